"""Helpers shared by the GPU parity tests: tolerances and explanations of
visibility flips.  Tolerances (per pixel, per component):
    |gpu - ref| <= 1e-4 |ref| + 1e-7 mean(ref)
VPL positions within 1e-6 of the scene diagonal, fluxes within 1e-6
relative; a GPU/oracle visibility disagreement counts as a flip when the
oracle finds the segment within 1e-5 of the scene diagonal of an edge or a
plane crossing."""
import numpy as np

PIX_RTOL = 1e-4
PIX_ATOL_FRAC = 1e-7
POS_TOL = 1e-6     # x scene diagonal
FLUX_RTOL = 1e-6
FLIP_MARGIN = 1e-5  # x scene diagonal
FLIP_FRACTION = 1e-5


def pixel_fail(gpu: np.ndarray, ref: np.ndarray) -> np.ndarray:
    """Boolean mask of pixels outside the tolerance (any channel)."""
    gpu = np.asarray(gpu, np.float64)[..., :3]
    ref = np.asarray(ref, np.float64)[..., :3]
    atol = PIX_ATOL_FRAC * max(float(np.abs(ref).mean()), 1e-30)
    bad = np.abs(gpu - ref) > PIX_RTOL * np.abs(ref) + atol
    return bad.reshape(-1, 3).any(axis=1)


def f32(a) -> np.ndarray:
    return np.asarray(a, np.float32).astype(np.float64)


def oracle_inputs_f32(gb: dict, vpl: dict) -> tuple:
    """Oracle G-buffer / VPLs rounded to FP32 (the GPU's input precision) and
    widened back, so both sides read identical inputs."""
    g = dict(pos=f32(gb["pos"]), nrm=f32(gb["nrm"]), rho=f32(gb["rho"]), tri=gb["tri"].copy())
    v = dict(pos=f32(vpl["pos"]), nrm=f32(vpl["nrm"]), flux=f32(vpl["flux"]))
    return g, v


def explain_pixel(oscene, y, ny, vpl, gpu_vis_row, d2_min, eps, L_diag):
    """Compare one pixel's GPU visibility bits with the oracle's.  Returns
    (n_flips, all_explained, flipped_term_sum).

    A flip is a pair that both sides evaluate (non-zero shading term and
    non-zero flux: the GPU skips zero-flux VPLs, which patch VPLs in the
    light's shadow are, and the oracle's term excludes the flux) with
    different V; each must lie within FLIP_MARGIN of an edge or a plane.  A
    pair that only one side evaluates is a cosine or distance decision at
    its rounding boundary: its term must be negligible (1e-6 of the pixel's
    terms), else the pixel is not explained."""
    term, vis, _ = oscene.pairs(y, ny, vpl, d2_min, eps, vis_mode=0)
    lit = np.abs(np.asarray(vpl["flux"], np.float64)).sum(axis=1) > 0
    traced = (vis >= 0) & lit
    g = np.asarray(gpu_vis_row)
    gpu_traced = g >= 0
    flips = traced & gpu_traced & (g != vis)
    one_sided = traced != gpu_traced
    ok = True
    if one_sided.any():
        ok = bool(np.abs(term[one_sided]).sum() <= 1e-6 * max(float(np.abs(term[traced]).sum()), 1e-300))
    if not flips.any():
        return 0, ok, 0.0
    _, _, margin = oscene.pairs(y, ny, vpl, d2_min, eps, vis_mode=0, want_margin=flips)
    ok = ok and bool((margin[flips] <= FLIP_MARGIN * L_diag).all())
    return int(flips.sum()), ok, float(np.abs(term[flips]).sum())


def _f16(a):
    return np.asarray(a, np.float32).astype(np.float16)


def image_errors(got, ref, keep=None) -> dict:
    """Max / mean relative error over pixels brighter than 1e-3 of the
    brightest, and PSNR (RGB); `keep` (boolean per pixel) limits both."""
    g, r = np.asarray(got)[:, :3].astype(np.float64), np.asarray(ref)[:, :3].astype(np.float64)
    if keep is not None:
        g, r = g[keep], r[keep]
    mask = r.max(axis=1) > 1e-3 * r.max()
    rel = np.abs(g - r)[mask] / np.abs(r)[mask].clip(1e-30)
    mse = ((g - r) ** 2).mean()
    psnr = 10 * np.log10(r.max() ** 2 / mse) if mse > 0 else float("inf")
    return dict(max_rel=float(rel.max()), mean_rel=float(rel.mean()), psnr_db=float(psnr))


def explain_failing_pixels(V, torch, ctx, sid, osc, gbuf, vset, params, g, v, got, ref, L_diag):
    """Pixels outside the pixel tolerance, each explained by visibility flips
    (the GPU's visibility bits of that pixel against the oracle's on the same
    inputs `g`, `v`, every flip within FLIP_MARGIN of an edge or a plane).
    Returns (failing pixel indices, total flips)."""
    bad = np.nonzero(pixel_fail(got, ref))[0]
    if not len(bad):
        return bad, 0
    M = len(v["pos"])
    pix = torch.as_tensor(bad.astype(np.int32)).cuda()
    vis = torch.zeros((len(bad), M), dtype=torch.int8, device="cuda")
    V.vpl_debug_visibility(ctx.h, sid, gbuf, vset, params, pix, vis)
    V.vpl_sync(ctx.h)
    vis = vis.cpu().numpy()
    total = 0
    for row, p in enumerate(bad):
        nf, ok, _ = explain_pixel(osc, g["pos"][p], g["nrm"][p], v, vis[row], params.d2_min,
                                  float(np.float32(params.ray_eps)), L_diag)
        assert nf > 0 and ok, (int(p), got[p], ref[p], nf)
        total += nf
    return bad, total


def precision_report(V, torch, ctx, sid, osc, view, pix, L_diag) -> dict:
    """Gathers the oracle's G-buffer rows of `pix` with the oracle's VPLs in
    FP32, FP16 + Kahan and FP16 plain, and measures each image against the
    FP64 oracle twice: on the original attributes (what a user gets) and on
    the attributes rounded the way the FP16 rows hold them (which leaves only
    the FP32 accumulation error).  FP16 VPL rows hold the flux colour divided
    by its largest channel, and that magnitude in pos.w (FP32).  Pixels off
    by visibility flips (each explained, counted against FLIP_FRACTION of the
    pairs) are left out of the error figures: they measure visibility, not
    precision."""
    from paper_2203_11484_gb300 import workloads as W
    cam = view.camera
    gb = osc.gbuffer(cam, pix)
    vp = osc.generate(cam, view.gen, vis_mode=0)
    g, v = oracle_inputs_f32(gb, vp)
    n, M = len(pix), len(v["pos"])
    pos = np.zeros((n, 4), np.float32)
    pos[:, :3] = g["pos"]
    pos[:, 3] = np.asarray(g["tri"], np.int32).view(np.float32)
    nrm = np.zeros((n, 4), np.float32)
    nrm[:, :3] = g["nrm"]
    alb = np.zeros((n, 4), np.float32)
    alb[:, :3] = g["rho"]
    vpos = np.zeros((M, 4), np.float32)
    vpos[:, :3] = v["pos"]
    vn = np.zeros((M, 4), np.float32)
    vn[:, :3] = v["nrm"]
    vf = np.zeros((M, 4), np.float32)
    vf[:, :3] = v["flux"]
    m = vf[:, :3].max(axis=1)
    inv = np.where(m > 0, np.float32(1.0) / np.where(m > 0, m, 1), 0).astype(np.float32)
    vpos16 = vpos.copy()
    vpos16[:, 3] = m
    vf16 = np.zeros((M, 4), np.float16)
    vf16[:, :3] = _f16(vf[:, :3] * inv[:, None])
    cuda = lambda a: torch.as_tensor(a).cuda()
    gb32 = V.GBuffer(cuda(pos), cuda(nrm), cuda(alb), n, 1)
    gb16 = V.GBuffer(cuda(pos), cuda(_f16(nrm)), cuda(_f16(alb)), n, 1, V.FORMAT_FP16)
    vs32 = V.VplSet(cuda(vpos), cuda(vn), cuda(vf))
    vs16 = V.VplSet(cuda(vpos16), cuda(_f16(vn)), cuda(vf16), V.FORMAT_FP16)
    ref = osc.gather(g, v, view.gather.d2_min, view.gather.ray_eps)
    g_h = dict(g, nrm=_f16(g["nrm"]).astype(np.float64), rho=_f16(g["rho"]).astype(np.float64))
    flux_h = (vf16[:, :3].astype(np.float32) * m[:, None]).astype(np.float64)
    v_h = dict(v, nrm=_f16(v["nrm"]).astype(np.float64), flux=flux_h)
    ref_h = osc.gather(g_h, v_h, view.gather.d2_min, view.gather.ray_eps)
    n_pairs = int((g["tri"] >= 0).sum()) * M
    outs, flip_pix, flips = {}, np.zeros(n, bool), {}
    for name, prec, gbuf, vset, gi, vi, r in (("fp32", W.PREC_FP32, gb32, vs32, g, v, ref),
                                              ("fp16_kahan", W.PREC_FP16_KAHAN, gb16, vs16, g_h, v_h, ref_h),
                                              ("fp16_plain", W.PREC_FP16_PLAIN, gb16, vs16, g_h, v_h, ref_h)):
        params = W.GatherParams(view.gather.d2_min, view.gather.ray_eps, prec, W.VIS_BVH)
        out = torch.zeros((n, 4), dtype=torch.float32, device="cuda")
        V.vpl_gather(ctx.h, sid, gbuf, vset, params, out)
        assert V.vpl_sync(ctx.h, check=False) == 0
        outs[name] = out.cpu().numpy()
        # each variant against the oracle on its own inputs: only flips may fail
        bad, nf = explain_failing_pixels(V, torch, ctx, sid, osc, gbuf, vset, params, gi, vi, outs[name], r,
                                         L_diag)
        assert nf <= max(3, FLIP_FRACTION * n_pairs), (name, nf)
        flip_pix[bad] = True
        flips[name] = dict(pixels=int(len(bad)), pairs=int(nf))
    keep = ~flip_pix
    report = {k: dict(vs_fp64=image_errors(o, ref, keep), vs_fp64_fp16_inputs=image_errors(o, ref_h, keep),
                      flips=flips[k]) for k, o in outs.items()}
    report["pixels_left_out"] = int(flip_pix.sum())
    return report


def check_precision_report(report: dict) -> None:
    """FP32 within the pixel tolerance on average; FP16 storage ~2^-11
    relative per attribute; with the input rounding taken out only the
    summation error is left, and compensated sums are no worse than plain."""
    assert report["fp32"]["vs_fp64"]["mean_rel"] < 1e-5
    for k in ("fp16_kahan", "fp16_plain"):
        assert report[k]["vs_fp64"]["mean_rel"] < 2e-3
        assert report[k]["vs_fp64"]["psnr_db"] > 50
        assert report[k]["vs_fp64_fp16_inputs"]["mean_rel"] < 1e-5
    assert (report["fp16_kahan"]["vs_fp64_fp16_inputs"]["mean_rel"]
            <= report["fp16_plain"]["vs_fp64_fp16_inputs"]["mean_rel"] * 1.25 + 1e-9)


def explain_render_pixels(V, torch, ctx, sid, osc, view, img, pix, ref_img, same_tri, L_diag):
    """Pixels of a full-size vpl_render (the benchmark's launch) that are
    outside the pixel tolerance against the oracle's whole pipeline, each
    explained.  The render is first checked to equal the G-buffer, the
    generation and the gather called one by one (bit for bit).  A failing
    pixel is then recomputed by the oracle's gather from the GPU's own
    G-buffer row and VPL rows: if it passes, the difference came from the
    FP32 inputs (bounded by the generation parity tests).  If not, the
    GPU's visibility bits of that pixel are taken with its whole tile as one
    packet, exactly as in the render, and the pixel must be explained by
    flips.  Returns (failing, failing on the GPU's inputs, flips)."""
    cam = view.camera
    W_, H_ = cam.width, cam.height
    gb = V.GBuffer.empty(W_, H_)
    V.vpl_gbuffer_build(ctx.h, sid, cam, gb)
    M = view.gen.m_close + view.gen.m_far
    vs = V.VplSet.empty(M)
    V.vpl_generate(ctx.h, sid, cam, view.gen, vs)
    out = torch.zeros((W_ * H_, 4), dtype=torch.float32, device="cuda")
    V.vpl_gather(ctx.h, sid, gb, vs, view.gather, out)
    assert V.vpl_sync(ctx.h, check=False) == 0
    assert np.array_equal(out.cpu().numpy()[pix], img[pix])
    bad = np.asarray(pix)[pixel_fail(img[pix], ref_img) & same_tri]
    if not len(bad):
        return 0, 0, 0
    rows = torch.as_tensor(bad.astype(np.int64)).cuda()
    gpos = gb.pos[rows].cpu().numpy()
    g = dict(pos=gpos[:, :3].astype(np.float64), nrm=gb.nrm[rows].cpu().numpy()[:, :3].astype(np.float64),
             rho=gb.albedo[rows].cpu().numpy()[:, :3].astype(np.float64),
             tri=gpos[:, 3].copy().view(np.int32).astype(np.int64))
    v = dict(pos=vs.pos.cpu().numpy()[:, :3].astype(np.float64), nrm=vs.nrm.cpu().numpy()[:, :3].astype(np.float64),
             flux=vs.flux.cpu().numpy()[:, :3].astype(np.float64))
    eps = float(np.float32(view.gather.ray_eps))
    ref2 = osc.gather(g, v, view.gather.d2_min, eps)
    still = np.nonzero(pixel_fail(img[bad], ref2))[0]
    if not len(still):
        return len(bad), 0, 0
    # each failing pixel's whole 8 x 4 tile, in lane order, as one packet
    tw, th = 8, 4
    lists, where = [], {}
    for k in still:
        p = int(bad[k])
        tx, ty = (p % W_) // tw, (p // W_) // th
        lanes = [(ty * th + l // tw) * W_ + tx * tw + l % tw for l in range(32)]
        if (tx + 1) * tw > W_ or (ty + 1) * th > H_:
            lanes = [p] + [p] * 31               # a ragged tile: the pixel alone
        where[p] = 32 * len(lists) + lanes.index(p)
        lists.append(lanes)
    plist = torch.as_tensor(np.asarray(lists, np.int32).reshape(-1)).cuda()
    vis = torch.zeros((plist.shape[0], M), dtype=torch.int8, device="cuda")
    V.vpl_debug_visibility(ctx.h, sid, gb, vs, view.gather, plist, vis)
    assert V.vpl_sync(ctx.h, check=False) == 0
    vis = vis.cpu().numpy()
    flips = 0
    for k in still:
        p = int(bad[k])
        nf, ok, _ = explain_pixel(osc, g["pos"][k], g["nrm"][k], v, vis[where[p]], view.gather.d2_min, eps, L_diag)
        assert nf > 0 and ok, (p, img[p], ref2[k], nf)
        flips += nf
    return len(bad), len(still), flips
