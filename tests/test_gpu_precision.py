"""FP16 attribute storage with FP32 shading (plain or Kahan-compensated sums).

FP16 rows must be exact roundings of the FP32 rows; the image error of each
variant is measured against the FP64 oracle twice: on the original
attributes (what a user gets) and on the attributes rounded the way the FP16
path stores them (which leaves only the FP32 accumulation error).
"""
import numpy as np
import pytest

from paper_2203_11484_gb300 import workloads as W
import parity as PY

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def V():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2203_11484_gb300 import build, vpl
    build.build_library()
    return vpl


@pytest.fixture(scope="module")
def room(V, orc):
    ctx = V.Context(0)
    wl = W.room200k_workload()
    sid = ctx.upload(wl.scene)
    yield ctx, wl, sid, orc.OracleScene(wl.scene)
    ctx.close()


def _f16(a):
    return np.asarray(a, np.float32).astype(np.float16)


def test_fp16_rows_are_roundings_of_fp32_rows(V, room):
    ctx, wl, sid, _ = room
    view = wl.views[0]
    cam = W.Camera(view.camera.eye, view.camera.forward, view.camera.up, view.camera.vfov_deg, 96, 64)
    g32, g16 = V.GBuffer.empty(96, 64), V.GBuffer.empty(96, 64, fmt=V.FORMAT_FP16)
    V.vpl_gbuffer_build(ctx.h, sid, cam, g32)
    V.vpl_gbuffer_build(ctx.h, sid, cam, g16)
    M = view.gen.m_close + view.gen.m_far
    v32, v16 = V.VplSet.empty(M), V.VplSet.empty(M, fmt=V.FORMAT_FP16)
    V.vpl_generate(ctx.h, sid, cam, view.gen, v32)
    V.vpl_generate(ctx.h, sid, cam, view.gen, v16)
    assert V.vpl_sync(ctx.h, check=False) == 0
    assert torch.equal(g32.pos, g16.pos)
    assert np.array_equal(g16.nrm.cpu().numpy(), _f16(g32.nrm.cpu().numpy()[:, :4] * [1, 1, 1, 0]))
    assert np.array_equal(g16.albedo.cpu().numpy(), _f16(g32.albedo.cpu().numpy()))
    p32, p16 = v32.pos.cpu().numpy(), v16.pos.cpu().numpy()
    phi = v32.flux.cpu().numpy()[:, :3]
    m = phi.max(axis=1).astype(np.float32)
    assert np.array_equal(p16[:, :3], p32[:, :3])
    assert np.array_equal(p16[:, 3], m)
    inv = np.where(m > 0, np.float32(1.0) / np.where(m > 0, m, 1), 0).astype(np.float32)
    want = np.zeros((M, 4), np.float16)
    want[:, :3] = _f16(phi.astype(np.float32) * inv[:, None])
    assert np.array_equal(v16.flux.cpu().numpy(), want)
    nn = np.zeros((M, 4), np.float16)
    nn[:, :3] = _f16(v32.nrm.cpu().numpy()[:, :3])
    assert np.array_equal(v16.nrm.cpu().numpy(), nn)


def _errors(got, ref):
    g, r = got[:, :3].astype(np.float64), ref[:, :3].astype(np.float64)
    mask = r.max(axis=1) > 1e-3 * r.max()
    rel = np.abs(g - r)[mask] / np.abs(r)[mask].clip(1e-30)
    mse = ((g - r) ** 2).mean()
    psnr = 10 * np.log10(r.max() ** 2 / mse) if mse > 0 else float("inf")
    return dict(max_rel=float(rel.max()), mean_rel=float(rel.mean()), psnr_db=float(psnr))


def test_precision_variants_error_report(V, room):
    """2048 sampled receivers of the 200k-triangle room, 4096 VPLs: FP32,
    FP16 + Kahan, FP16 plain against the FP64 oracle."""
    ctx, wl, sid, osc = room
    view = wl.views[0]
    cam = view.camera
    pix = np.random.default_rng(21).choice(cam.width * cam.height, 2048, replace=False)
    gb = osc.gbuffer(cam, pix)
    vp = osc.generate(cam, view.gen, vis_mode=0)
    g, v = PY.oracle_inputs_f32(gb, vp)
    n, M = len(pix), len(v["pos"])
    # device rows, FP32 and FP16
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
    gb32 = V.GBuffer(cuda(pos), cuda(nrm), cuda(alb), 64, 32)
    gb16 = V.GBuffer(cuda(pos), cuda(_f16(nrm)), cuda(_f16(alb)), 64, 32, V.FORMAT_FP16)
    vs32 = V.VplSet(cuda(vpos), cuda(vn), cuda(vf))
    vs16 = V.VplSet(cuda(vpos16), cuda(_f16(vn)), cuda(vf16), V.FORMAT_FP16)
    # the oracle on the original inputs, and on the inputs as FP16 rows hold them
    ref = osc.gather(g, v, view.gather.d2_min, view.gather.ray_eps)
    g_h = dict(g, nrm=_f16(g["nrm"]).astype(np.float64), rho=_f16(g["rho"]).astype(np.float64))
    flux_h = (vf16[:, :3].astype(np.float32) * m[:, None]).astype(np.float64)
    v_h = dict(v, nrm=_f16(v["nrm"]).astype(np.float64), flux=flux_h)
    ref_h = osc.gather(g_h, v_h, view.gather.d2_min, view.gather.ray_eps)
    report = {}
    for name, prec, gbuf, vset in (("fp32", W.PREC_FP32, gb32, vs32),
                                   ("fp16_kahan", W.PREC_FP16_KAHAN, gb16, vs16),
                                   ("fp16_plain", W.PREC_FP16_PLAIN, gb16, vs16)):
        params = W.GatherParams(view.gather.d2_min, view.gather.ray_eps, prec, W.VIS_BVH)
        out = torch.zeros((n, 4), dtype=torch.float32, device="cuda")
        V.vpl_gather(ctx.h, sid, gbuf, vset, params, out)
        assert V.vpl_sync(ctx.h, check=False) == 0
        got = out.cpu().numpy()
        report[name] = dict(vs_fp64=_errors(got, ref), vs_fp64_fp16_inputs=_errors(got, ref_h))
    print("precision report (2048 receivers x 4096 VPLs):", report)
    assert report["fp32"]["vs_fp64"]["mean_rel"] < 1e-5
    for k in ("fp16_kahan", "fp16_plain"):
        # FP16 storage: ~2^-11 relative per attribute
        assert report[k]["vs_fp64"]["mean_rel"] < 2e-3
        assert report[k]["vs_fp64"]["psnr_db"] > 50
        # with the rounding of the inputs taken out, only summation error is left
        assert report[k]["vs_fp64_fp16_inputs"]["mean_rel"] < 1e-5
    # compensated sums remove the summation rounding; the per-term FP32
    # rounding is common to both
    assert (report["fp16_kahan"]["vs_fp64_fp16_inputs"]["mean_rel"]
            <= report["fp16_plain"]["vs_fp64_fp16_inputs"]["mean_rel"] * 1.25 + 1e-9)


def test_render_fp16_matches_fp32_closely(V, room):
    """vpl_render in FP16 + Kahan against vpl_render in FP32, same view."""
    ctx, wl, sid, _ = room
    view = wl.views[0]
    cam = W.Camera(view.camera.eye, view.camera.forward, view.camera.up, view.camera.vfov_deg, 256, 256)
    outs = {}
    for prec in (W.PREC_FP32, W.PREC_FP16_KAHAN):
        params = W.GatherParams(view.gather.d2_min, view.gather.ray_eps, prec, W.VIS_BVH)
        out = torch.zeros((256 * 256, 4), dtype=torch.float32, device="cuda")
        V.vpl_render(ctx.h, sid, cam, view.gen, params, out)
        assert V.vpl_sync(ctx.h, check=False) == 0
        outs[prec] = out.cpu().numpy()[:, :3].astype(np.float64)
    a, b = outs[W.PREC_FP32], outs[W.PREC_FP16_KAHAN]
    mask = a.max(axis=1) > 1e-3 * a.max()
    rel = np.abs(a - b)[mask] / np.abs(a)[mask].clip(1e-30)
    assert np.median(rel) < 2e-3 and np.isfinite(b).all()
