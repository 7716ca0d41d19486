"""GPU parity: the CUDA path through the C ABI against the FP64 oracle on the
same seeded inputs (Jin et al., arXiv 2203.11484, Sec. 3 and Eqs. 1-2).

  Philox words, close-range sets, patch triangle assignment, VPL tags: bit-exact
  patch VPL positions: within 1e-6 of the scene diagonal; light-path VPL
  positions: within the bound derived per VPL from FP32 rounding along its
  path; fluxes: 1e-6 relative
  pixels: |gpu - ref| <= 1e-4 |ref| + 1e-7 mean(ref), except pixels whose
  error is explained by visibility flips (<= 1e-5 of the pairs, each passing
  an edge or plane within what FP32 rounding can move)
"""
import math

import dataclasses

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
def ctx(V):
    c = V.Context(0)
    yield c
    c.close()


@pytest.fixture(scope="module")
def cornell(V, ctx, orc):
    wl = W.cornell_workload()
    sid = ctx.upload(wl.scene)
    return wl, sid, orc.OracleScene(wl.scene)


@pytest.fixture(scope="module")
def room(V, ctx, orc):
    wl = W.room200k_workload()
    sid = ctx.upload(wl.scene)
    return wl, sid, orc.OracleScene(wl.scene)


def _dev(a, dtype=None):
    t = torch.as_tensor(np.ascontiguousarray(a))
    if dtype is not None:
        t = t.to(dtype)
    return t.cuda()


# ---------------------------------------------------------------------------
# random numbers: Philox4x64-10 words bit-exact
# ---------------------------------------------------------------------------
def test_philox_bit_exact(V, ctx, orc):
    rng = np.random.default_rng(2)
    n = 4096
    ctr = rng.integers(0, 2**63, size=(n, 4), dtype=np.uint64)
    ctr[:64, 2:] = 0
    ctr[:64, 0] = np.arange(64)
    key = rng.integers(0, 2**63, size=(n, 2), dtype=np.uint64)
    out = torch.zeros((n, 4), dtype=torch.int64, device="cuda")
    V.vpl_debug_philox(ctx.h, _dev(ctr.view(np.int64)), _dev(key.view(np.int64)), out)
    V.vpl_sync(ctx.h)
    got = out.cpu().numpy().view(np.uint64)
    for i in range(0, n, 7):
        assert np.array_equal(got[i], orc.philox4x64_10(ctr[i], key[i])), i


# ---------------------------------------------------------------------------
# BVH queries against the oracle (brute force and its own FP64 BVH)
# ---------------------------------------------------------------------------
def _ray_queries(V, ctx, sid, P, Q, mode, brute):
    n = P.shape[0]
    a = np.zeros((n, 4), np.float32)
    b = np.zeros((n, 4), np.float32)
    a[:, :3], b[:, :3] = P, Q
    tri = torch.zeros(n, dtype=torch.int32, device="cuda")
    t = torch.zeros(n, dtype=torch.float32, device="cuda")
    V.vpl_debug_rays(ctx.h, sid, mode, brute, _dev(a), _dev(b), tri, t)
    V.vpl_sync(ctx.h)
    return tri.cpu().numpy(), t.cpu().numpy()


@pytest.mark.parametrize("which", ["cornell", "room"])
def test_bvh_visibility_and_closest_hit(V, ctx, which, request):
    wl, sid, osc = request.getfixturevalue(which)
    sc = wl.scene
    Ld = sc.diag()
    rng = np.random.default_rng(11)
    lo, hi = sc.verts.min(0), sc.verts.max(0)
    n = 200000
    P = rng.uniform(lo, hi, size=(n, 3)).astype(np.float32)
    Q = rng.uniform(lo, hi, size=(n, 3)).astype(np.float32)
    # segments occluded test: at most 1e-5 of the segments differ, each explained
    for brute in ([0, 1] if which == "cornell" else [0]):
        occ, _ = _ray_queries(V, ctx, sid, P, Q, 0, brute)
        ref = osc.occluded(P.astype(np.float64), Q.astype(np.float64), vis_mode=0)
        diff = np.nonzero((occ != 0) != ref)[0]
        print(which, "brute" if brute else "bvh", "segments differing:", len(diff), "of", n)
        assert len(diff) <= max(1, int(PY.FLIP_FRACTION * n)), (brute, len(diff))
        for i in diff:
            assert PY.flip_explained(osc, P[i], Q[i]), i
    # closest hit along P + t (Q - P)
    D = (Q - P).astype(np.float32)
    tri, t = _ray_queries(V, ctx, sid, P, D, 1, 0)
    rtri, rt = osc.closest(P.astype(np.float64), D.astype(np.float64), 0.0, 0)
    same = tri == rtri
    # a closest hit is not a pair's visibility: faces that coincide (a box
    # standing on the floor) or share an edge make equal-t ties common in
    # these scenes, so the bound is 1e-3 of the rays, each one explained
    assert (~same).sum() <= max(2, 1e-3 * n)
    hit = same & (tri >= 0)
    assert np.allclose(t[hit], rt[hit], rtol=1e-5, atol=1e-6)
    n_tie = 0
    for i in np.nonzero(~same)[0]:
        # different triangle: two hits at equal t (faces that touch), or the
        # ray passes an edge within FP32 reach
        near_tie = (tri[i] >= 0 and rtri[i] >= 0 and abs(t[i] - rt[i]) <= 1e-5 * max(1.0, rt[i]))
        n_tie += near_tie
        q = P[i] + D[i] * (rt[i] if rtri[i] >= 0 else t[i])
        assert near_tie or PY.flip_explained(osc, P[i], P[i] + 2 * (q - P[i]), ends=0), i
    print(which, "closest hits differing:", int((~same).sum()), "of", n, "equal-t ties", n_tie)


# ---------------------------------------------------------------------------
# G-buffer (points y of Eq. 1)
# ---------------------------------------------------------------------------
def _gbuffer(V, ctx, sid, cam):
    gb = V.GBuffer.empty(cam.width, cam.height)
    V.vpl_gbuffer_build(ctx.h, sid, cam, gb)
    V.vpl_sync(ctx.h)
    pos = gb.pos.cpu().numpy()
    return dict(pos=pos[:, :3].astype(np.float64), tri=pos[:, 3].copy().view(np.int32).astype(np.int64),
                nrm=gb.nrm.cpu().numpy()[:, :3].astype(np.float64),
                rho=gb.albedo.cpu().numpy()[:, :3].astype(np.float64)), gb


@pytest.mark.parametrize("which", ["cornell", "room"])
def test_gbuffer_parity(V, ctx, which, request):
    wl, sid, osc = request.getfixturevalue(which)
    cam = wl.views[0].camera
    g, _ = _gbuffer(V, ctx, sid, cam)
    npx = cam.width * cam.height
    pix = np.arange(npx) if which == "cornell" else np.random.default_rng(3).choice(npx, 8192, replace=False)
    ref = osc.gbuffer(cam, pix)
    Ld = wl.scene.diag()
    same = g["tri"][pix] == ref["tri"]
    assert same.mean() >= 0.999
    ok = same & (ref["tri"] >= 0)
    assert np.abs(g["pos"][pix][ok] - ref["pos"][ok]).max() <= PY.POS_TOL * Ld
    assert np.abs(g["nrm"][pix][ok] - ref["nrm"][ok]).max() <= 1e-7
    assert np.array_equal(g["rho"][pix][ok], ref["rho"][ok])
    # pixels that hit another triangle: the primary ray passes an edge
    frame_eye = np.array(cam.eye, np.float32).astype(np.float64)
    for k in np.nonzero(~same)[0]:
        q = ref["pos"][k] if ref["tri"][k] >= 0 else g["pos"][pix[k]]
        far = frame_eye + 2.0 * (q - frame_eye)
        assert PY.flip_explained(osc, frame_eye, far), int(pix[k])


# ---------------------------------------------------------------------------
# VPL generation (Sec. 3 pipeline steps (1)-(3))
# ---------------------------------------------------------------------------
def _generate(V, ctx, sid, cam, gen):
    M = gen.m_close + gen.m_far
    vs = V.VplSet.empty(M)
    V.vpl_generate(ctx.h, sid, cam, gen, vs)
    rc = V.vpl_sync(ctx.h, check=False)
    info = V.vpl_generate_info(ctx.h)
    return dict(PY.vpl_rows(vs), status=rc, info=info), vs


@pytest.mark.parametrize("variant", ["centroid", "any_vertex", "ir_only"])
@pytest.mark.parametrize("which", ["cornell", "room"])
def test_generate_parity(V, ctx, which, variant, request):
    """Both close-range rules (centroid; centroid or any vertex), and plain
    instant radiosity (no close range, every VPL from light paths: the
    comparison method of the quality study).  Close set, f(N), strata ->
    faces and tags bit-exact; patch positions and fluxes as the module
    states (light-sample flips explained); light-path VPLs matched by tag,
    each within its derived position bound, any path that changed course
    explained by a ray near an edge."""
    wl, sid, osc = request.getfixturevalue(which)
    view = wl.views[0]
    cam, gen = view.camera, view.gen
    if variant == "any_vertex":
        gen = dataclasses.replace(gen, close_rule=1)
    elif variant == "ir_only":
        gen = dataclasses.replace(gen, m_close=0, m_far=gen.m_close + gen.m_far, d_close=0.0)
    g, _ = _generate(V, ctx, sid, cam, gen)
    r = osc.generate(cam, gen, vis_mode=0)
    assert g["status"] == 0 and r["status"] == 0
    assert g["info"]["m_far_kept"] == r["m_far_kept"] == gen.m_far
    flips, div = PY.check_generation(osc, cam, gen, g, r, g["info"])
    print(which, variant, "light-sample flips", flips, "divergent light paths", div, "paths", r["paths"])


@pytest.mark.parametrize("which", ["cornell", "room"])
def test_generate_parity_set_sum(V, ctx, which, request):
    """Set-sum rule: the face of every patch VPL (the one giving its stratum
    the most area) is exact, positions (area-weighted centroids) and normals
    agree to FP32, fluxes to 1e-6 except where the light segment of a face
    of the stratum flips between the FP32 and FP64 BVHs (each explained, at
    most 1% of the VPLs)."""
    wl, sid, osc = request.getfixturevalue(which)
    view = wl.views[0]
    cam, gen = view.camera, dataclasses.replace(view.gen, patch_rule=1)
    g, _ = _generate(V, ctx, sid, cam, gen)
    r = osc.generate(cam, gen, vis_mode=0)
    assert g["status"] == 0 and r["status"] == 0
    PY.check_generation(osc, cam, gen, g, r, g["info"])
    # the rule changed something on this view: some stratum spans several faces
    Mc = gen.m_close
    p0 = osc.generate(cam, view.gen, vis_mode=0)
    assert not np.array_equal(p0["pos"][:Mc], r["pos"][:Mc])


# ---------------------------------------------------------------------------
# gather (Eq. 1) on identical FP32 inputs made by the oracle
# ---------------------------------------------------------------------------
def _to_gbuffer(V, g, width, height):
    n = width * height
    pos = np.zeros((n, 4), np.float32)
    pos[:, :3] = g["pos"]
    pos[:, 3] = np.asarray(g["tri"], np.int32).view(np.float32)
    nrm = np.zeros((n, 4), np.float32)
    nrm[:, :3] = g["nrm"]
    alb = np.zeros((n, 4), np.float32)
    alb[:, :3] = g["rho"]
    return V.GBuffer(_dev(pos), _dev(nrm), _dev(alb), width, height)


def _to_vpls(V, v):
    M = len(v["pos"])
    out = []
    for key in ("pos", "nrm", "flux"):
        a = np.zeros((max(M, 0), 4), np.float32)
        a[:, :3] = v[key]
        out.append(_dev(a))
    return V.VplSet(*out)


def _gather(V, ctx, sid, gbuf, vpls, params):
    out = torch.zeros((gbuf.width * gbuf.height, 4), dtype=torch.float32, device="cuda")
    V.vpl_gather(ctx.h, sid, gbuf, vpls, params, out)
    assert V.vpl_sync(ctx.h, check=False) == 0
    return out.cpu().numpy()


def _check_gather(V, ctx, sid, osc, wl, gb_ref, vpl_ref, width, height, params, oracle_vis):
    g, v = PY.oracle_inputs_f32(gb_ref, vpl_ref)
    gbuf = _to_gbuffer(V, g, width, height)
    vpls = _to_vpls(V, v)
    got = _gather(V, ctx, sid, gbuf, vpls, params)
    ref = osc.gather(g, v, params.d2_min, params.ray_eps, vis_mode=oracle_vis)
    bad = np.nonzero(PY.pixel_fail(got, ref))[0]
    n_pairs = int((g["tri"] >= 0).sum()) * len(v["pos"])
    flips_total = 0
    if len(bad):
        assert params.visibility != W.VIS_NONE, "no visibility: nothing may differ"
        pix = torch.as_tensor(bad.astype(np.int32)).cuda()
        vis = torch.zeros((len(bad), len(v["pos"])), dtype=torch.int8, device="cuda")
        V.vpl_debug_visibility(ctx.h, sid, gbuf, vpls, params, pix, vis)
        V.vpl_sync(ctx.h)
        vis = vis.cpu().numpy()
        Ld = wl.scene.diag()
        for row, p in enumerate(bad):
            nf, ok, _ = PY.explain_pixel(osc, g["pos"][p], g["nrm"][p], v, vis[row], params.d2_min,
                                         float(np.float32(params.ray_eps)), Ld)
            assert nf > 0 and ok, (p, got[p], ref[p], nf)
            flips_total += nf
    assert flips_total <= max(3, PY.FLIP_FRACTION * n_pairs), flips_total
    return got, ref, len(bad)


@pytest.mark.parametrize("vis", [W.VIS_BRUTE, W.VIS_BVH, W.VIS_NONE])
def test_gather_parity_cornell(V, ctx, cornell, vis):
    wl, sid, osc = cornell
    view = wl.views[0]
    gb = osc.gbuffer(view.camera, vis_mode=1)
    vp = osc.generate(view.camera, view.gen, vis_mode=1)
    params = W.GatherParams(view.gather.d2_min, view.gather.ray_eps, W.PREC_FP32, vis)
    ovis = {W.VIS_BRUTE: 1, W.VIS_BVH: 0, W.VIS_NONE: 2}[vis]
    got, ref, nbad = _check_gather(V, ctx, sid, osc, wl, gb, vp, view.camera.width, view.camera.height,
                                   params, ovis)
    assert ref.max() > 0 and np.isfinite(got).all()


def test_gather_parity_room_sampled(V, ctx, room):
    """The 200k-triangle room with 4096 VPLs: 2048 sampled receivers laid out
    as a 64 x 32 G-buffer (every pixel is independent in Eq. 1)."""
    wl, sid, osc = room
    view = wl.views[0]
    cam = view.camera
    pix = np.random.default_rng(5).choice(cam.width * cam.height, 2048, replace=False)
    gb = osc.gbuffer(cam, pix)
    vp = osc.generate(cam, view.gen, vis_mode=0)
    got, ref, nbad = _check_gather(V, ctx, sid, osc, wl, gb, vp, 64, 32, view.gather, 0)
    assert ref.max() > 0


# ---------------------------------------------------------------------------
# the whole pipeline (steps (1)-(4)) through vpl_render
# ---------------------------------------------------------------------------
def _render(V, ctx, sid, view):
    cam = view.camera
    out = torch.zeros((cam.width * cam.height, 4), dtype=torch.float32, device="cuda")
    V.vpl_render(ctx.h, sid, cam, view.gen, view.gather, out)
    assert V.vpl_sync(ctx.h, check=False) == 0
    return out.cpu().numpy()


def _render_parity(V, ctx, sid, osc, wl, view, pix):
    import oracle as O
    img = _render(V, ctx, sid, view)
    r = O.render(osc, view, pix)
    # pixels whose primary ray hits another triangle are G-buffer flips
    g, _ = _gbuffer(V, ctx, sid, view.camera)
    same_tri = g["tri"][pix] == r["gbuffer"]["tri"]
    assert same_tri.mean() >= 0.999
    got = img[pix]
    bad = PY.pixel_fail(got, r["image"]) & same_tri
    return img, r, bad


def test_render_parity_cornell_full(V, ctx, cornell):
    wl, sid, osc = cornell
    view = wl.views[0]
    pix = np.arange(view.camera.width * view.camera.height)
    img, r, bad = _render_parity(V, ctx, sid, osc, wl, view, pix)
    # tiny scene, brute-force visibility: at most a handful of flip pixels
    assert bad.sum() <= 3, np.nonzero(bad)[0][:10]
    assert r["image"].max() > 0


def test_render_parity_room_full_size(V, ctx, room):
    """Full 1024 x 1024, 4096-VPL render (the benchmark's launch), sampled
    pixels checked against the oracle."""
    wl, sid, osc = room
    view = wl.views[0]
    pix = np.random.default_rng(9).choice(view.camera.width * view.camera.height, 512, replace=False)
    img, r, bad = _render_parity(V, ctx, sid, osc, wl, view, pix)
    g, _ = _gbuffer(V, ctx, sid, view.camera)
    same_tri = g["tri"][pix] == r["gbuffer"]["tri"]
    M = view.gen.m_close + view.gen.m_far
    n_bad, n_still, flips = PY.explain_render_pixels(V, torch, ctx, sid, osc, view, img, pix, r["image"], r["vpl"],
                                                     same_tri, wl.scene.diag())
    assert n_bad == int(bad.sum())
    assert flips <= max(3, PY.FLIP_FRACTION * len(pix) * M), flips
    assert np.isfinite(img).all()


# ---------------------------------------------------------------------------
# the beam walk against the per-lane packet walk: the same segments, so the
# same visibility, so the same image bit for bit
# ---------------------------------------------------------------------------
def test_beam_walk_equals_per_lane_walk_cornell(V, ctx, cornell):
    """The 64-triangle room (axis-aligned, coplanar and touching faces, the
    light just under the ceiling) with BVH visibility: both walks give the
    same image bit for bit, and it matches the brute-force gather."""
    wl, sid, osc = cornell
    view = wl.views[0]
    cam = view.camera
    gb = V.GBuffer.empty(cam.width, cam.height)
    vs = V.VplSet.empty(view.gen.m_close + view.gen.m_far)
    V.vpl_gbuffer_build(ctx.h, sid, cam, gb)
    V.vpl_generate(ctx.h, sid, cam, view.gen, vs)
    imgs = []
    for walk, vis in ((0, W.VIS_BVH), (1, W.VIS_BVH), (0, W.VIS_BRUTE)):
        out = torch.zeros((cam.width * cam.height, 4), dtype=torch.float32, device="cuda")
        V.vpl_gather(ctx.h, sid, gb, vs, dataclasses.replace(view.gather, walk=walk, visibility=vis), out)
        assert V.vpl_sync(ctx.h, check=False) == 0
        imgs.append(out)
    assert float(imgs[0].max()) > 0
    assert torch.equal(imgs[0], imgs[1])
    # brute force tests every triangle per segment; the BVH walks may differ
    # from it only where a segment's FP32 box tests and triangle tests disagree
    assert (imgs[0] != imgs[2]).any(dim=1).float().mean().item() <= 1e-3


@pytest.mark.parametrize("prec", [W.PREC_FP32, W.PREC_FP16_KAHAN])
def test_beam_walk_equals_per_lane_walk(V, ctx, room, prec):
    """The full 1024 x 1024 x 4096 room launch with walk = 0 (beam walk for
    narrow packets) and walk = 1 (per-lane packet walk only): identical
    images, and identical to the per-lane walk for every pixel tile shape
    and with the tiles taken most costly first (tile_order = 2)."""
    wl, sid, osc = room
    view = wl.views[0]
    cam = view.camera
    fmt = V.FORMAT_FP32 if prec == W.PREC_FP32 else V.FORMAT_FP16
    gb = V.GBuffer.empty(cam.width, cam.height, fmt=fmt)
    vs = V.VplSet.empty(view.gen.m_close + view.gen.m_far, fmt=fmt)
    V.vpl_gbuffer_build(ctx.h, sid, cam, gb)
    V.vpl_generate(ctx.h, sid, cam, view.gen, vs)
    imgs = {}
    for walk, tw, order in ((1, 8, 1), (0, 8, 0), (0, 4, 0), (0, 32, 0), (0, 8, 2), (0, 4, 2)):
        out = torch.zeros((cam.width * cam.height, 4), dtype=torch.float32, device="cuda")
        params = dataclasses.replace(view.gather, precision=prec, walk=walk, tile_w=tw, tile_order=order)
        V.vpl_gather(ctx.h, sid, gb, vs, params, out)
        assert V.vpl_sync(ctx.h, check=False) == 0
        imgs[(walk, tw, order)] = out
    ref = imgs[(1, 8, 1)]
    assert float(ref.max()) > 0
    for key, img in imgs.items():
        assert torch.equal(img, ref), key
