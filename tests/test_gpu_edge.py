"""Edge cases through the C ABI: empty and degenerate inputs, ragged sizes,
the method's degenerate cases (no close-range face, light paths that run
out), the point light of the paper's experiments, and argument errors."""
import ctypes as C

import numpy as np
import pytest

from paper_2203_11484_gb300 import workloads as W
import parity as PY

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def env(orc):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2203_11484_gb300 import build, vpl
    build.build_library()
    ctx = vpl.Context(0)
    wl = W.cornell_workload()
    sid = ctx.upload(wl.scene)
    yield vpl, ctx, wl, sid, orc.OracleScene(wl.scene), orc
    ctx.close()


def _render(V, ctx, sid, view):
    c = view.camera
    out = torch.full((c.width * c.height, 4), -1.0, dtype=torch.float32, device="cuda")
    V.vpl_render(ctx.h, sid, c, view.gen, view.gather, out)
    rc = V.vpl_sync(ctx.h, check=False)
    return out.cpu().numpy(), rc


def _view(wl, w=None, h=None, **gen):
    b = wl.views[0]
    cam = W.Camera(b.camera.eye, b.camera.forward, b.camera.up, b.camera.vfov_deg, w or b.camera.width,
                   h or b.camera.height)
    gat = W.GatherParams(b.gather.d2_min, b.gather.ray_eps, W.PREC_FP32, W.VIS_BVH)
    return W.View(cam, W.GenParams(**{**b.gen.__dict__, **gen}), gat)


def _parity(orc, osc, view, img, V=None, ctx=None, sid=None, max_bad_frac=0.005):
    """Pixels whose primary ray hits another triangle on the GPU (an edge
    between FP32 and FP64) are left out; of the rest at most max_bad_frac
    may differ (visibility flips, bounded in the main parity tests)."""
    r = orc.render(osc, view)
    same = np.ones(len(img), bool)
    if V is not None:
        cam = view.camera
        gb = V.GBuffer.empty(cam.width, cam.height)
        V.vpl_gbuffer_build(ctx.h, sid, cam, gb)
        V.vpl_sync(ctx.h, check=False)
        gpos = gb.pos.cpu().numpy()
        same = gpos[:, 3].copy().view(np.int32) == r["gbuffer"]["tri"]
        if len(img) >= 400:
            assert same.mean() >= 0.95
        # each pixel whose primary ray hits another triangle passes an edge
        eye = np.array(cam.eye, np.float32).astype(np.float64)
        for k in np.nonzero(~same)[0]:
            q = r["gbuffer"]["pos"][k] if r["gbuffer"]["tri"][k] >= 0 else gpos[k, :3].astype(np.float64)
            assert PY.flip_explained(osc, eye, eye + 2.0 * (q - eye)), int(k)
    bad = PY.pixel_fail(img, r["image"]) & same
    assert bad.sum() <= max(1, max_bad_frac * len(img)), int(bad.sum())
    return r


def test_no_vpls_gives_black(env):
    V, ctx, wl, sid, _, _ = env
    img, rc = _render(V, ctx, sid, _view(wl, m_close=0, m_far=0))
    assert rc == 0 and (img == 0).all()


@pytest.mark.parametrize("w,h", [(1, 1), (33, 17), (7, 65)])
def test_ragged_and_tiny_images(env, w, h):
    V, ctx, wl, sid, osc, orc = env
    view = _view(wl, w, h)
    img, rc = _render(V, ctx, sid, view)
    assert rc == 0 and np.isfinite(img).all() and (img[:, 3] == 0).all()
    _parity(orc, osc, view, img, V, ctx, sid)


def test_vpl_count_not_a_multiple_of_32(env):
    V, ctx, wl, sid, osc, orc = env
    view = _view(wl, 40, 30, m_close=29, m_far=8)
    img, rc = _render(V, ctx, sid, view)
    assert rc == 0
    _parity(orc, osc, view, img, V, ctx, sid)


def test_camera_looking_away_gives_empty_gbuffer(env):
    V, ctx, wl, sid, _, _ = env
    b = wl.views[0].camera
    cam = W.Camera((0.5, 0.5, 3.0), (0.0, 0.0, 1.0), (0.0, 1.0, 0.0), 60.0, 40, 20)
    gb = V.GBuffer.empty(40, 20)
    V.vpl_gbuffer_build(ctx.h, sid, cam, gb)
    assert V.vpl_sync(ctx.h, check=False) == 0
    assert (gb.pos.cpu().numpy()[:, 3].copy().view(np.int32) == -1).all()
    view = W.View(cam, W.GenParams(**{**wl.views[0].gen.__dict__, "m_close": 0}), wl.views[0].gather)
    img, rc = _render(V, ctx, sid, view)
    assert rc == 0 and (img == 0).all()


def test_single_triangle_scene(env, orc):
    V, ctx, _, _, _, _ = env
    verts = np.array([[-1, -1, 0], [1, -1, 0], [0, 1, 0]], np.float32)
    sc = W.Scene(verts, np.array([[0, 1, 2]], np.int32), np.array([[0.5, 0.6, 0.7]], np.float32),
                 W.Light((0.2, 0.1, 2.0), (0, 0, -1.0), (0.4, 0, 0), (0, 0.4, 0), (1, 1, 1), W.LIGHT_AREA))
    sid = ctx.upload(sc)
    info = V.vpl_scene_query(ctx.h, sid)
    assert info["n_tris"] == 1 and info["depth"] == 1
    cam = W.Camera((0.0, -0.2, 3.0), (0.0, 0.0, -1.0), (0.0, 1.0, 0.0), 50.0, 24, 24)
    gen = W.GenParams(d_close=10.0, m_close=40, m_far=10, seed=3, ray_eps=1e-5)
    view = W.View(cam, gen, W.GatherParams(1e-4, 1e-5))
    img, rc = _render(V, ctx, sid, view)
    # light paths end after one bounce (nothing else to hit) and the only face
    # is close range, so no distant VPL can be placed: VPL_ERR_PATHS_EXHAUSTED
    assert rc == 7
    r = orc.render(orc.OracleScene(sc), view)
    assert r["vpl"]["status"] == 7
    assert PY.pixel_fail(img, r["image"]).sum() == 0
    V.vpl_scene_release(ctx.h, sid)


def test_empty_close_set_status_and_far_vpls(env):
    V, ctx, wl, sid, osc, orc = env
    view = _view(wl, 32, 32, d_close=0.0)
    img, rc = _render(V, ctx, sid, view)
    assert rc == 6                                   # VPL_ERR_EMPTY_CLOSE
    r = _parity(orc, osc, view, img, V, ctx, sid)
    assert r["vpl"]["status"] == 6 and r["image"].max() > 0  # the distant VPLs still light it


def test_light_paths_exhausted(env):
    V, ctx, wl, sid, osc, orc = env
    view = _view(wl, 32, 32, m_far=64, ir_max_paths=5)
    img, rc = _render(V, ctx, sid, view)
    assert rc == 7                                   # VPL_ERR_PATHS_EXHAUSTED
    r = _parity(orc, osc, view, img, V, ctx, sid)
    assert r["vpl"]["status"] == 7 and r["vpl"]["paths"] == 5


def test_point_light_generation_and_render(env, orc):
    """Sec. 3.1: the paper's scenes are lit by point lights (Eq. 2 with 4 pi)."""
    V, ctx, wl, _, _, _ = env
    sc = W.cornell_scene(0)
    sc = W.Scene(sc.verts, sc.tris, sc.albedo, W.Light((0.5, 0.9, 0.5), (0, -1.0, 0), (0, 0, 0), (0, 0, 0),
                                                       (1, 1, 1), W.LIGHT_POINT))
    sid = ctx.upload(sc)
    view = _view(wl, 64, 64)
    M = view.gen.m_close + view.gen.m_far
    vs = V.VplSet.empty(M)
    V.vpl_generate(ctx.h, sid, view.camera, view.gen, vs)
    assert V.vpl_sync(ctx.h, check=False) == 0
    osc = orc.OracleScene(sc)
    ref = osc.generate(view.camera, view.gen, vis_mode=1)
    tri = vs.pos.cpu().numpy()[:, 3].copy().view(np.int32)
    assert np.array_equal(tri[: view.gen.m_close], ref["tri"][: view.gen.m_close])
    flux = vs.flux.cpu().numpy()[:, :3].astype(np.float64)
    assert np.allclose(flux, ref["flux"], rtol=1e-6, atol=1e-12)
    img, rc = _render(V, ctx, sid, view)
    assert rc == 0
    _parity(orc, osc, view, img, V, ctx, sid)
    V.vpl_scene_release(ctx.h, sid)


def test_argument_errors(env):
    V, ctx, wl, sid, _, _ = env
    L = V.load()
    view = wl.views[0]
    # unknown scene
    with pytest.raises(V.VplError) as e:
        V.vpl_render(ctx.h, 987654, view.camera, view.gen, view.gather,
                     torch.zeros((view.camera.width * view.camera.height, 4), device="cuda"))
    assert e.value.code == 5
    # G-buffer size differs from the camera's
    gb = V.GBuffer.empty(8, 8)
    cam = W.Camera(view.camera.eye, view.camera.forward, view.camera.up, 60.0, 9, 8)
    with pytest.raises(V.VplError) as e:
        V.vpl_gbuffer_build(ctx.h, sid, cam, gb)
    assert e.value.code == 1
    # VPL set count must equal the budget
    with pytest.raises(V.VplError):
        V.vpl_generate(ctx.h, sid, view.camera, view.gen, V.VplSet.empty(3))
    # bad tile width, bad precision / format pair
    with pytest.raises(V.VplError):
        V.vpl_gather(ctx.h, sid, V.GBuffer.empty(8, 8), V.VplSet.empty(4),
                     W.GatherParams(1e-4, 1e-5, tile_w=6), torch.zeros((64, 4), device="cuda"))
    with pytest.raises(V.VplError):
        V.vpl_gather(ctx.h, sid, V.GBuffer.empty(8, 8), V.VplSet.empty(4),
                     W.GatherParams(1e-4, 1e-5, walk=2), torch.zeros((64, 4), device="cuda"))
    for order in (-1, 3):             # tile orders are 0 (auto), 1 (scan) and 2 (cost)
        with pytest.raises(V.VplError):
            V.vpl_gather(ctx.h, sid, V.GBuffer.empty(8, 8), V.VplSet.empty(4),
                         W.GatherParams(1e-4, 1e-5, tile_order=order), torch.zeros((64, 4), device="cuda"))
    for vt in (8, 48, 128, -16):      # VPL tiles are 16, 32 or 64 (0 = 64)
        with pytest.raises(V.VplError):
            V.vpl_gather(ctx.h, sid, V.GBuffer.empty(8, 8), V.VplSet.empty(4),
                         W.GatherParams(1e-4, 1e-5, vpl_tile=vt), torch.zeros((64, 4), device="cuda"))
    with pytest.raises(V.VplError):
        V.vpl_gather(ctx.h, sid, V.GBuffer.empty(8, 8), V.VplSet.empty(4),
                     W.GatherParams(1e-4, 1e-5, precision=W.PREC_FP16_KAHAN), torch.zeros((64, 4), device="cuda"))
    # camera degenerate
    with pytest.raises(V.VplError):
        V.vpl_gbuffer_build(ctx.h, sid, W.Camera((0, 0, 0), (0, 1, 0), (0, 1, 0), 60.0, 8, 8), gb)
    # empty scene is refused, vertex indices out of range are reported by vpl_sync
    with pytest.raises(V.VplError):
        V.vpl_scene_upload(ctx.h, torch.zeros((3, 3), device="cuda"), torch.zeros((0, 3), dtype=torch.int32,
                           device="cuda"), torch.zeros((0, 3), device="cuda"), wl.scene.light)
    bad = torch.tensor([[0, 1, 7]], dtype=torch.int32, device="cuda")
    s2 = V.vpl_scene_upload(ctx.h, torch.zeros((3, 3), device="cuda") + torch.eye(3, device="cuda"), bad,
                            torch.full((1, 3), 0.5, device="cuda"), wl.scene.light)
    assert V.vpl_sync(ctx.h, check=False) == 1
    V.vpl_scene_release(ctx.h, s2)
    assert V.vpl_sync(ctx.h, check=False) == 0       # the status word was cleared


def test_debug_visibility_reports_pixels_outside_the_image(env):
    """A pixel index outside the G-buffer is reported through the device
    status and its row is left alone; the other rows are written."""
    V, ctx, wl, sid, _, _ = env
    view = wl.views[0]
    cam = view.camera
    gb = V.GBuffer.empty(cam.width, cam.height)
    V.vpl_gbuffer_build(ctx.h, sid, cam, gb)
    M = view.gen.m_close + view.gen.m_far
    vs = V.VplSet.empty(M)
    V.vpl_generate(ctx.h, sid, cam, view.gen, vs)
    assert V.vpl_sync(ctx.h, check=False) == 0
    n_px = cam.width * cam.height
    pix = torch.tensor([n_px // 2, n_px, -1, n_px // 2 + 1], dtype=torch.int32, device="cuda")
    vis = torch.full((4, M), 7, dtype=torch.int8, device="cuda")
    V.vpl_debug_visibility(ctx.h, sid, gb, vs, view.gather, pix, vis)
    assert V.vpl_sync(ctx.h, check=False) == 1          # VPL_ERR_INVALID_ARG
    v = vis.cpu().numpy()
    assert (v[1] == 7).all() and (v[2] == 7).all()      # rows of the bad indices untouched
    assert np.isin(v[[0, 3]], (-1, 0, 1)).all()
    # the status word is cleared by the read: the next call starts clean
    V.vpl_debug_visibility(ctx.h, sid, gb, vs, view.gather, pix[[0, 3]], vis[:2])
    assert V.vpl_sync(ctx.h, check=False) == 0
