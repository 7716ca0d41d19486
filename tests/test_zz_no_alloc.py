"""vpl_gather_noalloc: the gather for callers that may not allocate device
memory while they run (their device memory is reserved up front, or an
allocation could block on other work on the device).  Its scratch lives in
static device memory shared by every call, so two calls in a row must both
give what vpl_gather gives; oversized images are refused before any work.

This file is collected last on purpose and does not depend on other test
files: it passes alone in a fresh process and after the rest of the suite.
"""
import numpy as np
import pytest

from paper_2203_11484_gb300 import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

RTOL = 1e-4        # the pixel tolerance of the parity tests
ATOL_FRAC = 1e-7


@pytest.fixture(scope="module")
def setup():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2203_11484_gb300 import build, vpl
    build.build_library()
    ctx = vpl.Context(0)
    wl = W.cornell_workload()
    sid = ctx.upload(wl.scene)
    yield vpl, ctx, wl, sid
    ctx.close()


def _inputs(V, ctx, sid, view, width, height):
    cam = W.Camera(view.camera.eye, view.camera.forward, view.camera.up, view.camera.vfov_deg,
                   width, height)
    gb = V.GBuffer.empty(width, height)
    V.vpl_gbuffer_build(ctx.h, sid, cam, gb)
    vs = V.VplSet.empty(view.gen.m_close + view.gen.m_far)
    V.vpl_generate(ctx.h, sid, cam, view.gen, vs)
    assert V.vpl_sync(ctx.h, check=False) == 0
    return gb, vs


def _close(a, b):
    a = a[:, :3].astype(np.float64)
    b = b[:, :3].astype(np.float64)
    atol = ATOL_FRAC * max(float(np.abs(b).mean()), 1e-30)
    return bool((np.abs(a - b) <= RTOL * np.abs(b) + atol).all())


@pytest.mark.parametrize("vis", [W.VIS_BVH, W.VIS_BRUTE])
def test_noalloc_gather_matches_gather_twice(setup, vis):
    V, ctx, wl, sid = setup
    view = wl.views[0]
    params = W.GatherParams(view.gather.d2_min, view.gather.ray_eps, W.PREC_FP32, vis)
    # two calls in a row with different image sizes: the second must not see
    # the first call's scheduler state
    for width, height in ((128, 128), (72, 44)):
        gb, vs = _inputs(V, ctx, sid, view, width, height)
        ref = torch.zeros((width * height, 4), dtype=torch.float32, device="cuda")
        got = torch.full((width * height, 4), -1.0, dtype=torch.float32, device="cuda")
        V.vpl_gather(ctx.h, sid, gb, vs, params, ref)
        V.vpl_gather_noalloc(ctx.h, sid, gb, vs, params, got)
        assert V.vpl_sync(ctx.h, check=False) == 0
        r, g = ref.cpu().numpy(), got.cpu().numpy()
        assert r[:, :3].max() > 0
        assert _close(g, r), (width, height)


def test_noalloc_gather_rejects_oversized_image(setup):
    """Refused on the host before any device work (the buffer addresses are
    never touched)."""
    V, ctx, wl, sid = setup
    view = wl.views[0]
    gb = V.vpl_gbuffer()
    gb.pos = gb.nrm = gb.albedo = 256
    gb.width, gb.height, gb.format = 1 << 18, 1 << 18, 0   # 2^31 tiles
    vs = V.vpl_vpl_set()
    vs.pos = vs.nrm = vs.flux = 256
    vs.count, vs.format = 1, 0
    p = V.make_gather(view.gather)
    import ctypes as C
    rc = V.load().vpl_gather_noalloc(ctx.h, sid, C.byref(gb), C.byref(vs), C.byref(p), 256, None)
    assert rc == 1
    assert "2^30 tiles of 32 pixels" in V.vpl_last_error(ctx.h)


def test_noalloc_gather_allocates_nothing(setup):
    """What the entry point is for: a call takes no memory from the
    library's pool and none from the device.  vpl_gather on the same inputs
    does draw on the pool (tile counter, VPL sort), which shows the check can
    see an allocation."""
    V, ctx, wl, sid = setup
    view = wl.views[0]
    gb, vs = _inputs(V, ctx, sid, view, 128, 128)
    out = torch.zeros((128 * 128, 4), dtype=torch.float32, device="cuda")
    V.vpl_gather_noalloc(ctx.h, sid, gb, vs, view.gather, out)   # first call: address look-up
    assert V.vpl_sync(ctx.h, check=False) == 0
    torch.cuda.synchronize()
    before = V.vpl_pool_stats(ctx.h, reset_high=True)
    free0 = torch.cuda.mem_get_info()[0]
    for _ in range(3):
        V.vpl_gather_noalloc(ctx.h, sid, gb, vs, view.gather, out)
    assert V.vpl_sync(ctx.h, check=False) == 0
    after = V.vpl_pool_stats(ctx.h)
    free1 = torch.cuda.mem_get_info()[0]
    assert after["high"] == before["used"] == after["used"], (before, after)
    assert free1 >= free0, (free0, free1)
    # the same check sees vpl_gather's temporaries
    V.vpl_pool_stats(ctx.h, reset_high=True)
    V.vpl_gather(ctx.h, sid, gb, vs, view.gather, out)
    assert V.vpl_sync(ctx.h, check=False) == 0
    assert V.vpl_pool_stats(ctx.h)["high"] > after["used"]
