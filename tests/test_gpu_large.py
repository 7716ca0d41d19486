"""The large configuration: ~1M-triangle dense clutter, 1920 x 1080 pixels,
32768 VPLs (26214 patch / 6554 instant radiosity).  One full-size render on
the GPU; the oracle checks sampled pixels of the 256 x 144 crop, every VPL
of the generation (patch faces exact, positions and fluxes, light paths by
tag) and the precision variants on the crop."""
import numpy as np
import pytest

from paper_2203_11484_gb300 import workloads as W
import parity as PY

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def large(orc):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2203_11484_gb300 import build, vpl
    build.build_library()
    ctx = vpl.Context(0)
    wl = W.room1m_workload()
    sid = ctx.upload(wl.scene)
    yield vpl, ctx, wl, sid, orc.OracleScene(wl.scene)
    ctx.close()


def _crop_pixels(wl, n, seed):
    x0, y0, w, h = wl.crop
    W_ = wl.views[0].camera.width
    rng = np.random.default_rng(seed)
    xs = x0 + rng.integers(0, w, n)
    ys = y0 + rng.integers(0, h, n)
    return np.unique(ys * W_ + xs)


def test_large_scene_builds(large):
    V, ctx, wl, sid, _ = large
    info = V.vpl_scene_query(ctx.h, sid)
    assert info["n_tris"] == wl.scene.n_tris >= 1_000_000
    assert 0 < info["depth"] <= 96


def test_large_generation_parity(large):
    """All 32768 VPLs of the 1M-triangle view against the oracle: close set,
    f(N) and patch faces exact, patch positions and fluxes (26214 light
    segments, flips explained), and the 6554 light-path VPLs matched by tag
    within their derived position bounds, fluxes to 1e-6."""
    V, ctx, wl, sid, osc = large
    view = wl.views[0]
    M = view.gen.m_close + view.gen.m_far
    vs = V.VplSet.empty(M)
    V.vpl_generate(ctx.h, sid, view.camera, view.gen, vs)
    assert V.vpl_sync(ctx.h, check=False) == 0
    info = V.vpl_generate_info(ctx.h)
    r = osc.generate(view.camera, view.gen, vis_mode=0)
    assert r["status"] == 0
    assert info["n_close"] == r["n_close"] > 0
    assert info["m_far_kept"] == r["m_far_kept"] == view.gen.m_far
    flips, div = PY.check_generation(osc, view.camera, view.gen, PY.vpl_rows(vs), r, info)
    print("1M clutter generation: light-sample flips", flips, "divergent light paths", div, "paths", r["paths"])


def test_large_render_full_size_crop_parity(large):
    V, ctx, wl, sid, osc = large
    import oracle as O
    view = wl.views[0]
    cam = view.camera
    out = torch.zeros((cam.width * cam.height, 4), dtype=torch.float32, device="cuda")
    V.vpl_render(ctx.h, sid, cam, view.gen, view.gather, out)
    assert V.vpl_sync(ctx.h, check=False) == 0
    img = out.cpu().numpy()
    assert np.isfinite(img).all()
    pix = _crop_pixels(wl, 96, 3)
    r = O.render(osc, view, pix)
    gb = V.GBuffer.empty(cam.width, cam.height)
    V.vpl_gbuffer_build(ctx.h, sid, cam, gb)
    V.vpl_sync(ctx.h)
    gtri = gb.pos.cpu().numpy()[pix, 3].copy().view(np.int32)
    same = gtri == r["gbuffer"]["tri"]
    assert same.mean() >= 0.98
    M = view.gen.m_close + view.gen.m_far
    n_bad, n_still, flips = PY.explain_render_pixels(V, torch, ctx, sid, osc, view, img, pix, r["image"], r["vpl"],
                                                     same, wl.scene.diag())
    assert flips <= max(3, PY.FLIP_FRACTION * len(pix) * M), flips
    assert r["image"].max() > 0


def test_large_precision_variants_on_crop(large):
    """FP32, FP16 attributes + Kahan sums and FP16 plain sums against the
    FP64 oracle on 1024 receivers of the 256 x 144 crop, 32768 VPLs."""
    V, ctx, wl, sid, osc = large
    x0, y0, w, h = wl.crop
    k = np.random.default_rng(5).choice(w * h, 1024, replace=False)
    pix = (y0 + k // w) * wl.views[0].camera.width + (x0 + k % w)
    report = PY.precision_report(V, torch, ctx, sid, osc, wl.views[0], pix, wl.scene.diag())
    print("precision report, 1M clutter crop (1024 receivers x 32768 VPLs):", report)
    PY.check_precision_report(report)


def test_large_beam_walk_equals_per_lane_walk(large):
    """The full 1920 x 1080 x 32768 launch on the 1M-triangle clutter with
    the beam walk (walk = 0) and with the per-lane packet walk only
    (walk = 1), the tiles taken most costly first (tile_order 0 picks that
    order for 32768 VPLs) and in scan order: identical images."""
    import dataclasses
    V, ctx, wl, sid, _ = large
    view = wl.views[0]
    cam = view.camera
    gb = V.GBuffer.empty(cam.width, cam.height)
    vs = V.VplSet.empty(view.gen.m_close + view.gen.m_far)
    V.vpl_gbuffer_build(ctx.h, sid, cam, gb)
    V.vpl_generate(ctx.h, sid, cam, view.gen, vs)
    imgs = []
    for walk, order in ((0, 0), (1, 1), (0, 1)):
        out = torch.zeros((cam.width * cam.height, 4), dtype=torch.float32, device="cuda")
        V.vpl_gather(ctx.h, sid, gb, vs, dataclasses.replace(view.gather, walk=walk, tile_order=order), out)
        assert V.vpl_sync(ctx.h, check=False) == 0
        imgs.append(out)
    assert float(imgs[1].max()) > 0
    assert torch.equal(imgs[0], imgs[1])
    assert torch.equal(imgs[2], imgs[1])
