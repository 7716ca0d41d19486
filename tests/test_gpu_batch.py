"""Batched gather: many views of uneven size and VPL budget in one persistent
launch (and in a captured CUDA graph) give exactly the images of one
vpl_gather per view, for every tile shape the autotuner may pick."""
import numpy as np
import pytest

from paper_2203_11484_gb300 import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def env():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2203_11484_gb300 import batch, build, vpl
    build.build_library()
    ctx = vpl.Context(0)
    yield vpl, batch, ctx
    ctx.close()


def _views(wl, sizes_and_budgets):
    base = wl.views[0]
    out = []
    for k, ((w, h), m) in enumerate(sizes_and_budgets):
        cam = W.Camera(base.camera.eye, base.camera.forward, base.camera.up, base.camera.vfov_deg, w, h)
        mc, mf = W.split_budget(m, 0.75)
        gen = W.GenParams(**{**base.gen.__dict__, "m_close": mc, "m_far": mf, "seed": base.gen.seed + k})
        out.append(W.View(cam, gen, base.gather))
    return out


def _reference(V, ctx, sid, br):
    """One vpl_gather per view on the batch's own G-buffers and VPLs."""
    refs = []
    for v, gb, vs in zip(br.views, br.gbufs, br.vsets):
        o = torch.zeros((gb.width * gb.height, 4), dtype=torch.float32, device="cuda")
        V.vpl_gather(ctx.h, sid, gb, vs, br.base, o)
        refs.append(o)
    assert V.vpl_sync(ctx.h, check=False) == 0
    return [r.cpu().numpy() for r in refs]


@pytest.mark.parametrize("scene", ["cornell", "room"])
def test_batch_equals_per_view_gather_for_every_tile_shape(env, scene):
    V, B, ctx = env
    if scene == "cornell":
        wl = W.cornell_workload(visibility=W.VIS_BVH)
        # (a very narrow view would see no close-range face: VPL_ERR_EMPTY_CLOSE)
        spec = [((37, 29), 256), ((64, 64), 96), ((128, 96), 300), ((48, 40), 33), ((1, 1), 64), ((50, 3), 1)]
    else:
        wl = W.room200k_workload()
        spec = [((256, 256), 512), ((96, 200), 2000), ((512, 128), 777), ((33, 17), 4096)]
    sid = ctx.upload(wl.scene)
    br = B.BatchRenderer(ctx.h, sid, _views(wl, spec))
    br.prepare()
    assert V.vpl_sync(ctx.h, check=False) == 0
    refs = _reference(V, ctx, sid, br)
    assert max(r.max() for r in refs) > 0
    for cfg in B.CANDIDATES:
        for o in br.outs:
            o.fill_(-1.0)
        br.gather(config=cfg)
        assert V.vpl_sync(ctx.h, check=False) == 0
        for k, (o, r) in enumerate(zip(br.outs, refs)):
            assert np.array_equal(o.cpu().numpy(), r), (cfg, k)
    br.close()
    V.vpl_scene_release(ctx.h, sid)


def test_autotune_and_graph_replay(env):
    V, B, ctx = env
    wl = W.room200k_workload()
    sid = ctx.upload(wl.scene)
    spec = [((256, 256), 1024), ((128, 192), 512), ((320, 64), 2048)]
    br = B.BatchRenderer(ctx.h, sid, _views(wl, spec))
    cfg = br.autotune()
    assert cfg in B.CANDIDATES
    # eager reference, then the captured graph (gather only, and the whole batch)
    br.run()
    assert V.vpl_sync(ctx.h, check=False) == 0
    eager = [o.cpu().numpy().copy() for o in br.outs]
    for include_generation in (False, True):
        br.capture(include_generation=include_generation)
        for o in br.outs:
            o.fill_(-1.0)
        br.replay()
        br.replay()
        torch.cuda.synchronize()
        assert V.vpl_sync(ctx.h, check=False) == 0
        for o, e in zip(br.outs, eager):
            assert np.array_equal(o.cpu().numpy(), e)
    br.close()
    V.vpl_scene_release(ctx.h, sid)
