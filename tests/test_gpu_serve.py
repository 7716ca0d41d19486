"""Serving with continuous batching on the GPU: requests over two resident
scenes, admitted into groups while others run (generation on a stream per
group, gathers in admission order on one stream), give the same image as
each request rendered alone; the admission estimate bounds the memory a
group takes."""
import numpy as np
import pytest

from paper_2203_11484_gb300 import serve as S
from paper_2203_11484_gb300 import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def test_served_requests_equal_their_renders_alone():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2203_11484_gb300 import build, vpl as V
    build.build_library()
    ctx = V.Context(0)
    try:
        tiny = W.cornell_workload()
        room, lo, hi = W.room200k_scene()
        sids = {"tiny": ctx.upload(tiny.scene), "room": ctx.upload(room)}
        n_tris = {"tiny": tiny.scene.n_tris, "room": room.n_tris}
        rng = np.random.default_rng(8)
        reqs = []
        base = tiny.views[0]
        for k, ((w, h), m) in enumerate([((64, 48), 256), ((128, 128), 96), ((80, 80), 512), ((32, 96), 64)]):
            cam = W.Camera(base.camera.eye, base.camera.forward, base.camera.up, 60.0, w, h)
            mc, mf = W.split_budget(m, 0.75)
            gen = W.GenParams(**{**base.gen.__dict__, "m_close": mc, "m_far": mf, "seed": 50 + k})
            reqs.append(S.Request(len(reqs), "tiny", W.View(cam, gen, base.gather), 0.0))
        room_reqs = S.random_requests(rng, {"room": (room, lo, hi, W.ROOM_D_CLOSE)}, 6, rate=200.0,
                                      resolutions=((128, 128), (256, 144), (96, 200)), m_range=(500, 3000))
        for r in room_reqs:
            r.rid = len(reqs)
            reqs.append(r)
        srv = S.Server(S.GpuBackend(ctx.h, sids, lanes=3), n_tris, lanes=3, max_group=4,
                       reserve_bytes=256 << 20)
        stats = srv.run(reqs)
        torch.cuda.synchronize()
        assert V.vpl_sync(ctx.h, check=False) == 0
        assert stats["requests"] == len(reqs)
        assert srv.groups_launched < len(reqs)       # requests were batched
        assert srv.max_concurrent_groups >= 2        # groups overlapped
        lit = 0
        for r in reqs:
            c = r.view.camera
            alone = torch.zeros((c.width * c.height, 4), dtype=torch.float32, device="cuda")
            V.vpl_render(ctx.h, sids[r.scene], c, r.view.gen, r.view.gather, alone)
            assert V.vpl_sync(ctx.h, check=False) == 0
            assert torch.equal(alone, r.image), r.rid
            lit += float(alone.max()) > 0
        assert lit >= len(reqs) - 2       # a view may see no indirect light at all
    finally:
        ctx.close()


def test_generations_on_two_streams_at_once_match_one_at_a_time():
    """Each generation keeps its own device record of close-set size, area
    total and path count, so calls overlapping on two streams of one context
    give the VPL sets they give alone."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2203_11484_gb300 import build, vpl as V
    build.build_library()
    ctx = V.Context(0)
    try:
        room, lo, hi = W.room200k_scene()
        sid = ctx.upload(room)
        reqs = S.random_requests(np.random.default_rng(21), {"room": (room, lo, hi, W.ROOM_D_CLOSE)}, 6,
                                 rate=100.0, resolutions=((64, 64),), m_range=(500, 3000))
        views = [(r.view.camera, r.view.gen) for r in reqs]

        def run(streams):
            sets = []
            for k, (cam, gen) in enumerate(views):
                s = streams[k % len(streams)]
                with torch.cuda.stream(s):
                    vs = V.VplSet.empty(gen.m_close + gen.m_far, "cuda")
                    V.vpl_generate(ctx.h, sid, cam, gen, vs, s)
                sets.append(vs)
            torch.cuda.synchronize()
            return sets

        one = run([torch.cuda.current_stream()])
        assert V.vpl_sync(ctx.h, check=False) == 0
        for _ in range(3):
            two = run([torch.cuda.Stream(), torch.cuda.Stream()])
            assert V.vpl_sync(ctx.h, check=False) == 0
            for a, b in zip(one, two):
                assert torch.equal(a.pos, b.pos) and torch.equal(a.nrm, b.nrm) and torch.equal(a.flux, b.flux)
    finally:
        ctx.close()


def test_estimate_bytes_bounds_what_a_group_takes():
    """Admission charges estimate_bytes per request; what a group actually
    takes -- its tensors (G-buffers, VPL sets, images) plus the most the
    library's pool holds at once for its generations and batched gather
    (close-set sort, light-path slots, VPL order) -- must stay within it."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2203_11484_gb300 import build, vpl as V
    build.build_library()
    ctx = V.Context(0)
    try:
        room, lo, hi = W.room200k_scene()
        sid = ctx.upload(room)
        scenes = {"room": (room, lo, hi, W.ROOM_D_CLOSE)}
        rng = np.random.default_rng(31)
        for res, m_range, n in ((((1920, 1080),), (15000, 16000), 1), (((256, 256), (512, 512)), (1000, 4000), 4)):
            reqs = S.random_requests(rng, scenes, n, rate=100.0, resolutions=res, m_range=m_range)
            est = sum(S.estimate_bytes(r.view, room.n_tris) for r in reqs)
            be = S.GpuBackend(ctx.h, {"room": sid}, lanes=1)
            torch.cuda.synchronize()
            base = torch.cuda.memory_allocated()
            torch.cuda.reset_peak_memory_stats()
            used0 = V.vpl_pool_stats(ctx.h, reset_high=True)["used"]
            h = be.launch(reqs, 0)
            torch.cuda.synchronize()
            assert V.vpl_sync(ctx.h, check=False) == 0
            took = (torch.cuda.max_memory_allocated() - base) + (V.vpl_pool_stats(ctx.h)["high"] - used0)
            print("group of", n, "estimate", est, "took", took)
            assert 0 < took <= est, (took, est)
            del h
    finally:
        ctx.close()
