"""Benchmark of the hybrid close-range VPL renderer on GB300.

One step = one pass of the whole hot path over one synthetic view: scene upload
+ BVH build, G-buffer, VPL generation (close-range patch VPLs + sparse
instant radiosity) and the per-pixel gather with BVH shadow rays, through the
C ABI (vpl_scene_upload + vpl_render).  Workload: the procedural 200k-triangle
room, 1024 x 1024 pixels, 4096 VPLs (3072 patch / 1024 instant radiosity).

Metric: pixel-VPL contributions per second with visibility, i.e.
width * height * VPLs per step / step time, summed over ranks (each rank
renders its own view: replicas, weak scaling).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

# the headline value is the first quantity (pairs/s); batched views/s and the
# serving p99 latencies are in the line's "batch" and "serving" objects
METRIC = "pixel-VPL contributions/s with visibility; batched views/s and p99 latency"
UNIT = "pairs/s"

# executed FP32 operations per unit of gather work, counted from the source of
# gather_kernel / warp_occluded / tri_hit (an FMA counts 2)
FLOPS_PER_PAIR = 28       # d, |d|^2, two cosines, clamp, geometry factor, RGB FMA
FLOPS_PER_RAY = 15        # segment end points and reciprocal direction
FLOPS_PER_NODE = 80       # four slab tests per visited 4-wide node (per active lane)
FLOPS_PER_TRI = 47        # Moller-Trumbore (per active lane)


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


# ---- multi-GPU: independent replicas (no collective on the data path) --------
def replica_seed(base: int, rank: int) -> int:
    """Each rank renders its own close-up view of its own scene copy."""
    return base + rank


def max_over_ranks(value: float, device) -> float:
    """The slowest rank's time (the only collective of a run)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(units_per_step: int, steps: int, world: int, max_ms: float) -> float:
    """Whole-job units per second: every rank did `steps` steps in at most max_ms."""
    return units_per_step * steps * world / (max_ms / 1e3)


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during a region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.idx = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.idx}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except (OSError, FileNotFoundError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self) -> dict:
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.t.join(timeout=2)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def measured_traffic(workload: str, precision: str):
    """DRAM bytes per gather launch from the committed ncu summary, valid only
    while the kernel sources are the ones that were measured (else None)."""
    import hashlib
    import re
    h = hashlib.sha256()
    for f in ("gather.cu", "vpl_device.cuh", "build.cu"):
        with open(os.path.join(ROOT, "paper_2203_11484_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    try:
        with open(os.path.join(ROOT, "profiles", "gather_room200k_1024x1024_4096vpl_dram.md")) as fh:
            text = fh.read()
    except OSError:
        return None
    if f"source_sha256: {h.hexdigest()}" not in text or f"workload: {workload} {precision}" not in text:
        return None
    m = re.search(r"traffic_bytes_per_launch: (\d+)", text)
    return int(m.group(1)) if m else None


def _peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(p) as f:
            return json.load(f)
    except OSError:
        return {}


def cpu_baseline(workload, seconds: float = 12.0) -> dict:
    """The FP64 oracle on a bounded sample of the same view: G-buffer of the
    sampled pixels, full VPL generation, gather of the sampled pixels against
    all VPLs.  Pairs/s on all host cores."""
    import oracle
    view = workload.views[0]
    cam = view.camera
    osc = oracle.OracleScene(workload.scene)
    M = view.gen.m_close + view.gen.m_far
    rng = np.random.default_rng(77)
    n = 32
    t_used = 0.0
    pairs = 0
    runs = 0
    while True:
        pix = rng.choice(cam.width * cam.height, n, replace=False)
        t0 = time.perf_counter()
        oracle.render(osc, view, pix)
        dt = time.perf_counter() - t0
        t_used += dt
        pairs += n * M
        runs += 1
        if t_used >= seconds or runs >= 50:
            break
        # grow the sample towards the time budget
        n = int(min(4096, max(n, n * 0.5 * (seconds - t_used) / max(dt, 1e-3))))
    cores = oracle.num_threads()
    # the same on one core, a shorter sample
    one = None
    try:
        oracle.set_threads(1)
        pix = rng.choice(cam.width * cam.height, 256, replace=False)
        t0 = time.perf_counter()
        oracle.render(osc, view, pix)
        one = 256 * M / (time.perf_counter() - t0)
    finally:
        oracle.set_threads(cores)
    return {"value": pairs / t_used, "unit": UNIT, "cores": cores, "kind": "oracle", "value_1core": one,
            "sample": f"{runs} oracle renders (FP64, own BVH) of {pairs // M} sampled pixels x {M} VPLs "
                      f"incl. G-buffer of those pixels and full VPL generation, {t_used:.1f} s; "
                      f"value_1core: 256 pixels on one thread"}


def cpu_configs(room_pairs_per_s, room_workload) -> dict:
    """The oracle on the other workloads, each on a bounded sample timed on
    all host cores (the render of the sampled pixels: their G-buffer, the
    full VPL generation of the view, the gather): the 64-triangle room in
    full frame, two views of the 64-view batch (1024 sampled pixels each),
    1024 pixels of the 1M clutter's 256 x 144 crop.  Times beyond a sample
    (the full frame, the crop, all 64 views) are extrapolated from its
    pairs/s and marked so."""
    import oracle
    from paper_2203_11484_gb300 import workloads as W
    rng = np.random.default_rng(78)
    out = {}
    v0 = room_workload.views[0]
    room_pairs = v0.camera.width * v0.camera.height * (v0.gen.m_close + v0.gen.m_far)
    out["room200k"] = {"workload": room_workload.name, "pairs_per_s": room_pairs_per_s,
                       "sample": "the cpu_baseline sample", "full_frame_s": room_pairs / room_pairs_per_s,
                       "extrapolated": True}
    wl = W.cornell_workload()
    v = wl.views[0]
    osc = oracle.OracleScene(wl.scene)
    pairs = v.camera.width * v.camera.height * (v.gen.m_close + v.gen.m_far)
    t0 = time.perf_counter()
    oracle.render(osc, v)
    dt = time.perf_counter() - t0
    out["cornell"] = {"workload": wl.name, "pairs_per_s": pairs / dt, "sample": "full frame, brute-force visibility",
                      "full_frame_s": dt, "extrapolated": False}
    wl = W.batch_views()
    osc = oracle.OracleScene(wl.scene)
    pairs, dt = 0, 0.0
    for v in wl.views[:2]:
        M = v.gen.m_close + v.gen.m_far
        pix = rng.choice(v.camera.width * v.camera.height, 1024, replace=False)
        t0 = time.perf_counter()
        oracle.render(osc, v, pix)
        dt += time.perf_counter() - t0
        pairs += 1024 * M
    all_pairs = sum(v.camera.width * v.camera.height * (v.gen.m_close + v.gen.m_far) for v in wl.views)
    out["batch"] = {"workload": wl.name, "pairs_per_s": pairs / dt, "sample": "2 views x 1024 sampled pixels",
                    "full_frame_s": all_pairs / (pairs / dt), "extrapolated": True}
    wl = W.room1m_workload()
    v = wl.views[0]
    osc = oracle.OracleScene(wl.scene)
    M = v.gen.m_close + v.gen.m_far
    x0, y0, w, h = wl.crop
    k = rng.choice(w * h, 1024, replace=False)
    pix = (y0 + k // w) * v.camera.width + (x0 + k % w)
    t0 = time.perf_counter()
    oracle.render(osc, v, pix)
    dt = time.perf_counter() - t0
    rate = 1024 * M / dt
    out["clutter1m"] = {"workload": wl.name, "pairs_per_s": rate, "sample": "1024 pixels of the 256 x 144 crop",
                        "crop_s": w * h * M / rate, "full_frame_s": v.camera.width * v.camera.height * M / rate,
                        "extrapolated": True}
    return out


def batch_section(ctx, n_views: int, precision: int, reps: int = 2) -> dict:
    """Many close-up views of the resident 200k-triangle room with uneven
    resolutions and VPL budgets: one vpl_render per view (one launch sequence
    each) against the batched path (G-buffers and VPLs per view, one
    persistent gather for all views, autotuned tile shape, captured in a CUDA
    graph).  Same images either way."""
    import torch
    from paper_2203_11484_gb300 import batch as BT
    from paper_2203_11484_gb300 import vpl as V
    from paper_2203_11484_gb300 import workloads as W
    wl = W.batch_views(n_views=n_views, precision=precision)
    sc = wl.scene
    sid = V.vpl_scene_upload(ctx.h, torch.as_tensor(sc.verts).cuda(), torch.as_tensor(sc.tris).cuda(),
                             torch.as_tensor(sc.albedo).cuda(), sc.light)
    V.vpl_sync(ctx.h)
    stream = torch.cuda.current_stream()
    outs = [torch.zeros((v.camera.width * v.camera.height, 4), dtype=torch.float32, device="cuda")
            for v in wl.views]

    def single():
        for v, o in zip(wl.views, outs):
            V.vpl_render(ctx.h, sid, v.camera, v.gen, v.gather, o, stream)

    def timed(fn):
        fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(reps):
            fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / reps

    ms_single = timed(single)
    # tune on the first 16 views (same distribution), then the whole batch
    tuner = BT.BatchRenderer(ctx.h, sid, wl.views[:16], precision)
    cfg = tuner.autotune(candidates=BT.CANDIDATES)
    tune_ms = {f"tile_w={k[0]} blocks_per_sm={k[1]} vpl_tile={k[2]}": v for k, v in tuner.tune_ms.items()}
    tuner.close()
    br = BT.BatchRenderer(ctx.h, sid, wl.views, precision)
    br.config = cfg
    br.capture(include_generation=True)
    ms_batch = timed(br.replay)
    same = all(torch.equal(a, b) for a, b in zip(outs, br.outs))
    pairs = br.pairs()
    br.close()
    status = V.vpl_sync(ctx.h, check=False)  # a view without close-range faces reports EMPTY_CLOSE
    V.vpl_scene_release(ctx.h, sid)
    return {"workload": wl.name, "views": n_views, "pairs": pairs,
            "single_view_ms": ms_single, "batched_graph_ms": ms_batch,
            "views_per_s_single": n_views / (ms_single / 1e3), "views_per_s_batched": n_views / (ms_batch / 1e3),
            "pairs_per_s_batched": pairs / (ms_batch / 1e3), "speedup": ms_single / ms_batch,
            "tuned": {"tile_w": cfg[0], "blocks_per_sm": cfg[1], "vpl_tile": cfg[2]},
            "tuner_ms_first_16_views": tune_ms, "images_identical": bool(same),
            "device_status": V.STATUS_NAMES.get(status, status),
            "graph": "G-buffers + VPL generation per view + one batched gather, captured once"}


def large_section(ctx, peak_tflops: float, reps: int = 2) -> dict:
    """The large configuration: the ~1M-triangle clutter at 1920 x 1080 with
    32768 VPLs (26214 patch / 6554 light-path), gathered in FP32, FP16
    attributes + Kahan sums and FP16 attributes + plain sums.  Per precision:
    the gather's pairs/s (CUDA events, L2 flushed before each launch), its
    work counters and the FP32 roofline fraction with the same flop
    constants as the headline."""
    import torch
    from paper_2203_11484_gb300 import vpl as V
    from paper_2203_11484_gb300 import workloads as W
    wl = W.room1m_workload()
    sc = wl.scene
    sid = V.vpl_scene_upload(ctx.h, torch.as_tensor(sc.verts).cuda(), torch.as_tensor(sc.tris).cuda(),
                             torch.as_tensor(sc.albedo).cuda(), sc.light)
    stream = torch.cuda.current_stream()
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")
    out = {"workload": wl.name, "tris": sc.n_tris}
    for name, prec in (("fp32", W.PREC_FP32), ("fp16_kahan", W.PREC_FP16_KAHAN), ("fp16_plain", W.PREC_FP16_PLAIN)):
        import dataclasses
        view = wl.views[0]
        cam, gen = view.camera, view.gen
        gat = dataclasses.replace(view.gather, precision=prec)
        fmt = V.FORMAT_FP32 if prec == W.PREC_FP32 else V.FORMAT_FP16
        M = gen.m_close + gen.m_far
        gb = V.GBuffer.empty(cam.width, cam.height, fmt=fmt)
        vs = V.VplSet.empty(M, fmt=fmt)
        img = torch.zeros((cam.width * cam.height, 4), dtype=torch.float32, device="cuda")
        V.vpl_gbuffer_build(ctx.h, sid, cam, gb, stream)
        V.vpl_generate(ctx.h, sid, cam, gen, vs, stream)
        V.vpl_gather(ctx.h, sid, gb, vs, gat, img, stream)          # warm-up
        ms = []
        for k in range(reps):
            flush.fill_(float(k))
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            V.vpl_gather(ctx.h, sid, gb, vs, gat, img, stream)
            e1.record(stream)
            torch.cuda.synchronize()
            ms.append(e0.elapsed_time(e1))
        cnt = V.vpl_gather_counters(ctx.h, sid, gb, vs, gat, stream)
        status = V.vpl_sync(ctx.h, stream, check=False)
        t = statistics.mean(ms)
        pairs = cam.width * cam.height * M
        flops = (cnt[0] * FLOPS_PER_PAIR + cnt[1] * FLOPS_PER_RAY + cnt[2] * FLOPS_PER_NODE
                 + cnt[3] * FLOPS_PER_TRI)
        out[name] = {"gather_ms": t, "pairs_per_s": pairs / (t / 1e3), "width": cam.width, "height": cam.height,
                     "vpls": M, "achieved_tflops": flops / (t / 1e3) / 1e12,
                     "frac": flops / (t / 1e3) / 1e12 / peak_tflops,
                     "counters": {"pairs": cnt[0], "shadow_rays": cnt[1], "node_visits": cnt[2],
                                  "tri_tests": cnt[3], "blocked": cnt[4]},
                     "device_status": V.STATUS_NAMES.get(status, status)}
        del gb, vs, img
    V.vpl_scene_release(ctx.h, sid)
    return out


def serve_section(ctx, n_requests: int, factors, precision: int) -> dict:
    """Poisson arrivals of render requests over two resident scenes (the 200k
    room and the ~1M-triangle clutter); resolution 256^2 .. 1920x1080, VPL
    budgets log-uniform 1k .. 16k.  The rate is a multiple of the measured
    one-at-a-time capacity.  Continuous batching (two groups in flight, groups
    of up to 8, generation on a stream per group overlapping the previous
    group's gather, gathers in admission order on one high-priority stream,
    one batched gather per group) against a plain FIFO queue (one request per
    launch sequence, one at a time), on the same arrivals."""
    import numpy as np
    import torch
    from paper_2203_11484_gb300 import serve as S
    from paper_2203_11484_gb300 import vpl as V
    from paper_2203_11484_gb300 import workloads as W
    room, rlo, rhi = W.room200k_scene()
    clut, clo, chi = W.room1m_scene()
    scenes = {"room200k": (room, rlo, rhi, W.ROOM_D_CLOSE), "clutter1m": (clut, clo, chi, W.ROOM_D_CLOSE * 0.5)}
    sids = {k: ctx.upload(v[0]) for k, v in scenes.items()}
    n_tris = {k: v[0].n_tris for k, v in scenes.items()}

    def requests(rate, seed=11):
        return S.random_requests(np.random.default_rng(seed), scenes, n_requests, rate, precision=precision)

    # capacity: the same kind of requests rendered one at a time
    probe = requests(1.0, seed=5)[: max(8, n_requests // 4)]
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for r in probe:
        c = r.view.camera
        o = torch.empty((c.width * c.height, 4), dtype=torch.float32, device="cuda")
        V.vpl_render(ctx.h, sids[r.scene], c, r.view.gen, r.view.gather, o)
    torch.cuda.synchronize()
    capacity = len(probe) / (time.perf_counter() - t0)
    out = {"capacity_views_per_s": capacity, "requests_per_rate": n_requests, "rates": []}
    for f in factors:
        row = {"rate_factor": f, "rate_per_s": f * capacity}
        for name, lanes, group in (("plain_fifo", 1, 1), ("continuous_batching", 2, 8)):
            srv = S.Server(S.GpuBackend(ctx.h, sids, lanes), n_tris, lanes=lanes, max_group=group,
                           reserve_bytes=4 << 30)
            st = srv.run(requests(f * capacity))
            torch.cuda.synchronize()
            st["groups"] = srv.groups_launched
            st["max_concurrent_groups"] = srv.max_concurrent_groups
            row[name] = st
        out["rates"].append(row)
    status = V.vpl_sync(ctx.h, check=False)
    for s in sids.values():
        V.vpl_scene_release(ctx.h, s)
    out["device_status"] = V.STATUS_NAMES.get(status, status)
    return out


def run_reference(args):
    """Reference arm: the FP64 oracle timed on the host cores, steps of a
    bounded sample of the same workload."""
    ws, rank, _ = _dist()
    if rank != 0:
        return 0
    import oracle
    from paper_2203_11484_gb300 import workloads as W
    oracle.build()
    wl = W.room200k_workload()
    view = wl.views[0]
    cam = view.camera
    osc = oracle.OracleScene(wl.scene)
    M = view.gen.m_close + view.gen.m_far
    n_pix = 2048
    rng = np.random.default_rng(5)
    for _ in range(args.warmup):
        oracle.render(osc, view, rng.choice(cam.width * cam.height, 8, replace=False))
    times = []
    for _ in range(args.steps):
        pix = rng.choice(cam.width * cam.height, n_pix, replace=False)
        t0 = time.perf_counter()
        oracle.render(osc, view, pix)
        times.append(time.perf_counter() - t0)
    total = sum(times)
    value = n_pix * M * args.steps / total
    sample = f"per step: {n_pix} sampled pixels x {M} VPLs, G-buffer of those pixels + full generation"
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": wl.name, "width": cam.width, "height": cam.height,
                                            "vpls": M, "tris": wl.scene.n_tris, "sample_pixels": n_pix},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": oracle.num_threads(), "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def run_ours(args):
    import torch
    from paper_2203_11484_gb300 import build as B
    from paper_2203_11484_gb300 import vpl as V
    from paper_2203_11484_gb300 import workloads as W

    ws, rank, local = _dist()
    if ws > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    else:
        torch.cuda.set_device(0)
    dev = torch.cuda.current_device()
    B.build_library()

    prec = {"fp32": W.PREC_FP32, "fp16_kahan": W.PREC_FP16_KAHAN, "fp16_plain": W.PREC_FP16_PLAIN}[args.precision]
    fmt = V.FORMAT_FP32 if prec == W.PREC_FP32 else V.FORMAT_FP16
    # each rank renders its own close-up view
    if args.workload == "clutter1m":
        wl = W.room1m_workload(width=args.width or 1920, height=args.height or 1080, m_total=args.vpls or 32768,
                               precision=prec, seed=replica_seed(4, rank))
    else:
        wl = W.room200k_workload(width=args.width or 1024, height=args.height or 1024,
                                 m_total=args.vpls or 4096, precision=prec, seed=replica_seed(1, rank))
    view = wl.views[0]
    cam, gen, gat = view.camera, view.gen, view.gather
    M = gen.m_close + gen.m_far
    npx = cam.width * cam.height
    units = npx * M
    sc = wl.scene
    verts = torch.as_tensor(sc.verts).cuda()
    tris = torch.as_tensor(sc.tris).cuda()
    alb = torch.as_tensor(sc.albedo).cuda()
    out = torch.zeros((npx, 4), dtype=torch.float32, device="cuda")
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    stream = torch.cuda.current_stream()

    ctx = V.Context(dev)
    gb = V.GBuffer.empty(cam.width, cam.height, fmt=fmt)
    vs = V.VplSet.empty(M, fmt=fmt)

    def step(o, gev=None):
        """Whole hot path through the C ABI: upload + BVH, G-buffer, VPLs, gather."""
        sid = V.vpl_scene_upload(ctx.h, verts, tris, alb, sc.light, stream)
        V.vpl_gbuffer_build(ctx.h, sid, cam, gb, stream)
        V.vpl_generate(ctx.h, sid, cam, gen, vs, stream)
        if gev:
            gev[0].record(stream)
        V.vpl_gather(ctx.h, sid, gb, vs, gat, o, stream)
        if gev:
            gev[1].record(stream)
        return sid

    def barrier():
        if ws > 1:
            import torch.distributed as dist
            dist.barrier()

    # ---- warm-up -------------------------------------------------------
    sids = []
    for _ in range(args.warmup):
        sids.append(step(out))
    rc = V.vpl_sync(ctx.h, stream, check=False)
    if rc != 0:
        raise RuntimeError(f"device status {rc}: {V.vpl_last_error(ctx.h)}")
    for s in sids:
        V.vpl_scene_release(ctx.h, s)

    # ---- timed region: K steps, L2 flushed between steps ----------------
    mk = lambda: torch.cuda.Event(enable_timing=True)
    ev = [(mk(), mk()) for _ in range(args.steps)]
    gev = [(mk(), mk()) for _ in range(args.steps)]
    sids = []
    clocks = ClockSampler(dev)
    launches0 = V.vpl_launch_count(ctx.h)
    barrier()
    torch.cuda.synchronize()
    clocks.start()
    wall0 = time.perf_counter()
    for k in range(args.steps):
        flush.fill_(float(k))
        ev[k][0].record(stream)
        sids.append(step(out, gev[k]))
        ev[k][1].record(stream)
    torch.cuda.synchronize()
    wall = time.perf_counter() - wall0
    barrier()
    clk = clocks.stop()
    launches = V.vpl_launch_count(ctx.h) - launches0
    rc = V.vpl_sync(ctx.h, stream, check=False)
    if rc != 0:
        raise RuntimeError(f"device status {rc}: {V.vpl_last_error(ctx.h)}")
    step_ms = [a.elapsed_time(b) for a, b in ev]
    gather_ms = [a.elapsed_time(b) for a, b in gev]
    total_ms = max_over_ranks(sum(step_ms), "cuda")
    for s in sids:
        V.vpl_scene_release(ctx.h, s)
    value = job_throughput(units, args.steps, ws, total_ms)

    # ---- gather roofline: work counters of the last step's inputs (untimed) --
    sid = V.vpl_scene_upload(ctx.h, verts, tris, alb, sc.light, stream)
    V.vpl_gbuffer_build(ctx.h, sid, cam, gb, stream)
    V.vpl_generate(ctx.h, sid, cam, gen, vs, stream)
    cnt = V.vpl_gather_counters(ctx.h, sid, gb, vs, gat, stream)
    V.vpl_sync(ctx.h, stream)
    flops = (cnt[0] * FLOPS_PER_PAIR + cnt[1] * FLOPS_PER_RAY + cnt[2] * FLOPS_PER_NODE
             + cnt[3] * FLOPS_PER_TRI)
    gather_in_step_ms = statistics.mean(gather_ms)
    props = torch.cuda.get_device_properties(dev)
    sms = props.multi_processor_count
    max_mhz = (clk.get("sm_max_mhz") or _peaks().get("sm_max_mhz") or 2070.0)
    peak_tflops = sms * 128 * 2 * max_mhz * 1e6 / 1e12
    achieved = flops / (gather_in_step_ms / 1e3) / 1e12
    roofline = {"bound": "alu", "achieved": achieved, "peak": peak_tflops, "unit": "TFLOP/s",
                "frac": achieved / peak_tflops, "traffic": measured_traffic(wl.name, args.precision),
                "traffic_note": "DRAM bytes per launch (ncu, profiles/); the working set is L2-resident",
                "kernel": f"gather_kernel<BVH,{args.precision}>",
                "peak_note": f"FP32 FMA pipe: {sms} SMs x 128 lanes x 2 x {max_mhz:.0f} MHz",
                "counters": {"pairs": cnt[0], "shadow_rays": cnt[1], "node_visits": cnt[2],
                             "tri_tests": cnt[3], "blocked": cnt[4], "warp_steps": cnt[5],
                             "lane_utilisation": cnt[2] / max(1, 32 * cnt[5])},
                "gather_ms": gather_in_step_ms,
                "flops_per_unit": {"pair": FLOPS_PER_PAIR, "ray": FLOPS_PER_RAY, "node": FLOPS_PER_NODE,
                                   "tri": FLOPS_PER_TRI}}
    # ---- shading-only probe: the same launch with V = 1 (no shadow rays) ----
    # isolates the Eq. 1 arithmetic from the BVH walks; not part of the metric
    import dataclasses
    gat_v1 = dataclasses.replace(gat, visibility=W.VIS_NONE)
    probe_ms = []
    for k in range(4):
        flush.fill_(float(k))
        e0, e1 = mk(), mk()
        e0.record(stream)
        V.vpl_gather(ctx.h, sid, gb, vs, gat_v1, out, stream)
        e1.record(stream)
        torch.cuda.synchronize()
        if k:
            probe_ms.append(e0.elapsed_time(e1))
    V.vpl_sync(ctx.h, stream)
    v1_ms = statistics.mean(probe_ms)
    v1_tflops = cnt[0] * FLOPS_PER_PAIR / (v1_ms / 1e3) / 1e12
    med_mhz = clk.get("sm_mhz") or max_mhz
    roofline["shading_only"] = {
        "visibility": "none (V = 1)", "gather_ms": v1_ms, "pairs_per_s": cnt[0] / (v1_ms / 1e3),
        "achieved": v1_tflops, "frac": v1_tflops / peak_tflops,
        "frac_at_median_clock": v1_tflops / (sms * 128 * 2 * med_mhz * 1e6 / 1e12)}
    roofline["frac_at_median_clock"] = achieved / (sms * 128 * 2 * med_mhz * 1e6 / 1e12)

    # ---- direct term (Eq. 1's L_e(y)) as light-sample VPLs, composite image ----
    # reported beside the metric, which counts the indirect VPLs only
    direct = None
    if sc.light.type == W.LIGHT_AREA:
        n_light = 256
        both = V.VplSet.empty(M + n_light, fmt=fmt)
        V.vpl_generate(ctx.h, sid, cam, gen, both.rows(0, M), stream)
        V.vpl_light_vpls(ctx.h, sid, n_light, 1, both.rows(M, n_light), stream)
        times = {}
        for name, part in (("direct", both.rows(M, n_light)), ("composite", both)):
            ms = []
            for k in range(3):
                flush.fill_(float(k))
                e0, e1 = mk(), mk()
                e0.record(stream)
                V.vpl_gather(ctx.h, sid, gb, part, gat, out, stream)
                e1.record(stream)
                torch.cuda.synchronize()
                if k:
                    ms.append(e0.elapsed_time(e1))
            times[name] = statistics.mean(ms)
        V.vpl_sync(ctx.h, stream)
        direct = {"light_vpls": n_light, "direct_gather_ms": times["direct"],
                  "direct_pairs_per_s": npx * n_light / (times["direct"] / 1e3),
                  "composite_vpls": M + n_light, "composite_gather_ms": times["composite"],
                  "composite_pairs_per_s": npx * (M + n_light) / (times["composite"] / 1e3)}
    V.vpl_scene_release(ctx.h, sid)

    # ---- end to end: host buffers in, image out, through the same API -----
    e2e = None
    if not args.no_e2e:
        hv = torch.as_tensor(sc.verts).pin_memory()
        ht = torch.as_tensor(sc.tris).pin_memory()
        ha = torch.as_tensor(sc.albedo).pin_memory()
        hout = torch.empty((npx, 4), dtype=torch.float32).pin_memory()
        e_ms = []
        sids = []
        for k in range(max(1, min(args.steps, 5))):
            flush.fill_(2.0)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            s = V.vpl_scene_upload(ctx.h, hv, ht, ha, sc.light, stream)
            V.vpl_render(ctx.h, s, cam, gen, gat, out, stream)
            hout.copy_(out, non_blocking=True)
            e1.record(stream)
            torch.cuda.synchronize()
            e_ms.append(e0.elapsed_time(e1))
            sids.append(s)
        V.vpl_sync(ctx.h, stream)
        for s in sids:
            V.vpl_scene_release(ctx.h, s)
        h2d = hv.numel() * 4 + ht.numel() * 4 + ha.numel() * 4
        e2e = {"value": units * ws / (statistics.mean(e_ms) / 1e3), "unit": UNIT,
               "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": hout.numel() * 4,
               "ms_per_step": statistics.mean(e_ms)}

    batch = batch_fp16 = None
    if args.batch_views > 0 and args.workload == "room200k":
        batch = batch_section(ctx, args.batch_views, prec)
        if prec == W.PREC_FP32:
            batch_fp16 = batch_section(ctx, args.batch_views, W.PREC_FP16_KAHAN)
    large = None
    if args.large and args.workload == "room200k":
        large = large_section(ctx, peak_tflops)
    serving = None
    if args.serve_requests > 0 and args.workload == "room200k":
        serving = serve_section(ctx, args.serve_requests, [float(x) for x in args.serve_rates.split(",")], prec)

    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        try:
            cpu = cpu_baseline(wl, seconds=args.cpu_seconds)
            if args.workload == "room200k" and args.width == 0 and args.height == 0 and args.vpls == 0:
                cpu["configs"] = cpu_configs(cpu["value"], wl)
        except Exception as exc:  # the baseline is reported, never required
            cpu = {"value": None, "unit": UNIT, "cores": None, "kind": "oracle", "sample": f"failed: {exc}"}

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None,
                "dtype": "f32" if prec == W.PREC_FP32 else "f16 attributes, f32 shading", "data": "synthetic",
                "config": {"workload": wl.name, "width": cam.width, "height": cam.height, "vpls": M,
                           "m_close": gen.m_close, "m_far": gen.m_far, "tris": sc.n_tris,
                           "visibility": "bvh", "parallelism": f"replicas x{ws}",
                           "l2": "flushed (256 MB write) before every step; per-step CUDA events",
                           "step": "scene upload + BVH build + G-buffer + VPL generation + gather"},
                "views_per_s": ws * args.steps / (total_ms / 1e3),
                "gather_ms_per_step": gather_in_step_ms,
                "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e,
                "gpu_launches": int(launches), "clocks": clk, "wall_s": wall, "direct_term": direct, "batch": batch,
                "batch_fp16_kahan": batch_fp16, "large": large, "serving": serving}
        print(json.dumps(line), flush=True)
    ctx.close()
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--batch-views", type=int, default=64,
                    help="views of the batched comparison (0: skip)")
    ap.add_argument("--serve-requests", type=int, default=200,
                    help="requests per arrival rate in the serving comparison (0: skip)")
    ap.add_argument("--serve-rates", default="0.5,1.0,1.5",
                    help="arrival rates as multiples of the one-at-a-time capacity")
    ap.add_argument("--large", type=int, default=1,
                    help="1: add the 1M-triangle 1920x1080 x 32768 gather in three precisions (0: skip)")
    ap.add_argument("--workload", default="room200k", choices=["room200k", "clutter1m"])
    ap.add_argument("--precision", default="fp32", choices=["fp32", "fp16_kahan", "fp16_plain"])
    ap.add_argument("--width", type=int, default=0, help="0: the workload's size")
    ap.add_argument("--height", type=int, default=0)
    ap.add_argument("--vpls", type=int, default=0)
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
