"""Serving loop: render requests over resident scenes with continuous batching.

Scenes (and their BVHs) stay on the device.  Requests (a view of one scene:
camera, resolution, VPL budget) arrive over time and wait in a FIFO queue.
Whenever one of the `lanes` (groups in flight) is free, the scheduler admits
the oldest requests of one scene -- up to `max_group` of them, as long as
their estimated device memory fits the budget -- and launches them as a
group: per request the G-buffer and VPL generation, then ONE batched gather
for the whole group (vpl_gather_views).  Requests that arrive while others
are on the GPU are admitted as soon as a lane and memory free up.

On the device (GpuBackend) the groups form a two-stage pipeline: each
group's G-buffers and VPL generations run on a stream of its own, and the
gathers -- the persistent launches that fill the whole GPU -- run on ONE
high-priority stream in admission order.  So the oldest request's gather
never shares the SMs with a newer group's gather, while the next group's
generation overlaps the running gather; requests that queue up behind a
running gather are batched into the next group.  Every pixel is summed in
VPL order by one thread, so a request's image is the same alone and in any
mix.

The scheduler is independent of the GPU: `Backend` launches groups and
reports completion; `GpuBackend` does it with libvpl.
"""
from __future__ import annotations

import collections
import math
import time
from dataclasses import dataclass, field
from typing import Callable, Dict, List, Optional, Sequence

import numpy as np

from . import workloads as W


@dataclass
class Request:
    rid: int
    scene: str
    view: W.View
    arrival: float                    # seconds after the start of the run
    t_admit: Optional[float] = None
    t_done: Optional[float] = None
    image: object = None              # device tensor [H*W, 4] once done

    @property
    def latency(self) -> float:
        return self.t_done - self.arrival


def estimate_bytes(view: W.View, n_tris: int) -> int:
    """Device memory one request holds while it is in flight: its G-buffer,
    VPL set and image, plus VPL generation scratch (per triangle for the
    close-range sort and area scan, per light-path slot for the IR walks)."""
    c, g = view.camera, view.gen
    px = c.width * c.height
    m = g.m_close + g.m_far
    row = 16 + 2 * (8 if view.gather.precision != W.PREC_FP32 else 16)
    paths = g.resolved_max_paths()
    return px * (row + 16) + m * row + 64 * n_tris + 80 * paths * g.max_bounces


class Backend:
    def free_bytes(self) -> int:
        raise NotImplementedError

    def launch(self, group: List[Request], lane: int):
        raise NotImplementedError

    def done(self, handle) -> bool:
        raise NotImplementedError


class Server:
    def __init__(self, backend: Backend, n_tris: Dict[str, int], lanes: int = 4, max_group: int = 8,
                 reserve_bytes: int = 1 << 30, clock: Callable[[], float] = time.perf_counter):
        self.backend = backend
        self.n_tris = n_tris
        self.lanes = lanes
        self.max_group = max_group
        self.reserve = reserve_bytes
        self.clock = clock
        self.queue: collections.deque = collections.deque()
        self.running: Dict[int, tuple] = {}     # lane -> (group, handle, bytes)
        self.finished: List[Request] = []
        self.max_in_flight_bytes = 0
        self.max_concurrent_groups = 0
        self.groups_launched = 0
        # the server's device memory budget: what is free when it starts, less
        # the reserve; admission charges each group's estimate against it
        # (allocations of running groups may not have happened yet, so the
        # free memory of the moment is not a safe measure)
        self.budget = backend.free_bytes() - reserve_bytes

    def submit(self, r: Request) -> None:
        self.queue.append(r)

    def in_flight_bytes(self) -> int:
        return sum(b for _, _, b in self.running.values())

    def tick(self, now: float) -> bool:
        """Retire finished groups, admit new ones; True if anything changed."""
        changed = False
        for lane, (group, h, _) in list(self.running.items()):
            if self.backend.done(h):
                for r in group:
                    r.t_done = now
                    self.finished.append(r)
                del self.running[lane]
                changed = True
        budget = self.budget - self.in_flight_bytes()
        for lane in range(self.lanes):
            if lane in self.running or not self.queue:
                continue
            head = self.queue[0]
            group, need = [], 0
            while (self.queue and len(group) < self.max_group and self.queue[0].scene == head.scene
                   and self.queue[0].view.gather == head.view.gather):
                e = estimate_bytes(self.queue[0].view, self.n_tris[head.scene])
                if need + e > budget:
                    break
                group.append(self.queue.popleft())
                need += e
            if not group:
                break                               # memory is full: wait for a group to finish
            for r in group:
                r.t_admit = now
            self.running[lane] = (group, self.backend.launch(group, lane), need)
            self.groups_launched += 1
            budget -= need
            changed = True
            self.max_in_flight_bytes = max(self.max_in_flight_bytes, self.in_flight_bytes())
            self.max_concurrent_groups = max(self.max_concurrent_groups, len(self.running))
        return changed

    def run(self, requests: Sequence[Request], poll_s: float = 2e-4) -> dict:
        reqs = sorted(requests, key=lambda r: r.arrival)
        t0 = self.clock()
        i = 0
        while i < len(reqs) or self.queue or self.running:
            now = self.clock() - t0
            while i < len(reqs) and reqs[i].arrival <= now:
                self.submit(reqs[i])
                i += 1
            if not self.tick(now) and poll_s > 0:
                time.sleep(poll_s)
        return summarize(self.finished)


def summarize(done: Sequence[Request]) -> dict:
    if not done:
        return {"requests": 0}
    lat = np.array([r.latency for r in done])
    span = max(r.t_done for r in done) - min(r.arrival for r in done)
    return {"requests": len(done), "p50_ms": float(np.percentile(lat, 50) * 1e3),
            "p99_ms": float(np.percentile(lat, 99) * 1e3), "mean_ms": float(lat.mean() * 1e3),
            "views_per_s": len(done) / span if span > 0 else float("inf")}


def poisson_arrivals(rng, rate: float, n: int) -> List[float]:
    return list(np.cumsum(rng.exponential(1.0 / rate, size=n)))


def random_requests(rng, scenes: Dict[str, tuple], n: int, rate: float,
                    resolutions=((256, 256), (512, 512), (1280, 720), (1920, 1080)),
                    m_range=(1000, 16000), alpha=0.75, precision=W.PREC_FP32) -> List[Request]:
    """Requests with random close-up cameras over the named scenes.
    scenes[name] = (Scene, box_lo, box_hi, d_close)."""
    names = sorted(scenes)
    arrivals = poisson_arrivals(rng, rate, n)
    out = []
    for k in range(n):
        name = names[rng.integers(len(names))]
        sc, lo, hi, d_close = scenes[name]
        sx, sy = float(sc.verts[:, 0].max()), float(sc.verts[:, 1].max())
        w, h = resolutions[rng.integers(len(resolutions))]
        cam = W.close_up_camera(rng, lo, hi, (sx / 2, sy / 2), 6.0, (0.8, 2.0), (2.0, 5.0), int(w), int(h))
        m = int(round(math.exp(rng.uniform(math.log(m_range[0]), math.log(m_range[1])))))
        mc, mf = W.split_budget(m, alpha)
        gen = W.GenParams(d_close=d_close, m_close=mc, m_far=mf, seed=1000 + k, ray_eps=W.ROOM_RAY_EPS)
        gat = W.GatherParams(W.ROOM_D2_MIN, W.ROOM_RAY_EPS, precision)
        out.append(Request(k, name, W.View(cam, gen, gat), float(arrivals[k])))
    return out


class GpuBackend(Backend):
    """Groups through libvpl: generation on a low-priority stream per lane,
    gathers on one high-priority stream in launch order."""

    def __init__(self, ctx, scene_ids: Dict[str, int], lanes: int):
        import torch
        from . import vpl as V
        self.torch = torch
        self.V = V
        self.ctx = ctx
        self.sids = scene_ids
        self.streams = [torch.cuda.Stream(priority=0) for _ in range(lanes)]
        self.gather_stream = torch.cuda.Stream(priority=-1)

    def free_bytes(self) -> int:
        t = self.torch
        free, _ = t.cuda.mem_get_info()
        return int(free + t.cuda.memory_reserved() - t.cuda.memory_allocated())

    def launch(self, group: List[Request], lane: int):
        t, V = self.torch, self.V
        s, gs = self.streams[lane], self.gather_stream
        gbufs, vsets, outs = [], [], []
        with t.cuda.stream(s):
            for r in group:
                c, g = r.view.camera, r.view.gen
                fmt = V.FORMAT_FP32 if r.view.gather.precision == W.PREC_FP32 else V.FORMAT_FP16
                gb = V.GBuffer.empty(c.width, c.height, "cuda", fmt)
                vs = V.VplSet.empty(g.m_close + g.m_far, "cuda", fmt)
                out = t.empty((c.width * c.height, 4), dtype=t.float32, device="cuda")
                V.vpl_gbuffer_build(self.ctx, self.sids[r.scene], c, gb, s)
                V.vpl_generate(self.ctx, self.sids[r.scene], c, g, vs, s)
                gbufs.append(gb)
                vsets.append(vs)
                outs.append(out)
                r.image = out
            prepared = t.cuda.Event()
            prepared.record(s)
        # the group's buffers were allocated on stream s and are used on gs
        for x in gbufs:
            for a in (x.pos, x.nrm, x.albedo):
                a.record_stream(gs)
        for x in vsets:
            for a in (x.pos, x.nrm, x.flux):
                a.record_stream(gs)
        for a in outs:
            a.record_stream(gs)
        gs.wait_event(prepared)
        with t.cuda.stream(gs):
            V.vpl_gather_views(self.ctx, self.sids[group[0].scene], gbufs, vsets, outs, group[0].view.gather, gs)
            ev = t.cuda.Event()
            ev.record(gs)
        return (ev, gbufs, vsets)

    def done(self, handle) -> bool:
        return handle[0].query()
