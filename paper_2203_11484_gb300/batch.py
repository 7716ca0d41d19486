"""Many views of one resident scene, rendered as a batch.

Each view keeps its own G-buffer, VPL set and image (resolutions and VPL
budgets may all differ).  Per view, vpl_gbuffer_build and vpl_generate fill
the buffers; then ONE vpl_gather_batch launch gathers every view: its warps
take 32-pixel tiles of all views from one queue, so small views do not leave
the GPU idle and large ones do not serialise.  The whole sequence can be
captured once into a CUDA graph and replayed.

The gather's pixel tile shape (tile_w), VPL tile (vpl_tile: VPLs a warp
stages in shared memory at a time) and resident-block cap (blocks_per_sm)
only change speed, never the images; `autotune` times the candidates on the
batch itself and keeps the fastest per batch signature.
"""
from __future__ import annotations

from typing import Dict, List, Optional, Sequence, Tuple

import torch

from . import vpl as V
from . import workloads as W

Config = Tuple[int, int, int]  # (tile_w, blocks_per_sm, vpl_tile)

# pixel tile x VPL tile, then resident-block caps at the default tiles
CANDIDATES: List[Config] = ([(tw, 0, vt) for tw in (8, 4, 16, 32) for vt in (64, 32, 16)]
                            + [(8, 4, 64), (8, 3, 64)])
_TUNED: Dict[tuple, Config] = {}


class BatchRenderer:
    def __init__(self, ctx, scene_id: int, views: Sequence[W.View], precision: int = W.PREC_FP32,
                 device: str = "cuda"):
        self.ctx = ctx
        self.sid = scene_id
        self.views = list(views)
        self.precision = precision
        self.fmt = V.FORMAT_FP32 if precision == W.PREC_FP32 else V.FORMAT_FP16
        self.gbufs, self.vsets, self.outs = [], [], []
        for v in self.views:
            c = v.camera
            self.gbufs.append(V.GBuffer.empty(c.width, c.height, device, self.fmt))
            self.vsets.append(V.VplSet.empty(v.gen.m_close + v.gen.m_far, device, self.fmt))
            self.outs.append(torch.zeros((c.width * c.height, 4), dtype=torch.float32, device=device))
        g0 = self.views[0].gather
        self.base = W.GatherParams(g0.d2_min, g0.ray_eps, precision, g0.visibility)
        self._batches: Dict[int, int] = {}
        self.config: Optional[Config] = None
        self.tune_ms: Dict[Config, float] = {}   # every candidate's time in the last autotune
        self.graph: Optional[torch.cuda.CUDAGraph] = None
        self.graph_includes_generation = False

    # ------------------------------------------------------------------
    def signature(self) -> tuple:
        return (self.precision, self.base.visibility,
                tuple((v.camera.width, v.camera.height, v.gen.m_close + v.gen.m_far) for v in self.views))

    def pairs(self) -> int:
        return sum(v.camera.width * v.camera.height * (v.gen.m_close + v.gen.m_far) for v in self.views)

    def _batch(self, tile_w: int) -> int:
        if tile_w not in self._batches:
            self._batches[tile_w] = V.vpl_batch_create(self.ctx, self.gbufs, self.vsets, self.outs, tile_w)
        return self._batches[tile_w]

    def _params(self, cfg: Config) -> W.GatherParams:
        return W.GatherParams(self.base.d2_min, self.base.ray_eps, self.base.precision, self.base.visibility,
                              tile_w=cfg[0], blocks_per_sm=cfg[1], vpl_tile=cfg[2] if len(cfg) > 2 else 0)

    # ---- the pipeline -----------------------------------------------------
    def prepare(self, stream=None) -> None:
        """G-buffer and VPLs of every view (pipeline steps (1)-(3))."""
        for v, gb, vs in zip(self.views, self.gbufs, self.vsets):
            V.vpl_gbuffer_build(self.ctx, self.sid, v.camera, gb, stream)
            V.vpl_generate(self.ctx, self.sid, v.camera, v.gen, vs, stream)

    def gather(self, stream=None, config: Optional[Config] = None) -> None:
        """Step (4) for all views in one launch."""
        cfg = config or self.config or CANDIDATES[0]
        V.vpl_gather_batch(self.ctx, self.sid, self._batch(cfg[0]), self._params(cfg), stream)

    def run(self, stream=None) -> None:
        self.prepare(stream)
        self.gather(stream)

    # ---- tuning -----------------------------------------------------------------
    def autotune(self, candidates: Sequence[Config] = CANDIDATES, reps: int = 1) -> Config:
        sig = self.signature()
        if sig in _TUNED:
            self.config = _TUNED[sig]
            return self.config
        self.prepare()
        V.vpl_sync(self.ctx)
        best, best_ms = None, float("inf")
        self.tune_ms = {}
        stream = torch.cuda.current_stream()
        for cfg in candidates:
            self.gather(config=cfg)           # warm-up of this shape
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for _ in range(reps):
                self.gather(config=cfg)
            e1.record(stream)
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1) / reps
            self.tune_ms[tuple(cfg)] = ms
            if ms < best_ms:
                best, best_ms = cfg, ms
        V.vpl_sync(self.ctx)
        _TUNED[sig] = best
        self.config = best
        return best

    # ---- CUDA graph ---------------------------------------------------------------
    def capture(self, include_generation: bool = True) -> None:
        """Capture the batch into a CUDA graph (after warm-up and tuning).
        With include_generation the graph holds G-buffers, VPL generation and
        the gather; otherwise only the single batched gather launch."""
        self.run()
        V.vpl_sync(self.ctx)
        side = torch.cuda.Stream()
        side.wait_stream(torch.cuda.current_stream())
        g = torch.cuda.CUDAGraph()
        with torch.cuda.stream(side):
            with torch.cuda.graph(g, stream=side):
                if include_generation:
                    self.prepare(side)
                self.gather(side)
        torch.cuda.current_stream().wait_stream(side)
        self.graph = g
        self.graph_includes_generation = include_generation

    def replay(self) -> None:
        if self.graph is None:
            raise RuntimeError("capture() first")
        self.graph.replay()

    def close(self) -> None:
        for b in self._batches.values():
            V.vpl_batch_destroy(self.ctx, b)
        self._batches.clear()
        self.graph = None
