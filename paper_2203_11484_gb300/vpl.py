"""ctypes binding of libvpl's C ABI (include/vpl.h).

The functions below carry the names of the C entry points and only marshal
arguments: every step of the pipeline runs in the library's CUDA kernels.
Device buffers are torch tensors (PyTorch provides device memory and
streams); host arrays may be numpy arrays or CPU tensors.  There is no CPU
fallback: without the built library every call raises.
"""
from __future__ import annotations

import ctypes as C
import os
import threading
from dataclasses import dataclass
from typing import Optional, Sequence

import numpy as np

from . import build as _build
from . import workloads as W

VPL_OK = 0
STATUS_NAMES = {0: "OK", 1: "INVALID_ARG", 2: "OOM", 3: "CUDA", 4: "TRAVERSAL_LIMIT", 5: "NOT_FOUND",
                6: "EMPTY_CLOSE", 7: "PATHS_EXHAUSTED", 8: "UNSUPPORTED"}
FORMAT_FP32, FORMAT_FP16 = 0, 1


class VplError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"vpl error {code} ({STATUS_NAMES.get(code, '?')}): {msg}")
        self.code = code


# ---- structures mirroring include/vpl.h ------------------------------------
class vpl_light(C.Structure):
    _fields_ = [("center", C.c_float * 3), ("normal", C.c_float * 3), ("edge_u", C.c_float * 3),
                ("edge_v", C.c_float * 3), ("power", C.c_float * 3), ("type", C.c_int32)]


class vpl_camera(C.Structure):
    _fields_ = [("eye", C.c_float * 3), ("forward", C.c_float * 3), ("up", C.c_float * 3),
                ("vfov_deg", C.c_float), ("width", C.c_int32), ("height", C.c_int32)]


class vpl_gen_params(C.Structure):
    _fields_ = [("d_close", C.c_double), ("ray_eps", C.c_float), ("m_close", C.c_int32),
                ("m_far", C.c_int32), ("max_bounces", C.c_int32), ("light_samples", C.c_int32),
                ("rules", C.c_int32), ("ir_max_paths", C.c_int64), ("seed", C.c_uint64)]


class vpl_gather_params(C.Structure):
    _fields_ = [("d2_min", C.c_float), ("ray_eps", C.c_float), ("precision", C.c_int32),
                ("visibility", C.c_int32), ("tile_w", C.c_int32), ("blocks_per_sm", C.c_int32),
                ("vpl_tile", C.c_int32), ("walk", C.c_int32), ("tile_order", C.c_int32)]


class vpl_vpl_set(C.Structure):
    _fields_ = [("pos", C.c_void_p), ("nrm", C.c_void_p), ("flux", C.c_void_p),
                ("count", C.c_int32), ("format", C.c_int32)]


class vpl_gbuffer(C.Structure):
    _fields_ = [("pos", C.c_void_p), ("nrm", C.c_void_p), ("albedo", C.c_void_p),
                ("width", C.c_int32), ("height", C.c_int32), ("format", C.c_int32),
                ("reserved", C.c_int32)]


class vpl_scene_info(C.Structure):
    _fields_ = [("n_tris", C.c_int64), ("n_nodes", C.c_int64), ("depth", C.c_int64),
                ("device_bytes", C.c_int64), ("bounds_lo", C.c_float * 3),
                ("bounds_hi", C.c_float * 3)]


class vpl_gen_info(C.Structure):
    _fields_ = [("n_close", C.c_int64), ("shift_s", C.c_int64), ("f_total", C.c_uint64),
                ("paths", C.c_int64), ("m_far_kept", C.c_int64), ("status", C.c_int64)]


# ---- library loading -----------------------------------------------------------
_lock = threading.Lock()
_L: Optional[C.CDLL] = None

_P = C.c_void_p
_SIGS = {
    "vpl_create": (C.c_int, [C.POINTER(C.c_void_p), C.c_int]),
    "vpl_destroy": (None, [_P]),
    "vpl_last_error": (C.c_char_p, [_P]),
    "vpl_scene_upload": (C.c_int, [_P, _P, C.c_int64, _P, C.c_int64, _P, C.POINTER(vpl_light), _P,
                                   C.POINTER(C.c_uint64)]),
    "vpl_scene_release": (C.c_int, [_P, C.c_uint64]),
    "vpl_scene_query": (C.c_int, [_P, C.c_uint64, C.POINTER(vpl_scene_info)]),
    "vpl_gbuffer_build": (C.c_int, [_P, C.c_uint64, C.POINTER(vpl_camera), C.POINTER(vpl_gbuffer), _P]),
    "vpl_light_vpls": (C.c_int, [_P, C.c_uint64, C.c_int32, C.c_uint64, C.POINTER(vpl_vpl_set), _P]),
    "vpl_generate_rs": (C.c_int, [_P, C.c_uint64, C.POINTER(vpl_camera), C.POINTER(vpl_gen_params), C.c_int32,
                                  C.c_float, C.c_float, C.POINTER(vpl_vpl_set), _P]),
    "vpl_generate": (C.c_int, [_P, C.c_uint64, C.POINTER(vpl_camera), C.POINTER(vpl_gen_params),
                               C.POINTER(vpl_vpl_set), _P]),
    "vpl_generate_info": (C.c_int, [_P, C.POINTER(vpl_gen_info)]),
    "vpl_gather": (C.c_int, [_P, C.c_uint64, C.POINTER(vpl_gbuffer), C.POINTER(vpl_vpl_set),
                             C.POINTER(vpl_gather_params), _P, _P]),
    "vpl_gather_noalloc": (C.c_int, [_P, C.c_uint64, C.POINTER(vpl_gbuffer), C.POINTER(vpl_vpl_set),
                                     C.POINTER(vpl_gather_params), _P, _P]),
    "vpl_batch_create": (C.c_int, [_P, C.c_int32, C.POINTER(vpl_gbuffer), C.POINTER(vpl_vpl_set),
                                   C.POINTER(C.c_void_p), C.c_int32, C.POINTER(C.c_uint64)]),
    "vpl_batch_destroy": (C.c_int, [_P, C.c_uint64]),
    "vpl_gather_views": (C.c_int, [_P, C.c_uint64, C.c_int32, C.POINTER(vpl_gbuffer), C.POINTER(vpl_vpl_set),
                                   C.POINTER(C.c_void_p), C.POINTER(vpl_gather_params), _P]),
    "vpl_gather_batch": (C.c_int, [_P, C.c_uint64, C.c_uint64, C.POINTER(vpl_gather_params), _P]),
    "vpl_render": (C.c_int, [_P, C.c_uint64, C.POINTER(vpl_camera), C.POINTER(vpl_gen_params),
                             C.POINTER(vpl_gather_params), _P, _P]),
    "vpl_sync": (C.c_int, [_P, _P]),
    "vpl_debug_philox": (C.c_int, [_P, _P, _P, C.c_int64, _P, _P]),
    "vpl_debug_rays": (C.c_int, [_P, C.c_uint64, C.c_int32, C.c_int32, _P, _P, C.c_int64, _P, _P, _P]),
    "vpl_debug_visibility": (C.c_int, [_P, C.c_uint64, C.POINTER(vpl_gbuffer), C.POINTER(vpl_vpl_set),
                                       C.POINTER(vpl_gather_params), _P, C.c_int64, _P, _P]),
    "vpl_set_timing": (C.c_int, [_P, C.c_int32]),
    "vpl_stage_times": (C.c_int, [_P, C.POINTER(C.c_float), C.c_int32]),
    "vpl_launch_count": (C.c_int64, [_P]),
    "vpl_pool_stats": (C.c_int, [_P, C.c_int32, C.POINTER(C.c_uint64)]),
    "vpl_gather_counters": (C.c_int, [_P, C.c_uint64, C.POINTER(vpl_gbuffer), C.POINTER(vpl_vpl_set),
                                      C.POINTER(vpl_gather_params), C.POINTER(C.c_uint64), _P]),
}


def library_path() -> str:
    return _build.LIB


def load(path: Optional[str] = None) -> C.CDLL:
    """Loads libvpl.so (built by build.build_library()); raises if it is missing."""
    global _L
    with _lock:
        if _L is None:
            p = path or _build.LIB
            if not os.path.exists(p):
                raise RuntimeError(f"libvpl.so not found at {p}: build it first "
                                   "(python -m paper_2203_11484_gb300.build)")
            lib = C.CDLL(p)
            for name, (res, args) in _SIGS.items():
                f = getattr(lib, name)
                f.restype = res
                f.argtypes = args
            _L = lib
    return _L


def _check(ctx, rc: int, what: str):
    if rc != VPL_OK:
        msg = load().vpl_last_error(ctx) if ctx else b""
        raise VplError(rc, f"{what}: {(msg or b'').decode()}")


def _stream(stream) -> Optional[int]:
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def _ptr(x) -> Optional[int]:
    """Device or host address of a torch tensor / numpy array (contiguous)."""
    if x is None:
        return None
    if isinstance(x, np.ndarray):
        if not x.flags["C_CONTIGUOUS"]:
            raise ValueError("array must be C-contiguous")
        return x.ctypes.data
    if not x.is_contiguous():
        raise ValueError("tensor must be contiguous")
    return x.data_ptr()


# ---- structure builders ----------------------------------------------------------
def make_light(L: W.Light) -> vpl_light:
    s = vpl_light()
    for n in ("center", "normal", "edge_u", "edge_v", "power"):
        getattr(s, n)[:] = [float(v) for v in getattr(L, n)]
    s.type = int(L.type)
    return s


def make_camera(c: W.Camera) -> vpl_camera:
    s = vpl_camera()
    s.eye[:] = [float(v) for v in c.eye]
    s.forward[:] = [float(v) for v in c.forward]
    s.up[:] = [float(v) for v in c.up]
    s.vfov_deg = float(c.vfov_deg)
    s.width, s.height = int(c.width), int(c.height)
    return s


def make_gen(g: W.GenParams) -> vpl_gen_params:
    s = vpl_gen_params()
    s.d_close = float(g.d_close)
    s.ray_eps = float(g.ray_eps)
    s.m_close, s.m_far = int(g.m_close), int(g.m_far)
    s.max_bounces, s.light_samples = int(g.max_bounces), int(g.light_samples)
    s.ir_max_paths = int(g.ir_max_paths)
    s.seed = int(g.seed)
    s.rules = (1 if g.close_rule else 0) | (2 if g.patch_rule else 0)
    return s


def make_gather(p: W.GatherParams) -> vpl_gather_params:
    s = vpl_gather_params()
    s.d2_min, s.ray_eps = float(p.d2_min), float(p.ray_eps)
    s.precision, s.visibility = int(p.precision), int(p.visibility)
    s.tile_w, s.blocks_per_sm = int(getattr(p, "tile_w", 0)), int(getattr(p, "blocks_per_sm", 0))
    s.vpl_tile = int(getattr(p, "vpl_tile", 0))
    s.walk = int(getattr(p, "walk", 0))
    s.tile_order = int(getattr(p, "tile_order", 0))
    return s


# ---- device buffers (torch) --------------------------------------------------------
@dataclass
class GBuffer:
    pos: "torch.Tensor"      # float32 [H*W, 4]
    nrm: "torch.Tensor"      # float32 [H*W, 4] or float16 [H*W, 4]
    albedo: "torch.Tensor"
    width: int
    height: int
    format: int = FORMAT_FP32

    @staticmethod
    def empty(width: int, height: int, device="cuda", fmt: int = FORMAT_FP32) -> "GBuffer":
        import torch
        n = width * height
        adt = torch.float32 if fmt == FORMAT_FP32 else torch.float16
        return GBuffer(torch.empty((n, 4), dtype=torch.float32, device=device),
                       torch.empty((n, 4), dtype=adt, device=device),
                       torch.empty((n, 4), dtype=adt, device=device), width, height, fmt)

    def struct(self) -> vpl_gbuffer:
        s = vpl_gbuffer()
        s.pos, s.nrm, s.albedo = _ptr(self.pos), _ptr(self.nrm), _ptr(self.albedo)
        s.width, s.height, s.format = self.width, self.height, self.format
        return s


@dataclass
class VplSet:
    pos: "torch.Tensor"      # float32 [M, 4]
    nrm: "torch.Tensor"
    flux: "torch.Tensor"
    format: int = FORMAT_FP32

    @property
    def count(self) -> int:
        return int(self.pos.shape[0])

    @staticmethod
    def empty(count: int, device="cuda", fmt: int = FORMAT_FP32) -> "VplSet":
        import torch
        adt = torch.float32 if fmt == FORMAT_FP32 else torch.float16
        return VplSet(torch.empty((count, 4), dtype=torch.float32, device=device),
                      torch.empty((count, 4), dtype=adt, device=device),
                      torch.empty((count, 4), dtype=adt, device=device), fmt)

    def struct(self) -> vpl_vpl_set:
        s = vpl_vpl_set()
        s.pos, s.nrm, s.flux = _ptr(self.pos), _ptr(self.nrm), _ptr(self.flux)
        s.count, s.format = self.count, self.format
        return s

    def rows(self, first: int, count: int) -> "VplSet":
        """Rows [first, first + count) of this set (views, no copy): e.g. the
        indirect VPLs and the light samples of the direct term in one set."""
        return VplSet(self.pos[first:first + count], self.nrm[first:first + count],
                      self.flux[first:first + count], self.format)


# ---- the C entry points ----------------------------------------------------------------
def vpl_create(device: int = 0) -> C.c_void_p:
    h = C.c_void_p()
    rc = load().vpl_create(C.byref(h), int(device))
    _check(None, rc, "vpl_create")
    return h


def vpl_destroy(ctx) -> None:
    load().vpl_destroy(ctx)


def vpl_last_error(ctx) -> str:
    return (load().vpl_last_error(ctx) or b"").decode()


def vpl_scene_upload(ctx, verts, tris, albedo, light: W.Light, stream=None) -> int:
    sid = C.c_uint64()
    lt = make_light(light)
    rc = load().vpl_scene_upload(ctx, _ptr(verts), int(verts.shape[0]), _ptr(tris), int(tris.shape[0]),
                                 _ptr(albedo), C.byref(lt), _stream(stream), C.byref(sid))
    _check(ctx, rc, "vpl_scene_upload")
    return int(sid.value)


def vpl_scene_release(ctx, scene: int) -> None:
    _check(ctx, load().vpl_scene_release(ctx, scene), "vpl_scene_release")


def vpl_scene_query(ctx, scene: int) -> dict:
    info = vpl_scene_info()
    _check(ctx, load().vpl_scene_query(ctx, scene, C.byref(info)), "vpl_scene_query")
    return dict(n_tris=info.n_tris, n_nodes=info.n_nodes, depth=info.depth,
                device_bytes=info.device_bytes, bounds_lo=list(info.bounds_lo),
                bounds_hi=list(info.bounds_hi))


def vpl_gbuffer_build(ctx, scene: int, camera: W.Camera, gbuf: GBuffer, stream=None) -> None:
    cam, gb = make_camera(camera), gbuf.struct()
    _check(ctx, load().vpl_gbuffer_build(ctx, scene, C.byref(cam), C.byref(gb), _stream(stream)),
           "vpl_gbuffer_build")


def vpl_generate_rs(ctx, scene: int, camera: W.Camera, gen: W.GenParams, pilot: int, d2_min: float,
                    ray_eps: float, vpls: VplSet, stream=None) -> None:
    cam, g, vs = make_camera(camera), make_gen(gen), vpls.struct()
    _check(ctx, load().vpl_generate_rs(ctx, scene, C.byref(cam), C.byref(g), int(pilot), float(d2_min),
                                       float(ray_eps), C.byref(vs), _stream(stream)), "vpl_generate_rs")


def vpl_light_vpls(ctx, scene: int, n: int, seed: int, vpls: VplSet, stream=None) -> None:
    vs = vpls.struct()
    _check(ctx, load().vpl_light_vpls(ctx, scene, int(n), C.c_uint64(seed), C.byref(vs), _stream(stream)),
           "vpl_light_vpls")


def vpl_generate(ctx, scene: int, camera: W.Camera, gen: W.GenParams, vpls: VplSet, stream=None) -> None:
    cam, g, vs = make_camera(camera), make_gen(gen), vpls.struct()
    _check(ctx, load().vpl_generate(ctx, scene, C.byref(cam), C.byref(g), C.byref(vs), _stream(stream)),
           "vpl_generate")


def vpl_generate_info(ctx) -> dict:
    info = vpl_gen_info()
    _check(ctx, load().vpl_generate_info(ctx, C.byref(info)), "vpl_generate_info")
    return dict(n_close=info.n_close, shift_s=info.shift_s, f_total=int(info.f_total),
                paths=info.paths, m_far_kept=info.m_far_kept, status=info.status)


def vpl_gather(ctx, scene: int, gbuf: GBuffer, vpls: VplSet, params: W.GatherParams, out,
               stream=None) -> None:
    gb, vs, p = gbuf.struct(), vpls.struct(), make_gather(params)
    _check(ctx, load().vpl_gather(ctx, scene, C.byref(gb), C.byref(vs), C.byref(p), _ptr(out),
                                  _stream(stream)), "vpl_gather")


def vpl_gather_noalloc(ctx, scene: int, gbuf: GBuffer, vpls: VplSet, params: W.GatherParams, out,
                       stream=None) -> None:
    """vpl_gather without any device allocation (its scratch is static device
    memory shared by all calls; see include/vpl.h)."""
    gb, vs, p = gbuf.struct(), vpls.struct(), make_gather(params)
    _check(ctx, load().vpl_gather_noalloc(ctx, scene, C.byref(gb), C.byref(vs), C.byref(p), _ptr(out),
                                          _stream(stream)), "vpl_gather_noalloc")


def vpl_batch_create(ctx, gbufs, vsets, outs, tile_w: int = 0) -> int:
    n = len(gbufs)
    gb = (vpl_gbuffer * n)(*[g.struct() for g in gbufs])
    vs = (vpl_vpl_set * n)(*[v.struct() for v in vsets])
    op = (C.c_void_p * n)(*[_ptr(o) for o in outs])
    bid = C.c_uint64()
    _check(ctx, load().vpl_batch_create(ctx, n, gb, vs, op, int(tile_w), C.byref(bid)), "vpl_batch_create")
    return int(bid.value)


def vpl_gather_views(ctx, scene: int, gbufs, vsets, outs, params: W.GatherParams, stream=None) -> None:
    n = len(gbufs)
    gb = (vpl_gbuffer * n)(*[g.struct() for g in gbufs])
    vs = (vpl_vpl_set * n)(*[v.struct() for v in vsets])
    op = (C.c_void_p * n)(*[_ptr(o) for o in outs])
    p = make_gather(params)
    _check(ctx, load().vpl_gather_views(ctx, scene, n, gb, vs, op, C.byref(p), _stream(stream)),
           "vpl_gather_views")


def vpl_batch_destroy(ctx, batch: int) -> None:
    _check(ctx, load().vpl_batch_destroy(ctx, batch), "vpl_batch_destroy")


def vpl_gather_batch(ctx, scene: int, batch: int, params: W.GatherParams, stream=None) -> None:
    p = make_gather(params)
    _check(ctx, load().vpl_gather_batch(ctx, scene, batch, C.byref(p), _stream(stream)), "vpl_gather_batch")


def vpl_render(ctx, scene: int, camera: W.Camera, gen: W.GenParams, params: W.GatherParams, out,
               stream=None) -> None:
    cam, g, p = make_camera(camera), make_gen(gen), make_gather(params)
    _check(ctx, load().vpl_render(ctx, scene, C.byref(cam), C.byref(g), C.byref(p), _ptr(out),
                                  _stream(stream)), "vpl_render")


def vpl_sync(ctx, stream=None, check: bool = True) -> int:
    rc = load().vpl_sync(ctx, _stream(stream))
    if check:
        _check(ctx, rc, "vpl_sync")
    return rc


def vpl_debug_philox(ctx, ctr, key, out, stream=None) -> None:
    n = int(ctr.shape[0])
    _check(ctx, load().vpl_debug_philox(ctx, _ptr(ctr), _ptr(key), n, _ptr(out), _stream(stream)),
           "vpl_debug_philox")


def vpl_debug_rays(ctx, scene: int, mode: int, brute: int, a, b, out_tri, out_t=None, stream=None) -> None:
    n = int(a.shape[0])
    _check(ctx, load().vpl_debug_rays(ctx, scene, mode, brute, _ptr(a), _ptr(b), n, _ptr(out_tri),
                                      _ptr(out_t), _stream(stream)), "vpl_debug_rays")


def vpl_debug_visibility(ctx, scene: int, gbuf: GBuffer, vpls: VplSet, params: W.GatherParams, pixels,
                         vis, stream=None) -> None:
    gb, vs, p = gbuf.struct(), vpls.struct(), make_gather(params)
    _check(ctx, load().vpl_debug_visibility(ctx, scene, C.byref(gb), C.byref(vs), C.byref(p), _ptr(pixels),
                                            int(pixels.shape[0]), _ptr(vis), _stream(stream)),
           "vpl_debug_visibility")


def vpl_set_timing(ctx, on: bool) -> None:
    _check(ctx, load().vpl_set_timing(ctx, 1 if on else 0), "vpl_set_timing")


def vpl_stage_times(ctx) -> list:
    buf = (C.c_float * 4)()
    _check(ctx, load().vpl_stage_times(ctx, buf, 4), "vpl_stage_times")
    return [float(v) for v in buf]


def vpl_launch_count(ctx) -> int:
    return int(load().vpl_launch_count(ctx))


def vpl_pool_stats(ctx, reset_high: bool = False) -> dict:
    out = (C.c_uint64 * 3)()
    _check(ctx, load().vpl_pool_stats(ctx, 1 if reset_high else 0, out), "vpl_pool_stats")
    return dict(used=int(out[0]), high=int(out[1]), reserved=int(out[2]))


def vpl_gather_counters(ctx, scene: int, gbuf: GBuffer, vpls: VplSet, params: W.GatherParams,
                        stream=None) -> list:
    gb, vs, p = gbuf.struct(), vpls.struct(), make_gather(params)
    out = (C.c_uint64 * 6)()
    _check(ctx, load().vpl_gather_counters(ctx, scene, C.byref(gb), C.byref(vs), C.byref(p), out,
                                           _stream(stream)), "vpl_gather_counters")
    return [int(v) for v in out]


# ---- small conveniences over the entry points --------------------------------------------
class Context:
    """Owns a vpl_ctx; scenes uploaded through it are released with it."""

    def __init__(self, device: int = 0):
        self.h = vpl_create(device)
        self.device = device

    def close(self):
        if getattr(self, "h", None):
            vpl_destroy(self.h)
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def upload(self, scene: W.Scene, device: str = "cuda", stream=None) -> int:
        """Uploads from device copies of the scene arrays."""
        import torch
        v = torch.as_tensor(scene.verts, device=device).contiguous()
        t = torch.as_tensor(scene.tris, device=device).contiguous()
        a = torch.as_tensor(scene.albedo, device=device).contiguous()
        sid = vpl_scene_upload(self.h, v, t, a, scene.light, stream)
        vpl_sync(self.h, stream)
        return sid
