"""FP64 CPU oracle of the hybrid close-range VPL method (test infrastructure).

Only the test-suite, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The numerical work is plain C in
``vpl_oracle.c`` (FP64, no FMA contraction, OpenMP only across independent
pixels / rays); this module compiles it with gcc and marshals numpy arrays.
It imports nothing from the CUDA package.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading
from typing import Optional

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "vpl_oracle.c")
_LIBDIR = os.path.join(_HERE, "_lib")
_LIB = os.path.join(_LIBDIR, "liboracle.so")
_lock = threading.Lock()
_lib: Optional[C.CDLL] = None


def build(force: bool = False) -> str:
    """Compile liboracle.so next to the source (gcc, FP64, -ffp-contract=off)."""
    os.makedirs(_LIBDIR, exist_ok=True)
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    base = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fPIC",
            "-shared", _SRC, "-o", _LIB + ".tmp", "-lm"]
    try:
        subprocess.run(base[:1] + ["-fopenmp"] + base[1:], check=True,
                       capture_output=True, text=True)
    except subprocess.CalledProcessError:
        subprocess.run(base, check=True, capture_output=True, text=True)
    os.replace(_LIB + ".tmp", _LIB)
    return _LIB


class _Cam(C.Structure):
    _fields_ = [("eye", C.c_double * 3), ("fwd", C.c_double * 3), ("up", C.c_double * 3),
                ("vfov_deg", C.c_double), ("width", C.c_int32), ("height", C.c_int32)]


class _Light(C.Structure):
    _fields_ = [("center", C.c_double * 3), ("normal", C.c_double * 3),
                ("edge_u", C.c_double * 3), ("edge_v", C.c_double * 3),
                ("power", C.c_double * 3), ("type", C.c_int32)]


class _Gen(C.Structure):
    _fields_ = [("d_close", C.c_double), ("ray_eps", C.c_double), ("ir_max_paths", C.c_int64),
                ("seed", C.c_uint64), ("m_close", C.c_int32), ("m_far", C.c_int32),
                ("max_bounces", C.c_int32), ("light_samples", C.c_int32),
                ("vis_mode", C.c_int32), ("close_rule", C.c_int32), ("patch_rule", C.c_int32)]


class _Info(C.Structure):
    _fields_ = [("n_close", C.c_int64), ("shift_s", C.c_int64), ("f_total", C.c_uint64),
                ("paths", C.c_int64), ("m_far_kept", C.c_int64), ("a_rep", C.c_double),
                ("status", C.c_int64)]


_P = C.c_void_p
_D = C.POINTER(C.c_double)
_I64 = C.POINTER(C.c_int64)
_U8 = C.POINTER(C.c_uint8)


def lib() -> C.CDLL:
    global _lib
    with _lock:
        if _lib is None:
            L = C.CDLL(build())
            L.orc_philox4x64_10.argtypes = [C.POINTER(C.c_uint64), C.POINTER(C.c_uint64),
                                            C.POINTER(C.c_uint64)]
            L.orc_morton63.argtypes = [C.c_uint32] * 3
            L.orc_morton63.restype = C.c_uint64
            L.orc_scene_create.argtypes = [_P, C.c_int64, _P, C.c_int64, _P]
            L.orc_scene_create.restype = _P
            L.orc_scene_destroy.argtypes = [_P]
            L.orc_scene_info.argtypes = [_P, _D]
            L.orc_closest_batch.argtypes = [_P, C.c_int64, _D, _D, C.c_double, C.c_int32,
                                            _I64, _D]
            L.orc_occluded_batch.argtypes = [_P, C.c_int64, _D, _D, C.c_int32, _U8]
            L.orc_segment_margin.argtypes = [_P, _D, _D]
            L.orc_segment_margin.restype = C.c_double
            L.orc_classify.argtypes = [_P, C.POINTER(_Cam), C.POINTER(_Light), C.c_double, C.c_int32, _U8]
            L.orc_classify.restype = C.c_int64
            L.orc_generate.argtypes = [_P, C.POINTER(_Cam), C.POINTER(_Light), C.POINTER(_Gen),
                                       _D, _D, _D, _I64, _I64, C.POINTER(_Info)]
            L.orc_generate.restype = C.c_int64
            L.orc_gbuffer.argtypes = [_P, C.POINTER(_Cam), C.c_int64, _I64, C.c_int32,
                                      _D, _D, _D, _I64]
            L.orc_gather.argtypes = [_P, C.c_int64, _D, _D, _D, _I64, C.c_int64, _D, _D, _D,
                                     C.c_double, C.c_double, C.c_int32, _D]
            L.orc_pairs.argtypes = [_P, _D, _D, C.c_int64, _D, _D, C.c_double, C.c_double,
                                    C.c_int32, _U8, _D, C.POINTER(C.c_int8), _D]
            L.orc_generate_rs.argtypes = [_P, C.POINTER(_Cam), C.POINTER(_Light), C.POINTER(_Gen), C.c_int32,
                                          C.c_double, C.c_double, _D, _D, _D, _I64, _I64, C.POINTER(_Info)]
            L.orc_generate_rs.restype = C.c_int64
            L.orc_light_vpls.argtypes = [C.POINTER(_Light), C.c_int64, C.c_uint64, _D, _D, _D, _I64]
            L.orc_light_vpls.restype = C.c_int64
            L.orc_close_order.argtypes = [_P, _U8, _I64]
            L.orc_close_order.restype = C.c_int64
            L.orc_ir_path.argtypes = [_P, C.POINTER(_Light), C.POINTER(_Gen), C.c_int64, _D, _D, _I64, _D, _I64]
            L.orc_ir_path.restype = C.c_int64
            L.orc_flip_ratio.argtypes = [_P, _D, _D, C.c_double, C.c_double, C.c_int32]
            L.orc_flip_ratio.restype = C.c_double
            L.orc_num_threads.restype = C.c_int32
            L.orc_set_threads.argtypes = [C.c_int32]
            _lib = L
    return _lib


def _ptr(a: np.ndarray, ct):
    return a.ctypes.data_as(C.POINTER(ct))


def _f64(a, shape=None) -> np.ndarray:
    a = np.ascontiguousarray(np.asarray(a, dtype=np.float64))
    return a if shape is None else a.reshape(shape)


def set_threads(n: int) -> None:
    """Threads of the oracle's parallel loops from now on."""
    lib().orc_set_threads(int(n))


def num_threads() -> int:
    return int(lib().orc_num_threads())


def philox4x64_10(counter, key) -> np.ndarray:
    c = np.ascontiguousarray(np.asarray(counter, dtype=np.uint64))
    k = np.ascontiguousarray(np.asarray(key, dtype=np.uint64))
    out = np.zeros(4, dtype=np.uint64)
    lib().orc_philox4x64_10(_ptr(c, C.c_uint64), _ptr(k, C.c_uint64), _ptr(out, C.c_uint64))
    return out


def morton63(qx: int, qy: int, qz: int) -> int:
    return int(lib().orc_morton63(qx, qy, qz))


def cam_struct(cam) -> _Cam:
    c = _Cam()
    c.eye[:] = [float(np.float32(v)) for v in cam.eye]
    c.fwd[:] = [float(np.float32(v)) for v in cam.forward]
    c.up[:] = [float(np.float32(v)) for v in cam.up]
    c.vfov_deg = float(np.float32(cam.vfov_deg))
    c.width = int(cam.width)
    c.height = int(cam.height)
    return c


def light_struct(light) -> _Light:
    L = _Light()
    for name in ("center", "normal", "edge_u", "edge_v", "power"):
        getattr(L, name)[:] = [float(np.float32(v)) for v in getattr(light, name)]
    L.type = int(light.type)
    return L


def gen_struct(gen, vis_mode: int) -> _Gen:
    g = _Gen()
    g.d_close = float(gen.d_close)
    g.ray_eps = float(np.float32(gen.ray_eps))
    g.ir_max_paths = int(gen.resolved_max_paths())
    g.seed = int(gen.seed)
    g.m_close, g.m_far = int(gen.m_close), int(gen.m_far)
    g.max_bounces, g.light_samples = int(gen.max_bounces), int(gen.light_samples)
    g.vis_mode = int(vis_mode)
    g.close_rule = int(getattr(gen, "close_rule", 0))
    g.patch_rule = int(getattr(gen, "patch_rule", 0))
    return g


class OracleScene:
    """FP64 copy of a triangle scene plus the oracle's own FP64 BVH."""

    def __init__(self, scene):
        self.scene = scene
        v = np.ascontiguousarray(scene.verts, dtype=np.float32)
        t = np.ascontiguousarray(scene.tris, dtype=np.int32)
        a = np.ascontiguousarray(scene.albedo, dtype=np.float32)
        self._keep = (v, t, a)
        self.h = lib().orc_scene_create(v.ctypes.data, v.shape[0], t.ctypes.data, t.shape[0],
                                        a.ctypes.data)
        self.light = light_struct(scene.light)

    def close(self):
        if self.h:
            lib().orc_scene_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def info(self) -> dict:
        out = np.zeros(14)
        lib().orc_scene_info(self.h, _ptr(out, C.c_double))
        return dict(glo=out[0:3], ghi=out[3:6], vlo=out[6:9], vhi=out[9:12],
                    n_nodes=int(out[12]), n_tris=int(out[13]))

    def diag(self) -> float:
        i = self.info()
        return float(np.linalg.norm(i["vhi"] - i["vlo"]))

    # --- rays -----------------------------------------------------------
    def closest(self, o, d, tmin=0.0, vis_mode=0):
        o = _f64(o, (-1, 3))
        d = _f64(d, (-1, 3))
        n = o.shape[0]
        tri = np.zeros(n, np.int64)
        t = np.zeros(n)
        lib().orc_closest_batch(self.h, n, _ptr(o, C.c_double), _ptr(d, C.c_double), tmin,
                                vis_mode, _ptr(tri, C.c_int64), _ptr(t, C.c_double))
        return tri, t

    def occluded(self, p, q, vis_mode=0):
        p = _f64(p, (-1, 3))
        q = _f64(q, (-1, 3))
        out = np.zeros(p.shape[0], np.uint8)
        lib().orc_occluded_batch(self.h, p.shape[0], _ptr(p, C.c_double), _ptr(q, C.c_double),
                                 vis_mode, _ptr(out, C.c_uint8))
        return out.astype(bool)

    def segment_margin(self, p, q) -> float:
        p = _f64(p, (3,))
        q = _f64(q, (3,))
        return float(lib().orc_segment_margin(self.h, _ptr(p, C.c_double), _ptr(q, C.c_double)))

    def flip_ratio(self, p, q, c: float = 16.0, extra: float = 0.0, ends: int = 3) -> float:
        """orc_flip_ratio: <= 1 when FP32 rounding (c unit roundoffs of the
        coordinates, scaled by the incidence and the triangle's shape, plus
        `extra` of end-point error) can change segment p->q's answer; `ends`
        selects which end points' distances to a plane count (bit 0 p,
        bit 1 q)."""
        p = _f64(p, (3,))
        q = _f64(q, (3,))
        return float(lib().orc_flip_ratio(self.h, _ptr(p, C.c_double), _ptr(q, C.c_double), float(c),
                                          float(extra), int(ends)))

    # --- the method --------------------------------------------------------
    def classify(self, cam, d_close, rule: int = 0) -> np.ndarray:
        flags = np.zeros(self.scene.n_tris, np.uint8)
        c = cam_struct(cam)
        lib().orc_classify(self.h, C.byref(c), C.byref(self.light), float(d_close), int(rule),
                           _ptr(flags, C.c_uint8))
        return flags.astype(bool)

    def close_order(self, mask) -> np.ndarray:
        """Triangle indices of the faces with mask != 0 in the order the
        patch sampling walks them (orc_close_order)."""
        m = np.ascontiguousarray(np.asarray(mask, dtype=bool).astype(np.uint8))
        assert m.shape == (self.scene.n_tris,)
        out = np.zeros(max(int(m.sum()), 1), np.int64)
        n = lib().orc_close_order(self.h, _ptr(m, C.c_uint8), _ptr(out, C.c_int64))
        return out[:n]

    def ir_path(self, gen, p: int, vis_mode=0) -> dict:
        """The rays of instant-radiosity light path p (orc_ir_path): origin,
        direction, triangle hit (-1 miss), t and whether it was a front-face
        hit, one row per ray cast."""
        B = max(int(gen.max_bounces), 1)
        o, d, t = np.zeros((B, 3)), np.zeros((B, 3)), np.zeros(B)
        k, front = np.zeros(B, np.int64), np.zeros(B, np.int64)
        g = gen_struct(gen, vis_mode)
        n = lib().orc_ir_path(self.h, C.byref(self.light), C.byref(g), int(p), _ptr(o, C.c_double),
                              _ptr(d, C.c_double), _ptr(k, C.c_int64), _ptr(t, C.c_double),
                              _ptr(front, C.c_int64))
        return dict(o=o[:n], d=d[:n], k=k[:n], t=t[:n], front=front[:n].astype(bool))

    def generate(self, cam, gen, vis_mode=0) -> dict:
        M = int(gen.m_close) + int(gen.m_far)
        pos = np.zeros((max(M, 1), 3))
        nrm = np.zeros((max(M, 1), 3))
        flux = np.zeros((max(M, 1), 3))
        tri = np.zeros(max(M, 1), np.int64)
        tag = np.zeros(max(M, 1), np.int64)
        info = _Info()
        c = cam_struct(cam)
        g = gen_struct(gen, vis_mode)
        lib().orc_generate(self.h, C.byref(c), C.byref(self.light), C.byref(g),
                           _ptr(pos, C.c_double), _ptr(nrm, C.c_double), _ptr(flux, C.c_double),
                           _ptr(tri, C.c_int64), _ptr(tag, C.c_int64), C.byref(info))
        return dict(pos=pos[:M], nrm=nrm[:M], flux=flux[:M], tri=tri[:M], tag=tag[:M],
                    n_close=info.n_close, shift_s=info.shift_s, f_total=int(info.f_total),
                    paths=info.paths, m_far_kept=info.m_far_kept, a_rep=info.a_rep,
                    status=info.status)

    def generate_rs(self, cam, gen, pilot: int, d2_min: float, eps: float, vis_mode=0) -> dict:
        """Rejection-sampled instant radiosity (orc_generate_rs): gen.m_far
        VPLs; `cbar` is the mean candidate contribution on the pilot grid."""
        M = int(gen.m_far)
        pos = np.zeros((max(M, 1), 3))
        nrm = np.zeros((max(M, 1), 3))
        flux = np.zeros((max(M, 1), 3))
        tri = np.zeros(max(M, 1), np.int64)
        tag = np.zeros(max(M, 1), np.int64)
        info = _Info()
        c = cam_struct(cam)
        g = gen_struct(gen, vis_mode)
        lib().orc_generate_rs(self.h, C.byref(c), C.byref(self.light), C.byref(g), int(pilot), float(d2_min),
                              float(eps), _ptr(pos, C.c_double), _ptr(nrm, C.c_double), _ptr(flux, C.c_double),
                              _ptr(tri, C.c_int64), _ptr(tag, C.c_int64), C.byref(info))
        return dict(pos=pos[:M], nrm=nrm[:M], flux=flux[:M], tri=tri[:M], tag=tag[:M], paths=info.paths,
                    m_far_kept=info.m_far_kept, cbar=info.a_rep, status=info.status)

    def light_vpls(self, n: int, seed: int) -> dict:
        """Direct term of Eq. 1 as n light-sample VPLs (orc_light_vpls);
        None for a point light."""
        pos = np.zeros((max(n, 1), 3))
        nrm = np.zeros((max(n, 1), 3))
        flux = np.zeros((max(n, 1), 3))
        tag = np.zeros(max(n, 1), np.int64)
        r = lib().orc_light_vpls(C.byref(self.light), int(n), C.c_uint64(seed), _ptr(pos, C.c_double),
                                 _ptr(nrm, C.c_double), _ptr(flux, C.c_double), _ptr(tag, C.c_int64))
        if r < 0:
            return None
        return dict(pos=pos[:n], nrm=nrm[:n], flux=flux[:n], tag=tag[:n], tri=np.full(n, -1, np.int64))

    def gbuffer(self, cam, pixels=None, vis_mode=0) -> dict:
        if pixels is None:
            pixels = np.arange(int(cam.width) * int(cam.height), dtype=np.int64)
        pix = np.ascontiguousarray(np.asarray(pixels, dtype=np.int64))
        n = pix.shape[0]
        pos = np.zeros((n, 3))
        nrm = np.zeros((n, 3))
        rho = np.zeros((n, 3))
        tri = np.zeros(n, np.int64)
        c = cam_struct(cam)
        lib().orc_gbuffer(self.h, C.byref(c), n, _ptr(pix, C.c_int64), vis_mode,
                          _ptr(pos, C.c_double), _ptr(nrm, C.c_double), _ptr(rho, C.c_double),
                          _ptr(tri, C.c_int64))
        return dict(pos=pos, nrm=nrm, rho=rho, tri=tri, pixels=pix)

    def gather(self, gb: dict, vpl: dict, d2_min: float, eps: float, vis_mode=0) -> np.ndarray:
        y = _f64(gb["pos"], (-1, 3))
        ny = _f64(gb["nrm"], (-1, 3))
        rho = _f64(gb["rho"], (-1, 3))
        valid = np.ascontiguousarray(np.asarray(gb["tri"], dtype=np.int64))
        x = _f64(vpl["pos"], (-1, 3))
        nx = _f64(vpl["nrm"], (-1, 3))
        phi = _f64(vpl["flux"], (-1, 3))
        n, M = y.shape[0], x.shape[0]
        out = np.zeros((n, 3))
        lib().orc_gather(self.h, n, _ptr(y, C.c_double), _ptr(ny, C.c_double),
                         _ptr(rho, C.c_double), _ptr(valid, C.c_int64), M, _ptr(x, C.c_double),
                         _ptr(nx, C.c_double), _ptr(phi, C.c_double),
                         float(np.float32(d2_min)), float(np.float32(eps)),
                         vis_mode, _ptr(out, C.c_double))
        return out

    def pairs(self, y, ny, vpl: dict, d2_min, eps, vis_mode=0, want_margin=None):
        y = _f64(y, (3,))
        ny = _f64(ny, (3,))
        x = _f64(vpl["pos"], (-1, 3))
        nx = _f64(vpl["nrm"], (-1, 3))
        M = x.shape[0]
        term = np.zeros(M)
        vis = np.zeros(M, np.int8)
        margin = np.zeros(M)
        wm = None
        if want_margin is not None:
            wm = np.ascontiguousarray(np.asarray(want_margin, dtype=np.uint8))
        lib().orc_pairs(self.h, _ptr(y, C.c_double), _ptr(ny, C.c_double), M,
                        _ptr(x, C.c_double), _ptr(nx, C.c_double),
                        float(np.float32(d2_min)), float(np.float32(eps)),
                        vis_mode, None if wm is None else _ptr(wm, C.c_uint8),
                        _ptr(term, C.c_double), vis.ctypes.data_as(C.POINTER(C.c_int8)),
                        _ptr(margin, C.c_double))
        return term, vis, margin


def render(oscene: OracleScene, view, pixels=None, vis_mode=None) -> dict:
    """Whole pipeline (1)-(4) at the requested pixels: G-buffer, VPL
    generation and gather, all in FP64."""
    vm = view.gather.visibility if vis_mode is None else vis_mode
    gvm = 1 if vm == 1 else 0
    gb = oscene.gbuffer(view.camera, pixels, vis_mode=gvm)
    vpl = oscene.generate(view.camera, view.gen, vis_mode=gvm)
    img = oscene.gather(gb, vpl, view.gather.d2_min, float(np.float32(view.gather.ray_eps)),
                        vis_mode=vm)
    return dict(gbuffer=gb, vpl=vpl, image=img)
