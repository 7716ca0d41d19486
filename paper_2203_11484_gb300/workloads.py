"""Seeded synthetic workloads for the hybrid close-range VPL renderer.

This module only builds inputs: triangle soups, albedos, a light, cameras and
parameter records.  It holds none of the method's arithmetic (no close-range
test, no Morton order, no area sampling, no shading), so both the CUDA path and
the FP64 oracle can consume the same inputs without sharing method code.

The paper's own scenes (a desk, a stone carving with a tea set and a display
cabinet, Sec. 3.1) are not available; the scenes below stand in for them: closed
or half-open rooms with dense, mutually reflecting diffuse geometry seen by a
close-up camera.  All arrays are float32 / int32, triangles are wound
counter-clockwise when seen from their front side (front normal = (b-a)x(c-a)).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field, replace
from typing import List, Optional, Tuple

import numpy as np

F32 = np.float32

# Light types (the paper's experiments use point lights, Sec. 3.1; the
# benchmark scenes use a one-sided square area light).
LIGHT_AREA = 0
LIGHT_POINT = 1

# Gather precision modes.
PREC_FP32 = 0
PREC_FP16_KAHAN = 1
PREC_FP16_PLAIN = 2

# Gather visibility modes.
VIS_BVH = 0
VIS_BRUTE = 1
VIS_NONE = 2


@dataclass
class Light:
    center: Tuple[float, float, float]
    normal: Tuple[float, float, float]
    edge_u: Tuple[float, float, float]
    edge_v: Tuple[float, float, float]
    power: Tuple[float, float, float] = (1.0, 1.0, 1.0)
    type: int = LIGHT_AREA


@dataclass
class Camera:
    eye: Tuple[float, float, float]
    forward: Tuple[float, float, float]
    up: Tuple[float, float, float]
    vfov_deg: float
    width: int
    height: int


@dataclass
class GenParams:
    d_close: float
    m_close: int
    m_far: int
    max_bounces: int = 3
    light_samples: int = 1
    seed: int = 0
    ir_max_paths: int = 0        # 0 -> default 16*m_far + 4096
    ray_eps: float = 1e-5
    close_rule: int = 0          # 0 centroid, 1 centroid or any vertex in view and range
    patch_rule: int = 0          # 0 a point per stratum, 1 set sum when a stratum spans several faces

    def resolved_max_paths(self) -> int:
        return self.ir_max_paths if self.ir_max_paths > 0 else 16 * self.m_far + 4096


@dataclass
class GatherParams:
    d2_min: float
    ray_eps: float
    precision: int = PREC_FP32
    visibility: int = VIS_BVH
    tile_w: int = 0           # warp pixel tile width (0 = 8): speed only
    blocks_per_sm: int = 0    # persistent grid cap (0 = occupancy limit): speed only
    vpl_tile: int = 0         # VPLs staged per warp at a time (0 = 64): speed only
    walk: int = 0             # 0: beam walk for narrow shadow packets, 1: per-lane walk only: speed only
    tile_order: int = 0       # 0 auto, 1 scan order, 2 costliest tiles first (sampled): speed only


@dataclass
class Scene:
    verts: np.ndarray      # float32 [V, 3]
    tris: np.ndarray       # int32   [T, 3]
    albedo: np.ndarray     # float32 [T, 3]
    light: Light

    @property
    def n_tris(self) -> int:
        return int(self.tris.shape[0])

    def diag(self) -> float:
        lo = self.verts.min(axis=0).astype(np.float64)
        hi = self.verts.max(axis=0).astype(np.float64)
        return float(np.linalg.norm(hi - lo))


@dataclass
class View:
    camera: Camera
    gen: GenParams
    gather: GatherParams


@dataclass
class Workload:
    name: str
    scene: Scene
    views: List[View]
    crop: Optional[Tuple[int, int, int, int]] = None   # x0, y0, w, h
    note: str = ""


def split_budget(m_total: int, alpha: float) -> Tuple[int, int]:
    """VPL budget split: m_close = floor(alpha*M + 0.5), m_far = M - m_close."""
    mc = int(math.floor(alpha * m_total + 0.5))
    return mc, m_total - mc


# ----------------------------------------------------------------------------
# geometry builders (triangle soups, CCW front)
# ----------------------------------------------------------------------------
class _Soup:
    def __init__(self):
        self.v: List[np.ndarray] = []
        self.t: List[np.ndarray] = []
        self.a: List[np.ndarray] = []
        self.nv = 0

    def add(self, verts: np.ndarray, tris: np.ndarray, albedo_rgb):
        verts = np.asarray(verts, dtype=np.float64)
        tris = np.asarray(tris, dtype=np.int64)
        self.v.append(verts)
        self.t.append(tris + self.nv)
        self.a.append(np.broadcast_to(np.asarray(albedo_rgb, dtype=np.float64),
                                      (tris.shape[0], 3)))
        self.nv += verts.shape[0]

    def quad_grid(self, origin, u, v, nu: int, nv: int, albedo_fn):
        """Quad spanned by edge vectors u, v (front normal along u x v),
        tessellated into nu x nv sub-quads of two triangles each.  albedo_fn()
        is called once per sub-quad."""
        o = np.asarray(origin, np.float64)
        u = np.asarray(u, np.float64)
        v = np.asarray(v, np.float64)
        for i in range(nu):
            for j in range(nv):
                p00 = o + u * (i / nu) + v * (j / nv)
                p10 = o + u * ((i + 1) / nu) + v * (j / nv)
                p11 = o + u * ((i + 1) / nu) + v * ((j + 1) / nv)
                p01 = o + u * (i / nu) + v * ((j + 1) / nv)
                self.add(np.stack([p00, p10, p11, p01]),
                         np.array([[0, 1, 2], [0, 2, 3]]), albedo_fn())

    def box(self, lo, hi, albedo_rgb):
        """Axis-aligned box, outward-facing."""
        lo = np.asarray(lo, np.float64)
        hi = np.asarray(hi, np.float64)
        dx, dy, dz = hi - lo
        X = np.array([dx, 0, 0])
        Y = np.array([0, dy, 0])
        Z = np.array([0, 0, dz])
        faces = [
            (lo, Z, Y),                                # -x
            (np.array([hi[0], lo[1], lo[2]]), Y, Z),   # +x
            (lo, X, Z),                                # -y
            (np.array([lo[0], hi[1], lo[2]]), Z, X),   # +y
            (lo, Y, X),                                # -z
            (np.array([lo[0], lo[1], hi[2]]), X, Y),   # +z
        ]
        vs, ts = [], []
        for f, (o, u, v) in enumerate(faces):
            vs += [o, o + u, o + u + v, o + v]
            b = 4 * f
            ts += [[b, b + 1, b + 2], [b, b + 2, b + 3]]
        self.add(np.stack(vs), np.array(ts), albedo_rgb)

    def uv_sphere(self, center, radius, stacks: int, slices: int, albedo_rgb):
        """UV sphere, outward-facing: 2*slices cap triangles plus
        2*slices*(stacks-2) band triangles."""
        c = np.asarray(center, np.float64)
        verts = [c + np.array([0, 0, radius])]
        for i in range(1, stacks):
            th = math.pi * i / stacks
            for j in range(slices):
                ph = 2 * math.pi * j / slices
                verts.append(c + radius * np.array([math.sin(th) * math.cos(ph),
                                                    math.sin(th) * math.sin(ph),
                                                    math.cos(th)]))
        verts.append(c + np.array([0, 0, -radius]))
        tris = []
        ring = lambda i, j: 1 + (i - 1) * slices + (j % slices)
        south = len(verts) - 1
        for j in range(slices):
            tris.append([0, ring(1, j), ring(1, j + 1)])
        for i in range(1, stacks - 1):
            for j in range(slices):
                a, b = ring(i, j), ring(i, j + 1)
                c2, d = ring(i + 1, j), ring(i + 1, j + 1)
                tris.append([a, c2, d])
                tris.append([a, d, b])
        for j in range(slices):
            tris.append([south, ring(stacks - 1, j + 1), ring(stacks - 1, j)])
        self.add(np.stack(verts), np.array(tris), albedo_rgb)

    def finish(self, light: Light) -> Scene:
        v = np.concatenate(self.v).astype(F32)
        t = np.concatenate(self.t).astype(np.int32)
        a = np.concatenate(self.a).astype(F32)
        return Scene(np.ascontiguousarray(v), np.ascontiguousarray(t),
                     np.ascontiguousarray(a), light)


def _room_zup(s: _Soup, size, nx, ny, nz, albedo_fn):
    """Closed room [0,sx]x[0,sy]x[0,sz], z up, all faces looking inward."""
    sx, sy, sz = size
    s.quad_grid((0, 0, 0), (sx, 0, 0), (0, sy, 0), nx, ny, albedo_fn)          # floor  +z
    s.quad_grid((0, 0, sz), (0, sy, 0), (sx, 0, 0), ny, nx, albedo_fn)         # ceiling -z
    s.quad_grid((0, 0, 0), (0, 0, sz), (sx, 0, 0), nz, nx, albedo_fn)          # y=0   +y
    s.quad_grid((0, sy, 0), (sx, 0, 0), (0, 0, sz), nx, nz, albedo_fn)         # y=sy  -y
    s.quad_grid((0, 0, 0), (0, sy, 0), (0, 0, sz), ny, nz, albedo_fn)          # x=0   +x
    s.quad_grid((sx, 0, 0), (0, 0, sz), (0, sy, 0), nz, ny, albedo_fn)         # x=sx  -x


# ----------------------------------------------------------------------------
# tiny Cornell-box-like scene: 64 triangles
# ----------------------------------------------------------------------------
# close-range distance threshold for the tiny scene: the value whose close set
# comes nearest to 15% of the total area (8 of 64 triangles, 13.2% of the
# area); chosen once by sweeping the threshold and checked by the tests.
CORNELL_D_CLOSE = 0.875


def cornell_scene(seed: int = 0) -> Scene:
    rng = np.random.default_rng(seed)
    alb = lambda: rng.uniform(0.2, 0.8, size=3)
    s = _Soup()
    # unit room, y up, front (z = 1) open; each wall 2 x 2 quads
    s.quad_grid((0, 0, 0), (0, 0, 1), (1, 0, 0), 2, 2, alb)   # floor   +y
    s.quad_grid((0, 1, 0), (1, 0, 0), (0, 0, 1), 2, 2, alb)   # ceiling -y
    s.quad_grid((0, 0, 0), (1, 0, 0), (0, 1, 0), 2, 2, alb)   # back    +z
    s.quad_grid((0, 0, 0), (0, 1, 0), (0, 0, 1), 2, 2, alb)   # left    +x
    s.quad_grid((1, 0, 0), (0, 0, 1), (0, 1, 0), 2, 2, alb)   # right   -x
    # two axis-aligned boxes: one albedo per face (6 quads each)
    for lo, hi in (((0.55, 0.0, 0.10), (0.85, 0.6, 0.40)),     # tall box
                   ((0.15, 0.0, 0.35), (0.45, 0.3, 0.65))):    # short box
        lo = np.array(lo)
        hi = np.array(hi)
        d = hi - lo
        X, Y, Z = np.array([d[0], 0, 0]), np.array([0, d[1], 0]), np.array([0, 0, d[2]])
        for o, u, v in ((lo, Z, Y), (np.array([hi[0], lo[1], lo[2]]), Y, Z),
                        (lo, X, Z), (np.array([lo[0], hi[1], lo[2]]), Z, X),
                        (lo, Y, X), (np.array([lo[0], lo[1], hi[2]]), X, Y)):
            s.quad_grid(o, u, v, 1, 1, alb)
    light = Light(center=(0.5, 1.0 - 1e-3, 0.5), normal=(0.0, -1.0, 0.0),
                  edge_u=(0.2, 0.0, 0.0), edge_v=(0.0, 0.0, 0.2),
                  power=(1.0, 1.0, 1.0), type=LIGHT_AREA)
    return s.finish(light)


def cornell_workload(width: int = 128, height: int = 128, visibility: int = VIS_BRUTE,
                     seed: int = 0) -> Workload:
    scene = cornell_scene(seed)
    # eye 0.5 units in front of the tall box's front face centre (0.7, 0.3, 0.4)
    cam = Camera(eye=(0.7, 0.3, 0.9), forward=(0.0, 0.0, -1.0), up=(0.0, 1.0, 0.0),
                 vfov_deg=60.0, width=width, height=height)
    L = scene.diag()
    eps = float(F32(1e-5 * L))
    gen = GenParams(d_close=CORNELL_D_CLOSE, m_close=192, m_far=64, max_bounces=3,
                    light_samples=1, seed=seed, ray_eps=eps)
    gat = GatherParams(d2_min=float(F32((1e-2 * L) ** 2)), ray_eps=eps,
                       precision=PREC_FP32, visibility=visibility)
    return Workload("cornell-64tri-128x128-256vpl", scene, [View(cam, gen, gat)],
                    note="tiny Cornell-box-like room, brute-force visibility")


# ----------------------------------------------------------------------------
# procedural rooms with random boxes and tessellated spheres
# ----------------------------------------------------------------------------
@dataclass
class RoomRecipe:
    size: Tuple[float, float, float]
    room_quads: Tuple[int, int, int]
    n_boxes: int
    box_scale: float
    spheres: List[Tuple[Tuple[float, float, float], float]]  # (centre, radius)
    sphere_res: Tuple[int, int]
    light_size: float
    seed: int


def room_scene(r: RoomRecipe):
    """Returns (scene, box_lo, box_hi) -- the box extents are kept so that
    camera placement can avoid starting inside a box."""
    rng = np.random.default_rng(r.seed)
    alb = lambda: rng.uniform(0.1, 0.9, size=3)
    s = _Soup()
    sx, sy, sz = r.size
    _room_zup(s, r.size, *r.room_quads, albedo_fn=alb)
    sizes = r.box_scale * rng.lognormal(0.0, 0.5, size=(r.n_boxes, 3))
    sizes[:, 2] = np.minimum(sizes[:, 2], 0.8 * sz)
    ctr = rng.uniform((1.0, 1.0), (sx - 1.0, sy - 1.0), size=(r.n_boxes, 2))
    lo = np.zeros((r.n_boxes, 3))
    hi = np.zeros((r.n_boxes, 3))
    lo[:, :2] = np.clip(ctr - sizes[:, :2] / 2, 0.0, None)
    hi[:, :2] = np.minimum(ctr + sizes[:, :2] / 2, (sx, sy))
    hi[:, 2] = sizes[:, 2]
    for b in range(r.n_boxes):
        s.box(lo[b], hi[b], alb())
    for c, rad in r.spheres:
        s.uv_sphere(c, rad, r.sphere_res[0], r.sphere_res[1], alb())
    h = r.light_size
    light = Light(center=(sx / 2, sy / 2, sz - 1e-3), normal=(0.0, 0.0, -1.0),
                  edge_u=(h, 0.0, 0.0), edge_v=(0.0, h, 0.0),
                  power=(1.0, 1.0, 1.0), type=LIGHT_AREA)
    return s.finish(light), lo, hi


def _free_eye(rng, lo, hi, centre_xy, spread, z_range, clearance=0.3, tries=10000):
    for _ in range(tries):
        xy = np.asarray(centre_xy) + rng.uniform(-spread, spread, size=2)
        z = rng.uniform(*z_range)
        e = np.array([xy[0], xy[1], z])
        inside = np.all((e >= lo - clearance) & (e <= hi + clearance), axis=1)
        if not inside.any():
            return e
    raise RuntimeError("no free camera position found")


def close_up_camera(rng, lo, hi, centre_xy, spread, z_range, dist_range,
                    width, height, vfov=60.0) -> Camera:
    """Eye outside every box, looking at the centre of a box whose centre
    lies dist_range away."""
    for _ in range(1000):
        e = _free_eye(rng, lo, hi, centre_xy, spread, z_range)
        c = (lo + hi) / 2
        d = np.linalg.norm(c - e, axis=1)
        cand = np.nonzero((d >= dist_range[0]) & (d <= dist_range[1]))[0]
        if cand.size:
            t = c[rng.choice(cand)]
            f = t - e
            return Camera(eye=tuple(float(F32(x)) for x in e),
                          forward=tuple(float(F32(x)) for x in f),
                          up=(0.0, 0.0, 1.0), vfov_deg=vfov, width=width, height=height)
    raise RuntimeError("no close-up target found")


ROOM200K = RoomRecipe(size=(160.0, 160.0, 12.0), room_quads=(80, 80, 6), n_boxes=10913,
                      box_scale=1.0,
                      spheres=[((76.0, 86.0, 2.0), 2.0), ((86.0, 77.0, 2.0), 2.0)],
                      sphere_res=(100, 100), light_size=4.0, seed=1)

ROOM1M = RoomRecipe(size=(100.0, 100.0, 10.0), room_quads=(50, 50, 5), n_boxes=40000,
                    box_scale=0.35, spheres=[], sphere_res=(26, 40), light_size=4.0, seed=4)

# close-range distance thresholds of the procedural rooms (scene units)
ROOM_D_CLOSE = 6.0
ROOM_D2_MIN = 0.05 ** 2
ROOM_RAY_EPS = 1e-3

_scene_cache = {}


def room200k_scene():
    if "200k" not in _scene_cache:
        _scene_cache["200k"] = room_scene(ROOM200K)
    return _scene_cache["200k"]


def room1m_scene():
    if "1m" not in _scene_cache:
        rng = np.random.default_rng(ROOM1M.seed + 1000)
        sx, sy, _ = ROOM1M.size
        sph = [((float(x), float(y), float(r)), float(r)) for x, y, r in
               zip(rng.uniform(2, sx - 2, 260), rng.uniform(2, sy - 2, 260),
                   rng.uniform(0.2, 0.8, 260))]
        _scene_cache["1m"] = room_scene(replace(ROOM1M, spheres=sph))
    return _scene_cache["1m"]


def room200k_workload(width=1024, height=1024, m_total=4096, alpha=0.75,
                      visibility=VIS_BVH, precision=PREC_FP32, seed=1) -> Workload:
    scene, lo, hi = room200k_scene()
    rng = np.random.default_rng(seed)
    cam = close_up_camera(rng, lo, hi, (80.0, 80.0), 6.0, (1.5, 1.5), (3.0, 5.0),
                          width, height)
    mc, mf = split_budget(m_total, alpha)
    gen = GenParams(d_close=ROOM_D_CLOSE, m_close=mc, m_far=mf, max_bounces=3,
                    light_samples=1, seed=seed, ray_eps=ROOM_RAY_EPS)
    gat = GatherParams(d2_min=ROOM_D2_MIN, ray_eps=ROOM_RAY_EPS, precision=precision,
                       visibility=visibility)
    return Workload(f"room-200k-{width}x{height}-{m_total}vpl", scene, [View(cam, gen, gat)],
                    note="procedural room, 200k triangles, BVH visibility")


def room1m_workload(width=1920, height=1080, m_total=32768, alpha=0.8,
                    precision=PREC_FP32, seed=4) -> Workload:
    scene, lo, hi = room1m_scene()
    rng = np.random.default_rng(seed)
    cam = close_up_camera(rng, lo, hi, (50.0, 50.0), 6.0, (1.0, 1.0), (2.0, 4.0),
                          width, height)
    mc, mf = split_budget(m_total, alpha)
    gen = GenParams(d_close=ROOM_D_CLOSE * 0.5, m_close=mc, m_far=mf, max_bounces=3,
                    light_samples=1, seed=seed, ray_eps=ROOM_RAY_EPS)
    gat = GatherParams(d2_min=ROOM_D2_MIN, ray_eps=ROOM_RAY_EPS, precision=precision,
                       visibility=VIS_BVH)
    return Workload(f"clutter-1m-{width}x{height}-{m_total}vpl", scene, [View(cam, gen, gat)],
                    crop=(832, 468, 256, 144),
                    note="dense clutter, ~1M triangles; oracle on a 256x144 crop")


def batch_views(n_views=64, seed=2, scene_fn=room200k_scene,
                resolutions=((256, 256), (512, 512), (768, 768), (1024, 1024)),
                m_range=(512, 8192), alpha=0.75, precision=PREC_FP32) -> Workload:
    """Many close-up views of one resident scene with uneven resolutions and
    VPL budgets (log-uniform)."""
    scene, lo, hi = scene_fn()
    rng = np.random.default_rng(seed)
    sx, sy, _ = (float(v) for v in scene.verts.max(axis=0))
    views = []
    for i in range(n_views):
        w, h = resolutions[rng.integers(len(resolutions))]
        cam = close_up_camera(rng, lo, hi, (sx / 2, sy / 2), 10.0, (0.5, 3.0), (2.0, 6.0),
                              int(w), int(h))
        m = int(round(math.exp(rng.uniform(math.log(m_range[0]), math.log(m_range[1])))))
        mc, mf = split_budget(m, alpha)
        gen = GenParams(d_close=ROOM_D_CLOSE, m_close=mc, m_far=mf, seed=seed * 1000 + i,
                        ray_eps=ROOM_RAY_EPS)
        gat = GatherParams(d2_min=ROOM_D2_MIN, ray_eps=ROOM_RAY_EPS, precision=precision)
        views.append(View(cam, gen, gat))
    return Workload(f"batch-{n_views}views-room-200k", scene, views,
                    note="uneven resolutions and VPL budgets, one resident scene")


def workload(name: str) -> Workload:
    if name in ("cornell", "tiny"):
        return cornell_workload()
    if name in ("room200k", "room"):
        return room200k_workload()
    if name in ("clutter1m", "large"):
        return room1m_workload()
    if name == "batch":
        return batch_views()
    raise KeyError(name)
