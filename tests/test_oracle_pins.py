"""Pins of the FP64 oracle against facts fixed by the paper and by mathematics
(closed forms, invariants, library routines, brute force).  CPU only.

Each test names the passage of the paper (Jin et al., arXiv 2203.11484) it
pins and what independent fact it uses.
"""
import dataclasses
import math

import numpy as np
import pytest

from paper_2203_11484_gb300 import workloads as W

F32 = np.float32


def tri_scene(verts, tris, albedo, light=None):
    verts = np.asarray(verts, np.float32)
    tris = np.asarray(tris, np.int32)
    albedo = np.broadcast_to(np.asarray(albedo, np.float32), (tris.shape[0], 3)).copy()
    if light is None:
        light = W.Light(center=(0.0, 0.0, 10.0), normal=(0.0, 0.0, -1.0),
                        edge_u=(1.0, 0.0, 0.0), edge_v=(0.0, 1.0, 0.0), type=W.LIGHT_POINT)
    return W.Scene(verts, tris, albedo, light)


def plane_scene(half=10.0, z=0.0, up=True, albedo=0.5, light=None):
    """Square [-half, half]^2 at height z, facing +z (or -z)."""
    v = [(-half, -half, z), (half, -half, z), (half, half, z), (-half, half, z)]
    t = [(0, 1, 2), (0, 2, 3)] if up else [(0, 2, 1), (0, 3, 2)]
    return tri_scene(v, t, albedo, light)


def closed_box_scene(albedo=0.5, n=2):
    s = W._Soup()
    W._room_zup(s, (1.0, 1.0, 1.0), n, n, n, albedo_fn=lambda: (albedo,) * 3)
    light = W.Light(center=(0.5, 0.5, 1.0 - 1e-3), normal=(0.0, 0.0, -1.0),
                    edge_u=(0.2, 0.0, 0.0), edge_v=(0.0, 0.2, 0.0), type=W.LIGHT_AREA)
    return s.finish(light)


# ---------------------------------------------------------------------------
# Philox4x64-10: library routine (numpy ships the same generator)
# ---------------------------------------------------------------------------
def _numpy_philox_block(ctr, key):
    """numpy increments its 256-bit counter before producing a block, so the
    block for counter c is produced from state c - 1."""
    c = sum(int(ctr[i]) << (64 * i) for i in range(4))
    k = int(key[0]) | (int(key[1]) << 64)
    bg = np.random.Philox(key=k, counter=(c - 1) % (1 << 256))
    return bg.random_raw(4)


def test_philox_matches_numpy(orc):
    rng = np.random.default_rng(123)
    cases = [((0, 0, 0, 0), (0, 0)), ((1, 0, 0, 0), (0, 1)), ((5, 7, 0, 0), (99, 3)),
             ((2**64 - 1, 2**64 - 1, 2**64 - 1, 2**64 - 1), (2**64 - 1, 2**64 - 1))]
    for _ in range(300):
        cases.append((tuple(int(x) for x in rng.integers(0, 2**63, 4, dtype=np.uint64)),
                      tuple(int(x) for x in rng.integers(0, 2**63, 2, dtype=np.uint64))))
    for ctr, key in cases:
        got = orc.philox4x64_10(ctr, key)
        want = _numpy_philox_block(ctr, key)
        assert np.array_equal(got, want), (ctr, key)


# ---------------------------------------------------------------------------
# Morton order (Sec. 3, "Realization": spatial sort by Morton code)
# ---------------------------------------------------------------------------
def test_morton_bit_interleave(orc):
    assert orc.morton63(1, 0, 0) == 4
    assert orc.morton63(0, 1, 0) == 2
    assert orc.morton63(0, 0, 1) == 1
    m = 2**21 - 1
    assert orc.morton63(m, m, m) == 2**63 - 1
    rng = np.random.default_rng(7)
    for _ in range(500):
        q = [int(v) for v in rng.integers(0, 2**21, 3)]
        # independent restatement: read the bits of the code back out
        code = orc.morton63(*q)
        back = [0, 0, 0]
        for bit in range(63):
            if code >> bit & 1:
                axis = 2 - bit % 3
                back[axis] |= 1 << (bit // 3)
        assert back == q


def _morton_order_restated(verts, tris, mask, aabb="all", axes=(0, 1, 2), bits=21, ties=1):
    """The order of the close faces restated from Sec. 3 "Realization" (sort
    the faces by the Morton code of their position) and the reading that
    fixes its details: FP64 centroids ((a + b) + c) / 3 of the FP32
    vertices, normalised into the AABB of the centroids of ALL faces,
    floor(t 2^21) clamped to [0, 2^21 - 1] per axis, bit i of x, y, z at bit
    3i + 2, 3i + 1, 3i, and Python's sorted() on (code, index).  The keyword
    arguments plant the plausible slips the pin must catch (another box,
    swapped axes, another resolution, ties the other way)."""
    V = np.asarray(verts, np.float32).astype(np.float64)
    T = np.asarray(tris)
    g = ((V[T[:, 0]] + V[T[:, 1]]) + V[T[:, 2]]) / 3.0
    sel = np.nonzero(mask)[0]
    if aabb == "all":
        lo, hi = g.min(axis=0), g.max(axis=0)
    elif aabb == "close":
        lo, hi = g[sel].min(axis=0), g[sel].max(axis=0)
    else:  # the vertex box
        lo, hi = V[T.reshape(-1)].min(axis=0), V[T.reshape(-1)].max(axis=0)
    keys = []
    for t in sel:
        code = 0
        for slot, a in enumerate(axes):
            u = (g[t, a] - lo[a]) / (hi[a] - lo[a]) if hi[a] > lo[a] else 0.0
            q = min(max(math.floor(u * 2 ** bits), 0), 2 ** bits - 1)
            for bit in range(bits):
                code |= ((q >> bit) & 1) << (3 * bit + 2 - slot)
        keys.append((code, ties * int(t)))
    return [ties * t for _, t in sorted(keys)]


def _morton_pin_scene():
    """Faces whose centroids span very unequal extents (x 100, y 2, z 0.02,
    negative coordinates included), a few long faces that reach far beyond
    the centroid box (so the vertex box differs), exact duplicates (equal
    codes) and pairs closer than one quantisation cell (equal codes, unequal
    centroids); the faces that set the centroid box are left out of the
    mask, so the box of the masked centroids differs too."""
    rng = np.random.default_rng(21)
    cents = np.stack([rng.uniform(-50, 50, 400), rng.uniform(0, 2, 400), rng.uniform(-0.01, 0.01, 400)], 1)
    tv = []
    for c in cents:
        d1, d2 = rng.normal(0, 0.05, 3), rng.normal(0, 0.05, 3)
        tv.append([c + d1, c + d2, c - d1 - d2])
    for k in range(6):                      # long faces: vertices out to |x| = 300
        c = cents[k]
        tv.append([c + (250.0, 0, 0), c - (250.0, 0, 0), c + (0, 0.01, 0)])
    for k in range(20):                     # duplicates of faces 10..29
        tv.append([v.copy() for v in tv[10 + k]])
    for k in range(20):                     # 1e-9 of the box apart from faces 40..59
        tv.append([v + (1e-7, 0, 0) for v in tv[40 + k]])
    cell = 100.0 / 2 ** 21
    for k in range(20):                     # one 21-bit cell below faces 70..89 in x
        tv.append([v - (cell, 0, 0) for v in tv[70 + k]])
    verts = np.array([p for t in tv for p in t], np.float32)
    tris = np.arange(len(verts)).reshape(-1, 3)
    V = verts.astype(np.float64)
    g = ((V[tris[:, 0]] + V[tris[:, 1]]) + V[tris[:, 2]]) / 3.0
    mask = rng.random(len(tris)) < 0.7
    mask[10:30] = mask[400 + 6:400 + 26] = True
    mask[40:60] = mask[426:446] = True
    mask[70:90] = mask[446:466] = True
    for a in range(3):                      # the faces that set the centroid box
        mask[np.argmin(g[:, a])] = mask[np.argmax(g[:, a])] = False
    return tri_scene(verts, tris, 0.5), mask


def test_morton_close_order_restated(orc):
    """The order the patch sampling walks (orc_close_order) equals the
    restatement, and each planted slip gives another order, so the pin
    would see it."""
    sc, mask = _morton_pin_scene()
    o = orc.OracleScene(sc)
    got = o.close_order(mask).tolist()
    want = _morton_order_restated(sc.verts, sc.tris, mask)
    assert got == want
    assert len(got) == int(mask.sum())
    for slip in (dict(aabb="close"), dict(aabb="verts"), dict(axes=(2, 1, 0)), dict(axes=(1, 0, 2)),
                 dict(bits=20), dict(ties=-1)):
        assert _morton_order_restated(sc.verts, sc.tris, mask, **slip) != want, slip
    assert sorted(got) != got                # not the index order either
    # equal codes are ordered by index: a duplicate, and a copy less than one
    # cell away, directly follow their original; a copy one cell lower in x
    # comes first
    pos = {t: i for i, t in enumerate(got)}
    both = lambda a, b: a in pos and b in pos
    pairs = [(10 + k, 406 + k) for k in range(20)] + [(40 + k, 426 + k) for k in range(20)]
    assert sum(both(a, b) for a, b in pairs) >= 36
    for a, b in pairs:
        assert not both(a, b) or pos[b] == pos[a] + 1, (a, b)
    below = [(70 + k, 446 + k) for k in range(20) if both(70 + k, 446 + k)]
    assert len(below) >= 18 and sum(pos[b] < pos[a] for a, b in below) >= len(below) - 1


@pytest.mark.parametrize("which", ["cornell", "room"])
def test_patch_strata_follow_the_morton_order(orc, which):
    """orc_generate assigns strata along that order: the faces of consecutive
    patch VPLs are non-decreasing in the restated order, and with many VPLs
    every close face with a large enough area is reached."""
    wl = W.cornell_workload() if which == "cornell" else W.room200k_workload()
    v = wl.views[0]
    o = orc.OracleScene(wl.scene)
    close = o.classify(v.camera, v.gen.d_close)
    order = _morton_order_restated(wl.scene.verts, wl.scene.tris, close)
    assert o.close_order(close).tolist() == order
    K = 4000 if which == "cornell" else 20000
    gen = dataclasses.replace(v.gen, m_close=K, m_far=0)
    g = o.generate(v.camera, gen, vis_mode=1 if which == "cornell" else 0)
    rank = {t: i for i, t in enumerate(order)}
    r = np.array([rank[int(t)] for t in g["tri"]])
    assert (np.diff(r) >= 0).all()
    A = _areas(wl.scene)
    big = [t for t in order if A[t] * K > 2 * A[close].sum()]   # >= 2 strata wide: reached
    assert set(big) <= set(g["tri"].tolist())
    assert len(big) >= min(8, len(order))


# ---------------------------------------------------------------------------
# close/distant split (Sec. 3): one-sided, in the field of view, nearer than a
# threshold; patch sampling only on faces facing the light
# ---------------------------------------------------------------------------
def _cam(eye=(0, 0, 0), fwd=(0, 0, 1), up=(0, 1, 0), w=64, h=64, vfov=60.0):
    return W.Camera(eye=eye, forward=fwd, up=up, vfov_deg=vfov, width=w, height=h)


def test_classify_hand_cases(orc):
    light = W.Light(center=(0.0, 0.0, -1.0), normal=(0.0, 0.0, 1.0), edge_u=(0.1, 0, 0),
                    edge_v=(0, 0.1, 0), type=W.LIGHT_POINT)
    s = 0.1
    def facing_cam(cx, cy, cz):   # triangle facing -z (towards a camera at the origin)
        return [(cx - s, cy - s, cz), (cx, cy + s, cz), (cx + s, cy - s, cz)]
    tris_v = [
        facing_cam(0, 0, 1),          # 0 close
        facing_cam(0, 0, 10),         # 1 beyond the threshold
        facing_cam(5, 0, 1),          # 2 outside the horizontal field of view
        facing_cam(0, 5, 1),          # 3 outside the vertical field of view
        facing_cam(0, 0, -1),         # 4 behind the camera
        list(reversed(facing_cam(0, 0, 1.5))),  # 5 back face towards the camera
        facing_cam(0.4, 0.4, 1.0),    # 6 inside (corner of the frustum, tan 30deg = 0.577)
    ]
    verts = np.array([p for t in tris_v for p in t], np.float32)
    tris = np.arange(len(verts)).reshape(-1, 3)
    sc = tri_scene(verts, tris, 0.5, light)
    o = orc.OracleScene(sc)
    got = o.classify(_cam(), 3.0)
    assert got.tolist() == [True, False, False, False, False, False, True]
    # the light behind the faces: nothing faces it
    sc2 = tri_scene(verts, tris, 0.5, W.Light(center=(0.0, 0.0, 20.0), normal=(0, 0, -1),
                                             edge_u=(1, 0, 0), edge_v=(0, 1, 0),
                                             type=W.LIGHT_POINT))
    assert not orc.OracleScene(sc2).classify(_cam(), 3.0).any()
    # wider screen widens the horizontal field of view only
    wide = _cam(w=256, h=64)
    v2 = np.array(facing_cam(1.5, 0, 1), np.float32)
    sc3 = tri_scene(v2, [(0, 1, 2)], 0.5, light)
    assert orc.OracleScene(sc3).classify(wide, 3.0).tolist() == [True]
    assert orc.OracleScene(sc3).classify(_cam(), 3.0).tolist() == [False]


def test_classify_any_vertex_rule(orc):
    """Rule 1 also accepts a face whose centroid fails the view or distance
    test when one of its vertices passes it (camera at the origin looking
    down +z, vfov 60 deg: the view edge at z = 1 is |x| = tan 30 deg = 0.577)."""
    light = W.Light(center=(0.0, 0.0, -1.0), normal=(0.0, 0.0, 1.0), edge_u=(0.1, 0, 0),
                    edge_v=(0, 0.1, 0), type=W.LIGHT_POINT)
    def facing(a, b, c):          # front side towards the camera (normal -z)
        return [a, c, b]
    tris_v = [
        facing((0.5, 0, 1), (0.9, 0, 1), (0.9, 0.3, 1)),   # 0 centroid x 0.77 outside, vertex x 0.5 inside
        facing((0, 0, 2.9), (0.1, 0, 3.5), (0, 0.1, 3.5)),  # 1 centroid at z 3.3 > d_close 3, a vertex at 2.9
        facing((0, 0, 1), (0.1, 0, 1), (0, 0.1, 1)),        # 2 centroid inside: close under both rules
        facing((1.0, 0, 1), (1.2, 0, 1), (1.2, 0.2, 1)),    # 3 all outside: close under neither
        [(0.5, 0, 1), (0.9, 0, 1), (0.9, 0.3, 1)],           # 4 as 0 but its back towards the camera
    ]
    verts = np.array([p for t in tris_v for p in t], np.float32)
    tris = np.arange(len(verts)).reshape(-1, 3)
    o = orc.OracleScene(tri_scene(verts, tris, 0.5, light))
    assert o.classify(_cam(), 3.0, rule=0).tolist() == [False, False, True, False, False]
    assert o.classify(_cam(), 3.0, rule=1).tolist() == [True, True, True, False, False]
    # on a whole scene the any-vertex set contains the centroid set
    wl = W.cornell_workload()
    oc = orc.OracleScene(wl.scene)
    c0 = oc.classify(wl.views[0].camera, wl.views[0].gen.d_close, rule=0)
    c1 = oc.classify(wl.views[0].camera, wl.views[0].gen.d_close, rule=1)
    assert (c1 | c0).tolist() == c1.tolist() and c1.sum() > c0.sum()


def test_cornell_close_fraction(orc):
    wl = W.cornell_workload()
    o = orc.OracleScene(wl.scene)
    fl = o.classify(wl.views[0].camera, wl.views[0].gen.d_close)
    V = wl.scene.verts.astype(np.float64)
    T = wl.scene.tris
    A = 0.5 * np.linalg.norm(np.cross(V[T[:, 1]] - V[T[:, 0]], V[T[:, 2]] - V[T[:, 0]]), axis=1)
    frac = A[fl].sum() / A.sum()
    assert fl.sum() == 8 and 0.10 <= frac <= 0.20


# ---------------------------------------------------------------------------
# patch strata (Sec. 3, "Realization"): K equal-area strata over f, each VPL
# represents the same area; a big triangle gets several VPLs
# ---------------------------------------------------------------------------
def _areas(scene):
    V = scene.verts.astype(np.float64)
    T = scene.tris
    return 0.5 * np.linalg.norm(np.cross(V[T[:, 1]] - V[T[:, 0]], V[T[:, 2]] - V[T[:, 0]]), axis=1)


@pytest.mark.parametrize("m_close", [1, 7, 192, 1000])
def test_strata_counts_and_uniform_area(orc, m_close):
    wl = W.cornell_workload()
    v = wl.views[0]
    o = orc.OracleScene(wl.scene)
    gen = W.GenParams(**{**v.gen.__dict__, "m_close": m_close, "m_far": 0})
    g = o.generate(v.camera, gen, vis_mode=1)
    close = o.classify(v.camera, gen.d_close)
    A = _areas(wl.scene)
    S = g["shift_s"]
    q = np.array([int(np.rint(np.ldexp(a, S))) for a in A])   # numpy rint: half-even,
    # differs from llround only on exact .5 ties which cannot occur for these areas
    F = int(q[close].sum())
    assert g["f_total"] == F
    counts = np.bincount(g["tri"], minlength=len(A))
    # an interval of L strata (jittered: one uniform point per stratum) holds
    # at least floor(L) - 1 and at most ceil(L) + 1 of the points
    for t in np.nonzero(close)[0]:
        L = m_close * int(q[t]) / F
        assert max(0, math.floor(L) - 1) <= counts[t] <= math.ceil(L) + 1
    assert counts.sum() == m_close
    assert counts[~close].sum() == 0
    # every VPL represents the same area; together they cover the close area
    assert abs(g["a_rep"] * m_close - A[close].sum()) <= 1e-9 * A[close].sum()
    # the strata are contiguous in the sorted order: each triangle's VPLs form one run
    seen, prev = set(), None
    for t in g["tri"]:
        if t != prev:
            assert t not in seen
            seen.add(t)
            prev = t


def test_strata_expected_counts(orc):
    """Averaged over seeds, triangle t receives exactly K q_t / F VPLs."""
    wl = W.cornell_workload()
    v = wl.views[0]
    o = orc.OracleScene(wl.scene)
    K, n_seeds = 50, 400
    A = _areas(wl.scene)
    close = o.classify(v.camera, v.gen.d_close)
    tot = np.zeros(len(A))
    for seed in range(n_seeds):
        gen = W.GenParams(**{**v.gen.__dict__, "m_close": K, "m_far": 0, "seed": seed})
        g = o.generate(v.camera, gen, vis_mode=1)
        tot += np.bincount(g["tri"], minlength=len(A))
    want = K * A / A[close].sum() * close
    # per-seed variance of a count is at most 1/2 (two partial strata)
    assert np.all(np.abs(tot / n_seeds - want) <= 4 * math.sqrt(0.5 / n_seeds) + 1e-9)


def test_points_uniform_in_triangle(orc):
    """One close triangle, 100k strata: barycentrics valid, chi^2 over 16
    equal-area sub-triangles (uniform point in a triangle)."""
    v = [(-1.0, -1.0, 0.0), (1.0, -1.0, 0.0), (0.0, 1.0, 0.0)]
    sc = tri_scene(v, [(0, 1, 2)], 0.5)
    cam = _cam(eye=(0, 0, 3), fwd=(0, 0, -1), up=(0, 1, 0))
    o = orc.OracleScene(sc)
    K = 100_000
    gen = W.GenParams(d_close=10.0, m_close=K, m_far=0, seed=11)
    g = o.generate(cam, gen)
    assert g["status"] == 0 and (g["tri"] == 0).all()
    P = g["pos"]
    a, b, c = (np.array(x) for x in v)
    # barycentric coordinates
    m = np.stack([b - a, c - a], axis=1)[:2]
    uv = np.linalg.solve(m, (P[:, :2] - a[:2]).T).T
    assert (uv >= -1e-12).all() and (uv.sum(axis=1) <= 1 + 1e-12).all()
    assert np.abs(P[:, 2]).max() == 0.0
    # 16 sub-triangles of a 4x4 barycentric grid
    n = 4
    u, w = uv[:, 0] * n, uv[:, 1] * n
    iu, iw = np.floor(u).astype(int), np.floor(w).astype(int)
    upper = (u - iu) + (w - iw) > 1
    cell = (iu * n + iw) * 2 + upper
    hist = np.bincount(cell, minlength=2 * n * n)
    valid = [((i * n + j) * 2 + up) for i in range(n) for j in range(n) for up in (0, 1)
             if i + j + up <= n - 1]
    assert len(valid) == 16 and hist[valid].sum() == K
    exp = K / 16
    chi2 = ((hist[valid] - exp) ** 2 / exp).sum()
    assert chi2 < 37.7     # 15 dof, p = 0.001


# ---------------------------------------------------------------------------
# Eq. 2 (patch VPL value), point light: sum over patches = rho * P * Omega/(4 pi)
# ---------------------------------------------------------------------------
def _solid_angle(p, a, b, c):
    """Van Oosterom & Strackee (1983): solid angle of triangle abc seen from p."""
    A, B, C = a - p, b - p, c - p
    la, lb, lc = np.linalg.norm(A), np.linalg.norm(B), np.linalg.norm(C)
    num = abs(np.dot(A, np.cross(B, C)))
    den = la * lb * lc + np.dot(A, B) * lc + np.dot(A, C) * lb + np.dot(B, C) * la
    return 2.0 * math.atan2(num, den)


@pytest.mark.parametrize("K,tol", [(2000, 1.5e-2), (200000, 1.5e-3)])
def test_eq2_point_light_total_flux(orc, K, tol):
    light = W.Light(center=(0.3, -0.2, 2.0), normal=(0, 0, -1), edge_u=(1, 0, 0),
                    edge_v=(0, 1, 0), power=(1.0, 2.0, 0.5), type=W.LIGHT_POINT)
    rho = np.array([0.25, 0.5, 0.75])
    sc = plane_scene(half=1.5, albedo=rho, light=light)
    cam = _cam(eye=(0, 0, 4), fwd=(0, 0, -1), up=(0, 1, 0), vfov=80)
    o = orc.OracleScene(sc)
    g = o.generate(cam, W.GenParams(d_close=100.0, m_close=K, m_far=0, seed=3))
    assert g["status"] == 0 and g["n_close"] == 2
    V = sc.verts.astype(np.float64)
    p = np.array(light.center, np.float64)
    omega = sum(_solid_angle(p, *V[t]) for t in sc.tris)
    want = rho * np.array(light.power) * omega / (4 * math.pi)
    got = g["flux"].sum(axis=0)
    assert np.allclose(got, want, rtol=tol)     # about 6 sigma of the stratified estimate
    # each VPL: D cos(w)/(4 pi r^2) * rho * P with D the uniform represented area
    x = g["pos"]
    d = p - x
    r = np.linalg.norm(d, axis=1)
    each = g["a_rep"] * (d[:, 2] / r) / (4 * math.pi * r * r)
    assert np.allclose(g["flux"], each[:, None] * rho * np.array(light.power), rtol=1e-12)


# ---------------------------------------------------------------------------
# Eq. 2 with a Lambertian square light: per-VPL flux -> rho * D * E(x), with E
# Lambert's closed-form polygon-to-point irradiance
# ---------------------------------------------------------------------------
def _lambert_irradiance(x, n, poly, radiance):
    """E = (L/2) sum_i angle(u_i, u_i+1) * n . unit(u_i x u_i+1), polygon seen
    from x wound so that its emitting side faces x."""
    u = [(q - x) / np.linalg.norm(q - x) for q in poly]
    e = 0.0
    for i in range(len(u)):
        a, b = u[i], u[(i + 1) % len(u)]
        cr = np.cross(a, b)
        e += math.acos(np.clip(np.dot(a, b), -1, 1)) * np.dot(n, cr / np.linalg.norm(cr))
    return 0.5 * radiance * abs(e)


def test_eq2_area_light_matches_lambert(orc):
    eu, ev = np.array([0.4, 0.0, 0.0]), np.array([0.0, 0.4, 0.0])
    c = np.array([0.1, 0.2, 1.0])
    light = W.Light(center=tuple(c), normal=(0, 0, -1), edge_u=tuple(eu), edge_v=tuple(ev),
                    power=(2.0, 2.0, 2.0), type=W.LIGHT_AREA)
    sc = plane_scene(half=1.0, albedo=0.6, light=light)
    cam = _cam(eye=(0, 0, 4), fwd=(0, 0, -1), up=(0, 1, 0), vfov=80)
    o = orc.OracleScene(sc)
    S_L = 20000
    g = o.generate(cam, W.GenParams(d_close=100.0, m_close=8, m_far=0, light_samples=S_L,
                                    seed=5))
    poly = [c - eu / 2 - ev / 2, c + eu / 2 - ev / 2, c + eu / 2 + ev / 2, c - eu / 2 + ev / 2]
    L = 2.0 / (math.pi * 0.16)
    for k in range(8):
        E = _lambert_irradiance(g["pos"][k], np.array([0, 0, 1.0]), poly, L)
        want = 0.6 * g["a_rep"] * E
        assert abs(g["flux"][k, 0] - want) < 0.02 * want


# ---------------------------------------------------------------------------
# instant radiosity (Sec. 3, pipeline step (3)); flux = power x albedos / P
# ---------------------------------------------------------------------------
def test_ir_flux_exact_constant_albedo(orc):
    sc = closed_box_scene(albedo=0.5)
    cam = _cam(eye=(0.5, 0.5, 0.5), fwd=(1, 0, 0), up=(0, 0, 1))
    o = orc.OracleScene(sc)
    gen = W.GenParams(d_close=0.0, m_close=0, m_far=3001, max_bounces=3, seed=9, ray_eps=1e-6)
    g = o.generate(cam, gen)
    assert g["status"] == 0 and g["m_far_kept"] == 3001
    P = g["paths"]
    b = g["tag"] % 16
    p = g["tag"] // 16
    assert (np.diff(g["tag"]) > 0).all() and p.max() == P - 1
    want = 0.5 ** b / P
    assert np.array_equal(g["flux"][:, 0], want)
    # closed room, inward faces: no path is absorbed or escapes, so every
    # launched path leaves exactly max_bounces VPLs (the last one truncated)
    full = np.bincount(p, minlength=P)
    assert (full[:-1] == 3).all() and 1 <= full[-1] <= 3
    # first-bounce VPLs carry rho * power in total
    assert abs(g["flux"][b == 1, 0].sum() - 0.5) < 1e-12


def test_ir_rejects_close_hits(orc):
    wl = W.cornell_workload()
    v = wl.views[0]
    o = orc.OracleScene(wl.scene)
    g = o.generate(v.camera, v.gen, vis_mode=1)
    close = o.classify(v.camera, v.gen.d_close)
    M_c = v.gen.m_close
    assert g["status"] == 0
    assert close[g["tri"][:M_c]].all()
    assert not close[g["tri"][M_c:]].any()
    assert len(g["tri"]) == M_c + v.gen.m_far
    # far VPLs lie on their triangle's plane
    V = wl.scene.verts.astype(np.float64)
    T = wl.scene.tris[g["tri"][M_c:]]
    nrm = np.cross(V[T[:, 1]] - V[T[:, 0]], V[T[:, 2]] - V[T[:, 0]])
    nrm /= np.linalg.norm(nrm, axis=1, keepdims=True)
    dist = np.einsum("ij,ij->i", g["pos"][M_c:] - V[T[:, 0]], nrm)
    assert np.abs(dist).max() < 1e-12


def _first_bounce_dirs(orc, light, n_paths, seed):
    """First-bounce VPL positions of n_paths light paths in the closed unit
    box (every path hits a wall at its first bounce) and their directions
    from the light's centre."""
    sc = closed_box_scene(albedo=0.5)
    sc = dataclasses.replace(sc, light=light)
    o = orc.OracleScene(sc)
    cam = _cam(eye=(0.5, 0.5, 0.5), fwd=(1, 0, 0), up=(0, 0, 1))
    gen = W.GenParams(d_close=0.0, m_close=0, m_far=n_paths, max_bounces=1, seed=seed, ray_eps=1e-6)
    g = o.generate(cam, gen)
    assert g["status"] == 0 and g["paths"] == n_paths and (g["tag"] % 16 == 1).all()
    d = g["pos"] - np.asarray(light.center, np.float64)
    return g["pos"], d / np.linalg.norm(d, axis=1, keepdims=True)


def _view_factor_corner(X, Y):
    """View factor from a differential area to a parallel rectangle of sides
    X, Y (in units of the distance) with the area's normal through one
    corner (Howell's catalogue, configuration B-3)."""
    a, b = math.sqrt(1 + X * X), math.sqrt(1 + Y * Y)
    return (X / a * math.atan(Y / a) + Y / b * math.atan(X / b)) / (2 * math.pi)


def test_ir_emission_is_cosine_weighted(orc):
    """Light paths leave the square light in cosine-weighted directions
    (Lambertian emitter): with a light too small to matter, E[cos] = 2/3,
    E[cos^2] = 1/2, the azimuth is uniform, and the share of paths whose
    first hit is the floor is the view factor from the light's centre to the
    floor (closed form).  A uniform hemisphere gives E[cos] = 1/2."""
    n = 40000
    light = W.Light(center=(0.5, 0.5, 1.0 - 1e-3), normal=(0.0, 0.0, -1.0), edge_u=(1e-4, 0.0, 0.0),
                    edge_v=(0.0, 1e-4, 0.0), type=W.LIGHT_AREA)
    pos, d = _first_bounce_dirs(orc, light, n, seed=21)
    cos = -d[:, 2]
    se = 1.0 / math.sqrt(n)
    assert (cos > 0).all()
    assert abs(cos.mean() - 2 / 3) < 5 * math.sqrt(1 / 18) * se
    assert abs((cos ** 2).mean() - 0.5) < 5 * math.sqrt(1 / 12) * se
    for c in (d[:, 0], d[:, 1]):   # E[sin cos phi] = 0, E[sin^2 cos^2 phi] = 1/4
        assert abs(c.mean()) < 5 * 0.5 * se
        assert abs((c ** 2).mean() - 0.25) < 5 * 0.25 * se
    h = 1.0 - 1e-3
    f_floor = 4 * _view_factor_corner(0.5 / h, 0.5 / h)
    share = float((pos[:, 2] < 1e-9).mean())
    assert abs(share - f_floor) < 5 * math.sqrt(f_floor * (1 - f_floor)) * se


def test_ir_point_light_emits_uniformly_over_the_sphere(orc):
    """A point light (type 1, isotropic) at the centre of the closed unit
    cube: each face subtends 4 pi / 6, so each takes 1/6 of the first hits,
    and the directions have zero mean with E[d_k^2] = 1/3."""
    n = 36000
    light = W.Light(center=(0.5, 0.5, 0.5), normal=(0.0, 0.0, -1.0), edge_u=(0.0, 0.0, 0.0),
                    edge_v=(0.0, 0.0, 0.0), type=W.LIGHT_POINT)
    pos, d = _first_bounce_dirs(orc, light, n, seed=22)
    se = 1.0 / math.sqrt(n)
    faces = [pos[:, 0] < 1e-9, pos[:, 0] > 1 - 1e-9, pos[:, 1] < 1e-9, pos[:, 1] > 1 - 1e-9,
             pos[:, 2] < 1e-9, pos[:, 2] > 1 - 1e-9]
    assert sum(int(f.sum()) for f in faces) == n
    for f in faces:
        assert abs(f.mean() - 1 / 6) < 5 * math.sqrt(5 / 36) * se
    for k in range(3):
        assert abs(d[:, k].mean()) < 5 * math.sqrt(1 / 3) * se
        assert abs((d[:, k] ** 2).mean() - 1 / 3) < 5 * math.sqrt(4 / 45) * se


def test_ir_bounce_directions_are_cosine_weighted_about_the_hit_normal(orc):
    """Each bounce leaves its hit point in a cosine-weighted direction about
    the face's normal: between consecutive VPLs of one path in the closed
    box, E[cos] = 2/3 and E[cos^2] = 1/2 against the first VPL's normal, and
    the tangent components have zero mean (a frame that favours one tangent
    direction fails)."""
    sc = closed_box_scene(albedo=0.5)
    o = orc.OracleScene(sc)
    cam = _cam(eye=(0.5, 0.5, 0.5), fwd=(1, 0, 0), up=(0, 0, 1))
    n = 40000
    g = o.generate(cam, W.GenParams(d_close=0.0, m_close=0, m_far=2 * n, max_bounces=2, seed=23, ray_eps=1e-6))
    assert g["status"] == 0 and g["paths"] == n
    b = g["tag"] % 16
    first, second = np.flatnonzero(b == 1), np.flatnonzero(b == 2)
    assert np.array_equal(second, first + 1)
    d = g["pos"][second] - g["pos"][first]
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    nrm = g["nrm"][first]
    cos = np.einsum("ij,ij->i", d, nrm)
    se = 1.0 / math.sqrt(n)
    assert (cos > 0).all()
    assert abs(cos.mean() - 2 / 3) < 5 * math.sqrt(1 / 18) * se
    assert abs((cos ** 2).mean() - 0.5) < 5 * math.sqrt(1 / 12) * se
    # tangent components about each face's normal: the two axes the face spans
    for axis in range(3):
        on = np.abs(nrm[:, axis]) > 0.5
        for t in range(3):
            if t != axis:
                c = d[on, t]
                assert abs(c.mean()) < 5 * 0.5 / math.sqrt(on.sum())


# ---------------------------------------------------------------------------
# gather (Eq. 1 indirect part): closed form of one VPL over a plane, energy
# ---------------------------------------------------------------------------
def test_gather_single_vpl_closed_form(orc):
    sc = plane_scene(half=100.0, albedo=0.5)
    o = orc.OracleScene(sc)
    h, Phi = 0.7, 3.0
    s = np.linspace(0.0, 5.0, 41)
    y = np.stack([s, np.zeros_like(s), np.zeros_like(s)], axis=1)
    gb = dict(pos=y, nrm=np.tile([0, 0, 1.0], (len(s), 1)), rho=np.full((len(s), 3), 0.5),
              tri=np.zeros(len(s), np.int64))
    vpl = dict(pos=np.array([[0, 0, h]]), nrm=np.array([[0, 0, -1.0]]),
               flux=np.array([[Phi, Phi, Phi]]))
    out = o.gather(gb, vpl, d2_min=1e-8, eps=1e-6, vis_mode=1)
    want = 0.5 * Phi * h * h / (math.pi ** 2 * (h * h + s * s) ** 2)
    assert np.allclose(out[:, 0], want, rtol=1e-12)


def test_gather_energy_conservation(orc):
    """Irradiance E = pi L / rho of one VPL integrated over the receiving plane
    equals its power (radial quadrature)."""
    sc = plane_scene(half=1e4, albedo=1.0)
    o = orc.OracleScene(sc)
    h, Phi = 1.0, 1.0
    # substitution s = h tan(a) maps [0, inf) to [0, pi/2)
    a = (np.arange(20000) + 0.5) * (math.pi / 2) / 20000
    s = h * np.tan(a)
    y = np.stack([s, np.zeros_like(s), np.zeros_like(s)], axis=1)
    gb = dict(pos=y, nrm=np.tile([0, 0, 1.0], (len(s), 1)), rho=np.ones((len(s), 3)),
              tri=np.zeros(len(s), np.int64))
    vpl = dict(pos=np.array([[0, 0, h]]), nrm=np.array([[0, 0, -1.0]]), flux=np.ones((1, 3)))
    L = o.gather(gb, vpl, d2_min=1e-12, eps=1e-9, vis_mode=2)[:, 0]
    E = math.pi * L
    ds_da = h / np.cos(a) ** 2
    total = (2 * math.pi * s * E * ds_da).sum() * (math.pi / 2) / 20000
    assert abs(total - Phi) < 1e-6


def test_gather_clamp_and_backfaces(orc):
    sc = plane_scene(half=10.0, albedo=1.0)
    o = orc.OracleScene(sc)
    y = np.zeros((1, 3))
    gb = dict(pos=y, nrm=np.array([[0, 0, 1.0]]), rho=np.ones((1, 3)), tri=np.zeros(1, np.int64))
    # VPL facing away from the receiver contributes nothing
    v1 = dict(pos=np.array([[0, 0, 1.0]]), nrm=np.array([[0, 0, 1.0]]), flux=np.ones((1, 3)))
    assert o.gather(gb, v1, 1e-6, 1e-6, vis_mode=1)[0, 0] == 0.0
    # below the clamp distance: cos cos / (pi d2_min)
    h = 0.01
    v2 = dict(pos=np.array([[0, 0, h]]), nrm=np.array([[0, 0, -1.0]]), flux=np.ones((1, 3)))
    d2min = 0.04
    out = o.gather(gb, v2, d2min, 1e-6, vis_mode=1)[0, 0]
    assert abs(out - 1.0 / (math.pi ** 2 * float(F32(d2min)))) < 1e-9
    # empty pixel stays black
    gb_empty = dict(gb, tri=np.full(1, -1, np.int64))
    assert o.gather(gb_empty, v2, d2min, 1e-6, vis_mode=1)[0, 0] == 0.0


# ---------------------------------------------------------------------------
# visibility V (Eq. 1): a hand-built occluder, and BVH == brute force
# ---------------------------------------------------------------------------
def test_visibility_hand_occluder(orc):
    sc = plane_scene(half=0.5, z=0.5)
    o = orc.OracleScene(sc)
    p = np.array([[0, 0, 0], [0, 0, 0], [0.9, 0, 0], [0, 0, 0], [0.2, 0.1, 1.0]], float)
    q = np.array([[0, 0, 1], [0, 0, 0.49], [0.9, 0, 1], [0, 0, 0.5], [0.2, 0.1, 0.0]], float)
    for vm in (0, 1):
        assert o.occluded(p, q, vis_mode=vm).tolist() == [True, False, False, False, True]


def _random_soup(n, seed):
    rng = np.random.default_rng(seed)
    c = rng.uniform(0, 10, size=(n, 1, 3))
    v = (c + rng.normal(0, 0.6, size=(n, 3, 3))).reshape(-1, 3)
    return tri_scene(v, np.arange(3 * n).reshape(-1, 3), 0.5)


@pytest.mark.parametrize("make", ["soup", "cornell", "room"])
def test_bvh_equals_brute_force(orc, make):
    if make == "soup":
        sc = _random_soup(3000, 1)
    elif make == "cornell":
        sc = W.cornell_scene(0)
    else:
        s = W._Soup()
        W._room_zup(s, (4.0, 4.0, 2.0), 4, 4, 2, albedo_fn=lambda: (0.5,) * 3)
        rng = np.random.default_rng(3)
        for _ in range(150):
            lo = rng.uniform(0, 3.5, 3) * [1, 1, 0.3]
            s.box(lo, lo + rng.uniform(0.1, 0.6, 3), (0.5, 0.5, 0.5))
        sc = s.finish(W.cornell_scene(0).light)
    o = orc.OracleScene(sc)
    rng = np.random.default_rng(5)
    lo, hi = sc.verts.min(0), sc.verts.max(0)
    n = 3000
    p = rng.uniform(lo, hi, size=(n, 3))
    q = rng.uniform(lo, hi, size=(n, 3))
    # axis-aligned and vertex-grazing rays too
    q[: n // 4] = p[: n // 4] + np.eye(3)[rng.integers(0, 3, n // 4)] * 3.0
    q[n // 4: n // 2] = sc.verts[rng.integers(0, len(sc.verts), n // 4)]
    assert np.array_equal(o.occluded(p, q, 0), o.occluded(p, q, 1))
    t0, tt0 = o.closest(p, q - p, 0.0, 0)
    t1, tt1 = o.closest(p, q - p, 0.0, 1)
    assert np.array_equal(t0, t1)
    assert np.array_equal(tt0[t0 >= 0], tt1[t1 >= 0])


def test_segment_margin(orc):
    sc = plane_scene(half=0.5, z=0.5)
    o = orc.OracleScene(sc)
    # through the middle of a triangle: margin is the in-plane edge distance
    m = o.segment_margin([0.2, -0.1, 0], [0.2, -0.1, 1])
    assert 0.05 < m < 0.5
    # passing 1e-7 outside the square's edge
    m2 = o.segment_margin([0.5 + 1e-7, 0.1, 0], [0.5 + 1e-7, 0.1, 1])
    assert m2 < 2e-7
    # ending 1e-8 above the plane over the square
    m3 = o.segment_margin([0.2, 0.1, 0], [0.2, 0.1, 0.5 - 1e-8])
    assert m3 < 2e-8


# ---------------------------------------------------------------------------
# G-buffer: ray / plane intersection in closed form
# ---------------------------------------------------------------------------
def test_gbuffer_plane_closed_form(orc):
    z = 2.0
    sc = plane_scene(half=50.0, z=z, up=False)      # faces -z, towards the camera
    o = orc.OracleScene(sc)
    cam = _cam(eye=(0, 0, 0), fwd=(0, 0, 1), up=(0, 1, 0), w=16, h=8, vfov=50.0)
    gb = o.gbuffer(cam)
    tv = math.tan(math.radians(50.0) / 2)
    th = tv * 16 / 8
    for j in range(8):
        for i in range(16):
            k = j * 16 + i
            sx = 2 * (i + 0.5) / 16 - 1
            sy = 1 - 2 * (j + 0.5) / 8
            # camera right = f x up = (0,0,1)x(0,1,0) = (-1,0,0)
            want = np.array([-sx * th * z, sy * tv * z, z])
            assert np.allclose(gb["pos"][k], want, rtol=0, atol=1e-12)
            assert gb["tri"][k] in (0, 1)
            assert np.allclose(gb["nrm"][k], [0, 0, -1])
    # the same plane seen from behind leaves every pixel empty
    o2 = orc.OracleScene(plane_scene(half=50.0, z=z, up=True))
    assert (o2.gbuffer(cam)["tri"] == -1).all()


# ---------------------------------------------------------------------------
# whole pipeline on the tiny scene: budget split and counts
# ---------------------------------------------------------------------------
def test_pipeline_counts_tiny(orc):
    wl = W.cornell_workload(width=32, height=32)
    v = wl.views[0]
    o = orc.OracleScene(wl.scene)
    r = orc.render(o, v)
    g = r["vpl"]
    assert g["status"] == 0
    assert len(g["pos"]) == 256 and g["n_close"] == 8 and g["m_far_kept"] == 64
    assert (g["tag"][:192] == np.arange(192)).all()
    assert np.isfinite(r["image"]).all() and (r["image"] >= 0).all()
    assert r["image"].max() > 0
    # brute-force and BVH visibility give the same image on the tiny scene
    r0 = orc.render(o, v, vis_mode=0)
    assert np.array_equal(r0["image"], r["image"])


# ---------------------------------------------------------------------------
# direct term L_e(y) of Eq. 1: light-sample VPLs, gathered like the others
# ---------------------------------------------------------------------------
def _square_light(power=(2.0, 1.5, 1.0)):
    return W.Light(center=(0.1, 0.2, 1.0), normal=(0, 0, -1), edge_u=(0.4, 0.0, 0.0), edge_v=(0.0, 0.4, 0.0),
                   power=power, type=W.LIGHT_AREA)


def test_light_vpls_follow_philox_and_split_the_power(orc):
    """Sample s: point (2 s1 - 1) eu/2 + (2 s2 - 1) ev/2 from the centre with
    s1, s2 the top 24 bits of Philox words 0, 1 at key (seed, 4), counter
    (s, 0, 0, 0) -- numpy's Philox gives the words; flux P / S each."""
    light = _square_light()
    o = orc.OracleScene(plane_scene(light=light))
    S, seed = 257, 11
    v = o.light_vpls(S, seed)
    f = lambda a: np.array(a, np.float32).astype(np.float64)  # the light is given in FP32
    c, eu, ev = f(light.center), f(light.edge_u), f(light.edge_v)
    for s in range(S):
        w = _numpy_philox_block((s, 0, 0, 0), (seed, 4))
        s1, s2 = (int(w[0]) >> 40) / 2.0**24, (int(w[1]) >> 40) / 2.0**24
        want = c + (2 * s1 - 1) * 0.5 * eu + (2 * s2 - 1) * 0.5 * ev
        assert np.allclose(v["pos"][s], want, rtol=0, atol=1e-15)
    assert np.array_equal(v["nrm"], np.tile([0.0, 0.0, -1.0], (S, 1)))
    assert np.array_equal(v["tag"], -1 - np.arange(S))
    assert np.allclose(v["flux"].sum(0), f(light.power), rtol=1e-12)
    pt = W.Light(center=(0, 0, 1), normal=(0, 0, -1), edge_u=(0, 0, 0), edge_v=(0, 0, 0), power=(1, 1, 1),
                 type=W.LIGHT_POINT)
    assert orc.OracleScene(plane_scene(light=pt)).light_vpls(4, 1) is None


def test_direct_term_matches_lambert(orc):
    """Gathering the light samples over an unoccluded plane gives rho/pi times
    Lambert's closed-form irradiance of the square emitter (radiance
    P / (pi A_L)), within the Monte Carlo error; a receiver facing away or
    behind the emitter's plane gets nothing."""
    light = _square_light(power=(2.0, 2.0, 2.0))
    o = orc.OracleScene(plane_scene(half=100.0, albedo=0.6, light=light))
    v = o.light_vpls(40000, 7)
    xs = np.array([[0.1, 0.2, 0.0], [0.6, -0.3, 0.0], [-1.5, 1.0, 0.0], [3.0, 0.2, 0.0]])
    gb = dict(pos=xs, nrm=np.tile([0, 0, 1.0], (len(xs), 1)), rho=np.full((len(xs), 3), 0.6),
              tri=np.zeros(len(xs), np.int64))
    out = o.gather(gb, v, d2_min=1e-12, eps=1e-9, vis_mode=1)
    c, eu, ev = np.array(light.center), np.array(light.edge_u), np.array(light.edge_v)
    poly = [c - eu / 2 - ev / 2, c + eu / 2 - ev / 2, c + eu / 2 + ev / 2, c - eu / 2 + ev / 2]
    Lrad = 2.0 / (math.pi * 0.16)
    for k, x in enumerate(xs):
        want = 0.6 / math.pi * _lambert_irradiance(x, np.array([0, 0, 1.0]), poly, Lrad)
        assert abs(out[k, 0] - want) < 0.02 * want, (k, out[k, 0], want)
    away = dict(pos=np.array([[0.1, 0.2, 0.0], [0.1, 0.2, 2.0]]), nrm=np.array([[0, 0, -1.0], [0, 0, 1.0]]),
                rho=np.full((2, 3), 0.6), tri=np.zeros(2, np.int64))
    assert np.array_equal(o.gather(away, v, d2_min=1e-12, eps=1e-9, vis_mode=1), np.zeros((2, 3)))


# ---------------------------------------------------------------------------
# patch rule 1 (set sum): a stratum over several faces is one VPL whose value
# is the sum of the faces' Eq. 2 terms with the areas they give it
# ---------------------------------------------------------------------------
def _grid_scene(n, half, light, albedo=0.5):
    xs = np.linspace(-half, half, n + 1)
    verts = np.array([(x, y, 0.0) for y in xs for x in xs], np.float32)
    tris = []
    for j in range(n):
        for i in range(n):
            a, b = j * (n + 1) + i, j * (n + 1) + i + 1
            c, d = a + n + 1, b + n + 1
            tris += [(a, b, d), (a, d, c)]
    return tri_scene(verts, tris, albedo, light)


def test_set_sum_total_flux_and_placement(orc):
    """With faces much smaller than a stratum every VPL sums several faces:
    the total flux is exactly sum_t rho E(c_t) A_t (E of the point light at
    each face's centroid; the quantised areas split without loss), each VPL
    lies at the area-weighted centroid of its faces, on the plane, inside
    the grid, with the plane's normal."""
    light = W.Light(center=(0.3, -0.2, 2.0), normal=(0, 0, -1), edge_u=(1, 0, 0), edge_v=(0, 1, 0),
                    power=(1.0, 2.0, 0.5), type=W.LIGHT_POINT)
    sc = _grid_scene(40, 1.5, light, albedo=0.5)
    cam = _cam(eye=(0, 0, 4), fwd=(0, 0, -1), up=(0, 1, 0), vfov=80)
    o = orc.OracleScene(sc)
    K = 50
    g = o.generate(cam, W.GenParams(d_close=100.0, m_close=K, m_far=0, seed=3, patch_rule=1))
    assert g["status"] == 0 and g["n_close"] == 3200
    V = sc.verts.astype(np.float64)
    T = sc.tris
    cen = V[T].mean(axis=1)
    area = 0.5 * np.linalg.norm(np.cross(V[T[:, 1]] - V[T[:, 0]], V[T[:, 2]] - V[T[:, 0]]), axis=1)
    p = np.array(light.center, np.float64)
    dv = p - cen
    r = np.linalg.norm(dv, axis=1)
    E = np.maximum(dv[:, 2] / r, 0) / (4 * math.pi * r * r)
    want = 0.5 * np.array(light.power) * (E * area).sum()
    assert np.allclose(g["flux"].sum(axis=0), want, rtol=1e-9)
    assert np.allclose(g["pos"][:, 2], 0.0, atol=1e-12)
    assert (np.abs(g["pos"][:, :2]) <= 1.5).all()
    assert np.allclose(g["nrm"], [0, 0, 1.0])
    # consecutive strata cover consecutive runs of faces: their VPLs differ
    assert len({tuple(np.round(x, 9)) for x in g["pos"]}) == K


def test_set_sum_equals_point_rule_inside_single_faces(orc):
    """A stratum inside one face keeps the point rule: on two large faces
    only the stratum that straddles their common edge can differ."""
    light = W.Light(center=(0.3, -0.2, 2.0), normal=(0, 0, -1), edge_u=(1, 0, 0), edge_v=(0, 1, 0),
                    power=(1.0, 2.0, 0.5), type=W.LIGHT_POINT)
    sc = plane_scene(half=1.5, albedo=0.5, light=light)
    cam = _cam(eye=(0, 0, 4), fwd=(0, 0, -1), up=(0, 1, 0), vfov=80)
    o = orc.OracleScene(sc)
    a = o.generate(cam, W.GenParams(d_close=100.0, m_close=64, m_far=0, seed=9, patch_rule=0))
    b = o.generate(cam, W.GenParams(d_close=100.0, m_close=64, m_far=0, seed=9, patch_rule=1))
    same = (a["pos"] == b["pos"]).all(axis=1) & (a["flux"] == b["flux"]).all(axis=1)
    assert same.sum() >= 63 and np.array_equal(a["tri"][same], b["tri"][same])


# ---------------------------------------------------------------------------
# rejection-sampled instant radiosity (the comparison method cited as r3)
# ---------------------------------------------------------------------------
def _rs_view(seed=0, m=64):
    import dataclasses
    wl = W.cornell_workload()
    v = wl.views[0]
    gen = dataclasses.replace(v.gen, m_close=0, m_far=m, d_close=0.0, seed=seed)
    return wl, v, gen


def test_rs_vpls_are_ir_candidates_with_probabilities(orc):
    """Every kept VPL is the hit (path, bounce) of plain instant radiosity's
    walk -- same point, normal and face -- and its flux is the plain one
    divided by its acceptance probability p in (0, 1] (the same p in every
    channel); some VPLs were kept for sure (p = 1), some with p < 1."""
    import dataclasses
    wl, v, gen = _rs_view(seed=3)
    o = orc.OracleScene(wl.scene)
    rs = o.generate_rs(v.camera, gen, 8, v.gather.d2_min, v.gather.ray_eps, vis_mode=1)
    assert rs["status"] == 0 and rs["m_far_kept"] == gen.m_far
    big = dataclasses.replace(gen, m_far=3 * rs["paths"] + 3, ir_max_paths=rs["paths"])
    ir = o.generate(v.camera, big, vis_mode=1)
    assert (np.diff(rs["tag"]) > 0).all()
    where = {int(t): k for k, t in enumerate(ir["tag"])}
    ps = []
    for k, t in enumerate(rs["tag"]):
        j = where[int(t)]
        assert np.array_equal(rs["pos"][k], ir["pos"][j]) and np.array_equal(rs["nrm"][k], ir["nrm"][j])
        assert rs["tri"][k] == ir["tri"][j]
        # flux_ir = power * albedos / P_ir (P_ir = ir paths), flux_rs = power * albedos / (P_rs p)
        p = (ir["flux"][j] * ir["paths"]) / (rs["flux"][k] * rs["paths"])
        assert np.allclose(p, p[0], rtol=1e-12) and 0.0 < p[0] <= 1.0 + 1e-12
        ps.append(p[0])
    ps = np.array(ps)
    assert (ps > 1 - 1e-12).any() and (ps < 0.999).any()


def test_rs_total_flux_matches_plain_ir_in_expectation(orc):
    """Dividing by p keeps the estimator unbiased: over many seeds the mean
    total flux of the kept VPLs equals plain instant radiosity's, within
    four standard errors."""
    rs, ir = [], []
    wl, v, _ = _rs_view()
    o = orc.OracleScene(wl.scene)
    for seed in range(120):
        _, _, gen = _rs_view(seed=seed)
        rs.append(o.generate_rs(v.camera, gen, 8, v.gather.d2_min, v.gather.ray_eps, vis_mode=1)["flux"].sum(0))
        ir.append(o.generate(v.camera, gen, vis_mode=1)["flux"].sum(0))
    rs, ir = np.array(rs), np.array(ir)
    se = np.sqrt(rs.var(0) / len(rs) + ir.var(0) / len(ir))
    assert (np.abs(rs.mean(0) - ir.mean(0)) < 4 * se).all(), (rs.mean(0), ir.mean(0), se)


def test_rs_keeps_only_vpls_that_light_the_pilot_pixels(orc):
    """A candidate that reaches none of the pilot pixels has c = 0, p = 0."""
    wl, v, gen = _rs_view(seed=5)
    o = orc.OracleScene(wl.scene)
    pilot = 8
    rs = o.generate_rs(v.camera, gen, pilot, v.gather.d2_min, v.gather.ray_eps, vis_mode=1)
    cam = v.camera
    pc = W.Camera(cam.eye, cam.forward, cam.up, cam.vfov_deg, pilot, max(1, (pilot * cam.height + cam.width // 2) // cam.width))
    gb = o.gbuffer(pc, vis_mode=1)
    for k in range(len(rs["pos"])):
        one = dict(pos=rs["pos"][k:k + 1], nrm=rs["nrm"][k:k + 1], flux=np.ones((1, 3)))
        assert o.gather(gb, one, v.gather.d2_min, v.gather.ray_eps, vis_mode=1).sum() > 0, k


def test_ir_path_replay_matches_generation(orc):
    """orc_ir_path (the replay the GPU parity tests use to explain a light
    path that changed course) gives the rays of orc_generate's walks: each
    far VPL tagged (p, b) is the front hit of ray b of path p, at o + t d."""
    wl = W.room200k_workload()
    v = wl.views[0]
    o = orc.OracleScene(wl.scene)
    g = o.generate(v.camera, v.gen, vis_mode=0)
    Mc = v.gen.m_close
    for i in range(Mc, Mc + v.gen.m_far, 7):
        p, b = divmod(int(g["tag"][i]), 16)
        r = o.ir_path(v.gen, p)
        assert len(r["k"]) >= b and r["front"][b - 1] and r["k"][b - 1] == g["tri"][i]
        assert np.array_equal(r["o"][b - 1] + r["d"][b - 1] * r["t"][b - 1], g["pos"][i])
        assert (r["front"][:b]).all()
