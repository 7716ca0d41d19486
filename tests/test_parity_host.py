"""The parity checker itself, on the CPU: fed the oracle's own generation as
both sides it passes; fed a copy with a planted mistake (a light path that
changed course with no edge near it, a position outside its derived bound,
a flux off with no visibility flip, a shifted patch face) it fails.  The
mistakes are planted in a copy of the oracle's output, never in the oracle."""
import copy
import dataclasses

import numpy as np
import pytest

from paper_2203_11484_gb300 import workloads as W
import parity as PY


@pytest.fixture(scope="module")
def room(orc):
    wl = W.room200k_workload()
    view = wl.views[0]
    osc = orc.OracleScene(wl.scene)
    r = osc.generate(view.camera, view.gen, vis_mode=0)
    info = dict(n_close=r["n_close"], shift_s=r["shift_s"], f_total=r["f_total"], paths=r["paths"],
                m_far_kept=r["m_far_kept"])
    return osc, view, r, info


def test_checker_accepts_identical_rows(room):
    osc, view, r, info = room
    assert PY.check_generation(osc, view.camera, view.gen, copy.deepcopy(r), r, info) == (0, 0)


def test_ir_position_bounds_are_fp32_sized(room):
    """The derived bounds sit between one FP32 ulp of the coordinates and a
    few hundred ulps (grazing hits), never at the old blanket 1e-4 of the
    diagonal for the typical VPL."""
    osc, view, r, _ = room
    Mc, Ld = view.gen.m_close, osc.scene.diag()
    R = float(np.abs(osc.scene.verts).max())
    b = []
    for t in r["tag"][Mc:Mc + 200]:
        p, k = divmod(int(t), 16)
        b.append(PY.ir_replay(osc, view.gen, p)[1][k - 1])
    b = np.array(b)
    assert b.min() >= 2 ** -24 * R
    assert np.median(b) <= 1e-5 * Ld


def _drop_path(r, view, p):
    """The far VPLs of path p removed and the list refilled from a longer
    oracle run: what a GPU walk that lost that path's hits would report."""
    Mc, Mf = view.gen.m_close, view.gen.m_far
    g = copy.deepcopy(r)
    keep = [i for i in range(Mc, Mc + Mf) if int(r["tag"][i]) // 16 != p]
    n_drop = Mf - len(keep)
    return g, keep, n_drop


def test_checker_rejects_an_unexplained_divergent_path(room, orc):
    osc, view, r, info = room
    Mc, Mf = view.gen.m_close, view.gen.m_far
    gen2 = dataclasses.replace(view.gen, m_far=Mf + 64)
    r2 = osc.generate(view.camera, gen2, vis_mode=0)
    # a path none of whose rays passes near an edge
    reach = 2 * osc.scene.diag()
    for t in r["tag"][Mc + 10:Mc + 200]:
        p = int(t) // 16
        rp, _, carried = PY.ir_replay(osc, view.gen, p)
        if not any(PY.flip_explained(osc, rp["o"][b], PY._ray_end(rp, b, reach), carried[b], ends=0)
                   for b in range(len(rp["k"]))):
            break
    else:
        pytest.skip("every path grazes an edge")
    keep = [i for i in range(Mc, Mc + Mf + 64) if int(r2["tag"][i]) // 16 != p][:Mf]
    g = copy.deepcopy(r)
    for key in ("pos", "nrm", "flux", "tri", "tag"):
        g[key][Mc:] = r2[key][keep]
    gi = dict(info, paths=int(r2["tag"][keep[-1]]) // 16 + 1)
    g["flux"][Mc:] *= r2["paths"] / gi["paths"]
    with pytest.raises(AssertionError, match="changed course"):
        PY.check_far_vpls(osc, view.gen, g, r, gi["paths"], info["paths"])


def test_checker_rejects_a_position_outside_its_bound(room):
    osc, view, r, info = room
    Mc = view.gen.m_close
    g = copy.deepcopy(r)
    i = Mc + 5
    p, b = divmod(int(r["tag"][i]), 16)
    bound = PY.ir_replay(osc, view.gen, p)[1][b - 1]
    g["pos"][i, 0] += 3 * bound
    with pytest.raises(AssertionError):
        PY.check_far_vpls(osc, view.gen, g, r, info["paths"], info["paths"])


def test_checker_rejects_a_flux_off_without_a_flip(room):
    osc, view, r, info = room
    g = copy.deepcopy(r)
    k = int(np.nonzero(r["flux"][:view.gen.m_close, 0] > 0)[0][3])
    g["flux"][k] *= 1.0 + 1e-5                       # a lit patch VPL
    with pytest.raises(AssertionError):
        PY.check_patch_vpls(osc, view.camera, view.gen, g, r)
    g = copy.deepcopy(r)
    g["flux"][view.gen.m_close + 3] *= 1.0 + 1e-5    # a light-path VPL
    with pytest.raises(AssertionError):
        PY.check_far_vpls(osc, view.gen, g, r, info["paths"], info["paths"])


def test_checker_rejects_a_shifted_patch_face(room):
    osc, view, r, info = room
    g = copy.deepcopy(r)
    g["tri"][7] = g["tri"][8] if g["tri"][8] != g["tri"][7] else g["tri"][7] + 1
    with pytest.raises(AssertionError):
        PY.check_patch_vpls(osc, view.camera, view.gen, g, r)


def test_flip_ratio_scales_with_incidence_and_distance(orc):
    """orc_flip_ratio on a square at z = 0.5: a segment through the middle
    of a triangle is far from any flip, one 1e-7 outside an edge at normal
    incidence is within FP32 reach, and the same in-plane distance becomes
    easier to reach as the segment grazes the plane."""
    v = [(-0.5, -0.5, 0.5), (0.5, -0.5, 0.5), (0.5, 0.5, 0.5), (-0.5, 0.5, 0.5)]
    sc = W.Scene(np.array(v, np.float32), np.array([(0, 1, 2), (0, 2, 3)], np.int32),
                 np.full((2, 3), 0.5, np.float32),
                 W.Light((0, 0, 10.0), (0, 0, -1.0), (1, 0, 0), (0, 1, 0), type=W.LIGHT_POINT))
    o = orc.OracleScene(sc)
    assert o.flip_ratio([0.2, -0.1, 0], [0.2, -0.1, 1], 16.0) > 1e4
    assert o.flip_ratio([0.5 + 1e-7, 0.1, 0], [0.5 + 1e-7, 0.1, 1], 16.0) < 1.0
    assert o.flip_ratio([0.5 + 1e-5, 0.1, 0], [0.5 + 1e-5, 0.1, 1], 16.0) > 1.0
    # grazing at cos 1e-3: 1e-5 in the plane is within reach
    d = np.array([1.0, 0.0, 1e-3])
    mid = np.array([0.5 + 1e-5, 0.1, 0.5])
    assert o.flip_ratio(mid - 0.3 * d, mid + 0.3 * d, 16.0) < 1.0
    # extra end-point error widens the reach
    assert o.flip_ratio([0.5 + 1e-5, 0.1, 0], [0.5 + 1e-5, 0.1, 1], 16.0, 1e-4) < 1.0
