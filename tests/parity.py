"""Helpers shared by the GPU parity tests: tolerances and explanations of
visibility flips.  Tolerances (per pixel, per component):
    |gpu - ref| <= 1e-4 |ref| + 1e-7 mean(ref)
VPL positions within 1e-6 of the scene diagonal, fluxes within 1e-6
relative; a GPU/oracle visibility disagreement counts as a flip when the
oracle finds the segment within 1e-5 of the scene diagonal of an edge or a
plane crossing."""
import numpy as np

PIX_RTOL = 1e-4
PIX_ATOL_FRAC = 1e-7
POS_TOL = 1e-6     # x scene diagonal
FLUX_RTOL = 1e-6
FLIP_MARGIN = 1e-5  # x scene diagonal
FLIP_FRACTION = 1e-5


def pixel_fail(gpu: np.ndarray, ref: np.ndarray) -> np.ndarray:
    """Boolean mask of pixels outside the tolerance (any channel)."""
    gpu = np.asarray(gpu, np.float64)[..., :3]
    ref = np.asarray(ref, np.float64)[..., :3]
    atol = PIX_ATOL_FRAC * max(float(np.abs(ref).mean()), 1e-30)
    bad = np.abs(gpu - ref) > PIX_RTOL * np.abs(ref) + atol
    return bad.reshape(-1, 3).any(axis=1)


def f32(a) -> np.ndarray:
    return np.asarray(a, np.float32).astype(np.float64)


def oracle_inputs_f32(gb: dict, vpl: dict) -> tuple:
    """Oracle G-buffer / VPLs rounded to FP32 (the GPU's input precision) and
    widened back, so both sides read identical inputs."""
    g = dict(pos=f32(gb["pos"]), nrm=f32(gb["nrm"]), rho=f32(gb["rho"]), tri=gb["tri"].copy())
    v = dict(pos=f32(vpl["pos"]), nrm=f32(vpl["nrm"]), flux=f32(vpl["flux"]))
    return g, v


def explain_pixel(oscene, y, ny, vpl, gpu_vis_row, d2_min, eps, L_diag):
    """Compare one pixel's GPU visibility bits with the oracle's.  Returns
    (n_flips, all_explained, flipped_term_sum)."""
    term, vis, _ = oscene.pairs(y, ny, vpl, d2_min, eps, vis_mode=0)
    traced = vis >= 0
    g = np.asarray(gpu_vis_row)
    flips = traced & (g >= 0) & (g != vis)
    flips |= traced != (g >= 0)
    if not flips.any():
        return 0, True, 0.0
    _, _, margin = oscene.pairs(y, ny, vpl, d2_min, eps, vis_mode=0, want_margin=flips)
    ok = bool((margin[flips] <= FLIP_MARGIN * L_diag).all())
    return int(flips.sum()), ok, float(np.abs(term[flips]).sum())
