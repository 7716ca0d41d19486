"""Host logic of the quality study: the equal-RMSE interpolation."""
import math

from paper_2203_11484_gb300 import quality as Q


def test_interp_m_log_log():
    ms, errs = [1000, 2000, 4000, 8000], [0.08, 0.04, 0.02, 0.01]   # error ~ 1 / M
    assert abs(Q._interp_m(ms, errs, 0.04) - 2000) < 1e-9
    assert abs(Q._interp_m(ms, errs, 0.0283) - 1000 * 0.08 / 0.0283) < 1.0
    assert Q._interp_m(ms, errs, 0.005) == float("inf")      # never reached
    assert Q._interp_m(ms, errs, 0.1) == 1000.0              # already below at the first count
    assert math.isfinite(Q._interp_m([1, 2], [0.5, 0.5], 0.5))


def test_equal_rmse_recovers_a_known_ratio_with_an_interval():
    """Error ~ c / sqrt(M) with c twice as large for plain IR: IR needs 4x
    the VPLs for the hybrid's error; the bootstrap interval brackets it."""
    import numpy as np
    rng = np.random.default_rng(0)

    def curve(method, ms, c):
        rows = []
        for m in ms:
            e = list(c / np.sqrt(m) * (1 + 0.05 * rng.standard_normal(16)))
            rows.append(dict(method=method, vpls=m, rmse=float(np.mean(e)), errs=e, ms=m / 100.0))
        return rows
    hyb = curve("hybrid", [1024, 2048, 4096], 1.0)
    ir = curve("instant radiosity", [1024, 2048, 4096, 8192, 16384, 32768], 2.0)
    for r in Q.equal_rmse(hyb, ir, 16, n_boot=300):
        lo, hi = r["vpl_ratio_90ci"]
        assert 3.5 < r["vpl_ratio"] < 4.5 and lo <= r["vpl_ratio"] <= hi
        assert 3.5 < r["time_ratio"] < 4.5             # time ~ M here
