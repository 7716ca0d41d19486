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
