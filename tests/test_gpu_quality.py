"""The quality study end to end on a small case (GPU): errors shrink with
the VPL count and the report is complete."""
import math

import numpy as np
import pytest

from paper_2203_11484_gb300 import quality as Q
from paper_2203_11484_gb300 import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.mark.parametrize("light", ["area", "point"])
def test_quality_study_small(light):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    wl = W.room200k_workload(width=96, height=96, seed=1)
    scene = wl.scene if light == "area" else Q.point_light_scene(wl.scene)
    res = Q.study(wl.views[0], scene, ms=(256, 1024), ir_ms=(256, 1024, 4096), seeds=2, m_ref=16384, ref_renders=2,
                  bias_m=8192)
    ir = [r["rmse"] for r in res["instant_radiosity"]]
    assert all(math.isfinite(r["rmse"]) for r in res["rejection_sampling"])
    hy = [r["rmse"] for r in res["hybrid"]]
    assert all(math.isfinite(e) and e > 0 for e in ir + hy)
    assert ir[-1] < ir[0] and hy[-1] < hy[0]
    assert res["reference"]["mean"] > 0
    assert len(res["equal_rmse"]) == 2 and len(res["equal_vpls"]) == 2
    assert "| VPLs |" in Q.markdown(res, "t")
