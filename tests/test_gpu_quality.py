"""The quality study end to end on a small case (GPU): errors shrink with
the VPL count and the report is complete; the renders it compares (hybrid
and plain instant radiosity, square and point light) match the oracle."""
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


@pytest.mark.parametrize("light", ["area", "point"])
@pytest.mark.parametrize("method", ["hybrid", "instant radiosity"])
def test_study_renders_match_the_oracle(orc, light, method):
    """The renders the study compares are the oracle's: the hybrid (alpha
    0.75) and plain instant radiosity (m_close = 0, d_close = 0) of the
    study's view, with the square light and with the point light, against
    the FP64 pipeline on sampled pixels (VPL rows checked first, failing
    pixels explained by visibility flips)."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import dataclasses
    import oracle as O
    import parity as PY
    from paper_2203_11484_gb300 import build, vpl as V
    build.build_library()
    wl = W.room200k_workload(width=96, height=96, seed=1)
    scene = wl.scene if light == "area" else Q.point_light_scene(wl.scene)
    v = wl.views[0]
    mc, mf = W.split_budget(1024, 0.75 if method == "hybrid" else 0.0)
    gen = dataclasses.replace(v.gen, m_close=mc, m_far=mf, seed=100,
                              d_close=v.gen.d_close if mc > 0 else 0.0)
    view = W.View(v.camera, gen, v.gather)
    ctx = V.Context(0)
    try:
        sid = ctx.upload(scene)
        cam = view.camera
        img = torch.zeros((cam.width * cam.height, 4), dtype=torch.float32, device="cuda")
        V.vpl_render(ctx.h, sid, cam, gen, view.gather, img)
        assert V.vpl_sync(ctx.h, check=False) == 0
        img = img.cpu().numpy()
        osc = orc.OracleScene(scene)
        pix = np.random.default_rng(4).choice(cam.width * cam.height, 256, replace=False)
        r = O.render(osc, view, pix)
        gb = V.GBuffer.empty(cam.width, cam.height)
        V.vpl_gbuffer_build(ctx.h, sid, cam, gb)
        V.vpl_sync(ctx.h)
        same = gb.pos.cpu().numpy()[pix, 3].copy().view(np.int32) == r["gbuffer"]["tri"]
        assert same.mean() >= 0.99
        n_bad, n_still, flips = PY.explain_render_pixels(V, torch, ctx, sid, osc, view, img, pix, r["image"],
                                                         r["vpl"], same, scene.diag())
        assert flips <= max(3, PY.FLIP_FRACTION * len(pix) * (mc + mf)), flips
        assert r["image"].max() > 0
    finally:
        ctx.close()
