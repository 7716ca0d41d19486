"""Direct term L_e(y) of Eq. 1 on the GPU: light-sample VPLs against the
oracle (bit for bit in FP32), the composite gather (indirect VPLs and light
samples in one set) against the oracle on identical inputs, and the point
light refused."""
import dataclasses

import numpy as np
import pytest

from paper_2203_11484_gb300 import workloads as W
import parity as PY
from test_gpu_parity import V, ctx, cornell, room, _check_gather  # noqa: F401  (fixtures)

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _cat(a: dict, b: dict) -> dict:
    return {k: np.concatenate([a[k], b[k]]) for k in ("pos", "nrm", "flux")}


@pytest.mark.parametrize("fmt", [0, 1])
def test_light_vpls_bit_exact(V, ctx, cornell, fmt):
    wl, sid, osc = cornell
    n, seed = 777, 9
    vs = V.VplSet.empty(n, fmt=fmt)
    V.vpl_light_vpls(ctx.h, sid, n, seed, vs)
    assert V.vpl_sync(ctx.h, check=False) == 0
    ref = osc.light_vpls(n, seed)
    pos = vs.pos.cpu().numpy()
    assert np.array_equal(pos[:, :3], ref["pos"].astype(np.float32))
    if fmt == 0:
        assert np.array_equal(vs.nrm.cpu().numpy()[:, :3], ref["nrm"].astype(np.float32))
        assert np.array_equal(vs.flux.cpu().numpy()[:, :3], ref["flux"].astype(np.float32))
        assert np.array_equal(vs.nrm.cpu().numpy()[:, 3].copy().view(np.int32), ref["tag"].astype(np.int32))
        assert np.array_equal(pos[:, 3].copy().view(np.int32), np.full(n, -1, np.int32))
    else:  # FP16 rows: colour / max in half, magnitude in pos.w
        m = ref["flux"].max(1).astype(np.float32)
        assert np.array_equal(pos[:, 3], m)
        col = vs.flux.float().cpu().numpy()[:, :3] * pos[:, 3:4]
        assert np.allclose(col, ref["flux"], rtol=1e-3)
        assert np.allclose(vs.nrm.float().cpu().numpy()[:, :3], ref["nrm"], atol=1e-3)


def test_composite_gather_parity_cornell(V, ctx, cornell):
    """Indirect VPLs and light samples in one set: the GPU gather equals the
    oracle's on the same FP32 inputs (flips explained, within the bound)."""
    wl, sid, osc = cornell
    view = wl.views[0]
    gb = osc.gbuffer(view.camera, vis_mode=1)
    vp = _cat(osc.generate(view.camera, view.gen, vis_mode=1), osc.light_vpls(256, 3))
    params = W.GatherParams(view.gather.d2_min, view.gather.ray_eps, W.PREC_FP32, W.VIS_BVH)
    got, ref, _ = _check_gather(V, ctx, sid, osc, wl, gb, vp, view.camera.width, view.camera.height, params, 0)
    direct = osc.gather(*PY.oracle_inputs_f32(gb, osc.light_vpls(256, 3)), params.d2_min, params.ray_eps,
                        vis_mode=0)
    assert direct.max() > 0 and ref.max() > direct.max()  # the composite holds both terms


def test_composite_is_direct_plus_indirect_on_gpu(V, ctx, room):
    """GPU pipeline on the 200k-triangle room: generate into rows [0, M),
    light samples into rows [M, M + S) of one set; one gather of all rows
    equals the sum of the two gathers up to FP32 rounding."""
    wl, sid, osc = room
    view = wl.views[0]
    cam = dataclasses.replace(view.camera, width=256, height=256)
    gen = dataclasses.replace(view.gen, m_close=768, m_far=256)
    M, S = gen.m_close + gen.m_far, 128
    gb = V.GBuffer.empty(cam.width, cam.height)
    V.vpl_gbuffer_build(ctx.h, sid, cam, gb)
    vs = V.VplSet.empty(M + S)
    V.vpl_generate(ctx.h, sid, cam, gen, vs.rows(0, M))
    V.vpl_light_vpls(ctx.h, sid, S, 17, vs.rows(M, S))
    outs = []
    for part in (vs, vs.rows(0, M), vs.rows(M, S)):
        o = torch.zeros((cam.width * cam.height, 4), device="cuda")
        V.vpl_gather(ctx.h, sid, gb, part, view.gather, o)
        outs.append(o)
    assert V.vpl_sync(ctx.h, check=False) == 0
    both, ind, dire = (o.cpu().numpy()[:, :3].astype(np.float64) for o in outs)
    assert dire.max() > 0 and ind.max() > 0
    close = np.isclose(both, ind + dire, rtol=1e-5, atol=1e-7 * both.mean()).all(1)
    assert close.mean() >= 0.999, close.mean()  # a visibility tie may fall either way


def test_light_vpls_refuse_point_light_and_bad_counts(V, ctx, cornell):
    wl, sid, osc = cornell
    sc = dataclasses.replace(wl.scene, light=W.Light(center=(0.5, 0.9, 0.5), normal=(0, -1, 0), edge_u=(0, 0, 0),
                                                     edge_v=(0, 0, 0), power=(1, 1, 1), type=W.LIGHT_POINT))
    sid_pt = ctx.upload(sc)
    with pytest.raises(V.VplError) as e:
        V.vpl_light_vpls(ctx.h, sid_pt, 4, 1, V.VplSet.empty(4))
    assert e.value.code == 8
    V.vpl_scene_release(ctx.h, sid_pt)
    with pytest.raises(V.VplError) as e:
        V.vpl_light_vpls(ctx.h, sid, 5, 1, V.VplSet.empty(4))
    assert e.value.code == 1
    V.vpl_light_vpls(ctx.h, sid, 0, 1, V.VplSet.empty(0))   # nothing to do
    assert V.vpl_sync(ctx.h, check=False) == 0
