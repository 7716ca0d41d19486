"""FP16 attribute storage with FP32 shading (plain or Kahan-compensated sums).

FP16 rows must be exact roundings of the FP32 rows; the image error of each
variant is measured against the FP64 oracle twice: on the original
attributes (what a user gets) and on the attributes rounded the way the FP16
path stores them (which leaves only the FP32 accumulation error).
"""
import numpy as np
import pytest

from paper_2203_11484_gb300 import workloads as W
import parity as PY

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def V():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2203_11484_gb300 import build, vpl
    build.build_library()
    return vpl


@pytest.fixture(scope="module")
def room(V, orc):
    ctx = V.Context(0)
    wl = W.room200k_workload()
    sid = ctx.upload(wl.scene)
    yield ctx, wl, sid, orc.OracleScene(wl.scene)
    ctx.close()


def _f16(a):
    return np.asarray(a, np.float32).astype(np.float16)


def test_fp16_rows_are_roundings_of_fp32_rows(V, room):
    ctx, wl, sid, _ = room
    view = wl.views[0]
    cam = W.Camera(view.camera.eye, view.camera.forward, view.camera.up, view.camera.vfov_deg, 96, 64)
    g32, g16 = V.GBuffer.empty(96, 64), V.GBuffer.empty(96, 64, fmt=V.FORMAT_FP16)
    V.vpl_gbuffer_build(ctx.h, sid, cam, g32)
    V.vpl_gbuffer_build(ctx.h, sid, cam, g16)
    M = view.gen.m_close + view.gen.m_far
    v32, v16 = V.VplSet.empty(M), V.VplSet.empty(M, fmt=V.FORMAT_FP16)
    V.vpl_generate(ctx.h, sid, cam, view.gen, v32)
    V.vpl_generate(ctx.h, sid, cam, view.gen, v16)
    assert V.vpl_sync(ctx.h, check=False) == 0
    assert torch.equal(g32.pos, g16.pos)
    assert np.array_equal(g16.nrm.cpu().numpy(), _f16(g32.nrm.cpu().numpy()[:, :4] * [1, 1, 1, 0]))
    assert np.array_equal(g16.albedo.cpu().numpy(), _f16(g32.albedo.cpu().numpy()))
    p32, p16 = v32.pos.cpu().numpy(), v16.pos.cpu().numpy()
    phi = v32.flux.cpu().numpy()[:, :3]
    m = phi.max(axis=1).astype(np.float32)
    assert np.array_equal(p16[:, :3], p32[:, :3])
    assert np.array_equal(p16[:, 3], m)
    inv = np.where(m > 0, np.float32(1.0) / np.where(m > 0, m, 1), 0).astype(np.float32)
    want = np.zeros((M, 4), np.float16)
    want[:, :3] = _f16(phi.astype(np.float32) * inv[:, None])
    assert np.array_equal(v16.flux.cpu().numpy(), want)
    nn = np.zeros((M, 4), np.float16)
    nn[:, :3] = _f16(v32.nrm.cpu().numpy()[:, :3])
    assert np.array_equal(v16.nrm.cpu().numpy(), nn)


def test_precision_variants_error_report(V, room):
    """2048 sampled receivers of the 200k-triangle room, 4096 VPLs: FP32,
    FP16 + Kahan, FP16 plain against the FP64 oracle."""
    ctx, wl, sid, osc = room
    view = wl.views[0]
    pix = np.random.default_rng(21).choice(view.camera.width * view.camera.height, 2048, replace=False)
    report = PY.precision_report(V, torch, ctx, sid, osc, view, pix, wl.scene.diag())
    print("precision report (2048 receivers x 4096 VPLs):", report)
    PY.check_precision_report(report)


def test_render_fp16_matches_fp32_closely(V, room):
    """vpl_render in FP16 + Kahan against vpl_render in FP32, same view."""
    ctx, wl, sid, _ = room
    view = wl.views[0]
    cam = W.Camera(view.camera.eye, view.camera.forward, view.camera.up, view.camera.vfov_deg, 256, 256)
    outs = {}
    for prec in (W.PREC_FP32, W.PREC_FP16_KAHAN):
        params = W.GatherParams(view.gather.d2_min, view.gather.ray_eps, prec, W.VIS_BVH)
        out = torch.zeros((256 * 256, 4), dtype=torch.float32, device="cuda")
        V.vpl_render(ctx.h, sid, cam, view.gen, params, out)
        assert V.vpl_sync(ctx.h, check=False) == 0
        outs[prec] = out.cpu().numpy()[:, :3].astype(np.float64)
    a, b = outs[W.PREC_FP32], outs[W.PREC_FP16_KAHAN]
    mask = a.max(axis=1) > 1e-3 * a.max()
    rel = np.abs(a - b)[mask] / np.abs(a)[mask].clip(1e-30)
    assert np.median(rel) < 2e-3 and np.isfinite(b).all()
