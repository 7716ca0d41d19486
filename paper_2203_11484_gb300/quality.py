"""Quality study of the hybrid sampler against plain instant radiosity.

The paper (Sec. 4) compares its hybrid VPL sampling with instant radiosity and
rejection sampling (among others) on
close-up views: the RMSE of the indirect image against a reference made by
densely sampled instant radiosity (more than 200k VPLs) at equal VPL counts,
and the VPL count and time each method needs for equal RMSE.  This module
runs that comparison on the synthetic scenes through the library's own
calls: the hybrid is alpha * M patch VPLs plus the rest from light paths,
plain instant radiosity is m_close = 0 with no close range (d_close = 0: every
light-path hit is a VPL), the rejection sampling is vpl_generate_rs (plain light paths, candidates kept
in proportion to their estimated contribution), the reference is plain
instant radiosity with many VPLs.  Indirect light only,
as in the paper.  Light: the scene's square light, or a point light at its
centre with the same power (the paper's scenes use point lights).

    python -m paper_2203_11484_gb300.quality [--light area|point] [--width 256 --height 256]
"""
from __future__ import annotations

import argparse
import dataclasses
import json
import math
import statistics
from typing import Dict, List, Sequence

import numpy as np

from . import workloads as W


def _rmse(img, ref) -> float:
    d = (img[:, :3] - ref[:, :3]).double()
    return float(d.pow(2).mean().sqrt())


def _interp_m(ms: Sequence[int], errs: Sequence[float], target: float) -> float:
    """VPL count at which an error curve reaches `target` (log-log
    interpolation between measured counts; inf when it never does)."""
    for k in range(len(ms) - 1):
        e0, e1 = errs[k], errs[k + 1]
        if (e0 - target) * (e1 - target) <= 0 and e0 != e1:
            f = (math.log(target) - math.log(e0)) / (math.log(e1) - math.log(e0))
            return math.exp(math.log(ms[k]) + f * (math.log(ms[k + 1]) - math.log(ms[k])))
    return float(ms[0]) if target >= errs[0] else float("inf")


def equal_rmse(hyb: List[Dict], ir: List[Dict], seeds: int, n_boot: int = 2000, seed: int = 7) -> List[Dict]:
    """For each hybrid VPL count, the plain-IR VPL count (and render time)
    that reaches the hybrid's mean RMSE, by log-log interpolation of IR's
    mean-RMSE curve, with a 90% bootstrap interval: the seeds of every row
    are resampled with replacement, both curves' means recomputed and the
    count found again (5th and 95th percentiles; inf when IR's curve never
    reaches the hybrid's error within the measured counts)."""
    ir_m = [r["vpls"] for r in ir]
    ir_t = [r["ms"] for r in ir]
    rng = np.random.default_rng(seed)
    boot_ir = [np.array([np.mean(rng.choice(r["errs"], len(r["errs"]))) for _ in range(n_boot)]) for r in ir]
    out = []
    for r in hyb:
        m_ir = _interp_m(ir_m, [q["rmse"] for q in ir], r["rmse"])
        t_ir = float("inf") if math.isinf(m_ir) else float(np.interp(math.log(m_ir), np.log(ir_m), ir_t))
        bh = np.array([np.mean(rng.choice(r["errs"], len(r["errs"]))) for _ in range(n_boot)])
        ratios = np.array([_interp_m(ir_m, [b[k] for b in boot_ir], bh[k]) / r["vpls"] for k in range(n_boot)])
        lo, hi = np.percentile(ratios, [5, 95], method="nearest")
        out.append({"hybrid_vpls": r["vpls"], "rmse": r["rmse"], "ir_vpls_for_equal_rmse": m_ir,
                    "vpl_ratio": m_ir / r["vpls"], "vpl_ratio_90ci": [float(lo), float(hi)],
                    "time_ratio": t_ir / r["ms"], "ir_ms": t_ir, "hybrid_ms": r["ms"]})
    return out


def study(view: W.View, scene: W.Scene, ms: Sequence[int] = (1024, 2048, 4096, 8192),
          ir_ms: Sequence[int] = (1024, 2048, 4096, 8192, 16384, 32768), seeds: int = 4,
          m_ref: int = 262144, ref_renders: int = 4, alpha: float = 0.75, bias_m: int = 65536,
          ctx=None) -> Dict:
    """RMSE (RGB, all pixels) of hybrid and plain IR renders against a dense
    plain-IR reference (the mean of `ref_renders` renders of m_ref VPLs
    each), mean over `seeds` seeds, with the render time (generation +
    gather, CUDA events) of each; also one hybrid render of bias_m VPLs,
    whose error is mostly the hybrid's bias against plain IR (light that
    reaches a close-range face after more than one bounce is carried only by
    far VPLs)."""
    import torch
    from . import vpl as V
    own = ctx is None
    ctx = ctx or V.Context(0)
    try:
        sid = ctx.upload(scene)
        cam, gat = view.camera, view.gather
        npx = cam.width * cam.height
        gb = V.GBuffer.empty(cam.width, cam.height)
        V.vpl_gbuffer_build(ctx.h, sid, cam, gb)

        def render_rs(m: int, seed: int):
            # rejection-sampled instant radiosity (no close range), pilot 32 x 32
            gen = dataclasses.replace(view.gen, m_close=0, m_far=m, seed=seed, d_close=0.0)
            vs = V.VplSet.empty(m)
            out = torch.zeros((npx, 4), dtype=torch.float32, device="cuda")
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            V.vpl_generate_rs(ctx.h, sid, cam, gen, 32, gat.d2_min, gat.ray_eps, vs)
            V.vpl_gather(ctx.h, sid, gb, vs, gat, out)
            e1.record()
            torch.cuda.synchronize()
            rc = V.vpl_sync(ctx.h, check=False)
            if rc != 0:
                raise RuntimeError(f"device status {rc} in rejection sampling, m={m}")
            return out, e0.elapsed_time(e1)

        def render(m_close: int, m_far: int, seed: int):
            # plain instant radiosity has no close range: d_close = 0 keeps every
            # light-path hit (with d_close > 0, m_close = 0 would still drop the
            # hits on close-range faces and give the hybrid's far part alone)
            d_close = view.gen.d_close if m_close > 0 else 0.0
            gen = dataclasses.replace(view.gen, m_close=m_close, m_far=m_far, seed=seed, d_close=d_close)
            vs = V.VplSet.empty(m_close + m_far)
            out = torch.zeros((npx, 4), dtype=torch.float32, device="cuda")
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            V.vpl_generate(ctx.h, sid, cam, gen, vs)
            V.vpl_gather(ctx.h, sid, gb, vs, gat, out)
            e1.record()
            torch.cuda.synchronize()
            rc = V.vpl_sync(ctx.h, check=False)
            if rc != 0:
                raise RuntimeError(f"device status {rc} at m_close={m_close} m_far={m_far}")
            return out, e0.elapsed_time(e1)

        ref, ref_ms = render(0, m_ref, 10_000)
        for k in range(1, ref_renders):
            ref = ref + render(0, m_ref, 10_000 + k)[0]
        ref = ref / ref_renders

        def curve(label: str, counts: Sequence[int], frac: float) -> List[Dict]:
            rows = []
            for m in counts:
                mc, mf = W.split_budget(m, frac)
                errs, times = [], []
                for s in range(seeds):
                    img, t = render_rs(m, 100 + s) if label == "rejection sampling" else render(mc, mf, 100 + s)
                    errs.append(_rmse(img, ref))
                    times.append(t)
                sd = statistics.pstdev(errs)
                rows.append({"method": label, "vpls": m, "m_close": mc, "m_far": mf,
                             "rmse": statistics.mean(errs), "rmse_sd": sd,
                             "rmse_se": sd / math.sqrt(max(1, len(errs) - 1)),
                             "rmse_median": statistics.median(errs), "errs": errs,
                             "ms": statistics.median(times)})
            return rows

        hyb = curve("hybrid", ms, alpha)
        ir = curve("instant radiosity", ir_ms, 0.0)
        rs = curve("rejection sampling", ms, 0.0)
        equal = equal_rmse(hyb, ir, seeds)
        ir_m = [r["vpls"] for r in ir]
        same_m = [{"vpls": r["vpls"], "rmse_hybrid": r["rmse"],
                   "rmse_ir": next(q["rmse"] for q in ir if q["vpls"] == r["vpls"]),
                   "rmse_rs": next(q["rmse"] for q in rs if q["vpls"] == r["vpls"])}
                  for r in hyb if r["vpls"] in ir_m]
        for row in same_m:
            row["ir_over_hybrid"] = row["rmse_ir"] / row["rmse_hybrid"]
        bias = None
        if bias_m:
            mc, mf = W.split_budget(bias_m, alpha)
            img, t = render(mc, mf, 99)
            bias = {"vpls": bias_m, "rmse": _rmse(img, ref), "ms": t,
                    "mean_ratio": float(img[:, :3].double().mean() / ref[:, :3].double().mean())}
        V.vpl_scene_release(ctx.h, sid)
        return {"reference": {"method": "instant radiosity", "vpls": m_ref * ref_renders, "ms_each": ref_ms,
                              "mean": float(ref[:, :3].double().mean())}, "hybrid_large": bias,
                "hybrid": hyb, "instant_radiosity": ir, "rejection_sampling": rs, "equal_vpls": same_m,
                "equal_rmse": equal,
                "pixels": npx, "seeds": seeds, "alpha": alpha}
    finally:
        if own:
            ctx.close()


def point_light_scene(scene: W.Scene) -> W.Scene:
    """The scene with its square light replaced by a point light of the same
    power at the square's centre (the light of the paper's experiments)."""
    L = scene.light
    return dataclasses.replace(scene, light=W.Light(center=L.center, normal=L.normal, edge_u=(0.0, 0.0, 0.0),
                                                    edge_v=(0.0, 0.0, 0.0), power=L.power, type=W.LIGHT_POINT))


def markdown(res: Dict, title: str) -> str:
    def cell(row):
        return f"{row['rmse']:.3g} +- {row['rmse_se']:.1g} (med {row['rmse_median']:.3g})"
    lines = [f"{title}: reference = instant radiosity with {res['reference']['vpls']} VPLs, "
             f"{res['pixels']} pixels, mean +- standard error over {res['seeds']} seeds (median)", "",
             "| VPLs | RMSE hybrid | RMSE instant radiosity | RMSE rejection sampling | IR / hybrid | ms hybrid / IR / RS |",
             "|---:|---:|---:|---:|---:|---:|"]
    by = {(r["method"], r["vpls"]): r for key in ("hybrid", "instant_radiosity", "rejection_sampling")
          for r in res[key]}
    for r in res["equal_vpls"]:
        m = r["vpls"]
        h, i, q = by[("hybrid", m)], by[("instant radiosity", m)], by[("rejection sampling", m)]
        lines.append(f"| {m} | {cell(h)} | {cell(i)} | {cell(q)} | {r['ir_over_hybrid']:.2f} | "
                     f"{h['ms']:.1f} / {i['ms']:.1f} / {q['ms']:.1f} |")
    lines += ["", "| hybrid VPLs | hybrid RMSE | IR VPLs for that RMSE | VPL ratio (90% CI) | time ratio |",
              "|---:|---:|---:|---:|---:|"]
    for r in res["equal_rmse"]:
        m = r["ir_vpls_for_equal_rmse"]
        lo, hi = r["vpl_ratio_90ci"]
        fmt = lambda v: "inf" if math.isinf(v) else f"{v:.2f}"
        lines.append(f"| {r['hybrid_vpls']} | {r['rmse']:.3g} | {'> range' if math.isinf(m) else f'{m:.0f}'} | "
                     f"{fmt(r['vpl_ratio'])} ({fmt(lo)} - {fmt(hi)}) | {fmt(r['time_ratio'])} |")
    b = res.get("hybrid_large")
    if b:
        lines += ["", f"Hybrid with {b['vpls']} VPLs: RMSE {b['rmse']:.3g}, mean {b['mean_ratio']:.3f} x the "
                      f"reference's (the hybrid's bias against plain IR)."]
    return "\n".join(lines)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--light", default="area", choices=["area", "point"])
    ap.add_argument("--width", type=int, default=256)
    ap.add_argument("--height", type=int, default=256)
    ap.add_argument("--m-ref", type=int, default=262144)
    ap.add_argument("--ref-renders", type=int, default=4)
    ap.add_argument("--alpha", type=float, default=0.75)
    ap.add_argument("--seeds", type=int, default=16)
    ap.add_argument("--view-seed", type=int, default=1)
    args = ap.parse_args()
    wl = W.room200k_workload(width=args.width, height=args.height, seed=args.view_seed)
    scene = wl.scene if args.light == "area" else point_light_scene(wl.scene)
    res = study(wl.views[0], scene, seeds=args.seeds, m_ref=args.m_ref, ref_renders=args.ref_renders,
                alpha=args.alpha)
    res["light"] = args.light
    print(json.dumps(res))
    print(markdown(res, f"room 200k, {args.light} light, {args.width}x{args.height}, alpha {args.alpha}"))


if __name__ == "__main__":
    main()
