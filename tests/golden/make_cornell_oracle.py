"""Writes cornell_oracle.json: the FP64 oracle's results on the 64-triangle
room (128 x 128, 256 VPLs, seed 0, brute-force visibility), a regression
record of the oracle itself.  It calls only `oracle/` and the input
generator; nothing here comes from the CUDA path.  Re-run it only with a
change to the oracle's arithmetic whose commit names the passage of the
paper (or the reading of it) that justifies the change.

    python tests/golden/make_cornell_oracle.py
"""
import json
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

PIXELS = [0, 1, 127, 128, 4095, 5000, 6000, 7000, 8000, 8191, 8192, 9000, 10000, 10500, 11000, 12000,
          12345, 13000, 14000, 15000, 15500, 16000, 16256, 16383, 2048, 3000, 3333, 4444, 5555, 6666, 7777, 8888]


def record() -> dict:
    import oracle
    from paper_2203_11484_gb300 import workloads as W
    oracle.build()
    wl = W.cornell_workload()
    view = wl.views[0]
    osc = oracle.OracleScene(wl.scene)
    close = osc.classify(view.camera, view.gen.d_close)
    g = osc.generate(view.camera, view.gen, vis_mode=1)
    r = oracle.render(osc, view, np.asarray(PIXELS))
    Mc = view.gen.m_close
    return {
        "workload": wl.name,
        "close_faces": [int(i) for i in np.flatnonzero(close)],
        "n_close": int(g["n_close"]), "shift_s": int(g["shift_s"]), "f_total": int(g["f_total"]),
        "paths": int(g["paths"]), "m_far_kept": int(g["m_far_kept"]), "a_rep": float(g["a_rep"]),
        "patch_tri": [int(t) for t in g["tri"][:Mc]],
        "far_tri": [int(t) for t in g["tri"][Mc:]],
        "far_tag": [int(t) for t in g["tag"][Mc:]],
        "vpl_pos_sum": [float(x) for x in g["pos"].sum(axis=0)],
        "vpl_flux_sum": [float(x) for x in g["flux"].sum(axis=0)],
        "vpl_pos_first": [float(x) for x in g["pos"][0]],
        "vpl_flux_first_far": [float(x) for x in g["flux"][Mc]],
        "pixels": PIXELS,
        "gbuffer_tri": [int(t) for t in r["gbuffer"]["tri"]],
        "image": [[float(x) for x in row[:3]] for row in r["image"]],
    }


if __name__ == "__main__":
    rec = record()
    with open(os.path.join(HERE, "cornell_oracle.json"), "w") as f:
        f.write("{\n" + ",\n".join(f"{json.dumps(k)}: {json.dumps(v)}" for k, v in rec.items()) + "\n}\n")
