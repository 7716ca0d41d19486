"""The oracle against its own stored results on the 64-triangle room
(tests/golden/cornell_oracle.json, written by
tests/golden/make_cornell_oracle.py from `oracle/` alone).  Not a pin
against the paper: it fixes the oracle so that any change to its arithmetic
shows up here and has to be justified by a passage of the paper.  CPU only.
Integers (close set, quantised areas, patch assignment, path tags) exact;
floating point to 1e-9 relative (libm may differ by an ulp between hosts)."""
import json
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.join(HERE, "golden"))


def test_oracle_reproduces_stored_cornell_results(orc):
    import make_cornell_oracle as G
    with open(os.path.join(HERE, "golden", "cornell_oracle.json")) as f:
        want = json.load(f)
    got = G.record()
    for k in ("workload", "close_faces", "n_close", "shift_s", "f_total", "paths", "m_far_kept", "patch_tri",
              "far_tri", "far_tag", "pixels", "gbuffer_tri"):
        assert got[k] == want[k], k
    for k in ("a_rep", "vpl_pos_sum", "vpl_flux_sum", "vpl_pos_first", "vpl_flux_first_far", "image"):
        assert np.allclose(got[k], want[k], rtol=1e-9, atol=1e-15), k
