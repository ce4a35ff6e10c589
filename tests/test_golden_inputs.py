"""The three-mode workload's optical operators against the coefficients the paper prints in its
Tables I and II (tests/golden/water_optics_tables_I_II.txt)."""
import os

import numpy as np

from paper_2509_25840_b300 import inputs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "water_optics_tables_I_II.txt")


def _table():
    rows = []
    for line in open(GOLDEN):
        line = line.split("#")[0].split()
        if line:
            kind, s, s2, v = line
            rows.append((kind, int(s) - 3, None if s2 == "-" else int(s2) - 3, float(v)))
    return rows


def test_three_mode_optics_follow_tables_I_II():
    mu, Pi = inputs.three_mode_optics()
    ops = {"mu": mu, "mu_ss": mu, "Pi": Pi, "Pi_ss": Pi}
    rows = _table()
    assert len(rows) == 18
    for kind, s, s2, v in rows:
        op = ops[kind]
        if s2 is None:
            assert op.lin[s] == v, (kind, s)
        else:
            q = np.asarray(op.quad)
            assert q[s, s2] == v and q[s2, s] == v, (kind, s, s2)
