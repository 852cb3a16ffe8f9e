"""The oracle reproduces its stored fixture (a regression guard: the values were
written by tests/golden/make_golden.py, which calls only the oracle; the oracle's
correctness itself is pinned by closed forms in test_oracle_pins.py)."""
import os
import sys

import numpy as np

sys.path.insert(0, os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden"))

import make_golden  # noqa: E402


def test_oracle_reproduces_golden():
    data = np.loadtxt(make_golden.PATH)
    r = make_golden.compute()
    assert np.array_equal(data[:, 0].astype(np.int64), r["idx"])
    for col, k in ((1, "sl"), (2, "dl"), (3, "adl")):
        ref = data[:, col]
        assert np.abs(r[k] - ref).max() <= 1e-13 * np.abs(ref).max(), k
