"""The oracle still reproduces its committed regression fixture (see tests/golden)."""
import os

import numpy as np

from tests.golden.make_oracle_fixture import compute

HERE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "oracle_small.txt")


def test_oracle_matches_committed_fixture():
    rows = [ln.split() for ln in open(HERE) if ln.strip() and not ln.startswith("#")]
    npairs = int(rows[0][1])
    energy = np.array([float(v) for v in rows[1][1:]])
    F = np.array([[float(v) for v in r[1:]] for r in rows[2:]])
    s, res = compute()
    assert res.npairs == npairs
    np.testing.assert_allclose(res.energy, energy, rtol=1e-13)
    np.testing.assert_allclose(res.F, F, rtol=0, atol=1e-13 * np.abs(F).max())
