"""Capped steepest descent with the oracle's forces (oracle/relax.py), the relaxed start
of the NVE control run, pinned on a small box (no GPU): each step moves every atom along
its force as given by the whole-system oracle routine, the atom under the largest force
by exactly the cap; the potential energy falls; the worker split does not change the
result."""
import numpy as np

import oracle
from oracle import relax
from paper_1611_04474_gb300 import workloads as W


def _system():
    return W.small_random(90, (11.0, 12.0, 13.0), rc=3.5, seed=21, min_dist=0.6)


def test_each_step_moves_along_the_force_by_the_cap():
    s = _system()
    ff = oracle.ForceField.from_system(s)
    x = s.pos.astype(np.float64)
    for _ in range(3):
        F = oracle.forces_cells(x, s.q, s.type, s.box, ff).F
        y = relax.steepest_descent(x, s.q, s.type, s.box, ff, n_steps=1, max_step=0.01,
                                   workers=2, cache=False)
        d = y - x
        d -= s.box * np.round(d / s.box)
        step = np.linalg.norm(d, axis=1)
        assert abs(step.max() - 0.01) <= 1e-12
        # parallel to the force, with the length of 0.01 |F_i| / max |F|
        fn = np.linalg.norm(F, axis=1)
        np.testing.assert_allclose(d, 0.01 * F / fn.max(), rtol=0, atol=1e-12)
        x = y


def test_energy_falls_and_workers_agree():
    s = _system()
    ff = oracle.ForceField.from_system(s)
    x0 = s.pos.astype(np.float64)
    e = lambda x: oracle.forces_cells(x, s.q, s.type, s.box, ff).energy[:2].sum()  # noqa: E731
    a = relax.steepest_descent(x0, s.q, s.type, s.box, ff, n_steps=30, workers=1, cache=False)
    b = relax.steepest_descent(x0, s.q, s.type, s.box, ff, n_steps=30, workers=3, cache=False)
    np.testing.assert_array_equal(a, b)
    assert e(a) < e(x0)
    assert np.all((a >= 0) & (a < s.box))
