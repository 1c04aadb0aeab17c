"""The seeded input generators: shapes, determinism and the stated recipes."""
import numpy as np

from paper_1611_04474_gb300 import workloads as W


def test_random_gas_recipe():
    s = W.workload_random_3000()
    assert s.n == 3000 and s.ntypes == 4
    assert s.pos.dtype == np.float32 and s.q.dtype == np.float32 and s.type.dtype == np.int32
    assert np.all(s.pos >= 0) and np.all(s.pos.astype(np.float64) < s.box[None, :])
    assert float(s.q.astype(np.float64).sum()) == 0.0
    assert set(np.unique(s.q).tolist()) <= {-0.8, -0.4, 0.4, 0.8} | {np.float32(v) for v in (-0.8, -0.4, 0.4, 0.8)}
    assert np.all((s.sigma >= 2.5) & (s.sigma <= 3.8)) and np.all((s.eps >= 0.05) & (s.eps <= 0.2))
    assert np.all((s.mass >= 1) & (s.mass <= 16))
    from scipy.spatial import cKDTree
    assert len(cKDTree(s.pos.astype(np.float64), boxsize=s.box).query_pairs(1.0)) == 0
    s2 = W.workload_random_3000()
    assert np.array_equal(s.pos, s2.pos) and np.array_equal(s.q, s2.q)
    # velocities: zero centre-of-mass momentum
    p = (s.mass.astype(np.float64)[:, None] * s.vel).sum(axis=0)
    assert np.abs(p).max() < 1e-12


def test_lattice_recipe_apoa1_box():
    s = W.workload_lattice_92k()
    assert s.n == 92224 and s.ntypes == 8
    assert np.allclose(s.box, (108.86, 108.86, 77.76))
    assert abs(s.n / np.prod(s.box) - 0.10008) < 1e-4
    assert np.all(s.pos >= 0) and np.all(s.pos.astype(np.float64) < s.box[None, :])
    assert abs(float(s.q.astype(np.float64).sum())) < 1e-2


def test_sweep_sizes_keep_density():
    for n in W.sweep_sizes()[:2]:
        s = W.lattice_box(n=n)
        assert s.n == n
        assert abs(n / np.prod(s.box) - 0.10008) < 2e-4


def test_lj_table_convention():
    sigma = np.array([1.0, 2.0])
    eps = np.array([0.25, 1.0])
    AB = W.lj_table(sigma, eps).astype(np.float64)
    # Lorentz-Berthelot: sigma_01 = 1.5, eps_01 = 0.5
    np.testing.assert_allclose(AB[0, 1], [48 * 0.5 * 1.5**12, 24 * 0.5 * 1.5**6], rtol=1e-7)
    np.testing.assert_array_equal(AB[0, 1], AB[1, 0])
