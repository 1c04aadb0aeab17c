"""Pins of the FP64 oracle to things other than itself (no GPU).

The paper prints no force or energy value, so the oracle is pinned by
  * closed forms: the two-atom LJ force against the derivative of the textbook
    12-6 potential (taken symbolically with sympy), the zero of the LJ force at
    r = 2^(1/6) sigma, Coulomb's law;
  * scipy's periodic k-d tree: partner counts per atom under the cutoff;
  * symmetry: a perfect periodic lattice feels no net force, and every atom of
    a simple cubic lattice has the number of partners given by counting integer
    vectors;
  * invariants: Newton's third law, translation and permutation invariance,
    linearity in the charges and in epsilon;
  * the two independent oracle routines (Algorithm 1 cell list, brute force) on
    boxes with 1, 2, 3 and 4 cells per axis.
Each pin is chosen so that a plausible slip (a wrong exponent, sign, index,
missing minimum image, non-strict cutoff, a duplicated neighbour cell) fails it.
"""
import math

import numpy as np
import pytest

import oracle
from paper_1611_04474_gb300 import workloads as W


def _ff_two_types(sigma, eps, k=W.K_COULOMB, rc=12.0):
    sigma = np.asarray(sigma, dtype=np.float64)
    eps = np.asarray(eps, dtype=np.float64)
    s = 0.5 * (sigma[:, None] + sigma[None, :])
    e = np.sqrt(eps[:, None] * eps[None, :])
    # the 12-6 convention of the reading: A = 48 eps sigma^12, B = 24 eps sigma^6
    return oracle.ForceField(48 * e * s**12, 24 * e * s**6, k, rc)


def _pair_force(r, sigma=3.0, eps=0.2, q=(0.0, 0.0), rc=12.0, axis=(1.0, 0.0, 0.0)):
    ff = _ff_two_types([sigma], [eps], rc=rc)
    box = np.array([100.0, 100.0, 100.0])
    u = np.asarray(axis, dtype=np.float64)
    u = u / np.linalg.norm(u)
    xi = np.array([50.0, 50.0, 50.0]) + 0.5 * r * u
    xj = np.array([50.0, 50.0, 50.0]) - 0.5 * r * u
    F, U = oracle.pair(xi, xj, box, q[0], q[1], ff.A[0, 0], ff.B[0, 0], ff.k, rc)
    return F, U, u


def test_lj_force_is_textbook_derivative():
    sympy = pytest.importorskip("sympy")
    r_, s_, e_ = sympy.symbols("r sigma epsilon", positive=True)
    U = 4 * e_ * ((s_ / r_) ** 12 - (s_ / r_) ** 6)
    dUdr = sympy.diff(U, r_)
    sigma, eps = 3.1, 0.17
    for r in (2.5, 2.9, 3.3, 3.48, 4.0, 6.0, 9.5, 11.9):
        F, Upair, u = _pair_force(r, sigma, eps)
        expect = -float(dUdr.subs({r_: r, s_: sigma, e_: eps}))  # radial force on i along +u
        got = float(F @ u)
        assert abs(got - expect) <= 1e-12 * max(abs(expect), 1e-30) + 1e-14, (r, got, expect)
        # no tangential part
        assert np.linalg.norm(F - got * u) <= 1e-12 * abs(got) + 1e-15
        u_expect = float(U.subs({r_: r, s_: sigma, e_: eps}))
        assert abs(Upair[0] - u_expect) <= 1e-12 * abs(u_expect) + 1e-15


def test_lj_force_vanishes_at_minimum_and_signs():
    sigma, eps = 3.4, 0.1
    rmin = 2 ** (1 / 6) * sigma
    F, _, u = _pair_force(rmin, sigma, eps)
    scale = 48 * eps * sigma**12 / rmin**13
    assert abs(F @ u) <= 1e-12 * scale
    Fin, _, u = _pair_force(0.95 * rmin, sigma, eps)
    Fout, _, u = _pair_force(1.05 * rmin, sigma, eps)
    assert Fin @ u > 0  # repulsive: pushes i away from j
    assert Fout @ u < 0  # attractive


def test_coulomb_closed_form():
    for qi, qj in ((0.8, 0.4), (-0.8, 0.4), (-0.4, -0.4)):
        for r in (1.0, 3.7, 11.0):
            F, U, u = _pair_force(r, sigma=1.0, eps=0.0, q=(qi, qj), axis=(1.0, 2.0, -0.5))
            expect = W.K_COULOMB * qi * qj / r**2
            assert abs(F @ u - expect) <= 1e-12 * abs(expect)
            assert abs(U[1] - W.K_COULOMB * qi * qj / r) <= 1e-12 * abs(U[1])
            if qi * qj > 0:
                assert F @ u > 0  # like charges repel


def test_force_is_minus_energy_gradient():
    sigma, eps, q = 2.9, 0.13, (0.6, -0.3)
    for r in (2.4, 3.2, 5.0, 10.0):
        F, _, u = _pair_force(r, sigma, eps, q=q)
        h = 1e-6 * r
        _, Up, _ = _pair_force(r + h, sigma, eps, q=q)
        _, Um, _ = _pair_force(r - h, sigma, eps, q=q)
        dUdr = (Up.sum() - Um.sum()) / (2 * h)
        assert abs(F @ u + dUdr) <= 1e-6 * max(abs(dUdr), 1e-3)


def test_cutoff_is_strict():
    rc = 12.0
    F, _, _ = _pair_force(rc * (1 - 1e-6), sigma=3.0, eps=0.2, q=(0.5, 0.5), rc=rc)
    assert np.linalg.norm(F) > 0
    F, _, _ = _pair_force(rc * (1 + 1e-6), sigma=3.0, eps=0.2, q=(0.5, 0.5), rc=rc)
    assert np.linalg.norm(F) == 0
    ff = _ff_two_types([3.0], [0.2], rc=rc)
    box = np.array([100.0, 100.0, 100.0])
    for d in ((12.0, 0.0, 0.0), (8.0, 8.0, 4.0), (0.0, 4.0, 11.313708498984761)):
        xi = np.array([40.0, 40.0, 40.0])
        xj = xi + np.asarray(d)
        r2 = float(np.sum((xi - xj) ** 2))
        F, _ = oracle.pair(xi, xj, box, 0.5, 0.5, ff.A[0, 0], ff.B[0, 0], ff.k, rc)
        if r2 == rc * rc:
            assert np.linalg.norm(F) == 0, d
        else:
            assert (np.linalg.norm(F) > 0) == (r2 < rc * rc), d


def test_minimum_image_across_the_boundary():
    ff = _ff_two_types([3.0], [0.2], rc=10.0)
    box = np.array([30.0, 25.0, 40.0])
    xi = np.array([0.4, 24.0, 39.7])
    xj = np.array([29.1, 0.5, 0.9])  # across the x, y and z faces: d = (1.3, -1.5, -1.2)
    F1, _ = oracle.pair(xi, xj, box, 0.4, -0.8, ff.A[0, 0], ff.B[0, 0], ff.k, ff.rc)
    # the same pair moved to the middle of the box: image of xj next to xi
    shift = np.array([10.0, -12.0, -20.0])
    xj_img = xj + np.array([-30.0, 25.0, 40.0])
    F2, _ = oracle.pair(xi + shift, xj_img + shift, box, 0.4, -0.8, ff.A[0, 0], ff.B[0, 0],
                        ff.k, ff.rc)
    assert np.linalg.norm(F1) > 0
    np.testing.assert_allclose(F1, F2, rtol=1e-10)


BOXES = [
    # (n, box, rc): 1, 2, 3, 4 cells per axis and anisotropic mixes
    (60, (9.0, 9.0, 9.0), 4.4),       # 2x2x2
    (50, (7.0, 7.5, 8.0), 3.4),       # 2x2x2, anisotropic
    (80, (9.5, 13.0, 18.5), 3.0),     # 3x4x6
    (40, (6.5, 12.0, 6.6), 3.2),      # 2x3x2
    (120, (16.0, 16.0, 16.0), 4.0),   # 4x4x4
    (30, (7.0, 9.0, 10.0), 3.4),      # 2x2x2
    (70, (6.9, 20.0, 9.3), 3.4),      # 2x5x2
    (45, (7.2, 7.2, 14.9), 3.55),     # 2x2x4
]


@pytest.mark.parametrize("n,box,rc", BOXES)
def test_cell_list_equals_brute_force(n, box, rc):
    s = W.small_random(n, box, rc=rc, seed=n)
    ff = oracle.ForceField.from_system(s)
    p = s.pos.astype(np.float64)
    a = oracle.forces_cells(p, s.q, s.type, s.box, ff)
    b = oracle.forces_brute(p, s.q, s.type, s.box, ff)
    assert a.npairs == b.npairs and a.npairs > 0
    scale = np.abs(b.F).max()
    np.testing.assert_allclose(a.F, b.F, rtol=0, atol=1e-12 * scale)
    np.testing.assert_allclose(a.energy, b.energy, rtol=1e-12, atol=1e-12 * np.abs(b.energy).max())


def test_two_cells_per_axis_boxes():
    # rc just under L/2: two cells per axis, both stencil offsets name the same cell
    s = W.small_random(40, (7.0, 7.0, 7.0), rc=3.45, seed=5)
    ff = oracle.ForceField.from_system(s)
    assert list(oracle.cell_dims(s.box, s.rc)) == [2, 2, 2]
    s1 = W.small_random(40, (5.0, 6.0, 6.5), rc=2.45, seed=6)
    ff1 = oracle.ForceField.from_system(s1)
    assert list(oracle.cell_dims(s1.box, s1.rc)) == [2, 2, 2]
    s2 = W.small_random(30, (5.0, 5.0, 5.0), rc=2.4, seed=7)
    ff2 = oracle.ForceField.from_system(s2)
    for sys_, f_ in ((s, ff), (s1, ff1), (s2, ff2)):
        p = sys_.pos.astype(np.float64)
        a = oracle.forces_cells(p, sys_.q, sys_.type, sys_.box, f_)
        b = oracle.forces_brute(p, sys_.q, sys_.type, sys_.box, f_)
        assert a.npairs == b.npairs
        np.testing.assert_allclose(a.F, b.F, rtol=0, atol=1e-12 * np.abs(b.F).max())
    # a box with a single cell on one axis: L < 2 rc is rejected by the library, but
    # the oracle's rule floor(L/rc) = 1 still yields all-pairs on that axis
    dims = oracle.cell_dims((5.0, 12.0, 12.0), 3.0)
    assert list(dims) == [1, 4, 4]


@pytest.mark.parametrize("seed", [0, 1])
def test_partner_counts_match_periodic_kdtree(seed):
    from scipy.spatial import cKDTree

    s = W.lattice_box(n=3000, seed=seed, ntypes=4)
    ff = oracle.ForceField.from_system(s)
    p = s.pos.astype(np.float64)
    _, _, npart = oracle.forces_atoms(p, s.q, s.type, s.box, ff, np.arange(s.n))
    tree = cKDTree(p, boxsize=s.box)
    # strict cutoff: shrink the radius by far less than any pair's distance from it
    rq = s.rc * (1 - 1e-12)
    counts = np.array([len(x) - 1 for x in tree.query_ball_point(p, rq)])
    bij, _ = oracle.boundary_pairs(p, s.box, s.rc, 1e-9)
    assert bij.shape[0] == 0
    np.testing.assert_array_equal(npart, counts)
    full = oracle.forces_cells(p, s.q, s.type, s.box, ff)
    assert full.npairs == counts.sum() // 2


def test_simple_cubic_lattice_counts_and_zero_force():
    # 8x8x8 sites, spacing 1.25 A, all atoms identical and equally charged:
    # every atom has the same partners (integer vectors v != 0 with |v|^2 a^2 < rc^2),
    # and by symmetry the net force on each atom is zero.
    m, a, rc = 8, 1.25, 3.9
    g = np.stack(np.meshgrid(*[np.arange(m)] * 3, indexing="ij"), -1).reshape(-1, 3)
    pos = (g + 0.5) * a
    box = np.full(3, m * a)
    ff = _ff_two_types([1.1], [0.3], rc=rc)
    q = np.full(pos.shape[0], 0.3)
    t = np.zeros(pos.shape[0], np.int32)
    res = oracle.forces_cells(pos, q, t, box, ff)
    lim = int(math.ceil(rc / a))
    expect = sum(1 for x in range(-lim, lim + 1) for y in range(-lim, lim + 1)
                 for z in range(-lim, lim + 1) if 0 < (x * x + y * y + z * z) * a * a < rc * rc)
    assert res.npairs == pos.shape[0] * expect // 2
    assert np.abs(res.F).max() <= 1e-10 * res.cond.max()


def test_lattice_pairs_exactly_at_the_cutoff_are_excluded():
    # spacing 1.5 and rc = 3.0 are exact in binary: the second-neighbour pairs
    # along the axes sit at r^2 == rc^2 exactly and must not count (strict <)
    m, a, rc = 6, 1.5, 3.0
    g = np.stack(np.meshgrid(*[np.arange(m)] * 3, indexing="ij"), -1).reshape(-1, 3)
    pos = (g + 0.5) * a
    box = np.full(3, m * a)
    ff = _ff_two_types([1.0], [0.2], rc=rc)
    q = np.zeros(pos.shape[0])
    t = np.zeros(pos.shape[0], np.int32)
    expect = sum(1 for x in range(-2, 3) for y in range(-2, 3) for z in range(-2, 3)
                 if 0 < (x * x + y * y + z * z) < 4)
    assert expect == 26
    for fn in (oracle.forces_cells, oracle.forces_brute):
        res = fn(pos, q, t, box, ff)
        assert res.npairs == pos.shape[0] * expect // 2, fn.__name__


def test_newton_third_law_translation_permutation():
    s = W.small_random(150, (14.0, 15.0, 16.0), rc=4.5, seed=11)
    ff = oracle.ForceField.from_system(s)
    p = s.pos.astype(np.float64)
    base = oracle.forces_cells(p, s.q, s.type, s.box, ff)
    tot = np.abs(base.F).sum()
    assert np.abs(base.F.sum(axis=0)).max() <= 1e-12 * tot
    shift = np.array([3.7, -11.2, 25.9])
    moved = np.mod(p + shift, s.box)
    res = oracle.forces_cells(moved, s.q, s.type, s.box, ff)
    np.testing.assert_allclose(res.F, base.F, rtol=0, atol=1e-9 * np.abs(base.F).max())
    perm = np.random.default_rng(3).permutation(s.n)
    res = oracle.forces_cells(p[perm], s.q[perm], s.type[perm], s.box, ff)
    np.testing.assert_allclose(res.F, base.F[perm], rtol=0, atol=1e-12 * np.abs(base.F).max())
    assert res.npairs == base.npairs


def test_linear_in_charge_squared_and_epsilon():
    s = W.small_random(100, (12.0, 12.0, 12.0), rc=4.0, seed=4)
    p = s.pos.astype(np.float64)
    ff = oracle.ForceField.from_system(s)
    lj_only = oracle.forces_cells(p, 0 * s.q, s.type, s.box, ff).F
    full = oracle.forces_cells(p, s.q, s.type, s.box, ff).F
    twice = oracle.forces_cells(p, 2.0 * s.q.astype(np.float64), s.type, s.box, ff).F
    sc = np.abs(full).max()
    np.testing.assert_allclose(twice, lj_only + 4.0 * (full - lj_only), rtol=0, atol=1e-10 * sc)
    ff3 = oracle.ForceField(3.0 * ff.A, 3.0 * ff.B, ff.k, ff.rc)
    tripled = oracle.forces_cells(p, 0 * s.q, s.type, s.box, ff3).F
    np.testing.assert_allclose(tripled, 3.0 * lj_only, rtol=0, atol=1e-10 * np.abs(lj_only).max())


def test_cells_are_well_formed():
    s = W.lattice_box(n=2000, seed=9, ntypes=2)
    dims, cell_of, cell_start, order = oracle.build_cells(s.pos.astype(np.float64), s.box, s.rc)
    ncell = int(np.prod(dims))
    assert cell_start[0] == 0 and cell_start[-1] == s.n
    assert np.all(np.diff(cell_start) >= 0)
    assert np.array_equal(np.sort(order), np.arange(s.n))
    edge = s.box / dims
    p = s.pos.astype(np.float64)
    for c in range(ncell):
        members = order[cell_start[c]:cell_start[c + 1]]
        assert np.all(np.diff(members) > 0)  # ascending input order within a cell
        assert np.all(cell_of[members] == c)
        cx, cy, cz = c % dims[0], (c // dims[0]) % dims[1], c // (dims[0] * dims[1])
        lo = np.array([cx, cy, cz]) * edge
        assert np.all(p[members] >= lo - 1e-9) and np.all(p[members] < lo + edge + 1e-9)


def _bound_pair(dt, n_steps, r0_factor=1.06):
    sigma, eps = 2.0, 0.5
    ff = _ff_two_types([sigma], [eps], rc=6.0)
    box = np.array([20.0, 20.0, 20.0])
    r0 = 2 ** (1 / 6) * sigma * r0_factor
    pos = np.array([[10.0 + r0 / 2, 10.0, 10.0], [10.0 - r0 / 2, 10.0, 10.0]])
    vel = np.array([[0.0, 0.002, 0.0], [0.0, -0.002, 0.0]])
    inv_m = np.array([1 / 12.0, 1 / 12.0])
    q = np.zeros(2)
    t = np.zeros(2, np.int32)
    return oracle.vv_steps(pos, vel, q, t, box, ff, inv_m, dt, n_steps, f32_positions=False), inv_m


def test_velocity_verlet_energy_error_is_second_order():
    T = 400.0  # fs, several oscillations of the bound pair
    amps = []
    for dt in (2.0, 1.0):
        (pos, vel, F, log), inv_m = _bound_pair(dt, int(T / dt))
        e = log[:, 0] + log[:, 1] + log[:, 2]
        amps.append(e.max() - e.min())
    ratio = amps[0] / amps[1]
    assert 3.0 < ratio < 5.0, amps


def test_velocity_verlet_time_reversible():
    (pos, vel, F, log), inv_m = _bound_pair(1.0, 200)
    sigma, eps = 2.0, 0.5
    ff = _ff_two_types([sigma], [eps], rc=6.0)
    back = oracle.vv_steps(pos, -vel, np.zeros(2), np.zeros(2, np.int32), np.full(3, 20.0), ff,
                           inv_m, 1.0, 200, F=F, f32_positions=False)
    r0 = 2 ** (1 / 6) * sigma * 1.06
    start = np.array([[10.0 + r0 / 2, 10.0, 10.0], [10.0 - r0 / 2, 10.0, 10.0]])
    np.testing.assert_allclose(back[0], start, rtol=0, atol=1e-9)
