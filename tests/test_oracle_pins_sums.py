"""Pins of the oracle routines that the large-system checks rely on (no GPU).

The full-size GPU checks compare against three oracle outputs besides the
whole-system forces:
  * ``forces_atoms``: the forces on chosen atoms of a large system (Algorithm 1's
    neighbour cells of the atom's own cell only), the checker of every sampled
    comparison;
  * ``boundary_pairs``: the pairs whose FP64 r^2 lies within a window of rc^2,
    which decide where an FP32 filter may legitimately differ;
  * the term-size sums ``cond``, ``fabs_sum`` and ``energy_abs``: the denominators
    of the 1e-5 force criterion and of the energy tolerances.
Each is pinned here to something other than the oracle itself: an all-pairs numpy
enumeration written from the definitions of Eq. 1-2 (no cell list, no loop order),
closed forms of a lone pair, and the pinned whole-system routine.  The pins are
chosen so that a flipped sign, a narrowed window or a dropped term fails one.
"""
import math

import numpy as np
import pytest

import oracle
from paper_1611_04474_gb300 import workloads as W

from tests.test_oracle_pins import BOXES, _ff_two_types


def _all_pairs(pos, q, types, box, ff):
    """Every ordered pair i != j by minimum image, straight from Eq. 1-2.

    Returns per-atom force, term-size sum (cond), sum of |F_ij| and partner count,
    plus the sums over unordered pairs of |U_LJ| parts, |U_C| and cond_ij * r."""
    p = np.asarray(pos, np.float64)
    L = np.asarray(box, np.float64)
    d = p[:, None, :] - p[None, :, :]
    d = d - L * np.floor(d / L + 0.5)
    r2 = np.einsum("ijk,ijk->ij", d, d)
    n = p.shape[0]
    keep = (r2 < ff.rc * ff.rc) & ~np.eye(n, dtype=bool)
    r2s = np.where(keep, r2, 1.0)
    r = np.sqrt(r2s)
    A = ff.A[types[:, None], types[None, :]]
    B = ff.B[types[:, None], types[None, :]]
    kqq = ff.k * np.asarray(q, np.float64)[:, None] * np.asarray(q, np.float64)[None, :]
    f = A / r**14 - B / r**8 + kqq / r**3  # F_ij = f d_ij (Eq. 1 + Eq. 2)
    f = np.where(keep, f, 0.0)
    size = np.where(keep, (np.abs(A) / r**14 + np.abs(B) / r**8 + np.abs(kqq) / r**3) * r, 0.0)
    F = np.einsum("ij,ijk->ik", f, d)
    cond = size.sum(axis=1)
    fabs = (np.abs(f) * np.where(keep, r, 0.0)).sum(axis=1)
    npart = keep.sum(axis=1)
    upper = np.triu(keep, 1)
    u_lj_abs = np.where(upper, np.abs(A) / 12.0 / r**12 + np.abs(B) / 6.0 / r**6, 0.0).sum()
    u_c_abs = np.where(upper, np.abs(kqq) / r, 0.0).sum()
    w_abs = np.where(upper, size * r, 0.0).sum()
    return F, cond, fabs, npart, np.array([u_lj_abs, u_c_abs, w_abs])


def _close_rows(a, b, scale, rel=1e-12):
    """|a - b| <= rel * scale per row (scale: one size per row)."""
    err = np.abs(np.asarray(a) - np.asarray(b)).max(axis=1)
    bad = np.nonzero(err > rel * np.asarray(scale))[0]
    assert bad.size == 0, (bad[:5], err[bad[:5]], np.asarray(scale)[bad[:5]])


def _systems():
    for n, box, rc in BOXES:
        yield W.small_random(n, box, rc=rc, seed=n)
    yield W.small_random(60, (14.0, 13.0, 15.0), rc=4.5, seed=60)


@pytest.mark.parametrize("idx", range(len(BOXES) + 1))
def test_term_size_sums_against_all_pairs(idx):
    s = list(_systems())[idx]
    ff = oracle.ForceField.from_system(s)
    p = s.pos.astype(np.float64)
    res = oracle.forces_cells(p, s.q, s.type, s.box, ff)
    F, cond, fabs, npart, eabs = _all_pairs(p, s.q, s.type, s.box, ff)
    assert npart.sum() == 2 * res.npairs and res.npairs > 0
    np.testing.assert_allclose(res.F, F, rtol=0, atol=1e-12 * cond.max())
    np.testing.assert_allclose(res.cond, cond, rtol=1e-12, atol=0)
    np.testing.assert_allclose(res.fabs_sum, fabs, rtol=1e-12, atol=0)
    np.testing.assert_allclose(res.energy_abs, eabs, rtol=1e-12, atol=0)
    # the three sizes of a sum bound the sum: |F_i| <= sum |F_ij| <= cond_i
    nF = np.linalg.norm(res.F, axis=1)
    assert np.all(nF <= res.fabs_sum * (1 + 1e-12) + 1e-300)
    assert np.all(res.fabs_sum <= res.cond * (1 + 1e-12) + 1e-300)
    # and every energy is bounded by its absolute counterpart
    assert abs(res.energy[0]) <= res.energy_abs[0] * (1 + 1e-12)
    assert abs(res.energy[1]) <= res.energy_abs[1] * (1 + 1e-12)
    assert abs(res.energy[2]) <= res.energy_abs[2] * (1 + 1e-12)


def test_term_sizes_of_a_lone_pair_closed_form():
    # at the LJ minimum r = 2^(1/6) sigma the two LJ terms are equal, so with q = 0
    # cond = 2 B r^-7 = 2 * 24 eps sigma^6 r^-7 while the force is zero
    sigma, eps = 3.2, 0.15
    ff = _ff_two_types([sigma], [eps], rc=9.0)
    box = np.array([30.0, 30.0, 30.0])
    rmin = 2 ** (1 / 6) * sigma
    pos = np.array([[10.0, 10.0, 10.0], [10.0 + rmin, 10.0, 10.0]])
    t = np.zeros(2, np.int32)
    res = oracle.forces_cells(pos, np.zeros(2), t, box, ff)
    expect = 2 * 24 * eps * sigma**6 / rmin**7
    np.testing.assert_allclose(res.cond, [expect, expect], rtol=1e-12)
    assert np.abs(res.F).max() <= 1e-12 * expect
    # LJ and Coulomb sizes add: charges +0.5 / -0.7 at r = 4.1 with eps = 0
    ff0 = _ff_two_types([sigma], [0.0], rc=9.0)
    r = 4.1
    pos = np.array([[10.0, 10.0, 10.0], [10.0, 10.0 + r, 10.0]])
    res = oracle.forces_cells(pos, np.array([0.5, -0.7]), t, box, ff0)
    kq = W.K_COULOMB * 0.35
    np.testing.assert_allclose(res.cond, [kq / r**2] * 2, rtol=1e-12)
    np.testing.assert_allclose(res.fabs_sum, [kq / r**2] * 2, rtol=1e-12)
    np.testing.assert_allclose(res.energy_abs, [0.0, kq / r, kq / r], rtol=1e-12)
    # both: sizes of the LJ terms plus |k q q| r^-2
    res = oracle.forces_cells(pos, np.array([0.5, -0.7]), t, box, ff)
    A, B = ff.A[0, 0], ff.B[0, 0]
    np.testing.assert_allclose(res.cond, [A / r**13 + B / r**7 + kq / r**2] * 2, rtol=1e-12)
    fr = A / r**13 - B / r**7 - kq / r**2
    np.testing.assert_allclose(res.fabs_sum, [abs(fr)] * 2, rtol=1e-12)
    np.testing.assert_allclose(res.energy_abs,
                               [A / 12 / r**12 + B / 6 / r**6, kq / r,
                                (A / r**13 + B / r**7 + kq / r**2) * r], rtol=1e-12)


@pytest.mark.parametrize("idx", range(len(BOXES) + 1))
def test_forces_atoms_equals_whole_system(idx):
    s = list(_systems())[idx]
    ff = oracle.ForceField.from_system(s)
    p = s.pos.astype(np.float64)
    full = oracle.forces_cells(p, s.q, s.type, s.box, ff)
    F, cond, fabs, npart, _ = _all_pairs(p, s.q, s.type, s.box, ff)
    rng = np.random.default_rng(idx)
    for sel in (np.arange(s.n), rng.choice(s.n, size=max(1, s.n // 3), replace=False)):
        Fs, cs, ns = oracle.forces_atoms(p, s.q, s.type, s.box, ff, sel)
        _close_rows(Fs, full.F[sel], full.cond[sel])
        _close_rows(Fs, F[sel], cond[sel])
        np.testing.assert_allclose(cs, cond[sel], rtol=1e-12, atol=0)
        np.testing.assert_array_equal(ns, npart[sel])


def test_forces_atoms_equals_whole_system_on_a_lattice():
    s = W.lattice_box(n=3000, seed=3, ntypes=4)
    ff = oracle.ForceField.from_system(s)
    p = s.pos.astype(np.float64)
    full = oracle.forces_cells(p, s.q, s.type, s.box, ff)
    rng = np.random.default_rng(7)
    sel = np.concatenate([np.arange(s.n), rng.choice(s.n, size=400, replace=False)])
    Fs, cs, ns = oracle.forces_atoms(p, s.q, s.type, s.box, ff, sel)
    _close_rows(Fs, full.F[sel], full.cond[sel])
    np.testing.assert_allclose(cs, full.cond[sel], rtol=1e-12, atol=0)
    assert ns[: s.n].sum() == 2 * full.npairs
    # a selection in any order, with repeats, gives the same rows
    perm = rng.permutation(sel.shape[0])
    Fp, _, _ = oracle.forces_atoms(p, s.q, s.type, s.box, ff, sel[perm])
    np.testing.assert_array_equal(Fp, Fs[perm])


def _boundary_system(window):
    """A random background plus planted pairs at r^2 = rc^2 + delta, some across faces."""
    box = np.array([20.0, 21.0, 22.0])
    rc = 6.0
    rng = np.random.default_rng(17)
    bg = rng.uniform(0, 1, (60, 3)) * box
    deltas = np.array([-1.6, -0.95, -0.7, -0.55, -0.2, 0.0, 0.15, 0.6, 0.8, 0.97, 1.4, 2.5]) * window
    planted = []
    for k, dl in enumerate(deltas):
        r = math.sqrt(rc * rc + dl)
        u = rng.normal(size=3)
        u /= np.linalg.norm(u)
        a = rng.uniform(0, 1, 3) * box
        if k % 3 == 0:  # put the pair across a face: the partner's image is inside the box
            a[k % 2] = 0.3
        b = np.mod(a + r * u, box)
        planted.append((a, b, dl))
    pos = np.concatenate([bg] + [np.stack([a, b]) for a, b, _ in planted])
    return pos, box, rc, deltas, bg.shape[0]


def test_boundary_pairs_against_all_pairs():
    rc = 6.0
    window = 2e-3 * rc * rc
    pos, box, rc, deltas, nbg = _boundary_system(window)
    ij, r2 = oracle.boundary_pairs(pos, box, rc, window)
    # all-pairs enumeration from the definition
    d = pos[:, None, :] - pos[None, :, :]
    d = d - box * np.floor(d / box + 0.5)
    rr = np.einsum("ijk,ijk->ij", d, d)
    n = pos.shape[0]
    iu, ju = np.triu_indices(n, 1)
    gap = np.abs(rr[iu, ju] - rc * rc)
    sure = np.abs(gap - window) > 1e-9 * rc * rc  # not within rounding of the window's edge
    want = {(int(i), int(j)) for i, j, g in zip(iu, ju, gap) if g <= window}
    got = {(int(i), int(j)) for i, j in ij}
    unsure = {(int(i), int(j)) for i, j, s in zip(iu, ju, sure) if not s}
    assert got - unsure == want - unsure
    assert np.all(ij[:, 0] < ij[:, 1])
    np.testing.assert_allclose(r2, rr[ij[:, 0], ij[:, 1]], rtol=1e-13, atol=0)
    # the planted pairs: in the list iff |delta| <= window
    for k, dl in enumerate(deltas):
        i, j = nbg + 2 * k, nbg + 2 * k + 1
        assert ((i, j) in got) == (abs(dl) <= window), (k, dl / window)
    assert sum(1 for dl in deltas if abs(dl) <= window) >= 8


def test_boundary_pairs_on_a_lattice_at_the_cutoff():
    # spacing 1.5, rc = 3.0, 6 sites per axis: pair vectors v (integers) have
    # r^2 = 2.25 |v|^2.  |v|^2 = 4 sits at rc^2 exactly (3 unordered partners per atom),
    # |v|^2 = 3 and 5 sit 2.25 below and above it (4 and 12 per atom)
    m, a, rc = 6, 1.5, 3.0
    g = np.stack(np.meshgrid(*[np.arange(m)] * 3, indexing="ij"), -1).reshape(-1, 3)
    pos = (g + 0.5) * a
    box = np.full(3, m * a)
    ij, r2 = oracle.boundary_pairs(pos, box, rc, 1e-6)
    assert ij.shape[0] == pos.shape[0] * 3
    assert np.all(r2 == rc * rc)
    ij, r2 = oracle.boundary_pairs(pos, box, rc, 2.25)  # the window's edge is inclusive
    assert ij.shape[0] == pos.shape[0] * (3 + 4 + 12)
    assert sorted(set(r2.tolist())) == [6.75, 9.0, 11.25]
    ij, _ = oracle.boundary_pairs(pos, box, rc, 2.2)
    assert ij.shape[0] == pos.shape[0] * 3
