"""GPU parity: the CUDA path through the C ABI against the FP64 oracle, element by element.

Bars: cell lists identical (integer work, bit-exact); forces within the criterion of
tests/parity.py (1e-5 for FP32 pair math, 1e-12 for the FP64 mode); pair counts exact
up to boundary pairs; FIXED64 forces bit-reproducible, exactly antisymmetric and
permutation-invariant.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_1611_04474_gb300 import workloads as W
from tests.parity import boundary_alternatives, force_errors

pytestmark = pytest.mark.gpu

TOL_F32 = 1e-5
TOL_F64 = 1e-12

ALGOS_F32 = [1, 2, 3]  # full shell, half shell, cluster pairs

SYSTEMS = {
    "gas3000": lambda: W.workload_random_3000(),
    "lattice3000": lambda: W.lattice_box(n=3000, seed=5, ntypes=6),
    "box_3x4x6": lambda: W.small_random(700, (9.5, 13.0, 18.5), rc=3.0, seed=3, min_dist=0.7),
    "box_2x3x2": lambda: W.small_random(300, (6.5, 12.0, 6.6), rc=3.2, seed=4, min_dist=0.7),
    "box_5x5x7_ragged": lambda: W.small_random(2111, (20.0, 20.5, 28.9), rc=4.0, seed=8,
                                               min_dist=0.8, ntypes=5),
}


def _oracle_ref(s):
    ff = oracle.ForceField.from_system(s)
    p = s.pos.astype(np.float64)
    ref = oracle.forces_cells(p, s.q, s.type, s.box, ff)
    alts, nb = boundary_alternatives(p, s, ff, ref.F)
    return ff, p, ref, alts, nb


_cache = {}


def ref_for(name):
    if name not in _cache:
        s = SYSTEMS[name]()
        _cache[name] = (s,) + _oracle_ref(s)
    return _cache[name]


def run_forces(api, s, mode, algo=1, energy=True):
    eng = api.Engine(s, mode=mode, algo=algo)
    eng.build_cells()
    eng.compute_forces(energy=energy, count=True)
    torch.cuda.synchronize()
    return eng


@pytest.mark.parametrize("name", list(SYSTEMS))
def test_cells_identical_to_oracle(cuda_lib, name):
    api = cuda_lib
    s = SYSTEMS[name]()
    eng = api.Engine(s)
    eng.build_cells()
    torch.cuda.synchronize()
    dims, cell_of, cell_start, order = oracle.build_cells(s.pos.astype(np.float64), s.box, s.rc)
    assert list(dims) == eng.dims
    np.testing.assert_array_equal(eng.cells.cell_start.cpu().numpy(), cell_start)
    np.testing.assert_array_equal(eng.cells.perm.cpu().numpy(), order)
    pqs = eng.cells.pos_q_sorted.cpu().numpy()
    np.testing.assert_array_equal(pqs[:, :3], s.pos[order])
    np.testing.assert_array_equal(pqs[:, 3], s.q[order])
    np.testing.assert_array_equal(eng.cells.type_sorted.cpu().numpy(), s.type[order])
    assert int(eng.status.item()) == 0


def _face_coords(L, n, rng, count):
    """float32 coordinates on and next to the cell faces k L / n (k = 0..n), plus -0.0,
    float(L) and coordinates outside [0, L) that the build must wrap."""
    vals = []
    for k in range(n + 1):
        f = np.float32(k * L / n)
        up = np.nextafter(f, np.float32(np.inf))
        vals += [f, up, np.nextafter(up, np.float32(np.inf)), np.nextafter(f, np.float32(-np.inf))]
    vals += [np.float32(-0.0), np.float32(L), np.float32(-1e-7), np.float32(L + 1e-3),
             np.float32(-L + 0.5), np.float32(2.5 * L)]
    vals = np.array(vals, np.float32)
    return vals[rng.integers(0, len(vals), count)]


def _wrap_f32(x, L):
    """The documented wrap of float coordinates in FP64, rounded back to float."""
    x = x.astype(np.float64)
    w = np.where((x >= 0.0) & (x < L), x, x - L * np.floor(x / L))
    w = np.where(w < 0.0, w + L, w)
    w = np.where(w >= L, w - L, w)
    return w.astype(np.float32)


@pytest.mark.parametrize("box,rc", [((36.0, 37.3, 48.0001), 12.0), ((24.0, 25.2, 26.4), 4.0),
                                    ((10.1, 7.0, 13.37), 3.4)])
def test_cells_on_cell_faces(cuda_lib, box, rc):
    """Coordinates on, one and two float steps beside every cell face, and outside the
    box: the cell of each atom is decided exactly as the oracle's FP64 rule decides it."""
    api = cuda_lib
    s = W.small_random(900, box, rc=rc, seed=11)
    rng = np.random.default_rng(12)
    dims = oracle.cell_dims(np.array(box), rc)
    pos = s.pos.copy()
    for k in range(3):
        sel = rng.random(len(pos)) < 0.8
        pos[sel, k] = _face_coords(box[k], dims[k], rng, int(sel.sum()))
    s.pos = pos
    eng = api.Engine(s)
    eng.build_cells()
    torch.cuda.synchronize()
    dims_o, cell_of, cell_start, order = oracle.build_cells(pos.astype(np.float64), s.box, s.rc)
    assert list(dims_o) == eng.dims
    np.testing.assert_array_equal(eng.cells.cell_start.cpu().numpy(), cell_start)
    np.testing.assert_array_equal(eng.cells.perm.cpu().numpy(), order)
    pqs = eng.cells.pos_q_sorted.cpu().numpy()
    for k in range(3):
        np.testing.assert_array_equal(pqs[:, k], _wrap_f32(pos[order, k], box[k]))
    assert int(eng.status.item()) == 0


@pytest.mark.parametrize("name", list(SYSTEMS))
@pytest.mark.parametrize("mode", [0, 1, 2])
def test_forces_match_oracle(cuda_lib, name, mode):
    api = cuda_lib
    s, ff, p, ref, alts, nb = ref_for(name)
    for algo in (ALGOS_F32 if mode != 2 else [1]):
        eng = run_forces(api, s, mode, algo)
        F = api.forces_to_f64(eng.forces, mode).cpu().numpy()
        err = force_errors(F, ref.F, ref.cond, alts)
        tol = TOL_F64 if mode == 2 else TOL_F32
        assert err["max_norm"] <= tol, (name, mode, algo, err, nb)
        assert int(eng.status.item()) == 0
        cnt = int(eng.pair_count.item())
        assert abs(cnt - ref.npairs) <= nb, (cnt, ref.npairs, nb)
        ev = eng.energy_virial.cpu().numpy()
        etol = 1e-12 if mode == 2 else 1e-5
        for k in range(3):
            assert abs(ev[k] - ref.energy[k]) <= etol * ref.energy_abs[k] + 1e-9, (k, ev, ref.energy)


@pytest.mark.parametrize("name", list(SYSTEMS))
@pytest.mark.parametrize("count", [False, True])
def test_f32_forces_without_energies_match_oracle(cuda_lib, name, count):
    """The FP32 force call without energies, with and without the pair count, against the
    oracle (at these sizes the one-cluster-pair form runs: too few cells to fill the
    long-row grid); twice, so that nothing depends on what an earlier kernel left in
    shared memory."""
    api = cuda_lib
    s, ff, p, ref, alts, nb = ref_for(name)
    for _ in range(2):
        eng = api.Engine(s, mode=api.ACCUM_F32, algo=api.ALGO_CLUSTER)
        eng.build_cells()
        eng.compute_forces(energy=False, count=count)
        torch.cuda.synchronize()
        assert int(eng.status.item()) == 0
        F = api.forces_to_f64(eng.forces, api.ACCUM_F32).cpu().numpy()
        err = force_errors(F, ref.F, ref.cond, alts)
        assert err["max_norm"] <= TOL_F32, (name, count, err, nb)
        if count:
            assert abs(int(eng.pair_count.item()) - ref.npairs) <= nb


@pytest.mark.parametrize("name", ["gas3000", "lattice3000"])
def test_fixed_mode_exact_sum_and_reproducible(cuda_lib, name):
    api = cuda_lib
    s, ff, p, ref, alts, nb = ref_for(name)
    runs = []
    for algo in (1, 2, 3, 2, 3):
        eng = run_forces(api, s, api.ACCUM_FIXED64, algo)
        runs.append(eng.forces.cpu().numpy().copy())
    # the same integers from both kernels and from run to run
    for r in runs[1:]:
        assert np.array_equal(runs[0], r)
    # Newton's third law holds exactly in integer arithmetic
    assert np.all(runs[0].sum(axis=0, dtype=np.int64) == 0)


@pytest.mark.parametrize("algo", [2, 3])
def test_fixed_mode_permutation_invariant(cuda_lib, algo):
    api = cuda_lib
    s = SYSTEMS["box_5x5x7_ragged"]()
    base = run_forces(api, s, api.ACCUM_FIXED64, algo).forces.cpu().numpy()
    perm = np.random.default_rng(1).permutation(s.n)
    s2 = W.System(s.name, s.pos[perm], s.q[perm], s.type[perm], s.box, s.rc, s.sigma, s.eps, s.AB,
                  s.mass[perm], s.vel[perm])
    got = run_forces(api, s2, api.ACCUM_FIXED64, algo).forces.cpu().numpy()
    assert np.array_equal(got, base[perm])


def test_f64_mode_translation(cuda_lib):
    # translating every atom by a box vector changes nothing after the wrap
    api = cuda_lib
    s = SYSTEMS["box_3x4x6"]()
    base = run_forces(api, s, api.ACCUM_F64).forces.cpu().numpy()
    s2 = W.System(s.name, (s.pos.astype(np.float64) + s.box * np.array([1, -2, 3])).astype(np.float32),
                  s.q, s.type, s.box, s.rc, s.sigma, s.eps, s.AB, s.mass, s.vel)
    got = run_forces(api, s2, api.ACCUM_F64).forces.cpu().numpy()
    ff, p, ref, alts, nb = _oracle_ref(s2)
    err = force_errors(got, ref.F, ref.cond, alts)
    # the wrap of x + k L subtracts k L exactly, so both sides see the same coordinates
    assert err["max_norm"] <= TOL_F64
    # against the untranslated system only the float32 rounding of x + k L differs
    # (up to ulp(55 A)/2 per coordinate)
    assert np.abs(got - base).max() <= 1e-3 * np.abs(base).max()


def test_lattice_92k_full_system(cuda_lib):
    """The throughput workload itself (92,224 atoms, ApoA1 box), every atom checked."""
    api = cuda_lib
    s = W.workload_lattice_92k()
    ff, p, ref, alts, nb = _oracle_ref(s)
    for mode in (api.ACCUM_F32, api.ACCUM_FIXED64):
        for algo in ALGOS_F32:
            eng = run_forces(api, s, mode, algo)
            F = api.forces_to_f64(eng.forces, mode).cpu().numpy()
            err = force_errors(F, ref.F, ref.cond, alts)
            assert err["max_norm"] <= TOL_F32, (mode, algo, err, nb)
            assert abs(int(eng.pair_count.item()) - ref.npairs) <= nb
            assert int(eng.status.item()) == 0


# ------------------------------------------------------------------ edge cases

def _custom(pos, box, rc=3.0, ntypes=2, seed=0, q=None, types=None):
    rng = np.random.default_rng(seed)
    n = len(pos)
    sigma = rng.uniform(0.9, 1.1, ntypes)
    eps = rng.uniform(0.5, 1.0, ntypes)
    q = np.asarray(q if q is not None else rng.choice([-0.5, 0.5], n), np.float32)
    t = np.asarray(types if types is not None else rng.integers(0, ntypes, n), np.int32)
    mass = np.full(n, 12.0, np.float32)
    return W.System("custom", np.asarray(pos, np.float32).reshape(n, 3), q, t,
                    np.asarray(box, np.float64), float(np.float32(rc)), sigma, eps,
                    W.lj_table(sigma, eps), mass, np.zeros((n, 3)))


def _check_vs_oracle(api, s, modes=(0, 1, 2)):
    ff, p, ref, alts, nb = _oracle_ref(s)
    for mode in modes:
        for algo in (ALGOS_F32 if mode != 2 else [1]):
            eng = run_forces(api, s, mode, algo)
            F = api.forces_to_f64(eng.forces, mode).cpu().numpy()
            err = force_errors(F, ref.F, ref.cond, alts)
            assert err["max_norm"] <= (TOL_F64 if mode == 2 else TOL_F32), (mode, algo, err)
            assert int(eng.pair_count.item()) == ref.npairs or nb > 0
    return ref


def test_single_atom_and_empty_cells(cuda_lib):
    api = cuda_lib
    s = _custom([[1.0, 2.0, 3.0]], (10.0, 10.0, 10.0))
    ref = _check_vs_oracle(api, s)
    assert ref.npairs == 0
    # every atom in one corner of a 4x4x4 grid (a 4x4x4 lattice of spacing 0.9 A, jittered):
    # most cells empty, a few crowded
    rng = np.random.default_rng(2)
    g = np.stack(np.meshgrid(*[np.arange(4)] * 3, indexing="ij"), -1).reshape(-1, 3)
    pos = 0.2 + 0.9 * g + rng.uniform(-0.05, 0.05, g.shape)
    s = _custom(pos, (12.0, 12.0, 12.0), rc=2.9)
    _check_vs_oracle(api, s)


def test_pair_across_every_face(cuda_lib):
    api = cuda_lib
    box = (10.0, 11.0, 12.0)
    pos = [[0.2, 5.0, 6.0], [9.6, 5.3, 6.2],     # across x
           [3.0, 0.1, 3.0], [3.4, 10.8, 2.7],    # across y
           [7.0, 7.0, 11.9], [7.1, 6.6, 0.3],    # across z
           [0.1, 0.2, 0.3], [9.8, 10.9, 11.7]]   # across a corner
    s = _custom(pos, box, rc=3.0)
    ref = _check_vs_oracle(api, s)
    assert ref.npairs >= 4


def test_atoms_on_cell_boundaries_and_outside_the_box(cuda_lib):
    api = cuda_lib
    box = np.array([12.0, 12.0, 12.0])  # rc 3 -> 4x4x4 cells of edge 3 (exact)
    g = np.stack(np.meshgrid(*[np.arange(4)] * 3, indexing="ij"), -1).reshape(-1, 3) * 3.0
    pos = np.concatenate([g, g + 1.5])  # half on cell corners exactly
    s = _custom(pos, box, rc=3.0)
    _check_vs_oracle(api, s)
    rng = np.random.default_rng(5)
    pos = rng.uniform(-30.0, 40.0, (200, 3))  # far outside [0, L): wrapped by the build
    s = _custom(pos, box, rc=3.0)
    eng = run_forces(api, s, api.ACCUM_F64)
    wrapped = np.mod(pos.astype(np.float32).astype(np.float64), box)
    s_in = _custom(wrapped, box, rc=3.0, q=s.q, types=s.type)
    ff, p, ref, alts, nb = _oracle_ref(s_in)
    err = force_errors(eng.forces.cpu().numpy(), ref.F, ref.cond, alts)
    assert err["max_norm"] <= TOL_F64


def test_crowded_cells(cuda_lib):
    """Cells of more than one staged tile (512 atoms) and one cell beyond the cluster
    ordering's limit (1,331 atoms, kept in sorted order), against the oracle; FIXED64
    the same bits from every kernel."""
    api = cuda_lib
    g = np.stack(np.meshgrid(*[np.arange(24)] * 3, indexing="ij"), -1).reshape(-1, 3)
    rng = np.random.default_rng(11)
    dense = _custom(0.25 + 0.5 * g + rng.uniform(-0.03, 0.03, g.shape), (12.0, 12.0, 12.0), rc=4.0)
    b = np.stack(np.meshgrid(*[np.arange(11)] * 3, indexing="ij"), -1).reshape(-1, 3)
    blob = 0.2 + 0.33 * b + rng.uniform(-0.02, 0.02, b.shape)       # one cell, 1,331 atoms
    rest = rng.uniform((5.5, 0.0, 0.0), (12.0, 12.0, 12.0), (300, 3))  # away from the blob
    keep = np.ones(len(rest), bool)
    for k in range(len(rest)):  # at least 0.8 A apart
        d = np.linalg.norm(rest[:k][keep[:k]] - rest[k], axis=1)
        keep[k] = not np.any(d < 0.8)
    mixed = _custom(np.concatenate([blob, rest[keep]]), (12.0, 12.0, 12.0), rc=4.0)
    for s, least in ((dense, 257), (mixed, 1025)):
        c3 = np.minimum(np.floor(s.pos.astype(np.float64) / 4.0), 2).astype(int)
        counts = np.bincount(c3[:, 0] + 3 * (c3[:, 1] + 3 * c3[:, 2]), minlength=27)
        assert counts.max() >= least
        _check_vs_oracle(api, s, modes=(0, 1))
        fx = [run_forces(api, s, api.ACCUM_FIXED64, algo).forces.cpu().numpy() for algo in (1, 2, 3)]
        assert np.array_equal(fx[0], fx[1]) and np.array_equal(fx[0], fx[2])


def test_many_types(cuda_lib):
    api = cuda_lib
    s = W.small_random(900, (15.0, 15.0, 15.0), ntypes=32, rc=3.5, seed=12, min_dist=0.8)
    _check_vs_oracle(api, s, modes=(0, 1))


def test_status_flags(cuda_lib):
    api = cuda_lib
    pos = [[1.0, 1.0, 1.0], [np.nan, 2.0, 2.0], [3.0, 3.0, 3.0]]
    s = _custom(pos, (10.0, 10.0, 10.0))
    eng = run_forces(api, s, api.ACCUM_F32)
    assert int(eng.status.item()) & api.STATUS_NONFINITE
    s = _custom([[1.0, 1.0, 1.0], [1.5, 1.0, 1.0]], (10.0, 10.0, 10.0), types=[0, 7])
    eng = run_forces(api, s, api.ACCUM_F32)
    assert int(eng.status.item()) & api.STATUS_BAD_TYPE
    # two atoms 0.01 A apart: an LJ term far beyond 2^31 kcal/mol/A
    s = _custom([[1.0, 1.0, 1.0], [1.01, 1.0, 1.0]], (10.0, 10.0, 10.0), types=[0, 0])
    eng = run_forces(api, s, api.ACCUM_FIXED64)
    assert int(eng.status.item()) & api.STATUS_FIXED_OVERFLOW


def test_errors_from_the_abi(cuda_lib):
    api = cuda_lib
    s = W.small_random(50, (10.0, 10.0, 10.0), rc=3.0, seed=1)
    eng = api.Engine(s)
    eng.build_cells()
    small_ws = torch.empty(64, dtype=torch.uint8, device="cuda")
    with pytest.raises(api.MDError) as e:
        api.nonbonded_forces(eng.cells, eng.box, eng.ff, small_ws)
    assert e.value.code == -3
    ff_bad = api.ForceField(s.AB, s.k_coulomb, 5.0)  # rc >= L/2
    with pytest.raises(api.MDError) as e:
        api.nonbonded_forces(eng.cells, eng.box, ff_bad, eng.workspace)
    assert e.value.code == -2


# ------------------------------------------------------------------ full sizes

def _boundary_atoms(p, box, rc, sel):
    """Sampled atoms with a partner whose FP64 r^2 lies in the boundary window of rc^2."""
    from scipy.spatial import cKDTree

    from tests.parity import boundary_window

    w = np.mod(p, box)
    tree = cKDTree(w, boxsize=box)
    lo, hi = rc * rc - boundary_window(rc), rc * rc + boundary_window(rc)
    out = np.zeros(len(sel), bool)
    for k, i in enumerate(sel):
        for j in tree.query_ball_point(w[i], np.sqrt(hi)):
            if j == i:
                continue
            d = p[i] - p[j]
            d -= box * np.round(d / box)
            r2 = float(d @ d)
            if lo <= r2 <= hi:
                out[k] = True
                break
    return out


def _sampled_reference(n):
    """The lattice of n atoms, 2,048 sampled atoms, their oracle forces and which of them
    have no boundary pair (computed once per test session)."""
    key = ("sampled", n)
    if key not in _cache:
        s = W.lattice_box(n=n)
        sel = np.random.default_rng(3).choice(s.n, size=2048, replace=False).astype(np.int32)
        ff = oracle.ForceField.from_system(s)
        p = s.pos.astype(np.float64)
        Fo, cond, _ = oracle.forces_atoms(p, s.q, s.type, s.box, ff, sel)
        _cache[key] = (s, sel, Fo, cond, ~_boundary_atoms(p, s.box, s.rc, sel))
    return _cache[key]


def _lattice92k_reference():
    """The 92,224-atom lattice and the oracle's forces on every atom, with the boundary-pair
    alternatives (computed once per test session)."""
    if "92k" not in _cache:
        s = W.lattice_box(n=W.APOA1_N)
        ff = oracle.ForceField.from_system(s)
        p = s.pos.astype(np.float64)
        ref = oracle.forces_cells(p, s.q, s.type, s.box, ff)
        alts, nb = boundary_alternatives(p, s, ff, ref.F)
        _cache["92k"] = (s, ref, alts, nb)
    return _cache["92k"]


@pytest.mark.parametrize("count", [False, True])
def test_f32_long_rows_92k_whole_system(cuda_lib, count):
    """The FP32 force call on the 92,224-atom lattice (the long-row form of the cluster
    kernel: 486 cells fill its grid), every atom against the oracle, with and without
    the pair count; twice, so that nothing depends on what an earlier kernel left in
    shared memory."""
    api = cuda_lib
    s, ref, alts, nb = _lattice92k_reference()
    for _ in range(2):
        eng = api.Engine(s, mode=api.ACCUM_F32, algo=api.ALGO_CLUSTER)
        eng.build_cells()
        eng.compute_forces(energy=False, count=count)
        torch.cuda.synchronize()
        assert int(eng.status.item()) == 0
        F = api.forces_to_f64(eng.forces, api.ACCUM_F32).cpu().numpy()
        err = force_errors(F, ref.F, ref.cond, alts)
        assert err["max_norm"] <= TOL_F32, (count, err, nb)
        if count:
            assert abs(int(eng.pair_count.item()) - ref.npairs) <= nb


@pytest.mark.parametrize("n", [W.APOA1_N // 4, W.APOA1_N * 4, W.APOA1_N * 16])
@pytest.mark.parametrize("mode", ["f32", "fixed64"])
def test_sweep_sizes_sampled(cuda_lib, n, mode):
    """The other points of the size sweep (23,056, 368,896 and 1,475,584 atoms; the first
    runs the one-cluster-pair form, the others the long-row form in FP32), in the launch
    the force call makes: 2,048 sampled atoms against the oracle; in FIXED64 Newton's third
    law holds exactly over the whole system."""
    api = cuda_lib
    s, sel, Fo, cond, use = _sampled_reference(n)
    m = api.ACCUM_F32 if mode == "f32" else api.ACCUM_FIXED64
    eng = run_forces(api, s, m, algo=0, energy=False)
    assert int(eng.status.item()) == 0
    if m == api.ACCUM_FIXED64:
        assert np.all(eng.forces.cpu().numpy().sum(axis=0, dtype=np.int64) == 0)
    F = api.forces_to_f64(eng.forces, m).cpu().numpy()
    assert use.sum() > 1800
    err = np.linalg.norm(F[sel] - Fo, axis=1)[use] / cond[use]
    assert err.max() <= TOL_F32, err.max()
