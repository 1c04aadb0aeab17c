"""MD_ACCUM_FIXED_TILE: FP32 pair math and FP32 partial sums, each partial (a home
cluster's sums over one neighbour tile, a neighbour tile's reactions) rounded once to
the int64 grid of MD_ACCUM_FIXED64.

Bars: forces within the FP32 criterion of tests/parity.py against the FP64 oracle (the
pair terms are those of Eq. 1-2 in FP32, as in MD_ACCUM_F32); the same bits from run to
run for force calls and for MD steps; a batch gives each system the bits it gets alone;
the residual of Newton's third law (exactly zero in MD_ACCUM_FIXED64, where every pair
term is rounded on its own) stays at the size of FP32 rounding.
"""
import numpy as np
import pytest
import torch

from paper_1611_04474_gb300 import workloads as W
from tests.parity import force_errors
from tests.test_gpu_parity import TOL_F32, _oracle_ref, run_forces

pytestmark = pytest.mark.gpu

SYSTEMS = {
    "gas3000": lambda: W.workload_random_3000(),
    "box_3x4x6": lambda: W.small_random(700, (9.5, 13.0, 18.5), rc=3.0, seed=3, min_dist=0.7),
    "box_2x3x2": lambda: W.small_random(300, (6.5, 12.0, 6.6), rc=3.2, seed=4, min_dist=0.7),
    "box_5x5x7_ragged": lambda: W.small_random(2111, (20.0, 20.5, 28.9), rc=4.0, seed=8,
                                               min_dist=0.8, ntypes=5),
    "lattice_92224": lambda: W.workload_lattice_92k(),
}


@pytest.mark.parametrize("name", list(SYSTEMS))
def test_fixed_tile_matches_oracle(cuda_lib, name):
    api = cuda_lib
    s = SYSTEMS[name]()
    ff, p, ref, alts, nb = _oracle_ref(s)
    for algo in (api.ALGO_DEFAULT, api.ALGO_CLUSTER):
        eng = run_forces(api, s, api.ACCUM_FIXED_TILE, algo)
        F = api.forces_to_f64(eng.forces, api.ACCUM_FIXED_TILE).cpu().numpy()
        err = force_errors(F, ref.F, ref.cond, alts)
        assert err["max_norm"] <= TOL_F32, (name, algo, err, nb)
        assert int(eng.status.item()) == 0
        assert abs(int(eng.pair_count.item()) - ref.npairs) <= nb
        ev = eng.energy_virial.cpu().numpy()
        for k in range(3):
            assert abs(ev[k] - ref.energy[k]) <= 1e-5 * ref.energy_abs[k] + 1e-9, (k, ev, ref.energy)
        # Newton's third law: the action and the reaction of a pair are the same FP32
        # values summed in different partials, so the net force is FP32 rounding only
        net = np.abs(eng.forces.cpu().numpy().sum(axis=0, dtype=np.int64)).max() / 2.0**32
        assert net <= 1e-6 * np.abs(F).sum(), (net, np.abs(F).sum())


def _crowded():
    """3 x 3 x 3 cells of 512 atoms each: every cell pair takes two 256-atom home tiles and
    two neighbour tiles, so each home cluster's sums are rounded once per neighbour tile."""
    from tests.test_gpu_parity import _custom

    g = np.stack(np.meshgrid(*[np.arange(24)] * 3, indexing="ij"), -1).reshape(-1, 3)
    rng = np.random.default_rng(11)
    return _custom(0.25 + 0.5 * g + rng.uniform(-0.03, 0.03, g.shape), (12.0, 12.0, 12.0), rc=4.0)


_refs = {}


@pytest.mark.parametrize("name", list(SYSTEMS) + ["crowded_512"])
@pytest.mark.parametrize("count", [False, True])
def test_fixed_tile_forces_without_energies_match_oracle(cuda_lib, name, count):
    """Forces alone, with and without the pair count (the force call without energy
    sums), on regular boxes, a box with a 2-cell axis and crowded cells: against the
    oracle, the same bits on a second call, Newton's third law to FP32 size."""
    api = cuda_lib
    if name not in _refs:
        s = _crowded() if name == "crowded_512" else SYSTEMS[name]()
        _refs[name] = (s,) + _oracle_ref(s)
    s, ff, p, ref, alts, nb = _refs[name]
    runs = []
    for _ in range(2):
        eng = api.Engine(s, mode=api.ACCUM_FIXED_TILE, algo=api.ALGO_CLUSTER)
        eng.build_cells()
        eng.compute_forces(energy=False, count=count)
        torch.cuda.synchronize()
        assert int(eng.status.item()) == 0
        runs.append(eng.forces.cpu().numpy().copy())
        F = api.forces_to_f64(eng.forces, api.ACCUM_FIXED_TILE).cpu().numpy()
        err = force_errors(F, ref.F, ref.cond, alts)
        assert err["max_norm"] <= TOL_F32, (name, count, err, nb)
        if count:
            assert abs(int(eng.pair_count.item()) - ref.npairs) <= nb
        net = np.abs(runs[-1].sum(axis=0, dtype=np.int64)).max() / 2.0**32
        assert net <= 1e-6 * np.abs(F).sum(), (net, np.abs(F).sum())
    assert np.array_equal(runs[0], runs[1])


def test_fixed_tile_reproducible_run_to_run(cuda_lib):
    api = cuda_lib
    s = SYSTEMS["lattice_92224"]()
    runs = []
    for _ in range(3):
        eng = run_forces(api, s, api.ACCUM_FIXED_TILE, api.ALGO_CLUSTER, energy=False)
        runs.append(eng.forces.cpu().numpy().copy())
        # a second call on the same engine as well
        eng.compute_forces()
        torch.cuda.synchronize()
        runs.append(eng.forces.cpu().numpy().copy())
    for r in runs[1:]:
        assert np.array_equal(runs[0], r)
    # and it is a different rounding from the per-pair mode, within FP32 size of it
    fx = run_forces(api, s, api.ACCUM_FIXED64, api.ALGO_CLUSTER, energy=False).forces.cpu().numpy()
    d = np.abs(runs[0] - fx).max() / 2.0**32
    assert 0 < d <= 1e-3 * np.abs(fx).max() / 2.0**32


def test_fixed_tile_md_steps_reproducible(cuda_lib):
    api = cuda_lib
    s = W.lattice_box(n=23056, seed=2).with_forcefield(sigma_scale=0.5, mass_range=(12.0, 16.0),
                                                       seed=22)
    out = []
    for _ in range(2):
        eng = api.Engine(s, mode=api.ACCUM_FIXED_TILE)
        eng.step(10, dt_fs=1.0)
        torch.cuda.synchronize()
        assert int(eng.status.item()) == 0
        out.append((eng.pos.cpu().numpy(), eng.vel.cpu().numpy(), eng.forces.cpu().numpy()))
    for a, b in zip(out[0], out[1]):
        assert np.array_equal(a, b)
    # the trajectory follows the F32 one (the same pair terms, other roundings)
    e32 = api.Engine(s, mode=api.ACCUM_F32)
    e32.step(10, dt_fs=1.0)
    torch.cuda.synchronize()
    dx = out[0][0] - e32.pos.cpu().numpy()
    dx -= s.box * np.round(dx / s.box)
    assert np.abs(dx).max() < 1e-6


@pytest.mark.parametrize("shape", [0, 5])
@pytest.mark.parametrize("n_steps", [0, 3])
def test_fixed_tile_batch_is_bitwise_the_single_system_path(cuda_lib, shape, n_steps):
    api = cuda_lib
    systems = W.batch_of_systems(nsys=10, seed=7, n_range=(400, 6000))
    b = api.Batch(systems, mode=api.ACCUM_FIXED_TILE, tuning=(shape, shape))
    b.step(n_steps, dt_fs=1.0)
    torch.cuda.synchronize()
    assert int(b.status.item()) == 0
    Fb, Xb = b.forces.cpu().numpy(), b.pos.cpu().numpy()
    for k, s in enumerate(systems):
        eng = api.Engine(s, mode=api.ACCUM_FIXED_TILE)
        eng.step(n_steps, dt_fs=1.0)
        torch.cuda.synchronize()
        sl = b.system_slice(k)
        assert np.array_equal(Fb[sl], eng.forces.cpu().numpy()), k
        assert np.array_equal(Xb[sl], eng.pos.cpu().numpy()), k
