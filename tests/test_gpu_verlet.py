"""md_step_verlet: the MD step with cells kept across steps while every atom stays within
skin/2 of where it was when they were built (the cell method of Section II.A, reused).

Bars: in MD_ACCUM_FIXED64 the trajectory is md_step's bit for bit (the same pairs, the
same pair terms, the same integer sums), including atoms that cross a face of the box
while the cells are kept, boxes with an axis of two cells, a skin so small that every
step rebuilds, and a run split over several calls; in MD_ACCUM_F32 the forces of every
step match the FP64 oracle at the step's positions (the criterion of tests/parity.py);
MD_ACCUM_FIXED_TILE is bit-reproducible; the cells are reused (fewer builds than steps).
"""
import numpy as np
import pytest
import torch

import oracle
from paper_1611_04474_gb300 import workloads as W
from tests.parity import boundary_alternatives, force_errors

pytestmark = pytest.mark.gpu


def _gentle(n=92224):
    base = W.workload_lattice_92k() if n == 92224 else W.lattice_box(n=n, seed=2)
    return base.with_forcefield(sigma_scale=0.5, mass_range=(12.0, 16.0), seed=22)


def _state(eng):
    return (eng.pos.cpu().numpy().copy(), eng.vel.cpu().numpy().copy(),
            eng.forces.cpu().numpy().copy())


def _crossings(x0, x1, box):
    """Atoms whose wrapped coordinate jumped by more than half a box (crossed a face)."""
    return int((np.abs(x1 - x0) > 0.5 * box).any(axis=1).sum())


@pytest.mark.parametrize("skin", [1.0, 0.3])
def test_fixed64_verlet_is_md_step_bit_for_bit(cuda_lib, skin):
    api = cuda_lib
    s = _gentle()
    n_steps = 50
    plain = api.Engine(s, mode=api.ACCUM_FIXED64)
    plain.step(n_steps, dt_fs=1.0)
    ver = api.Engine(s, mode=api.ACCUM_FIXED64)
    ver.step_verlet(n_steps, dt_fs=1.0, skin=skin)
    torch.cuda.synchronize()
    assert int(plain.status.item()) == 0 and int(ver.status.item()) == 0
    for a, b in zip(_state(plain), _state(ver)):
        assert np.array_equal(a, b)
    builds = int(ver.rebuilds.item())
    assert 1 < builds < n_steps + 1, builds  # the cells were kept over several steps
    # atoms crossed faces of the box in the run (so kept cells saw wrapped atoms)
    assert _crossings(s.pos.astype(np.float64), ver.pos.cpu().numpy(), s.box) > 0


def test_fixed64_verlet_every_step_rebuilds_and_split_calls(cuda_lib):
    api = cuda_lib
    s = _gentle(23056)
    plain = api.Engine(s, mode=api.ACCUM_FIXED64)
    plain.step(30, dt_fs=1.0)
    # a skin so small that every step builds the cells again
    tiny = api.Engine(s, mode=api.ACCUM_FIXED64)
    tiny.step_verlet(30, dt_fs=1.0, skin=1e-4)
    # the same run in three calls (each call builds the cells at its first step)
    split = api.Engine(s, mode=api.ACCUM_FIXED64)
    for k in (7, 13, 10):
        split.step_verlet(k, dt_fs=1.0, skin=0.8)
    torch.cuda.synchronize()
    ref = _state(plain)
    for eng in (tiny, split):
        assert int(eng.status.item()) == 0
        for a, b in zip(ref, _state(eng)):
            assert np.array_equal(a, b)
    assert int(tiny.rebuilds.item()) == 31  # the initial forces and every step
    assert 3 <= int(split.rebuilds.item()) < 31


def test_fixed64_verlet_two_cells_per_axis(cuda_lib):
    """rc + skin close to L/2: the kept grid has an axis of two cells, where every pair
    takes the per-pair minimum image."""
    api = cuda_lib
    s = W.lattice_box(n=3000, seed=5, ntypes=6).with_forcefield(0.5, (12.0, 16.0), seed=1)
    skin = 0.4995 * float(s.box.min()) - s.rc  # the largest skin below min(L)/2 - rc
    assert skin > 0.2
    from paper_1611_04474_gb300 import api as _a
    assert min(_a.cell_dims(s.box, s.rc + skin)) == 2
    plain = api.Engine(s, mode=api.ACCUM_FIXED64)
    plain.step(20, dt_fs=1.0)
    ver = api.Engine(s, mode=api.ACCUM_FIXED64)
    ver.step_verlet(20, dt_fs=1.0, skin=skin)
    torch.cuda.synchronize()
    assert int(ver.status.item()) == 0
    for a, b in zip(_state(plain), _state(ver)):
        assert np.array_equal(a, b)


def test_f32_verlet_forces_match_oracle_every_step(cuda_lib):
    api = cuda_lib
    s = _gentle(23056)
    ff = oracle.ForceField.from_system(s)
    eng = api.Engine(s, mode=api.ACCUM_F32)
    for k in range(6):
        eng.step_verlet(3 if k else 1, dt_fs=1.0, skin=1.0)
        torch.cuda.synchronize()
        assert int(eng.status.item()) == 0
        x, _, F = _state(eng)
        p32 = x.astype(np.float32).astype(np.float64)
        ref = oracle.forces_cells(p32, s.q, s.type, s.box, ff)
        alts, nb = boundary_alternatives(p32, s, ff, ref.F)
        err = force_errors(F.astype(np.float64), ref.F, ref.cond, alts)
        assert err["max_norm"] <= 1e-5, (k, err)


def test_verlet_energy_log_matches_md_step(cuda_lib):
    api = cuda_lib
    s = _gentle(23056)
    logs = []
    for verlet in (False, True):
        eng = api.Engine(s, mode=api.ACCUM_FIXED64)
        log = torch.zeros((10, 4), dtype=torch.float64, device="cuda")
        if verlet:
            eng.step_verlet(10, dt_fs=1.0, skin=1.0, energy_log=log)
        else:
            eng.step(10, dt_fs=1.0, energy_log=log)
        torch.cuda.synchronize()
        logs.append(log.cpu().numpy())
    # the same states (FIXED64), so the same kinetic energy; the pair energies are summed
    # in FP32 per thread over other cells, so they agree to FP32 rounding
    np.testing.assert_array_equal(logs[1][:, 2], logs[0][:, 2])
    for col in (0, 1, 3):
        np.testing.assert_allclose(logs[1][:, col], logs[0][:, col], rtol=2e-6)


def test_fixed_tile_verlet_reproducible(cuda_lib):
    api = cuda_lib
    s = _gentle(23056)
    runs = []
    for _ in range(2):
        eng = api.Engine(s, mode=api.ACCUM_FIXED_TILE)
        eng.step_verlet(20, dt_fs=1.0, skin=1.0)
        torch.cuda.synchronize()
        assert int(eng.status.item()) == 0
        runs.append(_state(eng))
    for a, b in zip(runs[0], runs[1]):
        assert np.array_equal(a, b)
