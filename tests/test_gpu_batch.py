"""Batched systems (md_batch_*): every system's result in the batch equals running it
alone, bit for bit in FIXED64, and matches the FP64 oracle."""
import numpy as np
import pytest
import torch

import oracle
from paper_1611_04474_gb300 import workloads as W
from tests.parity import boundary_alternatives, force_errors

pytestmark = pytest.mark.gpu


def _systems():
    # small boxes (an axis of two cells: per-pair minimum image) and larger ones together
    return W.batch_of_systems(nsys=10, seed=7, n_range=(400, 6000))


def _alone(api, s, mode, n_steps):
    eng = api.Engine(s, mode=mode)
    eng.step(n_steps, dt_fs=1.0) if n_steps else eng.step(0, dt_fs=1.0)
    torch.cuda.synchronize()
    return eng


def test_batch_mixes_both_cell_regimes():
    from paper_1611_04474_gb300 import api  # noqa: F401 (import only)

    dims = [np.floor(s.box / s.rc) for s in _systems()]
    assert any(d.min() < 3 for d in dims) and any(d.min() >= 3 for d in dims)


@pytest.mark.parametrize("n_steps", [0, 4])
def test_fixed64_batch_is_bitwise_the_single_system_path(cuda_lib, n_steps):
    api = cuda_lib
    systems = _systems()
    b = api.Batch(systems, mode=api.ACCUM_FIXED64)
    b.step(n_steps, dt_fs=1.0, count_pairs=True)
    torch.cuda.synchronize()
    assert int(b.status.item()) == 0
    Fb = b.forces.cpu().numpy()
    Xb = b.pos.cpu().numpy()
    Vb = b.vel.cpu().numpy()
    counts = b.pair_count.cpu().numpy()
    for k, s in enumerate(systems):
        eng = _alone(api, s, api.ACCUM_FIXED64, n_steps)
        sl = b.system_slice(k)
        assert np.array_equal(Fb[sl], eng.forces.cpu().numpy()), k
        assert np.array_equal(Xb[sl], eng.pos.cpu().numpy()), k
        assert np.array_equal(Vb[sl], eng.vel.cpu().numpy()), k
        eng.build_cells()
        eng.compute_forces(count=True)
        torch.cuda.synchronize()
        if n_steps == 0:
            assert counts[k] == int(eng.pair_count.item()), k


def test_f32_batch_matches_oracle(cuda_lib):
    api = cuda_lib
    systems = _systems()
    b = api.Batch(systems, mode=api.ACCUM_F32)
    b.step(0)
    torch.cuda.synchronize()
    F = b.forces.cpu().numpy().astype(np.float64)
    for k in (0, 3, 9):
        s = systems[k]
        ff = oracle.ForceField.from_system(s)
        p = s.pos.astype(np.float64)
        ref = oracle.forces_cells(p, s.q, s.type, s.box, ff)
        alts, nb = boundary_alternatives(p, s, ff, ref.F)
        err = force_errors(F[b.system_slice(k)], ref.F, ref.cond, alts)
        assert err["max_norm"] <= 1e-5, (k, err)


@pytest.mark.parametrize("mode", ["fixed64", "f32"])
def test_every_kernel_shape_gives_the_same_result(cuda_lib, mode):
    """The tuning shapes change only the launch: FIXED64 forces and trajectories are the
    same bits and the pair counts are equal under every shape; F32 agrees to rounding."""
    api = cuda_lib
    m = api.ACCUM_FIXED64 if mode == "fixed64" else api.ACCUM_F32
    systems = _systems()
    ref = None
    for r in range(api.BATCH_SHAPES):
        for s in range(api.BATCH_SHAPES):
            if r and s and r != s:
                continue  # each shape in each regime, against the default in the other
            b = api.Batch(systems, mode=m, tuning=(r, s))
            # F32 trajectories differ by rounding between shapes: compare start forces
            b.step(2 if m == api.ACCUM_FIXED64 else 0, dt_fs=1.0, count_pairs=True)
            torch.cuda.synchronize()
            assert int(b.status.item()) == 0, (r, s)
            got = (b.forces.cpu().numpy(), b.pos.cpu().numpy(), b.pair_count.cpu().numpy())
            if ref is None:
                ref = got
                continue
            assert np.array_equal(got[2], ref[2]), (r, s)
            if m == api.ACCUM_FIXED64:
                assert np.array_equal(got[0], ref[0]), (r, s)
                assert np.array_equal(got[1], ref[1]), (r, s)
            else:
                scale = np.abs(ref[0]).max()
                assert np.abs(got[0].astype(np.float64) - ref[0]).max() <= 1e-5 * scale, (r, s)


def test_autotuner_leaves_the_trajectory_and_caches(cuda_lib, tmp_path):
    api = cuda_lib
    from paper_1611_04474_gb300 import autotune

    systems = _systems()
    plain = api.Batch(systems, mode=api.ACCUM_FIXED64)
    plain.step(3, dt_fs=1.0)
    tuned = api.Batch(systems, mode=api.ACCUM_FIXED64)
    cache = str(tmp_path / "tuning.json")
    e1 = autotune.tune(tuned, cache_path=cache, n_steps=1, reps=1)
    assert e1["measured"] and len(e1["ms"]) == 2  # both regimes are present
    tuned.step(3, dt_fs=1.0)
    torch.cuda.synchronize()
    assert np.array_equal(tuned.pos.cpu().numpy(), plain.pos.cpu().numpy())
    assert np.array_equal(tuned.forces.cpu().numpy(), plain.forces.cpu().numpy())
    again = api.Batch(systems, mode=api.ACCUM_FIXED64)
    e2 = autotune.tune(again, cache_path=cache)
    assert not e2["measured"] and tuple(e2["tuning"]) == tuple(e1["tuning"]) == again.tuning


def test_full_size_batch_sampled(cuda_lib):
    """The 256-system batch (1.24 M atoms, N 500-20,000) at full size: FIXED64 steps of
    sampled systems bitwise equal to running them alone, FP32 forces of sampled systems
    against the oracle."""
    api = cuda_lib
    systems = W.batch_of_systems()
    b = api.Batch(systems, mode=api.ACCUM_FIXED64)
    b.step(2, dt_fs=1.0)
    torch.cuda.synchronize()
    assert int(b.status.item()) == 0
    sizes = np.array([s.n for s in systems])
    dims = [np.floor(s.box / s.rc).min() for s in systems]
    picks = {int(np.argmax(sizes)), int(np.argmin(sizes)), int(np.argmax(dims)),
             int(np.argmin(dims)), 100}
    Xb, Fb = b.pos.cpu().numpy(), b.forces.cpu().numpy()
    for k in sorted(picks):
        eng = _alone(api, systems[k], api.ACCUM_FIXED64, 2)
        sl = b.system_slice(k)
        assert np.array_equal(Xb[sl], eng.pos.cpu().numpy()), k
        assert np.array_equal(Fb[sl], eng.forces.cpu().numpy()), k
    b32 = api.Batch(systems, mode=api.ACCUM_F32)
    b32.step(0)
    torch.cuda.synchronize()
    F32 = b32.forces.cpu().numpy().astype(np.float64)
    for k in sorted(picks):
        s = systems[k]
        ff = oracle.ForceField.from_system(s)
        p = s.pos.astype(np.float64)
        ref = oracle.forces_cells(p, s.q, s.type, s.box, ff)
        alts, nb = boundary_alternatives(p, s, ff, ref.F)
        err = force_errors(F32[b32.system_slice(k)], ref.F, ref.cond, alts)
        assert err["max_norm"] <= 1e-5, (k, err)


def test_cuda_graph_replay_is_the_plain_loop(cuda_lib):
    """md_batch_step captured once in a CUDA graph and replayed gives the same FIXED64
    bits as calling it step by step."""
    api = cuda_lib
    systems = _systems()
    plain = api.Batch(systems, mode=api.ACCUM_FIXED64)
    plain.step(1, dt_fs=1.0)
    graphed = api.Batch(systems, mode=api.ACCUM_FIXED64)
    graphed.step(1, dt_fs=1.0)  # one call outside the capture
    torch.cuda.synchronize()
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    g = torch.cuda.CUDAGraph()
    with torch.cuda.stream(s):
        with torch.cuda.graph(g, stream=s):
            graphed.step(3, dt_fs=1.0)
    torch.cuda.synchronize()
    g.replay()
    g.replay()
    plain.step(6, dt_fs=1.0)
    torch.cuda.synchronize()
    assert int(graphed.status.item()) == 0
    for name in ("pos", "vel", "forces"):
        assert np.array_equal(getattr(graphed, name).cpu().numpy(), getattr(plain, name).cpu().numpy()), name


def test_staged_prepare_behind_queued_work_is_the_plain_prepare(cuda_lib):
    """md_batch_prepare_staged enqueues its copy without waiting for the stream: a batch
    prepared that way while another batch's steps are still queued steps bit for bit like
    one prepared with md_batch_prepare on an idle stream."""
    api = cuda_lib
    systems = _systems()
    busy = api.Batch(W.batch_of_systems(nsys=4, seed=11, n_range=(20000, 40000)),
                     mode=api.ACCUM_FIXED_TILE)
    torch.cuda.synchronize()
    results = []
    for staged in (True, False):
        busy.step(20, dt_fs=1.0)  # queued ahead of the prepare's copy
        b = api.Batch(systems, mode=api.ACCUM_FIXED_TILE, staged=staged)
        b.step(5, dt_fs=1.0, count_pairs=True)
        torch.cuda.synchronize()
        assert int(b.status.item()) == 0
        results.append([t.cpu().numpy() for t in (b.pos, b.vel, b.forces, b.pair_count)])
    for a, c in zip(*results):
        assert np.array_equal(a, c)
