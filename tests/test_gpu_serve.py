"""Continuous-batching server: jobs that arrive while others run are admitted as memory
frees up; each job's result is the same, bit for bit in the deterministic modes, as
running it alone through md_step, and matches the FP64 oracle at its final positions."""
import numpy as np
import pytest
import torch

import oracle
from paper_1611_04474_gb300 import api, serve
from paper_1611_04474_gb300 import workloads as W
from tests.parity import boundary_alternatives, force_errors


def _jobs(n=10, seed=11):
    specs = W.serving_jobs(n_jobs=n, rate_per_s=500.0, seed=seed, n_range=(800, 4000),
                           steps_range=(3, 17))
    return [serve.Job(k, mk, st, arr, na) for k, (mk, st, arr, na) in enumerate(specs)]


@pytest.mark.gpu
@pytest.mark.parametrize("mode", [api.ACCUM_FIXED_TILE, api.ACCUM_FIXED64])
def test_results_equal_alone_and_budget_respected(cuda_lib, mode):
    jobs = _jobs()
    largest = max(serve.job_footprint_bytes(j.n_atoms) for j in jobs)
    srv = serve.Server(mode=mode, budget_bytes=2 * largest, tick_steps=4, max_wait_s=0.0)
    stats = srv.run(jobs)
    assert srv.max_footprint <= 2 * largest
    assert srv.rebuilds > 2  # jobs joined and left while others were running
    assert stats["latency_p99_s"] >= stats["latency_p50_s"] > 0
    assert all(np.isfinite(j.finished) and j.finished > j.arrival for j in jobs)
    for j in jobs:
        eng = api.Engine(j.make_system(), mode=mode)
        eng.step(j.n_steps)
        torch.cuda.synchronize()
        assert np.array_equal(j.state["pos"].cpu().numpy(), eng.pos.cpu().numpy()), j.id
        assert np.array_equal(j.state["vel"].cpu().numpy(), eng.vel.cpu().numpy()), j.id
        assert np.array_equal(j.state["forces"].cpu().numpy(), eng.forces.cpu().numpy()), j.id
        assert j.pairs > 0


@pytest.mark.gpu
@pytest.mark.parametrize("mode", [api.ACCUM_F32, api.ACCUM_FIXED_TILE])
def test_served_forces_match_oracle(cuda_lib, mode):
    """Every served job's final forces against the FP64 oracle at its final float32
    positions (the criterion of tests/parity.py)."""
    jobs = _jobs(n=8, seed=12)
    largest = max(serve.job_footprint_bytes(j.n_atoms) for j in jobs)
    srv = serve.Server(mode=mode, budget_bytes=3 * largest, tick_steps=5)
    srv.run(jobs)
    for j in jobs:
        s = j.make_system()
        ff = oracle.ForceField.from_system(s)
        x = j.state["pos"].cpu().numpy()
        p32 = x.astype(np.float32).astype(np.float64)
        ref = oracle.forces_cells(p32, s.q, s.type, s.box, ff)
        alts, nb = boundary_alternatives(p32, s, ff, ref.F)
        F = api.forces_to_f64(j.state["forces"], mode).cpu().numpy()
        err = force_errors(F, ref.F, ref.cond, alts)
        assert err["max_norm"] <= 1e-5, (j.id, err)
        # the counted pairs are those of its n_steps force evaluations, each close to
        # the oracle's count at the final positions
        assert 0.5 * j.n_steps * ref.npairs < j.pairs < 1.5 * j.n_steps * ref.npairs


def test_fifo_alone_model():
    class J:
        def __init__(self, a, p):
            self.arrival, self.pairs = a, p
    jobs = [J(0.0, 10), J(0.5, 10), J(0.6, 10)]
    r = serve.fifo_alone(jobs, [1.0, 1.0, 1.0])
    # finishes at 1, 2, 3 -> latencies 1, 1.5, 2.4
    assert r["latency_p50_s"] == pytest.approx(1.5)
    assert r["pairs_per_s"] == pytest.approx(10.0)
