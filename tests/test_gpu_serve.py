"""Continuous-batching server: jobs that arrive while others run are admitted as memory
frees up, and each job's result is the same, bit for bit in FIXED64, as running it
alone through md_step."""
import numpy as np
import pytest
import torch

from paper_1611_04474_gb300 import api, serve
from paper_1611_04474_gb300 import workloads as W

def _jobs(n=10, seed=11):
    specs = W.serving_jobs(n_jobs=n, rate_per_s=500.0, seed=seed, n_range=(800, 4000),
                           steps_range=(3, 17))
    return [serve.Job(k, mk, st, arr, na) for k, (mk, st, arr, na) in enumerate(specs)]


@pytest.mark.gpu
def test_results_equal_alone_and_budget_respected(cuda_lib):
    jobs = _jobs()
    largest = max(serve.job_footprint_bytes(j.n_atoms) for j in jobs)
    srv = serve.Server(mode=api.ACCUM_FIXED64, budget_bytes=2 * largest, tick_steps=4)
    stats = srv.run(jobs)
    assert srv.max_footprint <= 2 * largest
    assert srv.rebuilds > 2  # jobs joined and left while others were running
    assert stats["latency_p99_s"] >= stats["latency_p50_s"] > 0
    for j in jobs:
        eng = api.Engine(j.make_system(), mode=api.ACCUM_FIXED64)
        eng.step(j.n_steps)
        torch.cuda.synchronize()
        assert np.array_equal(j.state["pos"].cpu().numpy(), eng.pos.cpu().numpy()), j.id
        assert np.array_equal(j.state["vel"].cpu().numpy(), eng.vel.cpu().numpy()), j.id
        assert np.array_equal(j.state["forces"].cpu().numpy(), eng.forces.cpu().numpy()), j.id
        assert j.pairs > 0


def test_fifo_alone_model():
    class J:
        def __init__(self, a, p):
            self.arrival, self.pairs = a, p
    jobs = [J(0.0, 10), J(0.5, 10), J(0.6, 10)]
    r = serve.fifo_alone(jobs, [1.0, 1.0, 1.0])
    # finishes at 1, 2, 3 -> latencies 1, 1.5, 2.4
    assert r["latency_p50_s"] == pytest.approx(1.5)
    assert r["pairs_per_s"] == pytest.approx(10.0)
