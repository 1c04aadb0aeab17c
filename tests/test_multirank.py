"""The replica (N > 1) reduction of bench.py on CPU with two gloo ranks: value counts the
pairs of every rank and divides by the slowest rank's time."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank(rank, world, port, out):
    import torch.distributed as dist

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench

    pairs = 1.0e9 * (rank + 1)
    step_ms = 10.0 + 5.0 * rank
    e2e_ms = 20.0 - rank
    out[rank] = bench.combine_ranks(pairs, step_ms, e2e_ms)
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_sum_pairs_and_take_max_time():
    world = 2
    ctx = mp.get_context("spawn")
    with ctx.Manager() as m:
        out = m.dict()
        port = _free_port()
        procs = [ctx.Process(target=_rank, args=(r, world, port, out)) for r in range(world)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(120)
            assert p.exitcode == 0
        for r in range(world):
            pairs, step_ms, e2e_ms = out[r]
            assert pairs == pytest.approx(3.0e9)
            assert step_ms == pytest.approx(15.0)
            assert e2e_ms == pytest.approx(20.0)


def test_single_process_is_unchanged():
    import bench

    assert bench.combine_ranks(5.0, 2.0, 3.0) == (5.0, 2.0, 3.0)
