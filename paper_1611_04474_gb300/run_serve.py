"""Serving measurement: Poisson streams of MD jobs through the continuous-batching server,
against serving the same arrivals one job at a time with the plain md_step path, whose
stand-alone device time is measured for every job of the window.

    python -m paper_1611_04474_gb300.run_serve --rates 15,50,200 --jobs 300,600,2000
"""
from __future__ import annotations

import argparse
import json

from . import api
from . import serve
from . import workloads as W

MODES = {"f32": api.ACCUM_F32, "fixed64": api.ACCUM_FIXED64, "fixed_tile": api.ACCUM_FIXED_TILE}


def serve_window(rate: float, n_jobs: int, mode: int, seed: int = 5, tick: int = 10,
                 budget_gb: float = 16.0, n_range=(1000, 150000), steps_range=(10, 500),
                 **server_kwargs):
    """One window: serve, then time every job alone; returns the result dict.  A short
    untimed window runs first, so that one-time costs (loading each kernel on its first
    launch, allocator growth) fall outside both measurements."""
    warm = W.serving_jobs(n_jobs=8, rate_per_s=1000.0, seed=seed + 1000, n_range=n_range,
                          steps_range=(10, 20))
    warm_jobs = [serve.Job(k, mk, st, arr, n) for k, (mk, st, arr, n) in enumerate(warm)]
    serve.Server(mode=mode, budget_bytes=int(budget_gb * (1 << 30)), tick_steps=tick,
                 **server_kwargs).run(warm_jobs)
    for j in warm_jobs[:2]:
        serve.time_alone(j, mode, system=j.system)
    specs = W.serving_jobs(n_jobs=n_jobs, rate_per_s=rate, seed=seed, n_range=n_range,
                           steps_range=steps_range)
    jobs = [serve.Job(k, mk, st, arr, n) for k, (mk, st, arr, n) in enumerate(specs)]
    srv = serve.Server(mode=mode, budget_bytes=int(budget_gb * (1 << 30)), tick_steps=tick,
                       **server_kwargs)
    res = srv.run(jobs)
    res.update({"rate": rate, "tick_steps": tick, "ticks": srv.ticks, "step_calls": srv.calls,
                "rebuilds": srv.rebuilds, "max_footprint_gb": srv.max_footprint / (1 << 30),
                "loop_seconds": {k: round(v, 3) for k, v in srv.seconds.items()}})
    # one job at a time: each job's md_step run alone, on the system it was served with
    alone = [serve.time_alone(j, mode, system=j.system) for j in jobs]
    res["alone"] = serve.fifo_alone(jobs, alone)
    res["alone"]["device_seconds"] = float(sum(alone))
    res["alone"]["measured_jobs"] = len(alone)
    return res


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--rates", default="200", help="comma-separated Poisson rates (jobs/s)")
    ap.add_argument("--jobs", default="400", help="comma-separated window sizes, one per rate")
    ap.add_argument("--seed", type=int, default=5)
    ap.add_argument("--tick", type=int, default=10)
    ap.add_argument("--budget-gb", type=float, default=16.0)
    ap.add_argument("--mode", default="fixed_tile", choices=list(MODES))
    ap.add_argument("--active-atoms", type=int, default=None,
                    help="compute admission cap (atoms of live jobs in the arena)")
    ap.add_argument("--depth", type=int, default=None, help="ticks enqueued ahead of the GPU")
    ap.add_argument("--tick-ms", type=float, default=None, help="GPU time a tick aims for")
    args = ap.parse_args(argv)
    rates = [float(x) for x in args.rates.split(",")]
    sizes = [int(x) for x in args.jobs.split(",")]
    if len(sizes) == 1:
        sizes = sizes * len(rates)
    for rate, n in zip(rates, sizes):
        kw = {k: v for k, v in (("active_atoms", args.active_atoms), ("depth", args.depth),
                                ("tick_ms", args.tick_ms)) if v is not None}
        res = serve_window(rate, n, MODES[args.mode], seed=args.seed, tick=args.tick,
                           budget_gb=args.budget_gb, **kw)
        res.update(kw)
        res["mode"] = args.mode
        print(json.dumps(res), flush=True)


if __name__ == "__main__":
    main()
