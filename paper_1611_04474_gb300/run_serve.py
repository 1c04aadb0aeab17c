"""Serving measurement: a Poisson stream of MD jobs through the continuous-batching
server, against serving the same arrivals one job at a time with the plain md_step
path (stand-alone job times measured on a sample of the jobs and fitted as a linear
function of each job's pair count).

    python -m paper_1611_04474_gb300.run_serve --jobs 400 --rate 200
"""
from __future__ import annotations

import argparse
import json

import numpy as np

from . import api
from . import serve
from . import workloads as W


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--jobs", type=int, default=400)
    ap.add_argument("--rate", type=float, default=200.0)
    ap.add_argument("--seed", type=int, default=5)
    ap.add_argument("--tick", type=int, default=10)
    ap.add_argument("--budget-gb", type=float, default=16.0)
    ap.add_argument("--alone-sample", type=int, default=30)
    ap.add_argument("--mode", default="fixed64", choices=["f32", "fixed64"])
    args = ap.parse_args(argv)
    mode = api.ACCUM_F32 if args.mode == "f32" else api.ACCUM_FIXED64
    specs = W.serving_jobs(n_jobs=args.jobs, rate_per_s=args.rate, seed=args.seed)
    jobs = [serve.Job(k, mk, st, arr, n) for k, (mk, st, arr, n) in enumerate(specs)]
    srv = serve.Server(mode=mode, budget_bytes=int(args.budget_gb * (1 << 30)), tick_steps=args.tick)
    res = srv.run(jobs)
    res.update({"mode": args.mode, "rate": args.rate, "tick_steps": args.tick,
                "ticks": srv.ticks, "rebuilds": srv.rebuilds,
                "max_footprint_gb": srv.max_footprint / (1 << 30),
                "loop_seconds": {k: round(v, 3) for k, v in srv.seconds.items()}})
    # stand-alone times on a sample of jobs, fitted as a + b * pairs
    rng = np.random.default_rng(0)
    sample = rng.choice(len(jobs), size=min(args.alone_sample, len(jobs)), replace=False)
    xs, ys = [], []
    for k in sample:
        ys.append(serve.time_alone(jobs[k], mode))
        xs.append(jobs[k].pairs)
    A = np.vstack([np.ones(len(xs)), np.asarray(xs, dtype=np.float64)]).T
    coef = np.linalg.lstsq(A, np.asarray(ys), rcond=None)[0]
    alone = [max(coef[0] + coef[1] * j.pairs, 0.0) for j in jobs]
    res["alone"] = serve.fifo_alone(jobs, alone)
    res["alone_fit"] = {"seconds_fixed": float(coef[0]), "seconds_per_pair": float(coef[1]),
                        "sample": len(sample)}
    print(json.dumps(res))


if __name__ == "__main__":
    main()
