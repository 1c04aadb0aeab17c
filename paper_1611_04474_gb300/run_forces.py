"""Command-line driver: evaluate the non-bonded forces of a workload a few times through
the C ABI (for timing and profiling one kernel in isolation).

    python -m paper_1611_04474_gb300.run_forces --n 92224 --reps 3 --mode f32 --algo 2
"""
from __future__ import annotations

import argparse
import json

import torch

from . import api
from . import workloads as W


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--n", type=int, default=W.APOA1_N, help="atoms of the lattice workload")
    ap.add_argument("--gas", action="store_true", help="the 3,000-atom random gas instead")
    ap.add_argument("--reps", type=int, default=3)
    ap.add_argument("--mode", default="f32", choices=["f32", "fixed64", "f64", "fixed_tile"])
    ap.add_argument("--algo", type=int, default=0)
    ap.add_argument("--energy", action="store_true")
    args = ap.parse_args(argv)
    mode = {"f32": api.ACCUM_F32, "fixed64": api.ACCUM_FIXED64, "f64": api.ACCUM_F64,
            "fixed_tile": api.ACCUM_FIXED_TILE}[args.mode]
    s = W.workload_random_3000() if args.gas else (
        W.workload_lattice_92k() if args.n == W.APOA1_N else W.lattice_box(n=args.n))
    eng = api.Engine(s, mode=mode, algo=args.algo)
    eng.build_cells()
    times = []
    for _ in range(args.reps):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        eng.compute_forces(energy=args.energy, count=True)
        b.record()
        torch.cuda.synchronize()
        times.append(a.elapsed_time(b))
    print(json.dumps({"workload": s.name, "atoms": s.n, "mode": args.mode, "algo": args.algo,
                      "pairs": int(eng.pair_count.item()), "status": int(eng.status.item()),
                      "ms": times}))


if __name__ == "__main__":
    main()
