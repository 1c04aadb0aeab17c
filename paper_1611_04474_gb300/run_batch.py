"""Batched many-system throughput: the systems advanced together through md_batch_step
(optionally replayed from a captured CUDA graph), against advancing each system alone
with md_step one after the other on the same GPU.  The force launches' kernel shapes
come from the autotuner (``--tuning auto``, the default), a fixed pair, or the default.

    python -m paper_1611_04474_gb300.run_batch --nsys 256 --steps 50 --mode fixed_tile
"""
from __future__ import annotations

import argparse
import json

import torch

from . import api
from . import autotune
from . import workloads as W


def _time(fn, reps=1):
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    a.record()
    for _ in range(reps):
        fn()
    b.record()
    torch.cuda.synchronize()
    return a.elapsed_time(b) / reps


def measure_batch(systems, steps: int, mode: int, tuning=(0, 0), graph: bool = True,
                  alone: bool = True) -> dict:
    """The systems advanced `steps` steps together (a launch loop, and one captured CUDA
    graph replayed), and each alone with md_step one after the other; device times."""
    out = {"nsys": len(systems), "atoms": int(sum(s.n for s in systems)), "steps": steps,
           "tuning": list(tuning)}
    b = api.Batch(systems, mode=mode, tuning=tuning)
    b.step(1, count_pairs=True)  # forces of the start state + one step, outside timing
    torch.cuda.synchronize()
    b.pair_count.zero_()
    t_loop = _time(lambda: b.step(steps, count_pairs=True))
    pairs = float(b.pair_count.sum().item())
    out["pairs_per_step"] = pairs / steps
    out["batch_loop_ms"] = t_loop
    out["pairs_per_s_batch_loop"] = pairs / (t_loop / 1e3)
    if graph:
        # the same steps captured once in a CUDA graph and replayed
        st = torch.cuda.Stream()
        st.wait_stream(torch.cuda.current_stream())
        g = torch.cuda.CUDAGraph()
        with torch.cuda.stream(st):
            b.step(1)  # warm-up on the capture stream
            torch.cuda.synchronize()
            with torch.cuda.graph(g, stream=st):
                b.step(steps, count_pairs=True)
        torch.cuda.synchronize()
        b.pair_count.zero_()
        t_graph = _time(lambda: g.replay())
        out["batch_graph_ms"] = t_graph
        out["pairs_per_s_batch_graph"] = float(b.pair_count.sum().item()) / (t_graph / 1e3)
        out["md_steps_per_s_per_system_graph"] = steps / (t_graph / 1e3)
    out["status"] = int(b.status.item())
    if alone:
        engines = [api.Engine(sy, mode=mode) for sy in systems]
        for e in engines:
            e.step(1)
        torch.cuda.synchronize()

        def run_alone():
            for e in engines:
                e.step(steps)

        t_alone = _time(run_alone)
        out["alone_ms"] = t_alone
        out["pairs_per_s_alone"] = pairs / (t_alone / 1e3)
        out["speedup_vs_alone"] = t_alone / out.get("batch_graph_ms", t_loop)
    return out


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--nsys", type=int, default=256)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--seed", type=int, default=4)
    ap.add_argument("--mode", default="fixed_tile", choices=["f32", "fixed64", "fixed_tile"])
    ap.add_argument("--no-alone", action="store_true")
    ap.add_argument("--tuning", default="auto",
                    help="'auto' (autotuner with its cache), 'retune', or two shapes 'r,s'")
    ap.add_argument("--cache", default=autotune.DEFAULT_CACHE)
    args = ap.parse_args(argv)
    mode = {"f32": api.ACCUM_F32, "fixed64": api.ACCUM_FIXED64,
            "fixed_tile": api.ACCUM_FIXED_TILE}[args.mode]
    systems = W.batch_of_systems(nsys=args.nsys, seed=args.seed)
    tuning = (0, 0)
    extra = {}
    if args.tuning in ("auto", "retune"):
        probe = api.Batch(systems, mode=mode)
        tuned = autotune.tune(probe, cache_path=args.cache, retune=args.tuning == "retune")
        extra["autotune"] = {k: tuned[k] for k in ("key", "tuning", "measured", "ms") if k in tuned}
        tuning = tuple(probe.tuning)
        del probe
    else:
        tuning = tuple(int(v) for v in args.tuning.split(","))
    out = measure_batch(systems, args.steps, mode, tuning=tuning, alone=not args.no_alone)
    out.update(extra)
    out["mode"] = args.mode
    out["rc_clamped"] = sum(bool(s.meta["rc_clamped"]) for s in systems)
    print(json.dumps(out))


if __name__ == "__main__":
    main()
