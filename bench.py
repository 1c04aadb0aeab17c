#!/usr/bin/env python
"""Throughput benchmark of the cutoff non-bonded MD path on GB300.

One step = one velocity-Verlet MD step of the 92,224-atom ApoA1-box lattice through
the C ABI (md_step: kick, drift + wrap, cell rebuild, forces, kick).  The headline
metric is within-cutoff pair interactions per second (unique pairs with r^2 < rc^2
per step, divided by the device time per step); ms_per_step gives MD steps/s.

Prints ONE JSON line (rank 0).  Multi-GPU runs (torchrun) are independent replicas
(the path has no exchange step): every rank runs the same system, value = all ranks'
pairs / max-over-ranks time, scaling "weak".

--impl reference times the FP64 CPU oracle on the same workload and metric.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "within-cutoff pair interactions/sec"
UNIT = "pairs/s"
L2_FLUSH_BYTES = 256 << 20  # twice the 129 MB L2
# nominal FP32 multiply-add peak (context only; the roofline uses the measured figure)
FP32_LANES_PER_SM = 128
NOMINAL_SMS = 152
NOMINAL_SM_GHZ = 2.07
# algorithmic FLOPs (FMA = 2): per half-shell candidate pair (3 sub, 3 mul, 2 add) and
# per surviving pair (powers, Eq. 1-2 factor, F = f r, reaction)
FLOP_PER_CANDIDATE = 8
FLOP_PER_PAIR = 22


# DRAM bytes of one launch of the dominant kernel (dram__bytes_read.sum +
# dram__bytes_write.sum of k_cluster_rows, the FP32 force kernel, 92,224-atom lattice)
# from one ncu capture, with the SHA-256 of the kernel's sources it was taken on: the
# figure is reported as null once they have changed.
TRAFFIC_CAPTURE = {"bytes": 8233984, "atoms": 92224,
                   "kernel_source_sha256": "a05d780fda0f15f933ad41ab282904bfde9964d76b530e54f4dbde248b3a9ac3"}
KERNEL_SOURCES = [os.path.join(ROOT, "paper_1611_04474_gb300", "csrc", f)
                  for f in ("md_forces_cluster.cu", "md_pairgeom.cuh", "md_internal.cuh")]


def artifact_dir() -> str:
    """Where the raw clock and power samples go: $MDNB_ARTIFACT_DIR when set, else a
    fresh temporary directory (the JSON line carries their summaries either way)."""
    d = os.environ.get("MDNB_ARTIFACT_DIR")
    if not d:
        global _TMP_ARTIFACTS
        if _TMP_ARTIFACTS is None:
            _TMP_ARTIFACTS = tempfile.mkdtemp(prefix="mdnb_bench_")
        d = _TMP_ARTIFACTS
    return d


_TMP_ARTIFACTS = None


def kernel_source_sha256() -> str | None:
    import hashlib

    h = hashlib.sha256()
    try:
        for path in KERNEL_SOURCES:
            with open(path, "rb") as f:
                h.update(f.read())
    except OSError:
        return None
    return h.hexdigest()


def captured_traffic(n_atoms: int):
    sha = kernel_source_sha256()
    if sha is None or sha != TRAFFIC_CAPTURE["kernel_source_sha256"] or n_atoms != TRAFFIC_CAPTURE["atoms"]:
        return None
    return TRAFFIC_CAPTURE["bytes"]


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--n", type=int, default=92224, help="atoms (lattice at ApoA1 density)")
    ap.add_argument("--mode", default="f32", choices=["f32", "fixed64"])
    ap.add_argument("--algo", type=int, default=0)
    ap.add_argument("--no-energy", action="store_true", help="skip the board-energy run")
    ap.add_argument("--dt", type=float, default=1.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the batch, serving and Verlet-skin measurements")
    return ap.parse_args()


def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def workload(n):
    from paper_1611_04474_gb300 import workloads as W

    base = W.workload_lattice_92k() if n == W.APOA1_N else W.lattice_box(n=n, seed=2)
    # sigma halved and masses 12-16 amu: the same atoms, charges, box and cutoff (so the
    # same cell list and pair count), but a force field under which the dynamics stays
    # physical for the timed steps
    return base.with_forcefield(sigma_scale=0.5, mass_range=(12.0, 16.0), seed=22)


def half_shell_candidates(cell_start: np.ndarray, dims) -> int:
    """Candidate pairs of one force evaluation under the half-shell cell-pair scheme:
    n_c (n_c - 1)/2 per home cell plus n_c n_c' over its 13 forward neighbours."""
    nx, ny, nz = dims
    cnt = np.diff(cell_start.astype(np.int64)).reshape(nz, ny, nx)
    total = int((cnt * (cnt - 1) // 2).sum())
    offs = [(1, 0, 0), (-1, 1, 0), (0, 1, 0), (1, 1, 0)]
    offs += [(ox, oy, 1) for oy in (-1, 0, 1) for ox in (-1, 0, 1)]
    seen = set()
    for ox, oy, oz in offs:
        key = (ox % nx, oy % ny, oz % nz)
        if key in seen or key == (0, 0, 0):
            continue
        seen.add(key)
        other = np.roll(cnt, shift=(-oz, -oy, -ox), axis=(0, 1, 2))
        total += int((cnt * other).sum())
    return total


class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.idx = gpu_index
        self.proc = None
        self.path = os.path.join(artifact_dir(), f"clocks_gpu{gpu_index}.csv")

    def start(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.idx), "--query-gpu=" + self.FIELDS,
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.f.close()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": sorted(reasons),
                "samples": len(sm)}


def measure_energy(eng, stream, dev_index: int, seconds: float = 2.0, dt_fs: float = 0.01):
    """Board energy per MD step: a sustained run of steps (about `seconds`) with
    nvidia-smi sampling power.draw every 50 ms; J/step = mean power over the run x the
    event-timed time per step.  The run starts from a copy of the current state with a
    short time step (the cost of a step does not depend on dt) and the state is restored
    afterwards, so the trajectory of the timed steps is not changed."""
    import datetime

    import torch

    saved = {k: getattr(eng, k).clone() for k in ("pos", "vel", "forces", "pos_q")}
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    a.record(stream)
    eng.step(20, dt_fs=dt_fs)
    b.record(stream)
    torch.cuda.synchronize()
    n_steps = max(100, int(seconds * 1e3 / (a.elapsed_time(b) / 20)))
    path = os.path.join(artifact_dir(), f"power_gpu{dev_index}.csv")
    try:
        os.makedirs(os.path.dirname(path), exist_ok=True)
        f = open(path, "w")
        proc = subprocess.Popen(["nvidia-smi", "-i", str(dev_index), "--query-gpu=timestamp,power.draw",
                                 "--format=csv,noheader,nounits", "-lms", "50"],
                                stdout=f, stderr=subprocess.DEVNULL)
    except (OSError, FileNotFoundError):
        return None
    time.sleep(0.5)
    torch.cuda.synchronize()
    t0 = datetime.datetime.now()
    a.record(stream)
    eng.step(n_steps, dt_fs=dt_fs)
    b.record(stream)
    torch.cuda.synchronize()
    t1 = datetime.datetime.now()
    time.sleep(0.2)
    proc.terminate()
    try:
        proc.wait(timeout=5)
    except subprocess.TimeoutExpired:
        proc.kill()
    f.close()
    for k, v in saved.items():
        getattr(eng, k).copy_(v)
    torch.cuda.synchronize()
    ms = a.elapsed_time(b)
    watts = []
    for line in open(path):
        parts = [x.strip() for x in line.split(",")]
        try:
            ts = datetime.datetime.strptime(parts[0], "%Y/%m/%d %H:%M:%S.%f")
            w = float(parts[1])
        except (ValueError, IndexError):
            continue
        if t0 <= ts <= t1:
            watts.append(w)
    if len(watts) < 5:
        return None
    p_mean = statistics.mean(watts)
    return {"joules_per_step": p_mean * ms / 1e3 / n_steps, "mean_power_w": p_mean,
            "ms_per_step": ms / n_steps, "steps": n_steps, "samples": len(watts),
            "dt_fs": dt_fs, "source": "nvidia-smi power.draw, 50 ms samples within the run"}


def measure_peak(dev_index: int):
    """The FP32 multiply-add peak of this GPU (paper_1611_04474_gb300.peak), with the SM
    clock sampled while the probe runs."""
    from paper_1611_04474_gb300 import peak

    clocks = ClockSampler(dev_index)
    clocks.path = clocks.path.replace("clocks_gpu", "clocks_peak_gpu")
    clocks.start()
    time.sleep(0.3)
    out = peak.measure_fp32_peak()
    clk = clocks.stop()
    out["sm_mhz"] = clk.get("sm_mhz")
    out["reasons"] = clk.get("reasons")
    return out


def measure_extras(eng, args):
    """The project's other operating points on this GPU, each with its own timing: the
    256-system batch (FIXED_TILE, CUDA-graph replay, against each system alone with
    md_step), the serving loop on two Poisson windows (against one job at a time, every
    job's stand-alone time measured), and the MD step with a Verlet skin."""
    import torch

    from paper_1611_04474_gb300 import api
    from paper_1611_04474_gb300 import run_batch, run_serve
    from paper_1611_04474_gb300 import workloads as W

    out = {}
    t0 = time.perf_counter()
    systems = W.batch_of_systems()
    b = run_batch.measure_batch(systems, 50, api.ACCUM_FIXED_TILE)
    b64 = run_batch.measure_batch(systems, 50, api.ACCUM_FIXED64, graph=False, alone=False)
    b.update({"mode": "fixed_tile", "workload": "256 systems, N log-uniform 500-20,000, 50 steps",
              "fixed64_batch_loop_ms": b64["batch_loop_ms"],
              "fixed64_pairs_per_s_batch_loop": b64["pairs_per_s_batch_loop"],
              "seconds": time.perf_counter() - t0})
    out["batch"] = b
    t0 = time.perf_counter()
    serve = {}
    for rate, n in ((200.0, 150), (15.0, 100)):
        r = run_serve.serve_window(rate, n, api.ACCUM_FIXED_TILE)
        keep = ("jobs", "latency_p50_s", "latency_p99_s", "pairs_per_s", "offered_jobs_per_s",
                "achieved_jobs_per_s", "rebuilds", "ticks", "alone")
        serve[f"rate_{int(rate)}"] = {k: r[k] for k in keep}
    serve["mode"] = "fixed_tile"
    serve["workload"] = "Poisson arrivals, N log-uniform 1,000-150,000, 10-500 steps"
    serve["seconds"] = time.perf_counter() - t0
    out["serve"] = serve
    t0 = time.perf_counter()
    verlet = {}
    s = eng.system
    for skin in (0.5, 1.0):
        v = api.Engine(s, mode=eng.mode)
        v.step(3, dt_fs=args.dt)
        v.rebuilds = torch.zeros(1, dtype=torch.int64, device=v.pos.device)
        a, z = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        a.record()
        v.step_verlet(100, dt_fs=args.dt, skin=skin)
        z.record()
        torch.cuda.synchronize()
        verlet[f"skin_{skin}"] = {"ms_per_step": a.elapsed_time(z) / 100,
                                  "cell_builds_per_100_steps": int(v.rebuilds.item())}
    verlet["seconds"] = time.perf_counter() - t0
    out["verlet"] = verlet
    return out


def combine_ranks(pairs: float, step_ms: float, e2e_ms: float, device=None):
    """Whole-job figures over the ranks of a replica run: the pairs all ranks processed,
    and the slowest rank's device time (max over ranks).  Works on any initialised
    process group (nccl on GPUs, gloo in the CPU tests)."""
    import torch
    import torch.distributed as dist

    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return pairs, step_ms, e2e_ms
    t = torch.tensor([step_ms, e2e_ms], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    p = torch.tensor([pairs], dtype=torch.float64, device=device)
    dist.all_reduce(p, op=dist.ReduceOp.SUM)
    return float(p[0]), float(t[0]), float(t[1])


def bench_config(s, args, world: int) -> dict:
    """The workload description both arms print (the same config for the same run)."""
    return {"workload": f"lattice_{s.n}_apoa1_box", "atoms": s.n, "box": [float(x) for x in s.box],
            "rc": s.rc, "cells": [int(v) for v in np.floor(s.box / s.rc)],
            "step": "velocity-Verlet MD step (rebuild+forces+VV)",
            "force_field": "8 LJ types, sigma x0.5 (1.25-1.9 A), masses 12-16 amu, q~N(0,0.4)",
            "accum": args.mode, "algo": args.algo, "dt_fs": args.dt,
            "l2": "flushed (256 MB write) before every timed step",
            "parallelism": f"replicas x{world}"}


def cpu_oracle_whole(s, gpu_forces=None):
    """The FP64 oracle as it stands, single-threaded: one whole-system evaluation
    (orc_forces_cells, Algorithm 1 over every cell).  Returns (pairs/s, seconds, accuracy
    of gpu_forces against it on every atom, or None)."""
    import oracle

    ff = oracle.ForceField.from_system(s)
    p = s.pos.astype(np.float64)
    t0 = time.perf_counter()
    ref = oracle.forces_cells(p, s.q, s.type, s.box, ff)
    dt = time.perf_counter() - t0
    acc = None
    if gpu_forces is not None:
        # atoms with a pair whose FP64 r^2 lies within 16 float32 ulps of rc^2 may see that
        # pair kept by one side and dropped by the other; both are correct roundings, so
        # those atoms are left out of the figures (the tests check them separately)
        ij, _ = oracle.boundary_pairs(p, s.box, s.rc, 16 * 2.0**-24 * s.rc * s.rc)
        use = np.ones(s.n, dtype=bool)
        use[ij.ravel()] = False
        dF = np.linalg.norm(gpu_forces - ref.F, axis=1)[use]
        nF = np.linalg.norm(ref.F, axis=1)[use]
        raw = dF / np.maximum(nF, 1e-300)
        worst = int(np.argmax(raw))
        acc = {"atoms_checked": int(use.sum()), "boundary_atoms_excluded": int((~use).sum()),
               "max_err_over_term_sum": float((dF / ref.cond[use]).max()),
               "max_rel_err": float(raw.max()),
               "max_rel_err_atom": {"abs_F": float(nF[worst]), "term_sum": float(ref.cond[use][worst]),
                                    "abs_dF": float(dF[worst])},
               "rms_rel_err": float(np.sqrt((dF**2).sum() / (nF**2).sum())),
               "oracle": "orc_forces_cells, whole system"}
    return ref.npairs / dt, dt, acc


def cpu_oracle_rate(s, seconds: float, seed: int = 0, gpu_forces=None):
    """The FP64 oracle as it stands, single-threaded, on a sample of the workload's atoms:
    forces on sampled atoms over the full cell list.  Returns (pairs/s, sample text,
    accuracy of gpu_forces on the sampled atoms or None)."""
    import oracle

    ff = oracle.ForceField.from_system(s)
    p = s.pos.astype(np.float64)
    rng = np.random.default_rng(seed)
    sample = 2048
    done_pairs = 0.0
    t_total = 0.0
    rounds = 0
    worst_norm, worst_raw, d2, f2 = 0.0, 0.0, 0.0, 0.0
    skip = np.zeros(s.n, dtype=bool)
    if gpu_forces is not None:
        # atoms with a pair whose FP64 r^2 lies within 16 float32 ulps of rc^2 may see that
        # pair kept by one side and dropped by the other; both are correct roundings, so
        # those atoms are left out of the error figures (the tests check them separately)
        ij, _ = oracle.boundary_pairs(p, s.box, s.rc, 16 * 2.0**-24 * s.rc * s.rc)
        skip[ij.ravel()] = True
    while t_total < seconds:
        sel = rng.choice(s.n, size=sample, replace=False).astype(np.int32)
        t0 = time.perf_counter()
        F, cond, npart = oracle.forces_atoms(p, s.q, s.type, s.box, ff, sel)
        t_total += time.perf_counter() - t0
        done_pairs += float(npart.sum()) / 2.0  # each unique pair is met from both sides
        rounds += 1
        if gpu_forces is not None:
            use = ~skip[sel]
            dF = np.linalg.norm(gpu_forces[sel] - F, axis=1)[use]
            worst_norm = max(worst_norm, float((dF / cond[use]).max()))
            worst_raw = max(worst_raw, float((dF / np.linalg.norm(F[use], axis=1)).max()))
            d2 += float((dF**2).sum())
            f2 += float((F[use]**2).sum())
    acc = None
    if gpu_forces is not None:
        acc = {"atoms_checked": rounds * sample, "boundary_atoms_excluded": int(skip.sum()),
               "max_err_over_term_sum": worst_norm, "max_rel_err": worst_raw,
               "rms_rel_err": (d2 / f2) ** 0.5}
    return done_pairs / t_total, (f"oracle full-shell cell-list forces on {rounds} random samples of "
                                  f"{sample} of the {s.n} atoms ({t_total:.1f} s); unique-pair "
                                  f"equivalent = partner count / 2"), acc


def run_reference(args):
    world, rank, local = dist_env()
    if rank != 0:
        return 0
    s = workload(args.n)
    per_step_s = 2.0
    rates = []
    for k in range(args.warmup + args.steps):
        r, sample, _ = cpu_oracle_rate(s, per_step_s, seed=k)
        if k >= args.warmup:
            rates.append(r)
    value = statistics.mean(rates)
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": bench_config(s, args, world),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def run_ours(args):
    import torch

    world, rank, local = dist_env()
    if world > 1:
        import torch.distributed as dist

        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)
    from paper_1611_04474_gb300 import api

    api.load()
    dev = torch.device("cuda", torch.cuda.current_device())
    mode = api.ACCUM_F32 if args.mode == "f32" else api.ACCUM_FIXED64
    s = workload(args.n)
    eng = api.Engine(s, mode=mode, algo=args.algo, device=dev)
    stream = torch.cuda.current_stream(dev)
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)

    # pair count and candidate count of the starting state (counter run, untimed)
    eng.build_cells()
    eng.compute_forces(count=True)
    torch.cuda.synchronize()
    pairs_start = int(eng.pair_count.item())
    candidates = half_shell_candidates(eng.cells.cell_start.cpu().numpy(), eng.dims)
    forces_start = api.forces_to_f64(eng.forces, mode).cpu().numpy()

    # warm-up MD steps
    for _ in range(args.warmup):
        eng.step(1, dt_fs=args.dt)
    torch.cuda.synchronize()

    clocks = ClockSampler(dev.index)
    if world > 1:
        torch.distributed.barrier()
    clocks.start()
    time.sleep(0.3)
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    for k in range(args.steps):
        flush.fill_(k & 0xFF)
        ev[k][0].record(stream)
        eng.step(1, dt_fs=args.dt)
        ev[k][1].record(stream)
    torch.cuda.synchronize()
    step_ms = [a.elapsed_time(b) for a, b in ev]

    # the dominant kernel alone on the final state: forces after a rebuilt cell list
    eng.pos_q[:, :3] = eng.pos.to(torch.float32)
    eng.build_cells()
    fev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
           for _ in range(args.steps)]
    for k in range(args.steps):
        flush.fill_(k & 0xFF)
        fev[k][0].record(stream)
        eng.compute_forces()
        fev[k][1].record(stream)
    torch.cuda.synchronize()
    force_ms = [a.elapsed_time(b) for a, b in fev]
    eng.compute_forces(count=True)
    torch.cuda.synchronize()
    pairs_end = int(eng.pair_count.item())
    status = int(eng.status.item())
    clk = clocks.stop()
    energy = None if args.no_energy else measure_energy(eng, stream, dev.index)
    fp32_peak = measure_peak(dev.index)

    # end to end through the public API with host buffers: the step's state (positions,
    # velocities, forces) lives in one pinned host buffer and one device buffer, so that
    # each step is one copy in, the same md_step as the device-timed steps, and one copy
    # of the new state out
    n = s.n
    sizes = [n * 3 * 8, n * 3 * 8, n * 3 * eng.forces.element_size()]
    offs = [0]
    for b in sizes:
        offs.append(offs[-1] + ((b + 255) // 256) * 256)
    dev_buf = torch.empty(offs[-1], dtype=torch.uint8, device=dev)
    views = [dev_buf[offs[k]:offs[k] + sizes[k]] for k in range(3)]
    pos_d = views[0].view(torch.float64).view(n, 3)
    vel_d = views[1].view(torch.float64).view(n, 3)
    F_d = views[2].view(eng.forces.dtype).view(n, 3)
    pos_d.copy_(eng.pos)
    vel_d.copy_(eng.vel)
    F_d.copy_(eng.forces)
    eng.pos, eng.vel, eng.forces = pos_d, vel_d, F_d
    host_buf = dev_buf.cpu().pin_memory()
    h2d = d2h = offs[-1]
    e2e_ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
              for _ in range(args.steps)]
    for k in range(args.steps):
        flush.fill_(k & 0xFF)
        e2e_ev[k][0].record(stream)
        dev_buf.copy_(host_buf, non_blocking=True)
        eng.step(1, dt_fs=args.dt)
        host_buf.copy_(dev_buf, non_blocking=True)
        e2e_ev[k][1].record(stream)
    torch.cuda.synchronize()
    e2e_ms = [a.elapsed_time(b) for a, b in e2e_ev]

    t_force = statistics.mean(force_ms)
    pairs_per_step = 0.5 * (pairs_start + pairs_end)
    total_pairs, t_step, t_e2e = combine_ranks(pairs_per_step * args.steps, sum(step_ms),
                                               sum(e2e_ms), device=dev)
    value = total_pairs / (t_step / 1e3)
    e2e_value = total_pairs / (t_e2e / 1e3)

    if energy:
        energy["pairs_per_joule"] = pairs_per_step / energy["joules_per_step"]
    flops = FLOP_PER_CANDIDATE * candidates + FLOP_PER_PAIR * pairs_end
    nominal_tflops = NOMINAL_SMS * FP32_LANES_PER_SM * 2 * NOMINAL_SM_GHZ / 1e3
    peak_tflops = fp32_peak["tflops"]
    achieved = flops / (t_force / 1e3) / 1e12
    # per MD step: kick + drift + wrap + cell index and bin (+ scan of the cell counts in
    # its last block), cell sort into cluster order, force kernel, finalize + kick
    # (md_step always runs the default kernel); the counts are zeroed by a memset
    per_step_launches = 4
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": t_step / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32" if mode == api.ACCUM_F32 else "f32+int64",
        "data": "synthetic",
        "config": bench_config(s, args, world),
        "md_steps_per_s": 1e3 * args.steps / t_step,
        "pairs_per_step": pairs_per_step,
        "candidates_per_eval": candidates,
        "force_kernel_ms": t_force,
        "roofline": {"bound": "alu", "achieved": achieved, "peak": peak_tflops, "unit": "TFLOP/s",
                     "frac": achieved / peak_tflops, "traffic": captured_traffic(s.n),
                     "kernel": "md_nonbonded_forces",
                     "flop_per_eval": flops,
                     "work": f"{FLOP_PER_CANDIDATE} FLOP x {candidates} half-shell candidates + "
                             f"{FLOP_PER_PAIR} FLOP x {pairs_end} pairs, over the mean "
                             f"event-timed force call of {t_force:.5f} ms",
                     "peak_basis": "measured: FP32 multiply-add probe (best of FFMA and FFMA2, "
                                   f"{fp32_peak['sms']} SMs, median SM clock "
                                   f"{fp32_peak.get('sm_mhz')} MHz during the probe)",
                     "nominal_peak": nominal_tflops,
                     "frac_of_nominal": achieved / nominal_tflops},
        "fp32_peak": fp32_peak,
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h},
        "gpu_launches": args.steps * per_step_launches,
        "energy": energy,
        "clocks": clk,
        "status": status,
    }
    if rank == 0 and not args.no_extras:
        line.update(measure_extras(eng, args))
    if rank == 0 and not args.no_cpu_baseline:
        from paper_1611_04474_gb300 import workloads as W

        rate, secs, acc = cpu_oracle_whole(s, gpu_forces=forces_start)
        sweep = []
        for small in (W.workload_random_3000(), workload(23056)):
            r, t, _ = cpu_oracle_whole(small)
            sweep.append({"atoms": small.n, "seconds": t, "pairs_per_s": r})
        srate, sample, _ = cpu_oracle_rate(s, 3.0)
        line["cpu_baseline"] = {"value": rate, "unit": UNIT, "cores": 1, "kind": "oracle",
                                "sample": f"one whole-system evaluation of the {s.n}-atom workload "
                                          f"(orc_forces_cells, FP64, single thread, {secs:.1f} s)",
                                "sweep": sweep, "sampled_atoms": {"value": srate, "sample": sample}}
        # the same oracle forces also check the GPU's forces of the starting state
        line["accuracy_vs_oracle"] = acc
    if world > 1:
        torch.distributed.barrier()
        torch.distributed.destroy_process_group()
    if rank == 0:
        print(json.dumps(line), flush=True)
    return 0


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
