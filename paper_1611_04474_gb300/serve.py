"""Continuous-batching MD server over the batched C ABI.

Jobs (a periodic system and a number of velocity-Verlet steps) arrive over time.  The
server keeps every admitted job's state on the device and advances all active jobs
together: each tick is one md_batch_step over the current set, so the work of jobs
that arrived at different times overlaps on the GPU.  Between ticks finished jobs
leave and queued jobs join while their device-memory footprint fits the budget
(admission in arrival order).  When the set changes, the active jobs' state is written
back from the batch arena and a new arena is built, and their forces are recomputed
at the current positions; in MD_ACCUM_FIXED64 that recomputation gives the same bits,
so a job's result does not depend on the company it ran in.

Reported per run: job latencies (finish - arrival; p50, p99), the aggregate within-
cutoff pair rate, the achieved against the offered job rate, and the largest
footprint admitted.
"""
from __future__ import annotations

import collections
import math
import threading
import time
from dataclasses import dataclass, field

import numpy as np
import torch

from . import api

# bytes of device memory per atom while a job is active: its state (pos, vel and
# forces 3 x 8 B each, q, type, 1/mass 4 B each) plus its share of the batch
# workspace (cell arrays, sorted copies, accumulators, per-CTA partials)
STATE_BYTES_PER_ATOM = 3 * 24 + 12
WORKSPACE_BYTES_PER_ATOM = 160
JOB_FIXED_BYTES = 64 << 10


def job_footprint_bytes(n_atoms: int) -> int:
    return JOB_FIXED_BYTES + n_atoms * (STATE_BYTES_PER_ATOM + WORKSPACE_BYTES_PER_ATOM)


@dataclass
class Job:
    id: int
    make_system: object  # callable returning the System (drawn when the job is admitted)
    n_steps: int
    arrival: float
    n_atoms: int
    admitted: float = math.nan
    finished: float = math.nan
    pairs: int = 0
    remaining: int = 0
    system: object = None
    ff: object = None
    state: dict = field(default_factory=dict)
    ready: threading.Event = field(default_factory=threading.Event)  # system received


class Server:
    def __init__(self, mode=api.ACCUM_FIXED64, budget_bytes: int = 16 << 30, tick_steps: int = 10,
                 dt_fs: float = 1.0, device="cuda", lookahead: int = 32):
        self.mode = mode
        self.budget = int(budget_bytes)
        self.tick = int(tick_steps)
        self.dt = float(dt_fs)
        self.device = torch.device(device)
        self.lookahead = int(lookahead)
        self.max_footprint = 0
        self.ticks = 0
        self.rebuilds = 0
        # wall seconds of the serving loop by phase
        self.seconds = {"upload": 0.0, "rebuild": 0.0, "ticks": 0.0, "write_back": 0.0}

    # ---------------------------------------------------------------- job state
    def _receive(self, ordered, admitted_count, stop):
        """The request bodies: each job's system is materialised on the host off the
        serving loop, in arrival order, at most `lookahead` jobs ahead of admission (what
        a client upload would deliver with the request)."""
        for k, j in enumerate(ordered):
            with admitted_count:
                while k >= admitted_count.n + self.lookahead and not stop.is_set():
                    admitted_count.wait(0.05)
            if stop.is_set():
                return
            j.system = j.make_system()
            j.ready.set()

    def _load(self, j: Job):
        if not j.ready.is_set():
            j.ready.wait()
        s = j.system
        j.ff = api.ForceField.from_system(s, self.device)
        d = self.device
        j.state = {
            "pos": torch.as_tensor(s.pos.astype(np.float64)).to(d),
            "vel": torch.as_tensor(s.vel).to(d),
            "forces": torch.zeros((s.n, 3), dtype=api.FORCE_DTYPE[self.mode], device=d),
            "q": torch.as_tensor(s.q).to(d),
            "types": torch.as_tensor(s.type).to(d),
            "inv_mass": torch.as_tensor(s.inv_mass).to(d),
        }
        j.remaining = j.n_steps

    def _arena(self, active, prev=None, prev_active=()):
        """A batch over `active`: jobs that were in the previous arena bring their
        current state straight from it (device to device), new jobs from their own."""
        where = {id(j): k for k, j in enumerate(prev_active)}
        keys = ("pos", "vel", "forces", "q", "types", "inv_mass")

        def src(j, key):
            k = where.get(id(j))
            return j.state[key] if k is None else getattr(prev, key)[prev.system_slice(k)]
        state = {key: torch.cat([src(j, key) for j in active]).contiguous() for key in keys}
        return api.Batch([j.system for j in active], mode=self.mode, device=self.device,
                         state=state, ffs=[j.ff for j in active])

    def _write_back(self, batch, active, jobs):
        """The current state of `jobs` (a subset of `active`) into their own tensors."""
        for k, j in enumerate(active):
            if any(j is x for x in jobs):
                sl = batch.system_slice(k)
                for key in ("pos", "vel", "forces"):
                    j.state[key].copy_(getattr(batch, key)[sl])

    # ---------------------------------------------------------------- main loop
    def run(self, jobs, realtime: bool = True):
        """Serve `jobs` (list of Job) until all have finished; returns a stats dict.
        realtime: jobs become visible at their arrival times on the wall clock."""
        pending = collections.deque(sorted(jobs, key=lambda j: j.arrival))
        admitted_count = threading.Condition()
        admitted_count.n = 0
        stop = threading.Event()
        receiver = threading.Thread(target=self._receive, args=(list(pending), admitted_count, stop),
                                    daemon=True)
        receiver.start()
        try:
            return self._serve(pending, admitted_count, realtime)
        finally:
            stop.set()
            receiver.join()

    def _serve(self, pending, admitted_count, realtime):
        jobs = list(pending)
        queue = collections.deque()
        active = []
        footprint = 0
        batch = None
        in_batch = []  # the jobs of `batch`, in its order
        changed = True
        t0 = time.perf_counter()
        now = lambda: time.perf_counter() - t0  # noqa: E731
        while pending or queue or active:
            t = now() if realtime else math.inf
            while pending and pending[0].arrival <= t:
                queue.append(pending.popleft())
            while queue and footprint + job_footprint_bytes(queue[0].n_atoms) <= self.budget:
                j = queue.popleft()
                t1 = time.perf_counter()
                self._load(j)
                self.seconds["upload"] += time.perf_counter() - t1
                with admitted_count:
                    admitted_count.n += 1
                    admitted_count.notify_all()
                j.admitted = now()
                active.append(j)
                footprint += job_footprint_bytes(j.n_atoms)
                changed = True
            self.max_footprint = max(self.max_footprint, footprint)
            if not active:
                if queue:
                    raise RuntimeError(f"job {queue[0].id} alone exceeds the memory budget")
                if pending:
                    time.sleep(max(0.0, pending[0].arrival - now()))
                continue
            if changed:
                t1 = time.perf_counter()
                batch = self._arena(active, batch, in_batch)
                in_batch = list(active)
                batch.step(0)  # forces of the current positions (first call: not yet valid)
                self.rebuilds += 1
                changed = False
                self.seconds["rebuild"] += time.perf_counter() - t1
            k = min(self.tick, min(j.remaining for j in active))
            t1 = time.perf_counter()
            batch.pair_count.zero_()
            batch.step(k, dt_fs=self.dt, count_pairs=True)
            counts = batch.pair_count.cpu().numpy()  # waits for the tick
            self.seconds["ticks"] += time.perf_counter() - t1
            self.ticks += 1
            t = now()
            done = []
            for idx, j in enumerate(active):
                j.remaining -= k
                j.pairs += int(counts[idx])
                if j.remaining == 0:
                    done.append(j)
            if int(batch.status.item()) != 0:
                raise RuntimeError(f"device status {int(batch.status.item())} during serving")
            freed = sum(job_footprint_bytes(j.n_atoms) for j in done)
            head = queue[0] if queue else (pending[0] if pending and realtime and pending[0].arrival <= now() else None)
            joinable = head is not None and footprint - freed + job_footprint_bytes(head.n_atoms) <= self.budget
            if done or joinable:
                t1 = time.perf_counter()
                self._write_back(batch, active, done)
                self.seconds["write_back"] += time.perf_counter() - t1
                for j in done:
                    j.finished = t
                    active.remove(j)
                    footprint -= job_footprint_bytes(j.n_atoms)
                changed = True
        torch.cuda.synchronize()
        return summarize(jobs)


def summarize(jobs):
    lat = np.array([j.finished - j.arrival for j in jobs])
    pairs = float(sum(j.pairs for j in jobs))
    first = min(j.arrival for j in jobs)
    last_arr = max(j.arrival for j in jobs)
    last_fin = max(j.finished for j in jobs)
    span = last_fin - first
    return {"jobs": len(jobs), "latency_p50_s": float(np.percentile(lat, 50)),
            "latency_p99_s": float(np.percentile(lat, 99)), "latency_max_s": float(lat.max()),
            "pairs": pairs, "pairs_per_s": pairs / span, "makespan_s": span,
            "offered_jobs_per_s": (len(jobs) - 1) / max(last_arr - first, 1e-9),
            "achieved_jobs_per_s": len(jobs) / span}


def fifo_alone(jobs, alone_seconds):
    """Latencies of the same arrivals served one job at a time in arrival order, each
    taking its measured stand-alone time."""
    order = sorted(range(len(jobs)), key=lambda k: jobs[k].arrival)
    free = -math.inf
    lat = np.zeros(len(jobs))
    for k in order:
        start = max(free, jobs[k].arrival)
        free = start + alone_seconds[k]
        lat[k] = free - jobs[k].arrival
    pairs = float(sum(j.pairs for j in jobs))
    return {"latency_p50_s": float(np.percentile(lat, 50)), "latency_p99_s": float(np.percentile(lat, 99)),
            "pairs_per_s": pairs / float(sum(alone_seconds))}


def time_alone(job: Job, mode) -> float:
    """Device time of the job run alone through md_step (state freshly loaded)."""
    s = job.make_system()
    eng = api.Engine(s, mode=mode)
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    a.record()
    eng.step(job.n_steps)
    b.record()
    torch.cuda.synchronize()
    return a.elapsed_time(b) / 1e3
