"""Continuous-batching MD server over the batched C ABI.

Jobs (a periodic system and a number of velocity-Verlet steps) arrive over time.  The
server keeps every admitted job's state on the device and advances all active jobs
together in one arena (an md_batch_step over their concatenation), so the work of jobs
that arrived at different times overlaps on the GPU.

A tick advances the arena by up to `tick_steps` steps, split into md_batch_step calls
at the steps where jobs reach their last step: such a job's state is copied out right
after its last step (on the stream, no host wait) and it stays in the arena, advanced
but no longer counted, until the arena is next rebuilt.  The arena is rebuilt between
ticks when the jobs waiting to join carry enough atoms or have waited `max_wait_s`, or
when finished jobs fill half of it; rebuilding copies the live jobs' state from the old
arena (device to device) and recomputes their forces at the current positions.  In
the deterministic modes (MD_ACCUM_FIXED_TILE, the default, and MD_ACCUM_FIXED64) that
recomputation gives the same bits, and a system's result never depends on the other
systems of its batch, so a job's result is the same as running it alone.

The host enqueues ticks ahead of the GPU and learns of finished jobs from CUDA events;
it waits only while more than 2 x `depth` events (ends of ticks and of jobs) are
pending.  A deeper queue buys nothing once the GPU is busy and delays the next arrival,
which joins behind every queued tick.  Nothing else in the loop waits for the stream: job
uploads, batch descriptors and index lists go through page-locked memory
(md_batch_prepare_staged for the descriptors).  Pair counts accumulate on the device and
are read once at the end.

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
    def __init__(self, mode=api.ACCUM_FIXED_TILE, budget_bytes: int = 16 << 30,
                 tick_steps: int = 10, dt_fs: float = 1.0, device="cuda", lookahead: int = 32,
                 depth: int = 1, max_wait_s: float = 0.002, join_fraction: float = 0.2,
                 active_atoms: int = 1_000_000, tick_ms: float = 4.0, done_ratio: float = 2.0):
        self.mode = mode
        self.budget = int(budget_bytes)
        self.tick = int(tick_steps)
        self.dt = float(dt_fs)
        self.device = torch.device(device)
        self.lookahead = int(lookahead)
        self.depth = int(depth)
        self.max_wait = float(max_wait_s)
        self.join_fraction = float(join_fraction)
        # compute admission: jobs join the arena while its live atoms stay below this
        # (enough to fill the GPU; beyond it more company only slows every job down), so
        # that under overload jobs wait in arrival order instead of all sharing the GPU
        self.active_atoms = int(active_atoms)
        # a tick runs about tick_ms of GPU time (at least tick_steps steps), so that the
        # host's work per tick stays small beside the GPU's
        self.tick_ms = float(tick_ms)
        # finished jobs are dropped from the arena once their atoms reach this multiple
        # of the live jobs' atoms (they are still stepped until then)
        self.done_ratio = float(done_ratio)
        self.max_footprint = 0
        self.ticks = 0
        self.calls = 0
        self.rebuilds = 0
        self.ms_per_atom_step = None  # GPU ms per atom-step, from the last completed tick
        # wall seconds of the serving loop by phase (host time; the GPU runs ahead)
        self.seconds = {"upload": 0.0, "rebuild": 0.0, "enqueue": 0.0, "wait": 0.0}

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
        up = api.to_device_async  # through page-locked memory: no wait for the stream
        j.state = {
            "pos": up(s.pos, np.float64, d),
            "vel": up(s.vel, np.float64, d),
            "forces": torch.zeros((s.n, 3), dtype=api.FORCE_DTYPE[self.mode], device=d),
            "q": up(s.q, np.float32, d),
            "types": up(s.type, np.int32, d),
            "inv_mass": up(s.inv_mass, np.float32, d),
        }
        j.remaining = j.n_steps

    def _arena(self, members, prev=None, prev_members=()):
        """A batch over `members`: jobs that were in the previous arena bring their
        current state straight from it (device to device), new jobs from their own."""
        where = {id(j): k for k, j in enumerate(prev_members)}
        keys = ("pos", "vel", "forces", "q", "types", "inv_mass")

        def src(j, key):
            k = where.get(id(j))
            return j.state[key] if k is None else getattr(prev, key)[prev.system_slice(k)]
        state = {key: torch.cat([src(j, key) for j in members]).contiguous() for key in keys}
        return api.Batch([j.system for j in members], mode=self.mode, device=self.device,
                         state=state, ffs=[j.ff for j in members], staged=True)

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
        index = {id(j): k for k, j in enumerate(jobs)}
        dev = self.device
        pairs_dev = torch.zeros(len(jobs), dtype=torch.int64, device=dev)
        status_dev = torch.zeros(1, dtype=torch.int32, device=dev)
        queue = collections.deque()   # arrived, not admitted
        waiting = []                  # admitted, not yet in the arena
        members = []                  # the arena's jobs, in its order (live and finished)
        batch = None
        footprint = 0                 # admitted jobs' memory, finished ones until a rebuild
        inflight = collections.deque()  # (event, jobs whose last step precedes it, timing)
        t0 = time.perf_counter()
        now = lambda: time.perf_counter() - t0  # noqa: E731

        def retire(block):
            # finish times of the jobs whose last step the GPU has completed
            while inflight:
                ev, done, timing = inflight[0]
                if not ev.query():
                    if not block:
                        return
                    t1 = time.perf_counter()
                    ev.synchronize()
                    self.seconds["wait"] += time.perf_counter() - t1
                t = now()
                for j in done:
                    j.finished = t
                if timing is not None and timing[1] > 0:  # (start event, steps, atoms)
                    self.ms_per_atom_step = timing[0].elapsed_time(ev) / (timing[1] * max(timing[2], 1))
                inflight.popleft()
                block = False

        def counts_of(b, mem, which):
            # add the arena's counts of `which` (members) to the jobs' totals, on the stream
            ks = [k for k, j in enumerate(mem) if any(j is x for x in which)]
            if ks:
                sel = api.to_device_async(ks, np.int64, dev)
                dst = api.to_device_async([index[id(mem[k])] for k in ks], np.int64, dev)
                pairs_dev.index_add_(0, dst, b.pair_count.index_select(0, sel))

        while pending or queue or waiting or any(j.remaining for j in members):
            retire(False)
            t = now() if realtime else math.inf
            while pending and pending[0].arrival <= t:
                queue.append(pending.popleft())
            in_flight_atoms = sum(j.n_atoms for j in members if j.remaining > 0) + sum(j.n_atoms for j in waiting)
            while queue and footprint + job_footprint_bytes(queue[0].n_atoms) <= self.budget and (
                    in_flight_atoms == 0 or in_flight_atoms + queue[0].n_atoms <= self.active_atoms):
                j = queue.popleft()
                t1 = time.perf_counter()
                self._load(j)
                self.seconds["upload"] += time.perf_counter() - t1
                with admitted_count:
                    admitted_count.n += 1
                    admitted_count.notify_all()
                j.admitted = now()
                waiting.append(j)
                footprint += job_footprint_bytes(j.n_atoms)
                in_flight_atoms += j.n_atoms
            self.max_footprint = max(self.max_footprint, footprint)
            live = [j for j in members if j.remaining > 0]
            live_atoms = sum(j.n_atoms for j in live)
            done_atoms = sum(j.n_atoms for j in members if j.remaining == 0)
            wait_atoms = sum(j.n_atoms for j in waiting)
            if not live and not waiting:
                if queue and not members:
                    raise RuntimeError(f"job {queue[0].id} alone exceeds the memory budget")
                if not members and pending:
                    retire(True)
                    time.sleep(max(0.0, pending[0].arrival - now()))
                    continue
            done_bytes = sum(job_footprint_bytes(j.n_atoms) for j in members if j.remaining == 0)
            head_fits_after = bool(queue) and footprint - done_bytes + job_footprint_bytes(queue[0].n_atoms) <= self.budget
            rebuild = bool((not live and (waiting or members)) or (
                waiting and (wait_atoms >= self.join_fraction * live_atoms
                             or now() - min(j.admitted for j in waiting) >= self.max_wait)) or (
                members and done_atoms >= self.done_ratio * live_atoms) or (done_bytes and head_fits_after))
            if rebuild:
                t1 = time.perf_counter()
                if batch is not None:
                    counts_of(batch, members, live)
                    status_dev.bitwise_or_(batch.status)
                freed = sum(job_footprint_bytes(j.n_atoms) for j in members if j.remaining == 0)
                new_members = live + waiting
                batch = self._arena(new_members, batch, members) if new_members else None
                members, waiting = new_members, []
                footprint -= freed
                if batch is not None:
                    batch.step(0)  # forces of the current positions
                self.rebuilds += 1
                self.seconds["rebuild"] += time.perf_counter() - t1
                continue
            if not live:
                retire(True)
                if pending:
                    time.sleep(max(0.0, min(self.max_wait, pending[0].arrival - now())))
                continue
            # one tick: md_batch_step calls split where live jobs take their last step
            t1 = time.perf_counter()
            left = self.tick
            arena_atoms = sum(j.n_atoms for j in members)  # finished jobs are stepped too
            if self.ms_per_atom_step:
                left = max(self.tick, min(500, int(self.tick_ms / (self.ms_per_atom_step * arena_atoms))))
            tick_steps = left
            ev0 = torch.cuda.Event(enable_timing=True)
            ev0.record()
            while left > 0:
                live = [j for j in members if j.remaining > 0]
                if not live:
                    break
                k = min(left, min(j.remaining for j in live))
                batch.step(k, dt_fs=self.dt, count_pairs=True)
                self.calls += 1
                left -= k
                done = []
                for j in live:
                    j.remaining -= k
                    if j.remaining == 0:
                        done.append(j)
                if done:
                    # their final state and counts, right after their last step
                    for j in done:
                        sl = batch.system_slice(next(i for i, x in enumerate(members) if x is j))
                        for key in ("pos", "vel", "forces"):
                            j.state[key].copy_(getattr(batch, key)[sl])
                    counts_of(batch, members, done)
                    ev = torch.cuda.Event()
                    ev.record()
                    inflight.append((ev, done, None))
            ev = torch.cuda.Event(enable_timing=True)
            ev.record()
            inflight.append((ev, [], (ev0, tick_steps - left, arena_atoms)))
            self.ticks += 1
            self.seconds["enqueue"] += time.perf_counter() - t1
            while len(inflight) > 2 * self.depth:
                retire(True)
        while inflight:
            retire(True)
        torch.cuda.synchronize()
        if batch is not None:
            status_dev.bitwise_or_(batch.status)
        if int(status_dev.item()) != 0:
            raise RuntimeError(f"device status {int(status_dev.item())} during serving")
        totals = pairs_dev.cpu().numpy()
        for j in jobs:
            j.pairs = int(totals[index[id(j)]])
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


def time_alone(job: Job, mode, system=None) -> float:
    """Device time of the job run alone through md_step (state freshly loaded)."""
    s = system if system is not None else job.make_system()
    eng = api.Engine(s, mode=mode)
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    a.record()
    eng.step(job.n_steps)
    b.record()
    torch.cuda.synchronize()
    return a.elapsed_time(b) / 1e3
