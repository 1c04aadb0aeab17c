"""Autotuner for the batched force launches (md_batch_tuning).

The batched step launches the half-shell force kernel twice: once over the systems
whose boxes hold >= 3 cells on every axis and once over those with an axis of two
cells (per-pair minimum image).  Each launch can use any of ``api.BATCH_SHAPES``
kernel shapes (warps per block, survivors buffered per warp).  The best shape depends
on the atoms per cell, the number of cells and the LJ table size, so it is measured,
not guessed: the GPU counterpart of the paper's design-space exploration over the
ratio of distance units to force units (Section V, Table VI).

A choice is cached in a JSON file under a key made from what decides it: the
accumulation mode, log2 of the batch's atoms, the cell edge over the cutoff and the
largest LJ table.  The tuner runs the candidate shapes on a copy of the batch's
state, so tuning leaves the batch's trajectory untouched.
"""
from __future__ import annotations

import json
import math
import os
import threading

import numpy as np
import torch

from . import api

DEFAULT_CACHE = os.path.join(os.path.expanduser("~"), ".cache", "mdnb_batch_tuning.json")
_lock = threading.Lock()


def regimes(batch) -> tuple[bool, bool]:
    """(has systems with >= 3 cells on every axis, has systems with an axis of 2)."""
    reg = small = False
    for s in batch.systems:
        d = api.cell_dims(s.box, float(s.rc))
        if min(d) >= 3:
            reg = True
        else:
            small = True
    return reg, small


def cache_key(batch) -> str:
    """Mode, atom-count bucket, cell edge / cutoff bucket and largest type count."""
    ratios = []
    for s in batch.systems:
        d = api.cell_dims(s.box, float(s.rc))
        ratios.extend(float(s.box[k]) / d[k] / float(s.rc) for k in range(3))
    nb = int(math.floor(math.log2(max(batch.n, 1))))
    ratio = round(float(np.mean(ratios)) * 8) / 8 if ratios else 1.0
    nt = max(int(ff.ntypes) for ff in batch.ffs) if batch.ffs else 0
    return f"mode{batch.mode}|n2^{nb}|edge/rc{ratio:.3f}|types{nt}"


def _load(path):
    try:
        with open(path) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def _store(path, key, entry):
    with _lock:
        data = _load(path)
        data[key] = entry
        os.makedirs(os.path.dirname(os.path.abspath(path)), exist_ok=True)
        tmp = f"{path}.{os.getpid()}.tmp"
        with open(tmp, "w") as f:
            json.dump(data, f, indent=1, sort_keys=True)
        os.replace(tmp, path)


def shapes_for(mode) -> list:
    """The kernel shapes a mode can run: MD_ACCUM_FIXED_TILE exists in the cluster kernel
    only (shapes 0 and 5)."""
    if mode == api.ACCUM_FIXED_TILE:
        return [0, 5]
    return list(range(api.BATCH_SHAPES))


def _time_shape(batch, tuning, n_steps, reps):
    """Mean ms of ``batch.step(n_steps)`` with ``tuning`` (state restored by the caller)."""
    batch.tuning = tuning
    batch.step(1)  # warm-up (first launch of an instantiation sets its smem attribute)
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    a.record()
    for _ in range(reps):
        batch.step(n_steps)
    b.record()
    torch.cuda.synchronize()
    return a.elapsed_time(b) / reps


def measure(batch, n_steps=5, reps=3):
    """Time every shape of each present regime, one regime at a time (the other at its
    best so far).  Returns (best tuning, {"regular": [ms...], "small": [ms...]})."""
    saved = {k: getattr(batch, k).clone() for k in ("pos", "vel", "forces", "status")}
    valid = batch.forces_valid
    has_reg, has_small = regimes(batch)
    best = [0, 0]
    times = {}
    try:
        for idx, (name, present) in enumerate((("regular", has_reg), ("small", has_small))):
            if not present:
                continue
            t = []
            for shape in shapes_for(batch.mode):
                trial = list(best)
                trial[idx] = shape
                t.append((_time_shape(batch, tuple(trial), n_steps, reps), shape))
            best[idx] = min(t)[1]
            times[name] = {str(sh): ms for ms, sh in t}
    finally:
        for k, v in saved.items():
            getattr(batch, k).copy_(v)
        batch.forces_valid = valid
        torch.cuda.synchronize()
    return tuple(best), times


def tune(batch, cache_path: str | None = DEFAULT_CACHE, n_steps=5, reps=3, retune=False):
    """Set ``batch.tuning`` from the cache, measuring (and caching) on a miss.  Returns
    the cache entry ``{"tuning": [r, s], "ms": {...}, "measured": bool}``."""
    key = cache_key(batch)
    if cache_path and not retune:
        hit = _load(cache_path).get(key)
        if hit and all(int(v) in shapes_for(batch.mode) for v in hit.get("tuning", [])) \
                and len(hit.get("tuning", [])) == 2:
            batch.tuning = tuple(int(v) for v in hit["tuning"])
            return dict(hit, measured=False, key=key)
    best, times = measure(batch, n_steps=n_steps, reps=reps)
    batch.tuning = best
    entry = {"tuning": list(best), "ms": times, "n_steps": n_steps}
    if cache_path:
        _store(cache_path, key, entry)
    return dict(entry, measured=True, key=key)
