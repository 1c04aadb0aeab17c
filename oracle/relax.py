"""Capped steepest descent with the FP64 oracle's forces (test infrastructure).

Produces the relaxed start state of the NVE control run: the positions move along the
oracle's forces, x <- x + s F with s = max_step / max_i |F_i|, so that the atom under
the largest force moves exactly max_step and every other atom proportionally less; the
positions are wrapped into the box after each step.  The paper prescribes no start
state; this only removes the overlaps of a lattice whose LJ cores were drawn at random,
so that the control run starts near equilibrium.

Every force evaluation is the oracle's (orc_forces_atoms over the whole cell list),
split over worker processes by atoms: each worker computes the forces on a contiguous
slice of atoms from positions in shared memory.  The workers are started with the
'spawn' method (never forked from a process that may hold a CUDA context).  The result
is cached on disk, keyed by a hash of every input, so that repeated runs reuse it.
"""
from __future__ import annotations

import hashlib
import multiprocessing as mp
import os
import tempfile
from multiprocessing import shared_memory

import numpy as np

_W = {}


def _init(shm_name, n, q, types, box, A, B, k, rc):
    import oracle

    _W["shm"] = shared_memory.SharedMemory(name=shm_name)
    _W["pos"] = np.ndarray((n, 3), dtype=np.float64, buffer=_W["shm"].buf)
    _W["args"] = (q, types, box, oracle.ForceField(A, B, k, rc))


def _forces_slice(bounds):
    import oracle

    lo, hi = bounds
    q, types, box, ff = _W["args"]
    F, _, _ = oracle.forces_atoms(_W["pos"].copy(), q, types, box, ff,
                                  np.arange(lo, hi, dtype=np.int32))
    return lo, F


def _cache_path(pos, q, types, box, ff, n_steps, max_step):
    h = hashlib.sha256()
    for a in (pos, q, types, box, ff.A, ff.B):
        h.update(np.ascontiguousarray(a).tobytes())
    h.update(repr((float(ff.k), float(ff.rc), int(n_steps), float(max_step))).encode())
    base = os.environ.get("MDNB_CACHE_DIR") or os.path.join(tempfile.gettempdir(), "mdnb_oracle_cache")
    return os.path.join(base, f"relaxed_{h.hexdigest()[:24]}.npy")


def steepest_descent(pos, q, types, box, ff, n_steps: int = 200, max_step: float = 0.01,
                     workers: int | None = None, cache: bool = True):
    """Positions (float64 [N, 3]) after n_steps capped steepest-descent steps."""
    import oracle

    pos = np.ascontiguousarray(np.asarray(pos, dtype=np.float64))
    q = np.asarray(q, dtype=np.float64)
    types = np.asarray(types, dtype=np.int32)
    box = np.asarray(box, dtype=np.float64)
    path = _cache_path(pos, q, types, box, ff, n_steps, max_step) if cache else None
    if path and os.path.exists(path):
        return np.load(path)
    n = pos.shape[0]
    workers = workers or min(os.cpu_count() or 1, 32)
    shm = shared_memory.SharedMemory(create=True, size=pos.nbytes)
    try:
        x = np.ndarray(pos.shape, dtype=np.float64, buffer=shm.buf)
        x[:] = np.mod(pos, box)
        chunks = np.linspace(0, n, workers + 1).astype(int)
        bounds = [(int(a), int(b)) for a, b in zip(chunks[:-1], chunks[1:]) if b > a]
        ctx = mp.get_context("spawn")
        with ctx.Pool(len(bounds), initializer=_init,
                      initargs=(shm.name, n, q, types, box, ff.A, ff.B, ff.k, ff.rc)) as pool:
            F = np.zeros((n, 3))
            for _ in range(n_steps):
                for lo, f in pool.map(_forces_slice, bounds):
                    F[lo:lo + f.shape[0]] = f
                fmax = np.linalg.norm(F, axis=1).max()
                if fmax > 0:
                    x += (max_step / fmax) * F
                    x[:] = np.mod(x, box)
                    x[x >= box] -= np.broadcast_to(box, x.shape)[x >= box]  # [0, L)
        out = x.copy()
    finally:
        shm.close()
        shm.unlink()
    if path:
        os.makedirs(os.path.dirname(path), exist_ok=True)
        tmp = path + f".{os.getpid()}.tmp"
        np.save(tmp, out)
        os.replace(tmp if tmp.endswith(".npy") else tmp + ".npy", path)
    return out
