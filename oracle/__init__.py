"""FP64 CPU oracle for the cutoff non-bonded force path (test infrastructure).

Only the tests, ``__graft_entry__.smoke()`` and the benchmark's CPU-baseline leg
use this package.  The CUDA product path never imports it and shares no code
with it.  ``oracle.c`` holds the arithmetic (Eq. 1-2 and Algorithm 1 of the
paper, Section II.A); this module only marshals numpy arrays into it.

Every function takes positions as float64 [N, 3] (the float32 inputs promoted
exactly), charges float64 [N], types int32 [N], the box as float64 [3] and the
A/B tables as float64 [T, T].
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

ACCEL = 4.184e-4  # (kcal/mol/A)/amu in A/fs^2, the same constant oracle.c uses


def build(force: bool = False) -> str:
    """Compile oracle.c with gcc (IEEE semantics: no fast-math, no FMA contraction)."""
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-std=c99", "-fPIC", "-shared", "-ffp-contract=off", "-fno-fast-math",
               "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIB_PATH)
            P = ctypes.c_void_p
            i32, f64, i64 = ctypes.c_int, ctypes.c_double, ctypes.c_longlong
            lib.orc_cell_dims.argtypes = [P, f64, P]
            lib.orc_build_cells.argtypes = [i32, P, P, P, P, P, P]
            lib.orc_pair.argtypes = [P, P, P, f64, f64, f64, f64, f64, f64, P, P]
            lib.orc_forces_cells.argtypes = [i32, P, P, P, P, i32, P, P, f64, f64, P, P, P, P, P, P]
            lib.orc_forces_atoms.argtypes = [i32, P, P, P, P, i32, P, P, f64, f64, i32, P, P, P, P]
            lib.orc_forces_brute.argtypes = [i32, P, P, P, P, i32, P, P, f64, f64, P, P, P]
            lib.orc_boundary_pairs.argtypes = [i32, P, P, f64, f64, i32, P, P]
            lib.orc_boundary_pairs.restype = i64
            lib.orc_kinetic_energy.argtypes = [i32, P, P]
            lib.orc_kinetic_energy.restype = f64
            lib.orc_vv_steps.argtypes = [i32, P, P, P, i32, P, P, P, P, i32, P, P, f64, f64, f64,
                                         i32, i32, P]
            for name in ("orc_cell_dims", "orc_build_cells", "orc_pair", "orc_forces_cells",
                         "orc_forces_atoms", "orc_forces_brute", "orc_vv_steps"):
                getattr(lib, name).restype = i32
            _lib = lib
    return _lib


def _p(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _f64(a, shape=None):
    out = np.ascontiguousarray(np.asarray(a, dtype=np.float64))
    return out.reshape(shape) if shape is not None else out


def _i32(a):
    return np.ascontiguousarray(np.asarray(a, dtype=np.int32))


class ForceField:
    """A/B tables (float64 [T,T]), Coulomb constant and cutoff, as the oracle takes them."""

    def __init__(self, A, B, k, rc):
        self.A = _f64(A)
        self.B = _f64(B)
        self.ntypes = int(self.A.shape[0])
        self.k = float(k)
        self.rc = float(rc)

    @classmethod
    def from_system(cls, s):
        AB = np.asarray(s.AB, dtype=np.float64)
        return cls(AB[..., 0], AB[..., 1], s.k_coulomb, s.rc)


def cell_dims(box, rc):
    lib = _load()
    L = _f64(box)
    dims = np.zeros(3, dtype=np.int32)
    if lib.orc_cell_dims(_p(L), float(rc), _p(dims)):
        raise ValueError("bad box or cutoff")
    return dims


def build_cells(pos, box, rc):
    """(cell_of[N], cell_start[ncell+1], order[N]) under the oracle's cell rule."""
    lib = _load()
    pos = _f64(pos)
    L = _f64(box)
    dims = cell_dims(box, rc)
    n = pos.shape[0]
    ncell = int(np.prod(dims))
    cell_of = np.zeros(n, np.int32)
    cell_start = np.zeros(ncell + 1, np.int32)
    order = np.zeros(n, np.int32)
    rcode = lib.orc_build_cells(n, _p(pos), _p(L), _p(dims), _p(cell_of), _p(cell_start),
                                _p(order))
    if rcode:
        raise RuntimeError(f"orc_build_cells failed ({rcode})")
    return dims, cell_of, cell_start, order


def pair(xi, xj, box, qi, qj, A, B, k, rc):
    """Force on i from j and (U_LJ, U_C); zero when r^2 >= rc^2."""
    lib = _load()
    F = np.zeros(3)
    U = np.zeros(2)
    lib.orc_pair(_p(_f64(xi)), _p(_f64(xj)), _p(_f64(box)), float(qi), float(qj), float(A),
                 float(B), float(k), float(rc), _p(F), _p(U))
    return F, U


class Result:
    def __init__(self, F, energy, npairs, cond=None, fabs_sum=None, energy_abs=None):
        self.F = F  # float64 [N, 3]
        self.energy = energy  # float64 [3]: E_LJ, E_C, W
        self.energy_abs = energy_abs  # float64 [3]: the same sums over absolute term sizes
        self.npairs = npairs  # unique pairs within the cutoff
        self.cond = cond  # float64 [N]
        self.fabs_sum = fabs_sum  # float64 [N]


def forces_cells(pos, q, types, box, ff: ForceField, with_cond: bool = True) -> Result:
    """O1: full-shell cell-list forces in Algorithm 1 loop order."""
    lib = _load()
    pos = _f64(pos)
    n = pos.shape[0]
    F = np.zeros((n, 3))
    en = np.zeros(3)
    cond = np.zeros(n) if with_cond else None
    fabs_sum = np.zeros(n) if with_cond else None
    npairs = ctypes.c_longlong(0)
    eabs = np.zeros(3)
    rcode = lib.orc_forces_cells(n, _p(pos), _p(_f64(q)), _p(_i32(types)), _p(_f64(box)),
                                 ff.ntypes, _p(ff.A), _p(ff.B), ff.k, ff.rc, _p(F), _p(en),
                                 _p(cond) if with_cond else None,
                                 _p(fabs_sum) if with_cond else None, ctypes.byref(npairs),
                                 _p(eabs))
    if rcode:
        raise RuntimeError(f"orc_forces_cells failed ({rcode})")
    return Result(F, en, int(npairs.value), cond, fabs_sum, eabs)


def forces_atoms(pos, q, types, box, ff: ForceField, sel):
    """Forces (and term sizes, partner counts) on the atoms listed in ``sel`` only."""
    lib = _load()
    pos = _f64(pos)
    sel = _i32(sel)
    m = sel.shape[0]
    F = np.zeros((m, 3))
    cond = np.zeros(m)
    npart = np.zeros(m, np.int32)
    rcode = lib.orc_forces_atoms(pos.shape[0], _p(pos), _p(_f64(q)), _p(_i32(types)),
                                 _p(_f64(box)), ff.ntypes, _p(ff.A), _p(ff.B), ff.k, ff.rc, m,
                                 _p(sel), _p(F), _p(cond), _p(npart))
    if rcode:
        raise RuntimeError(f"orc_forces_atoms failed ({rcode})")
    return F, cond, npart


def forces_brute(pos, q, types, box, ff: ForceField) -> Result:
    """O2: every pair i<j, minimum image."""
    lib = _load()
    pos = _f64(pos)
    n = pos.shape[0]
    F = np.zeros((n, 3))
    en = np.zeros(3)
    npairs = ctypes.c_longlong(0)
    rcode = lib.orc_forces_brute(n, _p(pos), _p(_f64(q)), _p(_i32(types)), _p(_f64(box)),
                                 ff.ntypes, _p(ff.A), _p(ff.B), ff.k, ff.rc, _p(F), _p(en),
                                 ctypes.byref(npairs))
    if rcode:
        raise RuntimeError(f"orc_forces_brute failed ({rcode})")
    return Result(F, en, int(npairs.value))


def boundary_pairs(pos, box, rc, window, max_out=100000):
    """Pairs (i<j) with |r^2 - rc^2| <= window, and their r^2."""
    lib = _load()
    pos = _f64(pos)
    ij = np.zeros((max_out, 2), np.int32)
    r2 = np.zeros(max_out)
    cnt = lib.orc_boundary_pairs(pos.shape[0], _p(pos), _p(_f64(box)), float(rc), float(window),
                                 max_out, _p(ij), _p(r2))
    if cnt < 0:
        raise RuntimeError("orc_boundary_pairs failed")
    if cnt > max_out:
        raise RuntimeError(f"{cnt} boundary pairs exceed max_out={max_out}")
    return ij[:cnt].copy(), r2[:cnt].copy()


def kinetic_energy(vel, inv_mass):
    lib = _load()
    vel = _f64(vel)
    return float(lib.orc_kinetic_energy(vel.shape[0], _p(vel), _p(_f64(inv_mass))))


def vv_steps(pos, vel, q, types, box, ff: ForceField, inv_mass, dt, n_steps, F=None,
             f32_positions=True):
    """Velocity Verlet; returns (pos, vel, F, energy_log[n_steps, 4]) as new arrays."""
    lib = _load()
    pos = _f64(pos).copy()
    vel = _f64(vel).copy()
    n = pos.shape[0]
    f_valid = F is not None
    F = _f64(F).copy() if f_valid else np.zeros((n, 3))
    log = np.zeros((max(n_steps, 1), 4))
    rcode = lib.orc_vv_steps(n, _p(pos), _p(vel), _p(F), int(f_valid), _p(_f64(inv_mass)),
                             _p(_f64(q)), _p(_i32(types)), _p(_f64(box)), ff.ntypes, _p(ff.A),
                             _p(ff.B), ff.k, ff.rc, float(dt), int(n_steps), int(f32_positions),
                             _p(log))
    if rcode:
        raise RuntimeError(f"orc_vv_steps failed ({rcode})")
    return pos, vel, F, log[:n_steps]
