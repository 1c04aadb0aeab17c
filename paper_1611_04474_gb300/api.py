"""Thin Python binding of the C ABI in include/md_nonbonded.h (argument marshalling only).

Every computation runs in the CUDA kernels of libmdnb.so; this module checks
tensor dtypes, devices and shapes, passes raw device pointers and the current
CUDA stream, and turns negative return codes into exceptions.  There is no CPU
path: if the library is missing, ``load()`` raises.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import numpy as np
import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libmdnb.so")

ACCUM_F32 = 0
ACCUM_FIXED64 = 1
ACCUM_F64 = 2
ACCUM_FIXED_TILE = 3
ALGO_DEFAULT = 0
ALGO_FULL_SHELL = 1
ALGO_HALF_SHELL = 2
ALGO_CLUSTER = 3
STATUS_NONFINITE = 1
STATUS_FIXED_OVERFLOW = 2
STATUS_BAD_TYPE = 4
FIXED_SCALE = 2.0**32

EXPORTS = ("md_strerror", "md_abi_version", "md_cell_dims", "md_workspace_bytes", "md_build_cells",
           "md_build_cells_noalloc", "md_nonbonded_forces", "md_nonbonded_forces_algo", "md_step",
           "md_verlet_workspace_bytes", "md_step_verlet",
           "md_batch_workspace_bytes", "md_batch_prepare", "md_batch_staging_bytes",
           "md_batch_prepare_staged", "md_batch_step", "md_batch_step_tuned")
BATCH_SHAPES = 6  # MD_BATCH_SHAPES: kernel shapes of the batched force launches

_lib = None


class MDError(RuntimeError):
    def __init__(self, fn: str, code: int, text: str):
        super().__init__(f"{fn} failed: {text} ({code})")
        self.code = code


class md_forcefield(ctypes.Structure):
    _fields_ = [("ntypes", ctypes.c_int32), ("reserved", ctypes.c_int32),
                ("AB", ctypes.c_void_p), ("k_coulomb", ctypes.c_double), ("rc", ctypes.c_double)]


class md_system_desc(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int32), ("reserved", ctypes.c_int32),
                ("box_L", ctypes.c_double * 3), ("ff", md_forcefield)]


class md_batch_tuning(ctypes.Structure):
    _fields_ = [("shape_regular", ctypes.c_int32), ("shape_small", ctypes.c_int32)]


def load(path: str | None = None):
    """Load libmdnb.so (built by ``__graft_entry__.build()``).  Raises if it is missing."""
    global _lib
    if _lib is not None and path is None:
        return _lib
    p = path or LIB_PATH
    if not os.path.exists(p):
        raise RuntimeError(f"{p} is missing: build it with `python -c 'import __graft_entry__ as g; "
                           f"g.build()'` (there is no fallback implementation)")
    lib = ctypes.CDLL(p)
    V, P, i32, f64, sz = None, ctypes.c_void_p, ctypes.c_int32, ctypes.c_double, ctypes.c_size_t
    lib.md_strerror.argtypes = [ctypes.c_int]
    lib.md_strerror.restype = ctypes.c_char_p
    lib.md_abi_version.argtypes = []
    lib.md_abi_version.restype = ctypes.c_int
    lib.md_cell_dims.argtypes = [P, f64, P]
    lib.md_cell_dims.restype = ctypes.c_int
    lib.md_workspace_bytes.argtypes = [i32, P]
    lib.md_workspace_bytes.restype = sz
    lib.md_build_cells.argtypes = [P, P, i32, P, P, P, P, P, P, P, sz, P, P]
    lib.md_build_cells.restype = ctypes.c_int
    lib.md_nonbonded_forces.argtypes = [P, P, P, P, i32, P, P, P, i32, P, P, P, P, sz, P, P]
    lib.md_nonbonded_forces.restype = ctypes.c_int
    lib.md_nonbonded_forces_algo.argtypes = [P, P, P, P, i32, P, P, P, i32, i32, P, P, P, P, sz,
                                             P, P]
    lib.md_nonbonded_forces_algo.restype = ctypes.c_int
    lib.md_step.argtypes = [P, P, P, i32, P, P, P, i32, P, P, i32, f64, i32, P, P, sz, P, P]
    lib.md_step.restype = ctypes.c_int
    lib.md_verlet_workspace_bytes.argtypes = [i32, P, f64, f64]
    lib.md_verlet_workspace_bytes.restype = sz
    lib.md_step_verlet.argtypes = [P, P, P, i32, P, P, P, i32, P, P, i32, f64, i32, f64, P, P, P, sz,
                                   P, P]
    lib.md_step_verlet.restype = ctypes.c_int
    lib.md_batch_workspace_bytes.argtypes = [i32, P]
    lib.md_batch_workspace_bytes.restype = sz
    lib.md_batch_prepare.argtypes = [i32, P, P, sz, P]
    lib.md_batch_prepare.restype = ctypes.c_int
    lib.md_batch_staging_bytes.argtypes = [i32, P]
    lib.md_batch_staging_bytes.restype = sz
    lib.md_batch_prepare_staged.argtypes = [i32, P, P, sz, P, sz, P]
    lib.md_batch_prepare_staged.restype = ctypes.c_int
    lib.md_batch_step.argtypes = [i32, P, P, P, P, i32, P, P, P, i32, f64, i32, P, P, sz, P, P]
    lib.md_batch_step.restype = ctypes.c_int
    lib.md_batch_step_tuned.argtypes = [i32, P, P, P, P, i32, P, P, P, i32, f64, i32, P, P, sz, P,
                                        P, P]
    lib.md_batch_step_tuned.restype = ctypes.c_int
    del V
    if path is None:
        _lib = lib
    return lib


def _check(fn: str, code: int):
    if code != 0:
        raise MDError(fn, code, load().md_strerror(code).decode())


def _ptr(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _need(t, dtype, shape=None, name="tensor"):
    if not isinstance(t, torch.Tensor):
        raise TypeError(f"{name} must be a torch.Tensor")
    if not t.is_cuda:
        raise ValueError(f"{name} must be on a CUDA device")
    if t.dtype != dtype:
        raise TypeError(f"{name} must be {dtype}, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if shape is not None and tuple(t.shape) != tuple(shape):
        raise ValueError(f"{name} must have shape {tuple(shape)}, got {tuple(t.shape)}")


def _stream(stream):
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _box(box):
    return (ctypes.c_double * 3)(*[float(x) for x in box])


def _dims(dims):
    return (ctypes.c_int32 * 3)(*[int(x) for x in dims])


FORCE_DTYPE = {ACCUM_F32: torch.float32, ACCUM_FIXED64: torch.int64, ACCUM_F64: torch.float64,
               ACCUM_FIXED_TILE: torch.int64}


def to_device_async(a, dtype, device):
    """A host array on `device` without a host wait: copied through page-locked memory
    (the caching host allocator keeps that block until the copy has run)."""
    t = torch.as_tensor(np.ascontiguousarray(np.asarray(a, dtype=dtype)))
    if torch.device(device).type != "cuda":
        return t.to(device)
    return t.pin_memory().to(device, non_blocking=True)


# page-locked staging buffers of md_batch_prepare_staged, each kept with an event recorded
# after its copy until that event has completed
_staging_in_flight = []


def _keep_staging(buf, event):
    _staging_in_flight[:] = [(b, e) for b, e in _staging_in_flight if not e.query()]
    _staging_in_flight.append((buf, event))


class ForceField:
    """Force-field constants on the device: AB float32 [T, T, 2], k, rc."""

    def __init__(self, AB, k_coulomb: float, rc: float, device="cuda"):
        AB = to_device_async(AB, np.float32, device).contiguous()
        if AB.dim() != 3 or AB.shape[0] != AB.shape[1] or AB.shape[2] != 2:
            raise ValueError("AB must be [T, T, 2]")
        self.AB = AB
        self.ntypes = int(AB.shape[0])
        self.k_coulomb = float(k_coulomb)
        self.rc = float(rc)
        self._c = md_forcefield(self.ntypes, 0, AB.data_ptr(), self.k_coulomb, self.rc)

    @classmethod
    def from_system(cls, s, device="cuda"):
        return cls(s.AB, s.k_coulomb, s.rc, device)

    @property
    def c(self):
        return ctypes.byref(self._c)


def cell_dims(box, rc):
    d = (ctypes.c_int32 * 3)()
    _check("md_cell_dims", load().md_cell_dims(_box(box), float(rc), d))
    return [int(d[0]), int(d[1]), int(d[2])]


def workspace_bytes(n: int, dims) -> int:
    b = int(load().md_workspace_bytes(int(n), _dims(dims)))
    if b == 0:
        raise ValueError("invalid n or dims")
    return b


def make_workspace(n: int, dims, device="cuda"):
    return torch.empty(workspace_bytes(n, dims), dtype=torch.uint8, device=device)


@dataclass
class CellList:
    dims: list
    cell_start: torch.Tensor  # int32 [ncell+1]
    perm: torch.Tensor  # int32 [n]
    pos_q_sorted: torch.Tensor  # float32 [n, 4]
    type_sorted: torch.Tensor  # int32 [n]


def alloc_cells(n: int, dims, device="cuda") -> CellList:
    ncell = int(np.prod(dims))
    return CellList(list(dims), torch.empty(ncell + 1, dtype=torch.int32, device=device),
                    torch.empty(n, dtype=torch.int32, device=device),
                    torch.empty((n, 4), dtype=torch.float32, device=device),
                    torch.empty(n, dtype=torch.int32, device=device))


def build_cells(pos_q, types, box, dims, workspace, out: CellList | None = None, status=None,
                stream=None) -> CellList:
    """md_build_cells: bin atoms into cells; returns the sorted cell list."""
    n = int(pos_q.shape[0])
    _need(pos_q, torch.float32, (n, 4), "pos_q")
    _need(types, torch.int32, (n,), "types")
    _need(workspace, torch.uint8, None, "workspace")
    cl = out if out is not None else alloc_cells(n, dims, pos_q.device)
    if status is not None:
        _need(status, torch.int32, (1,), "status")
    _check("md_build_cells", load().md_build_cells(
        _ptr(pos_q), _ptr(types), n, _box(box), _dims(dims), _ptr(cl.cell_start), _ptr(cl.perm),
        _ptr(cl.pos_q_sorted), _ptr(cl.type_sorted), _ptr(workspace), workspace.numel(),
        _ptr(status), _stream(stream)))
    return cl


def nonbonded_forces(cl: CellList, box, ff: ForceField, workspace, mode=ACCUM_F32,
                     algo=ALGO_DEFAULT, forces_out=None, energy_virial=None, pair_count=None,
                     status=None, stream=None):
    """md_nonbonded_forces(_algo): forces [n, 3] in input order (dtype by mode)."""
    n = int(cl.perm.shape[0])
    dev = cl.perm.device
    F = forces_out if forces_out is not None else torch.empty((n, 3), dtype=FORCE_DTYPE[mode],
                                                             device=dev)
    _need(F, FORCE_DTYPE[mode], (n, 3), "forces_out")
    if energy_virial is not None:
        _need(energy_virial, torch.float64, (3,), "energy_virial")
    if pair_count is not None:
        _need(pair_count, torch.int64, (1,), "pair_count")
    if status is not None:
        _need(status, torch.int32, (1,), "status")
    _need(workspace, torch.uint8, None, "workspace")
    _check("md_nonbonded_forces_algo", load().md_nonbonded_forces_algo(
        _ptr(cl.cell_start), _ptr(cl.perm), _ptr(cl.pos_q_sorted), _ptr(cl.type_sorted), n,
        _box(box), _dims(cl.dims), ff.c, int(mode), int(algo), _ptr(F), _ptr(energy_virial),
        _ptr(pair_count), _ptr(workspace), workspace.numel(), _ptr(status), _stream(stream)))
    return F


def step(pos, vel, forces, forces_valid: bool, inv_mass, q, types, box, ff: ForceField, mode,
         dt_fs: float, n_steps: int, workspace, energy_log=None, status=None, stream=None):
    """md_step: n_steps of velocity Verlet, in place on pos/vel/forces."""
    n = int(pos.shape[0])
    _need(pos, torch.float64, (n, 3), "pos")
    _need(vel, torch.float64, (n, 3), "vel")
    _need(forces, FORCE_DTYPE[mode], (n, 3), "forces")
    _need(inv_mass, torch.float32, (n,), "inv_mass")
    _need(q, torch.float32, (n,), "q")
    _need(types, torch.int32, (n,), "types")
    _need(workspace, torch.uint8, None, "workspace")
    if energy_log is not None:
        _need(energy_log, torch.float64, (n_steps, 4), "energy_log")
    if status is not None:
        _need(status, torch.int32, (1,), "status")
    _check("md_step", load().md_step(
        _ptr(pos), _ptr(vel), _ptr(forces), int(bool(forces_valid)), _ptr(inv_mass), _ptr(q),
        _ptr(types), n, _box(box), ff.c, int(mode), float(dt_fs), int(n_steps), _ptr(energy_log),
        _ptr(workspace), workspace.numel(), _ptr(status), _stream(stream)))


def verlet_workspace_bytes(n: int, box, rc: float, skin: float) -> int:
    b = int(load().md_verlet_workspace_bytes(int(n), _box(box), float(rc), float(skin)))
    if b == 0:
        raise ValueError("invalid n, box, cutoff or skin (rc + skin must stay below min(L)/2)")
    return b


def step_verlet(pos, vel, forces, forces_valid: bool, inv_mass, q, types, box, ff: ForceField,
                mode, dt_fs: float, n_steps: int, skin: float, workspace, energy_log=None,
                rebuilds=None, status=None, stream=None):
    """md_step_verlet: n_steps of velocity Verlet with cells kept while every atom stays
    within skin/2 of where it was when they were built."""
    n = int(pos.shape[0])
    _need(pos, torch.float64, (n, 3), "pos")
    _need(vel, torch.float64, (n, 3), "vel")
    _need(forces, FORCE_DTYPE[mode], (n, 3), "forces")
    _need(inv_mass, torch.float32, (n,), "inv_mass")
    _need(q, torch.float32, (n,), "q")
    _need(types, torch.int32, (n,), "types")
    _need(workspace, torch.uint8, None, "workspace")
    if energy_log is not None:
        _need(energy_log, torch.float64, (n_steps, 4), "energy_log")
    if rebuilds is not None:
        _need(rebuilds, torch.int64, (1,), "rebuilds")
    if status is not None:
        _need(status, torch.int32, (1,), "status")
    _check("md_step_verlet", load().md_step_verlet(
        _ptr(pos), _ptr(vel), _ptr(forces), int(bool(forces_valid)), _ptr(inv_mass), _ptr(q),
        _ptr(types), n, _box(box), ff.c, int(mode), float(dt_fs), int(n_steps), float(skin),
        _ptr(energy_log), _ptr(rebuilds), _ptr(workspace), workspace.numel(), _ptr(status),
        _stream(stream)))


def forces_to_f64(F: torch.Tensor, mode: int) -> torch.Tensor:
    """Forces of any mode as float64 kcal/mol/A."""
    if mode in (ACCUM_FIXED64, ACCUM_FIXED_TILE):
        return F.to(torch.float64) / FIXED_SCALE
    return F.to(torch.float64)


class Engine:
    """Device-resident state of one system: inputs, cell list, forces, MD state and
    workspace allocated once; every call runs the CUDA path through the C ABI."""

    def __init__(self, system, mode=ACCUM_F32, algo=ALGO_DEFAULT, device="cuda"):
        s = system
        self.system = s
        self.n = s.n
        self.box = [float(x) for x in s.box]
        self.mode = mode
        self.algo = algo
        self.ff = ForceField.from_system(s, device)
        self.dims = cell_dims(self.box, s.rc)
        self.pos_q = torch.as_tensor(s.pos_q()).to(device)
        self.types = torch.as_tensor(s.type).to(device)
        self.q = torch.as_tensor(s.q).to(device)
        self.inv_mass = torch.as_tensor(s.inv_mass).to(device)
        self.pos = torch.as_tensor(s.pos.astype(np.float64)).to(device)
        self.vel = torch.as_tensor(s.vel).to(device)
        self.workspace = make_workspace(self.n, self.dims, device)
        self.cells = alloc_cells(self.n, self.dims, device)
        self.forces = torch.zeros((self.n, 3), dtype=FORCE_DTYPE[mode], device=device)
        self.energy_virial = torch.zeros(3, dtype=torch.float64, device=device)
        self.pair_count = torch.zeros(1, dtype=torch.int64, device=device)
        self.status = torch.zeros(1, dtype=torch.int32, device=device)
        self.forces_valid = False

    def build_cells(self, stream=None):
        return build_cells(self.pos_q, self.types, self.box, self.dims, self.workspace,
                           out=self.cells, status=self.status, stream=stream)

    def compute_forces(self, energy=False, count=False, algo=None, stream=None):
        return nonbonded_forces(self.cells, self.box, self.ff, self.workspace, self.mode,
                                self.algo if algo is None else algo, self.forces,
                                self.energy_virial if energy else None,
                                self.pair_count if count else None, self.status, stream)

    def step(self, n_steps=1, dt_fs=1.0, energy_log=None, stream=None):
        step(self.pos, self.vel, self.forces, self.forces_valid, self.inv_mass, self.q,
             self.types, self.box, self.ff, self.mode, dt_fs, n_steps, self.workspace,
             energy_log=energy_log, status=self.status, stream=stream)
        self.forces_valid = True

    # ------------------------------------------------------------ checkpoints
    def save_state(self, path: str):
        """Write the MD state (positions, velocities, forces of the current mode, whether
        they are valid) with the system's fingerprint to `path` (a numpy .npz); the
        device is synchronised first."""
        torch.cuda.synchronize(self.pos.device)
        np.savez(path, pos=self.pos.cpu().numpy(), vel=self.vel.cpu().numpy(),
                 forces=self.forces.cpu().numpy(), forces_valid=np.int32(self.forces_valid),
                 mode=np.int32(self.mode), fingerprint=np.frombuffer(self.fingerprint(), np.uint8))

    def load_state(self, path: str):
        """Restore a state written by save_state for the same system and mode (raises
        ValueError otherwise); the next step continues bit for bit where it left off."""
        with np.load(path) as z:
            if int(z["mode"]) != self.mode:
                raise ValueError(f"checkpoint mode {int(z['mode'])} != engine mode {self.mode}")
            if bytes(z["fingerprint"].tobytes()) != self.fingerprint():
                raise ValueError("checkpoint belongs to another system")
            for name in ("pos", "vel", "forces"):
                t = getattr(self, name)
                a = z[name]
                if a.shape != tuple(t.shape) or a.dtype != np.dtype(str(t.dtype).replace("torch.", "")):
                    raise ValueError(f"checkpoint {name} has shape {a.shape} / {a.dtype}")
                t.copy_(torch.as_tensor(a))
            self.forces_valid = bool(int(z["forces_valid"]))

    def fingerprint(self) -> bytes:
        """SHA-256 of what fixes the dynamics besides the state: charges, types, masses,
        box, cutoff and the LJ table."""
        import hashlib

        s = self.system
        h = hashlib.sha256()
        for a in (s.q, s.type, s.inv_mass, np.asarray(self.box, np.float64), np.float64(s.rc),
                  np.asarray(s.AB, np.float32), np.float64(s.k_coulomb)):
            h.update(np.ascontiguousarray(a).tobytes())
        return h.digest()

    def step_verlet(self, n_steps=1, dt_fs=1.0, skin=1.0, energy_log=None, stream=None):
        """md_step_verlet on this system's state; the number of cell builds accumulates in
        self.rebuilds (a device int64[1])."""
        need = verlet_workspace_bytes(self.n, self.box, self.ff.rc, skin)
        if getattr(self, "verlet_ws", None) is None or self.verlet_ws.numel() < need:
            self.verlet_ws = torch.empty(need, dtype=torch.uint8, device=self.pos.device)
        if getattr(self, "rebuilds", None) is None:
            self.rebuilds = torch.zeros(1, dtype=torch.int64, device=self.pos.device)
        step_verlet(self.pos, self.vel, self.forces, self.forces_valid, self.inv_mass, self.q,
                    self.types, self.box, self.ff, self.mode, dt_fs, n_steps, skin, self.verlet_ws,
                    energy_log=energy_log, rebuilds=self.rebuilds, status=self.status,
                    stream=stream)
        self.forces_valid = True


class Batch:
    """Independent systems advanced together (md_batch_*): the systems' arrays are
    concatenated on the device; every step is one set of launches for all of them.

    ``state`` (optional) gives the concatenated device arrays directly (keys pos, vel,
    forces, q, types, inv_mass) so that a caller keeping systems on the device builds a
    batch without a host round trip; ``ffs`` likewise reuses device force fields.
    ``tuning`` = (shape for the systems with >= 3 cells per axis, shape for those with an
    axis of 2 cells), each in 0 .. BATCH_SHAPES-1 (md_batch_tuning); a performance choice
    only, see ``autotune``.  ``staged`` prepares the batch through page-locked staging
    memory (md_batch_prepare_staged) without waiting for the stream, for callers that keep
    work queued on it; otherwise md_batch_prepare waits for the stream."""

    def __init__(self, systems, mode=ACCUM_FIXED64, device="cuda", state=None, ffs=None,
                 tuning=(0, 0), staged=False):
        if mode not in (ACCUM_F32, ACCUM_FIXED64, ACCUM_FIXED_TILE):
            raise ValueError("batched mode must be ACCUM_F32, ACCUM_FIXED64 or ACCUM_FIXED_TILE")
        self.systems = list(systems)
        self.mode = mode
        self.nsys = len(self.systems)
        self.ffs = list(ffs) if ffs is not None else [ForceField.from_system(s, device)
                                                      for s in self.systems]
        self.desc = (md_system_desc * self.nsys)()
        for k, (s, ff) in enumerate(zip(self.systems, self.ffs)):
            self.desc[k].n = s.n
            self.desc[k].reserved = 0
            for d in range(3):
                self.desc[k].box_L[d] = float(s.box[d])
            self.desc[k].ff = ff._c
        self.offsets = np.concatenate([[0], np.cumsum([s.n for s in self.systems])]).astype(np.int64)
        self.n = int(self.offsets[-1])
        if state is not None:
            self.pos, self.vel, self.forces = state["pos"], state["vel"], state["forces"]
            self.q, self.types, self.inv_mass = state["q"], state["types"], state["inv_mass"]
            for name, t, dt, shape in (("pos", self.pos, torch.float64, (self.n, 3)),
                                       ("vel", self.vel, torch.float64, (self.n, 3)),
                                       ("forces", self.forces, FORCE_DTYPE[mode], (self.n, 3)),
                                       ("q", self.q, torch.float32, (self.n,)),
                                       ("types", self.types, torch.int32, (self.n,)),
                                       ("inv_mass", self.inv_mass, torch.float32, (self.n,))):
                _need(t, dt, shape, name)
        else:
            cat = lambda f, dt: torch.as_tensor(np.concatenate([f(s) for s in self.systems]).astype(dt)).to(device)
            self.pos = cat(lambda s: s.pos.astype(np.float64), np.float64).contiguous()
            self.vel = cat(lambda s: s.vel, np.float64).contiguous()
            self.q = cat(lambda s: s.q, np.float32)
            self.types = cat(lambda s: s.type, np.int32)
            self.inv_mass = cat(lambda s: s.inv_mass, np.float32)
            self.forces = torch.zeros((self.n, 3), dtype=FORCE_DTYPE[mode], device=device)
        self.pair_count = torch.zeros(self.nsys, dtype=torch.int64, device=device)
        self.status = torch.zeros(1, dtype=torch.int32, device=device)
        nbytes = int(load().md_batch_workspace_bytes(self.nsys, ctypes.byref(self.desc)))
        if nbytes == 0:
            raise ValueError("invalid batch (a cutoff at or above L/2, bad n or force field)")
        self.workspace = torch.empty(nbytes, dtype=torch.uint8, device=device)
        self.forces_valid = False
        self.tuning = tuple(tuning)
        if staged:
            sb = int(load().md_batch_staging_bytes(self.nsys, ctypes.byref(self.desc)))
            buf = torch.empty(sb, dtype=torch.uint8, pin_memory=True)
            _check("md_batch_prepare_staged", load().md_batch_prepare_staged(
                self.nsys, ctypes.byref(self.desc), _ptr(self.workspace), nbytes,
                ctypes.c_void_p(buf.data_ptr()), sb, _stream(None)))
            ev = torch.cuda.Event()
            ev.record()
            _keep_staging(buf, ev)
        else:
            _check("md_batch_prepare", load().md_batch_prepare(
                self.nsys, ctypes.byref(self.desc), _ptr(self.workspace), nbytes,
                _stream(None)))

    def step(self, n_steps=1, dt_fs=1.0, count_pairs=False, stream=None):
        t = md_batch_tuning(int(self.tuning[0]), int(self.tuning[1]))
        _check("md_batch_step_tuned", load().md_batch_step_tuned(
            self.nsys, ctypes.byref(self.desc), _ptr(self.pos), _ptr(self.vel), _ptr(self.forces),
            int(self.forces_valid), _ptr(self.inv_mass), _ptr(self.q), _ptr(self.types),
            int(self.mode), float(dt_fs), int(n_steps),
            _ptr(self.pair_count) if count_pairs else None, _ptr(self.workspace),
            self.workspace.numel(), _ptr(self.status), ctypes.byref(t), _stream(stream)))
        self.forces_valid = True

    def system_slice(self, k):
        return slice(int(self.offsets[k]), int(self.offsets[k + 1]))
