"""md_build_cells_noalloc, the cell build for callers that cannot allocate device memory,
gives the same cell list as md_build_cells (which uses a caller workspace).

Its scratch is a fixed array inside the library shared by every call, so the test makes
two calls in a row on different inputs and checks each against the workspace entry
point: a second call must not see leftovers of the first.  Runs alone in a fresh process
or after the other tests; this file is collected last.
"""
import ctypes

import numpy as np
import pytest
import torch

from paper_1611_04474_gb300 import workloads as W

pytestmark = pytest.mark.gpu

MAX_ATOMS = 131072
MAX_CELLS = 16384


def _lib(api):
    lib = api.load()
    P = ctypes.c_void_p
    lib.md_build_cells_noalloc.argtypes = [P, P, ctypes.c_int32, P, P, P, P, P, P, P, P]
    lib.md_build_cells_noalloc.restype = ctypes.c_int
    return lib


def _noalloc(api, lib, pos_q, types, box, dims, status):
    n = int(pos_q.shape[0])
    cl = api.alloc_cells(n, dims, pos_q.device)
    rc = lib.md_build_cells_noalloc(
        ctypes.c_void_p(pos_q.data_ptr()), ctypes.c_void_p(types.data_ptr()), n,
        (ctypes.c_double * 3)(*box), (ctypes.c_int32 * 3)(*dims),
        ctypes.c_void_p(cl.cell_start.data_ptr()), ctypes.c_void_p(cl.perm.data_ptr()),
        ctypes.c_void_p(cl.pos_q_sorted.data_ptr()), ctypes.c_void_p(cl.type_sorted.data_ptr()),
        ctypes.c_void_p(status.data_ptr()),
        ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert rc == 0, rc
    return cl


def test_noalloc_cell_build_matches_workspace_entry_point(cuda_lib):
    api = cuda_lib
    lib = _lib(api)
    systems = [W.workload_lattice_92k(), W.small_random(1500, (14.0, 15.0, 16.5), rc=3.5, seed=3)]
    for s in systems:  # two calls in a row, different sizes and cell grids
        box = [float(x) for x in s.box]
        dims = api.cell_dims(box, s.rc)
        pos_q = torch.as_tensor(s.pos_q()).cuda()
        types = torch.as_tensor(s.type).cuda()
        st_a = torch.zeros(1, dtype=torch.int32, device="cuda")
        st_b = torch.zeros(1, dtype=torch.int32, device="cuda")
        got = _noalloc(api, lib, pos_q, types, box, dims, st_a)
        ws = api.make_workspace(s.n, dims)
        ref = api.build_cells(pos_q, types, box, dims, ws, status=st_b)
        torch.cuda.synchronize()
        for name in ("cell_start", "perm", "pos_q_sorted", "type_sorted"):
            a = getattr(got, name).cpu().numpy()
            b = getattr(ref, name).cpu().numpy()
            assert np.array_equal(a, b), name
        assert int(st_a.item()) == int(st_b.item()) == 0


def _uniform(n, box, seed):
    rng = np.random.default_rng(seed)
    box = np.asarray(box, dtype=np.float64)
    pos = W.to_f32_in_box(rng.uniform(0.0, 1.0, (n, 3)) * box, box)
    pos_q = np.concatenate([pos, rng.uniform(-1, 1, (n, 1)).astype(np.float32)], axis=1)
    return pos_q, rng.integers(0, 4, n).astype(np.int32), box


def test_noalloc_at_its_limits(cuda_lib):
    """The most atoms and cells the scratch holds: 131,072 atoms over 32 x 32 x 16 = 16,384
    cells fills the array to its last byte and takes the global-histogram path (more than
    8,192 cells); then 131,072 atoms over a small grid (the shared-memory histogram)."""
    api = cuda_lib
    lib = _lib(api)
    cases = [(MAX_ATOMS, (64.0, 64.0, 32.0), 1.99, (32, 32, 16)),
             (MAX_ATOMS, (60.0, 61.0, 62.5), 7.5, (8, 8, 8))]
    for k, (n, box, rc, want) in enumerate(cases):
        pos_q_np, types_np, box64 = _uniform(n, box, seed=k)
        dims = api.cell_dims(box, rc)
        assert tuple(dims) == want
        pos_q = torch.as_tensor(pos_q_np).cuda()
        types = torch.as_tensor(types_np).cuda()
        st_a = torch.zeros(1, dtype=torch.int32, device="cuda")
        st_b = torch.zeros(1, dtype=torch.int32, device="cuda")
        got = _noalloc(api, lib, pos_q, types, list(box), dims, st_a)
        ws = api.make_workspace(n, dims)
        ref = api.build_cells(pos_q, types, list(box), dims, ws, status=st_b)
        torch.cuda.synchronize()
        for name in ("cell_start", "perm", "pos_q_sorted", "type_sorted"):
            assert np.array_equal(getattr(got, name).cpu().numpy(), getattr(ref, name).cpu().numpy()), (k, name)
        assert int(st_a.item()) == int(st_b.item()) == 0


def test_noalloc_rejects_sizes_beyond_its_scratch(cuda_lib):
    api = cuda_lib
    lib = _lib(api)
    box = (ctypes.c_double * 3)(500.0, 500.0, 500.0)
    one = torch.zeros(4, dtype=torch.int32, device="cuda")
    p = ctypes.c_void_p(one.data_ptr())
    # too many atoms (nothing is read: the sizes are rejected first)
    assert lib.md_build_cells_noalloc(p, p, MAX_ATOMS + 1, box, (ctypes.c_int32 * 3)(4, 4, 4), p,
                                      p, p, p, None, None) == -5
    # too many cells
    assert lib.md_build_cells_noalloc(p, p, 10, box, (ctypes.c_int32 * 3)(64, 64, 8), p, p, p, p,
                                      None, None) == -5
