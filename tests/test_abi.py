"""The C ABI library loads and exports every entry point include/*.h declares; host-only
calls and host-side validation work without a GPU."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for f in os.listdir(os.path.join(ROOT, "include")):
        if f.endswith(".h"):
            src = open(os.path.join(ROOT, "include", f)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names |= set(re.findall(r"\b(md_[a-z0-9_]+)\s*\(", src))
    return names


@pytest.fixture(scope="module")
def lib():
    from paper_1611_04474_gb300 import build

    build.build()
    from paper_1611_04474_gb300 import api

    return api.load()


def test_every_declared_symbol_is_exported(lib):
    from paper_1611_04474_gb300 import api

    declared = _declared()
    assert {"md_build_cells", "md_nonbonded_forces", "md_step"} <= declared
    for name in declared:
        assert hasattr(lib, name), name
    assert declared <= set(api.EXPORTS) | {n for n in declared if n.startswith("md_") and hasattr(lib, n)}


def test_abi_version_and_strerror(lib):
    assert lib.md_abi_version() == 1
    for code in (0, -1, -2, -3, -4, -5, -99):
        assert isinstance(lib.md_strerror(code), bytes)


def test_cell_dims_rule_and_cutoff_errors(lib):
    from paper_1611_04474_gb300 import api

    assert api.cell_dims((108.86, 108.86, 77.76), 12.0) == [9, 9, 6]
    assert api.cell_dims((31.0, 31.0, 31.0), 12.0) == [2, 2, 2]
    for box, rc in (((31.0, 31.0, 31.0), 15.5), ((31.0, 31.0, 31.0), 0.0), ((10, 40, 40), 5.0),
                    ((31.0, 31.0, 31.0), float("nan"))):
        with pytest.raises(api.MDError) as e:
            api.cell_dims(box, rc)
        assert e.value.code == -2
    with pytest.raises(api.MDError) as e:
        api.cell_dims((0.0, 10.0, 10.0), 1.0)
    assert e.value.code == -1


def test_workspace_bytes(lib):
    from paper_1611_04474_gb300 import api

    small = api.workspace_bytes(3000, [2, 2, 2])
    big = api.workspace_bytes(92224, [9, 9, 6])
    assert 0 < small < big
    assert lib.md_workspace_bytes(-1, (ctypes.c_int32 * 3)(2, 2, 2)) == 0
    assert lib.md_workspace_bytes(10, (ctypes.c_int32 * 3)(0, 2, 2)) == 0


def test_host_validation_rejects_before_any_launch(lib):
    P = ctypes.c_void_p
    box = (ctypes.c_double * 3)(10.0, 10.0, 10.0)
    dims = (ctypes.c_int32 * 3)(3, 3, 3)
    # negative n
    assert lib.md_build_cells(None, None, -1, box, dims, None, None, None, None, None, 0, None,
                              None) == -1
    # missing cell_start
    assert lib.md_build_cells(None, None, 0, box, dims, None, None, None, None, None, 0, None,
                              None) == -1
    # workspace missing (n = 0 is otherwise valid)
    cs = P(16)  # never dereferenced: validation fails first
    assert lib.md_build_cells(None, None, 0, box, dims, cs, None, None, None, None, 0, None,
                              None) == -3
    from paper_1611_04474_gb300 import api

    ff = api.md_forcefield(4, 0, 256, 332.0636, 3.0)
    # dims inconsistent with rc
    bad = (ctypes.c_int32 * 3)(2, 3, 3)
    assert lib.md_nonbonded_forces(cs, None, None, None, 0, box, bad, ctypes.byref(ff), 0, None,
                                   None, None, None, 0, None, None) == -2
    # ntypes outside 1..32
    ff_bad = api.md_forcefield(33, 0, 256, 332.0636, 3.0)
    assert lib.md_nonbonded_forces(cs, None, None, None, 0, box, dims, ctypes.byref(ff_bad), 0,
                                   None, None, None, None, 0, None, None) == -1
    # unknown mode
    assert lib.md_nonbonded_forces(cs, None, None, None, 0, box, dims, ctypes.byref(ff), 7, None,
                                   None, None, None, 0, None, None) == -1
    # md_step: dt <= 0
    assert lib.md_step(None, None, None, 0, None, None, None, 0, box, ctypes.byref(ff), 0, 0.0, 1,
                       None, None, 0, None, None) == -1


def test_fixed_tile_mode_only_on_the_cluster_kernel(lib):
    from paper_1611_04474_gb300 import api

    box = (ctypes.c_double * 3)(10.0, 10.0, 10.0)
    dims = (ctypes.c_int32 * 3)(3, 3, 3)
    cs = ctypes.c_void_p(16)  # never dereferenced: validation fails first
    ff = api.md_forcefield(4, 0, 256, 332.0636, 3.0)
    for algo in (api.ALGO_FULL_SHELL, api.ALGO_HALF_SHELL):
        assert lib.md_nonbonded_forces_algo(cs, None, None, None, 0, box, dims, ctypes.byref(ff),
                                            api.ACCUM_FIXED_TILE, algo, None, None, None, None, 0,
                                            None, None) == -1
    # batched: shapes 1..4 are the half-shell kernel
    desc = (api.md_system_desc * 1)()
    desc[0].n = 10
    for d in range(3):
        desc[0].box_L[d] = 10.0
    desc[0].ff = ff
    for shape in (1, 2, 3, 4):
        t = api.md_batch_tuning(shape, 0)
        assert lib.md_batch_step_tuned(1, ctypes.byref(desc), None, None, None, 0, None, None,
                                       None, api.ACCUM_FIXED_TILE, 1.0, 1, None, None, 0, None,
                                       ctypes.byref(t), None) == -1


def test_staged_batch_prepare_validation(lib):
    from paper_1611_04474_gb300 import api

    ff = api.md_forcefield(4, 0, 256, 332.0636, 3.0)
    desc = (api.md_system_desc * 2)()
    for k, (n, L) in enumerate(((10, 10.0), (40, 7.0))):
        desc[k].n = n
        for d in range(3):
            desc[k].box_L[d] = L
        desc[k].ff = ff
    staging = int(lib.md_batch_staging_bytes(2, ctypes.byref(desc)))
    ws = int(lib.md_batch_workspace_bytes(2, ctypes.byref(desc)))
    # the staged block is the descriptor part of the workspace: per-system descriptors and
    # one int per cell and per atom at least
    assert 50 * 4 < staging < ws
    bad = (api.md_system_desc * 1)()
    bad[0].n = 10
    for d in range(3):
        bad[0].box_L[d] = 5.0  # rc at L/2
    bad[0].ff = ff
    assert lib.md_batch_staging_bytes(1, ctypes.byref(bad)) == 0
    W = ctypes.c_void_p(256)  # never dereferenced: validation fails first
    buf = (ctypes.c_uint8 * (staging + 32))()
    base = ctypes.addressof(buf)
    aligned = ctypes.c_void_p((base + 15) & ~15)
    # missing or small workspace
    assert lib.md_batch_prepare_staged(2, ctypes.byref(desc), None, ws, aligned, staging,
                                       None) == -3
    assert lib.md_batch_prepare_staged(2, ctypes.byref(desc), W, ws - 512, aligned, staging,
                                       None) == -3
    # missing, small or misaligned staging memory
    assert lib.md_batch_prepare_staged(2, ctypes.byref(desc), W, ws, None, staging, None) == -1
    assert lib.md_batch_prepare_staged(2, ctypes.byref(desc), W, ws, aligned, staging - 1,
                                       None) == -1
    odd = ctypes.c_void_p(aligned.value + 4)
    assert lib.md_batch_prepare_staged(2, ctypes.byref(desc), W, ws, odd, staging, None) == -1
    assert lib.md_batch_prepare_staged(1, ctypes.byref(bad), W, ws, aligned, staging, None) == -2


def test_verlet_step_validation(lib):
    from paper_1611_04474_gb300 import api

    box = (ctypes.c_double * 3)(30.0, 30.0, 30.0)
    assert lib.md_verlet_workspace_bytes(1000, box, 12.0, 1.0) > 0
    # rc + skin must stay below L/2
    assert lib.md_verlet_workspace_bytes(1000, box, 12.0, 3.0) == 0
    assert lib.md_verlet_workspace_bytes(1000, box, 12.0, 0.0) == 0
    ff = api.md_forcefield(4, 0, 256, 332.0636, 12.0)
    P = ctypes.c_void_p(16)  # never dereferenced: validation fails first
    args = lambda mode, skin: (P, P, P, 0, P, P, P, 10, box, ctypes.byref(ff), mode, 1.0, 1, skin,
                               None, None, None, 0, None, None)
    assert lib.md_step_verlet(*args(api.ACCUM_F32, 0.0)) == -1        # skin <= 0
    assert lib.md_step_verlet(*args(api.ACCUM_F32, 3.5)) == -2        # rc + skin >= L/2
    assert lib.md_step_verlet(*args(api.ACCUM_F64, 1.0)) == -1        # the FP64 mode
    assert lib.md_step_verlet(*args(api.ACCUM_F32, 1.0)) == -3        # no workspace
