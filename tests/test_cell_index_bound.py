"""The cell index of the GPU build takes floor(x * (n/L)) from an FP32 product and falls
back to the FP64 rule only within 2.5e-7 (relative) of an integer.  This checks the
error bound that decision rests on, on the CPU with IEEE float32 arithmetic: wherever
the FP32 test accepts, its floor equals the FP64 floor, for coordinates on, beside and
between cell faces of boxes with exact and inexact cell edges."""
import numpy as np


def _fast_accepts(x32, inv32):
    t = (x32 * inv32).astype(np.float32)  # one IEEE float32 rounding, as __fmul_rn
    fl = np.floor(t)
    fr = (t - fl).astype(np.float32)
    tol = (t * np.float32(2.5e-7)).astype(np.float32)
    ok = (fr > tol) & (fr < (np.float32(1.0) - tol).astype(np.float32))
    return ok, fl.astype(np.int64)


def _coords(L, n, rng):
    faces = np.array([np.float32(k * L / n) for k in range(n + 1)], np.float32)
    near = [faces]
    up = faces.copy()
    dn = faces.copy()
    for _ in range(4):
        up = np.nextafter(up, np.float32(np.inf))
        dn = np.nextafter(dn, np.float32(-np.inf))
        near += [up, dn]
    rnd = rng.uniform(0.0, L, 200000).astype(np.float32)
    x = np.concatenate(near + [rnd])
    return x[(x >= 0) & (x < np.float32(L))]


def test_fp32_cell_index_agrees_with_fp64_wherever_it_decides():
    rng = np.random.default_rng(3)
    for L, rc in ((36.0, 12.0), (37.3, 12.0), (48.0001, 12.0), (108.86, 12.0), (77.76, 12.0),
                  (435.44, 12.0), (24.0, 4.0), (10.1, 3.4), (1000.0, 9.0)):
        n = max(1, int(np.floor(L / rc)))
        inv64 = n / L
        inv32 = np.float32(inv64)
        x = _coords(L, n, rng)
        ok, fl32 = _fast_accepts(x, inv32)
        fl64 = np.floor(x.astype(np.float64) * inv64).astype(np.int64)
        assert np.array_equal(fl32[ok], fl64[ok]), (L, rc)
        # the band that falls back is narrow: nearly every random coordinate decides in FP32
        assert ok[-200000:].mean() > 0.999, (L, ok[-200000:].mean())
