"""Measured FP32 multiply-add throughput of the current GPU (the roofline denominator of
the force kernel, which is bound by FP32 arithmetic issue).

Runs the probe kernels of csrc_probe/fp32_peak.cu (libmdprobe.so): independent
multiply-add chains in every thread over several waves of CTAs per SM, scalar FFMA and
packed FFMA2, each timed with CUDA events; the best of a few launches of each form.
"""
from __future__ import annotations

import ctypes
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
PROBE_PATH = os.path.join(_HERE, "libmdprobe.so")


def _load():
    if not os.path.exists(PROBE_PATH):
        raise RuntimeError(f"{PROBE_PATH} is missing: run __graft_entry__.build()")
    lib = ctypes.CDLL(PROBE_PATH)
    lib.mdp_sm_count.restype = ctypes.c_int
    lib.mdp_fma_run.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_void_p,
                                ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double)]
    lib.mdp_fma_run.restype = ctypes.c_int
    return lib


def measure_fp32_peak(target_ms: float = 150.0, repeats: int = 3, blocks_per_sm: int = 8):
    """{'ffma_tflops', 'ffma2_tflops', 'tflops' (the larger), 'sms', ...}: FP32 FLOP/s
    (2 per multiply-add) of the device on torch's current stream."""
    import torch

    lib = _load()
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    ms, flop = ctypes.c_double(), ctypes.c_double()
    out = {"sms": int(lib.mdp_sm_count()), "blocks_per_sm": blocks_per_sm, "threads": 256,
           "chains_per_thread": 8}
    for name, packed in (("ffma", 0), ("ffma2", 1)):
        iters = 2000
        rc = lib.mdp_fma_run(packed, blocks_per_sm, iters, stream, ctypes.byref(ms), ctypes.byref(flop))
        if rc != 0:
            raise RuntimeError(f"mdp_fma_run failed ({rc})")
        # size one launch to about target_ms
        iters = max(2000, int(iters * target_ms / max(ms.value, 1e-3)))
        best = 0.0
        for _ in range(repeats):
            rc = lib.mdp_fma_run(packed, blocks_per_sm, iters, stream, ctypes.byref(ms),
                                 ctypes.byref(flop))
            if rc != 0:
                raise RuntimeError(f"mdp_fma_run failed ({rc})")
            best = max(best, flop.value / (ms.value * 1e-3) / 1e12)
        out[f"{name}_tflops"] = best
        out[f"{name}_ms"] = ms.value
    out["tflops"] = max(out["ffma_tflops"], out["ffma2_tflops"])
    return out
