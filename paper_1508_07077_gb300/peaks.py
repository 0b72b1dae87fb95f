"""Measured ALU-pipe ceilings of the GPU (``libhpmc_peaks.so``), the
denominators of the roofline fractions the benchmark reports.

The implicit-depletant path is bound by integer and floating-point issue,
not by tensor cores or HBM, so its ceilings are measured with
microbenchmarks on the GPU that runs it: Philox4x32-10 calls/s in both of the
library's forms (key bumped per round; round keys precomputed), FP32 FMA/s
and FP64 FMA/s, each the best of three launches over every SM."""
from __future__ import annotations

import ctypes
import os

_LIB = os.path.join(os.path.dirname(os.path.abspath(__file__)), "_lib", "libhpmc_peaks.so")


def measure() -> dict:
    """Rates on the current CUDA device (needs the library built)."""
    if not os.path.exists(_LIB):
        raise ImportError("libhpmc_peaks.so not built: " + _LIB)
    lib = ctypes.CDLL(_LIB)
    out = (ctypes.c_double * 5)()
    lib.hpmc_pipe_peaks.argtypes = [ctypes.POINTER(ctypes.c_double)]
    lib.hpmc_pipe_peaks.restype = ctypes.c_int
    if lib.hpmc_pipe_peaks(out) != 0:
        raise RuntimeError("hpmc_pipe_peaks failed")
    return {"philox_calls_per_s": out[0], "philox_rk_calls_per_s": out[4],
            "ffma_per_s": out[1], "dfma_per_s": out[2], "sms": int(out[3])}
