"""ctypes binding of libqhd_probe.so (include/qhd_probe.h): measured arithmetic
rates of the current GPU, used by the benchmark to state roofline peaks."""
from __future__ import annotations

import ctypes
import os

from . import build as _build

_lib = None


def load():
    global _lib
    if _lib is not None:
        return _lib
    _build.build()
    if not os.path.exists(_build.PROBE_LIB):
        raise RuntimeError(f"libqhd_probe.so not built ({_build.PROBE_LIB})")
    lib = ctypes.CDLL(_build.PROBE_LIB)
    lib.qhd_probe_alu_rates.argtypes = [ctypes.POINTER(ctypes.c_double)]
    lib.qhd_probe_alu_rates.restype = ctypes.c_int
    _lib = lib
    return lib


def alu_rates():
    """(FP32 FMAs/s, 32x32->64-bit integer multiply-adds/s, FP64 FMAs/s, hardware
    sine approximations/s) on the current device."""
    out = (ctypes.c_double * 4)()
    st = load().qhd_probe_alu_rates(out)
    if st != 0:
        raise RuntimeError(f"qhd_probe_alu_rates failed with status {st}")
    return tuple(out)
