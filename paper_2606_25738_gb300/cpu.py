"""ctypes binding of libphmm_cpu.so (include/phmm_cpu.h): the row-wise PairHMM forward
pass on the host CPU, one pair per SIMD lane, FP32 with FP64 rescue or FP64.  A
comparator for the GPU library, which never calls it."""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import phmm

LIB_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "_lib", "libphmm_cpu.so")
_lib = None


def _load() -> ctypes.CDLL:
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError("libphmm_cpu.so is not built (%s); run __graft_entry__.build()" % LIB_PATH)
        lib = ctypes.CDLL(LIB_PATH)
        lib.phmm_cpu_forward.argtypes = [ctypes.POINTER(phmm.Batch), ctypes.c_int, ctypes.c_int,
                                         ctypes.c_double]
        _lib = lib
    return _lib


def forward(b: dict, n_threads: int = 0, precision: str = "fp32", tolerance: float = 0.0):
    """log10 L and flags (phmm.PAIR_* bits) of every pair of a host batch, on n_threads
    host threads (0: one per online core); precision "fp32" (FP32 + FP64 rescue), "fp64"
    or "fp32_only"; tolerance: the FP32 pass's accepted error bound (0: 1e-3)."""
    n = len(b["pair_read"])
    out = np.empty(n, dtype=np.float64)
    fl = np.zeros(n, dtype=np.uint8)
    bb, keep = phmm._host_batch(b, out, fl)
    rc = _load().phmm_cpu_forward(ctypes.byref(bb), int(n_threads), phmm.PREC[precision], float(tolerance))
    del keep
    if rc != phmm.PHMM_OK:
        raise phmm.PhmmError(rc, "phmm_cpu_forward")
    return out, fl
