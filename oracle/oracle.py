"""ctypes wrapper around phmm_oracle.c (plain FP64 / long-double cell-by-cell PairHMM).

TEST INFRASTRUCTURE ONLY (see the package docstring).  Every function here follows
Eq. 1-4 of the paper (Section 2) as implemented in phmm_oracle.c; the long-double
variants (``precision="long"``) bound the oracle's own rounding.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "phmm_oracle.c")
_LIBDIR = os.path.join(_HERE, "_lib")
lib_path = os.path.join(_LIBDIR, "libphmm_oracle.so")
_lock = threading.Lock()
_lib = None

_u8p = ctypes.POINTER(ctypes.c_uint8)
_u32p = ctypes.POINTER(ctypes.c_uint32)
_u64p = ctypes.POINTER(ctypes.c_uint64)
_f64p = ctypes.POINTER(ctypes.c_double)
_i32p = ctypes.POINTER(ctypes.c_int)
_i64p = ctypes.POINTER(ctypes.c_long)


def build(force: bool = False) -> str:
    """Compile phmm_oracle.c (double and long double) into one shared library."""
    os.makedirs(_LIBDIR, exist_ok=True)
    if not force and os.path.exists(lib_path) and os.path.getmtime(lib_path) >= os.path.getmtime(_SRC):
        return lib_path
    tmp = lib_path + ".tmp.%d" % os.getpid()
    o_d = os.path.join(_LIBDIR, "orc_d.%d.o" % os.getpid())
    o_l = os.path.join(_LIBDIR, "orc_l.%d.o" % os.getpid())
    flags = ["-O2", "-fPIC", "-std=c11", "-ffp-contract=off"]
    subprocess.check_call(["gcc", *flags, "-c", _SRC, "-o", o_d])
    subprocess.check_call(["gcc", *flags, "-DORC_LONG", "-c", _SRC, "-o", o_l])
    subprocess.check_call(["gcc", "-shared", "-o", tmp, o_d, o_l, "-lm", "-lpthread"])
    os.replace(tmp, lib_path)
    for f in (o_d, o_l):
        os.remove(f)
    return lib_path


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(lib_path)
            for pre in ("orc_", "orcl_"):
                f = getattr(lib, pre + "loglik_probs")
                f.restype = ctypes.c_double
                f.argtypes = [ctypes.c_int, _u8p, _f64p, _f64p, _f64p, _f64p, _f64p, ctypes.c_int,
                              _u8p, ctypes.c_double, ctypes.c_int, _i32p]
                f = getattr(lib, pre + "forward_raw")
                f.restype = ctypes.c_double
                f.argtypes = [ctypes.c_int, _u8p, _f64p, _f64p, _f64p, _f64p, _f64p, ctypes.c_int,
                              _u8p, ctypes.c_double, ctypes.c_int, _i32p, _f64p, _i64p]
                f = getattr(lib, pre + "rowwise_eq7")
                f.restype = ctypes.c_double
                f.argtypes = [ctypes.c_int, _u8p, _f64p, _f64p, _f64p, _f64p, _f64p, ctypes.c_int,
                              _u8p, ctypes.c_double, _i32p]
                f = getattr(lib, pre + "loglik_phred")
                f.restype = ctypes.c_double
                f.argtypes = [ctypes.c_int, _u8p, _u8p, _u8p, _u8p, _u8p, ctypes.c_int, _u8p,
                              ctypes.c_double, ctypes.c_int, _i32p]
                f = getattr(lib, pre + "batch")
                f.restype = ctypes.c_long
                f.argtypes = [_u8p, _u64p, _u8p, _u8p, _u8p, _u8p, _u8p, _u64p, ctypes.c_uint32,
                              _u32p, _u32p, ctypes.c_double, ctypes.c_int, ctypes.c_int, _f64p]
            lib.orc_q_phred.restype = ctypes.c_double
            lib.orc_q_phred.argtypes = [ctypes.c_int]
            _lib = lib
    return _lib


def _pre(precision: str) -> str:
    if precision == "double":
        return "orc_"
    if precision == "long":
        return "orcl_"
    raise ValueError(precision)


def _bytes(x) -> np.ndarray:
    if isinstance(x, (bytes, bytearray)):
        return np.frombuffer(bytes(x), dtype=np.uint8).copy()
    if isinstance(x, str):
        return np.frombuffer(x.encode("ascii"), dtype=np.uint8).copy()
    return np.ascontiguousarray(x, dtype=np.uint8)


def _f64(x, n) -> np.ndarray:
    a = np.ascontiguousarray(np.broadcast_to(np.asarray(x, dtype=np.float64), (n,)), dtype=np.float64)
    return a


def _p(a, t):
    return a.ctypes.data_as(t)


def q_phred(x: int) -> float:
    """q(x) = 10^(-x/10) (Eq. 3, numeric Phred)."""
    return _load().orc_q_phred(int(x))


def _probs_args(read, eps, tmi, tmd, gcp, tmm):
    r = _bytes(read)
    l = len(r)
    eps, tmi, tmd, gcp = (_f64(v, l) for v in (eps, tmi, tmd, gcp))
    tmm = (1.0 - tmi - tmd) if tmm is None else _f64(tmm, l)
    tmm = np.ascontiguousarray(tmm, dtype=np.float64)
    return r, l, eps, tmi, tmd, gcp, tmm


def loglik_probs(read, hap, eps, tmi, tmd, gcp, tmm=None, log2C=1020.0, rescale=1,
                 precision="double") -> float:
    """log10 L from per-row probabilities (Eq. 1-4).  ``tmm`` defaults to 1 - tmi - tmd."""
    lib = _load()
    r, l, eps, tmi, tmd, gcp, tmm = _probs_args(read, eps, tmi, tmd, gcp, tmm)
    h = _bytes(hap)
    st = ctypes.c_int(0)
    v = getattr(lib, _pre(precision) + "loglik_probs")(
        l, _p(r, _u8p), _p(eps, _f64p), _p(tmi, _f64p), _p(tmd, _f64p), _p(gcp, _f64p),
        _p(tmm, _f64p), len(h), _p(h, _u8p), float(log2C), int(rescale), ctypes.byref(st))
    if st.value != 0:
        raise ValueError("invalid oracle input")
    return v


def forward_raw(read, hap, eps, tmi, tmd, gcp, tmm=None, log2C=1020.0, rescale=1,
                precision="double"):
    """(log10 L, S, E) with L * C = S * 2^E: the final Eq. 4 sum before log10."""
    lib = _load()
    r, l, eps, tmi, tmd, gcp, tmm = _probs_args(read, eps, tmi, tmd, gcp, tmm)
    h = _bytes(hap)
    st = ctypes.c_int(0)
    S = ctypes.c_double(0)
    E = ctypes.c_long(0)
    v = getattr(lib, _pre(precision) + "forward_raw")(
        l, _p(r, _u8p), _p(eps, _f64p), _p(tmi, _f64p), _p(tmd, _f64p), _p(gcp, _f64p),
        _p(tmm, _f64p), len(h), _p(h, _u8p), float(log2C), int(rescale), ctypes.byref(st),
        ctypes.byref(S), ctypes.byref(E))
    if st.value != 0:
        raise ValueError("invalid oracle input")
    return v, S.value, E.value


def rowwise_eq7(read, hap, eps, tmi, tmd, gcp, tmm=None, log2C=60.0, precision="double") -> float:
    """The paper's row-wise form (Section 3.1, Eq. 7) evaluated literally; small cases."""
    lib = _load()
    r, l, eps, tmi, tmd, gcp, tmm = _probs_args(read, eps, tmi, tmd, gcp, tmm)
    h = _bytes(hap)
    st = ctypes.c_int(0)
    v = getattr(lib, _pre(precision) + "rowwise_eq7")(
        l, _p(r, _u8p), _p(eps, _f64p), _p(tmi, _f64p), _p(tmd, _f64p), _p(gcp, _f64p),
        _p(tmm, _f64p), len(h), _p(h, _u8p), float(log2C), ctypes.byref(st))
    if st.value != 0:
        raise ValueError("invalid oracle input")
    return v


def loglik_phred(read, hap, base_q, ins_q, del_q, gcp_q, log2C=1020.0, rescale=1,
                 precision="double") -> float:
    """log10 L of one pair from numeric Phred qualities (0..93)."""
    lib = _load()
    r = _bytes(read)
    h = _bytes(hap)
    l = len(r)
    bq, iq, dq, gq = (np.ascontiguousarray(np.broadcast_to(np.asarray(q, dtype=np.uint8), (l,)))
                      for q in (base_q, ins_q, del_q, gcp_q))
    st = ctypes.c_int(0)
    v = getattr(lib, _pre(precision) + "loglik_phred")(
        l, _p(r, _u8p), _p(bq, _u8p), _p(iq, _u8p), _p(dq, _u8p), _p(gq, _u8p), len(h),
        _p(h, _u8p), float(log2C), int(rescale), ctypes.byref(st))
    if st.value != 0:
        raise ValueError("invalid oracle input")
    return v


def batch(b, pairs=None, n_threads: int | None = None, log2C=1020.0, rescale=1,
          precision="double") -> np.ndarray:
    """log10 L for every pair of a batch in the library's layout.

    ``b`` is a mapping with numpy arrays read_bases, read_off, base_q, ins_q, del_q,
    gcp_q, hap_bases, hap_off, pair_read, pair_hap.  ``pairs`` optionally selects a
    subset of pair indices.  NaN marks invalid pairs.
    """
    lib = _load()
    pr = np.ascontiguousarray(b["pair_read"], dtype=np.uint32)
    ph = np.ascontiguousarray(b["pair_hap"], dtype=np.uint32)
    if pairs is not None:
        pairs = np.asarray(pairs, dtype=np.int64)
        pr = np.ascontiguousarray(pr[pairs])
        ph = np.ascontiguousarray(ph[pairs])
    n = len(pr)
    out = np.empty(n, dtype=np.float64)
    if n == 0:
        return out
    if n_threads is None:
        n_threads = os.cpu_count() or 1
    arrs = {key: np.ascontiguousarray(b[key], dtype=np.uint8)
            for key in ("read_bases", "base_q", "ins_q", "del_q", "gcp_q", "hap_bases")}
    ro = np.ascontiguousarray(b["read_off"], dtype=np.uint64)
    ho = np.ascontiguousarray(b["hap_off"], dtype=np.uint64)
    getattr(lib, _pre(precision) + "batch")(
        _p(arrs["read_bases"], _u8p), _p(ro, _u64p), _p(arrs["base_q"], _u8p),
        _p(arrs["ins_q"], _u8p), _p(arrs["del_q"], _u8p), _p(arrs["gcp_q"], _u8p),
        _p(arrs["hap_bases"], _u8p), _p(ho, _u64p), n, _p(pr, _u32p), _p(ph, _u32p),
        float(log2C), int(rescale), int(n_threads), _p(out, _f64p))
    return out
