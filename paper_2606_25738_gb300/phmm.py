"""Thin ctypes binding of libphmm.so (C ABI in include/phmm.h).

Argument marshalling only: every step of the forward computation runs in the library's
CUDA kernels.  Inputs are numpy arrays (host) or torch CUDA tensors (device); PyTorch is
used for device memory and streams only.  Importing this module loads the library and
raises if it has not been built: there is no fallback implementation.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_lib", "libphmm.so")

PHMM_OK, PHMM_PENDING = 0, 1
PHMM_EINVAL, PHMM_ENOMEM, PHMM_EBUSY, PHMM_ECUDA = -1, -2, -3, -4
PHMM_ETIMEOUT, PHMM_ECANCELED, PHMM_ENOTFOUND = -5, -6, -7
PREC = {"fp32": 0, "fp64": 1, "fp32_only": 2}
VARIANTS = {"auto": 0, "packed": 1, "scalar": 2, "lean": 3, "pipe": 4, "pipe2": 5, "pipe2lean": 6}
F_NO_GRAPH, F_LAUNCH_PER_PAIR, F_FORCE_RESCUE = 0x1, 0x2, 0x4
F_LONG_LEAN, F_LONG_PIPE32, F_LONG_PIPE24, F_NO_TUNE, F_LONG_SERIAL = 0x10, 0x20, 0x40, 0x80, 0x100
F_LONG_PIPE4, F_LONG_CLUSTER, F_LONG_WAVE, F_LONG_WAVE16 = 0x200, 0x400, 0x800, 0x1000
PAIR_RESCUED, PAIR_RESCALED, PAIR_FP64, PAIR_ERROR = 0x1, 0x2, 0x4, 0x80
PAIR_DANGER, PAIR_NONFINITE, PAIR_SMALL_SUM, PAIR_DEGENERATE = 0x8, 0x10, 0x20, 0x40

# Every entry point declared in include/phmm.h.
SYMBOLS = ["phmm_create", "phmm_submit_batch", "phmm_poll", "phmm_get_stats", "phmm_destroy",
           "phmm_strerror", "phmm_abi_version", "phmm_device_info", "phmm_scan_test",
           "phmm_forward_noalloc", "phmm_batch_footprint", "phmm_server_create",
           "phmm_server_enqueue", "phmm_server_poll", "phmm_server_get_stats", "phmm_server_destroy",
           "phmm_plan_check", "phmm_wait_test"]


class PhmmError(RuntimeError):
    def __init__(self, status: int, what: str = ""):
        self.status = status
        msg = _lib.phmm_strerror(status).decode() if _lib else str(status)
        super().__init__("%s: %s (%d)" % (what, msg, status) if what else "%s (%d)" % (msg, status))


class Config(ctypes.Structure):
    _fields_ = [("device", ctypes.c_int), ("precision", ctypes.c_int),
                ("mem_budget_bytes", ctypes.c_size_t), ("max_inflight", ctypes.c_uint),
                ("flags", ctypes.c_uint), ("stream", ctypes.c_void_p),
                ("cols_per_lane", ctypes.c_int), ("kernel_variant", ctypes.c_int),
                ("fp32_tolerance", ctypes.c_double)]


class Batch(ctypes.Structure):
    _fields_ = [("n_reads", ctypes.c_uint32), ("read_bases", ctypes.c_void_p),
                ("read_off", ctypes.c_void_p), ("base_q", ctypes.c_void_p),
                ("ins_q", ctypes.c_void_p), ("del_q", ctypes.c_void_p), ("gcp_q", ctypes.c_void_p),
                ("n_haps", ctypes.c_uint32), ("hap_bases", ctypes.c_void_p),
                ("hap_off", ctypes.c_void_p), ("n_pairs", ctypes.c_uint32),
                ("pair_read", ctypes.c_void_p), ("pair_hap", ctypes.c_void_p),
                ("out_log10", ctypes.c_void_p), ("out_flags", ctypes.c_void_p),
                ("inputs_on_device", ctypes.c_int), ("outputs_on_device", ctypes.c_int)]


ABI_VERSION = 3  # PHMM_ABI_VERSION of include/phmm.h

# Kernel names behind phmm_stats.short_kernel / packed_kernel / long_kernel.
SHORT_KERNELS = ["k_short_scalar<32, 4>", "k_short_scalar<24, 4>", "k_short_scalar<24, 5>",
                 "k_short_scalar<16, 6>", "k_short_pipe<32, 3>", "k_short_pipe<24, 4>",
                 "k_short_pipe<16, 4>", "k_short_pipe2<32, 3, 1, 0>", "k_short_pipe2<24, 4, 1, 0>",
                 "k_short_pipe2<32, 4, 1, 1>"]
PACKED_KERNELS = ["k_short_packed<12, 4>", "k_short_packed<16, 3>"]
LONG_KERNELS = ["k_forward<float, 32, 0>", "k_forward_pipe<32, 12>", "k_forward_pipe<24, 16>",
                "k_forward_serial<32, 3, 0>", "k_forward_pipe<32, 4>", "k_forward_cluster<32, 4, 8>",
                "k_forward_wave<32, 3>", "k_forward_wave<32, 3> (2 CTAs/SM)", "k_forward_wave<16, 3>"]
# FP64 forward variant behind phmm_stats.short_kernel when the precision is FP64.
FP64_KERNELS = ["k_forward<double, 8, 1, 16>", "k_forward<double, 16, 1, 8>",
                "k_short_pipe64<16, 2, 0> + k_forward<double, 16, 0, 8>",
                "k_short_pipe64<32, 1, 1> + k_forward<double, 16, 0, 8>"]


class Stats(ctypes.Structure):
    _fields_ = [("cells", ctypes.c_uint64), ("n_pairs", ctypes.c_uint32),
                ("n_rescued", ctypes.c_uint32), ("n_long", ctypes.c_uint32),
                ("cols_per_lane", ctypes.c_uint32), ("ms_total", ctypes.c_float),
                ("ms_forward", ctypes.c_float), ("ms_rescue", ctypes.c_float),
                ("ms_h2d", ctypes.c_float), ("kernel_launches", ctypes.c_uint32),
                ("status_bits", ctypes.c_uint32), ("ms_host", ctypes.c_float),
                ("short_kernel", ctypes.c_int32), ("packed_kernel", ctypes.c_int32),
                ("long_kernel", ctypes.c_int32), ("cells_branch", ctypes.c_uint64 * 3),
                ("ms_branch", ctypes.c_float * 3)]

    def as_dict(self) -> dict:
        return {name: (list(v) if isinstance(v, ctypes.Array) else v)
                for name, v in ((n, getattr(self, n)) for n, _ in self._fields_)}


class ServerConfig(ctypes.Structure):
    _fields_ = [("mem_budget_bytes", ctypes.c_uint64), ("max_epoch_pairs", ctypes.c_uint32),
                ("max_inflight_epochs", ctypes.c_uint32), ("max_pending", ctypes.c_uint32),
                ("max_wait_ms", ctypes.c_uint32), ("epoch_cells", ctypes.c_uint64),
                ("small_cells", ctypes.c_uint64)]


class ServerStats(ctypes.Structure):
    _fields_ = [(n, ctypes.c_uint64) for n in ("enqueued", "admitted", "completed", "failed", "epochs",
                                               "pending", "inflight", "cells_completed", "bytes_inflight")]

    def as_dict(self) -> dict:
        return {name: getattr(self, name) for name, _ in self._fields_}


def _load() -> ctypes.CDLL:
    if not os.path.exists(LIB_PATH):
        raise RuntimeError("libphmm.so is not built (%s); run __graft_entry__.build() or "
                           "python -m paper_2606_25738_gb300.build" % LIB_PATH)
    lib = ctypes.CDLL(LIB_PATH)
    if lib.phmm_abi_version() != ABI_VERSION:
        raise RuntimeError("libphmm.so has ABI version %d, this binding expects %d: rebuild it"
                           % (lib.phmm_abi_version(), ABI_VERSION))
    lib.phmm_create.argtypes = [ctypes.POINTER(Config), ctypes.POINTER(ctypes.c_void_p)]
    lib.phmm_submit_batch.argtypes = [ctypes.c_void_p, ctypes.POINTER(Batch), ctypes.POINTER(ctypes.c_uint64)]
    lib.phmm_poll.argtypes = [ctypes.c_void_p, ctypes.c_uint64, ctypes.c_int]
    lib.phmm_get_stats.argtypes = [ctypes.c_void_p, ctypes.c_uint64, ctypes.POINTER(Stats)]
    lib.phmm_destroy.argtypes = [ctypes.c_void_p]
    lib.phmm_destroy.restype = None
    lib.phmm_strerror.argtypes = [ctypes.c_int]
    lib.phmm_strerror.restype = ctypes.c_char_p
    lib.phmm_device_info.argtypes = [ctypes.c_void_p, ctypes.POINTER(ctypes.c_int),
                                     ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double)]
    lib.phmm_scan_test.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int,
                                   ctypes.c_float]
    lib.phmm_forward_noalloc.argtypes = [ctypes.c_int, ctypes.c_void_p, ctypes.POINTER(Batch)]
    lib.phmm_batch_footprint.argtypes = [ctypes.c_void_p, ctypes.POINTER(Batch), ctypes.POINTER(ctypes.c_uint64)]
    lib.phmm_server_create.argtypes = [ctypes.c_void_p, ctypes.POINTER(ServerConfig),
                                       ctypes.POINTER(ctypes.c_void_p)]
    lib.phmm_server_enqueue.argtypes = [ctypes.c_void_p, ctypes.POINTER(Batch), ctypes.POINTER(ctypes.c_uint64)]
    lib.phmm_server_poll.argtypes = [ctypes.c_void_p, ctypes.c_uint64, ctypes.c_int,
                                     ctypes.POINTER(ctypes.c_double)]
    lib.phmm_server_get_stats.argtypes = [ctypes.c_void_p, ctypes.POINTER(ServerStats)]
    lib.phmm_server_destroy.argtypes = [ctypes.c_void_p]
    lib.phmm_server_destroy.restype = None
    lib.phmm_wait_test.argtypes = [ctypes.c_void_p]
    lib.phmm_plan_check.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_uint32,
                                    ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                    ctypes.POINTER(ctypes.c_uint64)]
    return lib


_lib = _load()


def library() -> ctypes.CDLL:
    return _lib


_KEYS_U8 = ("read_bases", "base_q", "ins_q", "del_q", "gcp_q", "hap_bases")


def _host_arrays(b: dict) -> dict:
    a = {k: np.ascontiguousarray(b[k], dtype=np.uint8) for k in _KEYS_U8}
    a["read_off"] = np.ascontiguousarray(b["read_off"], dtype=np.uint64)
    a["hap_off"] = np.ascontiguousarray(b["hap_off"], dtype=np.uint64)
    a["pair_read"] = np.ascontiguousarray(b["pair_read"], dtype=np.uint32)
    a["pair_hap"] = np.ascontiguousarray(b["pair_hap"], dtype=np.uint32)
    return a


def _host_batch(b: dict, out, out_flags):
    """ctypes Batch over host numpy arrays; returns (batch, arrays kept alive)."""
    arrs = _host_arrays(b)
    ptr = {k: ctypes.c_void_p(v.ctypes.data) for k, v in arrs.items()}
    bb = Batch(len(arrs["read_off"]) - 1, ptr["read_bases"], ptr["read_off"], ptr["base_q"], ptr["ins_q"],
               ptr["del_q"], ptr["gcp_q"], len(arrs["hap_off"]) - 1, ptr["hap_bases"], ptr["hap_off"],
               len(arrs["pair_read"]), ptr["pair_read"], ptr["pair_hap"],
               ctypes.c_void_p(out.ctypes.data) if out is not None else None,
               ctypes.c_void_p(out_flags.ctypes.data) if out_flags is not None else None, 0, 0)
    return bb, arrs


def to_device(b: dict, device: str = "cuda"):
    """Copies a host batch to torch CUDA tensors (offsets as int64, indices as int32:
    the same bits the ABI reads as uint64 / uint32)."""
    import torch
    d = {k: torch.from_numpy(np.ascontiguousarray(b[k], dtype=np.uint8)).to(device) for k in _KEYS_U8}
    d["read_off"] = torch.from_numpy(np.ascontiguousarray(b["read_off"]).astype(np.int64)).to(device)
    d["hap_off"] = torch.from_numpy(np.ascontiguousarray(b["hap_off"]).astype(np.int64)).to(device)
    d["pair_read"] = torch.from_numpy(np.ascontiguousarray(b["pair_read"]).astype(np.int32)).to(device)
    d["pair_hap"] = torch.from_numpy(np.ascontiguousarray(b["pair_hap"]).astype(np.int32)).to(device)
    return d


class Context:
    """One library context (device, stream, arenas, captured graphs)."""

    def __init__(self, device: int = 0, precision: str = "fp32", flags: int = 0, stream=None,
                 cols_per_lane: int = 0, mem_budget: int = 0, max_inflight: int = 2,
                 variant: str = "auto", tolerance: float = 0.0):
        cfg = Config(device, PREC[precision], mem_budget, max_inflight, flags,
                     ctypes.c_void_p(stream) if stream else None, cols_per_lane,
                     VARIANTS[variant], float(tolerance))
        h = ctypes.c_void_p()
        rc = _lib.phmm_create(ctypes.byref(cfg), ctypes.byref(h))
        if rc != PHMM_OK:
            raise PhmmError(rc, "phmm_create")
        self._h = h
        self._keep = {}

    def close(self):
        if getattr(self, "_h", None):
            _lib.phmm_destroy(self._h)
            self._h = None
            self._keep = {}

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def device_info(self) -> dict:
        sms, mhz, cups = ctypes.c_int(), ctypes.c_double(), ctypes.c_double()
        _lib.phmm_device_info(self._h, ctypes.byref(sms), ctypes.byref(mhz), ctypes.byref(cups))
        return {"sms": sms.value, "max_clock_mhz": mhz.value, "roofline_cups": cups.value}

    def submit(self, b: dict, out=None, out_flags=None) -> int:
        """Enqueue a batch.  ``b`` holds numpy arrays (host inputs) or torch CUDA tensors
        (device inputs).  ``out`` / ``out_flags``: numpy arrays (host outputs) or torch
        CUDA tensors (device outputs) of n_pairs float64 / uint8."""
        dev_in = not isinstance(b["read_bases"], np.ndarray)
        n_reads = len(b["read_off"]) - 1
        n_haps = len(b["hap_off"]) - 1
        n_pairs = len(b["pair_read"])
        if dev_in:
            arrs = b
            ptr = {k: ctypes.c_void_p(v.data_ptr()) for k, v in b.items() if hasattr(v, "data_ptr")}
        else:
            arrs = _host_arrays(b)
            ptr = {k: ctypes.c_void_p(v.ctypes.data) for k, v in arrs.items()}
        if out is None:
            out = np.empty(n_pairs, dtype=np.float64)
        dev_out = not isinstance(out, np.ndarray)
        if out_flags is None and not dev_out:
            out_flags = np.zeros(n_pairs, dtype=np.uint8)
        optr = ctypes.c_void_p(out.data_ptr() if dev_out else out.ctypes.data)
        fptr = None
        if out_flags is not None:
            fptr = ctypes.c_void_p(out_flags.data_ptr() if dev_out else out_flags.ctypes.data)
        bb = Batch(n_reads, ptr["read_bases"], ptr["read_off"], ptr["base_q"], ptr["ins_q"],
                   ptr["del_q"], ptr["gcp_q"], n_haps, ptr["hap_bases"], ptr["hap_off"], n_pairs,
                   ptr["pair_read"], ptr["pair_hap"], optr, fptr, int(dev_in), int(dev_out))
        t = ctypes.c_uint64()
        rc = _lib.phmm_submit_batch(self._h, ctypes.byref(bb), ctypes.byref(t))
        if rc != PHMM_OK:
            raise PhmmError(rc, "phmm_submit_batch")
        self._keep[t.value] = (arrs, out, out_flags)
        return t.value

    def poll(self, ticket: int, timeout_ms: int = -1) -> int:
        rc = _lib.phmm_poll(self._h, ticket, timeout_ms)
        if rc != PHMM_PENDING:
            self._keep.pop(ticket, None)
        return rc

    def stats(self, ticket: int) -> dict:
        s = Stats()
        rc = _lib.phmm_get_stats(self._h, ticket, ctypes.byref(s))
        if rc not in (PHMM_OK, PHMM_PENDING):
            raise PhmmError(rc, "phmm_get_stats")
        return s.as_dict()

    def run(self, b: dict, out=None, out_flags=None, check: bool = True):
        """submit + poll(forever).  Returns (log10 L, flags, status, stats)."""
        n = len(b["pair_read"])
        if out is None:
            out = np.empty(n, dtype=np.float64)
        if out_flags is None and isinstance(out, np.ndarray):
            out_flags = np.zeros(n, dtype=np.uint8)
        t = self.submit(b, out, out_flags)
        rc = self.poll(t, -1)
        st = self.stats(t)
        if check and rc not in (PHMM_OK,):
            raise PhmmError(rc, "phmm_poll")
        return out, out_flags, rc, st

    def footprint(self, b: dict) -> int:
        """phmm_batch_footprint: device bytes a host batch may hold while in flight."""
        bb, _arrs = _host_batch(b, None, None)
        v = ctypes.c_uint64()
        rc = _lib.phmm_batch_footprint(self._h, ctypes.byref(bb), ctypes.byref(v))
        if rc != PHMM_OK:
            raise PhmmError(rc, "phmm_batch_footprint")
        return v.value

    def wait_test(self) -> int:
        """phmm_wait_test: a bounded device wait on a boundary nothing writes; returns
        PHMM_ETIMEOUT when the wait gave up as designed."""
        return _lib.phmm_wait_test(self._h)

    def scan_test(self, y, a: float):
        """The lane + warp linear-recurrence scan on a torch CUDA float32 tensor y
        (1..1024 values): z[t] = sum_{s<=t} a^(t-s) y[s]."""
        import torch
        z = torch.empty_like(y)
        rc = _lib.phmm_scan_test(self._h, ctypes.c_void_p(y.data_ptr()), ctypes.c_void_p(z.data_ptr()),
                                 int(y.numel()), float(a))
        if rc != PHMM_OK:
            raise PhmmError(rc, "phmm_scan_test")
        return z


def plan_check(l, k, pair_read, precision: str = "fp32", scal_id: int = 4, pack_id: int = -1,
               long_kind: int = 1):
    """phmm_plan_check (host only): builds and checks the work plan for the given read /
    haplotype lengths.  Returns (status, stats dict)."""
    l = np.ascontiguousarray(l, dtype=np.uint32)
    k = np.ascontiguousarray(k, dtype=np.uint32)
    pr = np.ascontiguousarray(pair_read, dtype=np.uint32)
    st = (ctypes.c_uint64 * 8)()
    rc = _lib.phmm_plan_check(ctypes.c_void_p(l.ctypes.data), ctypes.c_void_p(k.ctypes.data),
                              ctypes.c_void_p(pr.ctypes.data), len(l), PREC[precision], scal_id, pack_id,
                              long_kind, st)
    names = ("teams", "warp_items", "packed_warp_items", "cta_items", "cta_pairs", "striped_pairs",
             "too_long", "failed_check")
    return rc, dict(zip(names, [int(v) for v in st]))


def forward_noalloc(d: dict, out, out_flags, device: int = 0, stream=None) -> int:
    """phmm_forward_noalloc: FP32 forward pass for callers that cannot allocate device
    memory (see include/phmm.h).  ``d`` holds torch CUDA tensors (see to_device), ``out``
    a float64 and ``out_flags`` a uint8 CUDA tensor of n_pairs.  Returns the status."""
    ptr = {k: ctypes.c_void_p(v.data_ptr()) for k, v in d.items() if hasattr(v, "data_ptr")}
    bb = Batch(len(d["read_off"]) - 1, ptr["read_bases"], ptr["read_off"], ptr["base_q"], ptr["ins_q"],
               ptr["del_q"], ptr["gcp_q"], len(d["hap_off"]) - 1, ptr["hap_bases"], ptr["hap_off"],
               len(d["pair_read"]), ptr["pair_read"], ptr["pair_hap"], ctypes.c_void_p(out.data_ptr()),
               ctypes.c_void_p(out_flags.data_ptr()), 1, 1)
    return _lib.phmm_forward_noalloc(device, ctypes.c_void_p(stream) if stream else None, ctypes.byref(bb))


class Server:
    """Continuous-batching request loop of the library (phmm_server_*), on a Context it
    takes over while it runs.  Requests are host batches; results land in numpy arrays."""

    def __init__(self, ctx: Context, mem_budget: int = 40 << 30, max_epoch_pairs: int = 0,
                 max_inflight_epochs: int = 2, max_pending: int = 0, max_wait_ms: int = 0,
                 epoch_cells: int = 0, small_cells: int = 0):
        self.ctx = ctx
        cfg = ServerConfig(mem_budget, max_epoch_pairs, max_inflight_epochs, max_pending, max_wait_ms,
                           epoch_cells, small_cells)
        h = ctypes.c_void_p()
        rc = _lib.phmm_server_create(ctx._h, ctypes.byref(cfg), ctypes.byref(h))
        if rc != PHMM_OK:
            raise PhmmError(rc, "phmm_server_create")
        self._h = h
        self._out = {}

    def enqueue(self, b: dict) -> int:
        """Queue a request; returns its id.  Raises PhmmError on rejection."""
        n = len(b["pair_read"])
        out = np.full(n, np.nan, dtype=np.float64)
        fl = np.zeros(n, dtype=np.uint8)
        bb, _arrs = _host_batch(b, out, fl)
        rid = ctypes.c_uint64()
        rc = _lib.phmm_server_enqueue(self._h, ctypes.byref(bb), ctypes.byref(rid))
        if rc != PHMM_OK:
            raise PhmmError(rc, "phmm_server_enqueue")
        self._out[rid.value] = (out, fl)
        return rid.value

    def poll(self, rid: int, timeout_ms: int = -1):
        """(status, latency_ms, log10 L, flags); results are None while pending."""
        lat = ctypes.c_double()
        rc = _lib.phmm_server_poll(self._h, rid, timeout_ms, ctypes.byref(lat))
        if rc == PHMM_PENDING:
            return rc, None, None, None
        out, fl = self._out.pop(rid, (None, None))
        return rc, lat.value, out, fl

    def stats(self) -> dict:
        s = ServerStats()
        _lib.phmm_server_get_stats(self._h, ctypes.byref(s))
        return s.as_dict()

    def close(self):
        if getattr(self, "_h", None):
            _lib.phmm_server_destroy(self._h)
            self._h = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
