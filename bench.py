"""Benchmark: GCUPS of the FP32 + FP64-rescue PairHMM forward path through the library's
C ABI, on seeded synthetic workloads shaped like the paper's (Section 4.1).

Headline (default ``--config uneven``): the largest single-GPU workload, 1M pairs with
read and haplotype lengths each log-uniform 50-20k bp (haplotype >= read), short-read
error and quality model, about 1.1e13 cell updates.  One step = one pass of the whole hot
path over that batch (coefficient prep, the three forward branches, log10 reduction,
rescue selection and the FP64 rescue pass) with inputs resident in device memory; the
batch is one submit, later steps replay its captured CUDA graph.  Extra legs in the same
JSON line: the short-read region batch and the long-read pairs (with their all-FP64 GPU
comparators), a row-wise CPU comparator, and a short open-loop run of the serving loop.

Other ``--config`` values time one workload alone: ``short`` (2000 regions x 50 reads of
150 bp x 1-8 haplotypes of 250-600 bp), ``long`` (64 pairs, haplotypes log-uniform
1k-100k bp), ``plain`` (64 short pairs) and ``sweep`` (equal lengths, the shape of the
paper's Section 4.3 scalability experiment).  ``--impl reference`` times the CPU oracle on
the host cores instead, on bounded samples of the same workload.  Prints one JSON line
(rank 0).
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "GCUPS (FP32+FP64-rescue vs plain FP64, |Δlog10|≤1e-3); serve p50/p99 ms"
TOL32, TOL64 = 1e-3, 1e-9
FLOP_PER_CELL = 12  # Eq. 2 as written: 6 multiplies + 6 adds per cell
L2_NOTE = "inputs larger than L2 (129 MB) and a 256 MB write between steps to evict it"

WORKLOADS = {
    # name: (default units, unit name, description template)
    "uneven": (1_000_000, "pairs", "uneven-length batch: %d pairs, read and haplotype lengths each "
                                   "log-uniform 50-20k bp (haplotype >= read), short-read error/quality model"),
    "short": (2000, "regions", "short-read batch: %d regions x 50 reads (150 bp) x 1-8 haplotypes (250-600 bp)"),
    "long": (64, "pairs", "long-read pairs: %d pairs, haplotypes log-uniform 1k-100k bp, reads 90-100%% "
                          "of the haplotype, 5%% substitutions, 3%% 1-3 bp indels, quals Phred 5-30"),
    "plain": (64, "pairs", "plain pairs: %d pairs, haplotypes 200-400 bp, reads 100-150 bp, 1%% "
                           "substitutions, 0.1%% indels"),
    "sweep": (0, "lengths", "equal-length sweep: read = haplotype length %s, %s per length"),
}


def _env_rank():
    return int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")), \
        int(os.environ.get("LOCAL_RANK", "0"))


# ----------------------------------------------------------------------------------------
# Workloads and the config dict both arms print
# ----------------------------------------------------------------------------------------

def sweep_lengths(args):
    out, L = [], args.min_len
    while L <= args.max_len:
        out.append(L)
        L *= 2
    return out


def make_workload(name: str, units: int, uneven_max: int = 20000):
    from paper_2606_25738_gb300 import workloads as W
    if name == "uneven":
        return W.uneven_pairs(units, seed=0, len_range=(50, uneven_max))
    if name == "short":
        return W.short_read_regions(units, seed=0)
    if name == "long":
        return W.long_pairs(units, seed=0)
    if name == "plain":
        return W.plain_pairs(units, seed=0)
    raise ValueError(name)


def sweep_batch(L: int, target_cells: float = 2e10, max_pairs: int = 1 << 20, pairs: int = 0):
    """Equal-length pairs of length L: ``pairs`` of them, or (0) about target_cells cells."""
    from paper_2606_25738_gb300 import workloads as W
    n = pairs if pairs > 0 else int(min(max_pairs, max(1, round(target_cells / (L * L)))))
    return W.equal_length(n, L, seed=0)


def config_dict(name: str, units: int, b, world: int, args) -> dict:
    """The workload description: identical in both arms for the same command line."""
    from paper_2606_25738_gb300 import workloads as W
    if name == "sweep":
        lens = sweep_lengths(args)
        sp = getattr(args, "sweep_pairs", 0)
        desc = WORKLOADS[name][2] % ("%d-%d bp" % (lens[0], lens[-1]),
                                     "%d pairs" % sp if sp > 0 else "about 2e10 cells")
        return {"workload": desc, "lengths": lens, "l2": L2_NOTE,
                "parallelism": "replicas" if world > 1 else "single GPU"}
    desc = WORKLOADS[name][2] % units
    if name == "uneven" and getattr(args, "uneven_max", 20000) != 20000:
        desc = desc.replace("50-20k bp", "50-%d bp" % args.uneven_max)
    return {"workload": desc, "pairs": int(len(b["pair_read"])), "reads": int(len(b["read_off"]) - 1),
            "haplotypes": int(len(b["hap_off"]) - 1), "cells": int(W.cells(b)), "l2": L2_NOTE,
            "parallelism": "replicas" if world > 1 else "single GPU"}


# ----------------------------------------------------------------------------------------
# Timing helpers
# ----------------------------------------------------------------------------------------

class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled every 200 ms during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device: int):
        self.device = device
        self.samples = []
        self._stop = threading.Event()
        self._t = None

    def _run(self):
        while not self._stop.is_set():
            try:
                r = subprocess.run(["nvidia-smi", "-i", str(self.device), "--query-gpu=" + self.FIELDS,
                                    "--format=csv,noheader,nounits"], capture_output=True, text=True,
                                   timeout=5)
                for line in r.stdout.strip().splitlines():
                    self.samples.append([x.strip() for x in line.split(",")])
            except Exception:
                pass
            self._stop.wait(0.2)

    def __enter__(self):
        self._t = threading.Thread(target=self._run, daemon=True)
        self._t.start()
        return self

    def __exit__(self, *a):
        self._stop.set()
        self._t.join(timeout=10)

    def summary(self) -> dict:
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for s in self.samples:
            try:
                sm.append(float(s[1]))
                mx.append(float(s[2]))
                for n, v in zip(names, s[5:9]):
                    if v.strip().lower() == "active":
                        reasons.add(n)
            except (ValueError, IndexError):
                continue
        return {"sm_mhz": float(np.median(sm)) if sm else None,
                "sm_max_mhz": float(max(mx)) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def max_over_ranks(values, world: int):
    """Element-wise maximum of per-rank values (step time, wall time) over the job's ranks:
    the job is as slow as its slowest rank.  NCCL jobs reduce on the GPU, gloo on the CPU."""
    if world <= 1:
        return [float(v) for v in values]
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([float(v) for v in values], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return [float(x) for x in t.cpu()]


def job_throughput(cells_per_rank: float, world: int, step_ms: float) -> float:
    """Whole-job GCUPS: every rank scores its own replica of the batch (pairs are
    independent; no exchange), so the job updates world x cells per slowest-rank step."""
    return cells_per_rank * world / (step_ms * 1e-3) / 1e9


def _peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return {}


def _nvtx(torch, name):
    try:
        if name:
            torch.cuda.nvtx.range_push(name)
        else:
            torch.cuda.nvtx.range_pop()
    except Exception:
        pass


# ----------------------------------------------------------------------------------------
# Oracle legs (test infrastructure: the cpu_baseline, the reference arm and the parity
# samples; nothing here is on the timed path)
# ----------------------------------------------------------------------------------------

def oracle_sample(b, seconds: float = 15.0, seed: int = 1, threads: int | None = None):
    """The CPU oracle on a random sample of the batch's pairs sized to about ``seconds``
    of work.  Returns (GCUPS, threads, description, seconds, sampled pair indices, their
    oracle log10 L)."""
    import oracle
    from paper_2606_25738_gb300 import workloads as W
    cores = threads or os.cpu_count() or 1
    rl, hl = W.pair_lengths(b)
    n = len(rl)
    rng = np.random.default_rng(seed)
    order = rng.permutation(n)
    # calibrate on a small sample (capped in cells so that huge pairs do not dominate)
    c = rl[order] * hl[order]
    csum = np.cumsum(c)
    m0 = int(min(n, max(cores * 4, min(64, np.searchsorted(csum, 2e8 * cores) + 1))))
    probe = order[:m0]
    t = time.perf_counter()
    oracle.batch(b, pairs=probe, n_threads=cores)
    dt = time.perf_counter() - t
    rate = float(np.sum(c[:m0])) / max(dt, 1e-6)
    m = int(min(n, max(m0, np.searchsorted(csum, rate * seconds) + 1)))
    pick = order[:m]
    cells = float(np.sum(c[:m]))
    t = time.perf_counter()
    ref = oracle.batch(b, pairs=pick, n_threads=cores)
    dt = time.perf_counter() - t
    return (cells / dt / 1e9, cores,
            "%d random pairs of the workload (%.3g cells), FP64 cell-by-cell, %d threads" % (m, cells, cores),
            dt, pick, ref)


def parity_block(b, res, flags, pick, ref) -> dict:
    """This run's outputs on the sampled pairs against the oracle's values for them."""
    from paper_2606_25738_gb300 import phmm
    dd = np.abs(res[pick] - ref)
    fp64 = (flags[pick] & (phmm.PAIR_RESCUED | phmm.PAIR_FP64)) != 0
    both_inf = ~np.isfinite(ref) & (res[pick] == ref)
    dd = np.where(both_inf, 0.0, dd)
    return {"sample_pairs": int(len(pick)),
            "max_abs_dlog10_fp32": float(dd[~fp64].max()) if (~fp64).any() else None,
            "max_abs_dlog10_fp64": float(dd[fp64].max()) if fp64.any() else None,
            "within_tolerance": bool(np.all(dd <= np.where(fp64, TOL64, TOL32)))}


def stratified_parity(b, res, flags, per_decile: int = 200, max_cells: float = 2e10) -> dict:
    """Parity on pairs from every decile of l*k plus every rescued pair (up to 300)."""
    import oracle
    from paper_2606_25738_gb300 import phmm
    from paper_2606_25738_gb300 import workloads as W
    pick = W.stratified_sample(b, per_decile, max_cells=max_cells)
    resc = np.flatnonzero(flags & phmm.PAIR_RESCUED)[:300]
    pick = np.unique(np.concatenate([pick, resc]))
    t = time.perf_counter()
    ref = oracle.batch(b, pairs=pick)
    r = parity_block(b, res, flags, pick, ref)
    r["oracle_s"] = time.perf_counter() - t
    r["how"] = "%d pairs per decile of l*k (under %.0e cells) + rescued pairs" % (per_decile, max_cells)
    return r


def run_reference(args):
    rank, world, _ = _env_rank()
    if rank != 0:
        return
    name = getattr(args, "config", "short")
    if name == "sweep":
        units = 0
        lens = sweep_lengths(args)
        batches = [sweep_batch(L, pairs=getattr(args, "sweep_pairs", 0)) for L in lens]
        cfg = config_dict(name, 0, None, world, args)
    else:
        units = getattr(args, "units", 0) or WORKLOADS[name][0]
        if getattr(args, "regions", None) and name == "short":
            units = args.regions
        batches = [make_workload(name, units, getattr(args, "uneven_max", 20000))]
        cfg = config_dict(name, units, batches[0], world, args)
    vals = []
    # each step is a bounded random sample of the workload, sized so that the whole run
    # stays within about three minutes of host time
    per_step = max(0.5, min(8.0, 150.0 / max(1, args.steps + args.warmup)))
    for w in range(args.warmup):
        oracle_sample(batches[w % len(batches)], seconds=min(2.0, per_step))
    desc, cores = "", 1
    for k in range(args.steps):
        v, cores, desc, _dt, _pick, _ref = oracle_sample(batches[k % len(batches)], seconds=per_step, seed=10 + k)
        vals.append(v)
    value = float(np.median(vals))
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "GCUPS",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic (seeded, shaped like the paper's workloads)", "config": cfg,
            "cpu_baseline": {"value": value, "unit": "GCUPS", "cores": cores, "kind": "oracle",
                             "sample": desc + "; median over %d steps" % args.steps},
            "e2e": {"value": value, "unit": "GCUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ----------------------------------------------------------------------------------------
# GPU legs
# ----------------------------------------------------------------------------------------

def _flag_bits(args, phmm):
    return {"auto": 0, "lean": phmm.F_LONG_LEAN, "pipe32": phmm.F_LONG_PIPE32, "pipe24": phmm.F_LONG_PIPE24,
            "serial": phmm.F_LONG_SERIAL, "pipe4": phmm.F_LONG_PIPE4,
            "cluster": phmm.F_LONG_CLUSTER, "wave": phmm.F_LONG_WAVE,
            "wave16": phmm.F_LONG_WAVE16}[args.long_kind]


def kernel_names(st: dict, phmm) -> list:
    """Names of the three forward branches' kernels of a ticket (None: no work)."""
    def nm(table, i):
        return table[i] if 0 <= i < len(table) else None
    return [nm(phmm.SHORT_KERNELS, st["short_kernel"]), nm(phmm.PACKED_KERNELS, st["packed_kernel"]),
            nm(phmm.LONG_KERNELS, st["long_kernel"])]


def dominant_branch(sts: list, phmm) -> dict:
    """The forward branch that scores the most cells, its cells and its mean launch
    duration over the timed steps (CUDA events on its own stream).  The branches run
    concurrently, so a small branch's duration can span the whole forward pass while its
    blocks wait for SMs: the cell count, not the duration, names the dominant kernel."""
    ms = np.mean([s["ms_branch"] for s in sts], axis=0)
    cells = sts[-1]["cells_branch"]
    names = kernel_names(sts[-1], phmm)
    q = int(np.argmax([c if names[i] else -1 for i, c in enumerate(cells)]))
    return {"branch": ["scalar short teams", "packed short teams", "multi-warp pairs"][q],
            "kernel": names[q], "ms": float(ms[q]), "cells": int(cells[q]),
            "all": [{"kernel": names[i], "cells": int(cells[i]), "ms": float(ms[i])} for i in range(3)]}


def fp64_forward(sts: list, phmm, cells: int) -> dict:
    """FP64 mode: the forward kernels of the chosen FP64 variant as one unit (the variant's
    branches both run FP64), their cells and the mean forward time."""
    ms = float(np.mean([s["ms_forward"] for s in sts]))
    name = phmm.FP64_KERNELS[sts[-1]["short_kernel"]]
    return {"branch": "FP64 forward", "kernel": name, "ms": ms, "cells": int(cells), "fp64": True,
            "all": [{"kernel": name, "cells": int(cells), "ms": ms}]}


def roofline(dom: dict, info: dict) -> dict:
    """Roofline entry of the dominant kernel.  `traffic` comes from
    profiles/forward_traffic.json, keyed by kernel name and by the launch's cell count (the
    exact work of a captured launch, scaled to this one in that file), else null."""
    peaks = _peaks()
    sm_max = float(peaks.get("sm_max_mhz", info["max_clock_mhz"]))
    fp64 = bool(dom.get("fp64"))
    lanes = 2 if fp64 else 128  # FMA lanes per SM per clock: FP64 (nominal) / FP32
    peak = 2.0 * lanes * info["sms"] * sm_max * 1e6 / 1e12
    achieved = FLOP_PER_CELL * dom["cells"] / (dom["ms"] * 1e-3) / 1e12 if dom["ms"] > 0 else 0.0
    traffic = None
    tfile = os.path.join(ROOT, "profiles", "forward_traffic.json")
    if os.path.exists(tfile) and dom["kernel"]:
        try:
            ent = json.load(open(tfile)).get(dom["kernel"], {}).get(str(dom["cells"]))
            if ent:
                traffic = ent.get("bytes_per_launch")
        except Exception:
            traffic = None
    return {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
            "frac": achieved / peak, "traffic": traffic, "kernel": dom["kernel"],
            "branch": dom["branch"], "cells_per_launch": dom["cells"], "ms_per_launch": dom["ms"],
            "flop_per_cell": FLOP_PER_CELL,
            "peak_note": "2 x %d %s FMA lanes x %d SMs x %.0f MHz (nominal unit count at the max SM clock of "
                         "MEASURED_PEAKS.json; no measured %s peak exists there)"
                         % (lanes, "FP64" if fp64 else "FP32", info["sms"], sm_max, "FP64" if fp64 else "FP32")}


def timed_steps(ctx, d, out, fl, steps, warmup, stream, flush, world, clocks: bool = True, dev: int = 0):
    """W untimed then K timed submits of one device-resident batch; the device time of a
    step comes from the library's CUDA events (first to last kernel of the ticket)."""
    import torch

    def step():
        with torch.cuda.stream(stream):
            flush.fill_(1.0)  # evict L2 between steps (outside the library's events)
        t = ctx.submit(d, out, fl)
        rc = ctx.poll(t, -1)
        if rc != 0:
            raise RuntimeError("poll status %d" % rc)
        return ctx.stats(t)

    for _ in range(warmup):
        step()
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    sts = []
    clk = ClockSampler(dev) if clocks else None
    if clk:
        clk.__enter__()
    try:
        torch.cuda.synchronize()
        _nvtx(torch, "timed")  # lets a profiler restrict itself to the timed steps
        t0 = time.perf_counter()
        for _ in range(steps):
            sts.append(step())
        torch.cuda.synchronize()
        wall = time.perf_counter() - t0
        _nvtx(torch, None)
    finally:
        if clk:
            clk.__exit__()
    if world > 1:
        torch.distributed.barrier()
    return sts, wall, (clk.summary() if clk else None)


def gpu_leg(name: str, b, dev: int, args, steps: int = 5, warmup: int = 3, precision: str = "fp32",
            flags: int = 0, parity: str = "stratified", flush=None) -> dict:
    """One workload on its own context: first submit (plan, tuning, graph capture), then
    timed replays; GCUPS for the forward kernels and the whole step, the dominant branch's
    roofline fraction, and sampled parity against the oracle."""
    import torch

    from paper_2606_25738_gb300 import phmm
    from paper_2606_25738_gb300 import workloads as W
    n = len(b["pair_read"])
    cells = W.cells(b)
    d = phmm.to_device(b)
    out = torch.empty(n, dtype=torch.float64, device="cuda")
    fl = torch.zeros(n, dtype=torch.uint8, device="cuda")
    stream = torch.cuda.Stream(device=dev)
    if flush is None:
        flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    with phmm.Context(device=dev, precision=precision, stream=stream.cuda_stream, max_inflight=1,
                      flags=flags) as ctx:
        info = ctx.device_info()
        t = time.perf_counter()
        ctx.poll(ctx.submit(d, out, fl), -1)
        first_s = time.perf_counter() - t
        sts, _wall, _ = timed_steps(ctx, d, out, fl, steps, warmup, stream, flush, 1, clocks=False)
    res, flg = out.cpu().numpy(), fl.cpu().numpy()
    del d, out, fl
    torch.cuda.empty_cache()
    tot = float(np.mean([s["ms_total"] for s in sts]))
    fwd = float(np.mean([s["ms_forward"] for s in sts]))
    row = {"workload": name, "precision": precision, "pairs": n, "cells": cells,
           "gcups_step": cells / tot / 1e6, "gcups_forward": cells / fwd / 1e6, "ms_per_step": tot,
           "ms_forward": fwd, "rescued_pairs": int(sts[-1]["n_rescued"]), "first_submit_s": first_s,
           "kernels": ([k for k in kernel_names(sts[-1], phmm) if k] if precision != "fp64"
                       else [phmm.FP64_KERNELS[sts[-1]["short_kernel"]]])}
    dom = dominant_branch(sts, phmm) if precision != "fp64" else fp64_forward(sts, phmm, cells)
    row["roofline"] = roofline(dom, info)
    if parity == "stratified":
        row["parity"] = stratified_parity(b, res, flg, per_decile=100, max_cells=1e10)
    elif parity == "all":
        import oracle
        ref = oracle.batch(b)
        row["parity"] = parity_block(b, res, flg, np.arange(n), ref)
    return row


def fp64_comparators(b, dev, args) -> dict:
    """The all-FP64 GPU comparators (outside the timed region): this library's batched
    FP64 mode over the whole batch, and a plain FP64 one-launch-per-pair run over a
    bounded random sample of its pairs."""
    import torch

    from paper_2606_25738_gb300 import phmm
    from paper_2606_25738_gb300 import workloads as W
    n = len(b["pair_read"])
    res = {}
    row = gpu_leg("fp64", b, dev, args, steps=3, warmup=1, precision="fp64", parity="none")
    res["fp64_batched"] = {"value": row["gcups_step"], "unit": "GCUPS", "ms_per_step": row["ms_per_step"],
                           "what": "this library, precision=fp64 (all pairs, one graph launch)"}
    m = min(n, args.lpp_pairs)
    pick = np.sort(np.random.default_rng(3).choice(n, m, replace=False))
    sb = W.subset(b, pick)
    sd = phmm.to_device(sb)
    scells = W.cells(sb)
    out2 = torch.empty(m, dtype=torch.float64, device="cuda")
    fl2 = torch.zeros(m, dtype=torch.uint8, device="cuda")
    with phmm.Context(device=dev, precision="fp64", flags=phmm.F_LAUNCH_PER_PAIR | phmm.F_NO_GRAPH,
                      max_inflight=1) as cl:
        cl.poll(cl.submit(sd, out2, fl2), -1)
        t = cl.submit(sd, out2, fl2)
        if cl.poll(t, -1) != 0:
            raise RuntimeError("fp64 launch-per-pair run failed")
        st = cl.stats(t)
    res["fp64_launch_per_pair"] = {"value": scells / (st["ms_total"] * 1e-3) / 1e9, "unit": "GCUPS",
                                   "ms": st["ms_total"], "sample_pairs": m, "sample_cells": scells,
                                   "what": "plain FP64, one kernel launch (one CTA) per pair, in order"}
    return res


def cpu_rowwise(b, pick, ref, cores):
    """The library's row-wise CPU path (libphmm_cpu.so, all host cores) on the pairs the
    cpu_baseline leg sampled, checked against the oracle's values for them."""
    from paper_2606_25738_gb300 import cpu
    from paper_2606_25738_gb300 import workloads as W
    sb = W.subset(b, pick)
    cells = float(W.cells(sb))
    cpu.forward(W.subset(b, pick[: min(len(pick), 256)]), cores)  # warm the library and caches
    t = time.perf_counter()
    out, _ = cpu.forward(sb, cores)
    dt = time.perf_counter() - t
    return {"value": cells / dt / 1e9, "unit": "GCUPS", "cores": cores, "seconds": dt,
            "max_abs_dlog10_vs_oracle": float(np.max(np.abs(out - ref))),
            "what": "row-wise CPU path on the cpu_baseline sample"}


def serve_leg(dev, rate, seconds, pool_n):
    """A short open-loop run of the library's serving loop on region requests (R reads
    U{10..500} x H haplotypes U{2..16}; 80% 150 bp reads, 20% log-uniform 1k-20k bp;
    haplotypes 1.5-3x the read length; 40 GB admission budget)."""
    from paper_2606_25738_gb300 import phmm
    from paper_2606_25738_gb300 import serving
    pool = serving.make_pool(pool_n, seed=0)
    with phmm.Context(device=dev, precision="fp32", max_inflight=3, flags=phmm.F_NO_TUNE) as c:
        r = serving.run(c, pool, rate=rate, duration=seconds, drain_s=60.0, max_inflight_epochs=3)
    r["pool"] = "%d seeded region requests, mean %.3g cells" % (len(pool), sum(p[1] for p in pool) / len(pool))
    return r


def run_sweep(args, dev, world):
    """Equal-length sweep: one batch per length (about 2e10 cells, at least one pair, or
    --sweep-pairs pairs), kernel-only and whole-step GCUPS per length, the forward time per
    row step, sampled parity where the oracle is cheap."""
    import oracle

    from paper_2606_25738_gb300 import phmm
    rows = []
    tot_cells, tot_ms = 0.0, 0.0
    for L in sweep_lengths(args):
        b = sweep_batch(L, pairs=args.sweep_pairs)
        row = gpu_leg("sweep", b, dev, args, steps=max(1, args.steps), warmup=max(1, min(args.warmup, 2)),
                      parity="none", flags=_flag_bits(args, phmm))
        row["us_per_row"] = row["ms_forward"] * 1e3 / L  # one row step along the pair's chain
        row["long_kernel"] = row["kernels"][-1] if row["kernels"] else None
        n = row["pairs"]
        m = int(max(1, min(n, 4e8 // (L * L)))) if L * L <= 4e8 else 0
        row["L"] = L
        if m:
            # a random sample of the length's pairs through the same path, against the oracle
            from paper_2606_25738_gb300 import phmm
            from paper_2606_25738_gb300 import workloads as W
            pick = np.sort(np.random.default_rng(L).choice(n, m, replace=False))
            sb = W.subset(b, pick)
            with phmm.Context(device=dev, precision="fp32", flags=_flag_bits(args, phmm)) as ctx:
                o, f, rc, _ = ctx.run(sb)
            row["parity"] = parity_block(sb, o, f, np.arange(m), oracle.batch(sb))
        tot_cells += row["cells"]
        tot_ms += row["ms_per_step"]
        rows.append(row)
    return rows, tot_cells, tot_ms


def run_ours(args):
    import torch

    from paper_2606_25738_gb300 import phmm
    from paper_2606_25738_gb300 import workloads as W

    rank, world, local = _env_rank()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    dev = local if world > 1 else 0
    torch.cuda.set_device(dev)
    name = args.config
    if name == "sweep":
        rows, tc, tms = run_sweep(args, dev, world)
        step_ms = max_over_ranks([tms], world)[0]
        if rank == 0:
            value = job_throughput(tc, world, step_ms)
            dom = max(rows, key=lambda r: r["cells"])
            print(json.dumps({
                "metric": METRIC, "value": value, "unit": "GCUPS", "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": step_ms, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "f32 (f64 rescue + reduction)",
                "data": "synthetic (seeded equal-length pairs)", "config": config_dict(name, 0, None, world, args),
                "roofline": dom.get("roofline"), "sweep": rows}), flush=True)
        return
    units = args.units or WORKLOADS[name][0]
    if args.regions and name == "short":
        units = args.regions
    t = time.perf_counter()
    # Replicas: every rank scores its own copy of the workload (pairs are independent;
    # there is no exchange step), so per-GPU work is fixed as N grows.
    b = make_workload(name, units, args.uneven_max)
    gen_s = time.perf_counter() - t
    n = len(b["pair_read"])
    cells = W.cells(b)
    stream = torch.cuda.Stream(device=dev)
    d = phmm.to_device(b)
    out = torch.empty(n, dtype=torch.float64, device="cuda")
    fl = torch.zeros(n, dtype=torch.uint8, device="cuda")
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")  # > L2 (129 MB)
    ctx = phmm.Context(device=dev, precision=args.precision, stream=stream.cuda_stream, max_inflight=2,
                       variant=args.variant, cols_per_lane=args.cols, flags=_flag_bits(args, phmm))
    info = ctx.device_info()
    t = time.perf_counter()
    ctx.poll(ctx.submit(d, out, fl), -1)  # plan, measured tuning, graph capture
    first_s = time.perf_counter() - t
    sts, wall, clocks = timed_steps(ctx, d, out, fl, args.steps, args.warmup, stream, flush, world, dev=dev)
    ms = np.array([s["ms_total"] for s in sts])
    ms_fwd = np.array([s["ms_forward"] for s in sts])
    step_ms, wall = max_over_ranks([float(ms.mean()), wall], world)
    value = job_throughput(cells, world, step_ms)
    res = out.cpu().numpy()
    flg = fl.cpu().numpy()
    dom = dominant_branch(sts, phmm) if args.precision != "fp64" else fp64_forward(sts, phmm, cells)

    # End to end through the C ABI with host buffers: every step copies its inputs from
    # pinned host memory to the device and its results back, both inside the timed region.
    # Same context (its plan, tuning and graph are reused); two batches in flight, as a
    # streaming caller would keep them: a step's upload overlaps the previous step's kernels.
    del d
    torch.cuda.empty_cache()
    keys = ("read_bases", "base_q", "ins_q", "del_q", "gcp_q", "hap_bases", "read_off", "hap_off",
            "pair_read", "pair_hap")
    hb = dict(b)
    for k in keys:
        hb[k] = torch.from_numpy(np.ascontiguousarray(b[k])).pin_memory().numpy()
    h2d = int(sum(hb[k].nbytes for k in keys))
    d2h = n * 9
    hout = [(torch.empty(n, dtype=torch.float64).pin_memory().numpy(),
             torch.zeros(n, dtype=torch.uint8).pin_memory().numpy()) for _ in range(2)]
    n_e2e = max(2, min(args.e2e_steps, args.steps) if args.e2e_steps > 0 else args.steps)

    overlap = [True]

    def e2e_run(k):
        pend = []
        for q in range(k):
            while True:
                try:
                    pend.append(ctx.submit(hb, *hout[q % 2]))
                    break
                except phmm.PhmmError as e:  # two batches do not fit the memory budget
                    if e.status != phmm.PHMM_EBUSY or not pend:
                        raise
                    overlap[0] = False
                    if ctx.poll(pend.pop(0), -1) != 0:
                        raise RuntimeError("e2e step failed")
            if len(pend) == 2 and ctx.poll(pend.pop(0), -1) != 0:
                raise RuntimeError("e2e step failed")
        while pend:
            if ctx.poll(pend.pop(0), -1) != 0:
                raise RuntimeError("e2e step failed")

    e2e_run(2)  # first copies into both slots' input arenas
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    e2e_run(n_e2e)
    e2e_ms = (time.perf_counter() - t0) * 1e3 / n_e2e
    e2e_ms = max_over_ranks([e2e_ms], world)[0]
    e2e_value = job_throughput(cells, world, e2e_ms)
    e2e_ok = all(bool(np.array_equal(np.nan_to_num(ho, nan=7.0), np.nan_to_num(res, nan=7.0)) or
                      np.max(np.abs(ho - res)) <= TOL32) for ho, _ in hout)
    ctx.close()
    del hb
    if rank != 0:
        return

    line = {
        "metric": METRIC, "value": value, "unit": "GCUPS", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": step_ms, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None,
        "dtype": {"fp32": "f32 (f64 rescue + reduction)", "fp64": "f64",
                  "fp32_only": "f32 (f64 reduction)"}[args.precision],
        "data": "synthetic (seeded, shaped like the paper's workloads)",
        "config": config_dict(name, units, b, world, args),
        "roofline": roofline(dom, info),
        "e2e": {"value": e2e_value, "unit": "GCUPS", "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                "ms_per_step": e2e_ms, "matches_device_run": e2e_ok,
                "how": "phmm_submit_batch/phmm_poll with pinned host inputs and pinned host outputs, "
                       "%s, %d steps, every step's H2D and D2H inside the timed region"
                       % ("two batches in flight (a step's upload overlaps the previous step's kernels)"
                          if overlap[0] else "one batch in flight (two exceed the memory budget)", n_e2e)},
        "gpu_launches": int(sum(s["kernel_launches"] for s in sts)),
        "clocks": clocks,
        "step": {"gcups_forward": cells / float(ms_fwd.mean()) / 1e6, "ms_forward": float(ms_fwd.mean()),
                 "branches": dom["all"], "rescued_pairs": int(sts[-1]["n_rescued"]),
                 "flagged_pairs": int(np.sum((flg & 0x78) != 0)), "first_submit_s": first_s,
                 "generate_s": gen_s, "wall_s": wall},
    }
    extras = args.extras
    if extras != "none":
        # cpu_baseline leg; its oracle values also check this run's outputs on those pairs
        cpu_v, cores, sdesc, cpu_s, pick, ref = oracle_sample(b, seconds=args.cpu_seconds)
        line["cpu_baseline"] = {"value": cpu_v, "unit": "GCUPS", "cores": cores, "kind": "oracle",
                                "sample": sdesc, "seconds": cpu_s}
        acc = {"random_sample": parity_block(b, res, flg, pick, ref)}
        acc["stratified"] = stratified_parity(b, res, flg)
        line["accuracy"] = acc
        comp = {"cpu_rowwise": cpu_rowwise(b, pick, ref, cores)}
        del b
        if name == "uneven" and extras == "all":
            legs = {}
            sb = make_workload("short", 2000)
            legs["short"] = gpu_leg("short", sb, dev, args, steps=10, warmup=3, flush=flush)
            legs["short"]["fp64_comparators"] = fp64_comparators(sb, dev, args)
            del sb
            lb = make_workload("long", 64)
            legs["long"] = gpu_leg("long", lb, dev, args, steps=5, warmup=2, flush=flush)
            f64 = gpu_leg("long fp64", lb, dev, args, steps=2, warmup=1, precision="fp64", parity="stratified",
                          flush=flush)
            legs["long"]["all_fp64_gpu"] = {k: f64[k] for k in ("gcups_step", "gcups_forward", "ms_per_step",
                                                                   "parity")}
            del lb
            line["legs"] = legs
        line["comparators"] = comp
        if args.serve_seconds > 0:
            line["serve"] = serve_leg(dev, args.serve_rate, args.serve_seconds, args.serve_pool)
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--config", default="uneven", choices=sorted(WORKLOADS),
                    help="workload (default: the 1M-pair uneven batch, the largest single-GPU workload)")
    ap.add_argument("--units", type=int, default=0,
                    help="pairs (uneven, long, plain) or regions (short) instead of the default; "
                         "smaller values only for profiling captures")
    ap.add_argument("--regions", type=int, default=0, help="same as --units for --config short")
    ap.add_argument("--min-len", type=int, default=32, help="sweep: shortest length")
    ap.add_argument("--max-len", type=int, default=16384, help="sweep: longest length")
    ap.add_argument("--sweep-pairs", type=int, default=0,
                    help="sweep: pairs per length (0: about 2e10 cells per length)")
    ap.add_argument("--variant", default="auto", choices=["auto", "packed", "scalar", "lean", "pipe", "pipe2", "pipe2lean"],
                    help="short-pair kernel family (default: the built-in tuner decides)")
    ap.add_argument("--cols", type=int, default=0, help="columns per lane (0: tuner)")
    ap.add_argument("--long-kind", default="auto",
                    choices=["auto", "lean", "pipe32", "pipe24", "serial", "pipe4", "cluster", "wave", "wave16"],
                    help="force one multi-warp kernel (default: the tuner decides)")
    ap.add_argument("--extras", default="all", choices=["all", "core", "none"],
                    help="all: cpu_baseline, parity, comparators, extra legs, serving; core: without the "
                         "extra workload legs; none: the timed headline only (profiling)")
    ap.add_argument("--uneven-max", type=int, default=20000,
                    help="uneven: longest read / haplotype (20000 = the benchmark; smaller only for "
                         "profiling captures)")
    ap.add_argument("--precision", default="fp32", choices=["fp32", "fp64", "fp32_only"],
                    help="precision of the timed run (fp32 = FP32 with FP64 rescue, the benchmark)")
    ap.add_argument("--e2e-steps", type=int, default=0,
                    help="end-to-end steps (host buffers); 0: as many as the timed steps")
    ap.add_argument("--cpu-seconds", type=float, default=12.0, help="cpu_baseline sample size in seconds")
    ap.add_argument("--lpp-pairs", type=int, default=4000,
                    help="pairs sampled for the FP64 launch-per-pair comparator")
    ap.add_argument("--serve-rate", type=float, default=8.0, help="requests per second of the serving leg")
    ap.add_argument("--serve-seconds", type=float, default=8.0, help="arrival window of the serving leg (0: skip)")
    ap.add_argument("--serve-pool", type=int, default=32, help="distinct region requests in the serving pool")
    args = ap.parse_args()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
