"""Benchmark: GCUPS of the FP32 + FP64-rescue PairHMM forward path on the short-read batch
workload (2000 active regions x 50 reads of 150 bp x 1-8 haplotypes of 250-600 bp, about
455k pairs / 2.9e10 cell updates), seeded synthetic data.

One step = one pass of the whole hot path over the batch (coefficient prep, the forward
kernel, log10 reduction, rescue selection and the FP64 rescue pass) with inputs resident
in device memory.  Prints one JSON line (rank 0).  ``--impl reference`` times the CPU
oracle on the host cores instead, on a bounded sample of the same workload.
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

METRIC = "GCUPS (FP32+FP64-rescue vs plain FP64, |\u0394log10|\u22641e-3); serve p50/p99 ms"
WORKLOAD = "short-read batch: 2000 regions x 50 reads (150 bp) x 1-8 haplotypes (250-600 bp)"


def _env_rank():
    return int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")), \
        int(os.environ.get("LOCAL_RANK", "0"))


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


def _oracle_sample(b, seconds: float = 15.0, seed: int = 1):
    """The cpu_baseline leg: the CPU oracle (test infrastructure) on a random sample of the
    batch's pairs sized to roughly ``seconds`` of work on all host cores.  Returns (GCUPS,
    cores, description, seconds, sampled pair indices, their oracle log10 L)."""
    import oracle
    from paper_2606_25738_gb300 import workloads as W
    cores = os.cpu_count() or 1
    rl, hl = W.pair_lengths(b)
    n = len(rl)
    rng = np.random.default_rng(seed)
    order = rng.permutation(n)
    # calibrate on a small sample
    probe = order[:max(cores * 4, 64)]
    t = time.perf_counter()
    oracle.batch(b, pairs=probe, n_threads=cores)
    dt = time.perf_counter() - t
    rate = float(np.sum(rl[probe] * hl[probe])) / max(dt, 1e-6)
    want = rate * seconds
    csum = np.cumsum(rl[order] * hl[order])
    m = int(min(n, max(len(probe), np.searchsorted(csum, want) + 1)))
    pick = order[:m]
    cells = float(np.sum(rl[pick] * hl[pick]))
    t = time.perf_counter()
    ref = oracle.batch(b, pairs=pick, n_threads=cores)
    dt = time.perf_counter() - t
    return (cells / dt / 1e9, cores,
            "%d random pairs of the workload (%.3g cells), FP64 cell-by-cell, %d threads" % (m, cells, cores),
            dt, pick, ref)


def run_reference(args):
    rank, world, _ = _env_rank()
    if rank != 0:
        return
    from paper_2606_25738_gb300 import workloads as W
    b = W.short_read_regions(args.regions, seed=0)
    vals = []
    # each step is a bounded random sample of the workload, sized so that the whole run
    # stays within about three minutes of host time
    per_step = max(0.5, min(8.0, 150.0 / max(1, args.steps + args.warmup)))
    for _ in range(args.warmup):
        _oracle_sample(b, seconds=min(2.0, per_step))
    desc = ""
    cores = 1
    for k in range(args.steps):
        v, cores, desc, _dt, _pick, _ref = _oracle_sample(b, seconds=per_step, seed=10 + k)
        vals.append(v)
    value = float(np.median(vals))
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "GCUPS",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic (seeded short-read regions)",
            "config": {"workload": WORKLOAD if args.regions == 2000 else WORKLOAD.replace("2000", str(args.regions)),
                       "pairs": int(len(b["pair_read"])), "reads": int(len(b["read_off"]) - 1),
                       "cells": int(W.cells(b))},
            "cpu_baseline": {"value": value, "unit": "GCUPS", "cores": cores, "kind": "oracle",
                             "sample": desc},
            "e2e": {"value": value, "unit": "GCUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def _nvtx(torch, name):
    try:
        if name:
            torch.cuda.nvtx.range_push(name)
        else:
            torch.cuda.nvtx.range_pop()
    except Exception:
        pass


def _serve_leg(dev, args):
    """A short open-loop run of the library's serving loop on region requests (R reads
    U{10..500} x H haplotypes U{2..16}; 80% 150 bp reads, 20% log-uniform 1k-20k bp;
    haplotypes 1.5-3x the read length; 40 GB admission budget)."""
    from paper_2606_25738_gb300 import phmm
    from paper_2606_25738_gb300 import serving
    pool = serving.make_pool(args.serve_pool, seed=0)
    with phmm.Context(device=dev, precision="fp32", max_inflight=3, flags=phmm.F_NO_TUNE) as c:
        r = serving.run(c, pool, rate=args.serve_rate, duration=args.serve_seconds, drain_s=60.0,
                        max_inflight_epochs=3)
    r["pool"] = "%d seeded region requests, mean %.3g cells" % (len(pool), sum(p[1] for p in pool) / len(pool))
    return r


def _cpu_rowwise(b, pick, ref, cores):
    """The library's row-wise CPU path (libphmm_cpu.so, FP64, all host cores) on the pairs
    the cpu_baseline leg sampled, checked against the oracle's values for them."""
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
            "what": "row-wise CPU path (FP64, vectorised loops, blocked deletion chain) on the "
                    "cpu_baseline sample"}


def _fp64_comparators(b, d, dev, args):
    """The all-FP64 GPU comparators on the same workload (outside the timed region):
    the batched FP64 path of this library over the whole batch, and a plain FP64
    one-launch-per-pair run over a bounded random sample of its pairs."""
    import torch

    from paper_2606_25738_gb300 import phmm
    from paper_2606_25738_gb300 import workloads as W
    n = len(b["pair_read"])
    cells = W.cells(b)
    res = {}
    out = torch.empty(n, dtype=torch.float64, device="cuda")
    fl = torch.zeros(n, dtype=torch.uint8, device="cuda")
    with phmm.Context(device=dev, precision="fp64", max_inflight=1) as c64:
        for _ in range(2):
            c64.poll(c64.submit(d, out, fl), -1)
        ms = []
        for _ in range(3):
            t = c64.submit(d, out, fl)
            if c64.poll(t, -1) != 0:
                raise RuntimeError("fp64 batched run failed")
            ms.append(c64.stats(t)["ms_total"])
        res["fp64_batched"] = {"value": cells / (float(np.mean(ms)) * 1e-3) / 1e9, "unit": "GCUPS",
                               "ms_per_step": float(np.mean(ms)),
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
    # Replicas: every rank scores its own copy of the workload (pairs are independent;
    # there is no exchange step), so per-GPU work is fixed as N grows.
    b = W.short_read_regions(args.regions, seed=0)
    n = len(b["pair_read"])
    cells = W.cells(b)
    stream = torch.cuda.Stream(device=dev)
    d = phmm.to_device(b)
    out = torch.empty(n, dtype=torch.float64, device="cuda")
    fl = torch.zeros(n, dtype=torch.uint8, device="cuda")
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")  # > L2 (129 MB)
    ctx = phmm.Context(device=dev, precision="fp32", stream=stream.cuda_stream, max_inflight=2,
                       variant=args.variant, cols_per_lane=args.cols)
    info = ctx.device_info()

    def step():
        with torch.cuda.stream(stream):
            flush.fill_(1.0)  # evict L2 between steps (outside the library's events)
        t = ctx.submit(d, out, fl)
        rc = ctx.poll(t, -1)
        if rc != 0:
            raise RuntimeError("poll status %d" % rc)
        return ctx.stats(t)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    sts = []
    with ClockSampler(dev) as clk:
        torch.cuda.synchronize()
        _nvtx(torch, "timed")  # lets a profiler restrict itself to the timed steps
        t0 = time.perf_counter()
        for _ in range(args.steps):
            sts.append(step())
        torch.cuda.synchronize()
        wall = time.perf_counter() - t0
        _nvtx(torch, None)
    if world > 1:
        torch.distributed.barrier()
    ms = np.array([s["ms_total"] for s in sts])
    ms_fwd = np.array([s["ms_forward"] for s in sts])
    step_ms = float(ms.mean())
    step_ms, wall = max_over_ranks([step_ms, wall], world)
    value = job_throughput(cells, world, step_ms)
    # accuracy gate on a sample of this run's outputs
    res = out.cpu().numpy()
    flg = fl.cpu().numpy()

    # End to end through the C ABI with host buffers: every step copies its inputs from
    # pinned host memory to the device and its results back, both inside the timed region.
    # The caller keeps two batches in flight (two slots), as a pipelined client would, so
    # one step's copies overlap the previous step's kernels.
    keys = ("read_bases", "base_q", "ins_q", "del_q", "gcp_q", "hap_bases", "read_off", "hap_off",
            "pair_read", "pair_hap")
    hb = dict(b)
    for k in keys:
        hb[k] = torch.from_numpy(np.ascontiguousarray(b[k])).pin_memory().numpy()
    h2d = int(sum(hb[k].nbytes for k in keys))
    d2h = n * 9
    bufs = [(np.empty(n, dtype=np.float64), np.zeros(n, dtype=np.uint8)) for _ in range(2)]
    n_e2e = max(4, args.steps // 2)
    with phmm.Context(device=dev, precision="fp32", max_inflight=2) as hctx:

        def pipelined(count):
            pending = []
            for q in range(count):
                if len(pending) == 2:
                    if hctx.poll(pending.pop(0), -1) != 0:
                        raise RuntimeError("e2e step failed")
                o, f = bufs[q % 2]
                pending.append(hctx.submit(hb, o, f))
            for t in pending:
                if hctx.poll(t, -1) != 0:
                    raise RuntimeError("e2e step failed")

        pipelined(4)  # plans, tuning and graphs of both slots
        t0 = time.perf_counter()
        pipelined(n_e2e)
        e2e_ms = [(time.perf_counter() - t0) * 1e3 / n_e2e]
    e2e_value = job_throughput(cells, world, max_over_ranks([float(np.median(e2e_ms))], world)[0])
    if rank != 0:
        ctx.close()
        return
    comparators = _fp64_comparators(b, d, dev, args)
    serve = _serve_leg(dev, args) if args.serve_seconds > 0 else None

    peaks = _peaks()
    sm_max = float(peaks.get("sm_max_mhz", info["max_clock_mhz"]))
    peak_tflops = 2.0 * 128 * info["sms"] * sm_max * 1e6 / 1e12
    fwd_ms = float(ms_fwd.mean())
    achieved = 12.0 * cells / (fwd_ms * 1e-3) / 1e12
    # cpu_baseline leg; the same oracle values check this run's results on the sampled pairs
    cpu_v, cores, sdesc, _, pick, ref = _oracle_sample(b, seconds=12.0)
    fp64 = (flg[pick] & 0x5) != 0
    err = float(np.max(np.abs(res[pick] - ref)[~fp64])) if (~fp64).any() else 0.0
    comparators["cpu_rowwise"] = _cpu_rowwise(b, pick, ref, cores)
    clocks = clk.summary()
    # the dominant kernel is the short-team kernel the plan ran; its DRAM bytes per launch
    # come from an ncu capture of that same kernel (null for any other kernel)
    sk = int(sts[-1]["short_kernel"])
    kname = phmm.SHORT_KERNELS[sk] if 0 <= sk < len(phmm.SHORT_KERNELS) else "none"
    traffic = None
    tfile = os.path.join(ROOT, "profiles", "forward_traffic.json")
    if os.path.exists(tfile):
        try:
            traffic = json.load(open(tfile)).get(kname, {}).get("bytes_per_launch")
        except Exception:
            traffic = None
    line = {
        "metric": METRIC, "value": value, "unit": "GCUPS", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": step_ms, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32 (f64 rescue + reduction)",
        "data": "synthetic (seeded short-read regions)",
        "config": {"workload": WORKLOAD if args.regions == 2000 else WORKLOAD.replace("2000", str(args.regions)), "pairs": n, "reads": len(b["read_off"]) - 1,
                   "cells": cells, "cols_per_lane": int(sts[-1]["cols_per_lane"]),
                   "l2": "flushed between steps (256 MB write outside the timed events)",
                   "parallelism": "replicas" if world > 1 else "single GPU"},
        "roofline": {"bound": "alu", "achieved": achieved, "peak": peak_tflops, "unit": "TFLOP/s",
                     "frac": achieved / peak_tflops, "traffic": traffic,
                     "kernel": "FP32 forward branches; short teams on %s" % kname,
                     "flop_per_cell": 12,
                     "peak_note": "2 x 128 FP32 lanes x %d SMs x %.0f MHz (max SM clock, MEASURED_PEAKS)" % (info["sms"], sm_max)},
        "cpu_baseline": {"value": cpu_v, "unit": "GCUPS", "cores": cores, "kind": "oracle",
                         "sample": sdesc},
        "e2e": {"value": e2e_value, "unit": "GCUPS", "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h, "ms_per_step": float(np.median(e2e_ms)),
                "how": "phmm_submit_batch/phmm_poll with pinned host inputs and host outputs, "
                       "2 batches in flight, %d steps" % n_e2e},
        "gpu_launches": int(sum(s["kernel_launches"] for s in sts)),
        "clocks": clocks,
        "accuracy": {"max_abs_dlog10_sample": err, "sample_pairs": int(len(pick)),
                     "rescued_pairs": int(sts[-1]["n_rescued"]),
                     "flagged": int(np.sum((flg & 0x78) != 0))},
        "comparators": comparators,
        "serve": serve,
        "ms_forward": fwd_ms, "wall_s": wall,
    }
    print(json.dumps(line), flush=True)
    ctx.close()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--variant", default="auto", choices=["auto", "packed", "scalar", "lean", "pipe"],
                    help="short-pair kernel family (default: the built-in tuner decides)")
    ap.add_argument("--cols", type=int, default=0, help="columns per lane (0: tuner)")
    ap.add_argument("--regions", type=int, default=2000,
                    help="active regions of the workload (2000 = the benchmark size; smaller "
                         "values only for profiling captures)")
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
