"""Throughput runs with sampled parity against the CPU oracle (test infrastructure).

    python tests/measure_parity.py configs --config long --precision both
    python tests/measure_parity.py sweep --min-len 32 --max-len 16384

``configs``: the named workload of paper_2606_25738_gb300.configs, timed on the GPU, then
checked on pairs sampled from every decile of the per-pair cell count plus every pair the
FP64 rescue recomputed (up to a cap); the oracle's own throughput on that sample is
reported for all host cores and for one core.  ``sweep``: the equal-length sweep, each
length checked on a sample of its pairs that the oracle finishes in seconds.
One JSON line per run.
"""
from __future__ import annotations

import argparse
import json
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_2606_25738_gb300 import configs, phmm, sweep  # noqa: E402
from paper_2606_25738_gb300 import workloads as W  # noqa: E402

TOL32, TOL64 = 1e-3, 1e-9


def check_sample(b, res, flags, pick, row):
    rl, hl = W.pair_lengths(b)
    t = time.perf_counter()
    ref = oracle.batch(b, pairs=pick)
    row["oracle_s"] = time.perf_counter() - t
    row["oracle_gcups_all_cores"] = float((rl[pick] * hl[pick]).sum()) / row["oracle_s"] / 1e9
    order = pick[np.argsort(rl[pick] * hl[pick])]
    csum = np.cumsum(rl[order] * hl[order])
    one = order[: max(1, int(np.searchsorted(csum, 3e8)))]
    t = time.perf_counter()
    oracle.batch(b, pairs=one, n_threads=1)
    row["oracle_gcups_1core"] = float((rl[one] * hl[one]).sum()) / (time.perf_counter() - t) / 1e9
    dd = np.abs(res[pick] - ref)
    fp64 = (flags[pick] & (phmm.PAIR_RESCUED | phmm.PAIR_FP64)) != 0
    row["checked_pairs"] = int(len(pick))
    row["max_abs_dlog10_fp32"] = float(dd[~fp64].max()) if (~fp64).any() else None
    row["max_abs_dlog10_fp64"] = float(dd[fp64].max()) if fp64.any() else None
    row["within_tolerance"] = bool(np.all(dd <= np.where(fp64, TOL64, TOL32)))
    return row


def run_configs(a):
    t = time.perf_counter()
    b = configs.MAKERS[a.config]()
    gen_s = time.perf_counter() - t
    precs = ["fp32", "fp64"] if a.precision == "both" else [a.precision]
    for p in precs:
        got = {}
        row = configs.run_config(a.config, b, p, steps=a.steps,
                                 on_result=lambda bb, res, fl: got.update(res=res, flags=fl))
        pick = configs.stratified_sample(b, a.per_decile)
        resc = np.flatnonzero(got["flags"] & phmm.PAIR_RESCUED)[:300]
        pick = np.unique(np.concatenate([pick, resc]))
        check_sample(b, got["res"], got["flags"], pick, row)
        row["gen_s"] = gen_s
        print(json.dumps(row), flush=True)


def run_sweep(a):
    lengths = []
    L = a.min_len
    while L <= a.max_len:
        lengths.append(L)
        L *= 2

    def on_result(L, b, res, flags):
        n = len(res)
        per = L * L
        m = int(max(1, min(n, 4e8 // per))) if per <= 4e8 else 0
        if not m:
            return {"checked_pairs": 0}
        pick = np.sort(np.random.default_rng(L).choice(n, m, replace=False))
        return check_sample(b, res, flags, pick, {})

    sweep.run(lengths, a.target_cells, precision=a.precision, steps=a.steps, log=sys.stdout,
              on_result=on_result)


def main():
    ap = argparse.ArgumentParser()
    sub = ap.add_subparsers(dest="what", required=True)
    c = sub.add_parser("configs")
    c.add_argument("--config", required=True, choices=sorted(configs.MAKERS))
    c.add_argument("--precision", default="fp32", choices=["fp32", "fp64", "fp32_only", "both"])
    c.add_argument("--steps", type=int, default=3)
    c.add_argument("--per-decile", type=int, default=200)
    s = sub.add_parser("sweep")
    s.add_argument("--min-len", type=int, default=32)
    s.add_argument("--max-len", type=int, default=16384)
    s.add_argument("--target-cells", type=float, default=2e10)
    s.add_argument("--precision", default="fp32", choices=["fp32", "fp64", "fp32_only"])
    s.add_argument("--steps", type=int, default=3)
    a = ap.parse_args()
    if a.what == "configs":
        run_configs(a)
    else:
        run_sweep(a)


if __name__ == "__main__":
    main()
