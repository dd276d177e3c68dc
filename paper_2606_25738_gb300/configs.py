"""Runs one named workload through the C ABI and reports its throughput.

    python -m paper_2606_25738_gb300.configs --config long --precision both

Workloads (see workloads.py): ``plain`` (64 short pairs), ``short`` (the short-read
region batch), ``long`` (64 long-read pairs, haplotypes 1k-100k bp), ``uneven`` (1M pairs
of log-uniform 50-20k bp lengths).  Each precision is run as one batch: one submit, the
timed steps replaying its captured graph.  One JSON line per (workload, precision).
``stratified_sample`` picks the pairs a parity check looks at (tests/measure_parity.py).
"""
from __future__ import annotations

import argparse
import json
import sys
import time

import numpy as np

from . import phmm
from . import workloads as W

MAKERS = {
    "plain": lambda: W.plain_pairs(64, seed=0),
    "short": lambda: W.short_read_regions(2000, seed=0),
    "long": lambda: W.long_pairs(64, seed=0),
    "uneven": lambda: W.uneven_pairs(1_000_000, seed=0),
}


def stratified_sample(b: dict, per_decile: int, seed: int = 0, max_cells: float = 4e10):
    """Pair indices: up to ``per_decile`` random pairs from each decile of l*k, keeping the
    sample's total cells under ``max_cells`` (largest deciles thinned first)."""
    rl, hl = W.pair_lengths(b)
    c = rl * hl
    order = np.argsort(c, kind="stable")
    rng = np.random.default_rng(seed)
    picks = []
    for dec in np.array_split(order, 10):
        if len(dec):
            picks.append(rng.choice(dec, min(per_decile, len(dec)), replace=False))
    pick = np.unique(np.concatenate(picks))
    while c[pick].sum() > max_cells and len(pick) > 10:
        big = np.argsort(c[pick])[::-1]
        pick = np.delete(pick, big[: max(1, len(pick) // 20)])
    return pick


def run_config(name: str, b: dict, precision: str, steps: int = 3, variant: str = "auto",
               on_result=None) -> dict:
    """One batch through the C ABI: a first submit (plan, tuning, graph capture), then
    ``steps`` timed replays.  ``on_result(b, log10_L, flags)`` (optional) receives the
    last step's host outputs, for a caller that checks them."""
    import torch
    n = len(b["pair_read"])
    cells = W.cells(b)
    d = phmm.to_device(b)
    out = torch.empty(n, dtype=torch.float64, device="cuda")
    fl = torch.zeros(n, dtype=torch.uint8, device="cuda")
    with phmm.Context(precision=precision, max_inflight=1, variant=variant) as ctx:
        t = time.perf_counter()
        ctx.poll(ctx.submit(d, out, fl), -1)
        first_s = time.perf_counter() - t
        st = []
        for _ in range(steps):
            tk = ctx.submit(d, out, fl)
            rc = ctx.poll(tk, -1)
            if rc != phmm.PHMM_OK:
                raise phmm.PhmmError(rc, "%s %s" % (name, precision))
            st.append(ctx.stats(tk))
    fwd = float(np.mean([s["ms_forward"] for s in st]))
    tot = float(np.mean([s["ms_total"] for s in st]))
    row = {"config": name, "precision": precision, "pairs": n, "cells": cells,
           "ms_forward": fwd, "ms_total": tot, "gcups_kernel": cells / fwd / 1e6,
           "gcups_total": cells / tot / 1e6, "rescued": int(st[-1]["n_rescued"]),
           "kernel_launches": int(st[-1]["kernel_launches"]), "first_submit_s": first_s}
    if on_result is not None:
        on_result(b, out.cpu().numpy(), fl.cpu().numpy())
    return row


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--config", required=True, choices=sorted(MAKERS))
    ap.add_argument("--precision", default="fp32", choices=["fp32", "fp64", "fp32_only", "both"])
    ap.add_argument("--steps", type=int, default=3)
    a = ap.parse_args(argv)
    t = time.perf_counter()
    b = MAKERS[a.config]()
    gen_s = time.perf_counter() - t
    precs = ["fp32", "fp64"] if a.precision == "both" else [a.precision]
    for p in precs:
        row = run_config(a.config, b, p, steps=a.steps)
        row["gen_s"] = gen_s
        print(json.dumps(row), flush=True)


if __name__ == "__main__":
    sys.exit(main())
