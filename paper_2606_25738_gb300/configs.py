"""Runs one named workload through the C ABI and reports its throughput.

    python -m paper_2606_25738_gb300.configs --config long --precision both
    python -m paper_2606_25738_gb300.configs --config uneven --units 5000 --long-kind serial

Workloads (see workloads.py): ``plain`` (64 short pairs), ``short`` (the short-read
region batch), ``long`` (64 long-read pairs, haplotypes 1k-100k bp), ``uneven`` (1M pairs
of log-uniform 50-20k bp lengths); ``--units`` scales a workload (pairs, or regions for
``short``) and ``--long-kind`` forces one multi-warp kernel.  Each precision is run as one
batch: one submit, the timed steps replaying its captured graph.  One JSON line per
(workload, precision).
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
    "plain": lambda n=64: W.plain_pairs(n, seed=0),
    "short": lambda n=2000: W.short_read_regions(n, seed=0),
    "long": lambda n=64: W.long_pairs(n, seed=0),
    "uneven": lambda n=1_000_000: W.uneven_pairs(n, seed=0),
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
               on_result=None, flags: int = 0) -> dict:
    """One batch through the C ABI: a first submit (plan, tuning, graph capture), then
    ``steps`` timed replays.  ``on_result(b, log10_L, flags)`` (optional) receives the
    last step's host outputs, for a caller that checks them."""
    import torch
    n = len(b["pair_read"])
    cells = W.cells(b)
    d = phmm.to_device(b)
    out = torch.empty(n, dtype=torch.float64, device="cuda")
    fl = torch.zeros(n, dtype=torch.uint8, device="cuda")
    with phmm.Context(precision=precision, max_inflight=1, variant=variant, flags=flags) as ctx:
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
           "kernel_launches": int(st[-1]["kernel_launches"]), "first_submit_s": first_s,
           "short_kernel": int(st[-1]["short_kernel"]), "long_kernel": int(st[-1]["long_kernel"])}
    if on_result is not None:
        on_result(b, out.cpu().numpy(), fl.cpu().numpy())
    return row


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--config", required=True, choices=sorted(MAKERS))
    ap.add_argument("--precision", default="fp32", choices=["fp32", "fp64", "fp32_only", "both"])
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--units", type=int, default=0,
                    help="pairs (plain, long, uneven) or regions (short) instead of the default")
    ap.add_argument("--long-kind", default="auto", choices=["auto", "lean", "pipe32", "pipe24", "serial", "pipe4"],
                    help="force one multi-warp kernel")
    a = ap.parse_args(argv)
    flags = {"auto": 0, "lean": phmm.F_LONG_LEAN, "pipe32": phmm.F_LONG_PIPE32,
             "pipe24": phmm.F_LONG_PIPE24, "serial": phmm.F_LONG_SERIAL, "pipe4": phmm.F_LONG_PIPE4}[a.long_kind]
    t = time.perf_counter()
    b = MAKERS[a.config](a.units) if a.units > 0 else MAKERS[a.config]()
    gen_s = time.perf_counter() - t
    precs = ["fp32", "fp64"] if a.precision == "both" else [a.precision]
    for p in precs:
        row = run_config(a.config, b, p, steps=a.steps, flags=flags)
        row["gen_s"] = gen_s
        print(json.dumps(row), flush=True)


if __name__ == "__main__":
    sys.exit(main())
