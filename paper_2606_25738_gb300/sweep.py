"""Equal-length scalability sweep (the shape of the paper's Section 4.3: read length =
haplotype length = 32 .. 131072 bp), through the library's C ABI.

For each length L the batch holds about ``target_cells`` cell updates (at least one
pair, at most ``max_pairs``).  GCUPS are reported for the forward kernels alone (the
paper's kernel-only convention for this experiment) and for the whole device pipeline
of a batch (prep, forward, reduction, rescue selection and rescue).  Parity of the sweep's
batches is checked by tests/measure_parity.py.

    python -m paper_2606_25738_gb300.sweep [--max-len 131072] [--precision fp32]
"""
from __future__ import annotations

import argparse
import json
import sys
import time

import numpy as np

from . import phmm
from . import workloads as W


def run(lengths, target_cells: float = 2e10, max_pairs: int = 1 << 20, precision: str = "fp32",
        steps: int = 3, device: int = 0, log=None, on_result=None):
    """One batch per length L of about ``target_cells`` cells (at least one pair, at most
    ``max_pairs``).  ``on_result(L, batch, log10_L, flags)`` (optional) receives each
    batch's host outputs, for a caller that checks them."""
    import torch
    rows = []
    for L in lengths:
        n = int(min(max_pairs, max(1, round(target_cells / (L * L)))))
        t = time.perf_counter()
        b = W.equal_length(n, L, seed=0)
        gen_s = time.perf_counter() - t
        cells = W.cells(b)
        d = phmm.to_device(b)
        out = torch.empty(n, dtype=torch.float64, device="cuda")
        fl = torch.zeros(n, dtype=torch.uint8, device="cuda")
        with phmm.Context(device=device, precision=precision, max_inflight=1) as ctx:
            ctx.poll(ctx.submit(d, out, fl), -1)  # plan, tune, capture
            st = []
            for _ in range(steps):
                tk = ctx.submit(d, out, fl)
                rc = ctx.poll(tk, -1)
                if rc != phmm.PHMM_OK:
                    raise phmm.PhmmError(rc, "sweep L=%d" % L)
                st.append(ctx.stats(tk))
        fwd = float(np.mean([s["ms_forward"] for s in st]))
        tot = float(np.mean([s["ms_total"] for s in st]))
        row = {"L": L, "pairs": n, "cells": cells, "ms_forward": fwd, "ms_total": tot,
               "gcups_kernel": cells / fwd / 1e6, "gcups_total": cells / tot / 1e6,
               "rescued": int(st[-1]["n_rescued"]), "cols_per_lane": int(st[-1]["cols_per_lane"]),
               "gen_s": gen_s}
        if on_result is not None:
            row.update(on_result(L, b, out.cpu().numpy(), fl.cpu().numpy()) or {})
        rows.append(row)
        if log:
            print(json.dumps(row), file=log, flush=True)
    return rows


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--min-len", type=int, default=32)
    ap.add_argument("--max-len", type=int, default=131072)
    ap.add_argument("--target-cells", type=float, default=2e10)
    ap.add_argument("--precision", default="fp32", choices=["fp32", "fp64", "fp32_only"])
    ap.add_argument("--steps", type=int, default=3)
    a = ap.parse_args(argv)
    lengths = []
    L = a.min_len
    while L <= a.max_len:
        lengths.append(L)
        L *= 2
    run(lengths, a.target_cells, precision=a.precision, steps=a.steps, log=sys.stdout)


if __name__ == "__main__":
    main()
