"""Open-loop load driver for the library's serving loop (phmm_server_*).

Requests (active regions, workloads.region_request) arrive as a Poisson stream at
``rate`` per second for ``duration`` seconds.  A submitter thread enqueues each one at
its arrival time; a collector thread waits for completions.  A request's latency runs
from its scheduled arrival to the completion of its results, so time spent behind a
lagging submitter counts too.  Request data comes from a seeded pool of distinct
regions (request i uses pool entry i mod pool size).

All scheduling, admission and batching happen in the library; this module only drives
arrivals and collects timings.  Give the context PHMM_F_NO_TUNE: every epoch is a batch of
a new shape, and measured tuning would re-run each one.
"""
from __future__ import annotations

import threading
import time

import numpy as np

from . import phmm
from . import workloads as W


def make_pool(n: int = 64, seed: int = 0, **kw) -> list:
    pool = W.serving_requests(n, seed=seed, **kw)
    return [(r, W.cells(r), len(r["pair_read"])) for r in pool]


def run(ctx: "phmm.Context", pool: list, rate: float, duration: float, seed: int = 1,
        drain_s: float = 60.0, mem_budget: int = 40 << 30, max_epoch_pairs: int = 0,
        max_inflight_epochs: int = 2, epoch_cells: int = 0, small_cells: int = 0,
        max_wait_ms: int = 0) -> dict:
    """Drive one open-loop run; returns latency percentiles (all requests, and the
    server's small and large size classes), throughput and counts."""
    rng = np.random.default_rng(seed)
    gaps = rng.exponential(1.0 / rate, size=int(rate * duration * 1.5) + 16)
    arr = np.cumsum(gaps)
    arr = arr[arr < duration]
    recs = {}  # rid -> [pool index, scheduled arrival, enqueue return]
    lock = threading.Lock()
    done = {}
    rejected = [0]
    stop_collect = threading.Event()

    with phmm.Server(ctx, mem_budget=mem_budget, max_epoch_pairs=max_epoch_pairs,
                     max_inflight_epochs=max_inflight_epochs, epoch_cells=epoch_cells,
                     small_cells=small_cells, max_wait_ms=max_wait_ms) as srv:
        t0 = time.perf_counter()

        def submitter():
            for i, ta in enumerate(arr):
                now = time.perf_counter() - t0
                if ta > now:
                    time.sleep(ta - now)
                req = pool[i % len(pool)][0]
                try:
                    rid = srv.enqueue(req)
                except phmm.PhmmError:
                    rejected[0] += 1
                    continue
                with lock:
                    recs[rid] = [i % len(pool), float(ta), time.perf_counter() - t0]

        def collector():
            while not stop_collect.is_set():
                with lock:
                    ids = [r for r in recs if r not in done]
                if not ids:
                    time.sleep(0.002)
                    continue
                for rid in ids:
                    rc, lat, out, fl = srv.poll(rid, 0)
                    if rc == phmm.PHMM_PENDING:
                        continue
                    with lock:
                        done[rid] = (rc, time.perf_counter() - t0, out, fl)
                time.sleep(0.0005)

        ts = threading.Thread(target=submitter)
        tc = threading.Thread(target=collector)
        ts.start()
        tc.start()
        ts.join()
        t_arrivals_end = time.perf_counter() - t0
        st_end = srv.stats()
        deadline = time.perf_counter() + drain_s
        while time.perf_counter() < deadline:
            with lock:
                if len(done) >= len(recs):
                    break
            time.sleep(0.01)
        stop_collect.set()
        tc.join()
        st = srv.stats()
        t_last = max([d[1] for d in done.values()], default=t_arrivals_end)
    # the server is destroyed here: requests still waiting were cancelled
    ok = [rid for rid, d in done.items() if d[0] in (phmm.PHMM_OK, phmm.PHMM_EINVAL)]
    lat = np.array([done[rid][1] - recs[rid][1] for rid in ok]) * 1e3
    cells_done = float(sum(pool[recs[rid][0]][1] for rid in ok))
    lag = np.array([recs[rid][2] - recs[rid][1] for rid in recs]) * 1e3 if recs else np.zeros(1)
    small_max = small_cells or (epoch_cells or 20_000_000_000) // 20
    by_class = {}
    for name, pick in (("small", lambda c: c <= small_max), ("large", lambda c: c > small_max)):
        ids = [rid for rid in ok if pick(pool[recs[rid][0]][1])]
        lc = np.array([done[rid][1] - recs[rid][1] for rid in ids]) * 1e3
        by_class[name] = {"completed": len(ids),
                          "p50_ms": float(np.percentile(lc, 50)) if len(lc) else None,
                          "p99_ms": float(np.percentile(lc, 99)) if len(lc) else None}
    by_class["small_max_cells"] = int(small_max)
    return {
        "by_class": by_class,
        "offered_rate": rate, "duration_s": duration, "arrivals": int(len(arr)),
        "enqueued": len(recs), "rejected": rejected[0], "completed": len(ok),
        "not_completed": len(recs) - len(ok),
        "backlog_at_arrivals_end": int(st_end["pending"] + st_end["inflight"]),
        "p50_ms": float(np.percentile(lat, 50)) if len(lat) else None,
        "p99_ms": float(np.percentile(lat, 99)) if len(lat) else None,
        "mean_ms": float(lat.mean()) if len(lat) else None,
        "gcups": cells_done / max(t_last, 1e-9) / 1e9,
        "cells_completed": cells_done, "epochs": int(st["epochs"]),
        "submit_lag_p99_ms": float(np.percentile(lag, 99)),
        "span_s": t_last,
    }
