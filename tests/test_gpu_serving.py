"""Concurrent batches and the serving loop (phmm_server_*), on the GPU.

Each request's results must be the same when it is scored alone and when it is scored
inside the mix of a continuous-batching run (|dlog10| <= 1e-3, the FP32 tolerance; the
request's pairs land at other offsets of a joined batch), and must match the oracle.
"""
import numpy as np
import pytest

import oracle
from paper_2606_25738_gb300 import workloads as W

pytestmark = pytest.mark.gpu

TOL32 = 1e-3


@pytest.fixture(scope="module")
def phmm():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2606_25738_gb300 import phmm as P
    return P


def _small_pool(n=10, seed=3):
    return W.serving_requests(n, seed=seed, reads_range=(4, 16), haps_range=(2, 4), long_frac=0.3,
                              long_range=(1000, 2000))


def test_concurrent_slots_match_sequential(phmm):
    """Two batches in flight at once on one context (separate slots and streams) give
    the same bits as the same batches run one at a time."""
    a = W.plain_pairs(300, seed=11, k_range=(200, 1200))
    b = W.long_pairs(4, seed=12, k_range=(1000, 3000))
    with phmm.Context(max_inflight=2) as ctx:
        ra, fa, _, _ = ctx.run(a)
        rb, fb, _, _ = ctx.run(b)
        oa, ob = np.empty_like(ra), np.empty_like(rb)
        ga, gb = np.zeros_like(fa), np.zeros_like(fb)
        ta = ctx.submit(a, oa, ga)
        tb = ctx.submit(b, ob, gb)
        assert ctx.poll(tb, -1) == 0
        assert ctx.poll(ta, -1) == 0
    assert np.array_equal(ra, oa) and np.array_equal(fa, ga)
    assert np.array_equal(rb, ob) and np.array_equal(fb, gb)


def test_server_alone_vs_mix(phmm):
    pool = _small_pool()
    with phmm.Context(max_inflight=2, variant="scalar", cols_per_lane=32) as ctx:
        alone = [ctx.run(r)[0] for r in pool]
    with phmm.Context(max_inflight=2, variant="scalar", cols_per_lane=32) as ctx:
        with phmm.Server(ctx, max_inflight_epochs=2) as srv:
            ids = [srv.enqueue(r) for r in pool] + [srv.enqueue(r) for r in pool[:4]]
            res = [srv.poll(i, -1) for i in ids]
            st = srv.stats()
    assert st["completed"] == len(ids) and st["failed"] == 0 and st["pending"] == 0
    assert 1 <= st["epochs"] <= len(ids)
    for q, (rc, lat, out, fl) in enumerate(res):
        assert rc == 0 and lat > 0
        r = q if q < len(pool) else q - len(pool)
        assert np.max(np.abs(out - alone[r])) <= TOL32
    for r in range(len(pool)):
        ref = oracle.batch(pool[r])
        out, fl = res[r][2], res[r][3]
        tol = np.where((fl & 0x5) != 0, 1e-9, TOL32)
        assert np.all(np.abs(out - ref) <= tol)


def test_server_chunks_large_requests_and_runs_small_first(phmm):
    """A request larger than the epoch cell budget is split into chunks of consecutive
    pairs across epochs and still gets the same results as alone; small requests queued
    behind it complete before it (they go ahead between its chunks)."""
    import time
    big = W.long_pairs(24, seed=31, k_range=(1500, 3000))
    smalls = [W.plain_pairs(3, seed=40 + q) for q in range(6)]
    big_cells = W.cells(big)
    with phmm.Context(max_inflight=2, variant="scalar", cols_per_lane=32) as ctx:
        alone = ctx.run(big)[0]
        with phmm.Server(ctx, max_inflight_epochs=2, epoch_cells=big_cells // 8,
                         small_cells=big_cells // 100) as srv:
            ib = srv.enqueue(big)
            time.sleep(0.001)
            ids = [srv.enqueue(r) for r in smalls]
            res = [srv.poll(i, -1) for i in ids]
            rb = srv.poll(ib, -1)
            st = srv.stats()
    assert rb[0] == 0 and np.max(np.abs(rb[2] - alone)) <= TOL32
    assert st["epochs"] >= 8 + 1  # the large request alone needs at least 8 chunks
    assert st["completed"] == 1 + len(smalls) and st["failed"] == 0 and st["pending"] == 0
    big_lat = rb[1]
    for q, (rc, lat, out, fl) in enumerate(res):
        assert rc == 0
        assert lat < big_lat
        assert np.max(np.abs(out - oracle.batch(smalls[q]))) <= TOL32


def test_server_error_isolated_to_its_request(phmm):
    good = W.plain_pairs(6, seed=21)
    bad = W.from_strings([("ACGT", "ACGT", 30, 45, 45, 10), ("AXGT", "ACGT", 30, 45, 45, 10)])
    with phmm.Context() as ctx:
        with phmm.Server(ctx) as srv:
            i1, i2, i3 = srv.enqueue(good), srv.enqueue(bad), srv.enqueue(good)
            r1, r2, r3 = srv.poll(i1, -1), srv.poll(i2, -1), srv.poll(i3, -1)
            assert srv.poll(i1, 0)[0] == phmm.PHMM_ENOTFOUND
    assert r1[0] == 0 and r3[0] == 0
    assert r2[0] == phmm.PHMM_EINVAL
    assert np.isfinite(r2[2][0]) and np.isnan(r2[2][1]) and (r2[3][1] & phmm.PAIR_ERROR)
    ref = oracle.batch(good)
    assert np.max(np.abs(r1[2] - ref)) <= TOL32 and np.max(np.abs(r3[2] - ref)) <= TOL32


def test_server_budget_rejects_oversize(phmm):
    b = W.plain_pairs(8, seed=22)
    with phmm.Context() as ctx:
        f = ctx.footprint(b)
        assert f > 0
        assert ctx.footprint(W.subset(b, [0, 1])) <= f
        with phmm.Server(ctx, mem_budget=f - 1) as srv:
            with pytest.raises(phmm.PhmmError) as e:
                srv.enqueue(b)
            assert e.value.status == phmm.PHMM_ENOMEM
        # a budget for one request at a time: requests are admitted one after another
        with phmm.Server(ctx, mem_budget=f + f // 2) as srv:
            ids = [srv.enqueue(b) for _ in range(5)]
            assert all(srv.poll(i, -1)[0] == 0 for i in ids)
            assert srv.stats()["epochs"] == 5


def test_open_loop_run(phmm):
    from paper_2606_25738_gb300 import serving
    pool = serving.make_pool(8, seed=5, reads_range=(4, 32), haps_range=(2, 6), long_frac=0.2,
                             long_range=(1000, 3000))
    with phmm.Context(max_inflight=2, flags=phmm.F_NO_TUNE) as ctx:
        r = serving.run(ctx, pool, rate=40.0, duration=1.5, drain_s=60.0)
    assert r["enqueued"] == r["arrivals"] and r["completed"] == r["enqueued"]
    assert r["p50_ms"] > 0 and r["p99_ms"] >= r["p50_ms"] and r["gcups"] > 0
    assert r["by_class"]["small"]["completed"] + r["by_class"]["large"]["completed"] == r["completed"]
