"""Full-size parity for the long-read and uneven-length workloads (GPU).

* Long-read pairs (64 pairs, haplotypes log-uniform 1k-100k bp, reads 90-100% of the
  haplotype, 5% substitutions, 3% indels, quals 5-30): every pair against the oracle,
  for FP32 + FP64 rescue (<= 1e-3; rescued pairs <= 1e-9) and for the all-FP64 GPU mode
  (<= 1e-9).
* Uneven lengths (1M pairs, read and haplotype lengths log-uniform 50-20k bp): one batch
  in the launch configuration the benchmark uses (one submit, one captured graph),
  checked on pairs sampled from every decile of the per-pair cell count plus pairs the
  rescue pass recomputed.
"""
import numpy as np
import pytest

import oracle
from paper_2606_25738_gb300 import workloads as W

pytestmark = [pytest.mark.gpu, pytest.mark.slow]


@pytest.fixture(scope="module")
def phmm():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2606_25738_gb300 import phmm as P
    return P


@pytest.fixture(scope="module")
def long_batch():
    b = W.long_pairs(64, seed=0)
    return b, oracle.batch(b)


def test_long_pairs_fp32_rescue_full(phmm, long_batch):
    b, ref = long_batch
    with phmm.Context(precision="fp32") as ctx:
        out, flags, rc, st = ctx.run(b)
    assert rc == 0
    assert np.all(np.isfinite(ref)) and np.all(ref < -100)
    fp64 = (flags & phmm.PAIR_RESCUED) != 0
    d = np.abs(out - ref)
    assert np.all(d[~fp64] <= 1e-3), d[~fp64].max()
    assert np.all(d[fp64] <= 1e-9)
    assert st["n_long"] > 0


def test_long_pairs_fp64_full(phmm, long_batch):
    b, ref = long_batch
    with phmm.Context(precision="fp64") as ctx:
        out, flags, rc, st = ctx.run(b)
    assert rc == 0
    assert np.max(np.abs(out - ref)) <= 1e-9


def test_uneven_million_pairs_sampled(phmm):
    import torch

    b = W.uneven_pairs(1_000_000, seed=0)
    n = len(b["pair_read"])
    d = phmm.to_device(b)
    out = torch.empty(n, dtype=torch.float64, device="cuda")
    fl = torch.zeros(n, dtype=torch.uint8, device="cuda")
    with phmm.Context(precision="fp32", max_inflight=1) as ctx:
        t = ctx.submit(d, out, fl)
        assert ctx.poll(t, -1) == 0
    res, flags = out.cpu().numpy(), fl.cpu().numpy()
    assert np.all(np.isfinite(res))
    pick = W.stratified_sample(b, 200, max_cells=2e10)
    resc = np.flatnonzero(flags & phmm.PAIR_RESCUED)[:200]
    pick = np.unique(np.concatenate([pick, resc]))
    ref = oracle.batch(b, pairs=pick)
    fp64 = (flags[pick] & phmm.PAIR_RESCUED) != 0
    dd = np.abs(res[pick] - ref)
    assert np.all(dd <= np.where(fp64, 1e-9, 1e-3)), dd.max()


def test_short_read_batch_full_sampled(phmm):
    """The benchmark's workload at full size (2000 regions, ~455k pairs) in the benchmark's
    launch configuration: device-resident inputs, one context, the tuned plan replayed as a
    captured graph.  Pairs sampled from every decile of the cell count plus every rescued
    pair match the oracle; a second replay gives the same bits."""
    import torch

    b = W.short_read_regions(2000, seed=0)
    n = len(b["pair_read"])
    d = phmm.to_device(b)
    out = torch.empty(n, dtype=torch.float64, device="cuda")
    fl = torch.zeros(n, dtype=torch.uint8, device="cuda")
    with phmm.Context(precision="fp32", max_inflight=3) as ctx:
        for _ in range(2):  # first submit plans and tunes, the second replays the graph
            assert ctx.poll(ctx.submit(d, out, fl), -1) == 0
        res1 = out.cpu().numpy().copy()
        t = ctx.submit(d, out, fl)
        assert ctx.poll(t, -1) == 0
        st = ctx.stats(t)
    res, flags = out.cpu().numpy(), fl.cpu().numpy()
    assert np.array_equal(res, res1)
    assert st["n_pairs"] == n and np.all(np.isfinite(res))
    pick = W.stratified_sample(b, 300)
    resc = np.flatnonzero(flags & phmm.PAIR_RESCUED)[:200]
    pick = np.unique(np.concatenate([pick, resc]))
    ref = oracle.batch(b, pairs=pick)
    fp64 = (flags[pick] & phmm.PAIR_RESCUED) != 0
    dd = np.abs(res[pick] - ref)
    assert np.all(dd <= np.where(fp64, 1e-9, 1e-3)), dd.max()
