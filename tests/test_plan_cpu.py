"""The work planner (host side, no GPU): phmm_plan_check builds the plan the runtime would
use and checks its invariants -- every pair scheduled exactly once, teams inside their
warp and wide enough, CTA warp ranges disjoint, strips of wide pairs tiling their columns
in work-item order with disjoint boundary buffers -- across length distributions and
every kernel choice."""
import numpy as np
import pytest

from paper_2606_25738_gb300 import workloads as W


@pytest.fixture(scope="module")
def P():
    from paper_2606_25738_gb300 import phmm
    return phmm


def _shapes():
    rng = np.random.default_rng(0)
    out = {}
    b = W.short_read_regions(60, seed=3)
    rl, hl = W.pair_lengths(b)
    out["short_regions"] = (rl, hl, b["pair_read"])
    lo, hi = np.log(50), np.log(20000)
    a = np.rint(np.exp(rng.uniform(lo, hi, 3000))).astype(np.int64)
    c = np.rint(np.exp(rng.uniform(lo, hi, 3000))).astype(np.int64)
    out["uneven"] = (np.minimum(a, c), np.maximum(a, c), np.arange(3000))
    k = np.rint(np.exp(rng.uniform(np.log(1000), np.log(200000), 200))).astype(np.int64)
    out["very_wide"] = ((k * rng.uniform(0.9, 1.0, 200)).astype(np.int64) // 10 + 1, k, np.arange(200))
    out["edges"] = (np.array([1, 1, 5, 1000, 3, 150, 150, 20000]),
                    np.array([1, 1024, 1025, 1, 16384, 16385, 65536, 131072]), np.arange(8))
    L = np.repeat([32, 512, 2048, 12288, 16384, 24577], 40)
    out["equal"] = (L, L, np.arange(len(L)))
    rr = rng.integers(0, 50, 800)
    out["shared_reads"] = (np.full(800, 150), rng.integers(100, 1500, 800), np.sort(rr))
    return out


SHAPES = _shapes()


@pytest.mark.parametrize("shape", sorted(SHAPES))
@pytest.mark.parametrize("scal,pack,kind", [(0, -1, 0), (4, -1, 1), (5, 1, 1), (7, 0, 0), (3, -1, 2), (8, 1, 2),
                                            (7, -1, 3), (5, 1, 3), (7, -1, 4), (4, 0, 4), (7, -1, 5),
                                            (5, 1, 5), (9, -1, 3), (9, 0, 1), (7, -1, 6), (5, 1, 6), (7, -1, 7),
                                            (7, -1, 8), (5, 1, 8)])
def test_fp32_plans_valid(P, shape, scal, pack, kind):
    l, k, pr = SHAPES[shape]
    rc, st = P.plan_check(l, k, pr, "fp32", scal, pack, kind)
    assert rc == P.PHMM_OK, st
    assert st["failed_check"] == 0 and st["too_long"] == 0


@pytest.mark.parametrize("shape", sorted(SHAPES))
@pytest.mark.parametrize("variant", [0, 1, 2, 3])
def test_fp64_plans_valid(P, shape, variant):
    """FP64 variants: 8 columns per lane in 16-warp CTAs, 16 in 8-warp CTAs, pipelined
    short teams of 16 (or 32) columns per lane with 8-warp CTA items."""
    l, k, pr = SHAPES[shape]
    rc, st = P.plan_check(l, k, pr, "fp64", variant)
    assert rc == P.PHMM_OK, st
    assert P.plan_check(l, k, pr, "fp64", 4)[0] == P.PHMM_EINVAL


def test_wide_pairs_are_striped_and_packed(P):
    l, k, pr = SHAPES["very_wide"]
    rc, st = P.plan_check(l, k, pr, "fp32", 4, -1, 1)
    assert rc == P.PHMM_OK
    assert st["striped_pairs"] > 0
    # strips of different pairs share CTAs: fewer items than strips in total
    rc0, st0 = P.plan_check(l, k, pr, "fp32", 4, -1, 0)
    assert rc0 == P.PHMM_OK and st0["cta_items"] <= st0["cta_pairs"]


def test_plan_check_rejects_bad_ids(P):
    l, k, pr = SHAPES["edges"]
    assert P.plan_check(l, k, pr, "fp32", 99, -1, 1)[0] == P.PHMM_EINVAL
    assert P.plan_check(l, k, pr, "fp32", 4, 7, 1)[0] == P.PHMM_EINVAL
    assert P.plan_check(l, k, pr, "fp32", 4, -1, 9)[0] == P.PHMM_EINVAL


def test_serial_plan_one_item_per_long_pair(P):
    """Long kind 3: every multi-warp pair is one item (one warp runs all its strips)."""
    l, k, pr = SHAPES["uneven"]
    rc, st = P.plan_check(l, k, pr, "fp32", 7, -1, 3)
    assert rc == P.PHMM_OK
    n_long = int(np.sum(k > 1024))
    assert st["cta_items"] == n_long and st["cta_pairs"] == n_long
    assert st["striped_pairs"] == int(np.sum(k > 1024))  # all of them span two or more strips


def test_wave_strip_widths(P):
    """The wave kinds make one work item per strip: 1024 columns per strip for kinds 6 and
    7, 512 for kind 8, so a pair of k columns has ceil(k / 1024) or ceil(k / 512) items."""
    k = np.array([1025, 4096, 20000, 131072])
    l = np.array([300, 50, 700, 150])
    pr = np.arange(len(k))
    for kind, width in ((6, 1024), (7, 1024), (8, 512)):
        rc, st = P.plan_check(l, k, pr, "fp32", 7, -1, kind)
        assert rc == P.PHMM_OK, st
        assert st["cta_items"] == int(np.sum((k + width - 1) // width)), (kind, st)
        assert st["cta_pairs"] == st["cta_items"]
