"""The seeded workload generators: determinism, layout and the configured shapes."""
import numpy as np

from paper_2606_25738_gb300 import workloads as W


def _check_layout(b):
    assert b["read_off"][0] == 0 and b["hap_off"][0] == 0
    assert np.all(np.diff(b["read_off"].astype(np.int64)) >= 1)
    assert np.all(np.diff(b["hap_off"].astype(np.int64)) >= 1)
    n = int(b["read_off"][-1])
    for k in ("base_q", "ins_q", "del_q", "gcp_q", "read_bases"):
        assert len(b[k]) == n
    assert len(b["hap_bases"]) == int(b["hap_off"][-1])
    assert b["pair_read"].max() < len(b["read_off"]) - 1
    assert b["pair_hap"].max() < len(b["hap_off"]) - 1
    assert set(np.unique(b["read_bases"])) <= set(b"ACGTN")
    assert set(np.unique(b["hap_bases"])) <= set(b"ACGT")


def test_plain_pairs_shape_and_determinism():
    a = W.plain_pairs(64, seed=0)
    b = W.plain_pairs(64, seed=0)
    for k in a:
        assert np.array_equal(a[k], b[k])
    _check_layout(a)
    rl, hl = W.pair_lengths(a)
    assert rl.min() >= 100 and rl.max() <= 150 and hl.min() >= 200 and hl.max() <= 400
    assert a["base_q"].min() >= 10 and a["base_q"].max() <= 40
    assert np.all(a["ins_q"] == 45) and np.all(a["gcp_q"] == 10)


def test_short_read_regions_shape():
    b = W.short_read_regions(n_regions=20, seed=0)
    _check_layout(b)
    rl, hl = W.pair_lengths(b)
    assert np.all(rl == 150)
    assert hl.min() >= 240 and hl.max() <= 620
    assert len(b["read_off"]) - 1 == 20 * 50
    assert (b["read_bases"] == ord("N")).mean() > 0.003
    q = b["base_q"]
    assert 0.75 < np.mean(q >= 30) < 0.95 and q.min() >= 2 and q.max() <= 41


def test_long_pairs_shape():
    b = W.long_pairs(8, seed=0, k_range=(1000, 5000))
    _check_layout(b)
    rl, hl = W.pair_lengths(b)
    assert np.all(rl <= hl) and np.all(rl >= 0.89 * hl)


def test_uneven_and_equal_length():
    b = W.uneven_pairs(50, seed=0)
    _check_layout(b)
    rl, hl = W.pair_lengths(b)
    assert np.all(hl >= rl) and rl.min() >= 50 and hl.max() <= 20000
    e = W.equal_length(4, 128)
    rl, hl = W.pair_lengths(e)
    assert np.all(rl == 128) and np.all(hl == 128)
    assert W.cells(e) == 4 * 128 * 128
