"""The row-wise CPU path (libphmm_cpu.so, include/phmm_cpu.h) against the CPU oracle, on
the CPU: edge cases of the blocked deletion chain and of the rescaling, invalid inputs,
and thread-count independence."""
import numpy as np
import pytest

import oracle
from paper_2606_25738_gb300 import workloads as W

TOL64 = 1e-9


@pytest.fixture(scope="module")
def cpu():
    from paper_2606_25738_gb300 import build
    build.build_cpu()
    from paper_2606_25738_gb300 import cpu as C
    return C


def _edge_batch():
    rng = np.random.default_rng(5)
    rs = lambda n: "".join(rng.choice(list("ACGT"), size=n))
    hap = rs(2100)
    pairs = [
        ("A", "A", 30, 45, 45, 10),                       # l = k = 1
        ("C", "ACGTA", 30, 45, 45, 10),                   # l = 1
        (rs(40), "G", 20, 45, 45, 10),                    # k = 1
        (rs(30), rs(31), 30, 45, 45, 10),                 # k < 32: plain deletion chain
        (rs(30), rs(32), 30, 45, 45, 10),                 # k = 32: first blocked row
        (rs(50), rs(33), 30, 45, 45, 10),                 # blocks with padding
        (hap[:100] + hap[150:250], hap[:400], 30, 45, 45, 10),   # 50 bp deletion
        (hap[:60] + rs(40) + hap[60:150], hap[:300], 30, 45, 45, 10),  # 40 bp insertion
        ("N" * 50, hap[:120], 30, 45, 45, 10),            # all-N read
        (hap[10:90], hap[:200].replace("A", "N"), 0, 45, 45, 10),  # N in the haplotype, Phred 0
        (hap[10:90], hap[:300], 93, 45, 45, 10),          # Phred 93
        (hap[5:60], hap[:300], 30, 10, 10, 10),           # frequent gaps
        (hap[:150], hap[:600], 25, 40, 40, np.arange(150) % 20 + 5),  # per-row gcp
        (rs(2000), hap, np.arange(2000) % 31 + 5, 45, 45, 10),  # 2000 unrelated rows: rescaling
        (hap[:150].lower(), hap[:500].lower(), 30, 45, 45, 10),  # lower case
    ]
    return W.from_strings(pairs)


def test_edge_cases_match_oracle(cpu):
    b = _edge_batch()
    out, fl = cpu.forward(b, 2)
    ref = oracle.batch(b)
    assert np.all(np.isfinite(out))
    assert np.all(fl == 0x4)
    assert np.max(np.abs(out - ref)) <= TOL64
    assert ref[-2] < -300  # the long read falls far below FP64's fixed-scale range


@pytest.mark.parametrize("maker", ["plain", "short", "long"])
def test_workloads_match_oracle(cpu, maker):
    b = {"plain": lambda: W.plain_pairs(60, seed=3, k_range=(1, 3000), l_range=(1, 400), indel_rate=0.01),
         "short": lambda: W.short_read_regions(4, seed=2),
         "long": lambda: W.long_pairs(3, seed=4, k_range=(1000, 3000))}[maker]()
    out, fl = cpu.forward(b, 4)
    assert np.max(np.abs(out - oracle.batch(b))) <= TOL64


def test_thread_count_does_not_change_bits(cpu):
    b = W.plain_pairs(40, seed=9, k_range=(1, 2000), l_range=(1, 300))
    o1, _ = cpu.forward(b, 1)
    o4, _ = cpu.forward(b, 4)
    assert np.array_equal(o1, o4)


def test_invalid_pairs_are_marked(cpu):
    b = W.from_strings([("ACGT", "ACGT", 30, 45, 45, 10), ("AXGT", "ACGT", 30, 45, 45, 10),
                        ("ACGT", "ACGT", 30, 45, 45, 10)])
    b["base_q"] = b["base_q"].copy()
    b["base_q"][int(b["read_off"][2])] = 94  # quality above 93 in the third pair's read
    out, fl = cpu.forward(b, 1)
    assert np.isfinite(out[0]) and np.isnan(out[1]) and np.isnan(out[2])
    assert fl[0] == 0x4 and fl[1] == 0x80 and fl[2] == 0x80


def test_malformed_batch_is_rejected(cpu):
    from paper_2606_25738_gb300 import phmm
    b = W.plain_pairs(4, seed=1)
    b["pair_read"] = b["pair_read"].copy()
    b["pair_read"][0] = 10_000
    with pytest.raises(phmm.PhmmError) as e:
        cpu.forward(b, 1)
    assert e.value.status == phmm.PHMM_EINVAL


def test_empty_batch(cpu):
    b = W.subset(W.plain_pairs(3, seed=1), [])
    out, fl = cpu.forward(b, 2)
    assert len(out) == 0 and len(fl) == 0
