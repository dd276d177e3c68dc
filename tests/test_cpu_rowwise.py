"""The row-wise CPU path (libphmm_cpu.so, include/phmm_cpu.h: one pair per SIMD lane)
against the CPU oracle, on the CPU: edge cases, packs of mixed lengths, rescaling, the FP32
pass with its FP64 rescue (including the a-priori rounding-bound trigger), invalid inputs,
and thread-count independence."""
import numpy as np
import pytest

import oracle
from paper_2606_25738_gb300 import workloads as W

TOL32, TOL64 = 1e-3, 1e-9


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


def _check(out, fl, ref):
    """FP32 values within 1e-3, FP64 (rescued or FP64 mode) within 1e-9."""
    fp64 = (fl & 0x4) != 0
    d = np.abs(out - ref)
    assert np.all(d <= np.where(fp64, TOL64, TOL32)), (d.max(), fl)
    return d


def test_edge_cases_match_oracle(cpu):
    b = _edge_batch()
    ref = oracle.batch(b)
    out, fl = cpu.forward(b, 2, "fp64")
    assert np.all(np.isfinite(out))
    assert np.all((fl & 0xFD) == 0x4)
    assert np.max(np.abs(out - ref)) <= TOL64
    assert ref[-2] < -300  # the long read falls far below FP64's fixed-scale range
    assert fl[-2] & 0x2  # ... so it was rescaled
    for prec in ("fp32", "fp32_only"):
        out, fl = cpu.forward(b, 2, prec)
        assert np.all(np.isfinite(out))
        _check(out, fl, ref)


@pytest.mark.parametrize("maker", ["plain", "short", "long", "uneven"])
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_workloads_match_oracle(cpu, maker, prec):
    b = {"plain": lambda: W.plain_pairs(60, seed=3, k_range=(1, 3000), l_range=(1, 400), indel_rate=0.01),
         "short": lambda: W.short_read_regions(4, seed=2),
         "long": lambda: W.long_pairs(3, seed=4, k_range=(1000, 3000)),
         "uneven": lambda: W.uneven_pairs(120, seed=5, len_range=(1, 1500))}[maker]()
    out, fl = cpu.forward(b, 4, prec)
    d = _check(out, fl, oracle.batch(b))
    if prec == "fp64":
        assert d.max() <= TOL64


def test_long_read_fp32_rescaling_and_drift():
    """A 20 kbp read against its haplotype: hundreds of rescalings, stochastically rounded
    coefficients; the FP32 pass stays within the tolerance without a rescue."""
    from paper_2606_25738_gb300 import cpu as C
    b = W.long_pairs(1, seed=6, k_range=(20000, 20001))
    out, fl = C.forward(b, 1, "fp32")
    ref = oracle.batch(b)
    assert fl[0] & 0x2 and not fl[0] & 0x1
    assert abs(out[0] - ref[0]) <= TOL32


def test_rounding_bound_triggers_fp64_rescue(cpu):
    """The a-priori FP32 rounding bound grows like sqrt(16 l + 4 k): under a tolerance
    that a 300-row pair exceeds, that pair (and only pairs as long) is flagged DANGER and
    recomputed in FP64; at the default tolerance (1e-3) nothing is."""
    b = W.plain_pairs(12, seed=4, k_range=(250, 400), l_range=(2, 300))
    rl, hl = W.pair_lengths(b)
    ref = oracle.batch(b)
    out, fl = cpu.forward(b, 2, "fp32")
    assert not np.any(fl & 0x1)
    bound = (6.5 * np.sqrt(16.0 * rl + 4.0 * hl) * 2.0 ** -23 + 8.0 * rl * 2.0 ** -46) / np.log(10.0)
    tol = float(np.median(bound))
    out, fl = cpu.forward(b, 2, "fp32", tolerance=tol)
    over = bound > tol
    assert over.any() and (~over).any()
    assert np.array_equal((fl & 0x1) != 0, over)
    assert np.all(fl[over] & 0x8) and np.all(fl[over] & 0x4)
    assert np.max(np.abs(out[over] - ref[over])) <= TOL64
    assert np.max(np.abs(out[~over] - ref[~over])) <= TOL32
    out2, fl2 = cpu.forward(b, 2, "fp32_only", tolerance=tol)
    assert np.array_equal((fl2 & 0x8) != 0, over) and not np.any(fl2 & 0x5)


def test_thread_count_does_not_change_bits(cpu):
    b = W.plain_pairs(40, seed=9, k_range=(1, 2000), l_range=(1, 300))
    for prec in ("fp32", "fp64"):
        o1, f1 = cpu.forward(b, 1, prec)
        o4, f4 = cpu.forward(b, 4, prec)
        assert np.array_equal(o1, o4) and np.array_equal(f1, f4)


def test_invalid_pairs_are_marked(cpu):
    b = W.from_strings([("ACGT", "ACGT", 30, 45, 45, 10), ("AXGT", "ACGT", 30, 45, 45, 10),
                        ("ACGT", "ACGT", 30, 45, 45, 10)])
    b["base_q"] = b["base_q"].copy()
    b["base_q"][int(b["read_off"][2])] = 94  # quality above 93 in the third pair's read
    for prec in ("fp64", "fp32"):
        out, fl = cpu.forward(b, 1, prec)
        assert np.isfinite(out[0]) and np.isnan(out[1]) and np.isnan(out[2])
        assert fl[1] == 0x80 and fl[2] == 0x80
        assert fl[0] == (0x4 if prec == "fp64" else 0x0)


def test_malformed_batch_is_rejected(cpu):
    from paper_2606_25738_gb300 import phmm
    b = W.plain_pairs(4, seed=1)
    b["pair_read"] = b["pair_read"].copy()
    b["pair_read"][0] = 10_000
    with pytest.raises(phmm.PhmmError) as e:
        cpu.forward(b, 1)
    assert e.value.status == phmm.PHMM_EINVAL
    with pytest.raises(phmm.PhmmError) as e:
        cpu.forward(W.plain_pairs(4, seed=1), 1, tolerance=-1.0)
    assert e.value.status == phmm.PHMM_EINVAL


def test_empty_batch(cpu):
    b = W.subset(W.plain_pairs(3, seed=1), [])
    out, fl = cpu.forward(b, 2)
    assert len(out) == 0 and len(fl) == 0


def test_degenerate_gap_row_goes_to_fp64(cpu):
    """FP32 takes T_IM = 1 - g out of the match update; a row with gap-continuation Phred 0
    (1 - g = 0) cannot be factored, so its pair is flagged DEGENERATE and recomputed in
    FP64 (to 1e-9), while the FP32-only pass leaves it flagged.  Pairs without such a row
    stay in FP32."""
    rng = np.random.default_rng(21)
    hap = "".join(rng.choice(list("ACGT"), size=600))
    read = hap[100:250]
    one_zero = np.full(len(read), 10)
    one_zero[70] = 0
    pairs = [(read, hap, 30, 45, 45, 10), (read, hap, 30, 45, 45, one_zero), (read, hap, 30, 45, 45, 1)]
    b = W.from_strings(pairs)
    ref = oracle.batch(b)
    assert np.all(np.isfinite(ref))
    out, fl = cpu.forward(b, 1, "fp32")
    assert fl[1] & 0x40 and fl[1] & 0x1 and fl[1] & 0x4
    assert not (fl[0] & 0x41) and not (fl[2] & 0x41)
    _check(out, fl, ref)
    out2, fl2 = cpu.forward(b, 1, "fp32_only")
    assert fl2[1] & 0x40 and not (fl2[1] & 0x5)
    assert np.max(np.abs(out2[[0, 2]] - ref[[0, 2]])) <= TOL32
