"""Pins for the CPU oracle (no GPU).

Every test here checks the oracle against something other than itself: exact rational
path sums, brute-force enumeration, closed forms, invariants, the paper's row-wise
reformulation (Eq. 7) evaluated literally, and a long-double build.  Each is chosen so
that a plausible slip in the oracle (a dropped term, a wrong row index, a transposed
transition, a wrong mismatch factor) fails at least one of them; test_oracle_mutants
demonstrates that by planting such slips.
"""
import math
import os
from fractions import Fraction

import numpy as np
import pytest

from oracle.brute import brute_force_loglik, brute_force_sum

HERE = os.path.dirname(os.path.abspath(__file__))


def _rand_case(rng, lmax, kmax, per_row=True, n_rate=0.1):
    l = int(rng.integers(1, lmax + 1))
    k = int(rng.integers(1, kmax + 1))
    alphabet = "ACGTN"
    p = [0.225, 0.225, 0.225, 0.225, 0.1] if n_rate else [0.25] * 4 + [0.0]
    read = "".join(rng.choice(list(alphabet), size=l, p=p))
    hap = "".join(rng.choice(list(alphabet), size=k, p=p))
    size = l if per_row else 1
    eps = rng.uniform(1e-4, 0.3, size)
    tmi = rng.uniform(1e-5, 0.1, size)
    tmd = rng.uniform(1e-5, 0.1, size)
    gcp = rng.uniform(0.01, 0.5, size)
    if not per_row:
        eps, tmi, tmd, gcp = (np.full(l, v[0]) for v in (eps, tmi, tmd, gcp))
    return read, hap, eps, tmi, tmd, gcp


# ---------------------------------------------------------------------------------------
# Exact values (rational arithmetic) and brute force
# ---------------------------------------------------------------------------------------

def test_golden_exact_rationals(oracle_mod):
    """Stored exact likelihoods (tests/golden/tiny_exact.txt, exhaustive path sums in
    rational arithmetic, Eq. 1-4) against the FP64 and long-double oracle."""
    rows = [ln.split() for ln in open(os.path.join(HERE, "golden", "tiny_exact.txt"))
            if ln.strip() and not ln.startswith("#")]
    assert len(rows) >= 10
    for read, hap, eps, tmi, tmd, gcp, frac, lg in rows:
        e, i, d, g = (float(Fraction(x)) for x in (eps, tmi, tmd, gcp))
        exact = Fraction(frac)
        want = math.log10(exact.numerator) - math.log10(exact.denominator)
        assert abs(float(lg) - want) < 1e-15
        for prec in ("double", "long"):
            got = oracle_mod.loglik_probs(read, hap, e, i, d, g, precision=prec)
            assert abs(got - want) < 1e-13, (read, hap, prec, got, want)


def test_golden_hand_values():
    """Two values derived by hand from Eq. 1-4: a single-base read against a one- and
    a two-base haplotype (T_DM = 1 - gcp = 0.9, e = 0.01)."""
    rows = {(r[0], r[1]): Fraction(r[6]) for r in
            (ln.split() for ln in open(os.path.join(HERE, "golden", "tiny_exact.txt"))
             if ln.strip() and not ln.startswith("#"))}
    assert rows[("A", "A")] == Fraction(9, 10) * Fraction(99, 100)
    assert rows[("A", "AC")] == Fraction(9, 10) / 2 * (Fraction(99, 100) + Fraction(1, 300))


@pytest.mark.parametrize("seed", range(40))
def test_brute_force_random(oracle_mod, seed):
    """Oracle (DP over Eq. 2) == explicit enumeration of every alignment path, on random
    reads/haplotypes of up to 6 bases with per-row probabilities and N bases."""
    rng = np.random.default_rng(seed)
    read, hap, eps, tmi, tmd, gcp = _rand_case(rng, 6, 6, per_row=bool(seed % 2))
    want = brute_force_loglik(read, hap, eps, tmi, tmd, gcp)
    got = oracle_mod.loglik_probs(read, hap, eps, tmi, tmd, gcp)
    assert abs(got - want) <= 1e-12 * max(1.0, abs(want)), (read, hap, got, want)


def test_brute_force_exact_fraction_random(oracle_mod):
    """Same, with exact rational path sums as the reference (no rounding on that side)."""
    rng = np.random.default_rng(123)
    for _ in range(8):
        l, k = int(rng.integers(1, 5)), int(rng.integers(1, 6))
        read = "".join(rng.choice(list("ACGT"), size=l))
        hap = "".join(rng.choice(list("ACGT"), size=k))
        fr = lambda lo, hi: [Fraction(int(x), 1000) for x in rng.integers(lo, hi, size=l)]
        eps, tmi, tmd, gcp = fr(1, 300), fr(1, 50), fr(1, 50), fr(10, 400)
        s = brute_force_sum(read, hap, eps, tmi, tmd, gcp)
        want = math.log10(s.numerator) - math.log10(s.denominator)
        got = oracle_mod.loglik_probs(read, hap, [float(x) for x in eps], [float(x) for x in tmi],
                                      [float(x) for x in tmd], [float(x) for x in gcp])
        assert abs(got - want) < 1e-13


# ---------------------------------------------------------------------------------------
# Closed forms
# ---------------------------------------------------------------------------------------

@pytest.mark.parametrize("k", [1, 2, 7, 64, 333])
def test_closed_form_single_row(oracle_mod, k):
    """l = 1: L = (1 - gcp_1)/k * sum_j P(r_1 | h_j)  (Eq. 1 row 0 of D, Eq. 2-4)."""
    rng = np.random.default_rng(k)
    hap = "".join(rng.choice(list("ACGTN"), size=k))
    for base in "ACGTN":
        e, g = 0.02, 0.1
        n_match = sum(1 for h in hap if h == base or h == "N" or base == "N")
        want = math.log10((1 - g) / k * (n_match * (1 - e) + (k - n_match) * e / 3))
        got = oracle_mod.loglik_probs(base, hap, e, 1e-3, 2e-3, g)
        assert abs(got - want) < 1e-14


@pytest.mark.parametrize("seed", range(6))
def test_closed_form_no_gaps(oracle_mod, seed):
    """T_MI = T_MD = 0: only M->M paths survive, so
    L = (1 - gcp_1)/k * sum_{s=1}^{k-l+1} prod_i P(r_i | h_{s+i-1})."""
    rng = np.random.default_rng(seed)
    l = int(rng.integers(1, 30))
    k = int(rng.integers(l, 60))
    read = rng.choice(list("ACGT"), size=l)
    hap = rng.choice(list("ACGT"), size=k)
    eps = rng.uniform(1e-3, 0.2, l)
    g = rng.uniform(0.05, 0.3, l)
    total = 0.0
    for s in range(k - l + 1):
        prod = 1.0
        for i in range(l):
            prod *= (1 - eps[i]) if read[i] == hap[s + i] else eps[i] / 3
        total += prod
    want = math.log10((1 - g[0]) / k * total)
    got = oracle_mod.loglik_probs("".join(read), "".join(hap), eps, 0.0, 0.0, g)
    assert abs(got - want) < 1e-12


def test_closed_form_identical(oracle_mod):
    """Read identical to the haplotype, l = k, no gaps: L = (1-gcp_1)/k * prod(1 - e_i)."""
    rng = np.random.default_rng(7)
    for l in (1, 5, 150, 1000):
        s = "".join(rng.choice(list("ACGT"), size=l))
        eps = rng.uniform(1e-4, 1e-2, l)
        want = math.log10(0.9 / l) + float(np.sum(np.log10(1 - eps)))
        got = oracle_mod.loglik_probs(s, s, eps, 0.0, 0.0, 0.1)
        assert abs(got - want) < 1e-11


def test_closed_form_identical_phred_gaps(oracle_mod):
    """With gap-open quals of 93 (T_MI = T_MD = 10^-9.3) the identical-read value moves
    by at most ~l*k*1e-9 relative from the no-gap closed form."""
    s = "ACGTTGCA" * 10
    q = np.full(len(s), 30, np.uint8)
    got = oracle_mod.loglik_phred(s, s, q, 93, 93, 10)
    e = 10 ** -3.0
    want = math.log10(0.9 / len(s)) + len(s) * math.log10(1 - e) + len(s) * math.log10(1 - 2 * 10 ** -9.3)
    assert abs(got - want) < len(s) ** 2 * 1e-9


# ---------------------------------------------------------------------------------------
# Invariants
# ---------------------------------------------------------------------------------------

@pytest.mark.parametrize("seed", range(10))
def test_probability_bounds(oracle_mod, seed):
    """0 < L <= 1 when ins/del quals are constant along the read (then every state's
    outgoing mass is at most 1 and the four emissions of a row sum to 1)."""
    rng = np.random.default_rng(seed)
    l, k = int(rng.integers(1, 80)), int(rng.integers(1, 120))
    read = "".join(rng.choice(list("ACGT"), size=l))
    hap = "".join(rng.choice(list("ACGT"), size=k))
    bq = rng.integers(2, 41, l).astype(np.uint8)
    v = oracle_mod.loglik_phred(read, hap, bq, 45, 40, 10)
    assert -math.inf < v <= 1e-15


def test_mismatch_monotone(oracle_mod):
    """Changing a read base to one that occurs nowhere in the haplotype never increases L,
    and strictly decreases it when e < 3/4 (Phred >= 2).  In FP64 the decrease can fall
    below one ulp when every path matching that base is negligible, so strictness is
    required in most cases rather than all."""
    rng = np.random.default_rng(11)
    strict = 0
    for _ in range(30):
        l, k = int(rng.integers(2, 40)), int(rng.integers(2, 60))
        hap = "".join(rng.choice(list("ACG"), size=k))  # 'T' absent
        read = list(rng.choice(list("ACG"), size=l))
        bq = rng.integers(2, 41, l).astype(np.uint8)
        a = oracle_mod.loglik_phred("".join(read), hap, bq, 45, 45, 10)
        pos = int(rng.integers(0, l))
        read[pos] = "T"
        b = oracle_mod.loglik_phred("".join(read), hap, bq, 45, 45, 10)
        assert b <= a
        strict += b < a
    assert strict >= 24


def test_first_row_symmetry(oracle_mod):
    """Eq. 1: every start column is equally likely (D[0][j] = C/k for all j including
    j = 0), so a one-base read scores the same against any rotation of the haplotype."""
    hap = "ACGTTGACCA"
    vals = {oracle_mod.loglik_probs("G", hap[r:] + hap[:r], 0.01, 0.001, 0.001, 0.1)
            for r in range(len(hap))}
    assert max(vals) - min(vals) < 1e-15


# ---------------------------------------------------------------------------------------
# Reformulation, rescaling and precision
# ---------------------------------------------------------------------------------------

@pytest.mark.parametrize("seed", range(12))
def test_rowwise_eq7_equals_cellwise(oracle_mod, seed):
    """The paper's row-wise form (Section 3.1, Eq. 7: D eliminated, D[i-1][j-1] as an
    explicit sum over row i-1) equals cell-by-cell Eq. 2 to 1e-12 relative."""
    rng = np.random.default_rng(100 + seed)
    read, hap, eps, tmi, tmd, gcp = _rand_case(rng, 40, 70, per_row=bool(seed % 2))
    a = oracle_mod.loglik_probs(read, hap, eps, tmi, tmd, gcp, log2C=60, rescale=0)
    b = oracle_mod.rowwise_eq7(read, hap, eps, tmi, tmd, gcp, log2C=60)
    assert abs(a - b) <= 1e-12 * max(1.0, abs(a))


@pytest.mark.parametrize("seed", range(6))
def test_rescaling_exact(oracle_mod, seed):
    """Power-of-two row rescaling after every row gives exactly the unrescaled sum
    (S_rescaled * 2^E == S_plain bit for bit) where nothing underflows."""
    rng = np.random.default_rng(200 + seed)
    l, k = int(rng.integers(5, 60)), int(rng.integers(5, 90))
    read = "".join(rng.choice(list("ACGT"), size=l))
    hap = "".join(rng.choice(list("ACGT"), size=k))
    eps = rng.uniform(1e-3, 0.05, l)
    _, s0, e0 = oracle_mod.forward_raw(read, hap, eps, 1e-3, 1e-3, 0.1, log2C=300, rescale=0)
    _, s1, e1 = oracle_mod.forward_raw(read, hap, eps, 1e-3, 1e-3, 0.1, log2C=300, rescale=2)
    assert e0 == 0 and e1 != 0
    assert math.ldexp(s1, e1) == s0


def test_rescaling_long_read_finite(oracle_mod):
    """A 3000-base read whose likelihood is far below the FP64 range (log10 L < -1000)
    stays finite with rescaling and matches the long-double oracle."""
    rng = np.random.default_rng(5)
    l = 3000
    hap = rng.choice(list("ACGT"), size=l)
    read = hap.copy()
    sub = rng.random(l) < 0.3
    read[sub] = rng.choice(list("ACGT"), size=int(sub.sum()))
    bq = np.full(l, 30, np.uint8)
    a = oracle_mod.loglik_phred("".join(read), "".join(hap), bq, 45, 45, 10)
    b = oracle_mod.loglik_phred("".join(read), "".join(hap), bq, 45, 45, 10, precision="long")
    assert a < -1000 and math.isfinite(a)
    assert abs(a - b) < 1e-9
    c = oracle_mod.loglik_phred("".join(read), "".join(hap), bq, 45, 45, 10, rescale=0)
    assert c == -math.inf  # without rescaling FP64 underflows


def test_double_vs_long_double(oracle_mod):
    """FP64 oracle within 1e-11 (log10) of the long-double build on short-read shapes:
    bounds the oracle's own rounding far below the 1e-9 FP64 parity tolerance."""
    from paper_2606_25738_gb300 import workloads as W
    b = W.plain_pairs(16, seed=3)
    d = oracle_mod.batch(b, precision="double")
    ld = oracle_mod.batch(b, precision="long")
    assert np.all(np.isfinite(d))
    assert np.max(np.abs(d - ld)) < 1e-11


def test_batch_matches_single(oracle_mod):
    """The threaded batch entry gives the single-pair result for every pair."""
    from paper_2606_25738_gb300 import workloads as W
    b = W.plain_pairs(8, seed=1)
    out = oracle_mod.batch(b, n_threads=3)
    for p in range(8):
        r0, r1 = b["read_off"][p], b["read_off"][p + 1]
        h0, h1 = b["hap_off"][p], b["hap_off"][p + 1]
        v = oracle_mod.loglik_phred(b["read_bases"][r0:r1], b["hap_bases"][h0:h1],
                                    b["base_q"][r0:r1], b["ins_q"][r0:r1],
                                    b["del_q"][r0:r1], b["gcp_q"][r0:r1])
        assert v == out[p]


def test_invalid_inputs(oracle_mod):
    """Bad bases, qualities above 93 and empty sequences are rejected."""
    with pytest.raises(ValueError):
        oracle_mod.loglik_probs("AXG", "ACG", 0.01, 0.001, 0.001, 0.1)
    with pytest.raises(ValueError):
        oracle_mod.loglik_probs("", "ACG", 0.01, 0.001, 0.001, 0.1)
    with pytest.raises(ValueError):
        oracle_mod.loglik_phred("ACG", "ACG", 94, 45, 45, 10)
    from paper_2606_25738_gb300 import workloads as W
    b = W.from_strings([("ACG", "ACG", 30, 45, 45, 10), ("AZG", "ACG", 30, 45, 45, 10)])
    out = oracle_mod.batch(b)
    assert math.isfinite(out[0]) and math.isnan(out[1])


def test_phred_table(oracle_mod):
    """q(x) = 10^(-x/10): q(10) = 0.1 (the paper's T_DD = T_II), q(0) = 1, q(30) = 1e-3."""
    assert oracle_mod.q_phred(10) == 0.1
    assert oracle_mod.q_phred(0) == 1.0
    assert abs(oracle_mod.q_phred(30) - 1e-3) < 1e-18
