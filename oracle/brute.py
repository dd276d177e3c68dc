"""Brute-force PairHMM likelihood by explicit enumeration of every alignment path.

TEST INFRASTRUCTURE ONLY.  This is a second, independent statement of what Eq. 1-4
(Section 2 of the paper) compute: instead of a dynamic programme it walks every state
path of the pair HMM one by one and adds up the path weights.  Exponential in l and k;
meant for reads and haplotypes of at most 6 bases.

Path model (read rows i = 1..l, haplotype columns j = 1..k), read off Eq. 1 and Eq. 2:
  * start in M(1, s), s = 1..k, with weight (1/k) * T_DM_1 * P(r_1 | h_s)
    (Eq. 1: row 0 of D holds C/k in every column; the C cancels in L);
  * M(i,j) -> M(i+1,j+1): T_MM_{i+1} * P(r_{i+1} | h_{j+1})
    I(i,j) -> M(i+1,j+1): T_IM_{i+1} * P(...);   D(i,j) -> M(i+1,j+1): T_DM_{i+1} * P(...)
  * M(i,j) -> I(i+1,j): T_MI_{i+1};              I(i,j) -> I(i+1,j): T_II_{i+1}
  * M(i,j) -> D(i,j+1): T_MD_i;                  D(i,j) -> D(i,j+1): T_DD_i
  * a path ends in M(l, j) or I(l, j) for any j (Eq. 4 sums the last row of M and I).
Coefficients of row i use row i's probabilities; T_IM = T_DM = 1 - g, T_II = T_DD = g.
'N' on either side is a match.
"""
from __future__ import annotations

import math


def _match(a: str, b: str) -> bool:
    a, b = a.upper(), b.upper()
    return a == "N" or b == "N" or a == b


def brute_force_sum(read: str, hap: str, eps, tmi, tmd, gcp, tmm=None):
    """L = sum of the weights of all paths (see module docstring), in the arithmetic of
    the inputs: floats give a float, fractions.Fraction gives the exact rational."""
    l, k = len(read), len(hap)
    eps, tmi, tmd, gcp = (list(v) if hasattr(v, "__len__") else [v] * l for v in (eps, tmi, tmd, gcp))
    if tmm is None:
        tmm = [1 - tmi[i] - tmd[i] for i in range(l)]
    elif not hasattr(tmm, "__len__"):
        tmm = [tmm] * l

    def emit(i: int, j: int) -> float:  # 1-based row i, column j
        e = eps[i - 1]
        return (1 - e) if _match(read[i - 1], hap[j - 1]) else e / 3

    total = 0 * eps[0]
    count = 0

    # Depth-first walk; state = (kind, i, j), w = weight of the path so far.
    def walk(kind: str, i: int, j: int, w: float) -> None:
        nonlocal total, count
        if w == 0:
            return
        if i == l and kind in ("M", "I"):
            total += w
            count += 1
        g_next = gcp[i] if i < l else None  # row i+1 coefficients (0-based index i)
        if kind == "M":
            if i < l and j < k:
                walk("M", i + 1, j + 1, w * tmm[i] * emit(i + 1, j + 1))
            if i < l:
                walk("I", i + 1, j, w * tmi[i])
            if j < k:
                walk("D", i, j + 1, w * tmd[i - 1])
        elif kind == "I":
            if i < l and j < k:
                walk("M", i + 1, j + 1, w * (1 - g_next) * emit(i + 1, j + 1))
            if i < l:
                walk("I", i + 1, j, w * g_next)
        else:  # D
            if i < l and j < k:
                walk("M", i + 1, j + 1, w * (1 - g_next) * emit(i + 1, j + 1))
            if j < k:
                walk("D", i, j + 1, w * gcp[i - 1])

    for s in range(1, k + 1):
        walk("M", 1, s, (1 - gcp[0]) * emit(1, s) / k)
    brute_force_sum.last_path_count = count
    return total


def brute_force_loglik(read: str, hap: str, eps, tmi, tmd, gcp, tmm=None) -> float:
    """log10 L by summing the weights of all paths (see module docstring)."""
    total = brute_force_sum(read, hap, eps, tmi, tmd, gcp, tmm)
    if total <= 0:
        return -math.inf
    if hasattr(total, "numerator"):
        return math.log10(total.numerator) - math.log10(total.denominator)
    return math.log10(total)
