"""Writes tiny_exact.txt: exact likelihoods of tiny pairs by exhaustive path enumeration
in rational arithmetic (oracle.brute with fractions.Fraction inputs).

Each case pins Eq. 1-4 of the paper (Section 2): the values come from summing every
alignment path's weight exactly (the path model is stated in oracle/brute.py), so they
do not depend on the dynamic programme or on floating-point rounding.  Probabilities are
exact rationals; the stored log10 value is the float nearest to log10 of the exact sum.

Run from the repository root:  python tests/golden/make_golden.py
"""
import math
import os
import sys
from fractions import Fraction as F

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__)))))
from oracle.brute import brute_force_sum  # noqa: E402

CASES = [
    # read, hap, eps, tmi, tmd, gcp   (each a rational, constant over the read)
    ("A", "A", F(1, 100), F(1, 1000), F(1, 1000), F(1, 10)),
    ("A", "AC", F(1, 100), F(1, 1000), F(1, 1000), F(1, 10)),
    ("AC", "AC", F(1, 1000), F(1, 10000), F(1, 10000), F(1, 10)),
    ("AC", "CA", F(1, 100), F(1, 1000), F(1, 1000), F(1, 10)),
    ("ACG", "AG", F(1, 100), F(1, 100), F(1, 100), F(1, 10)),
    ("AG", "ACG", F(1, 100), F(1, 100), F(1, 100), F(1, 10)),
    ("NNN", "ACGT", F(1, 10), F(1, 50), F(1, 20), F(1, 5)),
    ("ACGT", "ACNT", F(1, 20), F(1, 30), F(1, 40), F(1, 10)),
    ("GATTA", "GATCA", F(1, 100), F(1, 1000), F(1, 2000), F(1, 10)),
    ("TTT", "TTTTT", F(3, 100), F(1, 100), F(1, 100), F(1, 4)),
]


def main():
    here = os.path.dirname(os.path.abspath(__file__))
    lines = ["# Exact PairHMM likelihoods of tiny pairs (Eq. 1-4, Section 2), by exhaustive",
             "# path enumeration in rational arithmetic (tests/golden/make_golden.py).",
             "# columns: read hap eps tmi tmd gcp exact_L(as p/q) log10_L"]
    for read, hap, eps, tmi, tmd, gcp in CASES:
        s = brute_force_sum(read, hap, eps, tmi, tmd, gcp)
        lg = math.log10(s.numerator) - math.log10(s.denominator)
        lines.append("%s %s %s %s %s %s %s/%s %.17g" % (read, hap, eps, tmi, tmd, gcp,
                                                       s.numerator, s.denominator, lg))
    with open(os.path.join(here, "tiny_exact.txt"), "w") as f:
        f.write("\n".join(lines) + "\n")


if __name__ == "__main__":
    main()
