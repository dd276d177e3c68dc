"""Plants plausible slips in a copy of the oracle source (on the CPU) and checks that
the pins of test_oracle.py catch every one: exact rational path sums, brute force and
closed forms.  The committed oracle is never modified."""
import ctypes
import math
import os
import subprocess
import tempfile
from fractions import Fraction

import numpy as np
import pytest

from oracle.brute import brute_force_loglik

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "phmm_oracle.c")
GOLD = os.path.join(ROOT, "tests", "golden", "tiny_exact.txt")

MUTANTS = {
    "drop_D_term": ("+ t_gm * Dp[j - 1]);", ");"),
    "mismatch_0.33": ("real pm = (real)1 - e, px = e / (real)3;", "real pm = (real)1 - e, px = e * (real)0.33;"),
    "insert_uses_diagonal": ("Ic[j] = t_mi * Mp[j] + g * Ip[j];", "Ic[j] = t_mi * Mp[j - 1] + g * Ip[j];"),
    "D00_zero": ("Dp[j] = C / (real)k;", "Dp[j] = j ? C / (real)k : 0;"),
    "swap_MI_MD": ("t_mi = tmi[i - 1], t_md = tmd[i - 1];", "t_mi = tmd[i - 1], t_md = tmi[i - 1];"),
    "sum_includes_D": ("S += Mp[j] + Ip[j];\n        if (S > 0)", "S += Mp[j] + Ip[j] + Dp[j];\n        if (S > 0)"),
    "N_is_mismatch": ("return rc == 4 || hc == 4 || rc == hc;", "return rc == hc;"),
    "gap_from_prev_row": ("real g = gcp[i - 1], t_gm", "real g = gcp[i > 1 ? i - 2 : 0], t_gm"),
    "match_sign": ("real pm = (real)1 - e,", "real pm = (real)1 + e,"),
    "D_uses_prev_row_M": ("Dc[j] = t_md * Mc[j - 1] + g * Dc[j - 1];", "Dc[j] = t_md * Mp[j - 1] + g * Dc[j - 1];"),
}


def _build_mutant(name, tmp):
    src = open(SRC).read()
    old, new = MUTANTS[name]
    assert src.count(old) == 1, name
    path_c = os.path.join(tmp, name + ".c")
    path_so = os.path.join(tmp, name + ".so")
    open(path_c, "w").write(src.replace(old, new))
    subprocess.check_call(["gcc", "-O1", "-fPIC", "-shared", "-ffp-contract=off", path_c, "-o",
                           path_so, "-lm", "-lpthread"])
    lib = ctypes.CDLL(path_so)
    f = lib.orc_loglik_probs
    u8 = ctypes.POINTER(ctypes.c_uint8)
    f64 = ctypes.POINTER(ctypes.c_double)
    f.restype = ctypes.c_double
    f.argtypes = [ctypes.c_int, u8, f64, f64, f64, f64, f64, ctypes.c_int, u8, ctypes.c_double,
                  ctypes.c_int, ctypes.POINTER(ctypes.c_int)]

    def call(read, hap, eps, tmi, tmd, gcp):
        l = len(read)
        r = np.frombuffer(read.encode(), np.uint8).copy()
        h = np.frombuffer(hap.encode(), np.uint8).copy()
        arr = [np.ascontiguousarray(np.broadcast_to(np.asarray(v, np.float64), (l,))) for v in (eps, tmi, tmd, gcp)]
        tmm = 1.0 - arr[1] - arr[2]
        st = ctypes.c_int()
        return f(l, r.ctypes.data_as(u8), *(a.ctypes.data_as(f64) for a in arr), tmm.ctypes.data_as(f64),
                 len(h), h.ctypes.data_as(u8), 1020.0, 1, ctypes.byref(st))
    return call


def _pins_pass(call):
    """True when the mutant passes all of: golden exact values, 20 brute-force cases,
    the single-row and no-gap closed forms."""
    for ln in open(GOLD):
        if not ln.strip() or ln.startswith("#"):
            continue
        read, hap, eps, tmi, tmd, gcp, frac, lg = ln.split()
        v = call(read, hap, *(float(Fraction(x)) for x in (eps, tmi, tmd, gcp)))
        if not abs(v - float(lg)) < 1e-12:
            return False
    rng = np.random.default_rng(0)
    for _ in range(20):
        l, k = int(rng.integers(1, 6)), int(rng.integers(1, 6))
        read = "".join(rng.choice(list("ACGTN"), size=l))
        hap = "".join(rng.choice(list("ACGTN"), size=k))
        eps, tmi, tmd, gcp = rng.uniform(1e-3, 0.2, l), rng.uniform(1e-4, 0.05, l), rng.uniform(1e-4, 0.05, l), rng.uniform(0.05, 0.4, l)
        if not abs(call(read, hap, eps, tmi, tmd, gcp) - brute_force_loglik(read, hap, eps, tmi, tmd, gcp)) < 1e-12:
            return False
    hap = "ACGTNACGGT"
    n_match = sum(1 for h in hap if h in "GN")
    if not abs(call("G", hap, 0.02, 1e-3, 1e-3, 0.1) - math.log10(0.9 / 10 * (n_match * 0.98 + (10 - n_match) * 0.02 / 3))) < 1e-13:
        return False
    return True


def test_unmutated_copy_passes():
    with tempfile.TemporaryDirectory() as tmp:
        src = open(SRC).read()
        p = os.path.join(tmp, "orig.c")
        open(p, "w").write(src)
        MUTANTS["_identity"] = ("static int base_code", "static int base_code")
        try:
            assert _pins_pass(_build_mutant("_identity", tmp))
        finally:
            del MUTANTS["_identity"]


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_mutant_caught(name):
    with tempfile.TemporaryDirectory() as tmp:
        assert not _pins_pass(_build_mutant(name, tmp)), name
