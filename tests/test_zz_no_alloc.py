"""phmm_forward_noalloc: the FP32 forward pass for callers that cannot allocate device
memory at call time (a host framework that owns the device heap and forbids allocation on
its threads, a process that reserved all device memory up front).  Its scratch lives in
fixed arrays inside the library.

Checked through the C ABI against the CPU oracle (FP32 tolerance) and against the regular
entry point (phmm_submit_batch: same values within the tolerance, same rescue-reason
flags), on two calls in a row: the scratch keeps the previous call's contents, so the
second call must not depend on them.  Also covered: a flagged pair that still returns
PHMM_OK, the scratch-full error (PHMM_ENOMEM), and offsets that must be rejected before
any access through them.  This file is collected last.
"""
import numpy as np
import pytest

import oracle
from paper_2606_25738_gb300 import workloads as W

pytestmark = pytest.mark.gpu

TOL32 = 1e-3
REASONS = 0x78  # DANGER | NONFINITE | SMALL_SUM | DEGENERATE: why the FP64 pass would run
MAX_BASES = 1 << 20  # read bases the allocation-free scratch holds


@pytest.fixture(scope="module")
def phmm():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2606_25738_gb300 import phmm as P
    return P


def _regular(phmm, b):
    """The regular entry point on the same engine family (lean scalar teams, 32 columns
    per lane), FP32 with the FP64 rescue pass."""
    with phmm.Context(precision="fp32", variant="lean", cols_per_lane=32) as ctx:
        out, flags, rc, st = ctx.run(b)
    return out, flags


def _noalloc(phmm, d, n):
    import torch
    out = torch.full((n,), -7.0, dtype=torch.float64, device="cuda")
    fl = torch.full((n,), 0xFF, dtype=torch.uint8, device="cuda")
    rc = phmm.forward_noalloc(d, out, fl)
    return rc, out.cpu().numpy(), fl.cpu().numpy()


def test_noalloc_matches_oracle_and_regular_twice(phmm):
    batches = [W.plain_pairs(64, seed=0), W.plain_pairs(40, seed=9, k_range=(1, 1024), l_range=(1, 300))]
    for b in batches:
        ref = oracle.batch(b)
        reg, reg_flags = _regular(phmm, b)
        d = phmm.to_device(b)
        n = len(b["pair_read"])
        for _call in range(2):
            rc, o, f = _noalloc(phmm, d, n)
            assert rc == phmm.PHMM_OK, rc
            assert np.all(np.isfinite(o))
            assert np.max(np.abs(o - ref)) <= TOL32
            assert np.max(np.abs(o - reg)) <= TOL32
            assert np.array_equal(f & REASONS, reg_flags & REASONS)
            assert not np.any(f & (phmm.PAIR_ERROR | phmm.PAIR_RESCUED | phmm.PAIR_FP64))


def test_noalloc_flags_degenerate_pair_and_returns_ok(phmm):
    """A pair with gap-continuation Phred 0 (T_DD = 1) cannot use the factored FP32 form:
    the regular path flags it DEGENERATE and recomputes it in FP64.  The allocation-free
    call has no FP64 pass: it flags the same pair, returns PHMM_OK, and leaves the other
    pairs exact to the FP32 tolerance."""
    rng = np.random.default_rng(11)
    hap = "".join(rng.choice(list("ACGT"), size=700))
    pairs = [
        (hap[40:190], hap[:400], 30, 45, 45, 10),
        (hap[100:250], hap[60:500], 30, 45, 45, 0),  # degenerate
        (hap[300:450], hap[250:700], 20, 40, 40, 10),
    ]
    b = W.from_strings(pairs)
    ref = oracle.batch(b)
    reg, reg_flags = _regular(phmm, b)
    assert reg_flags[1] & phmm.PAIR_DEGENERATE and reg_flags[1] & phmm.PAIR_RESCUED
    d = phmm.to_device(b)
    for _call in range(2):
        rc, o, f = _noalloc(phmm, d, 3)
        assert rc == phmm.PHMM_OK, rc
        assert f[1] & phmm.PAIR_DEGENERATE
        assert np.array_equal(f & REASONS, reg_flags & REASONS)
        assert np.max(np.abs(o[[0, 2]] - ref[[0, 2]])) <= TOL32


def test_noalloc_scratch_full_then_recovers(phmm):
    """More read bases than the scratch holds (2^20 + 1): PHMM_ENOMEM, no pair computed;
    the next call with a batch that fits succeeds."""
    rng = np.random.default_rng(2)
    big = "".join(rng.choice(list("ACGT"), size=MAX_BASES))
    b = W.from_strings([(big, "ACGTACGTAC", 30, 45, 45, 10), ("A", "ACGT", 30, 45, 45, 10)])
    assert int(b["read_off"][-1]) == MAX_BASES + 1
    d = phmm.to_device(b)
    rc, o, f = _noalloc(phmm, d, 2)
    assert rc == phmm.PHMM_ENOMEM, rc
    assert np.all(np.isnan(o)) and np.all(f & phmm.PAIR_ERROR)
    small = W.plain_pairs(16, seed=3)
    rc, o, _f = _noalloc(phmm, phmm.to_device(small), 16)
    assert rc == phmm.PHMM_OK
    assert np.max(np.abs(o - oracle.batch(small))) <= TOL32


def test_noalloc_rejects_bad_offsets(phmm):
    """Offsets are checked on the device before any access through them: a read range
    that runs backwards and a haplotype range past the last offset give NaN and
    PHMM_PAIR_ERROR for their pairs and PHMM_EINVAL for the call; a valid pair in the same
    batch is still scored."""
    import torch
    good = W.from_strings([("ACGTACGTAC", "TTACGTACGTACAA", 30, 45, 45, 10)])
    ref = oracle.batch(good)[0]
    reads = b"ACGTACGTAC" + b"ACGTA" + b"GGGGCCCC"          # 23 read bases
    haps = b"TTACGTACGTACAA" + b"CCCCCC"                    # 20 haplotype bases
    read_off = np.array([0, 10, 5, 23], np.int64)            # read 1 runs backwards
    hap_off = np.array([0, 14, 5000, 20], np.int64)          # haplotype 1 ends past the last offset
    pair_read = np.array([0, 1, 0, 0], np.int32)
    pair_hap = np.array([0, 0, 1, 2], np.int32)              # haplotype 2 runs backwards
    nb = len(reads)
    u8 = lambda x: torch.from_numpy(np.frombuffer(x, np.uint8).copy()).cuda()
    d = {"read_bases": u8(reads), "base_q": torch.full((nb,), 30, dtype=torch.uint8, device="cuda"),
         "ins_q": torch.full((nb,), 45, dtype=torch.uint8, device="cuda"),
         "del_q": torch.full((nb,), 45, dtype=torch.uint8, device="cuda"),
         "gcp_q": torch.full((nb,), 10, dtype=torch.uint8, device="cuda"),
         "hap_bases": u8(haps), "read_off": torch.from_numpy(read_off).cuda(),
         "hap_off": torch.from_numpy(hap_off).cuda(), "pair_read": torch.from_numpy(pair_read).cuda(),
         "pair_hap": torch.from_numpy(pair_hap).cuda()}
    rc, o, f = _noalloc(phmm, d, 4)
    assert rc == phmm.PHMM_EINVAL, rc
    assert abs(o[0] - ref) <= TOL32 and not (f[0] & phmm.PAIR_ERROR)
    assert np.all(np.isnan(o[1:])) and np.all(f[1:] & phmm.PAIR_ERROR)


def test_noalloc_rejects_oversize(phmm):
    b = W.from_strings([("ACGT" * 10, "ACGT" * 300, 30, 45, 45, 10), ("ACGT", "ACGTA", 30, 45, 45, 10)])
    d = phmm.to_device(b)
    rc, o, f = _noalloc(phmm, d, 2)
    assert rc == phmm.PHMM_EINVAL  # haplotype of 1200 > 1024
    assert np.isnan(o[0]) and np.isfinite(o[1])
    assert (f[0] & phmm.PAIR_ERROR) != 0
