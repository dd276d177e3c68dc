"""GPU parity: the CUDA path through the C ABI against the CPU oracle, element by element.

Tolerances (absolute, in log10 L): 1e-3 for the FP32 path, 1e-9 for FP64 (the FP64 mode
and every pair the rescue pass recomputed).
"""
import math

import numpy as np
import pytest

import oracle
from paper_2606_25738_gb300 import workloads as W

pytestmark = pytest.mark.gpu

TOL32 = 1e-3
TOL64 = 1e-9


@pytest.fixture(scope="module")
def phmm():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2606_25738_gb300 import phmm as P
    return P


def _check(out, flags, ref, tol32=TOL32, tol64=TOL64):
    out = np.asarray(out)
    ref = np.asarray(ref)
    fin = np.isfinite(ref)
    assert np.array_equal(np.isfinite(out), fin), (out[~fin], ref[~fin])
    assert np.array_equal(out[~fin], ref[~fin]) or np.all(np.isnan(out[~fin]) == np.isnan(ref[~fin]))
    d = np.abs(out[fin] - ref[fin])
    tol = np.where((flags[fin] & 0x5) != 0, tol64, tol32)
    bad = np.flatnonzero(d > tol)
    assert bad.size == 0, "max |dlog10| %g at %s (flags %s)" % (d.max(), bad[:8], flags[fin][bad[:8]])
    return float(d.max()) if d.size else 0.0


def test_plain_64_pairs_fp32(phmm):
    """64 short pairs (200-400 bp haplotypes, 100-150 bp reads): FP32 + rescue vs oracle."""
    b = W.plain_pairs(64, seed=0)
    with phmm.Context(precision="fp32") as ctx:
        out, flags, rc, st = ctx.run(b)
    assert rc == 0
    _check(out, flags, oracle.batch(b))
    assert st["kernel_launches"] >= 4


@pytest.mark.parametrize("N,variant", [(0, "auto"), (8, "auto"), (16, "auto"), (0, "pipe"), (0, "pipe2")])
def test_plain_64_pairs_fp64(phmm, N, variant):
    """FP64 mode, every forward variant (unfactored: 8 columns per lane in 16-warp CTAs, 16
    in 8-warp CTAs; pipelined short teams of 16 or 32 columns per lane) and the tuner's
    choice; pairs up to 1200 columns (teams and linked warps)."""
    b = W.plain_pairs(64, seed=0, k_range=(200, 1200))
    with phmm.Context(precision="fp64", cols_per_lane=N, variant=variant) as ctx:
        out, flags, rc, st = ctx.run(b)
    assert np.all(flags & phmm.PAIR_FP64)
    if N or variant != "auto":
        assert st["short_kernel"] == ({8: 0, 16: 1}[N] if N else {"pipe": 2, "pipe2": 3}[variant])
    ref = oracle.batch(b)
    assert np.max(np.abs(out - ref)) <= TOL64


@pytest.mark.parametrize("variant,fid", [("pipe", 2), ("pipe2", 3)])
def test_fp64_pipelined_engine_range_and_degenerate_rows(phmm, variant, fid):
    """The pipelined FP64 engine carries J = I / T_MI with checkpoints like the FP32 one:
    long reads (rescaling), insertion Phred 93 next to 1, and a gap-continuation Phred 0
    row (1 - g = 0: the J-form is unusable) which must go to the unfactored pass."""
    rng = np.random.default_rng(8)
    hap = "".join(rng.choice(list("ACGT"), size=900))
    read = hap[100:400] + hap[410:500]
    l = len(read)
    alt = np.where(np.arange(l) % 2 == 0, 93, 1)
    pairs = [(read, hap, 30, 45, 45, 10), (read, hap, 30, alt, 45, 10), (read, hap, 30, 45, 45, 0),
             (read[:80], hap[:200], 20, 93, 93, 10)]
    b = W.from_strings(pairs)
    lb = W.long_pairs(3, seed=14, k_range=(2000, 9000))
    for batch in (b, lb):
        with phmm.Context(precision="fp64", variant=variant) as ctx:
            out, flags, rc, st = ctx.run(batch)
        assert st["short_kernel"] == fid
        ref = oracle.batch(batch)
        _check(out, flags, ref, tol32=TOL64)
        if batch is b:
            assert ref[2] == -np.inf and out[2] == -np.inf


def test_force_rescue_fp64_pass(phmm):
    """Every pair through the FP64 rescue pass: results within 1e-9 and flagged."""
    b = W.plain_pairs(32, seed=5)
    with phmm.Context(precision="fp32", flags=phmm.F_FORCE_RESCUE) as ctx:
        out, flags, rc, st = ctx.run(b)
    assert st["n_rescued"] == 32
    assert np.all(flags & phmm.PAIR_RESCUED)
    assert np.max(np.abs(out - oracle.batch(b))) <= TOL64


VARIANTS = [("packed", 12), ("packed", 16), ("lean", 24), ("lean", 32), ("pipe", 16), ("pipe", 24),
            ("pipe", 32), ("pipe2", 24), ("pipe2", 32), ("pipe2lean", 32)]


@pytest.mark.parametrize("variant,N", [("packed", 12), ("packed", 16)])
def test_packed_same_read_teams(phmm, variant, N):
    """Active-region batches: haplotypes of the same read packed two per thread."""
    b = W.short_read_regions(n_regions=30, seed=8)
    with phmm.Context(precision="fp32_only", cols_per_lane=N, variant=variant) as ctx:
        out, flags, rc, st = ctx.run(b)
    assert st["cols_per_lane"] == N
    ref = oracle.batch(b)
    assert np.max(np.abs(out - ref)) <= TOL32
    assert np.all((flags & 0x78) == 0)


@pytest.mark.parametrize("variant,N", VARIANTS)
def test_columns_per_lane(phmm, variant, N):
    """Every compiled short-team kernel (packed: two pairs per lane; scalar) gives
    oracle-equal results, together with multi-warp pairs beyond 32 N columns."""
    b = W.plain_pairs(40, seed=11, k_range=(1, 40 * N), l_range=(1, 300), indel_rate=0.01)
    with phmm.Context(precision="fp32", cols_per_lane=N, variant=variant) as ctx:
        out, flags, rc, st = ctx.run(b)
    _check(out, flags, oracle.batch(b))


LONG_KINDS = ["lean", "pipe32", "pipe24", "serial", "pipe4", "cluster", "wave", "wave16"]


def _long_flag(phmm, kind):
    return {"lean": phmm.F_LONG_LEAN, "pipe32": phmm.F_LONG_PIPE32, "pipe24": phmm.F_LONG_PIPE24,
            "serial": phmm.F_LONG_SERIAL, "pipe4": phmm.F_LONG_PIPE4, "cluster": phmm.F_LONG_CLUSTER,
            "wave": phmm.F_LONG_WAVE, "wave16": phmm.F_LONG_WAVE16}[kind]


@pytest.mark.parametrize("variant,N", VARIANTS)
@pytest.mark.parametrize("kind", LONG_KINDS)
def test_fp32_path_without_rescue(phmm, variant, N, kind):
    """The FP32 engines alone (no FP64 rescue pass): short teams and multi-warp pairs up to
    16384 columns (every multi-warp kernel, strips included) stay within 1e-3 and none is
    flagged for rescue."""
    if variant == "lean" and kind != "lean":
        pytest.skip("the lean variant keeps the lean multi-warp engine")
    b = W.plain_pairs(48, seed=12, k_range=(1, 16384), l_range=(1, 400), indel_rate=0.01)
    with phmm.Context(precision="fp32_only", cols_per_lane=N, variant=variant,
                      flags=_long_flag(phmm, kind)) as ctx:
        out, flags, rc, st = ctx.run(b)
    assert st["n_long"] > 0
    assert np.all((flags & 0x78) == 0), flags[(flags & 0x78) != 0]
    ref = oracle.batch(b)
    assert np.max(np.abs(out - ref)) <= TOL32


def _edge_batch(N=16):
    rng = np.random.default_rng(3)
    rs = lambda n: "".join(rng.choice(list("ACGT"), size=n))
    hap = rs(300)
    pairs = [
        ("A", "A", 30, 45, 45, 10),                  # l = k = 1
        ("C", "ACGTA", 30, 45, 45, 10),              # l = 1
        (rs(10), rs(3), 30, 45, 45, 10),             # l > k
        (rs(40), "G", 20, 45, 45, 10),               # k = 1
        ("N" * 50, hap[:120], 30, 45, 45, 10),       # all-N read
        (hap[10:90], hap, 0, 45, 45, 10),            # Phred 0 base quality
        (hap[10:90], hap, 93, 45, 45, 10),           # Phred 93
        (hap[5:60], hap, 30, 93, 93, 10),            # near-zero gap opens
        (hap[5:60], hap, 30, 10, 10, 10),            # frequent gaps
        (hap[:100] + hap[150:250], hap, 30, 45, 45, 10),   # 50 bp deletion
        (hap[:60] + rs(40) + hap[60:150], hap, 30, 45, 45, 10),  # 40 bp insertion
        (hap[:N], hap[:N], 30, 45, 45, 10),          # k = N
        (hap[:N + 1], hap[:N + 1], 30, 45, 45, 10),  # k = N + 1
        (rs(120), rs(32 * N), 30, 45, 45, 10),       # k = 32 N (one full packed team)
        (rs(120), rs(32 * N + 1), 30, 45, 45, 10),   # k = 32 N + 1 (multi-warp path)
        (rs(150), rs(3 * 1024 - 1), 30, 45, 45, 10), # three 1024-column warp segments
        (rs(150), rs(3 * 1024 + 1), 30, 45, 45, 10),
        (rs(30), rs(600), 30, 45, 45, 10),
        (hap[:200], hap, np.arange(200) % 41, np.arange(200) % 30 + 15, 40, 10),  # per-row quals
        (hap[:150], hap, 25, 40, 40, np.arange(150) % 20 + 5),  # per-row gap continuation
        (hap[:150].lower(), hap.lower(), 30, 45, 45, 10),  # lower case
    ]
    return W.from_strings(pairs)


@pytest.mark.parametrize("prec,variant", [("fp32", "packed"), ("fp32", "scalar"), ("fp32", "lean"),
                                          ("fp32", "pipe"), ("fp32", "pipe2"), ("fp64", "auto")])
def test_edge_cases(phmm, prec, variant):
    n = {"packed": 16, "scalar": 24, "lean": 32, "pipe": 32, "pipe2": 32}.get(variant, 0) if prec == "fp32" else 0
    b = _edge_batch(max(n, 16))
    with phmm.Context(precision=prec, cols_per_lane=n, variant=variant) as ctx:
        out, flags, rc, st = ctx.run(b)
    ref = oracle.batch(b)
    if prec == "fp64":
        fin = np.isfinite(ref)
        assert np.array_equal(np.isfinite(out), fin)
        assert np.max(np.abs(out[fin] - ref[fin])) <= TOL64
    else:
        _check(out, flags, ref)


def test_long_deletion_50bp(phmm):
    """A read whose best alignment needs a 50 bp deletion: the carry crosses lanes and
    warps through the scan and must not be dropped."""
    rng = np.random.default_rng(9)
    hap = "".join(rng.choice(list("ACGT"), size=2000))
    read = hap[100:700] + hap[750:1350]
    b = W.from_strings([(read, hap, 30, 45, 45, 10)])
    for N, v in ((12, "packed"), (16, "packed"), (24, "lean"), (32, "lean"), (16, "pipe"), (24, "pipe"),
                 (32, "pipe"), (24, "pipe2"), (32, "pipe2")):
        with phmm.Context(precision="fp32", cols_per_lane=N, variant=v) as ctx:
            out, flags, rc, st = ctx.run(b)
        _check(out, flags, oracle.batch(b))


def test_scan_unit(phmm):
    import torch
    rng = np.random.default_rng(1)
    with phmm.Context() as ctx:
        for n, a in ((1, 0.1), (31, 0.5), (33, 0.1), (1024, 0.1), (1000, 0.9), (517, 1.0)):
            y = rng.uniform(0.5, 2.0, n).astype(np.float32)
            z = ctx.scan_test(torch.from_numpy(y).cuda(), a).cpu().numpy()
            ref = np.zeros(n)
            acc = 0.0
            for t in range(n):
                acc = a * acc + float(y[t])
                ref[t] = acc
            assert np.allclose(z, ref, rtol=1e-5, atol=0), (n, a)


def test_device_inputs_outputs(phmm):
    import torch
    b = W.plain_pairs(24, seed=2)
    d = phmm.to_device(b)
    out = torch.empty(24, dtype=torch.float64, device="cuda")
    fl = torch.zeros(24, dtype=torch.uint8, device="cuda")
    with phmm.Context() as ctx:
        t = ctx.submit(d, out, fl)
        assert ctx.poll(t, -1) == 0
    _check(out.cpu().numpy(), fl.cpu().numpy(), oracle.batch(b))


def test_graph_replay_equals_eager(phmm):
    b = W.plain_pairs(48, seed=4, k_range=(100, 1500))
    with phmm.Context() as c1:
        a1, f1, _, _ = c1.run(b)
        a2, f2, _, _ = c1.run(b)  # graph replay
    with phmm.Context(flags=phmm.F_NO_GRAPH) as c2:
        a3, f3, _, _ = c2.run(b)
    assert np.array_equal(a1, a2) and np.array_equal(a1, a3)
    assert np.array_equal(f1, f3)


def test_invalid_input_reported(phmm):
    b = W.from_strings([("ACGT", "ACGT", 30, 45, 45, 10), ("AXGT", "ACGT", 30, 45, 45, 10),
                        ("ACGT", "ACGT", 94, 45, 45, 10), ("ACG", "AC?T", 30, 45, 45, 10)])
    with phmm.Context() as ctx:
        out, flags, rc, st = ctx.run(b, check=False)
    assert rc == phmm.PHMM_EINVAL
    assert math.isfinite(out[0]) and np.all(np.isnan(out[1:]))
    assert np.all(flags[1:] & phmm.PAIR_ERROR)


def test_launch_per_pair_fp64(phmm):
    b = W.plain_pairs(8, seed=6)
    with phmm.Context(precision="fp64", flags=phmm.F_LAUNCH_PER_PAIR) as ctx:
        out, flags, rc, st = ctx.run(b)
    assert st["kernel_launches"] == 8 + 3
    assert np.max(np.abs(out - oracle.batch(b))) <= TOL64


def _wide_batch(seed=30):
    """Pairs wider than one 16-warp CTA (strips), with moderate read lengths so the oracle
    stays fast: haplotypes 16k-60k bp, reads 200-600 bp from a random offset."""
    rng = np.random.default_rng(seed)
    pairs = []
    for k in (16385, 20000, 33000, 49153, 60000):
        hap = "".join(rng.choice(list("ACGT"), size=k))
        l = int(rng.integers(200, 601))
        off = int(rng.integers(0, k - l))
        read = list(hap[off:off + l])
        for p in rng.choice(l, size=l // 40, replace=False):
            read[p] = "ACGT"[("ACGT".index(read[p]) + 1) % 4]
        pairs.append(("".join(read), hap, rng.integers(10, 41, size=l), 45, 45, 10))
    return W.from_strings(pairs)


@pytest.mark.parametrize("kind", LONG_KINDS)
def test_wide_pairs_fp32_strips(phmm, kind):
    """Concurrent strips (global row boundaries between CTAs), FP32 only."""
    b = _wide_batch()
    with phmm.Context(precision="fp32_only", flags=_long_flag(phmm, kind)) as ctx:
        out, flags, rc, st = ctx.run(b)
    assert st["n_long"] == 5
    assert np.all((flags & 0x78) == 0)
    assert np.max(np.abs(out - oracle.batch(b))) <= TOL32


def test_cluster_kind_single_very_wide_pair(phmm):
    """One pair of 131072 columns on the cluster kind: 32 strips of 4096 columns in four
    groups of eight CTAs, neighbours inside a group linked through distributed shared
    memory, groups through global memory; the read is short enough for the oracle."""
    rng = np.random.default_rng(44)
    k = 131072
    hap = "".join(rng.choice(list("ACGT"), size=k))
    off = 70000
    read = hap[off:off + 180]
    b = W.from_strings([(read, hap, 30, 45, 45, 10), (read[:90], hap[:20000], 25, 45, 45, 10)])
    with phmm.Context(precision="fp32", flags=phmm.F_LONG_CLUSTER) as ctx:
        out, flags, rc, st = ctx.run(b)
    assert st["long_kernel"] == 5 and st["n_long"] == 2
    _check(out, flags, oracle.batch(b))


@pytest.mark.parametrize("kind", ["wave", "wave16"])
def test_wave_kind_very_wide_pairs(phmm, kind):
    """The wave kinds: 128 strips (256 at 512 columns) of one 131072-column pair run at
    the same time, each waiting for its left neighbour's progress once per 32 rows (a
    700-row read: 22 blocks), next to a pair of 20 (40) strips; both against the oracle."""
    rng = np.random.default_rng(45)
    k = 131072
    hap = "".join(rng.choice(list("ACGT"), size=k))
    read = hap[90000:90400] + hap[90410:90710]
    b = W.from_strings([(read, hap, 30, 45, 45, 10), (read[:333], hap[:20000], 25, 45, 45, 10)])
    with phmm.Context(precision="fp32", flags=_long_flag(phmm, kind)) as ctx:
        out, flags, rc, st = ctx.run(b)
    assert st["long_kernel"] in ((6, 7, 8) if kind == "wave" else (8,)) and st["n_long"] == 2
    assert not np.any(flags & phmm.PAIR_ERROR)
    _check(out, flags, oracle.batch(b))


@pytest.mark.parametrize("N", [8, 16])
def test_wide_pairs_fp64_strips(phmm, N):
    """Concurrent strips in the batched FP64 engine (4096 columns per CTA), both variants."""
    b = _wide_batch(seed=31)
    with phmm.Context(precision="fp64", cols_per_lane=N) as ctx:
        out, flags, rc, st = ctx.run(b)
    assert np.max(np.abs(out - oracle.batch(b))) <= TOL64


def test_wide_pairs_rescue_sequential_strips(phmm):
    """FP64 rescue of wide pairs: strips run one after another inside one CTA."""
    b = _wide_batch(seed=32)
    with phmm.Context(precision="fp32", flags=phmm.F_FORCE_RESCUE) as ctx:
        out, flags, rc, st = ctx.run(b)
    assert st["n_rescued"] == 5
    assert np.max(np.abs(out - oracle.batch(b))) <= TOL64


@pytest.mark.parametrize("kind", LONG_KINDS)
def test_long_reads_reduced(phmm, kind):
    """Long-read-like pairs (reads 90-100% of haplotypes of 1k-20k bp, 5% substitutions,
    3% indels, quals 5-30): FP32 + rescue within 1e-3 including multi-warp and strip
    pairs; checkpoint rescaling must have happened."""
    b = W.long_pairs(10, seed=4, k_range=(1000, 20000))
    with phmm.Context(precision="fp32", flags=_long_flag(phmm, kind)) as ctx:
        out, flags, rc, st = ctx.run(b)
    ref = oracle.batch(b)
    assert np.all(ref < -300)  # far below what a fixed 2^120 scale could hold
    _check(out, flags, ref)
    assert np.all(flags & phmm.PAIR_RESCALED)


def test_launch_per_pair_wide(phmm):
    b = _wide_batch(seed=33)
    with phmm.Context(precision="fp64", flags=phmm.F_LAUNCH_PER_PAIR) as ctx:
        out, flags, rc, st = ctx.run(b)
    assert np.max(np.abs(out - oracle.batch(b))) <= TOL64


@pytest.mark.parametrize("L", [32, 64, 128])
def test_short_equal_length_no_spurious_rescue(phmm, L):
    """Short equal-length pairs (the first lengths of the scalability sweep): the initial
    scale 2^120 / k is largest here, and no FP32 kernel may overflow on it, so no pair
    needs the rescue pass."""
    b = W.equal_length(1500, L, seed=1)
    ref = oracle.batch(b)
    for v, N in (("pipe", 32), ("pipe", 16), ("lean", 32), ("packed", 12), ("pipe2", 32)):
        with phmm.Context(precision="fp32", variant=v, cols_per_lane=N) as ctx:
            out, flags, rc, st = ctx.run(b)
        assert st["n_rescued"] == 0, (v, N, np.unique(flags, return_counts=True))
        _check(out, flags, ref)


def test_pipelined_engine_extreme_gap_qualities(phmm):
    """The pipelined engine carries J = I / T_MI: insertion Phred 93 next to 1, gap
    continuation 1-2 and mixed rows stress its range; every pair is within 1e-3 or
    flagged and rescued (then within 1e-9)."""
    rng = np.random.default_rng(5)
    hap = "".join(rng.choice(list("ACGT"), size=900))
    read = hap[100:400] + hap[410:700]
    l = len(read)
    alt = np.where(np.arange(l) % 2 == 0, 93, 1)
    pairs = [
        (read, hap, 30, 93, 93, 10),
        (read, hap, 30, alt, 45, 10),
        (read, hap, 30, 45, alt, 10),
        (read, hap, 30, 45, 45, 1),
        (read, hap, 30, 93, 0, 2),
        (read, hap, 30, np.arange(l) % 94, 40, np.arange(l) % 20 + 1),
        (read[:60], hap[:64], 30, 93, 93, 10),
    ]
    b = W.from_strings(pairs)
    for v, N in (("pipe", 16), ("pipe", 24), ("pipe", 32), ("pipe2", 24), ("pipe2", 32)):
        with phmm.Context(precision="fp32", variant=v, cols_per_lane=N) as ctx:
            out, flags, rc, st = ctx.run(b)
        _check(out, flags, oracle.batch(b))


def test_rounding_bound_triggers_fp64_rescue(phmm):
    """The a-priori FP32 rounding bound, (6.5 sqrt(16 l + 4 k) 2^-23 + 8 l 2^-46) / ln 10,
    grows with the pair's size.  Under a tolerance that half the pairs exceed, exactly
    those are flagged DANGER and recomputed in FP64 (within 1e-9 of the oracle); at the
    default tolerance (1e-3) none of them is."""
    b = W.plain_pairs(24, seed=4, k_range=(250, 400), l_range=(2, 300))
    rl, hl = W.pair_lengths(b)
    ref = oracle.batch(b)
    with phmm.Context(precision="fp32") as ctx:
        out, flags, rc, st = ctx.run(b)
    assert st["n_rescued"] == 0 and not np.any(flags & 0x8)
    bound = (6.5 * np.sqrt(16.0 * rl + 4.0 * hl) * 2.0 ** -23 + 8.0 * rl * 2.0 ** -46) / np.log(10.0)
    tol = float(np.median(bound))
    over = bound > tol
    assert over.any() and (~over).any()
    with phmm.Context(precision="fp32", tolerance=tol) as ctx:
        out, flags, rc, st = ctx.run(b)
    assert np.array_equal((flags & phmm.PAIR_RESCUED) != 0, over)
    assert np.all(flags[over] & phmm.PAIR_DANGER)
    assert st["n_rescued"] == int(over.sum())
    _check(out, flags, ref)
    assert np.max(np.abs(out[over] - ref[over])) <= TOL64


def test_bounded_wait_times_out_and_context_survives(phmm):
    """A device-side wait that can never be satisfied gives up within its poll limit and
    reports PHMM_ETIMEOUT; the same context then still scores a batch correctly."""
    import time
    b = W.plain_pairs(8, seed=40)
    with phmm.Context() as ctx:
        t = time.perf_counter()
        assert ctx.wait_test() == phmm.PHMM_ETIMEOUT
        assert time.perf_counter() - t < 30.0
        out, flags, rc, st = ctx.run(b)
    assert rc == 0
    _check(out, flags, oracle.batch(b))


def _strip_edge_batch():
    """Wide pairs at the serial kind's strip edges: one column in the last strip, exact
    multiples of 1024, one-row reads, reads longer than the haplotype."""
    rng = np.random.default_rng(41)
    rs = lambda n: "".join(rng.choice(list("ACGT"), size=n))
    hap = rs(5 * 1024 + 1)
    pairs = [
        (rs(120), hap[:1025], 30, 45, 45, 10),           # last strip: one column
        (rs(120), hap[:2048], 30, 45, 45, 10),           # exactly two strips
        (hap[100:400], hap[:4096], 30, 45, 45, 10),      # exactly four strips
        ("A", hap[:3000], 30, 45, 45, 10),               # one row
        (hap[:70], hap[:5121], 30, 45, 45, 10),          # five strips and one column
        (rs(1500), hap[:1100], 30, 45, 45, 10),          # more rows than columns
        (hap[:2000], hap[:2100], 30, 40, 40, np.arange(2000) % 20 + 5),  # per-row gcp
    ]
    return W.from_strings(pairs)


@pytest.mark.parametrize("prec,flag", [("fp32_only", "serial"), ("fp32", "serial"), ("fp32", "rescue")])
def test_serial_strip_edges(phmm, prec, flag):
    """The serial multi-warp kind at its strip boundaries; with forced rescue the FP64
    pass recomputes the same pairs."""
    b = _strip_edge_batch()
    f = phmm.F_LONG_SERIAL | (phmm.F_FORCE_RESCUE if flag == "rescue" else 0)
    with phmm.Context(precision=prec, flags=f) as ctx:
        out, flags, rc, st = ctx.run(b)
    assert st["long_kernel"] == 3
    ref = oracle.batch(b)
    if flag == "rescue":
        assert np.all(flags & phmm.PAIR_RESCUED)
        assert np.max(np.abs(out - ref)) <= TOL64
    else:
        assert np.all((flags & 0x78) == 0)
        assert np.max(np.abs(out - ref)) <= TOL32


def test_stats_name_the_kernels_and_no_tune(phmm):
    """Per-ticket stats report the kernels a plan ran; PHMM_F_NO_TUNE (cost model only)
    gives oracle-equal results too."""
    b = W.plain_pairs(40, seed=17, k_range=(100, 6000), l_range=(50, 300))
    ref = oracle.batch(b)
    with phmm.Context(precision="fp32", variant="pipe2", cols_per_lane=32, flags=phmm.F_LONG_SERIAL) as ctx:
        out, flags, rc, st = ctx.run(b)
    assert phmm.SHORT_KERNELS[st["short_kernel"]].startswith("k_short_pipe2<32")
    assert phmm.LONG_KERNELS[st["long_kernel"]] == "k_forward_serial<32, 3, 0>"
    assert st["packed_kernel"] == -1
    _check(out, flags, ref)
    with phmm.Context(precision="fp32", flags=phmm.F_NO_TUNE) as ctx:
        out2, flags2, rc2, st2 = ctx.run(b)
    _check(out2, flags2, ref)
    with phmm.Context(precision="fp64") as ctx:
        out3, flags3, rc3, st3 = ctx.run(b)
    # FP64: short_kernel names the FP64 forward variant
    assert st3["short_kernel"] in (0, 1, 2, 3) and st3["long_kernel"] == -1 and st3["packed_kernel"] == -1
    _check(out3, flags3, ref)


def test_empty_batch(phmm):
    """A batch with reads and haplotypes but no pairs completes with empty outputs."""
    b = W.subset(W.plain_pairs(3, seed=1), [])
    with phmm.Context() as ctx:
        out, flags, rc, st = ctx.run(b)
    assert rc == phmm.PHMM_OK and len(out) == 0 and len(flags) == 0
    assert st["n_pairs"] == 0 and st["cells"] == 0
