"""Seeded synthetic PairHMM workloads.

This module only draws inputs: reads, haplotypes, Phred qualities and the pair index,
in the library's batch layout.  It holds none of the forward algorithm's arithmetic and
is shared by the tests, the benchmark and the oracle legs, so that both sides of every
parity check see the same bytes.

Batch layout (a dict of numpy arrays):
    read_bases  uint8   ASCII A/C/G/T/N, all reads concatenated
    read_off    uint64  n_reads + 1 offsets into read_bases
    base_q, ins_q, del_q, gcp_q   uint8 numeric Phred 0..93, laid out like read_bases
    hap_bases   uint8   ASCII A/C/G/T/N, all haplotypes concatenated
    hap_off     uint64  n_haps + 1 offsets
    pair_read, pair_hap uint32 one (read, haplotype) index per pair

The shapes follow the workloads the paper evaluates on (GIAB short- and long-read sets,
Table "GIAB Dataset Description"; the 10s set; equal-length synthetic pairs of
32..131072 bp, Section 4.1) -- none of those datasets is used or reproduced; only their
length and error structure is imitated.
"""
from __future__ import annotations

import numpy as np

ACGT = np.frombuffer(b"ACGT", dtype=np.uint8)


def _rng(seed: int, stream: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(np.random.SeedSequence([seed, stream])))


def _random_bases(rng, n: int) -> np.ndarray:
    return ACGT[rng.integers(0, 4, size=n)]


def _substitute(rng, seq: np.ndarray, rate: float) -> np.ndarray:
    """Replace each base with probability ``rate`` by one of the other three."""
    out = seq.copy()
    m = rng.random(len(seq)) < rate
    if m.any():
        codes = np.searchsorted(ACGT, out[m])  # N never occurs in templates
        shift = rng.integers(1, 4, size=int(m.sum()))
        out[m] = ACGT[(codes + shift) % 4]
    return out


def _mutate(rng, template: np.ndarray, start: int, length: int, sub_rate: float,
            indel_rate: float) -> np.ndarray:
    """Read of exactly ``length`` bases copied from ``template[start:]`` with
    substitutions and 1-3 bp insertions/deletions (50:50).  Runs past the template end
    are filled with random bases."""
    if indel_rate <= 0.0:
        seg = template[start:start + length]
        if len(seg) < length:
            seg = np.concatenate([seg, _random_bases(rng, length - len(seg))])
        return _substitute(rng, seg, sub_rate)
    pieces = []
    have = 0
    pos = start
    n_t = len(template)
    # Events are drawn per template base with a geometric gap.
    while have < length:
        gap = int(rng.geometric(indel_rate)) if indel_rate < 1.0 else 1
        take = min(gap - 1, length - have, max(n_t - pos, 0))
        if take > 0:
            pieces.append(template[pos:pos + take])
            have += take
            pos += take
        if have >= length:
            break
        if pos >= n_t:
            pieces.append(_random_bases(rng, length - have))
            have = length
            break
        ln = int(rng.integers(1, 4))
        if rng.random() < 0.5:  # insertion into the read
            ins = _random_bases(rng, min(ln, length - have))
            pieces.append(ins)
            have += len(ins)
        else:  # deletion from the read
            pos += ln
    read = np.concatenate(pieces)[:length] if pieces else np.zeros(0, np.uint8)
    return _substitute(rng, read, sub_rate)


def _pack(reads, quals, haps, pair_read, pair_hap) -> dict:
    """Concatenate per-read / per-haplotype arrays into the batch layout."""
    rl = np.array([len(r) for r in reads], dtype=np.uint64)
    hl = np.array([len(h) for h in haps], dtype=np.uint64)
    b = {
        "read_bases": np.concatenate(reads).astype(np.uint8) if reads else np.zeros(0, np.uint8),
        "read_off": np.concatenate([[0], np.cumsum(rl)]).astype(np.uint64),
        "hap_bases": np.concatenate(haps).astype(np.uint8) if haps else np.zeros(0, np.uint8),
        "hap_off": np.concatenate([[0], np.cumsum(hl)]).astype(np.uint64),
        "pair_read": np.asarray(pair_read, dtype=np.uint32),
        "pair_hap": np.asarray(pair_hap, dtype=np.uint32),
    }
    for i, name in enumerate(("base_q", "ins_q", "del_q", "gcp_q")):
        b[name] = (np.concatenate([q[i] for q in quals]).astype(np.uint8) if quals
                   else np.zeros(0, np.uint8))
    return b


def cells(b: dict) -> int:
    """Sum over pairs of read length x haplotype length (the cell-update count)."""
    rl = np.diff(b["read_off"].astype(np.int64))
    hl = np.diff(b["hap_off"].astype(np.int64))
    return int(np.sum(rl[b["pair_read"]] * hl[b["pair_hap"]]))


def pair_lengths(b: dict):
    rl = np.diff(b["read_off"].astype(np.int64))
    hl = np.diff(b["hap_off"].astype(np.int64))
    return rl[b["pair_read"]], hl[b["pair_hap"]]


# ----------------------------------------------------------------------------------------
# Workloads
# ----------------------------------------------------------------------------------------

def plain_pairs(n_pairs: int = 64, seed: int = 0, k_range=(200, 400), l_range=(100, 150),
                sub_rate=0.01, indel_rate=0.001, q_range=(10, 40), gap_q=45, gcp_q=10) -> dict:
    """Short-read parity set: one haplotype per pair, uniform ACGT of length U{k_range};
    the read (length U{l_range}) starts at a random haplotype offset, with substitutions
    and 1-3 bp indels; base quals U{q_range}, ins/del quals ``gap_q``, gcp ``gcp_q``."""
    rng = _rng(seed, 1)
    reads, quals, haps = [], [], []
    for _ in range(n_pairs):
        k = int(rng.integers(k_range[0], k_range[1] + 1))
        l = int(rng.integers(l_range[0], l_range[1] + 1))
        hap = _random_bases(rng, k)
        off = int(rng.integers(0, max(k - l, 0) + 1))
        read = _mutate(rng, hap, off, l, sub_rate, indel_rate)
        bq = rng.integers(q_range[0], q_range[1] + 1, size=l).astype(np.uint8)
        q_i = np.full(l, gap_q, np.uint8)
        quals.append((bq, q_i, q_i.copy(), np.full(l, gcp_q, np.uint8)))
        reads.append(read)
        haps.append(hap)
    idx = np.arange(n_pairs)
    return _pack(reads, quals, haps, idx, idx)


def short_read_regions(n_regions: int = 2000, reads_per_region: int = 50, seed: int = 0,
                       max_haps: int = 8, read_len: int = 150, ref_range=(250, 600),
                       max_pairs: int | None = None) -> dict:
    """Active-region short-read batch: per region a random reference window of length
    U{ref_range}; H ~ U{1..max_haps} haplotypes = reference + SNPs (1e-3 per base) and
    1 bp indels (1e-4 per base); ``reads_per_region`` reads of ``read_len`` bp, each from
    a random haplotype at a random offset, with a per-read substitution rate
    U[0.5%, 2%] and then 1% of bases set to N.  Base quals: 85% U{30..41}, 15% U{2..29};
    ins/del quals U{40..45} per base; gcp 10.  Pairs = every read x every haplotype of
    its region (about 4.5 pairs per read).  ``max_pairs`` truncates in region order."""
    rng = _rng(seed, 2)
    reads, quals, haps = [], [], []
    pr, ph = [], []
    n_pairs = 0
    for _ in range(n_regions):
        rlen = int(rng.integers(ref_range[0], ref_range[1] + 1))
        ref = _random_bases(rng, rlen)
        h_count = int(rng.integers(1, max_haps + 1))
        h0 = len(haps)
        for _h in range(h_count):
            hap = _substitute(rng, ref, 1e-3)
            ev = np.flatnonzero(rng.random(rlen) < 1e-4)
            for p in ev[::-1]:
                if rng.random() < 0.5:
                    hap = np.concatenate([hap[:p], _random_bases(rng, 1), hap[p:]])
                elif len(hap) > 1:
                    hap = np.concatenate([hap[:p], hap[p + 1:]])
            haps.append(hap)
        r0 = len(reads)
        src = rng.integers(0, h_count, size=reads_per_region)
        err = rng.uniform(0.005, 0.02, size=reads_per_region)
        for r in range(reads_per_region):
            hap = haps[h0 + int(src[r])]
            off = int(rng.integers(0, max(len(hap) - read_len, 0) + 1))
            read = _mutate(rng, hap, off, read_len, float(err[r]), 0.0)
            nm = rng.random(read_len) < 0.01
            read[nm] = ord("N")
            hi = rng.random(read_len) < 0.85
            bq = np.where(hi, rng.integers(30, 42, size=read_len),
                          rng.integers(2, 30, size=read_len)).astype(np.uint8)
            iq = rng.integers(40, 46, size=read_len).astype(np.uint8)
            dq = rng.integers(40, 46, size=read_len).astype(np.uint8)
            quals.append((bq, iq, dq, np.full(read_len, 10, np.uint8)))
            reads.append(read)
        for r in range(reads_per_region):
            for h in range(h_count):
                pr.append(r0 + r)
                ph.append(h0 + h)
        n_pairs += reads_per_region * h_count
        if max_pairs is not None and n_pairs >= max_pairs:
            break
    if max_pairs is not None:
        pr, ph = pr[:max_pairs], ph[:max_pairs]
    return _pack(reads, quals, haps, pr, ph)


def long_pairs(n_pairs: int = 64, seed: int = 0, k_range=(1000, 100000), read_frac=(0.9, 1.0),
               sub_rate=0.05, indel_rate=0.03, q_range=(5, 30), gap_q=45, gcp_q=10) -> dict:
    """Long-read pairs: haplotype length log-uniform in ``k_range``; the read is
    90-100% of the haplotype length, copied from a random offset with substitutions and
    1-3 bp indels; base quals U{q_range}, ins/del quals ``gap_q``, gcp ``gcp_q``."""
    rng = _rng(seed, 3)
    reads, quals, haps = [], [], []
    for _ in range(n_pairs):
        k = int(round(np.exp(rng.uniform(np.log(k_range[0]), np.log(k_range[1])))))
        l = max(1, int(round(k * rng.uniform(read_frac[0], read_frac[1]))))
        hap = _random_bases(rng, k)
        off = int(rng.integers(0, k - l + 1))
        read = _mutate(rng, hap, off, l, sub_rate, indel_rate)
        bq = rng.integers(q_range[0], q_range[1] + 1, size=l).astype(np.uint8)
        q_i = np.full(l, gap_q, np.uint8)
        quals.append((bq, q_i, q_i.copy(), np.full(l, gcp_q, np.uint8)))
        reads.append(read)
        haps.append(hap)
    idx = np.arange(n_pairs)
    return _pack(reads, quals, haps, idx, idx)


def _unpack_bases(raw: np.ndarray, n: int) -> np.ndarray:
    """n uniform ACGT bases from random bytes (four 2-bit codes per byte)."""
    codes = np.empty(4 * len(raw), np.uint8)
    for s in range(4):
        codes[s::4] = (raw >> (2 * s)) & 3
    return ACGT[codes[:n]]


def uneven_pairs(n_pairs: int = 1_000_000, seed: int = 0, len_range=(50, 20000),
                 chunk: int = 16384, threads: int | None = None) -> dict:
    """Uneven-length batch: read and haplotype lengths each log-uniform in
    ``len_range``, drawn independently and swapped so that haplotype >= read; the read
    is copied from a random haplotype offset with the short-read error and quality model
    (substitutions at a per-read rate U[0.5%, 2%], 1% N, quals 85% U{30..41} / 15%
    U{2..29}, ins/del U{40..45}, gcp 10).  The million pairs hold about 1.1e9 read and
    5.6e9 haplotype bases: the lengths come from one stream, then every chunk of
    ``chunk`` pairs draws its bases and qualities from a stream of its own, so chunks run
    on ``threads`` threads (default: all cores) and the bytes do not depend on the thread
    count."""
    from concurrent.futures import ThreadPoolExecutor
    import os
    rng = _rng(seed, 4)
    lo, hi = np.log(len_range[0]), np.log(len_range[1])
    a = np.rint(np.exp(rng.uniform(lo, hi, size=n_pairs))).astype(np.int64)
    c = np.rint(np.exp(rng.uniform(lo, hi, size=n_pairs))).astype(np.int64)
    ls, ks = np.minimum(a, c), np.maximum(a, c)
    roff = np.zeros(n_pairs + 1, np.uint64)
    hoff = np.zeros(n_pairs + 1, np.uint64)
    roff[1:] = np.cumsum(ls)
    hoff[1:] = np.cumsum(ks)
    nb, nh = int(roff[-1]), int(hoff[-1])
    off = (rng.random(n_pairs) * (ks - ls + 1)).astype(np.int64)
    rate = rng.uniform(0.005, 0.02, size=n_pairs)
    hap = np.empty(nh, np.uint8)
    read = np.empty(nb, np.uint8)
    bq = np.empty(nb, np.uint8)
    iq = np.empty(nb, np.uint8)
    dq = np.empty(nb, np.uint8)

    def fill(ci: int) -> None:
        p0 = ci * chunk
        p1 = min(n_pairs, p0 + chunk)
        g = np.random.Generator(np.random.PCG64(np.random.SeedSequence([seed, 4, ci + 1])))
        h0, h1 = int(hoff[p0]), int(hoff[p1])
        hap[h0:h1] = _unpack_bases(np.frombuffer(g.bytes((h1 - h0 + 3) // 4), np.uint8), h1 - h0)
        L = ls[p0:p1]
        b0, b1 = int(roff[p0]), int(roff[p1])
        n = b1 - b0
        first = np.repeat(hoff[p0:p1].astype(np.int64) + off[p0:p1], L)
        within = np.arange(n, dtype=np.int64) - np.repeat(roff[p0:p1].astype(np.int64) - b0, L)
        r = hap[first + within]
        m = g.random(n) < np.repeat(rate[p0:p1], L)
        if m.any():
            codes = np.searchsorted(ACGT, r[m])
            r[m] = ACGT[(codes + g.integers(1, 4, size=int(m.sum()))) % 4]
        r[g.random(n) < 0.01] = ord("N")
        read[b0:b1] = r
        hq = g.random(n) < 0.85
        bq[b0:b1] = np.where(hq, g.integers(30, 42, size=n, dtype=np.uint8), g.integers(2, 30, size=n, dtype=np.uint8))
        iq[b0:b1] = g.integers(40, 46, size=n, dtype=np.uint8)
        dq[b0:b1] = g.integers(40, 46, size=n, dtype=np.uint8)

    n_chunks = (n_pairs + chunk - 1) // chunk
    with ThreadPoolExecutor(max_workers=threads or os.cpu_count() or 1) as ex:
        list(ex.map(fill, range(n_chunks)))
    idx = np.arange(n_pairs, dtype=np.uint32)
    return {"read_bases": read, "read_off": roff, "hap_bases": hap, "hap_off": hoff,
            "pair_read": idx, "pair_hap": idx.copy(), "base_q": bq, "ins_q": iq, "del_q": dq,
            "gcp_q": np.full(nb, 10, np.uint8)}


def stratified_sample(b: dict, per_decile: int, seed: int = 0, max_cells: float = 4e10) -> np.ndarray:
    """Pair indices for a parity check: up to ``per_decile`` random pairs from each decile
    of the per-pair cell count l*k, keeping the sample's total cells under ``max_cells``
    (largest pairs thinned first)."""
    rl, hl = pair_lengths(b)
    c = rl * hl
    order = np.argsort(c, kind="stable")
    rng = np.random.default_rng(seed)
    picks = [rng.choice(dec, min(per_decile, len(dec)), replace=False)
             for dec in np.array_split(order, 10) if len(dec)]
    pick = np.unique(np.concatenate(picks)) if picks else np.zeros(0, np.int64)
    while c[pick].sum() > max_cells and len(pick) > 10:
        big = np.argsort(c[pick])[::-1]
        pick = np.delete(pick, big[: max(1, len(pick) // 20)])
    return pick


def _short_read_quals(rng, n: int):
    """Base quals 85% U{30..41} / 15% U{2..29}; ins/del U{40..45}; gcp 10."""
    hi = rng.random(n) < 0.85
    bq = np.where(hi, rng.integers(30, 42, size=n), rng.integers(2, 30, size=n)).astype(np.uint8)
    return (bq, rng.integers(40, 46, size=n).astype(np.uint8),
            rng.integers(40, 46, size=n).astype(np.uint8), np.full(n, 10, np.uint8))


def region_request(rng, reads_range=(10, 500), haps_range=(2, 16), long_frac=0.2,
                   long_range=(1000, 20000), short_len=150, hap_factor=(1.5, 3.0)) -> dict:
    """One serving request: an active region of R ~ U{reads_range} reads x H ~
    U{haps_range} haplotypes, scored as all R x H pairs.  With probability ``long_frac``
    every read of the region has one length drawn log-uniform in ``long_range``, else
    ``short_len``.  The reference window is U[hap_factor] x the read length; haplotypes
    are the reference with SNPs (1e-3 per base) and 1 bp indels (1e-4 per base); reads
    come from a random haplotype at a random offset with the short-read error and
    quality model (substitutions U[0.5%, 2%], then 1% N)."""
    R = int(rng.integers(reads_range[0], reads_range[1] + 1))
    H = int(rng.integers(haps_range[0], haps_range[1] + 1))
    if rng.random() < long_frac:
        rl = int(round(np.exp(rng.uniform(np.log(long_range[0]), np.log(long_range[1])))))
    else:
        rl = short_len
    wl = max(rl, int(round(rl * rng.uniform(hap_factor[0], hap_factor[1]))))
    ref = _random_bases(rng, wl)
    haps = []
    for _ in range(H):
        hap = _substitute(rng, ref, 1e-3)
        ev = np.flatnonzero(rng.random(wl) < 1e-4)
        if len(ev):
            keep = np.ones(len(hap), bool)
            ins_at, ins_b = [], []
            for p in ev:
                if rng.random() < 0.5:
                    ins_at.append(p)
                    ins_b.append(_random_bases(rng, 1)[0])
                else:
                    keep[p] = False
            hap = np.insert(hap, ins_at, ins_b) if ins_at else hap
            if not keep.all():
                keep = np.insert(keep, ins_at, True) if ins_at else keep
                hap = hap[keep]
        haps.append(hap)
    reads, quals = [], []
    src = rng.integers(0, H, size=R)
    for r in range(R):
        hap = haps[int(src[r])]
        off = int(rng.integers(0, max(len(hap) - rl, 0) + 1))
        read = _mutate(rng, hap, off, rl, float(rng.uniform(0.005, 0.02)), 0.0)
        read[rng.random(rl) < 0.01] = ord("N")
        reads.append(read)
        quals.append(_short_read_quals(rng, rl))
    pr = np.repeat(np.arange(R), H)
    ph = np.tile(np.arange(H), R)
    return _pack(reads, quals, haps, pr, ph)


def serving_requests(n: int, seed: int = 0, **kw) -> list:
    """``n`` independent region requests (see region_request), seeded."""
    rng = _rng(seed, 5)
    return [region_request(rng, **kw) for _ in range(n)]


def equal_length(n_pairs: int, length: int, seed: int = 0) -> dict:
    """Equal-length synthetic pairs (read length = haplotype length), the shape of the
    paper's scalability sweep (Section 4.3): random haplotype, read = haplotype with 1%
    substitutions; quals U{10..40}, ins/del 45, gcp 10.  Vectorised (one array draw per
    field), so a million short pairs take seconds."""
    rng = _rng(seed + 1000 * length, 6)
    n, L = int(n_pairs), int(length)
    hap = ACGT[rng.integers(0, 4, size=n * L)]
    read = hap.copy()
    m = rng.random(n * L) < 0.01
    if m.any():
        codes = np.searchsorted(ACGT, read[m])
        read[m] = ACGT[(codes + rng.integers(1, 4, size=int(m.sum()))) % 4]
    off = np.arange(n + 1, dtype=np.uint64) * np.uint64(L)
    idx = np.arange(n, dtype=np.uint32)
    return {
        "read_bases": read, "read_off": off.copy(), "hap_bases": hap, "hap_off": off.copy(),
        "pair_read": idx, "pair_hap": idx.copy(),
        "base_q": rng.integers(10, 41, size=n * L).astype(np.uint8),
        "ins_q": np.full(n * L, 45, np.uint8), "del_q": np.full(n * L, 45, np.uint8),
        "gcp_q": np.full(n * L, 10, np.uint8),
    }


def subset(b: dict, pairs) -> dict:
    """Batch restricted to the given pair indices (reads/haplotypes are shared)."""
    out = dict(b)
    pairs = np.asarray(pairs, dtype=np.int64)
    out["pair_read"] = np.ascontiguousarray(b["pair_read"][pairs])
    out["pair_hap"] = np.ascontiguousarray(b["pair_hap"][pairs])
    return out


def from_strings(pairs) -> dict:
    """Batch from explicit (read, hap, base_q, ins_q, del_q, gcp_q) tuples; qualities may
    be scalars or sequences.  Used for hand-made edge cases."""
    reads, quals, haps = [], [], []
    for (r, h, bq, iq, dq, gq) in pairs:
        r = np.frombuffer(r.encode() if isinstance(r, str) else bytes(r), np.uint8).copy()
        h = np.frombuffer(h.encode() if isinstance(h, str) else bytes(h), np.uint8).copy()
        l = len(r)
        q = tuple(np.broadcast_to(np.asarray(x, dtype=np.uint8), (l,)).copy() for x in (bq, iq, dq, gq))
        reads.append(r)
        haps.append(h)
        quals.append(q)
    idx = np.arange(len(pairs))
    return _pack(reads, quals, haps, idx, idx)
