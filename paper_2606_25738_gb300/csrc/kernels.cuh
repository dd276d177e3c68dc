// Kernels of the row-wise PairHMM library: coefficient prep, the persistent forward
// kernel, the log10 reduction / rescue selection, the FP64 rescue pass, the FP64
// launch-per-pair comparator and the scan test.  Instantiated for float in
// kernels_f32.cu and for double in kernels_f64.cu.
#pragma once

#include <cmath>
#include <cooperative_groups.h>
#include <cstdint>
#include <type_traits>

#include "engine.cuh"
#include "phmm_internal.h"

namespace phmm {

namespace cg = cooperative_groups;


// ------------------------------------------------------------------------------------
// Double-float helpers for the FP32 prep (Phred tables: see PhredTables).
// ------------------------------------------------------------------------------------
__device__ __forceinline__ df quick_two_sum(float a, float b) {
    const float s = __fadd_rn(a, b);
    return {s, __fsub_rn(b, __fsub_rn(s, a))};
}
__device__ __forceinline__ df df_mul(df a, df b) {
    const float p = __fmul_rn(a.hi, b.hi);
    float e = fmaf(a.hi, b.hi, -p);
    e = fmaf(a.hi, b.lo, e);
    e = fmaf(a.lo, b.hi, e);
    return quick_two_sum(p, e);
}
__device__ __forceinline__ df df_sub(df a, df b) {
    const df s = two_sum(a.hi, -b.hi);
    return quick_two_sum(s.hi, __fadd_rn(s.lo, __fsub_rn(a.lo, b.lo)));
}
__device__ __forceinline__ df to_df(double v) {
    const float hi = (float)v;
    return {hi, (float)(v - (double)hi)};
}

// SplitMix64 output function (Steele, Lea, Flood 2014) as a counter-based mixer.
__device__ __forceinline__ uint64_t mix64(uint64_t z) {
    z += 0x9e3779b97f4a7c15ull;
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
    return z ^ (z >> 31);
}

// Unbiased stochastic rounding of hi + lo to float: rounding errors of per-row
// coefficients then average out over long reads instead of adding up.
__device__ __forceinline__ float sround(df v, uint32_t u24) {
    if (v.lo == 0.0f || !isfinite(v.hi)) return v.hi;
    const float nb = nextafterf(v.hi, v.lo > 0.0f ? INFINITY : -INFINITY);
    const float gap = fabsf(__fsub_rn(nb, v.hi));
    const float u = (float)u24 * 0x1p-24f;
    return (__fmul_rn(u, gap) < fabsf(v.lo)) ? nb : v.hi;
}

__device__ __forceinline__ int read_code(uint32_t c) { return base_code(c); }

// Per-base record inputs with validation.  Returns META_BAD-tagged meta on bad input.
struct BaseQ {
    int code, Q, ins, del, gcp, delp, insp;  // delp / insp: previous base of the batch
    bool bad;
};
__device__ __forceinline__ BaseQ base_inputs(const BatchHeader* __restrict__ H, uint64_t b) {
    BaseQ r;
    r.code = read_code(H->read_bases[b]);
    r.Q = H->base_q[b];
    r.ins = H->ins_q[b];
    r.del = H->del_q[b];
    r.gcp = H->gcp_q[b];
    r.delp = b > 0 ? H->del_q[b - 1] : 0;
    // the batch's first base has no predecessor: take its own insertion quality (its
    // record is a row 1, whose previous-row terms are never used; this keeps the prep's
    // range statistics free of an artificial T_MI = 1)
    r.insp = b > 0 ? H->ins_q[b - 1] : H->ins_q[b];
    r.bad = r.code < 0 || r.Q > kMaxPhred || r.ins > kMaxPhred || r.del > kMaxPhred ||
            r.gcp > kMaxPhred;
    r.code = r.code < 0 ? 4 : r.code;
    r.Q = min(r.Q, kMaxPhred);
    r.ins = min(r.ins, kMaxPhred);
    r.del = min(r.del, kMaxPhred);
    r.gcp = min(r.gcp, kMaxPhred);
    r.delp = min(r.delp, kMaxPhred);
    r.insp = min(r.insp, kMaxPhred);
    return r;
}

__device__ __forceinline__ Rec32 make_rec32(const BaseQ& x, const float2* tq, const float2* tom,
                                            const float2* tq3, const float2* tinv, uint32_t seed,
                                            uint64_t b) {
    const df q_i = {tq[x.ins].x, tq[x.ins].y};
    const df q_d = {tq[x.del].x, tq[x.del].y};
    const df om_g = {tom[x.gcp].x, tom[x.gcp].y};
    const df om_Q = {tom[x.Q].x, tom[x.Q].y};
    const df q3_Q = {tq3[x.Q].x, tq3[x.Q].y};
    const df inv_g = {tinv[x.gcp].x, tinv[x.gcp].y};
    const df one = {1.0f, 0.0f};
    const df tmm = df_sub(df_sub(one, q_i), q_d);  // T_MM = 1 - T_MI - T_MD
    const uint64_t h = mix64(((uint64_t)seed << 40) ^ (b * 4u));
    Rec32 r;
    r.pm = sround(df_mul(om_Q, om_g), (uint32_t)(h & 0xffffffu));          // (1-e)(1-g)
    r.px = sround(df_mul(q3_Q, om_g), (uint32_t)((h >> 24) & 0xffffffu));  // e/3 (1-g)
    r.a = sround(df_mul(tmm, inv_g), (uint32_t)((h >> 40) & 0xffffffu));   // T_MM/(1-g)
    r.b = tq[x.delp].x;                                                      // T_MD of the previous row
    r.mi = q_i.hi;
    r.g = tq[x.gcp].x;
    r.gm = om_g.hi;
    uint32_t meta = (uint32_t)x.code | ((uint32_t)x.gcp << META_GCP_SHIFT);
    if (x.bad) meta |= META_BAD;
    if (!(om_g.hi >= 0x1p-20f) || !isfinite(r.a)) meta |= META_DEGEN;
    r.meta = meta;
    return r;
}

// Record of the pipelined FP32 engine (see Rec32J).  first: row 1 of a read, where the
// previous row's T_MI is taken as 1.  All products in double-float, then stochastically
// rounded to FP32 (unbiased, so per-row rounding errors do not add up to a drift over
// long reads with constant qualities).
__device__ __forceinline__ Rec32J make_rec32j(const BaseQ& x, const float2* tq, const float2* tom,
                                              const float2* tq3, const float2* tinv, const float2* tiq,
                                              uint32_t seed, uint64_t b, bool first) {
    const df one = {1.0f, 0.0f};
    const df q_i = {tq[x.ins].x, tq[x.ins].y};
    const df q_d = {tq[x.del].x, tq[x.del].y};
    const df q_g = {tq[x.gcp].x, tq[x.gcp].y};
    const df om_g = {tom[x.gcp].x, tom[x.gcp].y};
    const df om_Q = {tom[x.Q].x, tom[x.Q].y};
    const df q3_Q = {tq3[x.Q].x, tq3[x.Q].y};
    const df inv_g = {tinv[x.gcp].x, tinv[x.gcp].y};
    const df iq_i = {tiq[x.ins].x, tiq[x.ins].y};
    const df q_dp = {tq[x.delp].x, tq[x.delp].y};
    const df mi_p = first ? one : df{tq[x.insp].x, tq[x.insp].y};    // mi_{i-1}
    const df imi_p = first ? one : df{tiq[x.insp].x, tiq[x.insp].y}; // 1 / mi_{i-1}
    const df tmm = df_sub(df_sub(one, q_i), q_d);
    const uint64_t h1 = mix64(((uint64_t)seed << 40) ^ (b * 4u + 1u));
    const uint64_t h2 = mix64(((uint64_t)seed << 40) ^ (b * 4u + 2u));
    Rec32J r;
    r.pm = sround(df_mul(df_mul(om_Q, om_g), mi_p), (uint32_t)(h1 & 0xffffffu));
    r.px = sround(df_mul(df_mul(q3_Q, om_g), mi_p), (uint32_t)((h1 >> 24) & 0xffffffu));
    r.a = sround(df_mul(df_mul(tmm, inv_g), imi_p), (uint32_t)((h1 >> 40) & 0xffffffu));
    r.b = sround(df_mul(q_dp, imi_p), (uint32_t)(h2 & 0xffffffu));
    r.h = sround(df_mul(df_mul(q_g, mi_p), iq_i), (uint32_t)((h2 >> 24) & 0xffffffu));
    r.g = q_g.hi;
    r.mi = q_i.hi;
    uint32_t meta = (uint32_t)x.code | ((uint32_t)x.gcp << META_GCP_SHIFT);
    if (x.bad) meta |= META_BAD;
    if (!(om_g.hi >= 0x1p-20f) || !isfinite(r.a) || !isfinite(r.b) || !isfinite(r.h)) meta |= META_DEGEN;
    r.meta = meta;
    return r;
}

__device__ __forceinline__ Rec64 make_rec64(const BaseQ& x, const PhredTables& T) {
    Rec64 r;
    r.pm = T.om[x.Q];
    r.px = T.q3[x.Q];
    r.a = 1.0 - T.q[x.ins] - T.q[x.del];
    r.b = T.q[x.delp];
    r.mi = T.q[x.ins];
    r.g = T.q[x.gcp];
    r.gm = T.om[x.gcp];
    uint64_t meta = (uint64_t)x.code | ((uint64_t)x.gcp << META_GCP_SHIFT);
    if (x.bad) meta |= META_BAD;
    r.meta = meta;
    return r;
}

// Record of the FP64 pipelined engine (see Rec64J), in plain double arithmetic.  first:
// row 1 of a read, where the previous row's T_MI is taken as 1.
__device__ __forceinline__ Rec64J make_rec64j(const BaseQ& x, const PhredTables& T, bool first) {
    const double mi_p = first ? 1.0 : T.q[x.insp], imi_p = first ? 1.0 : T.iq[x.insp];
    const double om_g = T.om[x.gcp];
    Rec64J r;
    r.pm = T.om[x.Q] * om_g * mi_p;
    r.px = T.q3[x.Q] * om_g * mi_p;
    r.a = (1.0 - T.q[x.ins] - T.q[x.del]) * T.inv[x.gcp] * imi_p;
    r.b = T.q[x.delp] * imi_p;
    r.h = T.q[x.gcp] * mi_p * T.iq[x.ins];
    r.g = T.q[x.gcp];
    r.mi = T.q[x.ins];
    uint64_t meta = (uint64_t)x.code | ((uint64_t)x.gcp << META_GCP_SHIFT);
    if (x.bad) meta |= META_BAD;
    if (!(om_g >= 0x1p-40) || !isfinite(r.a) || !isfinite(r.b) || !isfinite(r.h)) meta |= META_DEGEN;
    r.meta = meta;
    return r;
}

// Worst per-row drop and growth of the row max in bits (see checkpoint_interval):
// the max can fall by at most min(T_MI, g) per row and grow by at most
// max(|T_MM| + (1-g) + T_MD, T_MI + g).
__device__ __forceinline__ void drop_grow(const BaseQ& x, const PhredTables& T, uint32_t& d,
                                          uint32_t& g) {
    const float qi = (float)T.q[x.ins], qd = (float)T.q[x.del], qg = (float)T.q[x.gcp];
    const float drop = -log2f(fminf(qi, qg));
    const float tmm = fabsf(1.0f - qi - qd);
    const float grow = log2f(fmaxf(tmm + (1.0f - qg) + qd, qi + qg));
    d = (uint32_t)ceilf(fmaxf(drop, 0.0f) * 64.0f) + 1u;
    g = (uint32_t)ceilf(fmaxf(grow, 0.0f) * 64.0f) + 1u;
}

__device__ __forceinline__ void block_max2(uint32_t d, uint32_t g, uint32_t* out) {
    __shared__ uint32_t sd[32], sg[32];
    d = __reduce_max_sync(kFull, d);
    g = __reduce_max_sync(kFull, g);
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0) { sd[w] = d; sg[w] = g; }
    __syncthreads();
    if (w == 0) {
        const int nw = (blockDim.x + 31) >> 5;
        d = lane < nw ? sd[lane] : 0u;
        g = lane < nw ? sg[lane] : 0u;
        d = __reduce_max_sync(kFull, d);
        g = __reduce_max_sync(kFull, g);
        if (lane == 0) {
            atomicMax(out, d);
            atomicMax(out + 1, g);
        }
    }
}

__device__ __forceinline__ void load_tables(const PhredTables* __restrict__ G, PhredTables& S) {
    for (int i = threadIdx.x; i < kPhredTab; i += blockDim.x) {
        S.q[i] = G->q[i];
        S.om[i] = G->om[i];
        S.q3[i] = G->q3[i];
        S.inv[i] = G->inv[i];
        S.iq[i] = G->iq[i];
    }
}

// Pair descriptors (grid-stride): desc[p] = offsets and lengths of pair p.
__device__ __forceinline__ void build_desc(const BatchHeader* __restrict__ H) {
    const uint32_t n = H->n_pairs;
    for (uint32_t p = blockIdx.x * blockDim.x + threadIdx.x; p < n; p += gridDim.x * blockDim.x) {
        const uint32_t r = H->pair_read[p], h = H->pair_hap[p];
        PairDesc d;
        d.roff = H->read_off[r];
        d.hoff = H->hap_off[h];
        d.l = (uint32_t)(H->read_off[r + 1] - d.roff);
        d.k = (uint32_t)(H->hap_off[h + 1] - d.hoff);
        H->desc[p] = d;
    }
}

// ------------------------------------------------------------------------------------
// Forward kernel pieces
// ------------------------------------------------------------------------------------
template <typename T>
__device__ __forceinline__ const typename Num<T>::Rec* recs_of(const BatchHeader* H);
template <>
__device__ __forceinline__ const Rec32* recs_of<float>(const BatchHeader* H) { return H->rec32; }
template <>
__device__ __forceinline__ const Rec64* recs_of<double>(const BatchHeader* H) { return H->rec64; }

template <typename T>
struct CtaShared {
    unsigned long long ring[kCtaWarps * kRing * Num<T>::kWords];
    int cons[kCtaWarps + 1];
    SegOut out[kCtaWarps];
    uint32_t item;
};

template <typename T>
__device__ __forceinline__ void cta_clear(CtaShared<T>& sh) {
    constexpr int n = kCtaWarps * kRing * Num<T>::kWords;
    for (int q = threadIdx.x; q < n; q += blockDim.x) sh.ring[q] = 0ull;
    if (threadIdx.x <= kCtaWarps) sh.cons[threadIdx.x] = 0;
}

// Warps w0 .. w0+W-1 of the CTA run one strip of a pair: segment (warp) s covers
// columns col0 + s * 32 N .. + 32 N - 1.  Neighbouring warps link through the CTA's
// shared-memory rings; the strip's first / last warp links to the previous / next strip
// through global boundaries bnd_in / bnd_out (null: none).
template <typename T, int N>
__device__ __forceinline__ void cta_strip_run(const BatchHeader* __restrict__ H,
                                              const PowRow<T>* __restrict__ pow, uint32_t pair,
                                              int w0, int W, uint32_t col0, unsigned long long* bnd_in,
                                              unsigned long long* bnd_out, CtaShared<T>& sh, int R) {
    constexpr int KW = Num<T>::kWords;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int s = warp - w0;
    if (s < 0 || s >= W) return;
    const PairDesc d = H->desc[pair];
    SmemLink L;
    L.in_ring = sh.ring + warp * kRing * KW;
    L.out_ring = sh.ring + min(warp + 1, kCtaWarps - 1) * kRing * KW;
    L.my_cons = sh.cons + warp;
    L.next_cons = sh.cons + warp + 1;
    L.in_g = (s == 0) ? bnd_in : nullptr;
    L.out_g = (s == W - 1) ? bnd_out : nullptr;
    L.has_left = s > 0 || bnd_in != nullptr;
    L.has_right = s < W - 1 || bnd_out != nullptr;
    const int c0 = (int)col0 + (s * 32 + lane) * N;
    const SegOut o = seg_run<T, N, true>(recs_of<T>(H) + d.roff, (int)d.l, (int)d.l,
                                         H->hap_bases + d.hoff, (int)d.k, c0, lane, 31, 5,
                                         pow, R, L, H->status);
    if (lane == 0) sh.out[warp] = o;
}

// Combine the W segment partials of one pair: L * C = sum_s S_s 2^(E_s).
template <typename T>
__device__ __forceinline__ Partial cta_combine(const CtaShared<T>& sh, int w0, int W) {
    int Eref = INT_MIN;
    uint32_t f = 0;
    for (int w = w0; w < w0 + W; ++w) {
        f |= sh.out[w].flags;
        if (sh.out[w].S != 0.0) Eref = max(Eref, sh.out[w].E);
    }
    double S = 0.0;
    if (Eref == INT_MIN) Eref = sh.out[w0].E;
    else
        for (int w = w0; w < w0 + W; ++w)
            if (sh.out[w].S != 0.0) S += ldexp(sh.out[w].S, sh.out[w].E - Eref);
    Partial p;
    p.S = S;
    p.E = Eref;
    p.flags = f | PF_DONE;
    p.n_extra = 0;
    p.extra_base = 0;
    return p;
}

// Partial slot of a strip: strip 0 at the pair's slot (carrying where the other strips'
// partials live), strip s >= 1 at extra_base + s - 1.
__device__ __forceinline__ void write_strip_part(const BatchHeader* __restrict__ H, uint32_t pair,
                                                 uint32_t strip, uint32_t nstrip, uint32_t extra_base,
                                                 Partial p) {
    if (strip == 0) {
        p.n_extra = nstrip - 1;
        p.extra_base = extra_base;
        H->parts[pair] = p;
    } else {
        p.n_extra = 0;
        p.extra_base = 0;
        H->parts[extra_base + strip - 1] = p;
    }
}

// A whole pair on this CTA, strip after strip (rescue pass, launch-per-pair comparator):
// strip s reads boundary (s-1)&1 and writes boundary s&1 of this CTA's two scratch
// boundaries; each strip finishes before the next starts.  Returns the combined partial
// in thread 0.
template <typename T, int N>
__device__ Partial cta_pair_sequential(const BatchHeader* __restrict__ H, const PowRow<T>* __restrict__ pow,
                                       uint32_t pair, CtaShared<T>& sh, int R, unsigned long long* scratch,
                                       uint64_t half_words) {
    const PairDesc d = H->desc[pair];
    const uint32_t seg = 32u * N;
    const uint32_t Wt = (d.k + seg - 1) / seg;
    const uint32_t S = (Wt + kCtaWarps - 1) / kCtaWarps;
    int Eref = INT_MIN;
    double Sum = 0.0;
    uint32_t fl = 0;
    for (uint32_t st = 0; st < S; ++st) {
        const int W = (int)min((uint32_t)kCtaWarps, Wt - st * kCtaWarps);
        cta_clear<T>(sh);
        __syncthreads();
        unsigned long long* bin = st > 0 ? scratch + ((st - 1) & 1) * half_words : nullptr;
        unsigned long long* bout = st + 1 < S ? scratch + (st & 1) * half_words : nullptr;
        cta_strip_run<T, N>(H, pow, pair, 0, W, st * kCtaWarps * seg, bin, bout, sh, R);
        __syncthreads();
        if (threadIdx.x == 0) {
            const Partial q = cta_combine<T>(sh, 0, W);
            fl |= q.flags;
            if (q.S != 0.0) {
                if (Eref == INT_MIN) {
                    Eref = q.E;
                    Sum = q.S;
                } else if (q.E > Eref) {
                    Sum = ldexp(Sum, Eref - q.E) + q.S;
                    Eref = q.E;
                } else {
                    Sum += ldexp(q.S, q.E - Eref);
                }
            }
        }
        __syncthreads();
    }
    Partial r;
    r.S = Sum;
    r.E = Eref == INT_MIN ? 0 : Eref;
    r.flags = fl | PF_DONE;
    r.n_extra = 0;
    r.extra_base = 0;
    return r;
}

template <typename T>
__device__ const typename Num<T>::Rec* dummy_rec();

// One warp item.  FP64: scalar teams of seg_run.  FP32 (k_forward_short): kind 0 = lean
// scalar teams (width NS), kind 1 = packed teams of two haplotypes of the same read
// (width NP).
template <typename T, int N>
__device__ __forceinline__ void warp_item_run(const BatchHeader* __restrict__ H,
                                              const PowRow<T>* __restrict__ pow, uint32_t wi,
                                              int R) {
    using Rec = typename Num<T>::Rec;
    const int lane = threadIdx.x & 31;
    const WarpItem it = H->witems[wi];
    int tbase = lane, tsize = 1, maxG = 1;
    uint32_t pair = kNoPair;
    for (uint32_t t = 0; t < it.n_teams; ++t) {
        const Team tm = H->teams[it.first_team + t];
        maxG = max(maxG, (int)tm.size);
        if (lane >= tm.base && lane < tm.base + tm.size) {
            tbase = tm.base;
            tsize = tm.size;
            pair = tm.pair;
        }
    }
    int nsteps = 0;
    while ((1 << nsteps) < maxG) ++nsteps;
    const int lt = lane - tbase, tlast = tbase + tsize - 1;
    int l = 0, k = 0;
    const Rec* rec = dummy_rec<T>();
    const uint8_t* hap = H->hap_bases;
    if (pair != kNoPair) {
        const PairDesc d = H->desc[pair];
        l = (int)d.l;
        k = (int)d.k;
        rec = recs_of<T>(H) + d.roff;
        hap = H->hap_bases + d.hoff;
    }
    const int lmax = (int)__reduce_max_sync(kFull, (unsigned)l);
    SmemLink L{};
    const SegOut o = seg_run<T, N, false>(rec, l, lmax, hap, k, lt * N, lt, tlast, nsteps, pow, R,
                                          L, H->status);
    if (pair != kNoPair && lt == 0) {
        Partial p;
        p.S = o.S;
        p.E = o.E;
        p.flags = o.flags | PF_DONE;
        p.n_extra = 0;
        p.extra_base = 0;
        H->parts[pair] = p;
    }
}

__device__ __forceinline__ void write_part(const BatchHeader* __restrict__ H, uint32_t pair,
                                           const SegOut& o) {
    Partial p;
    p.S = o.S;
    p.E = o.E;
    p.flags = o.flags | PF_DONE;
    p.n_extra = 0;
    p.extra_base = 0;
    H->parts[pair] = p;
}

// Persistent forward kernel for multi-warp pairs: CTA items (longest first) taken from
// an atomic counter; with WARP_ITEMS it then also takes warp items (the FP64 engine, which
// has no packed short kernel).
template <typename T, int N, bool WARP_ITEMS, int CW = kCtaWarps>
__global__ void __launch_bounds__(CW * 32, 1)
k_forward(const BatchHeader* __restrict__ H, const PowRow<T>* __restrict__ pow) {
    __shared__ CtaShared<T> sh;
    const int R = checkpoint_interval<T>(H->dropgrow);
    const uint32_t n_c = H->n_citems;
    for (;;) {
        if (threadIdx.x == 0) sh.item = atomicAdd(&H->counters[0], 1u);
        cta_clear<T>(sh);
        __syncthreads();
        const uint32_t it = sh.item;
        if (it >= n_c) break;
        const CtaItem ci = H->citems[it];
        const int warp = threadIdx.x >> 5;
        for (uint32_t q = 0; q < ci.n; ++q) {
            const CtaPair cp = H->cpairs[ci.first + q];
            if (warp >= cp.w0 && warp < cp.w0 + cp.W)
                cta_strip_run<T, N>(H, pow, cp.pair, cp.w0, cp.W, cp.col0,
                                    cp.bnd_in == kNoBnd ? nullptr : H->bnd + cp.bnd_in,
                                    cp.bnd_out == kNoBnd ? nullptr : H->bnd + cp.bnd_out, sh, R);
        }
        __syncthreads();
        if ((threadIdx.x & 31) == 0) {
            for (uint32_t q = 0; q < ci.n; ++q) {
                const CtaPair cp = H->cpairs[ci.first + q];
                if (warp == cp.w0)
                    write_strip_part(H, cp.pair, cp.strip, cp.nstrip, cp.extra_base,
                                     cta_combine<T>(sh, cp.w0, cp.W));
            }
        }
        __syncthreads();
    }
    if constexpr (WARP_ITEMS) {
        const uint32_t n_w = H->n_witems;
        const int lane = threadIdx.x & 31;
        for (;;) {
            uint32_t wi = 0;
            if (lane == 0) wi = atomicAdd(&H->counters[1], 1u);
            wi = __shfl_sync(kFull, wi, 0);
            if (wi >= n_w) break;
            warp_item_run<T, N>(H, pow, wi, R);
        }
    }
}

// Multi-warp FP32 pairs on the pipelined engine: one warp per 32 N-column segment, up to
// kCtaWarpsPipe warps per CTA item (register budget of the engine), strips beyond that.
template <int N>
__device__ __forceinline__ void cta_strip_run_pipe(const BatchHeader* __restrict__ H,
                                                   const PowRow<float>* __restrict__ pow, uint32_t pair,
                                                   int w0, int W, uint32_t col0, unsigned long long* bnd_in,
                                                   unsigned long long* bnd_out, CtaShared<float>& sh,
                                                   const PipeRange& rng) {
    constexpr int KW = Num<float>::kWords;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int s = warp - w0;
    if (s < 0 || s >= W) return;
    const PairDesc d = H->desc[pair];
    SmemLink L;
    L.in_ring = sh.ring + warp * kRing * KW;
    L.out_ring = sh.ring + min(warp + 1, kCtaWarps - 1) * kRing * KW;
    L.my_cons = sh.cons + warp;
    L.next_cons = sh.cons + warp + 1;
    L.in_g = (s == 0) ? bnd_in : nullptr;
    L.out_g = (s == W - 1) ? bnd_out : nullptr;
    L.has_left = s > 0 || bnd_in != nullptr;
    L.has_right = s < W - 1 || bnd_out != nullptr;
    const int c0 = (int)col0 + (s * 32 + lane) * N;
    const SegOut o = seg_link_pipe<N>(H->rec32j + d.roff, (int)d.l, H->hap_bases + d.hoff, (int)d.k, c0,
                                      lane, pow, rng, L, H->status);
    if (lane == 0) sh.out[warp] = o;
}

constexpr int kCtaThreadsPipe = kCtaWarpsPipe * 32;

// CW warps per CTA: 12 at N = 32 (168 registers), 16 at N = 24 (128 registers), or 4 at
// N = 32 with three CTAs per SM: a very wide pair then spreads over many SMs, one warp per
// scheduler, instead of filling a few.
template <int N, int CW>
__global__ void __launch_bounds__(CW * 32, CW <= 4 ? 3 : 1)
k_forward_pipe(const BatchHeader* __restrict__ H, const PowRow<float>* __restrict__ pow) {
    __shared__ CtaShared<float> sh;
    const PipeRange rng = pipe_range(H->dropgrow);
    const uint32_t n_c = H->n_citems;
    for (;;) {
        if (threadIdx.x == 0) sh.item = atomicAdd(&H->counters[0], 1u);
        cta_clear<float>(sh);
        __syncthreads();
        const uint32_t it = sh.item;
        if (it >= n_c) break;
        const CtaItem ci = H->citems[it];
        const int warp = threadIdx.x >> 5;
        for (uint32_t q = 0; q < ci.n; ++q) {
            const CtaPair cp = H->cpairs[ci.first + q];
            if (warp >= cp.w0 && warp < cp.w0 + cp.W)
                cta_strip_run_pipe<N>(H, pow, cp.pair, cp.w0, cp.W, cp.col0,
                                      cp.bnd_in == kNoBnd ? nullptr : H->bnd + cp.bnd_in,
                                      cp.bnd_out == kNoBnd ? nullptr : H->bnd + cp.bnd_out, sh, rng);
        }
        __syncthreads();
        if ((threadIdx.x & 31) == 0) {
            for (uint32_t q = 0; q < ci.n; ++q) {
                const CtaPair cp = H->cpairs[ci.first + q];
                if (warp == cp.w0)
                    write_strip_part(H, cp.pair, cp.strip, cp.nstrip, cp.extra_base,
                                     cta_combine<float>(sh, cp.w0, cp.W));
            }
        }
        __syncthreads();
    }
}

// Multi-warp FP32 pairs in thread-block clusters (long kind 5): the plan's CTA items (as
// for 4-warp CTAs: strips of 4096 columns) are taken CS at a time by a cluster of CS CTAs,
// CTA rank r running item CS g + r.  Where consecutive strips of a pair sit in
// neighbouring ranks, the left strip's last warp writes each row's boundary values (M, J,
// D-hat and exponent of its last column) straight into the right strip's first-warp ring
// in the other CTA's shared memory (distributed shared memory, the paper's multi-CTA
// design); other strip boundaries go through global memory as for k_forward_pipe.
template <int N>
__device__ __forceinline__ void cta_strip_run_cluster(const BatchHeader* __restrict__ H,
                                                      const PowRow<float>* __restrict__ pow, const CtaPair& cp,
                                                      CtaShared<float>& sh, const PipeRange& rng, unsigned rank) {
    constexpr int KW = Num<float>::kWords;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int s = warp - cp.w0;
    if (s < 0 || s >= cp.W) return;
    const PairDesc d = H->desc[cp.pair];
    const bool din = is_dsmem_bnd(cp.bnd_in), dout = is_dsmem_bnd(cp.bnd_out);
    SmemLink L;
    L.in_ring = sh.ring + warp * kRing * KW;
    L.out_ring = sh.ring + min(warp + 1, kCtaWarps - 1) * kRing * KW;
    L.my_cons = sh.cons + warp;
    L.next_cons = sh.cons + warp + 1;
    if (s == cp.W - 1 && dout) {
        // the receiving strip's first warp w1 in the next CTA of the cluster
        const int w1 = (int)(cp.bnd_out & 0xffu);
        cg::cluster_group cl = cg::this_cluster();
        L.out_ring = cl.map_shared_rank(sh.ring + w1 * kRing * KW, rank + 1);
        L.next_cons = cl.map_shared_rank(sh.cons + w1, rank + 1);
    }
    L.in_g = (s == 0 && cp.bnd_in != kNoBnd && !din) ? H->bnd + cp.bnd_in : nullptr;
    L.out_g = (s == cp.W - 1 && cp.bnd_out != kNoBnd && !dout) ? H->bnd + cp.bnd_out : nullptr;
    L.has_left = s > 0 || cp.bnd_in != kNoBnd;
    L.has_right = s < cp.W - 1 || cp.bnd_out != kNoBnd;
    const int c0 = (int)cp.col0 + (s * 32 + lane) * N;
    const SegOut o = seg_link_pipe<N>(H->rec32j + d.roff, (int)d.l, H->hap_bases + d.hoff, (int)d.k, c0,
                                      lane, pow, rng, L, H->status);
    if (lane == 0) sh.out[warp] = o;
}

template <int N, int CW, int CS>
__global__ void __cluster_dims__(CS, 1, 1) __launch_bounds__(CW * 32, 3)
k_forward_cluster(const BatchHeader* __restrict__ H, const PowRow<float>* __restrict__ pow) {
    __shared__ CtaShared<float> sh;
    cg::cluster_group cl = cg::this_cluster();
    const unsigned rank = cl.block_rank();
    const PipeRange rng = pipe_range(H->dropgrow);
    const uint32_t n_c = H->n_citems;
    const uint32_t n_g = (n_c + CS - 1) / CS;
    const int warp = threadIdx.x >> 5;
    cl.sync();  // every CTA of the cluster runs before any shared memory of another is touched
    for (;;) {
        if (rank == 0 && threadIdx.x == 0) {
            const uint32_t g = atomicAdd(&H->counters[5], 1u);
            for (unsigned r = 0; r < CS; ++r) *cl.map_shared_rank(&sh.item, r) = g;
        }
        cta_clear<float>(sh);
        cl.sync();  // the group index is everywhere; every ring is clear before a neighbour writes
        const uint32_t g = sh.item;
        if (g >= n_g) break;
        const uint32_t it = g * CS + rank;
        CtaItem ci;
        ci.first = 0;
        ci.n = 0;
        if (it < n_c) ci = H->citems[it];
        for (uint32_t q = 0; q < ci.n; ++q) {
            const CtaPair cp = H->cpairs[ci.first + q];
            if (warp >= cp.w0 && warp < cp.w0 + cp.W) cta_strip_run_cluster<N>(H, pow, cp, sh, rng, rank);
        }
        __syncthreads();
        if ((threadIdx.x & 31) == 0) {
            for (uint32_t q = 0; q < ci.n; ++q) {
                const CtaPair cp = H->cpairs[ci.first + q];
                if (warp == cp.w0)
                    write_strip_part(H, cp.pair, cp.strip, cp.nstrip, cp.extra_base,
                                     cta_combine<float>(sh, cp.w0, cp.W));
            }
        }
        cl.sync();  // no CTA clears its rings for the next group while a neighbour still writes
    }
}

// Multi-warp pairs one warp at a time (long kind 3): each warp takes a whole pair and
// runs its strips of 32 N columns one after another (team_run_pipe2 in LINK mode), strip s
// reading the boundary strip s - 1 left in this warp's scratch.  No warp ever waits on
// another; the pair's S strips leave S partials, combined by the finalize kernel as for
// CTA strips.
template <int N, int MINB, bool L1P = false>
__global__ void __launch_bounds__(128, MINB)
k_forward_serial(const BatchHeader* __restrict__ H, const PowRow<float>* __restrict__ pow) {
    __shared__ float4 stage[4][64];    // per warp: two blocks of 32 left-boundary rows
    __shared__ float4 rstage[4][128];  // per warp: two blocks of 32 records (32 B each)
    const PipeRange rng = pipe_range(H->dropgrow);
    const uint32_t n_c = H->n_citems;
    const int lane = threadIdx.x & 31;
    const uint32_t gw = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (gw >= H->sbnd_warps) return;  // no scratch for this warp (grid larger than planned)
    float4* buf0 = H->sbnd + (size_t)gw * 2 * H->sbnd_rows;
    float4* buf1 = buf0 + H->sbnd_rows;
    for (;;) {
        uint32_t wi = 0;
        if (lane == 0) wi = atomicAdd(&H->counters[0], 1u);
        wi = __shfl_sync(kFull, wi, 0);
        if (wi >= n_c) break;
        const CtaPair cp = H->cpairs[H->citems[wi].first];
        const PairDesc d = H->desc[cp.pair];
        const uint32_t S = cp.nstrip;
        for (uint32_t s = 0; s < S; ++s) {
            const float4* in = (s & 1u) ? buf0 : buf1;  // what strip s - 1 wrote
            float4* outb = (s & 1u) ? buf1 : buf0;
            const int c0 = (int)(s * 32u * N) + lane * N;
            const SegOut o = team_run_pipe2<N, true, true, true, L1P>(H->rec32j + d.roff, (int)d.l, (int)d.l,
                                                           H->hap_bases + d.hoff, (int)d.k, c0, lane, 31, 5,
                                                           pow, rng, in, outb, s > 0, s + 1 < S,
                                                           stage[threadIdx.x >> 5], rstage[threadIdx.x >> 5]);
            __syncwarp();  // this strip's boundary stores before the next strip's loads
            if (lane == 0) {
                Partial p;
                p.S = o.S;
                p.E = o.E;
                p.flags = o.flags | PF_DONE;
                write_strip_part(H, cp.pair, s, S, cp.extra_base, p);
            }
        }
    }
}

// Wave multi-warp kind (long kind 6): every 1024-column strip of a wide pair is its own
// item, on its own warp, and the strips of a pair run at the same time.  Strip s stores its
// right boundary row by row (float4: M, J, D-hat, E of its last column) at wbnd + bnd_out
// and releases its progress (rows stored) in boundary word `pad` at every 32nd row and the
// last; strip s + 1 acquires that word before it copies the next 32 rows of the boundary
// (team_run_pipe2<..., WAVE>), so the strips hand over once per 32 rows.  Items are taken
// in order and a pair's strips are consecutive: a strip only waits for a strip that some
// warp already runs, so every wait ends (and each one is bounded).
template <int N, int MINB>
__global__ void __launch_bounds__(128, MINB)
k_forward_wave(const BatchHeader* __restrict__ H, const PowRow<float>* __restrict__ pow) {
    __shared__ float4 stage[4][64];    // per warp: two blocks of 32 left-boundary rows
    __shared__ float4 rstage[4][128];  // per warp: two blocks of 32 records (32 B each)
    const PipeRange rng = pipe_range(H->dropgrow);
    const uint32_t n_c = H->n_citems;
    const int lane = threadIdx.x & 31;
    for (;;) {
        uint32_t wi = 0;
        if (lane == 0) wi = atomicAdd(&H->counters[0], 1u);
        wi = __shfl_sync(kFull, wi, 0);
        if (wi >= n_c) break;
        const CtaPair cp = H->cpairs[H->citems[wi].first];
        const PairDesc d = H->desc[cp.pair];
        const uint32_t s = cp.strip, S = cp.nstrip;
        const bool has_left = s > 0, has_right = s + 1 < S;
        const float4* in = has_left ? H->wbnd + cp.bnd_in : nullptr;
        float4* outb = has_right ? H->wbnd + cp.bnd_out : nullptr;
        const unsigned long long* pl = has_left ? H->bnd + (cp.pad - 1) : nullptr;
        unsigned long long* pm = has_right ? H->bnd + cp.pad : nullptr;
        const int c0 = (int)cp.col0 + lane * N;
        const SegOut o = team_run_pipe2<N, true, true, true, false, true>(
            H->rec32j + d.roff, (int)d.l, (int)d.l, H->hap_bases + d.hoff, (int)d.k, c0, lane, 31, 5, pow, rng,
            in, outb, has_left, has_right, stage[threadIdx.x >> 5], rstage[threadIdx.x >> 5], pl, pm, H->status);
        __syncwarp();
        if (lane == 0) {
            Partial p;
            p.S = o.S;
            p.E = o.E;
            p.flags = o.flags | PF_DONE;
            write_strip_part(H, cp.pair, s, S, cp.extra_base, p);
        }
    }
}

// Team lookup of a warp item: this lane's team (first lane, size, pairs) and the scan
// steps of the widest team.
struct TeamOf {
    int lt, tlast, nsteps;
    uint32_t pair, pair2;
};
__device__ __forceinline__ TeamOf team_of(const Team* __restrict__ teams, const WarpItem& it) {
    const int lane = threadIdx.x & 31;
    int tbase = lane, tsize = 1, maxG = 1;
    uint32_t pair = kNoPair, pair2 = kNoPair;
    for (uint32_t t = 0; t < it.n_teams; ++t) {
        const Team tm = teams[it.first_team + t];
        maxG = max(maxG, (int)tm.size);
        if (lane >= tm.base && lane < tm.base + tm.size) {
            tbase = tm.base;
            tsize = tm.size;
            pair = tm.pair;
            pair2 = tm.pair2;
        }
    }
    int nsteps = 0;
    while ((1 << nsteps) < maxG) ++nsteps;
    return {lane - tbase, tbase + tsize - 1, nsteps, pair, pair2};
}

// Persistent kernels for short pairs in FP32 (warp items taken from atomic counters).
// Small CTAs: residency is set by registers, not by a CTA-wide shape.
constexpr int kShortThreads = 128;

// Lean scalar teams, N columns per lane (item list witems / counters[1]); MINB resident
// CTAs per SM bound the registers per thread.
template <int N, int MINB>
__global__ void __launch_bounds__(kShortThreads, MINB)
k_short_scalar(const BatchHeader* __restrict__ H, const PowRow<float>* __restrict__ pow) {
    const int R = checkpoint_interval<float>(H->dropgrow);
    const uint32_t n_w = H->n_witems;
    const int lane = threadIdx.x & 31;
    for (;;) {
        uint32_t wi = 0;
        if (lane == 0) wi = atomicAdd(&H->counters[1], 1u);
        wi = __shfl_sync(kFull, wi, 0);
        if (wi >= n_w) break;
        const TeamOf t = team_of(H->teams, H->witems[wi]);
        int l = 0, k = 0;
        const Rec32* rec = dummy_rec<float>();
        const uint8_t* hap = H->hap_bases;
        if (t.pair != kNoPair) {
            const PairDesc d = H->desc[t.pair];
            l = (int)d.l;
            k = (int)d.k;
            rec = H->rec32 + d.roff;
            hap = H->hap_bases + d.hoff;
        }
        const int lmax = (int)__reduce_max_sync(kFull, (unsigned)l);
        const SegOut o = team_run_lean<N>(rec, l, lmax, hap, k, t.lt * N, t.lt, t.tlast, t.nsteps, pow, R);
        if (t.pair != kNoPair && t.lt == 0) write_part(H, t.pair, o);
    }
}

// Pipelined scalar teams (team_run_pipe, Rec32J records), same work list as
// k_short_scalar.
template <int N, int MINB>
__global__ void __launch_bounds__(kShortThreads, MINB)
k_short_pipe(const BatchHeader* __restrict__ H, const PowRow<float>* __restrict__ pow) {
    const PipeRange rng = pipe_range(H->dropgrow);
    const uint32_t n_w = H->n_witems;
    const int lane = threadIdx.x & 31;
    for (;;) {
        uint32_t wi = 0;
        if (lane == 0) wi = atomicAdd(&H->counters[1], 1u);
        wi = __shfl_sync(kFull, wi, 0);
        if (wi >= n_w) break;
        const TeamOf t = team_of(H->teams, H->witems[wi]);
        int l = 0, k = 0;
        const Rec32J* rec = reinterpret_cast<const Rec32J*>(dummy_rec<float>());
        const uint8_t* hap = H->hap_bases;
        if (t.pair != kNoPair) {
            const PairDesc d = H->desc[t.pair];
            l = (int)d.l;
            k = (int)d.k;
            rec = H->rec32j + d.roff;
            hap = H->hap_bases + d.hoff;
        }
        const int lmax = (int)__reduce_max_sync(kFull, (unsigned)l);
        const SegOut o = team_run_pipe<N>(rec, l, lmax, hap, k, t.lt * N, t.lt, t.tlast, t.nsteps, pow, rng);
        if (t.pair != kNoPair && t.lt == 0) write_part(H, t.pair, o);
    }
}

// FP64 mode, pipelined variant: short pairs on the pipelined engine in FP64
// (team_run_pipe<N, double>, Rec64J records), same work list as k_short_scalar; the
// multi-warp pairs run on k_forward<double> (CTA items) on the other branch.  A pair with a
// degenerate row (1 - g = 0) or a range the engine cannot hold is flagged and goes to the
// unfactored FP64 pass.
template <int N, int MINB, bool FUSE = false>
__global__ void __launch_bounds__(kShortThreads, MINB)
k_short_pipe64(const BatchHeader* __restrict__ H, const PowRow<double>* __restrict__ pow) {
    const PipeRange rng = pipe_range<double>(H->dropgrow);
    const uint32_t n_w = H->n_witems;
    const int lane = threadIdx.x & 31;
    for (;;) {
        uint32_t wi = 0;
        if (lane == 0) wi = atomicAdd(&H->counters[1], 1u);
        wi = __shfl_sync(kFull, wi, 0);
        if (wi >= n_w) break;
        const TeamOf t = team_of(H->teams, H->witems[wi]);
        int l = 0, k = 0;
        const Rec64J* rec = reinterpret_cast<const Rec64J*>(dummy_rec<double>());
        const uint8_t* hap = H->hap_bases;
        if (t.pair != kNoPair) {
            const PairDesc d = H->desc[t.pair];
            l = (int)d.l;
            k = (int)d.k;
            rec = H->rec64j + d.roff;
            hap = H->hap_bases + d.hoff;
        }
        const int lmax = (int)__reduce_max_sync(kFull, (unsigned)l);
        const SegOut o = team_run_pipe<N, double, FUSE>(rec, l, lmax, hap, k, t.lt * N, t.lt, t.tlast, t.nsteps, pow, rng);
        if (t.pair != kNoPair && t.lt == 0) write_part(H, t.pair, o);
    }
}

// Pipelined scalar teams with packed column halves (team_run_pipe2).  LEAN: the fused row
// (no partials array) with records and carry powers read from L1 each row, which fits
// 128 registers and so four CTAs of four warps per SM.
template <int N, int MINB, bool PACKED, bool LEAN = false>
__global__ void __launch_bounds__(kShortThreads, MINB)
k_short_pipe2(const BatchHeader* __restrict__ H, const PowRow<float>* __restrict__ pow) {
    const PipeRange rng = pipe_range(H->dropgrow);
    const uint32_t n_w = H->n_witems;
    const int lane = threadIdx.x & 31;
    for (;;) {
        uint32_t wi = 0;
        if (lane == 0) wi = atomicAdd(&H->counters[1], 1u);
        wi = __shfl_sync(kFull, wi, 0);
        if (wi >= n_w) break;
        const TeamOf t = team_of(H->teams, H->witems[wi]);
        int l = 0, k = 0;
        const Rec32J* rec = reinterpret_cast<const Rec32J*>(dummy_rec<float>());
        const uint8_t* hap = H->hap_bases;
        if (t.pair != kNoPair) {
            const PairDesc d = H->desc[t.pair];
            l = (int)d.l;
            k = (int)d.k;
            rec = H->rec32j + d.roff;
            hap = H->hap_bases + d.hoff;
        }
        const int lmax = (int)__reduce_max_sync(kFull, (unsigned)l);
        const SegOut o = team_run_pipe2<N, PACKED, false, LEAN, LEAN>(rec, l, lmax, hap, k, t.lt * N, t.lt, t.tlast, t.nsteps, pow, rng);
        if (t.pair != kNoPair && t.lt == 0) write_part(H, t.pair, o);
    }
}

// Packed teams of two haplotypes of the same read, N columns per lane (item list
// witems2 / counters[4]).
template <int N, int MINB>
__global__ void __launch_bounds__(kShortThreads, MINB)
k_short_packed(const BatchHeader* __restrict__ H, const PowRow<float>* __restrict__ pow) {
    const int R = checkpoint_interval<float>(H->dropgrow);
    const uint32_t n_w = H->n_witems2;
    const int lane = threadIdx.x & 31;
    for (;;) {
        uint32_t wi = 0;
        if (lane == 0) wi = atomicAdd(&H->counters[4], 1u);
        wi = __shfl_sync(kFull, wi, 0);
        if (wi >= n_w) break;
        const TeamOf t = team_of(H->teams, H->witems2[wi]);
        int l = 0, k = 0, k2 = 0;
        const Rec32* rec = dummy_rec<float>();
        const uint8_t* hap = H->hap_bases;
        const uint8_t* hap2 = H->hap_bases;
        if (t.pair != kNoPair) {
            const PairDesc d = H->desc[t.pair];
            l = (int)d.l;
            k = (int)d.k;
            rec = H->rec32 + d.roff;
            hap = H->hap_bases + d.hoff;
        }
        if (t.pair2 != kNoPair) {
            const PairDesc d = H->desc[t.pair2];
            k2 = (int)d.k;
            hap2 = H->hap_bases + d.hoff;
        }
        const int lmax = (int)__reduce_max_sync(kFull, (unsigned)l);
        const PairOut2 o = team_run_sr2<N>(rec, l, lmax, hap, k, hap2, k2, t.lt * N, t.lt, t.tlast,
                                           t.nsteps, pow, R);
        if (t.lt == 0) {
            if (t.pair != kNoPair) write_part(H, t.pair, o.a);
            if (t.pair2 != kNoPair) write_part(H, t.pair2, o.b);
        }
    }
}

// A-priori bound on |log10 L(FP32) - log10 L| for a pair of l rows and k columns.  The
// forward sum adds products of nonnegative factors, so nothing cancels and the relative
// error of L is set by the roundings along one path: at most 16 per row (the per-row
// coefficients and the cell arithmetic of Eq. 7 in its factored form) and 4 per column
// (the deletion chain, the scan and its carries), each below u = 2^-23.  The coefficients
// are stochastically rounded (independent, mean-zero errors) and the cell roundings are
// modelled the same way, so m of them add up to less than lambda sqrt(m) u except with
// probability 2 exp(-lambda^2 / 2) (probabilistic rounding-error analysis: Higham & Mary
// 2019; stochastic rounding: Connolly, Higham & Mary 2021); lambda = 6.5 makes that
// 1.4e-9.  The deterministic part is the double-float accuracy of the coefficients
// (8 per row at 2^-46).
__device__ __forceinline__ double fp32_bound_log10(double l, double k) {
    return (6.5 * sqrt(16.0 * l + 4.0 * k) * 0x1.0p-23 + 8.0 * l * 0x1.0p-46) * 0.43429448190325182765;
}

// log10 L per pair (Eq. 4 with C divided out) and selection for the FP64 rescue pass.
// mode: 0 FP32 + rescue, 1 FP64, 2 FP32 only.
template <typename T>
__global__ void k_finalize(const BatchHeader* __restrict__ H) {
    using NT = Num<T>;
    const uint32_t n = H->n_pairs;
    const uint32_t mode = H->mode;
    for (uint32_t p = blockIdx.x * blockDim.x + threadIdx.x; p < n; p += gridDim.x * blockDim.x) {
        Partial q = H->parts[p];
        const PairDesc d = H->desc[p];
        if ((q.flags & PF_DONE) && q.n_extra > 0) {
            // strips of a wide pair: L * C = sum_s S_s 2^(E_s)
            int Eref = q.S != 0.0 ? q.E : INT_MIN;
            for (uint32_t e = 0; e < q.n_extra; ++e) {
                const Partial x = H->parts[q.extra_base + e];
                q.flags |= x.flags;
                if (!(x.flags & PF_DONE)) q.flags &= ~PF_DONE;
                if (x.S != 0.0) Eref = max(Eref, x.E);
            }
            double Sum = 0.0;
            if (Eref != INT_MIN) {
                if (q.S != 0.0) Sum += ldexp(q.S, q.E - Eref);
                for (uint32_t e = 0; e < q.n_extra; ++e) {
                    const Partial x = H->parts[q.extra_base + e];
                    if (x.S != 0.0) Sum += ldexp(x.S, x.E - Eref);
                }
                q.E = Eref;
            }
            q.S = Sum;
        }
        uint32_t f = q.flags;
        double v;
        uint8_t of = 0;
        bool rescue = false;
        if (!(f & PF_DONE)) {
            v = NAN;
            of |= 0x80u;
            atomicOr(H->status, ST_TOO_LONG);
        } else if (f & PF_BAD) {
            v = NAN;
            of |= 0x80u;
            atomicOr(H->status, ST_BAD_INPUT);
        } else {
            if (q.S > 0.0 && isfinite(q.S))
                v = log10(q.S) + (double)(q.E - NT::kLog2C) * 0.30102999566398119521;
            else
                v = q.S == 0.0 ? -INFINITY : NAN;
            if (f & PF_RESCALED) of |= 0x2u;
            if (mode == 1) of |= 0x4u;
            if (f & PF_TIMEOUT) of |= 0x80u;
            if (mode == 1) {
                // FP64: the pipelined engine's own flags (a degenerate row, a range it
                // cannot hold, a non-finite value) send the pair to the unfactored pass
                if (f & PF_DANGER) of |= 0x8u;
                if ((f & PF_NONFINITE) || !isfinite(q.S)) of |= 0x10u;
                if (f & PF_DEGEN) of |= 0x40u;
                rescue = (of & 0x58u) != 0;
            }
            if (mode == 0) {
                // Underflow test (the FP32 sum in stored units against 1e4 * 3 l k FLT_MIN)
                // plus the kernel's own danger / non-finite / degenerate flags.
                const double tau = 3.0e4 * (double)d.l * (double)d.k * 1.1754943508222875e-38;
                if ((f & PF_DANGER) || fp32_bound_log10((double)d.l, (double)d.k) > H->tol32) of |= 0x8u;
                if ((f & PF_NONFINITE) || !isfinite(q.S)) of |= 0x10u;
                if (!(q.S > tau)) of |= 0x20u;
                if (f & PF_DEGEN) of |= 0x40u;
                rescue = H->force_rescue || (of & 0x78u) || !isfinite(v);
            }
        }
        H->out[p] = v;
        H->out_flags[p] = of;
        if (rescue) {
            const uint32_t idx = atomicAdd(&H->counters[2], 1u);
            H->rescue_list[idx] = p;
        }
    }
}

}  // namespace phmm
