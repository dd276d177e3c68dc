// Row-wise PairHMM forward engine (device side).
//
// What one lane does (paper Section 3.4, mapped to sm_103a): a pair's haplotype columns
// are split across the G lanes of a team (a sub-warp, or a whole warp per segment of a
// multi-warp pair); lane t owns N consecutive columns and keeps their M and I values of
// the previous row in registers.  Per read row i:
//
//  1. M and I of row i from row i-1 (Eq. 2 / Eq. 7), left to right over the lane's N
//     columns.  The deletion term D[i-1][j-1] is carried along the lane as
//     D-hat = D / T_MD (so one FMA advances it: D-hat[j] = M[j-1] + g D-hat[j-1]), and the
//     FP32 form is factored so each cell costs 7 FMA-pipe operations:
//        S  = fma(T_MD_{i-1}, Dhat[i-1][j-1], I[i-1][j-1])          I' + D'
//        u  = fma(T_MM_i / (1-g_i), M[i-1][j-1], S)
//        M  = P(r_i|h_j) (1-g_i) * u                                  (Eq. 2, M)
//        I  = fma(T_MI_i, M[i-1][j], g_i * I[i-1][j])                (Eq. 2, I)
//        Dhat[i-1][j] = fma(g_{i-1}, Dhat[i-1][j-1], M[i-1][j-1])    (carry of row i-1)
//        y  = fma(g_i, y, M[i][j])                                    (local D-hat of row i)
//     The FP64 instantiation keeps the unfactored product (one more multiply) so that
//     g = 1 stays exact.
//  2. The deletion recurrence of row i across lanes is a first-order linear recurrence
//     D-hat[j+N] = g^N D-hat[j] + y_lane: an exclusive Kogge-Stone scan over the team with
//     the operator (a, b) o (a', b') = (a a', a' b + b') and a = g^N (Algorithm 1, but
//     the exclusive value comes straight out of the scan: no subtraction, no division).
//     Powers are applied as two factors so products that are representable stay so.
//  3. Between warps of one pair, the last lane publishes its last column's M, I, D-hat
//     and exponent for row i into the next warp's shared-memory ring (tagged 64-bit
//     words, no fences), the next warp folds that carry in.  Warps run skewed by about
//     one row, so the hand-off latency is paid once per segment, not once per row.
//  4. Every R rows the segment's largest |M|, |I| is checked; values are multiplied by
//     an exact power of two when it leaves [2^lo, 2^hi] (the paper is silent on
//     rescaling; the initial scale 2^120 / k alone cannot hold long reads).  A row max
//     below the danger level flags the pair for the FP64 rescue pass.
//  5. After row l: S = sum over the team's columns of M + I (Eq. 4) in FP64.
#pragma once

#include <climits>
#include <cstdint>

#include "phmm_internal.h"

namespace phmm {

constexpr unsigned kFull = 0xffffffffu;

template <typename T>
struct Num;

template <>
struct Num<float> {
    using Rec = Rec32;
    using RecJ = Rec32J;
    static constexpr int kLog2C = 120;      // C = 2^120 (FP32 initial scale of D)
    static constexpr int kHi = 100;         // rescale when the row max >= 2^kHi ...
    static constexpr int kLo = 40;          // ... or < 2^kLo
    static constexpr int kTarget = 96;      // new row max in [2^95, 2^96)
    static constexpr int kDanger = -100;    // below: flag for the FP64 rescue pass
    static constexpr int kDropBudget = 140; // kLo - kDanger
    static constexpr int kGrowBudget = 26;  // (127 - 1) - kHi
    static constexpr int kMinExp = -126, kMaxExp = 127;
    static constexpr bool kFactored = true;
    static constexpr int kWords = 4;        // mailbox words per row: M, I, D-hat, E
    __device__ static __forceinline__ float pow2(int e) {
        return __uint_as_float((uint32_t)(e + 127) << 23);
    }
    // frexp-style exponent: m in [2^(e-1), 2^e) for normal m > 0; INT_MIN for 0 and
    // subnormals; INT_MAX for inf / nan.
    __device__ static __forceinline__ int expo(float m) {
        const uint32_t b = __float_as_uint(m) & 0x7fffffffu;
        const int f = (int)(b >> 23);
        if (f == 0) return INT_MIN;
        if (f == 255) return INT_MAX;
        return f - 126;
    }
};

template <>
struct Num<double> {
    using Rec = Rec64;
    using RecJ = Rec64J;
    static constexpr int kLog2C = 1020;     // C = 2^1020 (Eq. 1)
    static constexpr int kHi = 900;
    static constexpr int kLo = 300;
    static constexpr int kTarget = 800;
    static constexpr int kDanger = -950;
    static constexpr int kDropBudget = 1250;
    static constexpr int kGrowBudget = 120;
    static constexpr int kMinExp = -1022, kMaxExp = 1023;
    static constexpr bool kFactored = false;
    static constexpr int kWords = 8;        // M, I, D-hat as two 32-bit halves each, E
    __device__ static __forceinline__ double pow2(int e) {
        return __longlong_as_double((long long)((uint64_t)(e + 1023) << 52));
    }
    __device__ static __forceinline__ int expo(double m) {
        const uint64_t b = (uint64_t)__double_as_longlong(m) & 0x7fffffffffffffffull;
        const int f = (int)(b >> 52);
        if (f == 0) return INT_MIN;
        if (f == 2047) return INT_MAX;
        return f - 1022;
    }
};

// x * 2^s (two exact steps when 2^s alone is not representable; shifts beyond twice the
// exponent range saturate: to 0 downwards, to the largest factors upwards, where a
// nonzero x overflows to inf and the next checkpoint flags it).
template <typename T>
__device__ __forceinline__ T scale2(T x, int s) {
    using NT = Num<T>;
    if (s >= NT::kMinExp && s <= NT::kMaxExp) return x * NT::pow2(s);
    if (s < 2 * NT::kMinExp) return T(0);
    if (s > 2 * NT::kMaxExp) s = 2 * NT::kMaxExp;
    const int s1 = s / 2;
    return (x * NT::pow2(s1)) * NT::pow2(s - s1);
}

__device__ __forceinline__ Rec32 load_rec(const Rec32* p) {
    const float4 a = __ldg(reinterpret_cast<const float4*>(p));
    const float4 b = __ldg(reinterpret_cast<const float4*>(p) + 1);
    Rec32 r;
    r.pm = a.x; r.px = a.y; r.a = a.z; r.b = a.w;
    r.mi = b.x; r.g = b.y; r.gm = b.z; r.meta = __float_as_uint(b.w);
    return r;
}
__device__ __forceinline__ Rec32J load_recj(const Rec32J* p) {
    const float4 a = __ldg(reinterpret_cast<const float4*>(p));
    const float4 b = __ldg(reinterpret_cast<const float4*>(p) + 1);
    Rec32J r;
    r.pm = a.x; r.px = a.y; r.a = a.z; r.b = a.w;
    r.h = b.x; r.g = b.y; r.mi = b.z; r.meta = __float_as_uint(b.w);
    return r;
}
__device__ __forceinline__ Rec64J load_recj(const Rec64J* p) {
    const double2 a = __ldg(reinterpret_cast<const double2*>(p));
    const double2 b = __ldg(reinterpret_cast<const double2*>(p) + 1);
    const double2 c = __ldg(reinterpret_cast<const double2*>(p) + 2);
    const double2 d = __ldg(reinterpret_cast<const double2*>(p) + 3);
    Rec64J r;
    r.pm = a.x; r.px = a.y; r.a = b.x; r.b = b.y;
    r.h = c.x; r.g = c.y; r.mi = d.x; r.meta = (uint64_t)__double_as_longlong(d.y);
    return r;
}
__device__ __forceinline__ Rec64 load_rec(const Rec64* p) {
    const double2* q = reinterpret_cast<const double2*>(p);
    const double2 a = __ldg(q), b = __ldg(q + 1), c = __ldg(q + 2), d = __ldg(q + 3);
    Rec64 r;
    r.pm = a.x; r.px = a.y; r.a = b.x; r.b = b.y; r.mi = c.x; r.g = c.y; r.gm = d.x;
    r.meta = (uint64_t)__double_as_longlong(d.y);
    return r;
}


// Powers of g for the lane's scan (see PowRow): a pointer to the table row of the
// current gcp; the factors are read through L1 when used (uniform addresses), which
// keeps them out of the register file.
template <typename T>
struct Pow {
    const PowRow<T>* row;
    int gcp;
    __device__ __forceinline__ void load(const PowRow<T>* __restrict__ tab, int gq) {
        row = tab + gq;
        gcp = gq;
    }
    __device__ __forceinline__ T sp1(int s) const { return __ldg(&row->sp1[s]); }
    __device__ __forceinline__ T sp2(int s) const { return __ldg(&row->sp2[s]); }
    __device__ __forceinline__ T lp1(int t) const { return __ldg(&row->lp1[t]); }
    __device__ __forceinline__ T lp2(int t) const { return __ldg(&row->lp2[t]); }
    __device__ __forceinline__ T last1() const { return __ldg(&row->last1); }
    __device__ __forceinline__ T last2() const { return __ldg(&row->last2); }
};

// Inclusive segmented scan z_t = sum_{s<=t} a^(t-s) x_s over the team (lt = lane in
// team); a^(2^s) = sp1[s] * sp2[s].  nsteps is warp-uniform.
template <typename T>
__device__ __forceinline__ T team_scan(T x, int lt, const Pow<T>& pw, int nsteps) {
#pragma unroll
    for (int s = 0; s < 5; ++s) {
        if (s < nsteps) {
            const int off = 1 << s;
            const T up = __shfl_up_sync(kFull, x, off);
            const T t = up * pw.sp1(s);
            if (lt >= off) x = fma(t, pw.sp2(s), x);
        }
    }
    return x;
}

template <typename V>
__device__ __forceinline__ V team_sum(V x, int lt, int last_lane, int nsteps) {
#pragma unroll
    for (int s = 0; s < 5; ++s) {
        if (s < nsteps) {
            const int off = 1 << s;
            const V up = __shfl_up_sync(kFull, x, off);
            if (lt >= off) x += up;
        }
    }
    return __shfl_sync(kFull, x, last_lane);
}

template <typename V>
__device__ __forceinline__ V team_max(V x, int lt, int last_lane, int nsteps) {
#pragma unroll
    for (int s = 0; s < 5; ++s) {
        if (s < nsteps) {
            const int off = 1 << s;
            const V up = __shfl_up_sync(kFull, x, off);
            if (lt >= off) x = fmax(x, up);
        }
    }
    return __shfl_sync(kFull, x, last_lane);
}

// Maximum of non-negative FP32 values over a team (lanes last_lane - lt .. last_lane), in
// every lane of the team: one warp reduction on the bit patterns, which order like the
// values for x >= 0 (the team's mask keeps other teams apart).  Same result as team_max.
__device__ __forceinline__ float team_max_pos(float x, int lt, int last_lane) {
    const int base = (int)(threadIdx.x & 31) - lt, size = last_lane - base + 1;
    const unsigned mask = size >= 32 ? kFull : ((1u << size) - 1u) << base;
    return __uint_as_float(__reduce_max_sync(mask, __float_as_uint(x)));
}

__device__ __forceinline__ uint32_t team_or(uint32_t x, int lt, int last_lane, int nsteps) {
#pragma unroll
    for (int s = 0; s < 5; ++s) {
        if (s < nsteps) {
            const int off = 1 << s;
            const uint32_t up = __shfl_up_sync(kFull, x, off);
            if (lt >= off) x |= up;
        }
    }
    return __shfl_sync(kFull, x, last_lane);
}

// Base code of an ASCII haplotype / read byte: A=0 C=1 G=2 T=3 N=4, -1 otherwise.
__device__ __forceinline__ int base_code(uint32_t c) {
    c |= 0x20u;  // lower case
    switch (c) {
    case 'a': return 0;
    case 'c': return 1;
    case 'g': return 2;
    case 't': return 3;
    case 'n': return 4;
    default: return -1;
    }
}

// ------------------------------------------------------------------------------------
// Shared-memory mailbox between consecutive warp segments of one pair.
// Word = (payload32 << 32) | row tag; a row is complete when every word carries its tag.
// ------------------------------------------------------------------------------------
constexpr long long kSpinLimit = 1ll << 22;  // polls (with backoff) before giving up
constexpr long long kSpinFast = 256;         // polls without backoff first: a neighbour
                                             // segment is usually a few hundred cycles
                                             // behind, far less than one sleep

struct SmemLink {
    unsigned long long* in_ring;   // my inbound ring  [kRing][words]
    unsigned long long* out_ring;  // next segment's ring
    volatile int* my_cons;         // rows I have consumed (written by me)
    volatile int* next_cons;       // rows the next segment consumed (read by me)
    unsigned long long* in_g;      // strip boundary in global memory (row-indexed), or null
    unsigned long long* out_g;     // ... outbound, or null
    bool has_left, has_right;
};

__device__ __forceinline__ void st_vol(unsigned long long* p, unsigned long long v) {
    *reinterpret_cast<volatile unsigned long long*>(p) = v;
}
__device__ __forceinline__ unsigned long long ld_vol(const unsigned long long* p) {
    return *reinterpret_cast<const volatile unsigned long long*>(p);
}
__device__ __forceinline__ unsigned long long tagw(uint32_t payload, int row) {
    return ((unsigned long long)payload << 32) | (uint32_t)row;
}

template <typename T>
__device__ __forceinline__ void pack_vals(T m, T i, T d, int e, uint32_t* w);
template <>
__device__ __forceinline__ void pack_vals<float>(float m, float i, float d, int e, uint32_t* w) {
    w[0] = __float_as_uint(m); w[1] = __float_as_uint(i); w[2] = __float_as_uint(d);
    w[3] = (uint32_t)e;
}
template <>
__device__ __forceinline__ void pack_vals<double>(double m, double i, double d, int e, uint32_t* w) {
    const unsigned long long a = (unsigned long long)__double_as_longlong(m);
    const unsigned long long b = (unsigned long long)__double_as_longlong(i);
    const unsigned long long c = (unsigned long long)__double_as_longlong(d);
    w[0] = (uint32_t)a; w[1] = (uint32_t)(a >> 32); w[2] = (uint32_t)b; w[3] = (uint32_t)(b >> 32);
    w[4] = (uint32_t)c; w[5] = (uint32_t)(c >> 32); w[6] = (uint32_t)e; w[7] = 0;
}
template <typename T>
__device__ __forceinline__ void unpack_vals(const uint32_t* w, T& m, T& i, T& d, int& e);
template <>
__device__ __forceinline__ void unpack_vals<float>(const uint32_t* w, float& m, float& i, float& d, int& e) {
    m = __uint_as_float(w[0]); i = __uint_as_float(w[1]); d = __uint_as_float(w[2]); e = (int)w[3];
}
template <>
__device__ __forceinline__ void unpack_vals<double>(const uint32_t* w, double& m, double& i, double& d, int& e) {
    m = __longlong_as_double((long long)(((unsigned long long)w[1] << 32) | w[0]));
    i = __longlong_as_double((long long)(((unsigned long long)w[3] << 32) | w[2]));
    d = __longlong_as_double((long long)(((unsigned long long)w[5] << 32) | w[4]));
    e = (int)w[6];
}

// Producer side (called by the segment's last lane): wait for ring space, then publish.
template <typename T>
__device__ bool link_send(const SmemLink& L, int row, T m, T i, T d, int e) {
    constexpr int W = Num<T>::kWords;
    bool ok = true;
    long long spins = 0;
    while (*L.next_cons < row - kRing) {
        if (++spins > kSpinLimit) { ok = false; break; }
        if (spins > kSpinFast) __nanosleep(64);
    }
    uint32_t w[W];
    pack_vals<T>(m, i, d, e, w);
    unsigned long long* slot = L.out_ring + (row % kRing) * W;
#pragma unroll
    for (int q = 0; q < W; ++q) st_vol(slot + q, tagw(w[q], row));
    return ok;
}

// Consumer side (called by the segment's first lane): wait for the row, read it.
template <typename T>
__device__ bool link_recv(const SmemLink& L, int row, T& m, T& i, T& d, int& e) {
    constexpr int W = Num<T>::kWords;
    const unsigned long long* slot = L.in_ring + (row % kRing) * W;
    uint32_t w[W];
    bool ok = true;
    long long spins = 0;
    for (;;) {
        bool all = true;
#pragma unroll
        for (int q = 0; q < W; ++q) {
            const unsigned long long v = ld_vol(slot + q);
            w[q] = (uint32_t)(v >> 32);
            all &= ((uint32_t)v == (uint32_t)row);
        }
        if (all) break;
        if (++spins > kSpinLimit) { ok = false; break; }
        if (spins > kSpinFast) __nanosleep(32);
    }
    unpack_vals<T>(w, m, i, d, e);
    *L.my_cons = row;
    return ok;
}

// Strip boundaries in global memory: one slot of kWords tagged words per row (no ring,
// no back-pressure: the buffer holds every row), written once per launch.
template <typename T>
__device__ __forceinline__ void link_send_g(unsigned long long* base, int row, T m, T i, T d, int e) {
    constexpr int W = Num<T>::kWords;
    uint32_t w[W];
    pack_vals<T>(m, i, d, e, w);
    unsigned long long* slot = base + (size_t)(row - 1) * W;
#pragma unroll
    for (int q = 0; q < W; ++q) st_vol(slot + q, tagw(w[q], row));
}
template <typename T>
__device__ bool link_recv_g(const unsigned long long* base, int row, T& m, T& i, T& d, int& e) {
    constexpr int W = Num<T>::kWords;
    const unsigned long long* slot = base + (size_t)(row - 1) * W;
    uint32_t w[W];
    bool ok = true;
    long long spins = 0;
    for (;;) {
        bool all = true;
#pragma unroll
        for (int q = 0; q < W; ++q) {
            const unsigned long long v = ld_vol(slot + q);
            w[q] = (uint32_t)(v >> 32);
            all &= ((uint32_t)v == (uint32_t)row);
        }
        if (all) break;
        if (++spins > kSpinLimit) { ok = false; break; }
        if (spins > kSpinFast) __nanosleep(64);
    }
    unpack_vals<T>(w, m, i, d, e);
    return ok;
}

// Checkpoint interval R from the batch's worst per-row drop and growth (bits * 64),
// so that between checkpoints no value can overflow and the row max cannot fall from
// 2^lo to below the danger level.
template <typename T>
__device__ __forceinline__ int checkpoint_interval(const uint32_t* dropgrow) {
    using NT = Num<T>;
    const uint32_t d = max(dropgrow[0], 1u), g = max(dropgrow[1], 1u);
    int r1 = (int)((uint64_t)NT::kDropBudget * 64u / d);
    int r2 = (int)((uint64_t)NT::kGrowBudget * 64u / g);
    int r = min(r1, r2);
    return max(1, min(r, 64));
}

// Range control of the pipelined FP32 engine.  Its match-update partial U = a M' + J' and
// the term b D-hat' are up to 2^rbits times the row maximum (rbits from prep: a, b/(1-g)
// and 1/T_MI of the previous row), and M can sit 2^rbits below J; so the rescale ceiling
// leaves rbits + 16 bits of headroom, the danger level rises by rbits, and the checkpoint
// interval R keeps the worst-case drift of the maximum within both budgets (J grows by at
// most 1 + h per row).  ok = false: the range does not fit (the pairs go to the rescue).
struct PipeRange {
    int R, hi, target, danger;
    bool ok;
};
template <typename T = float>
__device__ __forceinline__ PipeRange pipe_range(const uint32_t* dropgrow) {
    using NT = Num<T>;
    const int rbits = (int)min(dropgrow[2], 200u);
    PipeRange r;
    r.hi = min(NT::kHi, NT::kMaxExp - 17 - rbits);
    r.target = r.hi - 4;
    r.danger = NT::kDanger + rbits;
    r.ok = r.hi >= NT::kLo + 16 && r.danger <= NT::kLo - 32;
    const uint32_t d = max(dropgrow[0], 1u), g = max(max(dropgrow[1], dropgrow[3]), 1u);
    const int drop_budget = max(NT::kLo - r.danger, 1), grow_budget = max(NT::kMaxExp - 1 - rbits - r.hi, 1);
    const int r1 = (int)((uint64_t)drop_budget * 64u / d), r2 = (int)((uint64_t)grow_budget * 64u / g);
    r.R = max(1, min(min(r1, r2), 64));
    return r;
}

struct SegOut {
    double S;
    int E;
    uint32_t flags;
};

// ------------------------------------------------------------------------------------
// One team / segment: rows 1..lmax over the lane's N columns.  Returns the team's
// final (S, E, flags) in every lane of the team (valid when the team's l <= lmax).
//   rec      the read's records (row i at rec[i-1]), l rows; lmax >= l is the warp's
//            row count (rows beyond l recompute row l harmlessly)
//   hap, k   the haplotype (ASCII) and its length; col0 = the lane's first column - 1
//   lt       lane in team; tlast = absolute lane of the team's last lane; nsteps = scan
//            steps (warp-uniform)
//   R        checkpoint interval
// ------------------------------------------------------------------------------------
template <typename T, int N, bool LINKED>
__device__ SegOut seg_run(const typename Num<T>::Rec* __restrict__ rec, int l, int lmax,
                          const uint8_t* __restrict__ hap, int k, int col0, int lt, int tlast,
                          int nsteps, const PowRow<T>* __restrict__ pow_tab, int R,
                          const SmemLink& link, uint32_t* __restrict__ status) {
    using NT = Num<T>;
    using Rec = typename NT::Rec;
    static_assert(N <= 32, "match masks hold 32 columns");

    // Match masks of the lane's columns (Eq. 3; an N matches every base).
    uint32_t bmA = 0, bmC = 0, bmG = 0, bmT = 0;
    uint32_t flags = 0;
    const bool has_left = LINKED && link.has_left, has_right = LINKED && link.has_right;
    const int nvalid = max(0, min(k - col0, N));
#pragma unroll
    for (int c = 0; c < N; ++c) {
        if (c < nvalid) {
            const int code = base_code(hap[col0 + c]);
            const uint32_t bit = 1u << c;
            if (code < 0) flags |= PF_BAD;
            if (code == 0 || code == 4) bmA |= bit;
            if (code == 1 || code == 4) bmC |= bit;
            if (code == 2 || code == 4) bmG |= bit;
            if (code == 3 || code == 4) bmT |= bit;
        }
    }

    T M[N], I[N];
    int E = 0;
    T ml = T(0), sl = T(0), dt = T(0), gprev = T(0);
    Pow<T> pw;
    pw.row = pow_tab;
    pw.gcp = -1;
    SegOut out;
    out.S = 0.0;
    out.E = 0;
    out.flags = 0;
    const bool active = l > 0;
    const T cinit = active && k > 0 ? (T)(ldexp(1.0, NT::kLog2C) / (double)k) : T(0);

    Rec cur = load_rec(rec);
    for (int i = 1; i <= lmax; ++i) {
        Rec nxt = cur;
        if (i < lmax) nxt = load_rec(rec + min(i, max(l, 1) - 1));
        const uint32_t meta = (uint32_t)cur.meta;
        const int gq = (int)((meta >> META_GCP_SHIFT) & 0xffu);
        if (gq != pw.gcp) pw.load(pow_tab, min(gq, kMaxPhred));
        if (i <= l) {
            if (meta & META_BAD) flags |= PF_BAD;
            if (NT::kFactored && (meta & META_DEGEN)) flags |= PF_DEGEN;
        }
        const int code = (int)(meta & META_CODE_MASK);
        const uint32_t mask = code == 0 ? bmA : code == 1 ? bmC : code == 2 ? bmG
                            : code == 3 ? bmT : 0xffffffffu;
        const T pim = cur.pm, pix = cur.px, rg = cur.g;
        T y = T(0), yprev = T(0);
        if (i == 1) {
            // Row 1 (Eq. 1-2): M = P (1 - g_1) C / k, I = 0.
            const T c1 = NT::kFactored ? cinit : cinit * cur.gm;
#pragma unroll
            for (int c = 0; c < N; ++c) {
                const T p = ((mask >> c) & 1u) ? pim : pix;
                M[c] = p * c1;
                I[c] = T(0);
                if (c == N - 1) yprev = y;
                y = fma(rg, y, M[c]);
            }
        } else {
            const T ra = cur.a, rb = cur.b, rmi = cur.mi, rgm = cur.gm;
#pragma unroll
            for (int c = 0; c < N; ++c) {
                const T S = fma(rb, dt, sl);
                T u;
                if (NT::kFactored) u = fma(ra, ml, S);
                else u = fma(ra, ml, rgm * S);
                const T p = ((mask >> c) & 1u) ? pim : pix;
                const T mn = p * u;
                const T in = fma(rmi, M[c], rg * I[c]);
                dt = fma(gprev, dt, ml);
                ml = M[c];
                sl = I[c];
                M[c] = mn;
                I[c] = in;
                if (c == N - 1) yprev = y;
                y = fma(rg, y, mn);
            }
        }

        // Deletion scan of row i across the team: W = D-hat at the lane's first column.
        const T Z = team_scan<T>(y, lt, pw, nsteps);
        T Wd = __shfl_up_sync(kFull, Z, 1);
        if (lt == 0) Wd = T(0);

        // Carry from the previous warp segment (multi-warp pairs): lane 0 waits for it, then
        // the (converged) warp takes it.
        T lM = T(0), lI = T(0), lD = T(0);
        int Eleft = INT_MIN;
        if (LINKED) {
            int e_in = INT_MIN;
            if (has_left && (threadIdx.x & 31) == 0) {
                const bool ok = link.in_g ? link_recv_g<T>(link.in_g, i, lM, lI, lD, e_in)
                                          : link_recv<T>(link, i, lM, lI, lD, e_in);
                if (!ok) {
                    flags |= PF_TIMEOUT;
                    atomicOr(status, ST_TIMEOUT);
                }
            }
            __syncwarp();
            lM = __shfl_sync(kFull, lM, 0);
            lI = __shfl_sync(kFull, lI, 0);
            lD = __shfl_sync(kFull, lD, 0);
            Eleft = __shfl_sync(kFull, e_in, 0);
        }

        // Checkpoint: power-of-two rescaling of the segment (uniform across the warp).
        int Enew = E;
        if (i == 1 || (i - 1) % R == 0) {
            T m = T(0);
#pragma unroll
            for (int c = 0; c < N; ++c) m = fmax(m, fmax(fabs(M[c]), fabs(I[c])));
            m = team_max<T>(m, lt, tlast, nsteps);
            const int e = NT::expo(m);
            int desired = E;
            if (e == INT_MAX) {
                if (i <= l) flags |= PF_NONFINITE;
            } else if (e == INT_MIN) {
                // Nothing representable in this segment: follow the left neighbour's scale,
                // so that mass arriving later from the left is not converted across a
                // gap wider than the format's range.
                if (has_left) desired = INT_MIN;
            } else if (e > NT::kHi || e <= NT::kLo) {
                desired = E + (e - NT::kTarget);
            }
            Enew = desired;
            bool forced = false;
            if (has_left && Eleft > Enew) {
                Enew = Eleft;
                forced = true;
            }
            if (Enew == INT_MIN) Enew = E;
            // A segment whose largest value is zero or subnormal holds no mass of its
            // own (it sits beside the alignment band); an empty row as a whole is caught
            // by the underflow test on the final sum.
            if (!forced && e != INT_MIN && e <= NT::kDanger && i <= l) flags |= PF_DANGER;
        }
        if (Enew != E) {
            const int s = E - Enew;
#pragma unroll
            for (int c = 0; c < N; ++c) {
                M[c] = scale2(M[c], s);
                I[c] = scale2(I[c], s);
            }
            Wd = scale2(Wd, s);
            yprev = scale2(yprev, s);
            if (i <= l) flags |= PF_RESCALED;
            E = Enew;
        }
        if (has_left) {
            // Left values into this segment's scale (E >= Eleft always holds here).
            const int d = Eleft - E;
            lM = scale2(lM, d);
            lI = scale2(lI, d);
            lD = scale2(lD, d);
            const T Wseg = fma(rg, lD, lM);  // D-hat at the segment's first column
            Wd = fma(Wseg * pw.lp1(lt), pw.lp2(lt), Wd);
        }
        // D-hat at the lane's last column (needed by the next lane's first cell).
        const T Dlast = fma(Wd * pw.last1(), pw.last2(), yprev);

        if (has_right && (threadIdx.x & 31) == 31) {
            if (link.out_g) {
                link_send_g<T>(link.out_g, i, M[N - 1], I[N - 1], Dlast, E);
            } else if (!link_send<T>(link, i, M[N - 1], I[N - 1], Dlast, E)) {
                flags |= PF_TIMEOUT;
                atomicOr(status, ST_TIMEOUT);
            }
        }

        // Eq. 4 when a team of this warp finishes (warp-uniform participation).
        if (__any_sync(kFull, i == l)) {
            double s = 0.0;
#pragma unroll
            for (int c = 0; c < N; ++c)
                if (c < nvalid) s += (double)M[c] + (double)I[c];
            s = team_sum<double>(s, lt, tlast, nsteps);
            const uint32_t f = team_or(flags, lt, tlast, nsteps);
            if (i == l) {
                out.S = s;
                out.E = E;
                out.flags = f;
            }
        }

        // Inputs of the next row's first column.
        T nm = __shfl_up_sync(kFull, M[N - 1], 1);
        T ni = __shfl_up_sync(kFull, I[N - 1], 1);
        T nd = __shfl_up_sync(kFull, Dlast, 1);
        if (lt == 0) {
            nm = lM;
            ni = lI;
            nd = lD;
        }
        ml = nm;
        sl = ni;
        dt = nd;
        gprev = rg;
        cur = nxt;
    }
    return out;
}

}  // namespace phmm

namespace phmm {


}  // namespace phmm

namespace phmm {

// ------------------------------------------------------------------------------------
// Helpers of the packed FP32 engines (float2 halves) and of the double-float prep.
// ------------------------------------------------------------------------------------
__device__ __forceinline__ float2 f2(float a, float b) { return make_float2(a, b); }

// Exact sum of two floats as hi + lo (Knuth's two-sum).
struct df {
    float hi, lo;
};
__device__ __forceinline__ df two_sum(float a, float b) {
    const float s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    return {s, __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb))};
}
__device__ __forceinline__ float2 shfl_up2(float2 v, int off) {
    return f2(__shfl_up_sync(kFull, v.x, off), __shfl_up_sync(kFull, v.y, off));
}

struct PairOut2 {
    SegOut a, b;
};

// ------------------------------------------------------------------------------------
// Lean scalar FP32 team (short pairs, no neighbour link): seg_run's algorithm with the
// per-row work cut down -- scan powers cached in registers (reloaded only when gcp
// changes), a countdown for checkpoints, record flag bits folded with one OR per row.
// ------------------------------------------------------------------------------------
template <int N>
__device__ SegOut team_run_lean(const Rec32* __restrict__ rec, int l, int lmax,
                                const uint8_t* __restrict__ hap, int k, int col0, int lt,
                                int tlast, int nsteps, const PowRow<float>* __restrict__ pow_tab,
                                int R) {
    using NT = Num<float>;
    static_assert(N <= 32, "match masks hold 32 columns");
    uint32_t bmA = 0, bmC = 0, bmG = 0, bmT = 0, flags = 0, mflags = 0;
    const int nvalid = max(0, min(k - col0, N));
#pragma unroll
    for (int c = 0; c < N; ++c) {
        if (c < nvalid) {
            const int code = base_code(hap[col0 + c]);
            const uint32_t bit = 1u << c;
            if (code < 0) flags |= PF_BAD;
            if (code == 0 || code == 4) bmA |= bit;
            if (code == 1 || code == 4) bmC |= bit;
            if (code == 2 || code == 4) bmG |= bit;
            if (code == 3 || code == 4) bmT |= bit;
        }
    }
    float M[N], I[N];
    int E = 0;
    float ml = 0.f, sl = 0.f, dt = 0.f, gprev = 0.f;
    float sp1[5], sp2[5], last1 = 0.f, last2 = 0.f;
    int gcp = -1;
    SegOut out;
    out.S = 0.0;
    out.E = 0;
    out.flags = 0;
    const float cinit = l > 0 && k > 0 ? (float)(0x1p120 / (double)k) : 0.f;
    const int l1 = max(l, 1) - 1;
    Rec32 cur = load_rec(rec);
    int until = 0;
    for (int i = 1; i <= lmax; ++i) {
        Rec32 nxt = cur;
        if (i < lmax) nxt = load_rec(rec + min(i, l1));
        const uint32_t meta = cur.meta;
        mflags |= meta;
        const int gq = (int)((meta >> META_GCP_SHIFT) & 0xffu);
        if (gq != gcp) {
            const PowRow<float>* pr = pow_tab + min(gq, kMaxPhred);
#pragma unroll
            for (int s = 0; s < 5; ++s) {
                sp1[s] = __ldg(&pr->sp1[s]);
                sp2[s] = __ldg(&pr->sp2[s]);
            }
            last1 = __ldg(&pr->last1);
            last2 = __ldg(&pr->last2);
            gcp = gq;
        }
        const int code = (int)(meta & META_CODE_MASK);
        const uint32_t mask = code == 0 ? bmA : code == 1 ? bmC : code == 2 ? bmG
                            : code == 3 ? bmT : 0xffffffffu;
        const float pim = cur.pm, pix = cur.px, rg = cur.g;
        float y = 0.f, yprev = 0.f;
        if (i == 1) {
#pragma unroll
            for (int c = 0; c < N; ++c) {
                M[c] = (((mask >> c) & 1u) ? pim : pix) * cinit;
                I[c] = 0.f;
                if (c == N - 1) yprev = y;
                y = fmaf(rg, y, M[c]);
            }
        } else {
            const float ra = cur.a, rb = cur.b, rmi = cur.mi;
#pragma unroll
            for (int c = 0; c < N; ++c) {
                const float S = fmaf(rb, dt, sl);
                const float u = fmaf(ra, ml, S);
                const float mn = (((mask >> c) & 1u) ? pim : pix) * u;
                const float in = fmaf(rmi, M[c], rg * I[c]);
                dt = fmaf(gprev, dt, ml);
                ml = M[c];
                sl = I[c];
                M[c] = mn;
                I[c] = in;
                if (c == N - 1) yprev = y;
                y = fmaf(rg, y, mn);
            }
        }
        float Z = y;
#pragma unroll
        for (int s = 0; s < 5; ++s) {
            if (s < nsteps) {
                const int off = 1 << s;
                const float up = __shfl_up_sync(kFull, Z, off);
                const float t = up * sp1[s];
                if (lt >= off) Z = fmaf(t, sp2[s], Z);
            }
        }
        float Wd = __shfl_up_sync(kFull, Z, 1);
        if (lt == 0) Wd = 0.f;
        if (until == 0) {
            until = R;
            float m = 0.f;
#pragma unroll
            for (int c = 0; c < N; ++c) m = fmaxf(m, fmaxf(fabsf(M[c]), fabsf(I[c])));
            m = team_max<float>(m, lt, tlast, nsteps);
            const int e = NT::expo(m);
            if (e == INT_MAX) {
                flags |= PF_NONFINITE;
            } else if (e != INT_MIN) {
                if (e <= NT::kDanger) flags |= PF_DANGER;
                if (e > NT::kHi || e <= NT::kLo) {
                    const int sh = e - NT::kTarget;  // multiply by 2^-sh in two exact steps
                    const float f1 = NT::pow2((-sh) / 2), f2v = NT::pow2(-sh - (-sh) / 2);
#pragma unroll
                    for (int c = 0; c < N; ++c) {
                        M[c] = (M[c] * f1) * f2v;
                        I[c] = (I[c] * f1) * f2v;
                    }
                    Wd = (Wd * f1) * f2v;
                    yprev = (yprev * f1) * f2v;
                    flags |= PF_RESCALED;
                    E += sh;
                }
            }
        }
        --until;
        const float Dlast = fmaf(Wd * last1, last2, yprev);
        if (__any_sync(kFull, i == l)) {
            double s = 0.0;
#pragma unroll
            for (int c = 0; c < N; ++c)
                if (c < nvalid) s += (double)M[c] + (double)I[c];
            s = team_sum<double>(s, lt, tlast, nsteps);
            uint32_t f = flags;
            if (mflags & META_BAD) f |= PF_BAD;
            if (mflags & META_DEGEN) f |= PF_DEGEN;
            f = team_or(f, lt, tlast, nsteps);
            if (i == l) {
                out.S = s;
                out.E = E;
                out.flags = f;
            }
        }
        float nm = __shfl_up_sync(kFull, M[N - 1], 1);
        float ni = __shfl_up_sync(kFull, I[N - 1], 1);
        float nd = __shfl_up_sync(kFull, Dlast, 1);
        if (lt == 0) {
            nm = 0.f;
            ni = 0.f;
            nd = 0.f;
        }
        ml = nm;
        sl = ni;
        dt = nd;
        gprev = rg;
        cur = nxt;
    }
    return out;
}

}  // namespace phmm

namespace phmm {

// ------------------------------------------------------------------------------------
// Pipelined scalar FP32 team (short pairs, no neighbour link).  Same recurrences as
// team_run_lean (Eq. 2 in the row-wise form of Eq. 7), rearranged so that the part of
// row i+1 that does not depend on row i's deletion scan runs while that scan's shuffles
// are in flight:
//   phase B (row i):  u = b D-hat_{i-1,j-1} + U_ij,  M_ij = P' u,  D-hat_{i-1} chain
//                     (carry from the left lane), lane-local D-hat_i chain y;
//   scan of y over the team (Algorithm 1), and alongside it
//   phase A (row i+1): U_{i+1,j} = a M_{i,j-1} + J_{i,j-1},  J_{i+1,j} = M_{i,j} + h J_{i,j}.
// J = I / T_MI (see Rec32J) makes the insertion update a single FMA.  The scan always
// takes five steps (steps beyond the team width change nothing), so it is one basic
// block that the compiler can interleave with phase A.
// ------------------------------------------------------------------------------------
template <int N, typename T = float, bool FUSE = false>
__device__ SegOut team_run_pipe(const typename Num<T>::RecJ* __restrict__ rec, int l, int lmax,
                                const uint8_t* __restrict__ hap, int k, int col0, int lt,
                                int tlast, int nsteps, const PowRow<T>* __restrict__ pow_tab,
                                const PipeRange& rng) {
    using NT = Num<T>;
    using RecJ = typename NT::RecJ;
    static_assert(N <= 32, "match masks hold 32 columns");
    uint32_t bmA = 0, bmC = 0, bmG = 0, bmT = 0, flags = rng.ok ? 0u : PF_DEGEN, mflags = 0;
    const int nvalid = max(0, min(k - col0, N));
#pragma unroll
    for (int c = 0; c < N; ++c) {
        if (c < nvalid) {
            const int code = base_code(hap[col0 + c]);
            const uint32_t bit = 1u << c;
            if (code < 0) flags |= PF_BAD;
            if (code == 0 || code == 4) bmA |= bit;
            if (code == 1 || code == 4) bmC |= bit;
            if (code == 2 || code == 4) bmG |= bit;
            if (code == 3 || code == 4) bmT |= bit;
        }
    }
    T M[N], J[N];
    T U[FUSE ? 1 : N];  // unfused: row i + 1's partials, formed after row i's scan
    T nj = T(0);        // fused: row i's J at the column before the lane
    int E = NT::kLog2C - rng.target;  // see cinit
    T ml = T(0), dt = T(0), gprev = T(0);
    T sp1[5], sp2[5], last1 = T(0), last2 = T(0);
    int gcp = -1;
    SegOut out;
    out.S = 0.0;
    out.E = 0;
    out.flags = 0;
    // Eq. 1's scale C taken as already rescaled to 2^target (E records the difference),
    // so that row 1 and the partials U formed from it start in range
    const T cinit = l > 0 && k > 0 ? (T)(ldexp(1.0, rng.target) / (double)k) : T(0);
    const int l1 = max(l, 1) - 1;
    RecJ cur = load_recj(rec);
    int until = 0;
    for (int i = 1; i <= lmax; ++i) {
        RecJ nxt = cur;
        if (i < lmax) nxt = load_recj(rec + min(i, l1));
        const uint32_t meta = (uint32_t)cur.meta;
        mflags |= meta;
        const int gq = (int)((meta >> META_GCP_SHIFT) & 0xffu);
        if (gq != gcp) {
            const PowRow<T>* pr = pow_tab + min(gq, kMaxPhred);
#pragma unroll
            for (int s = 0; s < 5; ++s) {
                sp1[s] = lt >= (1 << s) ? __ldg(&pr->sp1[s]) : T(0);
                sp2[s] = __ldg(&pr->sp2[s]);
            }
            last1 = __ldg(&pr->last1);
            last2 = __ldg(&pr->last2);
            gcp = gq;
        }
        const int code = (int)(meta & META_CODE_MASK);
        const uint32_t mask = code == 0 ? bmA : code == 1 ? bmC : code == 2 ? bmG
                            : code == 3 ? bmT : 0xffffffffu;
        const T pim = cur.pm, pix = cur.px, rg = cur.g;
        T y = T(0), yprev = T(0);
        // phase B
        if (i == 1) {
#pragma unroll
            for (int c = 0; c < N; ++c) {
                M[c] = (((mask >> c) & 1u) ? pim : pix) * cinit;
                J[c] = T(0);
                if (c == N - 1) yprev = y;
                y = fma(rg, y, M[c]);
            }
        } else if constexpr (FUSE) {
            // Row i's partials U = a M' + J' and insertions J = M' + h J' (primes: row i - 1)
            // formed column by column inside phase B, as in team_run_pipe2's fused row
            const T rb = cur.b, na = cur.a, nh = cur.h;
#pragma unroll
            for (int c = 0; c < N; ++c) {
                const T uq = fma(na, ml, c == 0 ? nj : J[c - 1]);
                if (c > 0) J[c - 1] = fma(nh, J[c - 1], ml);
                const T u = fma(rb, dt, uq);
                dt = fma(gprev, dt, ml);
                ml = M[c];
                const T mn = (((mask >> c) & 1u) ? pim : pix) * u;
                M[c] = mn;
                if (c == N - 1) yprev = y;
                y = fma(rg, y, mn);
            }
            J[N - 1] = fma(nh, J[N - 1], ml);
        } else {
            const T rb = cur.b;
#pragma unroll
            for (int c = 0; c < N; ++c) {
                const T u = fma(rb, dt, U[c]);
                dt = fma(gprev, dt, ml);
                ml = M[c];
                const T mn = (((mask >> c) & 1u) ? pim : pix) * u;
                M[c] = mn;
                if (c == N - 1) yprev = y;
                y = fma(rg, y, mn);
            }
        }
        // Eq. 4 when a pair of this warp finishes (I = T_MI J on the last row)
        if (__any_sync(kFull, i == l)) {
            const double rmi = (double)cur.mi;
            double s = 0.0;
#pragma unroll
            for (int c = 0; c < N; ++c)
                if (c < nvalid) s += (double)M[c] + rmi * (double)J[c];
            s = team_sum<double>(s, lt, tlast, nsteps);
            uint32_t f = flags;
            if (mflags & META_BAD) f |= PF_BAD;
            if (mflags & META_DEGEN) f |= PF_DEGEN;
            f = team_or(f, lt, tlast, nsteps);
            if (i == l) {
                out.S = s;
                out.E = E;
                out.flags = f;
            }
        }
        // the deletion scan of row i and, independent of it, phase A of row i+1
        T nm = __shfl_up_sync(kFull, M[N - 1], 1);
        nj = __shfl_up_sync(kFull, J[N - 1], 1);
        T yp = __shfl_up_sync(kFull, yprev, 1);
        if (lt == 0) {
            nm = T(0);
            nj = T(0);
            yp = T(0);
        }
        T Z = y;
#pragma unroll
        for (int s = 0; s < 5; ++s) {
            const int off = 1 << s;
            const T up = __shfl_up_sync(kFull, Z, off);
            Z = fma(up * sp1[s], sp2[s], Z);
        }
        if constexpr (!FUSE) {
            const T na = nxt.a, nh = nxt.h;
#pragma unroll
            for (int c = N - 1; c >= 1; --c) {
                U[c] = fma(na, M[c - 1], J[c - 1]);
                J[c] = fma(nh, J[c], M[c]);
            }
            U[0] = fma(na, nm, nj);
            J[0] = fma(nh, J[0], M[0]);
        }
        T zz = __shfl_up_sync(kFull, Z, 2);
        if (lt < 2) zz = T(0);
        if (until == 0) {
            // checkpoint: M holds row i, J and U row i+1 when unfused (linear in row i, so
            // they take the same power of two; U was formed before this test, which the
            // headroom of the range bounds covers), J row i when fused
            until = rng.R;
            T m = T(0);
#pragma unroll
            for (int c = 0; c < N; ++c) m = fmax(m, fmax(fabs(M[c]), fabs(J[c])));
            if constexpr (sizeof(T) == 4) m = team_max_pos(m, lt, tlast);
            else m = team_max<T>(m, lt, tlast, nsteps);
            const int e = NT::expo(m);
            if (e == INT_MAX) {
                flags |= PF_NONFINITE;
            } else if (e != INT_MIN) {
                if (e <= rng.danger) flags |= PF_DANGER;
                if (e > rng.hi || e <= NT::kLo) {
                    const int sh = e - rng.target;  // multiply by 2^-sh
                    if (sh >= NT::kMinExp && sh <= NT::kMaxExp - 1) {
                        const T f = NT::pow2(-sh);
#pragma unroll
                        for (int c = 0; c < N; ++c) {
                            M[c] *= f;
                            J[c] *= f;
                            if constexpr (!FUSE) U[c] *= f;
                        }
                        nm *= f;
                        nj *= f;
                        zz *= f;
                        yp *= f;
                    } else {  // two exact steps
                        const T f1 = NT::pow2((-sh) / 2), f2v = NT::pow2(-sh - (-sh) / 2);
#pragma unroll
                        for (int c = 0; c < N; ++c) {
                            M[c] = (M[c] * f1) * f2v;
                            J[c] = (J[c] * f1) * f2v;
                            if constexpr (!FUSE) U[c] = (U[c] * f1) * f2v;
                        }
                        nm = (nm * f1) * f2v;
                        nj = (nj * f1) * f2v;
                        zz = (zz * f1) * f2v;
                        yp = (yp * f1) * f2v;
                    }
                    flags |= PF_RESCALED;
                    E += sh;
                }
            }
        }
        --until;
        ml = nm;
        dt = fma(zz * last1, last2, yp);
        gprev = rg;
        cur = nxt;
    }
    return out;
}

// ------------------------------------------------------------------------------------
// team_run_pipe with each lane's columns split in two halves that advance side by side:
// column q of the first half and column N/2 + q of the second sit in one float2 and share
// a packed FFMA2 / FMUL2 (PACKED) or go through two scalar instructions (two independent
// dependency chains per lane).  Both halves run the D-hat chains
// of phase B at once, each from its own carry: the first half's comes from the left lane
// (as in team_run_pipe), the second half's is the first half's D-hat at its last column,
// formed after the scan.  The lane's scan aggregate joins the two half chains with
// g^(N/2).  Phase A is not a separate pass here: row i's partials U and insertions J are
// formed column by column inside phase B of row i, from row i - 1's M (the value the D-hat
// chain reads anyway) and J, so no partials array is kept between rows (32 registers at
// N = 32); the scan's latency is then left to the other warps.  Same results as
// team_run_pipe up to rounding order.
// ------------------------------------------------------------------------------------
// Asynchronous 16-byte copy global -> shared through L2 only (cp.async.cg: the source was
// written by this warp's previous strip with L2-only stores, so L1 may hold stale lines),
// and the group bookkeeping around it.
__device__ __forceinline__ void cp_async16_cg(void* smem_dst, const void* gmem_src) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(smem_dst);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(d), "l"(gmem_src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_1() { asm volatile("cp.async.wait_group 1;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_0() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }

// float2 FMA / multiply as one packed instruction (PACKED) or as two scalar ones (two
// independent dependency chains for the scheduler to interleave).
template <bool PACKED>
__device__ __forceinline__ float2 ffma2_sel(float2 a, float2 b, float2 c) {
    if constexpr (PACKED) return __ffma2_rn(a, b, c);
    else return make_float2(fmaf(a.x, b.x, c.x), fmaf(a.y, b.y, c.y));
}
template <bool PACKED>
__device__ __forceinline__ float2 fmul2_sel(float2 a, float2 b) {
    if constexpr (PACKED) return __fmul2_rn(a, b);
    else return make_float2(a.x * b.x, a.y * b.y);
}

// LINK: the team is a whole warp running one 32 N-column strip of a wider pair whose
// strips run one after another on this warp (the serial multi-warp kind).  As in
// seg_link_pipe<N, true>: the finished left strip's boundary (float4 per row: M, J, D-hat,
// E of its last column; `sin`) enters lane 0 and, as a carry g^(N t - 1), every lane's
// D-hat; checkpoints keep E >= E_left; lane 31 stores this strip's boundary (`sout`).
// The left boundary and the records are staged in shared memory (`stg`, `rstg`: two
// blocks of 32 rows each for this warp), each block copied asynchronously (cp.async, one
// row per lane) while the warp computes the 32 rows before it; every row then reads its
// boundary and record as broadcasts (no record is held in registers across a row).
// The lane's carry power g^(N lt - 1) stays in registers (reloaded when gcp changes):
// reading it from L1 every row measured 2% slower on the 1M-pair uneven batch.
// Progress of a strip of the wave kind (the rows whose boundary it has stored): released
// by its writer after those stores, acquired by the right neighbour before it copies them.
__device__ __forceinline__ unsigned long long ld_acquire_gpu(const unsigned long long* p) {
    unsigned long long v;
    asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_release_gpu(unsigned long long* p, unsigned long long v) {
    asm volatile("st.release.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
// Waits (bounded, with backoff) until the left strip has stored rows 1..need.
__device__ __forceinline__ bool wave_wait(const unsigned long long* p, unsigned long long need) {
    long long spins = 0;
    while (ld_acquire_gpu(p) < need) {
        if (++spins > kSpinLimit) return false;
        if (spins > kSpinFast) __nanosleep(64);
    }
    return true;
}

template <int N, bool PACKED, bool LINK = false, bool FUSE = LINK, bool L1P = false, bool WAVE = false>
__device__ SegOut team_run_pipe2(const Rec32J* __restrict__ rec, int l, int lmax,
                                 const uint8_t* __restrict__ hap, int k, int col0, int lt,
                                 int tlast, int nsteps, const PowRow<float>* __restrict__ pow_tab,
                                 const PipeRange& rng, const float4* sin = nullptr, float4* sout = nullptr,
                                 bool has_left = false, bool has_right = false, float4* stg = nullptr,
                                 float4* rstg = nullptr, const unsigned long long* prog_left = nullptr,
                                 unsigned long long* prog_me = nullptr, uint32_t* status = nullptr) {
    using NT = Num<float>;
    static_assert(N <= 32 && N % 2 == 0, "match masks hold 32 columns; two halves");
    static_assert(FUSE || !(LINK || L1P), "the serial strips and the L1 tables need the fused row");
    static_assert(LINK || !WAVE, "the wave kind runs strips in link mode");
    constexpr int H = N / 2;
    uint32_t bmA = 0, bmC = 0, bmG = 0, bmT = 0, flags = rng.ok ? 0u : PF_DEGEN, mflags = 0;
    const int nvalid = max(0, min(k - col0, N));
#pragma unroll
    for (int c = 0; c < N; ++c) {
        if (c < nvalid) {
            const int code = base_code(hap[col0 + c]);
            // match bits in the order phase B reads them: bit 2q for column q of the first
            // half, bit 2q + 1 for column H + q of the second
            const uint32_t bit = 1u << (c < H ? 2 * c : 2 * (c - H) + 1);
            if (code < 0) flags |= PF_BAD;
            if (code == 0 || code == 4) bmA |= bit;
            if (code == 1 || code == 4) bmC |= bit;
            if (code == 2 || code == 4) bmG |= bit;
            if (code == 3 || code == 4) bmT |= bit;
        }
    }
    float2 M2[H], J2[H];  // .x: column q, .y: column H + q of the lane
    float2 U2[FUSE ? 1 : H];  // unfused: row i + 1's partials, formed after row i's scan
    int E = 120 - rng.target;    // see team_run_pipe's cinit
    float2 dt2 = make_float2(0.f, 0.f), ml2 = make_float2(0.f, 0.f);
    float nj = 0.f;  // J of row i - 1 at the column before the lane (previous lane's last)
    float gprev = 0.f;
    float sp1[5], sp2[5], last1 = 0.f, last2 = 0.f, hh1 = 0.f, hh2 = 0.f, hm1 = 0.f, hm2 = 0.f;
    int gcp = -1;
    float qa1 = 0.f, qa2 = 0.f;
    float lsc = 1.f;  // LINK: 2^(E_left - E), constant between checkpoints
    const int l1 = max(l, 1) - 1;
    if constexpr (LINK) {
        // block 0 (rows 1..32): records and, with a left strip, its boundary rows
        const float4* src = reinterpret_cast<const float4*>(rec + min(lt, l1));
        cp_async16_cg(rstg + 2 * lt, src);
        cp_async16_cg(rstg + 2 * lt + 1, src + 1);
        if constexpr (WAVE) {  // the left strip runs concurrently: its rows 1..32 first
            if (has_left && !wave_wait(prog_left, (unsigned long long)min(l, 32))) {
                flags |= PF_TIMEOUT;
                atomicOr(status, ST_TIMEOUT);
            }
        }
        if (has_left && lt + 1 <= l) cp_async16_cg(stg + lt, sin + lt);
        cp_async_commit();
        cp_async_wait_0();
        __syncwarp();
    }
    SegOut out;
    out.S = 0.0;
    out.E = 0;
    out.flags = 0;
    const float cinit = l > 0 && k > 0 ? (float)(ldexp(1.0, rng.target) / (double)k) : 0.f;
    Rec32J cur;
    if constexpr (!LINK && !L1P) cur = load_recj(rec);
    int until = 0;
    for (int i = 1; i <= lmax; ++i) {
        Rec32J nxt;
        if constexpr (LINK) {
            // Stage blocks of 32 rows (records and left boundary), two buffers: block b + 1
            // is copied while block b is computed; at block b's first row the warp waits
            // for block b (issued 32 rows earlier) and then issues block b + 1.  Row i
            // sits in slot (i - 1) mod 64 of the two buffers taken together.
            const int slot = (i - 1) & 63;
            if ((slot & 31) == 0) {
                cp_async_wait_0();
                __syncwarp();  // block b has landed; every lane is done with block b - 1's buffer
                const int r = i + 32 + lt;
                const int ns = (slot + 32 + lt) & 63;  // row r's slot
                const float4* src = reinterpret_cast<const float4*>(rec + min(r - 1, l1));
                cp_async16_cg(rstg + 2 * ns, src);
                cp_async16_cg(rstg + 2 * ns + 1, src + 1);
                if constexpr (WAVE) {  // the next block's rows of the concurrent left strip
                    if (has_left && i + 32 <= l && !wave_wait(prog_left, (unsigned long long)min(l, i + 63))) {
                        flags |= PF_TIMEOUT;
                        atomicOr(status, ST_TIMEOUT);
                    }
                }
                if (has_left && r <= l) cp_async16_cg(stg + ns, sin + (r - 1));
                cp_async_commit();
            }
            const float4 a = rstg[2 * slot], b = rstg[2 * slot + 1];
            cur.pm = a.x; cur.px = a.y; cur.a = a.z; cur.b = a.w;
            cur.h = b.x; cur.g = b.y; cur.mi = b.z; cur.meta = __float_as_uint(b.w);
        } else if constexpr (L1P) {
            // the row's record from L1 at the row's start; a few rows ahead are prefetched
            const Rec32J* rp = rec + min(i - 1, l1);
            cur = load_recj(rp);
            asm volatile("prefetch.global.L1 [%0];" ::"l"(rec + min(i + 7, l1)));
        } else {
            nxt = cur;
            if (i < lmax) nxt = load_recj(rec + min(i, l1));
        }
        const uint32_t meta = cur.meta;
        mflags |= meta;
        const int gq = (int)((meta >> META_GCP_SHIFT) & 0xffu);
        const PowRow<float>* pr = pow_tab + min(gq, kMaxPhred);
        if constexpr (L1P) {
            // carry powers read from L1 where they are used (no registers across the row)
            if constexpr (LINK) {
                if (gq != gcp) {
                    qa1 = __ldg(&pr->lq1[lt]);
                    qa2 = __ldg(&pr->lq2[lt]);
                    gcp = gq;
                }
            }
        } else if (LINK ? __any_sync(kFull, gq != gcp) : gq != gcp) {
            // (link mode: every lane holds the same row, so the vote is exact and the
            // branch is warp-uniform)
#pragma unroll
            for (int s = 0; s < 5; ++s) {
                sp1[s] = lt >= (1 << s) ? __ldg(&pr->sp1[s]) : 0.f;
                sp2[s] = __ldg(&pr->sp2[s]);
            }
            last1 = (!LINK || lt >= 2) ? __ldg(&pr->last1) : 0.f;  // link: zz of lanes 0, 1 drops out
            last2 = __ldg(&pr->last2);
            hh1 = __ldg(&pr->hh1);
            hh2 = __ldg(&pr->hh2);
            hm1 = __ldg(&pr->hm1);
            hm2 = __ldg(&pr->hm2);
            if constexpr (LINK) {
                qa1 = __ldg(&pr->lq1[lt]);
                qa2 = __ldg(&pr->lq2[lt]);
            }
            gcp = gq;
        }
        // the row's carry powers: registers, or L1 reads at their use
        const auto P_sp1 = [&](int s) { if constexpr (L1P) return lt >= (1 << s) ? __ldg(&pr->sp1[s]) : 0.f; else return sp1[s]; };
        const auto P_sp2 = [&](int s) { if constexpr (L1P) return __ldg(&pr->sp2[s]); else return sp2[s]; };
        const auto P_last1 = [&]() { if constexpr (L1P) return __ldg(&pr->last1); else return last1; };
        const auto P_last2 = [&]() { if constexpr (L1P) return __ldg(&pr->last2); else return last2; };
        const auto P_hh1 = [&]() { if constexpr (L1P) return __ldg(&pr->hh1); else return hh1; };
        const auto P_hh2 = [&]() { if constexpr (L1P) return __ldg(&pr->hh2); else return hh2; };
        const auto P_hm1 = [&]() { if constexpr (L1P) return __ldg(&pr->hm1); else return hm1; };
        const auto P_hm2 = [&]() { if constexpr (L1P) return __ldg(&pr->hm2); else return hm2; };
        const int code = (int)(meta & META_CODE_MASK);
        const uint32_t mask = code == 0 ? bmA : code == 1 ? bmC : code == 2 ? bmG
                            : code == 3 ? bmT : 0xffffffffu;
        const float pim = cur.pm, pix = cur.px, rg = cur.g;
        const float2 rg2 = make_float2(rg, rg);
        float2 y2 = make_float2(0.f, 0.f), yp2 = make_float2(0.f, 0.f);
        // phase B (both halves at once)
        if (i == 1) {
#pragma unroll
            for (int q = 0; q < H; ++q) {
                const float2 mn = make_float2((((mask >> (2 * q)) & 1u) ? pim : pix) * cinit,
                                              (((mask >> (2 * q + 1)) & 1u) ? pim : pix) * cinit);
                M2[q] = mn;
                J2[q] = make_float2(0.f, 0.f);
                if (q == H - 1) yp2 = y2;
                y2 = ffma2_sel<PACKED>(rg2, y2, mn);
            }
        } else if constexpr (!FUSE) {
            const float2 rb2 = make_float2(cur.b, cur.b), gp2 = make_float2(gprev, gprev);
#pragma unroll
            for (int q = 0; q < H; ++q) {
                const float2 u2 = ffma2_sel<PACKED>(rb2, dt2, U2[q]);
                dt2 = ffma2_sel<PACKED>(gp2, dt2, ml2);
                ml2 = M2[q];
                const float2 p2 = make_float2(((mask >> (2 * q)) & 1u) ? pim : pix,
                                              ((mask >> (2 * q + 1)) & 1u) ? pim : pix);
                const float2 mn = fmul2_sel<PACKED>(p2, u2);
                M2[q] = mn;
                if (q == H - 1) yp2 = y2;
                y2 = ffma2_sel<PACKED>(rg2, y2, mn);
            }
        } else {
            // Row i's partials U = a M' + J' and insertions J = M' + h J' (primes: row
            // i - 1, from the column before for U, the same column for J) are formed
            // column by column as phase B reaches them, from the old M and J.  Row i - 1's
            // D-hat chain runs one column ahead (dA: the D-hat of the column before q; dB:
            // that of column q, formed from column q - 1's old M), so column q's old M and
            // J have their last uses (dB, column q + 1's partial, column q's J) before
            // column q's new M is formed, and the new values take the old ones' registers.
            const float2 rb2 = make_float2(cur.b, cur.b), gp2 = make_float2(gprev, gprev);
            const float2 na2 = make_float2(cur.a, cur.a), nh2 = make_float2(cur.h, cur.h);
            float2 uq = ffma2_sel<PACKED>(na2, ml2, make_float2(nj, J2[H - 1].x));
            float2 dA = dt2, dB = ffma2_sel<PACKED>(gp2, dt2, ml2);
#pragma unroll
            for (int q = 0; q < H; ++q) {
                const float2 u2 = ffma2_sel<PACKED>(rb2, dA, uq);
                const float2 mo = M2[q];
                if (q + 1 < H) {
                    dA = dB;
                    dB = ffma2_sel<PACKED>(gp2, dB, mo);
                    uq = ffma2_sel<PACKED>(na2, mo, J2[q]);
                }
                J2[q] = ffma2_sel<PACKED>(nh2, J2[q], mo);
                const float2 p2 = make_float2(((mask >> (2 * q)) & 1u) ? pim : pix,
                                              ((mask >> (2 * q + 1)) & 1u) ? pim : pix);
                const float2 mn = fmul2_sel<PACKED>(p2, u2);
                M2[q] = mn;
                if (q == H - 1) yp2 = y2;
                y2 = ffma2_sel<PACKED>(rg2, y2, mn);
            }
        }
        // Eq. 4 when a pair of this warp finishes (I = T_MI J on the last row); a strip
        // of the serial kind is one pair on the whole warp
        bool ends;
        if constexpr (LINK) ends = false;  // one pair on the whole warp: summed after the loop
        else ends = __any_sync(kFull, i == l);
        if (ends) {
            const double rmi = (double)cur.mi;
            double s = 0.0;
#pragma unroll
            for (int q = 0; q < H; ++q) {
                if (q < nvalid) s += (double)M2[q].x + rmi * (double)J2[q].x;
                if (q + H < nvalid) s += (double)M2[q].y + rmi * (double)J2[q].y;
            }
            s = team_sum<double>(s, lt, tlast, nsteps);
            uint32_t f = flags;
            if (mflags & META_BAD) f |= PF_BAD;
            if (mflags & META_DEGEN) f |= PF_DEGEN;
            f = team_or(f, lt, tlast, nsteps);
            if (i == l) {
                out.S = s;
                out.E = E;
                out.flags = f;
            }
        }
        // lane aggregates of the local (zero-carry) D-hat chain: one past the lane's last
        // column (scan input) and at its last column (the right neighbour's carry)
        const float zl = fmaf(y2.x * P_hh1(), P_hh2(), y2.y);
        float ypl = fmaf(y2.x * P_hm1(), P_hm2(), yp2.y);
        float jl = 0.f;
        if constexpr (LINK) jl = J2[H - 1].y;  // this lane's last J of row i (sent right)
        float yA = yp2.x;  // first half, at its last column
        float nm = __shfl_up_sync(kFull, M2[H - 1].y, 1);
        nj = __shfl_up_sync(kFull, J2[H - 1].y, 1);
        float yp = __shfl_up_sync(kFull, ypl, 1);
        if (!LINK && lt == 0) {  // link mode replaces lane 0's three after the checkpoint
            nm = 0.f;
            nj = 0.f;
            yp = 0.f;
        }
        float Z = zl;
#pragma unroll
        for (int s = 0; s < 5; ++s) {
            const float up = __shfl_up_sync(kFull, Z, 1 << s);
            Z = fmaf(up * P_sp1(s), P_sp2(s), Z);
        }
        if constexpr (!FUSE) {  // phase A: row i + 1's partials and insertions
            const float2 na2 = make_float2(nxt.a, nxt.a), nh2 = make_float2(nxt.h, nxt.h);
            const float mal = M2[H - 1].x, jal = J2[H - 1].x;
#pragma unroll
            for (int q = H - 1; q >= 1; --q) {
                U2[q] = ffma2_sel<PACKED>(na2, M2[q - 1], J2[q - 1]);
                J2[q] = ffma2_sel<PACKED>(nh2, J2[q], M2[q]);
            }
            U2[0] = ffma2_sel<PACKED>(na2, make_float2(nm, mal), make_float2(nj, jal));
            J2[0] = ffma2_sel<PACKED>(nh2, J2[0], M2[0]);
        }
        float zz = __shfl_up_sync(kFull, Z, 2);
        if ((!LINK || L1P) && lt < 2) zz = 0.f;
        if constexpr (LINK) {
            // one broadcast read, taken with or without a left strip (without one the slot is
            // stale and only selected away: no branch in the row)
            const float4 v = stg[(i - 1) & 63];
            float lM = has_left ? v.x : 0.f, lJ = has_left ? v.y : 0.f, lD = has_left ? v.z : 0.f;
            const int Eleft = has_left ? __float_as_int(v.w) : INT_MIN;
            // checkpoint (same rows in every strip of the pair): E >= E_left, so that left
            // values only ever scale down
            int Enew = E;
            if (until == 0) {
                until = rng.R;
                float2 m2 = make_float2(0.f, 0.f);
#pragma unroll
                for (int q = 0; q < H; ++q) {
                    m2.x = fmaxf(m2.x, fmaxf(fabsf(M2[q].x), fabsf(J2[q].x)));
                    m2.y = fmaxf(m2.y, fmaxf(fabsf(M2[q].y), fabsf(J2[q].y)));
                }
                // the strip is the whole warp: one reduction over the lanes' maxima (values
                // >= 0, so their bit patterns order like the values)
                const float m = __uint_as_float(__reduce_max_sync(kFull, __float_as_uint(fmaxf(m2.x, m2.y))));
                const int e = NT::expo(m);
                int desired = E;
                if (e == INT_MAX) {
                    flags |= PF_NONFINITE;
                } else if (e == INT_MIN) {
                    if (has_left) desired = INT_MIN;  // nothing representable: follow the left
                } else if (e > rng.hi || e <= NT::kLo) {
                    desired = E + (e - rng.target);
                }
                Enew = desired;
                bool forced = false;
                if (has_left && Eleft > Enew) {
                    Enew = Eleft;
                    forced = true;
                }
                if (Enew == INT_MIN) Enew = E;
                if (!forced && e != INT_MIN && e != INT_MAX && e <= rng.danger) flags |= PF_DANGER;
                if (Enew != E) {  // only a checkpoint row changes the exponent
                    const int sdn = E - Enew;
#pragma unroll
                    for (int q = 0; q < H; ++q) {
                        M2[q] = make_float2(scale2(M2[q].x, sdn), scale2(M2[q].y, sdn));
                        J2[q] = make_float2(scale2(J2[q].x, sdn), scale2(J2[q].y, sdn));
                    }
                    nm = scale2(nm, sdn);
                    nj = scale2(nj, sdn);
                    zz = scale2(zz, sdn);
                    yp = scale2(yp, sdn);
                    yA = scale2(yA, sdn);
                    ypl = scale2(ypl, sdn);
                    jl = scale2(jl, sdn);
                    flags |= PF_RESCALED;
                    E = Enew;
                }
                // both exponents change only on checkpoint rows (the same rows in every
                // strip of the pair), so the left values' scale 2^(E_left - E) <= 1 is
                // formed here (exactly, subnormal or zero below 2^-126) and kept
                const int dsh = has_left ? Eleft - E : 0;
                lsc = dsh >= -126 ? NT::pow2(dsh) : dsh >= -149 ? __uint_as_float(1u << (dsh + 149)) : 0.f;
            }
            --until;
            // left values into this strip's scale (no left: zeros stay zero)
            lM *= lsc;
            lJ *= lsc;
            lD *= lsc;
            const float Wseg = fmaf(rg, lD, lM);  // D-hat at the strip's first column
            float ndA = fmaf(zz * P_last1(), P_last2(), yp);
            ndA = fmaf(Wseg * qa1, qa2, ndA);
            if (lt == 0) {
                ndA = lD;
                nm = lM;
                nj = lJ;
            }
            if (has_right && lt == 31) {
                // D-hat at the strip's last column: the lane's own chain from ndA (the
                // column before it, carry included) over its N columns, g^N ndA + ypl
                const float dl = fmaf((ndA * rg) * P_last1(), P_last2(), ypl);
                __stcg(sout + (i - 1), make_float4(M2[H - 1].y, jl, dl, __int_as_float(E)));
                if constexpr (WAVE) {  // rows 1..i stored: publish at block ends and the last row
                    if ((i & 31) == 0 || i == l) st_release_gpu(prog_me, (unsigned long long)i);
                }
            }
            const float wl = fmaf(rg, ndA, nm);         // D-hat at the lane's first column
            const float ndB = fmaf(wl * P_hm1(), P_hm2(), yA);  // D-hat at the first half's last column
            dt2 = make_float2(ndA, ndB);
            ml2 = make_float2(nm, M2[H - 1].x);
            gprev = rg;
            continue;
        }
        if (until == 0) {
            until = rng.R;
            float2 m2 = make_float2(0.f, 0.f);
#pragma unroll
            for (int q = 0; q < H; ++q) {
                m2.x = fmaxf(m2.x, fmaxf(fabsf(M2[q].x), fabsf(J2[q].x)));
                m2.y = fmaxf(m2.y, fmaxf(fabsf(M2[q].y), fabsf(J2[q].y)));
            }
            const float m = team_max_pos(fmaxf(m2.x, m2.y), lt, tlast);
            const int e = NT::expo(m);
            if (e == INT_MAX) {
                flags |= PF_NONFINITE;
            } else if (e != INT_MIN) {
                if (e <= rng.danger) flags |= PF_DANGER;
                if (e > rng.hi || e <= NT::kLo) {
                    const int sh = e - rng.target;
                    float f1 = 1.f, f2v;
                    if (sh >= -126 && sh <= 126) {
                        f2v = NT::pow2(-sh);
                    } else {
                        f1 = NT::pow2((-sh) / 2);
                        f2v = NT::pow2(-sh - (-sh) / 2);
                    }
                    const float2 a2 = make_float2(f1, f1), b2 = make_float2(f2v, f2v);
#pragma unroll
                    for (int q = 0; q < H; ++q) {
                        M2[q] = fmul2_sel<PACKED>(fmul2_sel<PACKED>(M2[q], a2), b2);
                        J2[q] = fmul2_sel<PACKED>(fmul2_sel<PACKED>(J2[q], a2), b2);
                        if constexpr (!FUSE) U2[q] = fmul2_sel<PACKED>(fmul2_sel<PACKED>(U2[q], a2), b2);
                    }
                    nm = (nm * f1) * f2v;
                    nj = (nj * f1) * f2v;
                    zz = (zz * f1) * f2v;
                    yp = (yp * f1) * f2v;
                    yA = (yA * f1) * f2v;
                    flags |= PF_RESCALED;
                    E += sh;
                }
            }
        }
        --until;
        const float ndA = fmaf(zz * P_last1(), P_last2(), yp);  // D-hat at the column before the lane
        const float wl = fmaf(rg, ndA, nm);                      // D-hat at the lane's first column
        const float ndB = fmaf(wl * P_hm1(), P_hm2(), yA);       // D-hat at the first half's last column
        dt2 = make_float2(ndA, ndB);
        ml2 = make_float2(nm, M2[H - 1].x);
        gprev = rg;
        if constexpr (!LINK && !L1P) cur = nxt;
    }
    if constexpr (LINK) {
        cp_async_wait_0();  // nothing may land in the stage after this strip
        // Eq. 4 on the pair's last row l (= lmax; a checkpoint on it rescaled M, J and E
        // together, and its flags count)
        const double rmi = (double)cur.mi;
        double s = 0.0;
#pragma unroll
        for (int q = 0; q < H; ++q) {
            if (q < nvalid) s += (double)M2[q].x + rmi * (double)J2[q].x;
            if (q + H < nvalid) s += (double)M2[q].y + rmi * (double)J2[q].y;
        }
        s = team_sum<double>(s, lt, tlast, nsteps);
        uint32_t f = flags;
        if (mflags & META_BAD) f |= PF_BAD;
        if (mflags & META_DEGEN) f |= PF_DEGEN;
        out.S = s;
        out.E = E;
        out.flags = team_or(f, lt, tlast, nsteps);
    }
    return out;
}

// ------------------------------------------------------------------------------------
// Pipelined FP32 engine for one warp segment of a multi-warp pair (32 N columns, all 32
// lanes; rows 1..l).  The row work is team_run_pipe's; the segment exchange is
// seg_run<LINKED>'s: after the scan and phase A of row i, lane 0 takes the left segment's
// (M, J, D-hat, E) of its last column for row i (shared-memory ring, or the global
// boundary of the previous strip), the checkpoint keeps E >= E_left, the left values are
// brought into this segment's scale, and lane 31 hands this segment's last column on.
// The segment carry enters lane t's previous column with the power g^(N t - 1).
// ------------------------------------------------------------------------------------
template <int N>
__device__ SegOut seg_link_pipe(const Rec32J* __restrict__ rec, int l, const uint8_t* __restrict__ hap,
                                int k, int col0, int lane, const PowRow<float>* __restrict__ pow_tab,
                                const PipeRange& rng, const SmemLink& link, uint32_t* __restrict__ status) {
    using NT = Num<float>;
    static_assert(N <= 32, "match masks hold 32 columns");
    uint32_t bmA = 0, bmC = 0, bmG = 0, bmT = 0, flags = rng.ok ? 0u : PF_DEGEN, mflags = 0;
    const int nvalid = max(0, min(k - col0, N));
    const bool has_left = link.has_left, has_right = link.has_right;
#pragma unroll
    for (int c = 0; c < N; ++c) {
        if (c < nvalid) {
            const int code = base_code(hap[col0 + c]);
            const uint32_t bit = 1u << c;
            if (code < 0) flags |= PF_BAD;
            if (code == 0 || code == 4) bmA |= bit;
            if (code == 1 || code == 4) bmC |= bit;
            if (code == 2 || code == 4) bmG |= bit;
            if (code == 3 || code == 4) bmT |= bit;
        }
    }
    float M[N], J[N], U[N];
    int E = 120 - rng.target;  // see team_run_pipe's cinit
    float ml = 0.f, dt = 0.f, gprev = 0.f;
    float sp1[5], sp2[5], last1 = 0.f, last2 = 0.f, qa1 = 0.f, qa2 = 0.f, qb1 = 0.f, qb2 = 0.f;
    int gcp = -1;
    SegOut out;
    out.S = 0.0;
    out.E = 0;
    out.flags = 0;
    const float cinit = l > 0 && k > 0 ? (float)(ldexp(1.0, rng.target) / (double)k) : 0.f;
    const int l1 = max(l, 1) - 1;
    Rec32J cur = load_recj(rec);
    int until = 0;
    for (int i = 1; i <= l; ++i) {
        Rec32J nxt = cur;
        if (i < l) nxt = load_recj(rec + min(i, l1));
        const uint32_t meta = cur.meta;
        mflags |= meta;
        const int gq = (int)((meta >> META_GCP_SHIFT) & 0xffu);
        if (gq != gcp) {
            const PowRow<float>* pr = pow_tab + min(gq, kMaxPhred);
#pragma unroll
            for (int s = 0; s < 5; ++s) {
                sp1[s] = lane >= (1 << s) ? __ldg(&pr->sp1[s]) : 0.f;
                sp2[s] = __ldg(&pr->sp2[s]);
            }
            last1 = __ldg(&pr->last1);
            last2 = __ldg(&pr->last2);
            qa1 = __ldg(&pr->lq1[lane]);      // g^(N lane - 1) (lane 0: unused)
            qa2 = __ldg(&pr->lq2[lane]);
            qb1 = __ldg(&pr->lq1[lane + 1]);  // g^(N (lane + 1) - 1): this lane's last column
            qb2 = __ldg(&pr->lq2[lane + 1]);
            gcp = gq;
        }
        const int code = (int)(meta & META_CODE_MASK);
        const uint32_t mask = code == 0 ? bmA : code == 1 ? bmC : code == 2 ? bmG
                            : code == 3 ? bmT : 0xffffffffu;
        const float pim = cur.pm, pix = cur.px, rg = cur.g;
        float y = 0.f, yprev = 0.f;
        // phase B
        if (i == 1) {
#pragma unroll
            for (int c = 0; c < N; ++c) {
                M[c] = (((mask >> c) & 1u) ? pim : pix) * cinit;
                J[c] = 0.f;
                if (c == N - 1) yprev = y;
                y = fmaf(rg, y, M[c]);
            }
        } else {
            const float rb = cur.b;
#pragma unroll
            for (int c = 0; c < N; ++c) {
                const float u = fmaf(rb, dt, U[c]);
                dt = fmaf(gprev, dt, ml);
                ml = M[c];
                const float mn = (((mask >> c) & 1u) ? pim : pix) * u;
                M[c] = mn;
                if (c == N - 1) yprev = y;
                y = fmaf(rg, y, mn);
            }
        }
        // Eq. 4 on the last row (I = T_MI J); all lanes of the warp run the same pair
        if (i == l) {
            const double rmi = (double)cur.mi;
            double s = 0.0;
#pragma unroll
            for (int c = 0; c < N; ++c)
                if (c < nvalid) s += (double)M[c] + rmi * (double)J[c];
            s = team_sum<double>(s, lane, 31, 5);
            uint32_t f = flags;
            if (mflags & META_BAD) f |= PF_BAD;
            if (mflags & META_DEGEN) f |= PF_DEGEN;
            f = team_or(f, lane, 31, 5);
            out.S = s;
            out.E = E;
            out.flags = f;
        }
        // deletion scan of row i, phase A of row i+1 (all but lane 0's first partial)
        float nm = __shfl_up_sync(kFull, M[N - 1], 1);
        float nj = __shfl_up_sync(kFull, J[N - 1], 1);
        float yp = __shfl_up_sync(kFull, yprev, 1);
        float jl = J[N - 1];  // this segment's last J of row i (sent right)
        float Z = y;
#pragma unroll
        for (int s = 0; s < 5; ++s) {
            const float up = __shfl_up_sync(kFull, Z, 1 << s);
            Z = fmaf(up * sp1[s], sp2[s], Z);
        }
        const float na = nxt.a, nh = nxt.h;
        {
#pragma unroll
            for (int c = N - 1; c >= 1; --c) {
                U[c] = fmaf(na, M[c - 1], J[c - 1]);
                J[c] = fmaf(nh, J[c], M[c]);
            }
            U[0] = fmaf(na, nm, nj);  // lane 0: replaced from the left segment below
            J[0] = fmaf(nh, J[0], M[0]);
        }
        float zz = __shfl_up_sync(kFull, Z, 2);
        float Wd = __shfl_up_sync(kFull, Z, 1);
        if (lane < 2) zz = 0.f;
        if (lane == 0) {
            Wd = 0.f;
            yp = 0.f;
        }
        // the left segment's last column of row i: lane 0 waits for it, then the whole
        // (converged) warp takes it
        float lM = 0.f, lJ = 0.f, lD = 0.f;
        int e_in = INT_MIN;
        if (has_left && lane == 0) {
            const bool ok = link.in_g ? link_recv_g<float>(link.in_g, i, lM, lJ, lD, e_in)
                                      : link_recv<float>(link, i, lM, lJ, lD, e_in);
            if (!ok) {
                flags |= PF_TIMEOUT;
                atomicOr(status, ST_TIMEOUT);
            }
        }
        __syncwarp();
        lM = __shfl_sync(kFull, lM, 0);
        lJ = __shfl_sync(kFull, lJ, 0);
        lD = __shfl_sync(kFull, lD, 0);
        const int Eleft = __shfl_sync(kFull, e_in, 0);
        // checkpoint (same rows in every segment of the pair): power-of-two rescaling,
        // with E >= E_left so that left values only ever scale down
        int Enew = E;
        if (until == 0) {
            until = rng.R;
            float m = 0.f;
#pragma unroll
            for (int c = 0; c < N; ++c) m = fmaxf(m, fmaxf(fabsf(M[c]), fabsf(J[c])));
            m = team_max_pos(m, lane, 31);
            const int e = NT::expo(m);
            int desired = E;
            if (e == INT_MAX) {
                if (i <= l) flags |= PF_NONFINITE;
            } else if (e == INT_MIN) {
                // nothing representable here: follow the left neighbour's scale
                if (has_left) desired = INT_MIN;
            } else if (e > rng.hi || e <= NT::kLo) {
                desired = E + (e - rng.target);
            }
            Enew = desired;
            bool forced = false;
            if (has_left && Eleft > Enew) {
                Enew = Eleft;
                forced = true;
            }
            if (Enew == INT_MIN) Enew = E;
            if (!forced && e != INT_MIN && e <= rng.danger) flags |= PF_DANGER;
        }
        --until;
        if (Enew != E) {
            const int sdn = E - Enew;
#pragma unroll
            for (int c = 0; c < N; ++c) {
                M[c] = scale2(M[c], sdn);
                J[c] = scale2(J[c], sdn);
                U[c] = scale2(U[c], sdn);
            }
            nm = scale2(nm, sdn);
            yp = scale2(yp, sdn);
            zz = scale2(zz, sdn);
            Wd = scale2(Wd, sdn);
            yprev = scale2(yprev, sdn);
            jl = scale2(jl, sdn);
            flags |= PF_RESCALED;
            E = Enew;
        }
        // left values into this segment's scale (E >= E_left here; no left: zeros stay zero)
        const int dsh = has_left ? Eleft - E : 0;
        if (dsh != 0) {  // warp-uniform; the scales differ only after a checkpoint
            lM = scale2(lM, dsh);
            lJ = scale2(lJ, dsh);
            lD = scale2(lD, dsh);
        }
        const float Wseg = fmaf(rg, lD, lM);  // D-hat at the segment's first column
        // D-hat at the column before this lane: the left lanes' part plus the carry
        float nd = fmaf(zz * last1, last2, yp);
        nd = fmaf(Wseg * qa1, qa2, nd);
        if (lane == 0) {
            nd = lD;
            nm = lM;
            U[0] = fmaf(na, lM, lJ);
        }
        if (has_right && lane == 31) {
            // D-hat at the segment's last column
            const float dl = fmaf(Wseg * qb1, qb2, fmaf(Wd * last1, last2, yprev));
            if (link.out_g) {
                link_send_g<float>(link.out_g, i, M[N - 1], jl, dl, E);
            } else if (!link_send<float>(link, i, M[N - 1], jl, dl, E)) {
                flags |= PF_TIMEOUT;
                atomicOr(status, ST_TIMEOUT);
            }
        }
        ml = nm;
        dt = nd;
        gprev = rg;
        cur = nxt;
    }
    return out;
}

// ------------------------------------------------------------------------------------
// Packed FP32 team for two haplotypes of the SAME read (pair A in x, pair B in y halves).
// Both halves share the row records and the scan powers, so the per-row work is that of
// one pair while every cell operation (FFMA2 / FMUL2) serves two cells.  Match masks of
// both haplotypes live in one register per base (bits 0..15: A, 16..31: B; N <= 16).
// ------------------------------------------------------------------------------------
template <int N>
__device__ PairOut2 team_run_sr2(const Rec32* __restrict__ rec, int l, int lmax,
                                 const uint8_t* __restrict__ hapA, int kA,
                                 const uint8_t* __restrict__ hapB, int kB, int col0, int lt,
                                 int tlast, int nsteps, const PowRow<float>* __restrict__ pow_tab,
                                 int R) {
    using NT = Num<float>;
    static_assert(N <= 16, "two 16-bit match masks per register");
    uint32_t mA = 0, mC = 0, mG = 0, mT = 0, flA = 0, flB = 0, mflags = 0;
    const int nvA = max(0, min(kA - col0, N)), nvB = max(0, min(kB - col0, N));
#pragma unroll
    for (int c = 0; c < N; ++c) {
        if (c < nvA) {
            const int code = base_code(hapA[col0 + c]);
            const uint32_t bit = 1u << c;
            if (code < 0) flA |= PF_BAD;
            if (code == 0 || code == 4) mA |= bit;
            if (code == 1 || code == 4) mC |= bit;
            if (code == 2 || code == 4) mG |= bit;
            if (code == 3 || code == 4) mT |= bit;
        }
        if (c < nvB) {
            const int code = base_code(hapB[col0 + c]);
            const uint32_t bit = 1u << (c + 16);
            if (code < 0) flB |= PF_BAD;
            if (code == 0 || code == 4) mA |= bit;
            if (code == 1 || code == 4) mC |= bit;
            if (code == 2 || code == 4) mG |= bit;
            if (code == 3 || code == 4) mT |= bit;
        }
    }
    float2 M[N], I[N];
    int EA = 0, EB = 0;
    float2 ml = f2(0.f, 0.f), sl = f2(0.f, 0.f), dt = f2(0.f, 0.f);
    float gprev = 0.f;
    float sp1[5], sp2[5], last1 = 0.f, last2 = 0.f;
    int gcp = -1;
    const float2 cinit = f2(l > 0 && kA > 0 ? (float)(0x1p120 / (double)kA) : 0.f,
                            l > 0 && kB > 0 ? (float)(0x1p120 / (double)kB) : 0.f);
    PairOut2 out;
    out.a = {0.0, 0, 0};
    out.b = {0.0, 0, 0};
    const int l1 = max(l, 1) - 1;
    Rec32 cur = load_rec(rec);
    int until = 0;
    for (int i = 1; i <= lmax; ++i) {
        Rec32 nxt = cur;
        if (i < lmax) nxt = load_rec(rec + min(i, l1));
        const uint32_t meta = cur.meta;
        mflags |= meta;
        const int gq = (int)((meta >> META_GCP_SHIFT) & 0xffu);
        if (gq != gcp) {
            const PowRow<float>* pr = pow_tab + min(gq, kMaxPhred);
#pragma unroll
            for (int s = 0; s < 5; ++s) {
                sp1[s] = __ldg(&pr->sp1[s]);
                sp2[s] = __ldg(&pr->sp2[s]);
            }
            last1 = __ldg(&pr->last1);
            last2 = __ldg(&pr->last2);
            gcp = gq;
        }
        const int code = (int)(meta & META_CODE_MASK);
        const uint32_t mask = code == 0 ? mA : code == 1 ? mC : code == 2 ? mG
                            : code == 3 ? mT : 0xffffffffu;
        const float pim = cur.pm, pix = cur.px, g = cur.g;
        const float2 rg = f2(g, g);
        float2 y = f2(0.f, 0.f), yprev = f2(0.f, 0.f);
        if (i == 1) {
#pragma unroll
            for (int c = 0; c < N; ++c) {
                const float2 p = f2(((mask >> c) & 1u) ? pim : pix, ((mask >> (c + 16)) & 1u) ? pim : pix);
                M[c] = __fmul2_rn(p, cinit);
                I[c] = f2(0.f, 0.f);
                if (c == N - 1) yprev = y;
                y = __ffma2_rn(rg, y, M[c]);
            }
        } else {
            const float2 ra = f2(cur.a, cur.a), rb = f2(cur.b, cur.b), rmi = f2(cur.mi, cur.mi);
            const float2 gp = f2(gprev, gprev);
#pragma unroll
            for (int c = 0; c < N; ++c) {
                const float2 S = __ffma2_rn(rb, dt, sl);
                const float2 u = __ffma2_rn(ra, ml, S);
                const float2 p = f2(((mask >> c) & 1u) ? pim : pix, ((mask >> (c + 16)) & 1u) ? pim : pix);
                const float2 mn = __fmul2_rn(p, u);
                const float2 in = __ffma2_rn(rmi, M[c], __fmul2_rn(rg, I[c]));
                dt = __ffma2_rn(gp, dt, ml);
                ml = M[c];
                sl = I[c];
                M[c] = mn;
                I[c] = in;
                if (c == N - 1) yprev = y;
                y = __ffma2_rn(rg, y, mn);
            }
        }
        // Deletion scan over the team, both halves with the same powers.
        float zx = y.x, zy = y.y;
#pragma unroll
        for (int s = 0; s < 5; ++s) {
            if (s < nsteps) {
                const int off = 1 << s;
                const float ux = __shfl_up_sync(kFull, zx, off);
                const float uy = __shfl_up_sync(kFull, zy, off);
                if (lt >= off) {
                    zx = fmaf(ux * sp1[s], sp2[s], zx);
                    zy = fmaf(uy * sp1[s], sp2[s], zy);
                }
            }
        }
        float2 Wd = f2(__shfl_up_sync(kFull, zx, 1), __shfl_up_sync(kFull, zy, 1));
        if (lt == 0) Wd = f2(0.f, 0.f);
        if (until == 0) {
            until = R;
            float ma = 0.f, mb = 0.f;
#pragma unroll
            for (int c = 0; c < N; ++c) {
                ma = fmaxf(ma, fmaxf(fabsf(M[c].x), fabsf(I[c].x)));
                mb = fmaxf(mb, fmaxf(fabsf(M[c].y), fabsf(I[c].y)));
            }
            ma = team_max<float>(ma, lt, tlast, nsteps);
            mb = team_max<float>(mb, lt, tlast, nsteps);
            const int ea = NT::expo(ma), eb = NT::expo(mb);
            int sa = 0, sb = 0;
            if (ea == INT_MAX) flA |= PF_NONFINITE;
            else if (ea != INT_MIN) {
                if (ea <= NT::kDanger) flA |= PF_DANGER;
                if (ea > NT::kHi || ea <= NT::kLo) sa = ea - NT::kTarget;
            }
            if (eb == INT_MAX) flB |= PF_NONFINITE;
            else if (eb != INT_MIN) {
                if (eb <= NT::kDanger) flB |= PF_DANGER;
                if (eb > NT::kHi || eb <= NT::kLo) sb = eb - NT::kTarget;
            }
            if (sa != 0 || sb != 0) {
                const float2 f1 = f2(NT::pow2((-sa) / 2), NT::pow2((-sb) / 2));
                const float2 f2v = f2(NT::pow2(-sa - (-sa) / 2), NT::pow2(-sb - (-sb) / 2));
#pragma unroll
                for (int c = 0; c < N; ++c) {
                    M[c] = __fmul2_rn(__fmul2_rn(M[c], f1), f2v);
                    I[c] = __fmul2_rn(__fmul2_rn(I[c], f1), f2v);
                }
                Wd = __fmul2_rn(__fmul2_rn(Wd, f1), f2v);
                yprev = __fmul2_rn(__fmul2_rn(yprev, f1), f2v);
                if (sa) flA |= PF_RESCALED;
                if (sb) flB |= PF_RESCALED;
                EA += sa;
                EB += sb;
            }
        }
        --until;
        const float2 Dlast = f2(fmaf(Wd.x * last1, last2, yprev.x), fmaf(Wd.y * last1, last2, yprev.y));
        if (__any_sync(kFull, i == l)) {
            // lane sums in FP32 with compensation (two-sum), the team sum in FP64
            float sa = 0.f, ca = 0.f, sb = 0.f, cb = 0.f;
#pragma unroll
            for (int c = 0; c < N; ++c) {
                if (c < nvA) {
                    const df t = two_sum(sa, M[c].x + I[c].x);
                    sa = t.hi;
                    ca += t.lo;
                }
                if (c < nvB) {
                    const df t = two_sum(sb, M[c].y + I[c].y);
                    sb = t.hi;
                    cb += t.lo;
                }
            }
            const double da = team_sum<double>((double)sa + (double)ca, lt, tlast, nsteps);
            const double db = team_sum<double>((double)sb + (double)cb, lt, tlast, nsteps);
            uint32_t fa = flA, fb = flB;
            if (mflags & META_BAD) {
                fa |= PF_BAD;
                fb |= PF_BAD;
            }
            if (mflags & META_DEGEN) {
                fa |= PF_DEGEN;
                fb |= PF_DEGEN;
            }
            fa = team_or(fa, lt, tlast, nsteps);
            fb = team_or(fb, lt, tlast, nsteps);
            if (i == l) {
                out.a = {da, EA, fa};
                out.b = {db, EB, fb};
            }
        }
        float2 nm = shfl_up2(M[N - 1], 1), ni = shfl_up2(I[N - 1], 1), nd = shfl_up2(Dlast, 1);
        if (lt == 0) {
            nm = f2(0.f, 0.f);
            ni = f2(0.f, 0.f);
            nd = f2(0.f, 0.f);
        }
        ml = nm;
        sl = ni;
        dt = nd;
        gprev = g;
        cur = nxt;
    }
    return out;
}

}  // namespace phmm
