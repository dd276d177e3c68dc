// Internal data structures shared by the host runtime and the CUDA kernels of the
// row-wise PairHMM library.  Nothing here is part of the public C ABI (include/phmm.h).
#pragma once

#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>

namespace phmm {

// ----------------------------------------------------------------------------------
// Per read-row coefficient records, written by the prep kernels, one per read base,
// in the layout of the concatenated reads (record of row i of read r sits at
// read_off[r] + i - 1).
//
// FP32 record (factored form of Eq. 2 for row i, see engine.cuh):
//   pm = (1 - e_i)(1 - g_i), px = (e_i / 3)(1 - g_i)        match / mismatch factor
//   a  = T_MM_i / (1 - g_i)                                  M -> M over I/D weight
//   b  = T_MD_{i-1}                                          D-hat -> D of row i-1
//   mi = T_MI_i, g = T_II_i = T_DD_i, gm = 1 - g_i
// FP64 record (unfactored, robust for g = 1):
//   pm = 1 - e_i, px = e_i / 3, a = T_MM_i, b = T_MD_{i-1}, mi, g, gm as above.
// meta: bits 0..2 read base code (A=0 C=1 G=2 T=3 N=4), bits 8..15 gcp Phred
// (row of the power table), META_DEGEN, META_BAD.
// ----------------------------------------------------------------------------------
struct alignas(16) Rec32 {
    float pm, px, a, b, mi, g, gm;
    uint32_t meta;
};
struct alignas(16) Rec64 {
    double pm, px, a, b, mi, g, gm;
    uint64_t meta;
};
// FP32 record of the pipelined engine, which carries J_i = I_i / T_MI_i instead of I_i,
// so that Eq. 2's insertion update becomes J_ij = M_{i-1,j} + h_i J_{i-1,j} (one FMA) and
// the factor T_MI_{i-1} of the I term of the match update moves into the coefficients
// (mi_0 := 1 for the first row of a read):
//   pm = (1 - e_i)(1 - g_i) mi_{i-1},  px = (e_i / 3)(1 - g_i) mi_{i-1}
//   a  = T_MM_i / ((1 - g_i) mi_{i-1}),  b = T_MD_{i-1} / mi_{i-1}
//   h  = g_i mi_{i-1} / mi_i,  g = g_i,  mi = T_MI_i
// so that M_ij = P' (a M' + J' + b D-hat'), with the primes on row i-1, column j-1.
struct alignas(16) Rec32J {
    float pm, px, a, b, h, g, mi;
    uint32_t meta;
};
// The same J-form record in FP64, for the pipelined engine of the FP64 mode (plain double
// arithmetic; rows with 1 - g_i = 0 are flagged degenerate and go to the unfactored FP64
// pass).
struct alignas(16) Rec64J {
    double pm, px, a, b, h, g, mi;
    uint64_t meta;
};

constexpr uint32_t META_CODE_MASK = 0x7u;
constexpr int META_GCP_SHIFT = 8;
constexpr uint32_t META_DEGEN = 1u << 16;  // 1 - g_i too small for the factored form
constexpr uint32_t META_BAD = 1u << 17;    // invalid base or quality > 93

constexpr int kMaxPhred = 93;
constexpr int kPhredTab = 96;  // table rows (>= kMaxPhred + 1)

// Per-pair descriptor (built on the device from the pair index and the offsets).
struct PairDesc {
    uint64_t roff;  // offset of the read's first base / record
    uint64_t hoff;  // offset of the haplotype's first base
    uint32_t l;     // read length (rows)
    uint32_t k;     // haplotype length (columns)
};

// Partial result of one segment (a team or one warp of a multi-warp pair):
// L * C = S * 2^E summed over its columns of the last row (Eq. 4).
struct alignas(16) Partial {
    double S;
    int32_t E;
    uint32_t flags;      // PF_* below
    uint32_t n_extra;    // segment 0 of a multi-warp pair: number of further partials
    uint32_t extra_base; // ... and where they start in the partial array
};

// Partial / pair flags (device side)
constexpr uint32_t PF_DONE = 1u << 0;       // written
constexpr uint32_t PF_DANGER = 1u << 1;     // a checkpoint row max fell below the danger level
constexpr uint32_t PF_NONFINITE = 1u << 2;  // inf / nan met
constexpr uint32_t PF_DEGEN = 1u << 3;      // factored FP32 form not applicable
constexpr uint32_t PF_BAD = 1u << 4;        // invalid input
constexpr uint32_t PF_RESCALED = 1u << 5;   // a power-of-two rescale happened
constexpr uint32_t PF_TIMEOUT = 1u << 6;    // a bounded wait gave up
constexpr uint32_t PF_TOO_LONG = 1u << 7;   // pair exceeds what this kernel can hold

// Device status word bits
constexpr uint32_t ST_BAD_INPUT = 1u << 0;
constexpr uint32_t ST_TIMEOUT = 1u << 1;
constexpr uint32_t ST_TOO_LONG = 1u << 2;
constexpr uint32_t ST_NONFINITE = 1u << 3;

// ----------------------------------------------------------------------------------
// Work plan (host-built).
//   Short pairs (k <= 32 N): a team of G = ceil(k / N) lanes; teams are packed into
//   warps (sum of G <= 32).  A warp item lists its teams.
//   Long pairs (k > 32 N): W = ceil(k / (32 N)) warps of one CTA (W <= kCtaWarps),
//   one warp per column segment, carries passed through shared memory.  A CTA item
//   lists pairs with their warp ranges.
// ----------------------------------------------------------------------------------
constexpr int kCtaWarps = 16;
constexpr int kCtaWarpsPipe = 12;  // FP32 multi-warp CTAs of the pipelined engine (register budget)
constexpr int kCtaThreads = kCtaWarps * 32;
constexpr int kRing = 8;  // rows buffered between two warp segments

constexpr uint32_t kNoPair = 0xffffffffu;

// A team: G lanes of one warp running one pair, or (FP32) two pairs packed into the x / y
// halves of float2 registers (pair2 = kNoPair when there is no second pair).
struct Team {
    uint32_t pair;
    uint32_t pair2;
    uint8_t base;   // first lane
    uint8_t size;   // lanes (G)
    uint16_t pad;
};
struct WarpItem {
    uint32_t first_team;
    uint32_t n_teams;
};
// One strip of a multi-warp pair in a CTA item: warps w0 .. w0+W-1 run columns
// col0 .. col0 + W * 32 N - 1.  A pair wider than one CTA is split into nstrip strips
// (consecutive CTA items, dequeued in order); strips pass each row's boundary values
// through the global buffer `bnd` (bnd_in / bnd_out: word offsets, kNoBnd if none).
constexpr uint64_t kNoBnd = ~0ull;
// Cluster kind: a strip whose neighbouring strip runs in the next (previous) CTA of the
// same thread-block cluster passes its boundary rows through that CTA's shared memory
// (DSMEM) instead of `bnd`.  bnd_out = kDsmemBnd | first warp of the receiving strip;
// bnd_in = kDsmemBnd.
constexpr uint64_t kDsmemBnd = 0xFFFFFFFF00000000ull;
__host__ __device__ inline bool is_dsmem_bnd(uint64_t b) {
    return b != kNoBnd && (b & 0xFFFFFFFF00000000ull) == kDsmemBnd;
}
constexpr int kClusterCtas = 8;   // CTAs per cluster of the cluster kind (portable size)
constexpr int kClusterWarps = 4;  // warps per CTA of the cluster kind
struct CtaPair {
    uint32_t pair;
    uint8_t w0;          // first warp
    uint8_t W;           // warps
    uint16_t strip;      // strip index
    uint32_t nstrip;     // strips of this pair
    uint32_t col0;       // first column of the strip (0-based)
    uint32_t extra_base; // partial slots of strips 1..nstrip-1
    uint32_t pad;
    uint64_t bnd_in, bnd_out;
};
struct CtaItem {
    uint32_t first;
    uint32_t n;
};

// Power table row for one gcp Phred value g = q(gcp) and one N (columns per lane):
// every power p is stored as two factors p1 * p2 = p so that a product v * p1 * p2 stays
// representable whenever v * p is (see engine.cuh, scan).
template <typename T>
struct PowRow {
    T sp1[5], sp2[5];   // g^(N * 2^s), s = 0..4: Kogge-Stone steps
    T lp1[32], lp2[32]; // g^(N * t), t = 0..31: segment carry into lane t
    T last1, last2;     // g^(N - 1): from a lane's first column to its last
    T pad1, pad2;
    T lq1[33], lq2[33]; // g^(N * t - 1), t = 1..32 (t = 0 unused): segment carry to the
                        // column before lane t (t = 32: the segment's last column)
    T hh1, hh2;         // g^(N/2): across the first half of a lane's columns
    T hm1, hm2;         // g^(N/2 - 1)
};

// Phred tables staged in shared memory by the prep kernels.  Each value is a pair
// (hi, lo) with hi + lo the FP64 value (host-computed), so FP32 prep can form the
// record coefficients in double-float arithmetic and round them stochastically.
//   q[x] = 10^(-x/10)      om[x] = 1 - q[x]      q3[x] = q[x] / 3      inv[x] = 1 / om[x]
// ------------------------------------------------------------------------------------
struct PhredTables {
    double q[kPhredTab], om[kPhredTab], q3[kPhredTab], inv[kPhredTab], iq[kPhredTab];  // iq = 1 / q
};

// Everything a batch's kernels read, in one device-resident header (so a captured CUDA
// graph stays valid while arrays move).
struct BatchHeader {
    // inputs (device pointers)
    const uint8_t *read_bases, *base_q, *ins_q, *del_q, *gcp_q, *hap_bases;
    const uint64_t *read_off, *hap_off;
    const uint32_t *pair_read, *pair_hap;
    uint64_t n_read_bases;
    uint32_t n_reads, n_haps, n_pairs;
    // derived
    PairDesc *desc;
    Rec32 *rec32;
    Rec32J *rec32j;  // pipelined-engine records (nullptr when no kernel of the plan uses them)
    Rec64 *rec64;
    Rec64J *rec64j;  // FP64 pipelined-engine records (FP64 mode, variant 2; else nullptr)
    // plan
    const WarpItem *witems;   // FP32: scalar teams; FP64: all teams
    const WarpItem *witems2;  // FP32: packed same-read teams
    const Team *teams;
    const CtaItem *citems;
    const CtaPair *cpairs;
    uint32_t n_witems, n_citems, n_witems2;
    uint32_t n_partials;
    uint32_t force_rescue;   // 1: every pair goes to the FP64 rescue pass
    Partial *parts;          // n_pairs slots, then extra slots of strips 1.. of wide pairs
    unsigned long long *bnd; // strip boundaries (tagged 64-bit words), cleared per launch
    uint64_t n_bnd_words;
    unsigned long long *rbnd;   // rescue / single-launch scratch: 2 boundaries per CTA
    uint64_t rbnd_words_per_cta;
    float4 *wbnd;            // strips of the wave kind: each strip's right boundary (l rows)
    float4 *sbnd;            // serial multi-warp pairs: 2 strip boundaries of sbnd_rows rows
    uint32_t sbnd_rows;      // per resident warp of k_forward_serial (not cleared)
    uint32_t sbnd_warps;     // warps the scratch holds (the kernel's grid x warps per CTA)
    uint32_t l_max;          // longest read of the batch
    // outputs
    double *out;             // n_pairs log10 L
    uint8_t *out_flags;      // n_pairs PHMM_PAIR_* bits
    uint32_t *rescue_list;   // pairs needing the FP64 pass
    // scratch counters (zeroed per launch by k_reset)
    uint32_t *counters;      // 8 words: [0] CTA items [1] warp items [2] rescue count
                             // [3] rescue items [4] packed warp items
    uint32_t *status;        // ST_* bits
    uint32_t *dropgrow;      // [0] max drop bits * 64, [1] max grow bits * 64 (prep);
                             // pipelined-engine records: [2] range bits (ceil log2 of the
                             // largest of a, b / (1 - g), 1 / mi_{i-1}), [3] J growth bits * 64
    uint32_t seed;
    uint32_t mode;           // 0 FP32+rescue, 1 FP64, 2 FP32 only
    double tol32;            // FP32 tolerance of |log10 L| for the a-priori rounding bound
};

}  // namespace phmm
