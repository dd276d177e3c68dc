// FP32 instantiation: coefficient prep (double-float + stochastic rounding), the
// persistent FP32 forward kernel for N = 16 / 24 / 32 columns per lane, finalize, and
// the scan test.
#include "kernels.cuh"
#include "launch.h"

namespace phmm {

__device__ __align__(16) Rec32 g_dummy32;  // read as two float4

template <>
__device__ const Rec32* dummy_rec<float>() { return &g_dummy32; }

// Zeroes the work counters and status words, and clears the strip boundary buffer (its
// row tags must not survive from an earlier launch).
__global__ void k_reset(const BatchHeader* __restrict__ H) {
    if (blockIdx.x == 0) {
        if (threadIdx.x < 8) H->counters[threadIdx.x] = 0u;
        if (threadIdx.x == 0) {
            H->status[0] = 0u;
            H->dropgrow[0] = 0u;
            H->dropgrow[1] = 0u;
            H->dropgrow[2] = 0u;
            H->dropgrow[3] = 0u;
        }
    }
    const uint64_t n = H->n_bnd_words;
    for (uint64_t q = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; q < n; q += (uint64_t)gridDim.x * blockDim.x)
        H->bnd[q] = 0ull;
}

// Phred tables as double-float pairs in shared memory.
struct Tables32 {
    float2 tq[kPhredTab], tom[kPhredTab], tq3[kPhredTab], tinv[kPhredTab], tiq[kPhredTab];
};
__device__ __forceinline__ void stage_tables32(const PhredTables* __restrict__ TG, Tables32& T) {
    for (int i = threadIdx.x; i < kPhredTab; i += blockDim.x) {
        const df a = to_df(TG->q[i]), b = to_df(TG->om[i]), c = to_df(TG->q3[i]),
                 d = to_df(TG->inv[i]), e = to_df(TG->iq[i]);
        T.tq[i] = make_float2(a.hi, a.lo);
        T.tom[i] = make_float2(b.hi, b.lo);
        T.tq3[i] = make_float2(c.hi, c.lo);
        T.tinv[i] = make_float2(d.hi, d.lo);
        T.tiq[i] = make_float2(e.hi, e.lo);
    }
    __syncthreads();
}

__device__ __forceinline__ void store_rec32j(Rec32J* dst, const Rec32J& r) {
    float4* d = reinterpret_cast<float4*>(dst);
    d[0] = make_float4(r.pm, r.px, r.a, r.b);
    d[1] = make_float4(r.h, r.g, r.mi, __uint_as_float(r.meta));
}

// One record per read base (both FP32 layouts), plus pair descriptors and the batch's
// drop / grow maxima.
// Input staging of the prep kernel: a tile of kPrepTile read bases of each byte stream
// (bases and the four quality strings) and the 16 bytes before it, copied into shared
// memory with 16-byte loads where the chunk is aligned and inside the array (byte loads
// at unaligned or ragged edges, zeros outside), so each thread then reads its bases from
// shared memory and the records it writes stay consecutive across the warp.
constexpr int kPrepThreads = 256, kPrepTile = kPrepThreads * 16;
__device__ __forceinline__ void stage_bytes(const uint8_t* __restrict__ src, uint64_t n, uint64_t t0,
                                            uint4* __restrict__ dst) {
    const bool al = ((uintptr_t)src & 15u) == 0;
    for (int c = threadIdx.x; c < kPrepTile / 16 + 1; c += blockDim.x) {
        const int64_t g = (int64_t)t0 - 16 + 16 * (int64_t)c;  // first byte of chunk c
        uint4 v;
        if (al && g >= 0 && g + 16 <= (int64_t)n) {
            v = __ldg(reinterpret_cast<const uint4*>(src + g));
        } else {
            uint32_t w[4] = {0u, 0u, 0u, 0u};
#pragma unroll
            for (int q = 0; q < 16; ++q) {
                const int64_t bi = g + q;
                const uint32_t byte = (bi >= 0 && bi < (int64_t)n) ? (uint32_t)src[bi] : 0u;
                w[q >> 2] |= byte << (8 * (q & 3));
            }
            v = make_uint4(w[0], w[1], w[2], w[3]);
        }
        dst[c] = v;
    }
}

__global__ void __launch_bounds__(kPrepThreads) k_prep32(const BatchHeader* __restrict__ H,
                                                         const PhredTables* __restrict__ TG) {
    __shared__ Tables32 T;
    __shared__ uint4 sb[5][kPrepTile / 16 + 1];  // bases, Q, ins, del, gcp; byte 16 = tile start
    stage_tables32(TG, T);
    const float2 *tq = T.tq, *tom = T.tom, *tq3 = T.tq3, *tinv = T.tinv;
    Rec32J* const rj = H->rec32j;
    uint32_t dmax = 0, gmax = 0, jmax = 0, hmax = 0;
    const uint64_t n = H->n_read_bases;
    const uint32_t seed = H->seed;
    const uint8_t* const s8[5] = {H->read_bases, H->base_q, H->ins_q, H->del_q, H->gcp_q};
    for (uint64_t t0 = (uint64_t)blockIdx.x * kPrepTile; t0 < n; t0 += (uint64_t)gridDim.x * kPrepTile) {
        __syncthreads();  // the previous tile's reads are done
#pragma unroll
        for (int q = 0; q < 5; ++q) stage_bytes(s8[q], n, t0, sb[q]);
        __syncthreads();
        const uint8_t* const sbase = reinterpret_cast<const uint8_t*>(sb[0]);
        const uint8_t* const sq = reinterpret_cast<const uint8_t*>(sb[1]);
        const uint8_t* const si = reinterpret_cast<const uint8_t*>(sb[2]);
        const uint8_t* const sd = reinterpret_cast<const uint8_t*>(sb[3]);
        const uint8_t* const sg = reinterpret_cast<const uint8_t*>(sb[4]);
        for (int m = 0; m < kPrepTile / kPrepThreads; ++m) {
            const int o = 16 + m * kPrepThreads + (int)threadIdx.x;  // byte of base b in the stage
            const uint64_t b = t0 + (uint64_t)(o - 16);
            if (b >= n) break;
            // the same fields and clamps as base_inputs(), from the staged bytes
            BaseQ x;
            x.code = read_code(sbase[o]);
            x.Q = sq[o];
            x.ins = si[o];
            x.del = sd[o];
            x.gcp = sg[o];
            x.delp = b > 0 ? sd[o - 1] : 0;
            x.insp = b > 0 ? si[o - 1] : si[o];
            x.bad = x.code < 0 || x.Q > kMaxPhred || x.ins > kMaxPhred || x.del > kMaxPhred || x.gcp > kMaxPhred;
            x.code = x.code < 0 ? 4 : x.code;
            x.Q = min(x.Q, kMaxPhred);
            x.ins = min(x.ins, kMaxPhred);
            x.del = min(x.del, kMaxPhred);
            x.gcp = min(x.gcp, kMaxPhred);
            x.delp = min(x.delp, kMaxPhred);
            x.insp = min(x.insp, kMaxPhred);
            if (H->rec32) {
                const Rec32 r = make_rec32(x, tq, tom, tq3, tinv, seed, b);
                float4* dst = reinterpret_cast<float4*>(H->rec32 + b);
                dst[0] = make_float4(r.pm, r.px, r.a, r.b);
                dst[1] = make_float4(r.mi, r.g, r.gm, __uint_as_float(r.meta));
            }
            if (rj) {
                const Rec32J r2 = make_rec32j(x, tq, tom, tq3, tinv, T.tiq, seed, b, false);
                store_rec32j(rj + b, r2);
                // range of the pipelined engine's intermediates relative to the row maximum
                const float om = fmaxf(1.0f - r2.g, 0x1p-60f);
                const float big = fmaxf(fmaxf(fabsf(r2.a), fabsf(r2.b) / om), T.tiq[x.insp].x);
                jmax = max(jmax, (uint32_t)fmaxf(ceilf(log2f(fmaxf(big, 1.0f))), 0.0f));
                hmax = max(hmax, (uint32_t)ceilf(log2f(1.0f + fabsf(r2.h)) * 64.0f) + 1u);
            }
            if (x.bad) atomicOr(H->status, ST_BAD_INPUT);
            const float qi = tq[x.ins].x, qd = tq[x.del].x, qg = tq[x.gcp].x;
            const float drop = -log2f(fminf(qi, qg));
            const float grow = log2f(fmaxf(fabsf(1.0f - qi - qd) + (1.0f - qg) + qd, qi + qg));
            dmax = max(dmax, (uint32_t)ceilf(fmaxf(drop, 0.0f) * 64.0f) + 1u);
            gmax = max(gmax, (uint32_t)ceilf(fmaxf(grow, 0.0f) * 64.0f) + 1u);
        }
    }
    block_max2(dmax, gmax, H->dropgrow);
    __syncthreads();
    block_max2(jmax, hmax, H->dropgrow + 2);
    build_desc(H);
}

// Row 1 of every read in the pipelined-engine records: the previous row's T_MI is 1
// there (k_prep32 used the previous base of the batch).  Runs after k_prep32.
__global__ void __launch_bounds__(256) k_prep32_first(const BatchHeader* __restrict__ H,
                                                      const PhredTables* __restrict__ TG) {
    __shared__ Tables32 T;
    stage_tables32(TG, T);
    Rec32J* const rj = H->rec32j;
    if (!rj) return;
    for (uint32_t r = blockIdx.x * blockDim.x + threadIdx.x; r < H->n_reads; r += gridDim.x * blockDim.x) {
        const uint64_t b = H->read_off[r];
        if (b >= H->read_off[r + 1]) continue;
        const BaseQ x = base_inputs(H, b);
        store_rec32j(rj + b, make_rec32j(x, T.tq, T.tom, T.tq3, T.tinv, T.tiq, H->seed, b, true));
    }
}

template __global__ void k_forward<float, kNLong32, false>(const BatchHeader*, const PowRow<float>*);
template __global__ void k_forward_pipe<32, kCtaWarpsPipe>(const BatchHeader*, const PowRow<float>*);
template __global__ void k_forward_pipe<24, kCtaWarps>(const BatchHeader*, const PowRow<float>*);
template __global__ void k_forward_serial<32, 3>(const BatchHeader*, const PowRow<float>*);
template __global__ void k_forward_wave<32, 3>(const BatchHeader*, const PowRow<float>*);
template __global__ void k_forward_wave<16, 3>(const BatchHeader*, const PowRow<float>*);
template __global__ void k_forward_pipe<32, 4>(const BatchHeader*, const PowRow<float>*);
template __global__ void k_forward_cluster<32, kClusterWarps, kClusterCtas>(const BatchHeader*, const PowRow<float>*);
template __global__ void k_short_scalar<32, 4>(const BatchHeader*, const PowRow<float>*);
template __global__ void k_short_scalar<24, 4>(const BatchHeader*, const PowRow<float>*);
template __global__ void k_short_scalar<24, 5>(const BatchHeader*, const PowRow<float>*);
template __global__ void k_short_scalar<16, 6>(const BatchHeader*, const PowRow<float>*);
template __global__ void k_short_pipe<32, 3>(const BatchHeader*, const PowRow<float>*);
template __global__ void k_short_pipe<24, 4>(const BatchHeader*, const PowRow<float>*);
template __global__ void k_short_pipe<16, 4>(const BatchHeader*, const PowRow<float>*);
template __global__ void k_short_pipe2<32, 3, true>(const BatchHeader*, const PowRow<float>*);
template __global__ void k_short_pipe2<24, 4, true>(const BatchHeader*, const PowRow<float>*);
template __global__ void k_short_pipe2<32, 4, true, true>(const BatchHeader*, const PowRow<float>*);

template __global__ void k_short_packed<12, 4>(const BatchHeader*, const PowRow<float>*);
template __global__ void k_short_packed<16, 3>(const BatchHeader*, const PowRow<float>*);

// Scan test: one warp, lane t owns y[32t .. 32t+31]; `row` is in global memory.
__global__ void k_scan_test(const float* __restrict__ y, float* __restrict__ z, int n,
                            const PowRow<float>* __restrict__ row) {
    const int lane = threadIdx.x & 31;
    Pow<float> pw;
    pw.row = row;
    pw.gcp = 0;
    const float a = row->pad1;  // the multiplier itself
    float loc[32];
    float v = 0.0f;
#pragma unroll
    for (int c = 0; c < 32; ++c) {
        const int e = lane * 32 + c;
        v = fmaf(a, v, e < n ? y[e] : 0.0f);
        loc[c] = v;
    }
    const float Z = team_scan<float>(v, lane, pw, 5);
    float W = __shfl_up_sync(kFull, Z, 1);
    if (lane == 0) W = 0.0f;
#pragma unroll
    for (int c = 0; c < 32; ++c) {
        W *= a;
        const int e = lane * 32 + c;
        if (e < n) z[e] = loc[c] + W;
    }
}

// Bounded-wait test: lane 0 waits for row 1 of a strip boundary that nothing writes (the
// words hold tag 0); the wait gives up after its poll limit and reports ST_TIMEOUT.
__global__ void k_wait_test(const unsigned long long* __restrict__ bnd, uint32_t* __restrict__ status) {
    if (threadIdx.x == 0) {
        float m, i, d;
        int e;
        if (!link_recv_g<float>(bnd, 1, m, i, d, e)) atomicOr(status, ST_TIMEOUT);
    }
}

void launch_wait_test(const void* bnd, uint32_t* status, cudaStream_t s) {
    k_wait_test<<<1, 32, 0, s>>>(static_cast<const unsigned long long*>(bnd), status);
}

void launch_reset(const BatchHeader* H, int grid, cudaStream_t s) { k_reset<<<grid, 256, 0, s>>>(H); }

void launch_prep32(const BatchHeader* H, const PhredTables* T, int grid, cudaStream_t s) {
    k_prep32<<<grid, kPrepThreads, 0, s>>>(H, T);
}

void launch_prep32_first(const BatchHeader* H, const PhredTables* T, int grid, cudaStream_t s) {
    k_prep32_first<<<grid, 256, 0, s>>>(H, T);
}

void launch_forward32_long(const BatchHeader* H, const void* pow, int grid, cudaStream_t s) {
    k_forward<float, kNLong32, false><<<grid, kCtaThreads, 0, s>>>(H, static_cast<const PowRow<float>*>(pow));
}

void launch_forward32_long_pipe(int kind, const BatchHeader* H, const void* pow, int grid, cudaStream_t s) {
    const PowRow<float>* p = static_cast<const PowRow<float>*>(pow);
    if (kind == 5) k_forward_cluster<32, kClusterWarps, kClusterCtas><<<grid, kClusterWarps * 32, 0, s>>>(H, p);
    else if (kind == 3) k_forward_serial<32, 3><<<grid, kSerialThreads, 0, s>>>(H, p);
    else if (kind == 6 || kind == 7) k_forward_wave<32, 3><<<grid, kSerialThreads, 0, s>>>(H, p);
    else if (kind == 8) k_forward_wave<16, 3><<<grid, kSerialThreads, 0, s>>>(H, p);
    else if (kind == 4) k_forward_pipe<32, 4><<<grid, 4 * 32, 0, s>>>(H, p);
    else if (kind == 2) k_forward_pipe<24, kCtaWarps><<<grid, kCtaWarps * 32, 0, s>>>(H, p);
    else k_forward_pipe<32, kCtaWarpsPipe><<<grid, kCtaWarpsPipe * 32, 0, s>>>(H, p);
}

// Short-pair kernel variants (ids used by the runtime's tuner):
//   scalar id 0: N 32, 4 CTAs/SM   1: N 24, 4   2: N 24, 5   3: N 16, 6   (lean)
//             4: N 32, 3            5: N 24, 4   6: N 16, 4                 (pipelined)
//             7: N 32, 3 halves     8: N 24, 4 halves   9: N 32, 4 halves, lean (fused row, L1 tables)
//   packed id 0: N 12, 4 CTAs/SM   1: N 16, 3
template <typename K>
static int occ_of(K kern) {
    cudaFuncSetAttribute((const void*)kern, cudaFuncAttributePreferredSharedMemoryCarveout,
                         cudaSharedmemCarveoutMaxShared);
    int b = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, kern, kShortThreads, 0);
    return b > 0 ? b : 1;
}

void launch_short_scalar(int id, const BatchHeader* H, const void* pow, int grid, cudaStream_t s) {
    const PowRow<float>* p = static_cast<const PowRow<float>*>(pow);
    switch (id) {
    case 1: k_short_scalar<24, 4><<<grid, kShortThreads, 0, s>>>(H, p); break;
    case 2: k_short_scalar<24, 5><<<grid, kShortThreads, 0, s>>>(H, p); break;
    case 3: k_short_scalar<16, 6><<<grid, kShortThreads, 0, s>>>(H, p); break;
    case 4: k_short_pipe<32, 3><<<grid, kShortThreads, 0, s>>>(H, p); break;
    case 5: k_short_pipe<24, 4><<<grid, kShortThreads, 0, s>>>(H, p); break;
    case 6: k_short_pipe<16, 4><<<grid, kShortThreads, 0, s>>>(H, p); break;
    case 7: k_short_pipe2<32, 3, true><<<grid, kShortThreads, 0, s>>>(H, p); break;
    case 8: k_short_pipe2<24, 4, true><<<grid, kShortThreads, 0, s>>>(H, p); break;
    case 9: k_short_pipe2<32, 4, true, true><<<grid, kShortThreads, 0, s>>>(H, p); break;

    default: k_short_scalar<32, 4><<<grid, kShortThreads, 0, s>>>(H, p); break;
    }
}

void launch_short_packed(int id, const BatchHeader* H, const void* pow, int grid, cudaStream_t s) {
    const PowRow<float>* p = static_cast<const PowRow<float>*>(pow);
    if (id == 0) k_short_packed<12, 4><<<grid, kShortThreads, 0, s>>>(H, p);
    else k_short_packed<16, 3><<<grid, kShortThreads, 0, s>>>(H, p);
}

int occupancy_short_scalar(int id) {
    switch (id) {
    case 1: return occ_of(k_short_scalar<24, 4>);
    case 2: return occ_of(k_short_scalar<24, 5>);
    case 3: return occ_of(k_short_scalar<16, 6>);
    case 4: return occ_of(k_short_pipe<32, 3>);
    case 5: return occ_of(k_short_pipe<24, 4>);
    case 6: return occ_of(k_short_pipe<16, 4>);
    case 7: return occ_of(k_short_pipe2<32, 3, true>);
    case 8: return occ_of(k_short_pipe2<24, 4, true>);
    case 9: return occ_of(k_short_pipe2<32, 4, true, true>);

    default: return occ_of(k_short_scalar<32, 4>);
    }
}

int occupancy_short_packed(int id) {
    return id == 0 ? occ_of(k_short_packed<12, 4>) : occ_of(k_short_packed<16, 3>);
}

int occupancy_forward32_long() {
    int b = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_forward<float, kNLong32, false>, kCtaThreads, 0);
    return b > 0 ? b : 1;
}

int occupancy_forward32_long_pipe(int kind) {
    int b = 0;
    if (kind == 5) {
        // clusters that fit on the GPU at once (the grid of the persistent cluster kernel)
        cudaLaunchConfig_t c = {};
        c.gridDim = dim3(kClusterCtas, 1, 1);
        c.blockDim = dim3(kClusterWarps * 32, 1, 1);
        c.dynamicSmemBytes = 0;
        c.attrs = nullptr;
        c.numAttrs = 0;
        if (cudaOccupancyMaxActiveClusters(&b, (const void*)k_forward_cluster<32, kClusterWarps, kClusterCtas>, &c) !=
            cudaSuccess)
            b = 0;
        cudaGetLastError();
        return b > 0 ? b : 1;
    }
    if (kind == 3)
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_forward_serial<32, 3>, kSerialThreads, 0);
    else if (kind == 6 || kind == 7) {
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_forward_wave<32, 3>, kSerialThreads, 0);
        if (kind == 7) b = b < 2 ? b : 2;  // the two-CTA grid
    }
    else if (kind == 8)
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_forward_wave<16, 3>, kSerialThreads, 0);
    else if (kind == 4)
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_forward_pipe<32, 4>, 4 * 32, 0);
    else if (kind == 2)
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_forward_pipe<24, kCtaWarps>, kCtaWarps * 32, 0);
    else
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_forward_pipe<32, kCtaWarpsPipe>, kCtaWarpsPipe * 32, 0);
    return b > 0 ? b : 1;
}

void launch_finalize32(const BatchHeader* H, int grid, cudaStream_t s) {
    k_finalize<float><<<grid, 256, 0, s>>>(H);
}

void launch_scan_test(const float* y, float* z, int n, const void* pow_row, cudaStream_t s) {
    k_scan_test<<<1, 32, 0, s>>>(y, z, n, static_cast<const PowRow<float>*>(pow_row));
}

}  // namespace phmm
