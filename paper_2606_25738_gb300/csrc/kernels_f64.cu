// FP64 instantiation: prep of FP64 records (all reads, or only the reads of pairs
// selected for rescue), the FP64 forward kernel, the rescue pass, the one-launch-per-
// pair comparator kernel and finalize.
#include "kernels.cuh"
#include "launch.h"

namespace phmm {

__device__ Rec64 g_dummy64;

template <>
__device__ const Rec64* dummy_rec<double>() { return &g_dummy64; }

__global__ void __launch_bounds__(256) k_prep64_all(const BatchHeader* __restrict__ H,
                                                    const PhredTables* __restrict__ TG) {
    __shared__ PhredTables T;
    load_tables(TG, T);
    __syncthreads();
    uint32_t dmax = 0, gmax = 0, jmax = 0, hmax = 0;
    const uint64_t n = H->n_read_bases;
    Rec64J* const rj = H->rec64j;
    for (uint64_t b = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; b < n;
         b += (uint64_t)gridDim.x * blockDim.x) {
        const BaseQ x = base_inputs(H, b);
        H->rec64[b] = make_rec64(x, T);
        if (rj) {
            // J-form records of the pipelined FP64 engine and the range of its
            // intermediates relative to the row maximum (as in the FP32 prep)
            const Rec64J r2 = make_rec64j(x, T, false);
            rj[b] = r2;
            const double om = fmax(1.0 - r2.g, 0x1p-60);
            const double big = fmax(fmax(fabs(r2.a), fabs(r2.b) / om), T.iq[x.insp]);
            jmax = max(jmax, (uint32_t)fmax(ceil(log2(fmax(big, 1.0))), 0.0));
            hmax = max(hmax, (uint32_t)ceil(log2(1.0 + fabs(r2.h)) * 64.0) + 1u);
        }
        if (x.bad) atomicOr(H->status, ST_BAD_INPUT);
        uint32_t d, g;
        drop_grow(x, T, d, g);
        dmax = max(dmax, d);
        gmax = max(gmax, g);
    }
    block_max2(dmax, gmax, H->dropgrow);
    __syncthreads();
    block_max2(jmax, hmax, H->dropgrow + 2);
    build_desc(H);
}

// Row 1 of every read in the FP64 J-form records: the previous row's T_MI is 1 there
// (k_prep64_all used the previous base of the batch).  Runs after k_prep64_all.
__global__ void __launch_bounds__(256) k_prep64_first(const BatchHeader* __restrict__ H,
                                                      const PhredTables* __restrict__ TG) {
    __shared__ PhredTables T;
    load_tables(TG, T);
    __syncthreads();
    Rec64J* const rj = H->rec64j;
    if (!rj) return;
    for (uint32_t r = blockIdx.x * blockDim.x + threadIdx.x; r < H->n_reads; r += gridDim.x * blockDim.x) {
        const uint64_t b = H->read_off[r];
        if (b >= H->read_off[r + 1]) continue;
        rj[b] = make_rec64j(base_inputs(H, b), T, true);
    }
}

// Records of the reads of the pairs selected for rescue (one block per pair).
__global__ void __launch_bounds__(256) k_prep64_list(const BatchHeader* __restrict__ H,
                                                     const PhredTables* __restrict__ TG) {
    __shared__ PhredTables T;
    load_tables(TG, T);
    __syncthreads();
    const uint32_t n = H->counters[2];
    for (uint32_t r = blockIdx.x; r < n; r += gridDim.x) {
        const PairDesc d = H->desc[H->rescue_list[r]];
        for (uint32_t i = threadIdx.x; i < d.l; i += blockDim.x) {
            const uint64_t b = d.roff + i;
            H->rec64[b] = make_rec64(base_inputs(H, b), T);
        }
    }
}

template __global__ void k_forward<double, kN64, true>(const BatchHeader*, const PowRow<double>*);
template __global__ void k_forward<double, kF64N[1], true, kF64CW[1]>(const BatchHeader*, const PowRow<double>*);
template __global__ void k_forward<double, kF64N[2], false, kF64CW[2]>(const BatchHeader*, const PowRow<double>*);
template __global__ void k_short_pipe64<kF64NS[2], 2>(const BatchHeader*, const PowRow<double>*);
template __global__ void k_short_pipe64<kF64NS[3], 1, true>(const BatchHeader*, const PowRow<double>*);
template __global__ void k_finalize<double>(const BatchHeader*);

__device__ __forceinline__ double log10_of(const Partial& q) {
    if (q.S > 0.0 && isfinite(q.S))
        return log10(q.S) + (double)(q.E - Num<double>::kLog2C) * 0.30102999566398119521;
    return q.S == 0.0 ? -INFINITY : NAN;
}

// FP64 rescue pass: one CTA per selected pair, persistent over the rescue list; pairs
// wider than the CTA run strip after strip through this CTA's boundary scratch.
__global__ void __launch_bounds__(kCtaThreads, 1)
k_rescue(const BatchHeader* __restrict__ H, const PowRow<double>* __restrict__ pow) {
    __shared__ CtaShared<double> sh;
    const int R = checkpoint_interval<double>(H->dropgrow);
    const uint32_t n = H->counters[2];
    unsigned long long* scratch = H->rbnd + (size_t)blockIdx.x * 2 * H->rbnd_words_per_cta;
    for (;;) {
        if (threadIdx.x == 0) sh.item = atomicAdd(&H->counters[3], 1u);
        __syncthreads();
        const uint32_t r = sh.item;
        __syncthreads();
        if (r >= n) break;
        const uint32_t p = H->rescue_list[r];
        const Partial q = cta_pair_sequential<double, kN64>(H, pow, p, sh, R, scratch, H->rbnd_words_per_cta);
        if (threadIdx.x == 0) {
            uint8_t of = (uint8_t)((H->out_flags[p] & 0x78u) | 0x1u | 0x4u);
            const double v = log10_of(q);
            if (q.flags & PF_RESCALED) of |= 0x2u;
            if (q.flags & (PF_TIMEOUT | PF_BAD)) of |= 0x80u;
            if (!isfinite(q.S)) atomicOr(H->status, ST_NONFINITE);
            H->out[p] = v;
            H->out_flags[p] = of;
        }
        __syncthreads();
    }
}

// Plain FP64 comparator: one launch (one CTA) per pair, strips in sequence.
__global__ void __launch_bounds__(kCtaThreads, 1)
k_single(const BatchHeader* __restrict__ H, const PowRow<double>* __restrict__ pow, uint32_t pair) {
    __shared__ CtaShared<double> sh;
    const int R = checkpoint_interval<double>(H->dropgrow);
    const Partial q = cta_pair_sequential<double, kN64>(H, pow, pair, sh, R, H->rbnd, H->rbnd_words_per_cta);
    if (threadIdx.x == 0) H->parts[pair] = q;
}

void launch_prep64_all(const BatchHeader* H, const PhredTables* T, int grid, cudaStream_t s) {
    k_prep64_all<<<grid, 256, 0, s>>>(H, T);
}
void launch_prep64_list(const BatchHeader* H, const PhredTables* T, int grid, cudaStream_t s) {
    k_prep64_list<<<grid, 256, 0, s>>>(H, T);
}
void launch_forward64(int id, const BatchHeader* H, const void* pow, int grid, cudaStream_t s) {
    const PowRow<double>* p = static_cast<const PowRow<double>*>(pow);
    if (f64_pipelined(id)) k_forward<double, kF64N[2], false, kF64CW[2]><<<grid, kF64CW[2] * 32, 0, s>>>(H, p);
    else if (id == 1) k_forward<double, kF64N[1], true, kF64CW[1]><<<grid, kF64CW[1] * 32, 0, s>>>(H, p);
    else k_forward<double, kN64, true><<<grid, kCtaThreads, 0, s>>>(H, p);
}
void launch_short_pipe64(int id, const BatchHeader* H, const void* pow, int grid, cudaStream_t s) {
    const PowRow<double>* p = static_cast<const PowRow<double>*>(pow);
    if (id == 3) k_short_pipe64<kF64NS[3], 1, true><<<grid, kShortThreads, 0, s>>>(H, p);
    else k_short_pipe64<kF64NS[2], 2><<<grid, kShortThreads, 0, s>>>(H, p);
}
int occupancy_short_pipe64(int id) {
    int b = 0;
    if (id == 3) cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_short_pipe64<kF64NS[3], 1, true>, kShortThreads, 0);
    else cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_short_pipe64<kF64NS[2], 2>, kShortThreads, 0);
    return b > 0 ? b : 1;
}
void launch_prep64_first(const BatchHeader* H, const PhredTables* T, int grid, cudaStream_t s) {
    k_prep64_first<<<grid, 256, 0, s>>>(H, T);
}
void launch_finalize64(const BatchHeader* H, int grid, cudaStream_t s) {
    k_finalize<double><<<grid, 256, 0, s>>>(H);
}
void launch_rescue64(const BatchHeader* H, const void* pow, int grid, cudaStream_t s) {
    k_rescue<<<grid, kCtaThreads, 0, s>>>(H, static_cast<const PowRow<double>*>(pow));
}
void launch_single64(const BatchHeader* H, const void* pow, uint32_t pair, cudaStream_t s) {
    k_single<<<1, kCtaThreads, 0, s>>>(H, static_cast<const PowRow<double>*>(pow), pair);
}
int occupancy_forward64(int id) {
    int b = 0;
    if (f64_pipelined(id))
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_forward<double, kF64N[2], false, kF64CW[2]>,
                                                      kF64CW[2] * 32, 0);
    else if (id == 1)
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_forward<double, kF64N[1], true, kF64CW[1]>,
                                                      kF64CW[1] * 32, 0);
    else
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_forward<double, kN64, true>, kCtaThreads, 0);
    return b > 0 ? b : 1;
}

}  // namespace phmm
