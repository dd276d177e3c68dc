// Allocation-free variant of the FP32 forward path (phmm_forward_noalloc, include/phmm.h).
//
// Who needs it: callers that must not allocate device memory at call time -- code running
// inside a host framework that owns the device heap and forbids cudaMalloc / cudaFree on
// its threads, a process that has reserved all of device memory up front, or a caller on
// a latency path where an allocation (which can synchronise the device) is not allowed.
// The regular API (phmm_create / phmm_submit_batch) allocates its arenas and tables; this
// entry point uses only the caller's input/output buffers plus fixed scratch arrays that
// are part of the library image (file-scope __device__ arrays below), so it calls no
// allocating routine at all.
//
// Limits: at most kNaMaxBases read bases per call (records scratch: 32 bytes each) and
// haplotypes of at most kNaMaxCols columns (one warp of 32 lanes x 32 columns per pair).
// Every call uses the same scratch: calls that overlap on the GPU (other streams, other
// host threads) race on it and must be serialised by the caller.
#include <cmath>
#include <mutex>

#include "kernels.cuh"
#include "phmm.h"

namespace phmm {
namespace {

constexpr uint64_t kNaMaxBases = 1ull << 20;  // records scratch: 32 MiB
constexpr int kNaN = 32;                      // columns per lane
constexpr uint32_t kNaMaxCols = 32u * kNaN;   // one warp per pair
constexpr uint32_t kNaScratchFull = 1u << 8;  // status bit: more read bases than the scratch holds
// Seed of the stochastic rounding of the per-row coefficients: the same value a context
// uses by default, so the records (and hence the results) equal the regular path's.
constexpr uint32_t kNaRoundingSeed = 0x5eed1234u;

// Scratch (every GPU that loads the library holds these until the process exits).
static __device__ __align__(256) Rec32 na_rec[kNaMaxBases];
static __device__ __align__(256) PowRow<float> na_pow[kPhredTab];
static __device__ __align__(256) PhredTables na_tab;
static __device__ __align__(256) uint32_t na_words[16];  // [0] status [1] drop [2] grow

// Host-side device addresses of the scratch, taken once per device (cudaGetSymbolAddress;
// the array names themselves are only host stand-ins in host code).
struct NaAddrs {
    Rec32* rec = nullptr;
    PowRow<float>* pow = nullptr;
    PhredTables* tab = nullptr;
    uint32_t* words = nullptr;
    bool ready = false;
};
constexpr int kNaMaxDevices = 64;
NaAddrs g_na[kNaMaxDevices];
std::mutex g_na_mu;

// Power row of gcp value x: each power g^m as two factors whose product is g^m (see
// PowRow); computed in FP64 on the device.
__device__ void na_split(int gq, double m, float& p1, float& p2) {
    const double lg = -(double)gq / 10.0 * m;
    if (lg >= -37.9) {
        p1 = (float)pow(10.0, lg);
        p2 = 1.0f;
    } else {
        const float h = (float)pow(10.0, lg / 2.0);
        p1 = h;
        p2 = h;
    }
}

// Tables and cleared status words (one block).
__global__ void k_na_tables(PowRow<float>* pw, PhredTables* tab, uint32_t* words) {
    for (int x = threadIdx.x; x < kPhredTab; x += blockDim.x) {
        const int q = min(x, kMaxPhred);
        const double v = pow(10.0, -(double)q / 10.0);
        tab->q[x] = v;
        tab->om[x] = 1.0 - v;
        tab->q3[x] = v / 3.0;
        tab->inv[x] = 1.0 / (1.0 - v);
        PowRow<float>& r = pw[x];
        for (int s = 0; s < 5; ++s) na_split(q, (double)kNaN * (double)(1 << s), r.sp1[s], r.sp2[s]);
        for (int t = 0; t < 32; ++t) na_split(q, (double)kNaN * t, r.lp1[t], r.lp2[t]);
        na_split(q, (double)(kNaN - 1), r.last1, r.last2);
        r.pad1 = (float)v;
        r.pad2 = 0.0f;
    }
    if (threadIdx.x < 16) words[threadIdx.x] = 0u;
}

// Records of every read base (as k_prep32) into the scratch.
__global__ void __launch_bounds__(256) k_na_prep(const uint8_t* __restrict__ rb, const uint8_t* __restrict__ bq,
                                                 const uint8_t* __restrict__ iq, const uint8_t* __restrict__ dq,
                                                 const uint8_t* __restrict__ gq, const uint64_t* __restrict__ read_off,
                                                 uint32_t n_reads, const PhredTables* __restrict__ TG,
                                                 Rec32* __restrict__ rec, uint32_t* __restrict__ words) {
    __shared__ float2 tq[kPhredTab], tom[kPhredTab], tq3[kPhredTab], tinv[kPhredTab];
    for (int i = threadIdx.x; i < kPhredTab; i += blockDim.x) {
        const df a = to_df(TG->q[i]), b = to_df(TG->om[i]), c = to_df(TG->q3[i]), d = to_df(TG->inv[i]);
        tq[i] = make_float2(a.hi, a.lo);
        tom[i] = make_float2(b.hi, b.lo);
        tq3[i] = make_float2(c.hi, c.lo);
        tinv[i] = make_float2(d.hi, d.lo);
    }
    __syncthreads();
    const uint64_t n = read_off[n_reads];
    uint32_t dmax = 0, gmax = 0;
    if (n <= kNaMaxBases) {
        for (uint64_t b = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; b < n;
             b += (uint64_t)gridDim.x * blockDim.x) {
            BaseQ x;
            x.code = base_code(rb[b]);
            x.Q = bq[b];
            x.ins = iq[b];
            x.del = dq[b];
            x.gcp = gq[b];
            x.delp = b > 0 ? dq[b - 1] : 0;
            x.bad = x.code < 0 || x.Q > kMaxPhred || x.ins > kMaxPhred || x.del > kMaxPhred || x.gcp > kMaxPhred;
            x.code = x.code < 0 ? 4 : x.code;
            x.Q = min(x.Q, kMaxPhred);
            x.ins = min(x.ins, kMaxPhred);
            x.del = min(x.del, kMaxPhred);
            x.gcp = min(x.gcp, kMaxPhred);
            x.delp = min(x.delp, kMaxPhred);
            const Rec32 r = make_rec32(x, tq, tom, tq3, tinv, kNaRoundingSeed, b);
            float4* dst = reinterpret_cast<float4*>(rec + b);
            dst[0] = make_float4(r.pm, r.px, r.a, r.b);
            dst[1] = make_float4(r.mi, r.g, r.gm, __uint_as_float(r.meta));
            if (x.bad) atomicOr(words, ST_BAD_INPUT);
            const float qi = tq[x.ins].x, qd = tq[x.del].x, qg = tq[x.gcp].x;
            const float drop = -log2f(fminf(qi, qg));
            const float grow = log2f(fmaxf(fabsf(1.0f - qi - qd) + (1.0f - qg) + qd, qi + qg));
            dmax = max(dmax, (uint32_t)ceilf(fmaxf(drop, 0.0f) * 64.0f) + 1u);
            gmax = max(gmax, (uint32_t)ceilf(fmaxf(grow, 0.0f) * 64.0f) + 1u);
        }
    } else if (blockIdx.x == 0 && threadIdx.x == 0) {
        atomicOr(words, kNaScratchFull);
    }
    block_max2(dmax, gmax, words + 1);
}

// One pair per warp (a full-warp lean team, N = 32 columns per lane); writes log10 L.
__global__ void __launch_bounds__(128) k_na_forward(const uint8_t* __restrict__ hap_bases,
                                                    const uint64_t* __restrict__ read_off,
                                                    const uint64_t* __restrict__ hap_off,
                                                    const uint32_t* __restrict__ pair_read,
                                                    const uint32_t* __restrict__ pair_hap, uint32_t n_reads,
                                                    uint32_t n_haps, uint32_t n_pairs, const Rec32* __restrict__ rec,
                                                    const PowRow<float>* __restrict__ pw, uint32_t* __restrict__ words,
                                                    double* __restrict__ out, uint8_t* __restrict__ out_flags) {
    const int lane = threadIdx.x & 31;
    const uint32_t warps = (gridDim.x * blockDim.x) >> 5;
    const int R = checkpoint_interval<float>(words + 1);
    const uint64_t read_end = read_off[n_reads], hap_end = hap_off[n_haps];
    const bool scratch_ok = read_end <= kNaMaxBases;
    for (uint32_t p = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; p < n_pairs; p += warps) {
        const uint32_t r = pair_read[p], h = pair_hap[p];
        bool ok = scratch_ok && r < n_reads && h < n_haps;
        int l = 0, k = 0;
        uint64_t roff = 0, hoff = 0;
        if (ok) {
            // Offsets are checked here, before any access through them: each read and
            // haplotype must be a non-empty range inside [0, last offset] (the records
            // scratch holds exactly the bases below read_off[n_reads]).  Lengths stay
            // 64-bit until they are known to be small.
            const uint64_t r0 = read_off[r], r1 = read_off[r + 1];
            const uint64_t h0 = hap_off[h], h1 = hap_off[h + 1];
            ok = r0 < r1 && r1 <= read_end && h0 < h1 && h1 <= hap_end && h1 - h0 <= kNaMaxCols;
            if (ok) {
                roff = r0;
                hoff = h0;
                l = (int)(r1 - r0);  // <= kNaMaxBases
                k = (int)(h1 - h0);  // <= kNaMaxCols
            }
        }
        if (!ok) {
            if (lane == 0) {
                out[p] = NAN;
                out_flags[p] = 0x80u;
                atomicOr(words, ST_TOO_LONG);
            }
            continue;
        }
        const SegOut o = team_run_lean<kNaN>(rec + roff, l, l, hap_bases + hoff, k, lane * kNaN, lane, 31, 5,
                                             pw, R);
        if (lane == 0) {
            uint8_t f = 0;
            double v;
            if (o.flags & PF_BAD) {
                v = NAN;
                f = 0x80u;
                atomicOr(words, ST_BAD_INPUT);
            } else {
                v = o.S > 0.0 && isfinite(o.S)
                        ? log10(o.S) + (double)(o.E - Num<float>::kLog2C) * 0.30102999566398119521
                        : (o.S == 0.0 ? -INFINITY : NAN);
                // The regular path's selection for its FP64 pass: the engine's flags plus
                // the underflow test on the FP32 sum in stored units (1e4 * 3 l k FLT_MIN).
                const double tau = 3.0e4 * (double)l * (double)k * 1.1754943508222875e-38;
                if (o.flags & PF_RESCALED) f |= 0x2u;
                if ((o.flags & PF_DANGER) || fp32_bound_log10((double)l, (double)k) > 1e-3) f |= 0x8u;
                if ((o.flags & PF_NONFINITE) || !isfinite(o.S)) f |= 0x10u;
                if (!(o.S > tau)) f |= 0x20u;
                if (o.flags & PF_DEGEN) f |= 0x40u;
            }
            out[p] = v;
            out_flags[p] = f;
        }
    }
}

}  // namespace
}  // namespace phmm

using namespace phmm;

extern "C" int phmm_forward_noalloc(int device, void* stream, const phmm_batch* b) {
    if (!b || device < 0 || device >= kNaMaxDevices) return PHMM_EINVAL;
    if (!b->inputs_on_device || !b->outputs_on_device || !b->out_flags || !b->out_log10) return PHMM_EINVAL;
    if (b->n_pairs == 0) return PHMM_OK;
    if (!b->read_bases || !b->read_off || !b->base_q || !b->ins_q || !b->del_q || !b->gcp_q ||
        !b->hap_bases || !b->hap_off || !b->pair_read || !b->pair_hap || b->n_reads == 0 || b->n_haps == 0)
        return PHMM_EINVAL;
    int cur = -1;
    if (cudaGetDevice(&cur) != cudaSuccess) return PHMM_ECUDA;
    if (cur != device && cudaSetDevice(device) != cudaSuccess) return PHMM_ECUDA;
    NaAddrs a;
    {
        // First call on a device: take the scratch addresses (with that device current).
        std::lock_guard<std::mutex> lock(g_na_mu);
        NaAddrs& g = g_na[device];
        if (!g.ready) {
            if (cudaGetSymbolAddress((void**)&g.rec, na_rec) != cudaSuccess ||
                cudaGetSymbolAddress((void**)&g.pow, na_pow) != cudaSuccess ||
                cudaGetSymbolAddress((void**)&g.tab, na_tab) != cudaSuccess ||
                cudaGetSymbolAddress((void**)&g.words, na_words) != cudaSuccess) {
                if (cur != device) cudaSetDevice(cur);
                return PHMM_ECUDA;
            }
            g.ready = true;
        }
        a = g;
    }
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
    k_na_tables<<<1, 128, 0, s>>>(a.pow, a.tab, a.words);
    k_na_prep<<<sms * 4, 256, 0, s>>>(b->read_bases, b->base_q, b->ins_q, b->del_q, b->gcp_q, b->read_off,
                                      b->n_reads, a.tab, a.rec, a.words);
    const uint32_t blocks = (b->n_pairs + 3u) / 4u;
    k_na_forward<<<blocks < (uint32_t)(sms * 16) ? blocks : (uint32_t)(sms * 16), 128, 0, s>>>(
        b->hap_bases, b->read_off, b->hap_off, b->pair_read, b->pair_hap, b->n_reads, b->n_haps, b->n_pairs,
        a.rec, a.pow, a.words, b->out_log10, b->out_flags);
    uint32_t status = 0;
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemcpyAsync(&status, a.words, sizeof(status), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (cur != device) cudaSetDevice(cur);
    if (e != cudaSuccess) return PHMM_ECUDA;
    if (status & kNaScratchFull) return PHMM_ENOMEM;
    if (status & (ST_BAD_INPUT | ST_TOO_LONG)) return PHMM_EINVAL;
    return PHMM_OK;
}
