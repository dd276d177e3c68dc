// Host-side launchers of the kernels (defined in kernels_f32.cu / kernels_f64.cu).
#pragma once

#include <cuda_runtime.h>

#include "phmm_internal.h"

namespace phmm {

struct PhredTables;

// FP32 unit
void launch_reset(const BatchHeader* H, int grid, cudaStream_t s);
void launch_prep32(const BatchHeader* H, const PhredTables* T, int grid, cudaStream_t s);
void launch_prep32_first(const BatchHeader* H, const PhredTables* T, int grid, cudaStream_t s);
void launch_forward32_long(const BatchHeader* H, const void* pow, int grid, cudaStream_t s);
// FP32 multi-warp kernels: kind 0 = lean engine (N 32, 16-warp CTAs), 1 = pipelined
// (N 32, 12-warp CTAs), 2 = pipelined (N 24, 16-warp CTAs), 3 = pipelined with packed
// column halves, one warp per pair running its 1024-column strips one after another
// (k_forward_serial, 4-warp CTAs), 4 = pipelined in 4-warp CTAs (3 per SM): strips of
// 4096 columns, so that a few very wide pairs spread over many SMs, 5 = the same 4-warp
// strips taken eight at a time by thread-block clusters, neighbouring strips linked
// through distributed shared memory (k_forward_cluster), 6 = every 1024-column strip of a
// pair on its own warp at the same time, the strips linked through global memory in blocks
// of 32 rows (a strip waits for its left neighbour's progress counter once per block,
// k_forward_wave), 7 = kind 6 on a grid of two CTAs per SM (fewer warps share each
// scheduler, so a long strip chain's row step is shorter), 8 = kind 6 with 16 columns per
// lane (512-column strips: twice the strips, each row step with half the in-lane chain).
constexpr int kNumLong = 9;
constexpr int kLongN[kNumLong] = {32, 32, 24, 32, 32, 32, 32, 32, 16};
constexpr int kLongCW[kNumLong] = {16, 12, 16, 1, 4, kClusterWarps, 1, 1, 1};
constexpr bool kLongSerial[kNumLong] = {false, false, false, true, false, false, false, false, false};
constexpr bool kLongWave[kNumLong] = {false, false, false, false, false, false, true, true, true};
constexpr int kSerialThreads = 128;
void launch_forward32_long_pipe(int kind, const BatchHeader* H, const void* pow, int grid, cudaStream_t s);
// Short-pair kernels by variant id (see kShortScalar / kShortPacked).
void launch_short_scalar(int id, const BatchHeader* H, const void* pow, int grid, cudaStream_t s);
void launch_short_packed(int id, const BatchHeader* H, const void* pow, int grid, cudaStream_t s);
void launch_finalize32(const BatchHeader* H, int grid, cudaStream_t s);
int occupancy_forward32_long();          // resident CTAs per SM
int occupancy_forward32_long_pipe(int kind);  // kind 5: resident clusters on the GPU
int occupancy_short_scalar(int id);
int occupancy_short_packed(int id);
// pow_row: a device pointer to one PowRow<float>
void launch_scan_test(const float* y, float* z, int n, const void* pow_row, cudaStream_t s);
// bnd: device buffer of at least 4 zero words; status: device word
void launch_wait_test(const void* bnd, uint32_t* status, cudaStream_t s);

// FP64 unit
void launch_prep64_all(const BatchHeader* H, const PhredTables* T, int grid, cudaStream_t s);
void launch_prep64_list(const BatchHeader* H, const PhredTables* T, int grid, cudaStream_t s);
// FP64 forward kernels (precision FP64): variant 0 = N 8 in 16-warp CTAs, 1 = N 16 in
// 8-warp CTAs (fewer padded columns and per-row operations per cell for pairs up to 512
// columns; the same 4096-column CTA width for wider pairs), both on the unfactored engine;
// 2 = short pairs (up to 512 columns) on the pipelined FP64 engine (J-form records, six
// FP64 operations per cell) and multi-warp pairs on the unfactored engine in 8-warp CTAs
// (CTA items only), two concurrent branches; 3 = as 2 with 32-column short teams (pairs
// up to 1024 columns) on the fused pipelined engine (no partials array).  pow: the FP64
// power table of that N (kF64N for the multi-warp kernel, kF64NS for the short teams).
constexpr int kNumF64 = 4;
constexpr int kF64N[kNumF64] = {8, 16, 16, 16};   // multi-warp (CTA) kernel: columns per lane
constexpr int kF64NS[kNumF64] = {8, 16, 16, 32};  // short teams: columns per lane
constexpr int kF64CW[kNumF64] = {16, 8, 8, 8};
constexpr bool f64_pipelined(int id) { return id >= 2; }
void launch_forward64(int id, const BatchHeader* H, const void* pow, int grid, cudaStream_t s);
void launch_short_pipe64(int id, const BatchHeader* H, const void* pow, int grid, cudaStream_t s);
int occupancy_short_pipe64(int id);
void launch_prep64_first(const BatchHeader* H, const PhredTables* T, int grid, cudaStream_t s);
void launch_finalize64(const BatchHeader* H, int grid, cudaStream_t s);
void launch_rescue64(const BatchHeader* H, const void* pow, int grid, cudaStream_t s);
void launch_single64(const BatchHeader* H, const void* pow, uint32_t pair, cudaStream_t s);
int occupancy_forward64(int id);

constexpr int kN64 = 8;       // columns per lane of the FP64 kernels
constexpr int kNLong32 = 32;  // columns per lane of FP32 multi-warp pairs
// FP32 short-pair kernel variants: columns per lane of scalar teams / packed teams.
constexpr int kNumScalar = 10;
constexpr int kShortScalarN[kNumScalar] = {32, 24, 24, 16, 32, 24, 16, 32, 24, 32};
// scalar ids whose kernel is the pipelined engine (Rec32J records)
constexpr bool kShortScalarPipe[kNumScalar] = {false, false, false, false, true, true, true, true, true, true};
// scalar ids whose pipelined engine packs the two column halves of a lane (FFMA2)
constexpr bool kShortScalarHalves[kNumScalar] = {false, false, false, false, false, false, false, true, true, true};
// scalar ids of the lean halves engine: fused row, records and carry powers from L1, four
// CTAs per SM
constexpr bool kShortScalarLean[kNumScalar] = {false, false, false, false, false, false, false, false, false, true};
constexpr int kNumPacked = 2;
constexpr int kShortPackedN[kNumPacked] = {12, 16};

}  // namespace phmm
