/*
 * phmm_cpu -- the row-wise PairHMM forward pass on the host CPU (a comparator for the GPU
 * library; a separate shared library, libphmm_cpu.so, that libphmm.so never calls).
 *
 * It evaluates the same recurrences as the GPU path (Section 2, Eq. 1-4) with the paper's
 * CPU mapping (Section 3.5): one (read, haplotype) pair per SIMD lane, pairs of similar
 * length packed side by side (on AArch64 8 pairs per FP32 pack, 4 per FP64 pack), every
 * instruction updating one cell of each pair of a pack.  Per lane, rows are computed in
 * order and the deletion chain D_ij = T_MD M_i,j-1 + g_i D_i,j-1 left to right, so no scan
 * is needed.  Power-of-two rescaling per lane keeps long reads in range.
 *
 * Inputs use the phmm_batch layout of phmm.h; every pointer must be a host pointer
 * (inputs_on_device and outputs_on_device must be 0).
 */
#ifndef PHMM_CPU_H
#define PHMM_CPU_H

#include "phmm.h"

#ifdef __cplusplus
extern "C" {
#endif

/* log10 L for every pair of b into b->out_log10 (caller-owned, n_pairs doubles).
 *   n_threads       POSIX threads taking packs from a shared counter (<= 0: one per
 *                   online core); results do not depend on it.
 *   precision       PHMM_PREC_FP32_RESCUE: FP32, then FP64 for every pair the FP32 pass
 *                   flags (a non-finite value, a checkpoint maximum below the danger
 *                   level, the last-row sum below 1e4 * 3 l k FLT_MIN, or an a-priori
 *                   rounding bound above fp32_tolerance); PHMM_PREC_FP64: every pair in
 *                   FP64; PHMM_PREC_FP32_ONLY: FP32, flagged pairs keep their FP32 value.
 *   fp32_tolerance  largest |error of log10 L| accepted from the FP32 pass (0: 1e-3).
 * b->out_flags (optional) gets the PHMM_PAIR_* bits of phmm.h per pair: RESCALED, FP64,
 * RESCUED, the reason bits (DANGER also covers the rounding bound), or ERROR for an
 * invalid pair (its result is NaN).  Returns PHMM_OK, or PHMM_EINVAL for a malformed
 * batch (NULL arrays, offsets out of order or out of range, a bad precision or
 * tolerance) -- per-pair problems (a base other than ACGTN, a quality above 93, an empty
 * read or haplotype) mark only that pair.  PHMM_ENOMEM if scratch memory cannot be
 * allocated. */
int phmm_cpu_forward(const phmm_batch *b, int n_threads, int precision, double fp32_tolerance);

#ifdef __cplusplus
}
#endif

#endif /* PHMM_CPU_H */
