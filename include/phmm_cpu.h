/*
 * phmm_cpu -- the row-wise PairHMM forward pass on the host CPU (a comparator for the GPU
 * library; a separate shared library, libphmm_cpu.so, that libphmm.so never calls).
 *
 * It evaluates the same recurrences as the GPU path (Section 2, Eq. 1-4) in the paper's
 * row-wise CPU form (Section 3.1, Eq. 5-7): per row, every column's Match and Insertion
 * value from the previous row in vectorisable loops, then the deletion chain
 * D_ij = T_MD M_i,j-1 + g_i D_i,j-1 as a first-order linear recurrence, split into blocks
 * that run as independent chains and are then joined by their carries g^m.  Arithmetic is
 * FP64 with power-of-two rescaling every 16 rows, so no pair needs a second pass.
 *
 * Inputs use the phmm_batch layout of phmm.h; every pointer must be a host pointer
 * (inputs_on_device and outputs_on_device are ignored and must be 0).
 */
#ifndef PHMM_CPU_H
#define PHMM_CPU_H

#include "phmm.h"

#ifdef __cplusplus
extern "C" {
#endif

/* log10 L for every pair of b into b->out_log10 (caller-owned, n_pairs doubles); when
 * b->out_flags is not NULL, each pair's flags get PHMM_PAIR_FP64, or PHMM_PAIR_ERROR for an
 * invalid pair (its result is NaN).  n_threads POSIX threads take pairs from a shared
 * counter (n_threads <= 0: one per online core).  Returns PHMM_OK, or PHMM_EINVAL for a
 * malformed batch (NULL arrays, offsets out of order or out of range) -- per-pair problems
 * (a base other than ACGTN, a quality above 93, an empty read or haplotype) mark only
 * that pair.  PHMM_ENOMEM if scratch memory cannot be allocated. */
int phmm_cpu_forward(const phmm_batch *b, int n_threads);

#ifdef __cplusplus
}
#endif

#endif /* PHMM_CPU_H */
