/*
 * phmm.h -- C ABI of the GB300 (sm_103a) row-wise PairHMM forward library.
 *
 * The library scores every (read, haplotype) pair of a batch as log10 P(read | hap)
 * with the PairHMM forward algorithm over the Match / Insertion / Deletion matrices
 * (paper, Section 2, Eq. 1-4), evaluated row by row as the paper's Section 3.1
 * reformulation proposes: each row's M and I cells come from the previous row in
 * parallel, and the in-row deletion dependency D[i][j] = T_MD_i M[i][j-1] + T_DD_i D[i][j-1]
 * (Eq. 2, unrolled in Eq. 5-6) is evaluated as a first-order linear-recurrence scan
 * (Section 3.4, Algorithm 1).  Every step runs in this library's CUDA kernels; the
 * ABI exposes plain pointers and sizes only.
 *
 * Conventions for every entry point:
 *   - Return value: PHMM_OK (0), PHMM_PENDING (1) or a negative phmm_status.  Errors are
 *     returned, never thrown across the ABI.  phmm_strerror() names them.
 *   - A context is bound to one CUDA device and one stream.  Calls on one context are
 *     serialised by an internal mutex (thread-safe per context).
 *
 * Input model (paper Section 2): a read of length l with four per-base quality strings
 * (base quality Q_i, insertion ins_i, deletion del_i, gap continuation gcp_i) and a
 * haplotype of length k.  Qualities are numeric Phred 0..93 (the paper's "Q - 33" is
 * the ASCII offset; subtract 33 before calling).  q(x) = 10^(-x/10):
 *   P(r_i|h_j) = 1 - q(Q_i) on a match, q(Q_i)/3 on a mismatch (Eq. 3); an 'N' on
 *   either side counts as a match;  T_MI_i = q(ins_i), T_MD_i = q(del_i),
 *   T_MM_i = 1 - T_MI_i - T_MD_i, T_II_i = T_DD_i = q(gcp_i), T_IM_i = T_DM_i = 1 - q(gcp_i)
 *   (Section 2 fixes 0.1 / 0.9, i.e. gcp = 10).
 * Output: log10 L with L = sum_j M[l][j] + I[l][j] / C (Eq. 4), where C = D[0][j] * k is
 * the initial scale of Eq. 1 (so L keeps the 1/k start prior).
 */
#ifndef PHMM_H
#define PHMM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define PHMM_ABI_VERSION 3

/* Opaque context: device arenas, stream, captured graphs, pending tickets. */
typedef struct phmm_ctx phmm_ctx;

typedef enum {
    PHMM_OK = 0,          /* done */
    PHMM_PENDING = 1,     /* phmm_poll: submitted work not finished yet */
    PHMM_EINVAL = -1,     /* bad argument, base other than ACGTN, quality > 93, empty
                             read or haplotype, non-monotone offsets, pair index out
                             of range */
    PHMM_ENOMEM = -2,     /* the batch's device footprint exceeds the memory budget */
    PHMM_EBUSY = -3,      /* max_inflight tickets already pending */
    PHMM_ECUDA = -4,      /* a CUDA runtime call failed (context unusable) */
    PHMM_ETIMEOUT = -5,   /* phmm_poll timed out, or a device-side bounded wait gave up */
    PHMM_ECANCELED = -6,  /* work cancelled by phmm_destroy */
    PHMM_ENOTFOUND = -7   /* unknown or already retired ticket */
} phmm_status;

typedef enum {
    PHMM_PREC_FP32_RESCUE = 0, /* FP32 bulk with power-of-two rescaling; pairs flagged
                                  by the underflow test are recomputed in FP64 (default) */
    PHMM_PREC_FP64 = 1,        /* every pair in FP64 (same batched engine) */
    PHMM_PREC_FP32_ONLY = 2    /* FP32 without the FP64 rescue pass (diagnostics) */
} phmm_precision;

/* phmm_config.flags */
#define PHMM_F_NO_GRAPH 0x1u        /* launch kernels directly instead of replaying a
                                       captured CUDA graph */
#define PHMM_F_LAUNCH_PER_PAIR 0x2u /* with PHMM_PREC_FP64: one kernel launch per pair
                                       (the plain FP64 comparator) */
#define PHMM_F_FORCE_RESCUE 0x4u    /* flag every pair for the FP64 rescue pass (tests) */
/* FP32 multi-warp pairs (k > 1024): force one kernel instead of the tuner's choice --
 * the lean engine (16-warp CTAs), the pipelined engine with 32 columns per lane
 * (12-warp CTAs) or with 24 columns per lane (16-warp CTAs), or the serial one below.
 * At most one may be set. */
#define PHMM_F_LONG_LEAN 0x10u
#define PHMM_F_LONG_PIPE32 0x20u
#define PHMM_F_LONG_PIPE24 0x40u
/* ... or one warp per multi-warp pair, running its 1024-column strips one after
 * another (no warp waits on another; for batches with many long pairs). */
#define PHMM_F_LONG_SERIAL 0x100u
/* ... or the pipelined engine in 4-warp CTAs (strips of 4096 columns: a few very wide
 * pairs spread over many SMs). */
#define PHMM_F_LONG_PIPE4 0x200u
/* ... or the same 4-warp strips run by thread-block clusters of eight CTAs, neighbouring
 * strips exchanging their boundary rows through distributed shared memory. */
#define PHMM_F_LONG_CLUSTER 0x400u
/* ... or every strip of a pair on its own warp at the same time, strips linked through
 * global memory in blocks of 32 rows (a strip waits for its left neighbour once per
 * block: for a few very wide pairs); the tuner picks the strip width and grid (1024
 * columns on the resident maximum or on two CTAs per SM, or 512 columns). */
#define PHMM_F_LONG_WAVE 0x800u
/* ... or only the 512-column wave strips (multi-warp kind 8). */
#define PHMM_F_LONG_WAVE16 0x1000u
/* No measured tuning: the built-in cost model and defaults choose the kernels.  For
 * serving, where nearly every batch (epoch) has a new shape and tuning would re-run it. */
#define PHMM_F_NO_TUNE 0x80u

typedef struct {
    int device;               /* CUDA device ordinal */
    int precision;            /* phmm_precision */
    size_t mem_budget_bytes;  /* admission budget for one batch's device footprint;
                                 0 = 90% of the device's free memory at create time */
    unsigned max_inflight;    /* tickets that may be pending at once; 0 = 4 */
    unsigned flags;           /* PHMM_F_* */
    void *stream;             /* cudaStream_t to run on; NULL = a stream owned by the
                                 context.  The caller keeps a passed stream alive until
                                 phmm_destroy. */
    int cols_per_lane;        /* haplotype columns per thread (the paper's N) for FP32 short
                                 pairs: 12 or 16 fixes the packed-team width, 24 or 32 the
                                 scalar-team width, 0 = chosen by the built-in tuner.
                                 Multi-warp pairs use 32 (FP32).  With PHMM_PREC_FP64: 8
                                 or 16 fixes the unfactored FP64 variant (8 columns per lane
                                 in 16-warp CTAs, 16 in 8-warp CTAs), 0 = tuner. */
    int kernel_variant;       /* FP32 short-pair kernels the tuner may use: 0 = any; 1 =
                                 pairs of the same read share packed teams (two haplotypes
                                 per thread in float2 halves), the rest run in scalar
                                 teams; 2 = scalar teams only (lean or pipelined engine);
                                 3 = lean scalar engine only; 4 = pipelined scalar engine
                                 only (the next row's scan-independent work overlaps the
                                 deletion scan); 5 = pipelined engine with each lane's two
                                 column halves in packed FP32 pairs; 6 = its lean form
                                 (the next row's partials formed inside the row, records
                                 and carry powers read from L1: four CTAs per SM).  With
                                 PHMM_PREC_FP64, 4 fixes the pipelined FP64 variant with
                                 16-column short teams (pairs up to 512 columns on the
                                 J-form engine, six FP64 operations per cell), 5 or 6 the
                                 one with 32-column fused teams (pairs up to 1024
                                 columns) */
    double fp32_tolerance;    /* largest |error of log10 L| accepted from the FP32 pass
                                 (0 = 1e-3): with PHMM_PREC_FP32_RESCUE a pair whose
                                 a-priori FP32 rounding bound exceeds it is recomputed in
                                 FP64 (flag PHMM_PAIR_DANGER) */
} phmm_config;

/*
 * One batch.  Reads and haplotypes are concatenated; offsets have n+1 entries and must
 * be non-decreasing with lengths >= 1.  Bases are ASCII A/C/G/T/N (either case).  The
 * four quality arrays have the layout of read_bases.  A pair is (pair_read[p],
 * pair_hap[p]).  All pointers are host pointers unless inputs_on_device (then every
 * input array is a device pointer of the context's device) or outputs_on_device.
 */
typedef struct {
    uint32_t n_reads;
    const uint8_t *read_bases;
    const uint64_t *read_off;
    const uint8_t *base_q;
    const uint8_t *ins_q;
    const uint8_t *del_q;
    const uint8_t *gcp_q;
    uint32_t n_haps;
    const uint8_t *hap_bases;
    const uint64_t *hap_off;
    uint32_t n_pairs;
    const uint32_t *pair_read;
    const uint32_t *pair_hap;
    double *out_log10;        /* n_pairs results, caller-owned */
    uint8_t *out_flags;       /* optional (may be NULL): per pair PHMM_PAIR_* bits */
    int inputs_on_device;
    int outputs_on_device;
} phmm_batch;

/* out_flags bits */
#define PHMM_PAIR_RESCUED 0x1u  /* recomputed in FP64 by the rescue pass */
#define PHMM_PAIR_RESCALED 0x2u /* power-of-two rescaling was applied */
#define PHMM_PAIR_FP64 0x4u     /* final value computed in FP64 */
/* why the FP32 pass selected a pair for the FP64 rescue (kept when it was rescued) */
#define PHMM_PAIR_DANGER 0x8u     /* FP32 accuracy not assured: a checkpoint row maximum
                                     fell below the danger level, or the pair's a-priori
                                     FP32 rounding bound exceeds the FP32 tolerance */
#define PHMM_PAIR_NONFINITE 0x10u /* an inf / nan appeared */
#define PHMM_PAIR_SMALL_SUM 0x20u /* the FP32 last-row sum failed the underflow test */
#define PHMM_PAIR_DEGENERATE 0x40u /* gcp Phred 0 (T_DD = 1): factored FP32 form unusable */
#define PHMM_PAIR_ERROR 0x80u   /* invalid input or device error for this pair */

/* Per-ticket statistics (device times from CUDA events on the context's stream). */
typedef struct {
    uint64_t cells;           /* sum over pairs of l * k */
    uint32_t n_pairs;
    uint32_t n_rescued;       /* pairs recomputed in FP64 by the rescue pass */
    uint32_t n_long;          /* pairs that spanned more than one warp */
    uint32_t cols_per_lane;   /* N used */
    float ms_total;           /* device time from first to last kernel of the ticket */
    float ms_forward;         /* the main FP32 (or FP64) forward kernel(s) */
    float ms_rescue;          /* FP64 rescue pass (0 if nothing was rescued) */
    float ms_h2d;             /* host-to-device copies (host inputs only) */
    uint32_t kernel_launches; /* kernels launched for the ticket */
    uint32_t status_bits;     /* device status word (0 = clean) */
    float ms_host;            /* host time of phmm_submit_batch's planning and enqueue */
    /* Kernels the plan ran (-1: that branch had no work).  FP64 precision: short_kernel =
     * the FP64 forward variant (0: 8 columns per lane in 16-warp CTAs, 1: 16 columns per
     * lane in 8-warp CTAs, 2: short pairs on the pipelined FP64 engine, 16 columns per
     * lane, and multi-warp pairs as in 1, 3: as 2 with 32-column fused short teams), the
     * other two -1.  FP32:
     * short_kernel = scalar-team variant 0..9 (k_short_scalar<32,4>, <24,4>, <24,5>,
     * <16,6>, k_short_pipe<32,3>, <24,4>, <16,4>, k_short_pipe2<32,3>, <24,4>, and the
     * lean k_short_pipe2<32,4>);
     * packed_kernel = packed-team variant 0..1 (k_short_packed<12,4>, <16,3>);
     * long_kernel = multi-warp kind 0..8 (lean k_forward<32>, k_forward_pipe<32,12>,
     * k_forward_pipe<24,16>, k_forward_serial<32,3>, k_forward_pipe<32,4>,
     * k_forward_cluster<32,4,8>, k_forward_wave<32,3>, the same on two CTAs per SM,
     * k_forward_wave<16,3>). */
    int32_t short_kernel;
    int32_t packed_kernel;
    int32_t long_kernel;
    /* The FP32 forward pass runs three branches concurrently, each a persistent kernel on
     * its own stream: [0] scalar short teams, [1] packed short teams, [2] multi-warp pairs.
     * cells_branch = sum of l * k over the pairs each branch scored; ms_branch = device time
     * of each branch's kernel (CUDA events on its stream).  FP64: [0] holds the whole
     * forward pass. */
    uint64_t cells_branch[3];
    float ms_branch[3];
} phmm_stats;

/* Create a context on cfg->device.  *out receives the handle.  PHMM_EINVAL on a bad
 * config, PHMM_ECUDA if the device cannot be used. */
int phmm_create(const phmm_config *cfg, phmm_ctx **out);

/* Validate a batch, copy host inputs to device arenas (before returning, so the caller
 * may reuse host input buffers immediately), and enqueue the forward computation.
 * *ticket identifies it for phmm_poll.  Device inputs and all outputs must stay valid
 * until phmm_poll returns a terminal status for the ticket.
 * Each in-flight batch occupies one of max_inflight slots with its own device arenas and
 * streams, so batches submitted back to back run concurrently on the device.  They are
 * ordered after work already queued on the context's stream (config.stream) at submit
 * time, and work queued on that stream afterwards waits for their outputs.
 * PHMM_EINVAL (bad offsets, index or length) / PHMM_ENOMEM (the batch alone exceeds the
 * memory budget: it can never be admitted) / PHMM_EBUSY (no free slot, or the in-flight
 * batches hold too much of the budget: retry after polling) / PHMM_ECUDA. */
int phmm_submit_batch(phmm_ctx *ctx, const phmm_batch *batch, uint64_t *ticket);

/* Upper bound of the device bytes a batch with host inputs needs while in flight (inputs,
 * per-base coefficient records, per-pair descriptors and work items, strip boundaries
 * of very wide pairs, FP64 rescue scratch), as counted against the memory budget.
 * Offsets and pair indices must be valid (PHMM_EINVAL otherwise); bases and qualities
 * are not read. */
int phmm_batch_footprint(phmm_ctx *ctx, const phmm_batch *batch, uint64_t *bytes);

/* Wait up to timeout_ms (0 = just test, < 0 = forever) for a ticket.  PHMM_OK when its
 * outputs are written, PHMM_PENDING if not finished, PHMM_EINVAL if a base or quality of
 * the batch was invalid (those pairs carry PHMM_PAIR_ERROR and NaN), PHMM_ETIMEOUT if a
 * device-side wait gave up.  A terminal status retires the ticket. */
int phmm_poll(phmm_ctx *ctx, uint64_t ticket, int timeout_ms);

/* Statistics of a finished (not yet retired, or the most recently retired) ticket. */
int phmm_get_stats(phmm_ctx *ctx, uint64_t ticket, phmm_stats *out);

/* Cancel pending work (waits for the stream), free every device and host resource. */
void phmm_destroy(phmm_ctx *ctx);

/* Static description of a status code. */
const char *phmm_strerror(int status);

/* ABI version of the loaded library (PHMM_ABI_VERSION at build time). */
int phmm_abi_version(void);

/* Number of SMs and the FP32 cell-update roofline of the context's device:
 * 2 * 128 FP32 lanes * SMs * max SM clock / 12 FLOP per cell (Eq. 2 as written:
 * 6 multiplies and 6 adds per cell).  Writes cells per second into *cups. */
int phmm_device_info(phmm_ctx *ctx, int *sms, double *max_clock_mhz, double *cups);

/*
 * Test entry: the lane-level linear-recurrence scan of Section 3.4 (Algorithm 1) on its
 * own, as the forward kernels run it: one warp, each lane owns 32 consecutive elements,
 * a sequential pass inside the lane, then a warp shuffle scan of the lane aggregates
 * with multiplier a^32.  For n values y[0..n) (device pointer, FP32, 1 <= n <= 1024)
 * writes z[t] = sum_{s <= t} a^(t-s) y[s] (device pointer).  Runs synchronously.
 */
int phmm_scan_test(phmm_ctx *ctx, const float *y, float *z, int n, float a);

/*
 * Test entry: the bounded device-side wait that links column strips (and, in shared
 * memory, warp segments) run on a boundary that is never written.  The wait gives up
 * after its poll limit (about a second) instead of hanging, and the call returns
 * PHMM_ETIMEOUT; the context stays usable.  Runs synchronously on the context's stream.
 */
int phmm_wait_test(phmm_ctx *ctx);

/*
 * Test entry (host only, no device needed): builds the work plan the runtime would use
 * for a batch with read lengths l[p], haplotype lengths k[p] and read index pair_read[p]
 * (n pairs), for precision (PHMM_PREC_*) and, in FP32, the short-pair kernel ids (scalar
 * 0..9, packed -1..1) and the multi-warp kernel kind (0..8, as phmm_stats.long_kernel),
 * and checks it: every pair scheduled exactly once; teams inside their warp, disjoint and
 * wide enough, packed pairs sharing a read; CTA warp ranges inside the CTA and disjoint; a
 * wide pair's strips tiling its columns in order, never placed in an earlier work item
 * than the strip to their left, with matching and disjoint boundary buffers and partial
 * slots; in the serial kind one item per wide pair, its strips' partial slots disjoint and
 * its rows within the serial scratch.  stats[8] receives:
 * teams, warp items, packed warp items, CTA items, CTA pairs, striped pairs, pairs too
 * long, and the number of the failed check (0 = none).  PHMM_OK or PHMM_EINVAL.
 */
int phmm_plan_check(const uint32_t *l, const uint32_t *k, const uint32_t *pair_read, uint32_t n,
                    int precision, int scal_id, int pack_id, int long_kind, uint64_t *stats);

/*
 * Serving: continuous batching of independent requests (an active region: R reads x H
 * haplotypes, scored as one phmm_batch).  The paper has no serving layer; this loop is
 * built on phmm_submit_batch / phmm_poll of one context.  A scheduler thread keeps the
 * waiting requests in arrival order.  Whenever an epoch slot is free it forms an epoch
 * (one batch) whose summed footprint (phmm_batch_footprint) fits in the budget left by
 * epochs still on the device, and submits it.  Up to max_inflight_epochs epochs run
 * concurrently, so requests that arrive while others are on the GPU start as soon as a
 * slot and memory free up.  Size classes keep small requests from waiting behind large
 * ones: requests of at most small_cells cells (sum of l * k) form epochs of their own and
 * go first; larger requests follow in arrival order, split into chunks of consecutive
 * pairs of at most epoch_cells cells, each chunk an epoch (so no epoch holds the device
 * for long); large epochs use at most max_inflight_epochs - 1 slots; a large request that
 * has waited longer than max_wait_ms goes ahead of small ones.  When an epoch finishes,
 * its results are copied to the requests' output buffers; a request completes when all
 * its pairs are done.
 */
typedef struct phmm_server phmm_server;

typedef struct {
    uint64_t mem_budget_bytes;     /* device bytes admitted across in-flight epochs (0: 40 GiB) */
    uint32_t max_epoch_pairs;      /* pairs per epoch (0: 2^20) */
    uint32_t max_inflight_epochs;  /* concurrent epochs (0: 2); the context needs as many slots */
    uint32_t max_pending;          /* waiting requests before enqueue returns PHMM_EBUSY (0: no limit) */
    uint32_t max_wait_ms;          /* a large request waiting longer goes ahead of small ones (0: 2000) */
    uint64_t epoch_cells;          /* cell budget of one epoch; larger requests are split (0: 2e10) */
    uint64_t small_cells;          /* requests of at most this many cells are small (0: epoch_cells / 20) */
} phmm_server_config;

typedef struct {
    uint64_t enqueued, admitted, completed, failed; /* requests */
    uint64_t epochs;                                /* batches submitted */
    uint64_t pending;                               /* requests waiting for admission */
    uint64_t inflight;                              /* requests admitted, not completed */
    uint64_t cells_completed;                       /* sum of l * k over completed requests */
    uint64_t bytes_inflight;                        /* admitted footprint on the device */
} phmm_server_stats;

/* Start a server on ctx (which must outlive it and must not be used by the caller while
 * the server runs).  PHMM_EINVAL on a bad argument. */
int phmm_server_create(phmm_ctx *ctx, const phmm_server_config *cfg, phmm_server **out);

/* Queue one request (a phmm_batch with host inputs and host outputs).  Inputs are copied
 * before the call returns; out_log10 / out_flags must stay valid until phmm_server_poll
 * returns a terminal status for *req_id.  PHMM_EINVAL (bad offsets, indices or lengths),
 * PHMM_ENOMEM (footprint above the whole budget), PHMM_EBUSY (max_pending reached). */
int phmm_server_enqueue(phmm_server *srv, const phmm_batch *request, uint64_t *req_id);

/* Wait up to timeout_ms (0 = test, < 0 = forever) for a request.  PHMM_OK when its outputs
 * are written, PHMM_PENDING, PHMM_EINVAL when one of its pairs had an invalid base or
 * quality (that pair holds NaN and PHMM_PAIR_ERROR), or the error of its epoch.
 * *latency_ms (optional) receives enqueue-to-completion time.  A terminal status retires
 * the id (PHMM_ENOTFOUND afterwards). */
int phmm_server_poll(phmm_server *srv, uint64_t req_id, int timeout_ms, double *latency_ms);

/* Counters since creation. */
int phmm_server_get_stats(phmm_server *srv, phmm_server_stats *out);

/* Stop admitting, wait for epochs on the device, fail waiting requests with
 * PHMM_ECANCELED, stop the scheduler and free the server (not the context). */
void phmm_server_destroy(phmm_server *srv);

/*
 * Allocation-free FP32 forward pass (the paper has no counterpart: this is an interface
 * for callers that cannot allocate device memory at call time -- code inside a host
 * framework that owns the device heap and forbids cudaMalloc/cudaFree on its threads, or
 * a process that reserved all device memory up front).  It needs no context and calls no
 * allocating routine: besides the caller's buffers it uses fixed scratch arrays built
 * into the library (about 32 MiB of read-row records plus small tables), which every GPU
 * that loads the library keeps until the process exits.
 *   device   CUDA device ordinal; the call makes it current for its duration.  The first
 *            call on a device looks up the scratch addresses (cudaGetSymbolAddress), so
 *            make that first call outside any stream capture.
 *   stream   cudaStream_t to run on (NULL = legacy default stream); the call waits for
 *            its own work to finish before returning (it reads its status word back), so
 *            it blocks the host and cannot be captured into a CUDA graph.
 *   batch    as for phmm_submit_batch, with inputs_on_device = outputs_on_device = 1 (all
 *            pointers are device pointers) and out_flags required.
 * Offsets are checked on the device before they are used: a pair whose read or
 * haplotype is empty, runs backwards or ends past the last offset gets NaN and
 * PHMM_PAIR_ERROR, and the call returns PHMM_EINVAL (as phmm_submit_batch would).
 * Limits: at most 2^20 read bases in the batch (PHMM_ENOMEM beyond) and haplotypes of at
 * most 1024 bases (such pairs get NaN and PHMM_PAIR_ERROR; the call returns PHMM_EINVAL).
 * FP32 only (no FP64 rescue pass): out_flags sets PHMM_PAIR_DANGER / NONFINITE /
 * SMALL_SUM / DEGENERATE by the same tests the regular API uses to pick pairs for its FP64
 * pass, and the call still returns PHMM_OK for such pairs.  The per-row coefficients are
 * rounded with the regular API's default seed, so they equal a default context's.  All
 * calls share the scratch, so calls that overlap on the GPU (other streams or threads)
 * race and must be serialised.
 */
int phmm_forward_noalloc(int device, void *stream, const phmm_batch *batch);

#ifdef __cplusplus
}
#endif

#endif /* PHMM_H */
