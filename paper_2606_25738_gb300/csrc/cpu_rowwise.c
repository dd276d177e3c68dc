/*
 * Row-wise PairHMM forward pass on the host CPU (include/phmm_cpu.h).
 *
 * Per pair, rows i = 1..l over columns j = 1..k (Section 2, Eq. 1-4):
 *   M_ij = P_ij (T_MM_i M_i-1,j-1 + T_IM_i I_i-1,j-1 + T_DM_i D_i-1,j-1)
 *   I_ij = T_MI_i M_i-1,j + g_i I_i-1,j
 *   D_ij = T_MD_i M_i,j-1 + g_i D_i,j-1
 * with D_0j = C/k for every j (row 0), column 0 zero for i >= 1, and L = sum_j M_lj + I_lj
 * over C.  T_MI = q(ins), T_MD = q(del), T_MM = 1 - T_MI - T_MD, g = q(gcp),
 * T_IM = T_DM = 1 - g; P = 1 - q(base) on a match (an N on either side matches), else
 * q(base) / 3; q(x) = 10^(-x / 10).
 *
 * CPU mapping (the paper's Section 3.5): one pair per SIMD lane.  Pairs are sorted by
 * length (read-length class, then haplotype length) and taken in packs of equal-ish
 * shape; a pack's lanes step through their rows and columns together, so every
 * instruction updates one cell of every pair of the pack (cpu_engine.inc).  The vectors
 * are the compiler's generic vector types: the same source builds for NEON on Arm and
 * SSE2 on x86, with no intrinsics and no target flags.
 *
 * Range: power-of-two rescaling per lane at checkpoints every R rows (R from the pack's
 * worst per-row drop and growth), folded into the next row's coefficients.
 * Precision (phmm_precision): FP32 with FP64 rescue of flagged pairs, FP64 for every
 * pair, or FP32 alone.  The FP32 pass flags a pair for the FP64 pass on the same tests
 * as the GPU library: a non-finite value, a checkpoint maximum below the danger level,
 * the last-row sum below tau(l, k) = 1e4 * 3 l k FLT_MIN (on x86 hosts, which flush
 * cells below 2^-106 to zero, 2^-106 instead of FLT_MIN), or an a-priori rounding bound
 * above the FP32 tolerance.  FP32 per-row coefficients are stochastically rounded from
 * double, so their rounding errors average out over long reads instead of drifting.
 */
#include "phmm_cpu.h"

#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <unistd.h>

/* Lanes per pack: one 128-bit register per operation (wider generic vectors measured
 * slower on Neoverse-V2: the per-row coefficients no longer fit the register file). */
#define W32 4 /* FP32 lanes per pack */
#define W64 2 /* FP64 lanes per pack */

/* Cells at or below FLUSH are stored as zero.  x86 cores compute with subnormal values
 * far slower, so there they are flushed (2^-106 FP32, 2^-1000 FP64); AArch64 cores
 * handle them at full speed (measured on Neoverse-V2: flushing cost more than it saved),
 * so there nothing is flushed beyond what the format itself does. */
#if defined(__aarch64__)
#define FLUSH32 0.0f
#define FLUSH64 0.0
#else
#define FLUSH32 0x1.0p-106f
#define FLUSH64 0x1.0p-1000
#endif
typedef float v32f __attribute__((vector_size(W32 * sizeof(float))));
typedef int32_t v32i __attribute__((vector_size(W32 * sizeof(int32_t))));
typedef double v64d __attribute__((vector_size(W64 * sizeof(double))));
typedef int64_t v64i __attribute__((vector_size(W64 * sizeof(int64_t))));

static double q_tab[94];
static pthread_once_t q_once = PTHREAD_ONCE_INIT;
static void q_init(void) {
    for (int x = 0; x < 94; ++x) q_tab[x] = pow(10.0, -(double)x / 10.0);
}

/* base as a bit set: A 1, C 2, G 4, T 8, N 15 (an N matches everything); 0 = invalid */
static int32_t base_bits(uint8_t c) {
    switch (c) {
    case 'A': case 'a': return 1;
    case 'C': case 'c': return 2;
    case 'G': case 'g': return 4;
    case 'T': case 't': return 8;
    case 'N': case 'n': return 15;
    default: return 0;
    }
}

/* SplitMix64 finaliser (Steele, Lea & Flood 2014): a counter-based uniform source. */
static uint64_t mix64(uint64_t z) {
    z += 0x9e3779b97f4a7c15ull;
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
    return z ^ (z >> 31);
}

/* x rounded to float stochastically: to one of the two neighbouring floats, with
 * probabilities that make the expected value x (unbiased up to 2^-16 of a unit in the last
 * place), from a 16-bit uniform u16 (a quarter of one hash of the read base index). */
static float sr_round(double x, uint32_t u16) {
    const float f = (float)x; /* nearest */
    const double e = x - (double)f;
    if (e == 0.0 || !(fabs(x) < 3.0e38)) return f;
    float g;
    if (f != 0.0f) {
        /* the neighbour on the side of x: one step of the bit pattern away from or
         * towards zero */
        uint32_t fb;
        memcpy(&fb, &f, 4);
        fb += ((e > 0.0) == (f > 0.0f)) ? 1u : (uint32_t)-1;
        memcpy(&g, &fb, 4);
    } else {
        g = nextafterf(f, e > 0.0 ? INFINITY : -INFINITY);
    }
    const double gap = fabs((double)g - (double)f);
    return ((double)u16 + 0.5) * 0x1.0p-16 * gap < fabs(e) ? g : f;
}

/* A-priori bound on |log10 L(FP32) - log10 L| for a pair of l rows and k columns.
 * Every term of the forward sum is a product of nonnegative factors and every sum adds
 * nonnegative terms, so no cancellation occurs and the relative error of L is bounded by
 * the roundings along one path: at most 16 per row (coefficients and cell arithmetic)
 * and 4 per column (the deletion chain and its carries), each below u = 2^-23.  The
 * coefficient roundings are stochastic (independent, mean zero) and the cell roundings
 * are modelled the same way, so the sum of m of them stays below lambda sqrt(m) u except
 * with probability 2 exp(-lambda^2 / 2) (probabilistic rounding-error analysis, Higham &
 * Mary 2019; for stochastic rounding, Connolly, Higham & Mary 2021); lambda = 6.5 makes
 * that 1.4e-9.  A deterministic part covers the coefficients' own double precision
 * (8 per row, 2^-46 each). */
static double fp32_bound_log10(double l, double k) {
    const double u = 0x1.0p-23, lambda = 6.5;
    return (lambda * sqrt(16.0 * l + 4.0 * k) * u + 8.0 * l * 0x1.0p-46) / log(10.0);
}

typedef struct {
    int n;                 /* pairs in the pack (lanes beyond n are idle) */
    uint32_t lmax, kmax, R;
    uint32_t idx[W32];     /* pair indices */
    uint32_t l[W32], k[W32];
    uint64_t r0[W32], h0[W32];
    uint64_t c0[W32];      /* the lane's read in the coefficient table (records) */
} pack;

/* Per-row coefficients of every read base the pass uses, computed once per read (a read
 * is shared by all its pairs) and in parallel, as NC values per base.  FP64: 1 - e, e / 3,
 * T_MM, T_DM = 1 - g, T_MI, g, (1 - g) T_MD of the previous row (1 on a read's first row),
 * and the read base's bit set.  FP32 takes the factor T_IM = T_DM = 1 - g of Eq. 2 out of
 * the match update (one multiply less per cell): (1 - e)(1 - g), (e / 3)(1 - g),
 * T_MM / (1 - g), 1, T_MI, g, T_MD of the previous row, the bit set; a row with
 * 1 - g < 2^-20 cannot be factored and carries DEGEN_BIT in its bit set instead (its pair
 * goes to the FP64 pass).  FP32 tables hold the values stochastically rounded. */
#define NC 8
#define DEGEN_BIT 0x100

typedef struct {
    double S;
    int E;
    uint32_t flags;
    int nomem;
} pair_result;

typedef struct {
    void *buf;
    size_t cap;
} cpu_scratch;

static int scratch_reserve(cpu_scratch *s, size_t bytes) {
    if (bytes <= s->cap) return 1;
    free(s->buf);
    bytes = (bytes + 63) & ~(size_t)63;
    s->buf = aligned_alloc(64, bytes);
    s->cap = s->buf ? bytes : 0;
    return s->buf != NULL;
}

/* FP32 engine: C = 2^120; the lane maximum is brought back to 2^96 when it leaves
 * (2^40, 2^100]; below 2^-100 the pair is flagged; cells at or below 2^-106 are flushed
 * to zero (the underflow test below accounts for them). */
#define ENG_NAME pack_forward32
#define ENG_T float
#define ENG_V v32f
#define ENG_VI v32i
#define ENG_W W32
#define ENG_SR 1
#define ENG_FACTOR 1
#define ENG_LOG2C 120
#define ENG_HI 100
#define ENG_LO 40
#define ENG_TARGET 96
#define ENG_DANGER (-100)
#define ENG_MAXSHIFT 126
#define ENG_FLUSH FLUSH32
#include "cpu_engine.inc"
#undef ENG_NAME
#undef ENG_T
#undef ENG_V
#undef ENG_VI
#undef ENG_W
#undef ENG_SR
#undef ENG_FACTOR
#undef ENG_LOG2C
#undef ENG_HI
#undef ENG_LO
#undef ENG_TARGET
#undef ENG_DANGER
#undef ENG_MAXSHIFT
#undef ENG_FLUSH

/* FP64 engine: C = 2^1020; maximum kept in (2^300, 2^900], target 2^800; cells at or
 * below 2^-1000 are flushed to zero. */
#define ENG_NAME pack_forward64
#define ENG_T double
#define ENG_V v64d
#define ENG_VI v64i
#define ENG_W W64
#define ENG_SR 0
#define ENG_FACTOR 0
#define ENG_LOG2C 1020
#define ENG_HI 900
#define ENG_LO 300
#define ENG_TARGET 800
#define ENG_DANGER (-950)
#define ENG_MAXSHIFT 1020
#define ENG_FLUSH FLUSH64
#include "cpu_engine.inc"

/* Checkpoint interval of a pack: between checkpoints the lane maximum can fall by at most
 * min(T_MI, g) per row (I_ij >= T_MI M_i-1,j and >= g I_i-1,j) and grow by at most the
 * row's largest transition sum; R keeps both within the range budgets. */
static uint32_t pack_interval(const phmm_batch *b, const pack *pk, double drop_budget, double grow_budget) {
    double dmax = 1e-3, gmax = 1e-3;
    for (int w = 0; w < pk->n; ++w) {
        const uint64_t r0 = pk->r0[w];
        for (uint32_t i = 0; i < pk->l[w]; ++i) {
            const double qi = q_tab[b->ins_q[r0 + i]], qd = q_tab[b->del_q[r0 + i]], g = q_tab[b->gcp_q[r0 + i]];
            const double lo = qi < g ? qi : g;
            const double drop = lo > 0.0 ? -log2(lo) : 1e9;
            /* D adds up to T_MD / (1 - g) times the row's M (k times at g = 1) */
            const double dg = 1.0 - g > 1.0 / (double)pk->k[w] ? qd / (1.0 - g) : qd * (double)pk->k[w];
            const double grow = log2(fmax(fmax(1.0 - qi - qd + (1.0 - g) * (1.0 + dg), qi + g), 1.0));
            if (drop > dmax) dmax = drop;
            if (grow > gmax) gmax = grow;
        }
    }
    double r = fmin(drop_budget / dmax, grow_budget / gmax);
    if (r > 32.0) r = 32.0;
    /* even when it can be: rows go through the columns two at a time, and a checkpoint
     * then always follows the second row of a pair (its maximum taken in that pass) */
    const uint32_t R = r < 1.0 ? 1u : (uint32_t)r;
    return R >= 2 ? R & ~1u : R;
}

/* ------------------------------------------------------------------------------------ */

typedef struct {
    const phmm_batch *b;
    pack *packs;
    uint32_t n_packs;
    int fp64;
    uint32_t next;
    pthread_mutex_t mu;
    int nomem;
    pair_result *res; /* per pair */
    const void *coef; /* coefficient table of the pass (float or double records) */
} job;

static void *worker(void *arg) {
    job *J = (job *)arg;
    cpu_scratch s = {NULL, 0};
    pair_result pr[W32];
    for (;;) {
        pthread_mutex_lock(&J->mu);
        const uint32_t q = J->next < J->n_packs ? J->next++ : J->n_packs;
        pthread_mutex_unlock(&J->mu);
        if (q >= J->n_packs) break;
        const pack *pk = &J->packs[q];
        for (int w = 0; w < W32; ++w) {
            pr[w].S = NAN;
            pr[w].E = 0;
            pr[w].flags = 0;
            pr[w].nomem = 0;
        }
        if (J->fp64) pack_forward64(J->b, pk, (const double *)J->coef, &s, pr);
        else pack_forward32(J->b, pk, (const float *)J->coef, &s, pr);
        for (int w = 0; w < pk->n; ++w) {
            J->res[pk->idx[w]] = pr[w];
            if (pr[w].nomem) {
                pthread_mutex_lock(&J->mu);
                J->nomem = 1;
                pthread_mutex_unlock(&J->mu);
            }
        }
    }
    free(s.buf);
    return NULL;
}

static int run_packs(job *J, int n_threads) {
    J->next = 0;
    pthread_mutex_init(&J->mu, NULL);
    pthread_t th[1024];
    int started = 0;
    for (int t = 1; t < n_threads && (uint32_t)t < J->n_packs; ++t) {
        if (pthread_create(&th[started], NULL, worker, J) != 0) break;
        ++started;
    }
    worker(J);
    for (int t = 0; t < started; ++t) pthread_join(th[t], NULL);
    pthread_mutex_destroy(&J->mu);
    return J->nomem ? PHMM_ENOMEM : PHMM_OK;
}

typedef struct {
    uint32_t p, l, k, cls;
} pair_key;

static int key_cmp(const void *a, const void *b) {
    const pair_key *x = (const pair_key *)a, *y = (const pair_key *)b;
    if (x->cls != y->cls) return x->cls > y->cls ? -1 : 1; /* longer reads first */
    if (x->k != y->k) return x->k > y->k ? -1 : 1;
    if (x->l != y->l) return x->l > y->l ? -1 : 1;
    return x->p < y->p ? -1 : x->p > y->p;
}

/* Packs of up to w pairs from the listed pairs: sorted by read-length class (ratio
 * 2^(1/4)), then haplotype length, so a pack's lanes have similar l and k. */
static pack *make_packs(const phmm_batch *b, const uint32_t *list, uint32_t n, int w, uint32_t *n_packs,
                        int fp64, const uint64_t *coff) {
    pair_key *key = (pair_key *)malloc(sizeof(pair_key) * (n ? n : 1));
    const uint32_t np = (n + (uint32_t)w - 1) / (uint32_t)w;
    pack *pk = (pack *)calloc(np ? np : 1, sizeof(pack));
    if (!key || !pk) {
        free(key);
        free(pk);
        return NULL;
    }
    for (uint32_t q = 0; q < n; ++q) {
        const uint32_t p = list[q], r = b->pair_read[p], h = b->pair_hap[p];
        key[q].p = p;
        key[q].l = (uint32_t)(b->read_off[r + 1] - b->read_off[r]);
        key[q].k = (uint32_t)(b->hap_off[h + 1] - b->hap_off[h]);
        key[q].cls = (uint32_t)floor(4.0 * log2((double)key[q].l));
    }
    qsort(key, n, sizeof(pair_key), key_cmp);
    for (uint32_t t = 0; t < np; ++t) {
        pack *P = &pk[t];
        P->n = 0;
        for (uint32_t q = t * (uint32_t)w; q < n && q < (t + 1) * (uint32_t)w; ++q) {
            const uint32_t p = key[q].p;
            const int x = P->n++;
            P->idx[x] = p;
            P->l[x] = key[q].l;
            P->k[x] = key[q].k;
            P->r0[x] = b->read_off[b->pair_read[p]];
            P->h0[x] = b->hap_off[b->pair_hap[p]];
            P->c0[x] = coff[b->pair_read[p]];
            if (key[q].l > P->lmax) P->lmax = key[q].l;
            if (key[q].k > P->kmax) P->kmax = key[q].k;
        }
        P->R = fp64 ? pack_interval(b, P, 300.0 + 950.0, 1023.0 - 900.0) : pack_interval(b, P, 40.0 + 100.0, 127.0 - 100.0);
    }
    free(key);
    *n_packs = np;
    return pk;
}

/* The coefficient table: reads used by the listed pairs get consecutive records
 * (coff[r] = first record of read r), filled by n_threads threads over the reads. */
typedef struct {
    const phmm_batch *b;
    const uint32_t *reads; /* used reads */
    uint32_t n_reads, next;
    const uint64_t *coff;
    void *tab;
    int fp64;
    pthread_mutex_t mu;
} coef_job;

static void coef_read(const phmm_batch *b, uint32_t r, uint64_t c0, void *tab, int fp64) {
    const uint64_t r0 = b->read_off[r], l = b->read_off[r + 1] - r0;
    for (uint64_t i = 0; i < l; ++i) {
        const uint64_t bi = r0 + i;
        const double e = q_tab[b->base_q[bi]], qi = q_tab[b->ins_q[bi]], qd = q_tab[b->del_q[bi]],
                     g = q_tab[b->gcp_q[bi]];
        const double qdp = i > 0 ? q_tab[b->del_q[bi - 1]] : 1.0;
        const double c[NC - 1] = {1.0 - e, e / 3.0, 1.0 - qi - qd, 1.0 - g, qi, g, (1.0 - g) * qdp};
        int32_t bits = base_bits(b->read_bases[bi]);
        if (fp64) {
            double *d = (double *)tab + (c0 + i) * NC;
            for (int q = 0; q < NC - 1; ++q) d[q] = c[q];
            const int64_t b64 = bits;
            memcpy(&d[NC - 1], &b64, 8);
        } else {
            /* two hashes of the read base give the eight 16-bit uniforms */
            const uint64_t h0 = mix64(0x5eed1234ull << 32 ^ (bi * 2u)), h1 = mix64(0x5eed1234ull << 32 ^ (bi * 2u + 1u));
            const double omg = 1.0 - g;
            double cf[NC - 1] = {c[0] * omg, c[1] * omg, c[2] / omg, 1.0, qi, g, qdp};
            if (!(omg >= 0x1p-20)) {
                bits |= DEGEN_BIT;
                cf[0] = cf[1] = cf[2] = 0.0;
            }
            float *f = (float *)tab + (c0 + i) * NC;
            for (int q = 0; q < NC - 1; ++q)
                f[q] = sr_round(cf[q], (uint32_t)(((q < 4 ? h0 : h1) >> (16 * (q & 3))) & 0xffffu));
            memcpy(&f[NC - 1], &bits, 4);
        }
    }
}

static void *coef_worker(void *arg) {
    coef_job *J = (coef_job *)arg;
    for (;;) {
        pthread_mutex_lock(&J->mu);
        const uint32_t q0 = J->next;
        J->next = q0 + 64 < J->n_reads ? q0 + 64 : J->n_reads;
        pthread_mutex_unlock(&J->mu);
        if (q0 >= J->n_reads) break;
        const uint32_t q1 = q0 + 64 < J->n_reads ? q0 + 64 : J->n_reads;
        for (uint32_t q = q0; q < q1; ++q) coef_read(J->b, J->reads[q], J->coff[J->reads[q]], J->tab, J->fp64);
    }
    return NULL;
}

/* Returns the table (caller frees) and fills coff (n_reads entries); NULL if out of memory. */
static void *build_coef(const phmm_batch *b, const uint32_t *list, uint32_t n, int fp64, uint64_t *coff,
                        int n_threads) {
    uint8_t *used = (uint8_t *)calloc(b->n_reads ? b->n_reads : 1, 1);
    uint32_t *reads = (uint32_t *)malloc(sizeof(uint32_t) * (b->n_reads ? b->n_reads : 1));
    if (!used || !reads) {
        free(used);
        free(reads);
        return NULL;
    }
    for (uint32_t q = 0; q < n; ++q) used[b->pair_read[list[q]]] = 1;
    uint64_t total = 0;
    uint32_t nr = 0;
    for (uint32_t r = 0; r < b->n_reads; ++r)
        if (used[r]) {
            coff[r] = total;
            total += b->read_off[r + 1] - b->read_off[r];
            reads[nr++] = r;
        }
    free(used);
    void *tab = malloc((size_t)(total ? total : 1) * NC * (fp64 ? sizeof(double) : sizeof(float)));
    if (!tab) {
        free(reads);
        return NULL;
    }
    coef_job J;
    J.b = b;
    J.reads = reads;
    J.n_reads = nr;
    J.next = 0;
    J.coff = coff;
    J.tab = tab;
    J.fp64 = fp64;
    pthread_mutex_init(&J.mu, NULL);
    pthread_t th[1024];
    int started = 0;
    for (int t = 1; t < n_threads && (uint32_t)t * 64 < nr; ++t) {
        if (pthread_create(&th[started], NULL, coef_worker, &J) != 0) break;
        ++started;
    }
    coef_worker(&J);
    for (int t = 0; t < started; ++t) pthread_join(th[t], NULL);
    pthread_mutex_destroy(&J.mu);
    free(reads);
    return tab;
}

/* Per-pair validity: lengths >= 1, bases ACGTN, qualities <= 93. */
static int pair_valid(const phmm_batch *b, uint32_t p) {
    const uint32_t r = b->pair_read[p], h = b->pair_hap[p];
    const uint64_t r0 = b->read_off[r], r1 = b->read_off[r + 1], h0 = b->hap_off[h], h1 = b->hap_off[h + 1];
    if (r1 <= r0 || h1 <= h0) return 0;
    for (uint64_t x = r0; x < r1; ++x)
        if (!base_bits(b->read_bases[x]) || b->base_q[x] > 93 || b->ins_q[x] > 93 || b->del_q[x] > 93 ||
            b->gcp_q[x] > 93)
            return 0;
    for (uint64_t x = h0; x < h1; ++x)
        if (!base_bits(b->hap_bases[x])) return 0;
    return 1;
}

int phmm_cpu_forward(const phmm_batch *b, int n_threads, int precision, double fp32_tolerance) {
    if (!b || !b->out_log10 || !b->read_bases || !b->read_off || !b->base_q || !b->ins_q || !b->del_q ||
        !b->gcp_q || !b->hap_bases || !b->hap_off || (b->n_pairs && (!b->pair_read || !b->pair_hap)))
        return PHMM_EINVAL;
    if (b->inputs_on_device || b->outputs_on_device) return PHMM_EINVAL;
    if (precision < PHMM_PREC_FP32_RESCUE || precision > PHMM_PREC_FP32_ONLY) return PHMM_EINVAL;
    if (!(fp32_tolerance >= 0.0)) return PHMM_EINVAL;
    if (fp32_tolerance == 0.0) fp32_tolerance = 1e-3;
    for (uint32_t r = 0; r < b->n_reads; ++r)
        if (b->read_off[r + 1] < b->read_off[r]) return PHMM_EINVAL;
    for (uint32_t h = 0; h < b->n_haps; ++h)
        if (b->hap_off[h + 1] < b->hap_off[h]) return PHMM_EINVAL;
    for (uint32_t p = 0; p < b->n_pairs; ++p)
        if (b->pair_read[p] >= b->n_reads || b->pair_hap[p] >= b->n_haps) return PHMM_EINVAL;
    pthread_once(&q_once, q_init);
    if (n_threads <= 0) {
        const long c = sysconf(_SC_NPROCESSORS_ONLN);
        n_threads = c > 0 ? (int)c : 1;
    }
    if (n_threads > 1024) n_threads = 1024;
    const uint32_t n = b->n_pairs;
    uint32_t *list = (uint32_t *)malloc(sizeof(uint32_t) * (n ? n : 1));
    pair_result *res = (pair_result *)calloc(n ? n : 1, sizeof(pair_result));
    uint64_t *coff = (uint64_t *)malloc(sizeof(uint64_t) * (b->n_reads ? b->n_reads : 1));
    if (!list || !res || !coff) {
        free(list);
        free(res);
        free(coff);
        return PHMM_ENOMEM;
    }
    uint32_t nv = 0;
    for (uint32_t p = 0; p < n; ++p) {
        if (pair_valid(b, p)) list[nv++] = p;
        else {
            b->out_log10[p] = NAN;
            if (b->out_flags) b->out_flags[p] = PHMM_PAIR_ERROR;
        }
    }
    int rc = PHMM_OK;
    const int fp64_all = precision == PHMM_PREC_FP64;
    for (int pass = 0; pass < 2 && rc == PHMM_OK && nv > 0; ++pass) {
        const int fp64 = fp64_all || pass == 1;
        uint32_t np = 0;
        void *coef = build_coef(b, list, nv, fp64, coff, n_threads);
        pack *pk = coef ? make_packs(b, list, nv, fp64 ? W64 : W32, &np, fp64, coff) : NULL;
        if (!pk) {
            free(coef);
            rc = PHMM_ENOMEM;
            break;
        }
        job J;
        memset(&J, 0, sizeof(J));
        J.b = b;
        J.packs = pk;
        J.n_packs = np;
        J.fp64 = fp64;
        J.res = res;
        J.coef = coef;
        rc = run_packs(&J, n_threads);
        free(pk);
        free(coef);
        if (rc != PHMM_OK) break;
        /* results; the FP32 pass collects the pairs its tests send to the FP64 pass */
        uint32_t nr = 0;
        for (uint32_t q = 0; q < nv; ++q) {
            const uint32_t p = list[q], r = b->pair_read[p], h = b->pair_hap[p];
            const double l = (double)(b->read_off[r + 1] - b->read_off[r]);
            const double k = (double)(b->hap_off[h + 1] - b->hap_off[h]);
            const pair_result *x = &res[p];
            const int log2c = fp64 ? 1020 : 120;
            const double v = x->S > 0.0 && isfinite(x->S)
                                 ? log10(x->S) + (double)(x->E - log2c) * 0.30102999566398119521
                                 : (x->S == 0.0 ? -INFINITY : NAN);
            uint32_t f = x->flags & (PHMM_PAIR_RESCALED | PHMM_PAIR_DANGER | PHMM_PAIR_NONFINITE | PHMM_PAIR_DEGENERATE);
            if (fp64) {
                f |= PHMM_PAIR_FP64;
                if (pass == 1) f |= PHMM_PAIR_RESCUED | (b->out_flags ? b->out_flags[p] & 0x78u : 0u);
            } else {
                /* underflow test: at most 3 l k cells lost to the flush (or to the format's
                 * own underflow), each below max(FLUSH32, FLT_MIN) and each reaching L with
                 * total weight <= 1; the relative loss must stay <= 1e-4 */
                const double lost = FLUSH32 > 1.1754943508222875e-38 ? (double)FLUSH32 : 1.1754943508222875e-38;
                if (!(x->S > 3.0e4 * l * k * lost)) f |= PHMM_PAIR_SMALL_SUM;
                if (fp32_bound_log10(l, k) > fp32_tolerance) f |= PHMM_PAIR_DANGER;
                if (precision == PHMM_PREC_FP32_RESCUE && ((f & 0x78u) || !isfinite(v))) list[nr++] = p;
            }
            b->out_log10[p] = v;
            if (b->out_flags) b->out_flags[p] = (uint8_t)f;
        }
        if (fp64) break;
        nv = nr;
    }
    free(list);
    free(res);
    free(coff);
    return rc;
}
