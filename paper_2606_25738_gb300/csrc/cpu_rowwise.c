/*
 * Row-wise PairHMM forward pass on the host CPU (include/phmm_cpu.h).
 *
 * Per pair, rows i = 1..l over columns j = 1..k (Section 2, Eq. 1-4; row-wise form of
 * Section 3.1, Eq. 5-7):
 *   M_ij = P_ij (T_MM_i M_i-1,j-1 + T_IM_i I_i-1,j-1 + T_DM_i D_i-1,j-1)
 *   I_ij = T_MI_i M_i-1,j + g_i I_i-1,j
 *   D_ij = T_MD_i M_i,j-1 + g_i D_i,j-1
 * with D_0j = C/k for every j (row 0), column 0 zero for i >= 1, and L = sum_j M_lj + I_lj
 * over C.  T_MI = q(ins), T_MD = q(del), T_MM = 1 - T_MI - T_MD, g = q(gcp),
 * T_IM = T_DM = 1 - g; P = 1 - q(base) on a match (an N on either side matches), else
 * q(base) / 3; q(x) = 10^(-x / 10).
 *
 * The M and I loops of a row read only the previous row: they vectorise.  The deletion
 * chain is the first-order recurrence d_j = a_j + g d_j-1 (a_j = T_MD M_i,j-1); it is
 * evaluated in NB blocks of the row at once (NB independent dependency chains, each from
 * a zero carry), then each block's true carry enters as carry * g^(m + 1) at its m-th
 * column (a vectorisable fix-up).  FP64 throughout; every 16 rows the row is multiplied by
 * a power of two that brings its maximum to 2^500 (exact), and the exponents are summed.
 *
 * Portable C: no intrinsics, no target flags; the compiler vectorises the loops for the
 * host's SIMD unit (NEON / SVE on Arm, SSE on x86).
 */
#include "phmm_cpu.h"

#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <unistd.h>

#define NB 8             /* deletion-chain blocks per row */
#define RESCALE_ROWS 16  /* rows between power-of-two rescalings */

static double q_tab[94];
static pthread_once_t q_once = PTHREAD_ONCE_INIT;
static void q_init(void) {
    for (int x = 0; x < 94; ++x) q_tab[x] = pow(10.0, -(double)x / 10.0);
}

/* base code: A C G T = 0..3, N = 4, anything else -1 */
static int code_of(uint8_t c) {
    switch (c) {
    case 'A': case 'a': return 0;
    case 'C': case 'c': return 1;
    case 'G': case 'g': return 2;
    case 'T': case 't': return 3;
    case 'N': case 'n': return 4;
    default: return -1;
    }
}

typedef struct {
    double *M, *I, *D, *Mn, *In, *Dn;  /* previous and new row, k + 1 columns each */
    double *match;                     /* 5 x n match indicators (1.0 / 0.0) per read base A C G T N */
    double *gp;                        /* g^1 .. g^gp_n for g = gp_g */
    size_t cap_k, cap_n, gp_n;
    double gp_g;
} scratch;

static int scratch_fit(scratch *s, size_t k) {
    if (k <= s->cap_k) return 1;
    free(s->M);
    size_t n = ((k + NB - 1) / NB) * NB + 1; /* whole deletion-chain blocks */
    /* one block: 6 rows of n, 5 x n match indicators, the powers (<= n) */
    double *p = (double *)malloc(sizeof(double) * (6 * n + 5 * n + n));
    if (!p) {
        s->M = NULL;
        s->cap_k = 0;
        return 0;
    }
    s->M = p;
    s->I = p + n;
    s->D = p + 2 * n;
    s->Mn = p + 3 * n;
    s->In = p + 4 * n;
    s->Dn = p + 5 * n;
    s->match = p + 6 * n;
    s->gp = s->match + 5 * n;
    s->cap_k = k;
    s->cap_n = n;
    s->gp_g = -1.0;
    s->gp_n = 0;
    return 1;
}

/* d[1..k] from d_j = a_j + g d_j-1 with d_0 = 0, where a_j = tmd * m[j - 1]. */
static void deletion_row(const double *m, double *d, size_t k, double tmd, double g, scratch *s) {
    d[0] = 0.0;
    if (k < 4 * NB) {  /* short rows: plain chain */
        double x = 0.0;
        for (size_t j = 1; j <= k; ++j) {
            x = tmd * m[j - 1] + g * x;
            d[j] = x;
        }
        return;
    }
    const size_t blk = (k + NB - 1) / NB;
    if (s->gp_g != g || s->gp_n < blk) {  /* g^1 .. g^blk (rows usually share one g) */
        double p = 1.0;
        for (size_t t = 0; t < blk; ++t) {
            p *= g;
            s->gp[t] = p;
        }
        s->gp_g = g;
        s->gp_n = blk;
    }
    /* NB independent chains, block b covering columns b*blk+1 .. (b+1)*blk (the rows are
     * padded to whole blocks; columns beyond k are computed and ignored) */
    double x[NB];
    for (int b = 0; b < NB; ++b) x[b] = 0.0;
    for (size_t t = 0; t < blk; ++t) {
        const double *mm = m + t;
        double *dd = d + t + 1;
        for (int b = 0; b < NB; ++b) {
            x[b] = tmd * mm[(size_t)b * blk] + g * x[b];
            dd[(size_t)b * blk] = x[b];
        }
    }
    /* carries: block b's chain starts from the true d at the end of block b - 1 */
    for (int b = 1; b < NB; ++b) {
        const size_t j0 = (size_t)b * blk; /* last column of block b - 1 */
        if (j0 >= k) break;
        const double carry = d[j0];
        const size_t n = (j0 + blk <= k) ? blk : k - j0;
        double *dd = d + j0 + 1;
        const double *gp = s->gp;
        for (size_t t = 0; t < n; ++t) dd[t] += carry * gp[t];
    }
}

/* M and I of a row i >= 2 from row i - 1 (columns 1..k; index 0 is column 0); the
 * emission of column j is px + (pm - px) mt[j - 1]. */
static void mi_row(double *restrict Mn, double *restrict In, const double *restrict M,
                   const double *restrict I, const double *restrict D, const double *restrict mt, size_t k,
                   double px, double dp, double tmm, double tgm, double tmi, double g) {
    for (size_t j = 1; j <= k; ++j) {
        Mn[j] = (px + dp * mt[j - 1]) * (tmm * M[j - 1] + tgm * I[j - 1] + tgm * D[j - 1]);
        In[j] = tmi * M[j] + g * I[j];
    }
}

/* One pair; NaN for an invalid one. */
static double pair_forward(const phmm_batch *b, uint32_t p, scratch *s, int *bad) {
    *bad = 0;
    const uint32_t r = b->pair_read[p], h = b->pair_hap[p];
    const uint64_t r0 = b->read_off[r], r1 = b->read_off[r + 1];
    const uint64_t h0 = b->hap_off[h], h1 = b->hap_off[h + 1];
    const size_t l = (size_t)(r1 - r0), k = (size_t)(h1 - h0);
    if (l == 0 || k == 0) {
        *bad = 1;
        return NAN;
    }
    if (!scratch_fit(s, k)) {
        *bad = 2;
        return NAN;
    }
    /* match indicators of the haplotype per read base A, C, G, T, N (an N matches all) */
    const size_t n = s->cap_n;
    const uint8_t *hb = b->hap_bases + h0;
    for (size_t j = 0; j < k; ++j) {
        const int c = code_of(hb[j]);
        if (c < 0) {
            *bad = 1;
            return NAN;
        }
        for (int x = 0; x < 4; ++x) s->match[(size_t)x * n + j] = (c == x || c == 4) ? 1.0 : 0.0;
        s->match[4 * n + j] = 1.0;
    }
    /* padding beyond column k (whole deletion-chain blocks) stays zero */
    for (size_t j = k + 1; j < n; ++j) s->M[j] = s->I[j] = s->D[j] = s->Mn[j] = s->In[j] = s->Dn[j] = 0.0;
    const uint8_t *rb = b->read_bases + r0, *bq = b->base_q + r0, *iq = b->ins_q + r0, *dq = b->del_q + r0,
                  *gq = b->gcp_q + r0;
    for (size_t i = 0; i < l; ++i)
        if (code_of(rb[i]) < 0 || bq[i] > 93 || iq[i] > 93 || dq[i] > 93 || gq[i] > 93) {
            *bad = 1;
            return NAN;
        }
    double *M = s->M, *I = s->I, *D = s->D, *Mn = s->Mn, *In = s->In, *Dn = s->Dn;
    /* Row 1 is formed from D_0j = 1/k instead of C/k, so the stored values are L's terms
     * (true values over C) times 2^lg2s, the sum of the rescaling shifts. */
    long lg2s = 0;
    for (size_t i = 0; i < l; ++i) {
        const double e = q_tab[bq[i]], pm = 1.0 - e, px = e / 3.0;
        const double tmi = q_tab[iq[i]], tmd = q_tab[dq[i]], g = q_tab[gq[i]];
        const double tmm = 1.0 - tmi - tmd, tgm = 1.0 - g;
        const double *mt = s->match + (size_t)code_of(rb[i]) * n, dp = pm - px;
        Mn[0] = 0.0;
        In[0] = 0.0;
        if (i == 0) {
            /* row 0: M = I = 0, D = C/k in every column (stored as 1/k) */
            const double d0 = 1.0 / (double)k;
            for (size_t j = 1; j <= k; ++j) {
                Mn[j] = (px + dp * mt[j - 1]) * (tgm * d0);
                In[j] = 0.0;
            }
        } else {
            mi_row(Mn, In, M, I, D, mt, k, px, dp, tmm, tgm, tmi, g);
        }
        deletion_row(Mn, Dn, k, tmd, g, s);
        /* the new row becomes the previous one */
        double *t;
        t = M; M = Mn; Mn = t;
        t = I; I = In; In = t;
        t = D; D = Dn; Dn = t;
        if ((i + 1) % RESCALE_ROWS == 0 && i + 1 < l) {
            double mx = 0.0;
            for (size_t j = 1; j <= k; ++j) {
                const double a = fabs(M[j]), b2 = fabs(I[j]), c2 = fabs(D[j]);
                const double m2 = a > b2 ? a : b2;
                mx = mx > m2 ? mx : m2;
                mx = mx > c2 ? mx : c2;
            }
            if (mx > 0.0 && isfinite(mx)) {
                int ex;
                frexp(mx, &ex);
                const int sh = 500 - ex; /* multiply by 2^sh: maximum near 2^500 */
                /* two exact power-of-two factors (2^sh alone may not be representable) */
                const double f1 = ldexp(1.0, sh / 2), f2 = ldexp(1.0, sh - sh / 2);
                for (size_t j = 1; j <= k; ++j) {
                    M[j] = (M[j] * f1) * f2;
                    I[j] = (I[j] * f1) * f2;
                    D[j] = (D[j] * f1) * f2;
                }
                lg2s += sh;
            }
        }
    }
    double S = 0.0;
    for (size_t j = 1; j <= k; ++j) S += M[j] + I[j];
    return log10(S) - (double)lg2s * log10(2.0); /* log10 L = log10(S 2^-lg2s) */
}

typedef struct {
    const phmm_batch *b;
    uint32_t next;
    pthread_mutex_t mu;
    int nomem;
} job;

static void *worker(void *arg) {
    job *J = (job *)arg;
    scratch s;
    memset(&s, 0, sizeof(s));
    for (;;) {
        uint32_t p0;
        pthread_mutex_lock(&J->mu);
        p0 = J->next;
        J->next = p0 + 64 < p0 ? J->b->n_pairs : p0 + 64;
        pthread_mutex_unlock(&J->mu);
        if (p0 >= J->b->n_pairs) break;
        uint32_t p1 = p0 + 64 < J->b->n_pairs ? p0 + 64 : J->b->n_pairs;
        for (uint32_t p = p0; p < p1; ++p) {
            int bad = 0;
            const double v = pair_forward(J->b, p, &s, &bad);
            J->b->out_log10[p] = v;
            if (J->b->out_flags) J->b->out_flags[p] = bad ? (uint8_t)PHMM_PAIR_ERROR : (uint8_t)PHMM_PAIR_FP64;
            if (bad == 2) {
                pthread_mutex_lock(&J->mu);
                J->nomem = 1;
                pthread_mutex_unlock(&J->mu);
            }
        }
    }
    free(s.M);
    return NULL;
}

int phmm_cpu_forward(const phmm_batch *b, int n_threads) {
    if (!b || !b->out_log10 || !b->read_bases || !b->read_off || !b->base_q || !b->ins_q || !b->del_q ||
        !b->gcp_q || !b->hap_bases || !b->hap_off || (b->n_pairs && (!b->pair_read || !b->pair_hap)))
        return PHMM_EINVAL;
    if (b->inputs_on_device || b->outputs_on_device) return PHMM_EINVAL;
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
    job J;
    J.b = b;
    J.next = 0;
    J.nomem = 0;
    pthread_mutex_init(&J.mu, NULL);
    pthread_t th[1024];
    int started = 0;
    for (int t = 1; t < n_threads; ++t) {
        if (pthread_create(&th[started], NULL, worker, &J) != 0) break;
        ++started;
    }
    worker(&J);
    for (int t = 0; t < started; ++t) pthread_join(th[t], NULL);
    pthread_mutex_destroy(&J.mu);
    return J.nomem ? PHMM_ENOMEM : PHMM_OK;
}
