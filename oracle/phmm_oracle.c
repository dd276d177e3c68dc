/*
 * phmm_oracle.c -- plain, slow, obviously-correct CPU PairHMM forward algorithm.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the parity oracle for the GPU library.
 * Only tests/, __graft_entry__.smoke() and bench.py's cpu_baseline / reference legs
 * may load it.  The product (the CUDA library and its Python binding) never links,
 * imports or calls it, and it shares no code, header, table or constant with the
 * CUDA path.
 *
 * What it computes (paper: Endeavor, "Efficient PairHMM for Detection of DNA
 * Variants in Genome-Scale Datasets", Section 2):
 *
 *   Eq. 1 (initialisation):  M[i][0] = I[i][0] = D[i][0] = 0 for i >= 1,
 *                            M[0][j] = I[0][j] = 0, D[0][j] = C / k for j = 0..k
 *                            (D[0][0] = C/k: the first row is P*T_DM*C/k in every
 *                            column, Section 3.4).
 *   Eq. 2 (recurrences), cell by cell, row i = 1..l, column j = 1..k:
 *       M[i][j] = P(r_i|h_j) * (T_MM_i M[i-1][j-1] + T_IM_i I[i-1][j-1] + T_DM_i D[i-1][j-1])
 *       I[i][j] = T_MI_i M[i-1][j] + T_II_i I[i-1][j]
 *       D[i][j] = T_MD_i M[i][j-1] + T_DD_i D[i][j-1]
 *   Eq. 3 (emission):  P = 1 - e_i on a match, e_i / 3 on a mismatch, e_i = 10^(-Q_i/10)
 *   Eq. 4 (likelihood): L = sum_j M[l][j] + I[l][j], reported as log10(L) with the
 *                       initial scale C divided back out.
 *
 * Transition probabilities per read row i (Section 2; the per-row forms of T_MM,
 * T_MI, T_MD follow the CPU listing of Section 3.3):
 *   T_MI_i = q(ins_i), T_MD_i = q(del_i), T_MM_i = 1 - q(ins_i) - q(del_i),
 *   T_II_i = T_DD_i = q(gcp_i), T_IM_i = T_DM_i = 1 - q(gcp_i)   (0.1 / 0.9 at gcp = 10),
 *   with q(x) = 10^(-x/10) for numeric Phred x in 0..93.
 *
 * Readings where the paper is silent or ambiguous (each one is listed in the
 * design notes of the repository):
 *   - qualities are numeric Phred (the paper's "Q - 33" is the ASCII offset);
 *   - mismatch emission is exactly e/3 (not 0.33);
 *   - the initial divisor is k = |haplotype| (Eq. 1), not a kernel constant;
 *   - every coefficient producing row i uses row i's qualities;
 *   - an 'N' in the read or in the haplotype counts as a match;
 *   - L keeps the 1/k start prior.
 *
 * Rescaling (the paper is silent; needed for long reads): after a row is complete,
 * if its largest value leaves [2^-500, 2^500], the whole row (M, I, D) is multiplied
 * by an exact power of two and the exponent is accumulated.  Power-of-two scaling is
 * exact, so the result equals unbounded-exponent evaluation except where subnormal
 * values would have occurred.
 *
 * The same source is compiled twice: REAL = double (prefix orc_) and
 * REAL = long double (prefix orcl_), the latter to bound the oracle's own rounding.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <pthread.h>

#ifndef ORC_LONG
typedef double real;
#define FN(name) orc_##name
#define R_POW pow
#define R_FREXP frexp
#define R_LDEXP ldexp
#define R_LOG10 log10
#else
typedef long double real;
#define FN(name) orcl_##name
#define R_POW powl
#define R_FREXP frexpl
#define R_LDEXP ldexpl
#define R_LOG10 log10l
#endif

/* Base code: A=0 C=1 G=2 T=3 N=4, anything else -1 (case-insensitive). */
static int base_code(uint8_t b)
{
    switch (b) {
    case 'A': case 'a': return 0;
    case 'C': case 'c': return 1;
    case 'G': case 'g': return 2;
    case 'T': case 't': return 3;
    case 'N': case 'n': return 4;
    default: return -1;
    }
}

/* Eq. 3 match rule with the 'N' reading: N on either side is a match. */
static int is_match(int rc, int hc)
{
    return rc == 4 || hc == 4 || rc == hc;
}

/* q(x) = 10^(-x/10): Phred to probability (Eq. 3 without the ASCII offset). */
real FN(q_phred)(int x)
{
    return R_POW((real)10, -(real)x / (real)10);
}

/*
 * Cell-by-cell Eq. 1-4 on per-row probabilities.
 *   l, read[l]            read bases (ASCII)
 *   eps[l]                base-error probability e_i (Eq. 3)
 *   tmi[l], tmd[l]        T_MI_i and T_MD_i
 *   gcp[l]                T_II_i = T_DD_i; T_IM_i = T_DM_i = 1 - gcp_i
 *   tmm[l]                T_MM_i (callers pass 1 - tmi - tmd, or anything else)
 *   k, hap[k]             haplotype bases (ASCII)
 *   log2C                 log2 of the initial scale C (Eq. 1 uses C = 2^1020)
 *   rescale               0: never, 1: when a row max leaves [2^-500, 2^500],
 *                         2: after every row (exactness test)
 * Returns log10 L; sets *status to 0, or -1 on invalid input (bad base, l or k < 1).
 */
static double forward_core(int l, const uint8_t *read, const real *eps, const real *tmi,
                           const real *tmd, const real *gcp, const real *tmm, int k,
                           const uint8_t *hap, double log2C, int rescale, int *status,
                           double *raw_S, long *raw_E)
{
    *status = -1;
    if (l < 1 || k < 1)
        return NAN;
    real *Mp = calloc((size_t)k + 1, sizeof(real)), *Ip = calloc((size_t)k + 1, sizeof(real));
    real *Dp = calloc((size_t)k + 1, sizeof(real)), *Mc = calloc((size_t)k + 1, sizeof(real));
    real *Ic = calloc((size_t)k + 1, sizeof(real)), *Dc = calloc((size_t)k + 1, sizeof(real));
    int *hc = malloc(sizeof(int) * (size_t)k);
    if (!Mp || !Ip || !Dp || !Mc || !Ic || !Dc || !hc) {
        free(Mp); free(Ip); free(Dp); free(Mc); free(Ic); free(Dc); free(hc);
        return NAN;
    }
    double result = NAN;
    for (int j = 0; j < k; j++) {
        hc[j] = base_code(hap[j]);
        if (hc[j] < 0)
            goto done;
    }
    /* Row 0 (Eq. 1): M = I = 0, D = C/k in every column j = 0..k. */
    real C = R_LDEXP((real)1, (int)log2C);
    for (int j = 0; j <= k; j++) {
        Mp[j] = 0;
        Ip[j] = 0;
        Dp[j] = C / (real)k;
    }
    long E = 0; /* true value = stored value * 2^E */
    for (int i = 1; i <= l; i++) {
        int rc = base_code(read[i - 1]);
        if (rc < 0)
            goto done;
        real e = eps[i - 1];
        real pm = (real)1 - e, px = e / (real)3;
        real t_mm = tmm[i - 1], t_mi = tmi[i - 1], t_md = tmd[i - 1];
        real g = gcp[i - 1], t_gm = (real)1 - g;
        /* Column 0 (Eq. 1): zero for every row i >= 1. */
        Mc[0] = 0;
        Ic[0] = 0;
        Dc[0] = 0;
        real rowmax = 0;
        for (int j = 1; j <= k; j++) {
            real p = is_match(rc, hc[j - 1]) ? pm : px;
            Mc[j] = p * (t_mm * Mp[j - 1] + t_gm * Ip[j - 1] + t_gm * Dp[j - 1]);
            Ic[j] = t_mi * Mp[j] + g * Ip[j];
            Dc[j] = t_md * Mc[j - 1] + g * Dc[j - 1];
            real a = Mc[j] > Ic[j] ? Mc[j] : Ic[j];
            a = a > Dc[j] ? a : Dc[j];
            rowmax = a > rowmax ? a : rowmax;
        }
        int do_scale = 0, s = 0;
        if (rescale == 2 && rowmax > 0) {
            int ex;
            R_FREXP(rowmax, &ex);
            s = -ex;
            do_scale = 1;
        } else if (rescale == 1 && rowmax > 0 &&
                   (rowmax < R_LDEXP((real)1, -500) || rowmax > R_LDEXP((real)1, 500))) {
            int ex;
            R_FREXP(rowmax, &ex);
            s = -ex; /* brings the row max into [0.5, 1) */
            do_scale = 1;
        }
        if (do_scale) {
            for (int j = 0; j <= k; j++) {
                Mc[j] = R_LDEXP(Mc[j], s);
                Ic[j] = R_LDEXP(Ic[j], s);
                Dc[j] = R_LDEXP(Dc[j], s);
            }
            E -= s;
        }
        real *t;
        t = Mp; Mp = Mc; Mc = t;
        t = Ip; Ip = Ic; Ic = t;
        t = Dp; Dp = Dc; Dc = t;
    }
    /* Eq. 4 on the last row (now in Mp/Ip). */
    {
        real S = 0;
        for (int j = 1; j <= k; j++)
            S += Mp[j] + Ip[j];
        if (S > 0)
            result = (double)(R_LOG10(S) + ((real)E - (real)log2C) * R_LOG10((real)2));
        else
            result = -INFINITY;
        if (raw_S)
            *raw_S = (double)S;
        if (raw_E)
            *raw_E = E;
        *status = 0;
    }
done:
    free(Mp); free(Ip); free(Dp); free(Mc); free(Ic); free(Dc); free(hc);
    return result;
}

/*
 * The paper's row-wise reformulation (Section 3.1, Eq. 7), evaluated literally:
 * D is never stored; every M[i][j] recomputes
 *     D[i-1][j-1] = T_MD_{i-1} * sum_{b=1}^{j-2} M[i-1][b] * T_DD_{i-1}^{j-2-b}
 * as an explicit sum over the previous row (row 1 uses D[0][j-1] = C/k from Eq. 1).
 * O(l k^2): small cases only.  No rescaling.  Same argument meaning as loglik_probs.
 */
double FN(rowwise_eq7)(int l, const uint8_t *read, const double *eps, const double *tmi,
                       const double *tmd, const double *gcp, const double *tmm, int k,
                       const uint8_t *hap, double log2C, int *status)
{
    *status = -1;
    if (l < 1 || k < 1)
        return NAN;
    real *Mp = calloc((size_t)k + 1, sizeof(real)), *Ip = calloc((size_t)k + 1, sizeof(real));
    real *Mc = calloc((size_t)k + 1, sizeof(real)), *Ic = calloc((size_t)k + 1, sizeof(real));
    double result = NAN;
    if (!Mp || !Ip || !Mc || !Ic)
        goto done;
    for (int j = 0; j < k; j++)
        if (base_code(hap[j]) < 0)
            goto done;
    real C = R_LDEXP((real)1, (int)log2C);
    for (int i = 1; i <= l; i++) {
        int rc = base_code(read[i - 1]);
        if (rc < 0)
            goto done;
        real e = eps[i - 1], pm = (real)1 - e, px = e / (real)3;
        real t_gm = (real)1 - gcp[i - 1];
        for (int j = 1; j <= k; j++) {
            real p = is_match(rc, base_code(hap[j - 1])) ? pm : px;
            real dprev;
            if (i == 1) {
                dprev = C / (real)k;
            } else {
                real sum = 0, gprev = gcp[i - 2];
                for (int b = 1; b <= j - 2; b++)
                    sum += Mp[b] * R_POW(gprev, (real)(j - 2 - b));
                dprev = tmd[i - 2] * sum;
            }
            Mc[j] = p * (tmm[i - 1] * Mp[j - 1] + t_gm * Ip[j - 1] + t_gm * dprev);
            Ic[j] = tmi[i - 1] * Mp[j] + gcp[i - 1] * Ip[j];
        }
        Mc[0] = Ic[0] = 0;
        real *t;
        t = Mp; Mp = Mc; Mc = t;
        t = Ip; Ip = Ic; Ic = t;
    }
    {
        real S = 0;
        for (int j = 1; j <= k; j++)
            S += Mp[j] + Ip[j];
        result = S > 0 ? (double)(R_LOG10(S) - (real)log2C * R_LOG10((real)2)) : -INFINITY;
        *status = 0;
    }
done:
    free(Mp); free(Ip); free(Mc); free(Ic);
    return result;
}

/* Widen double per-row probabilities to REAL; NULL on allocation failure. */
static real *widen(int l, const double *a, const double *b, const double *c, const double *d,
                   const double *e)
{
    real *buf = malloc(sizeof(real) * 5 * (size_t)l);
    if (!buf)
        return NULL;
    for (int i = 0; i < l; i++) {
        buf[i] = a[i];
        buf[l + i] = b[i];
        buf[2 * l + i] = c[i];
        buf[3 * l + i] = d[i];
        buf[4 * l + i] = e[i];
    }
    return buf;
}

/* Exported form of forward_core on double per-row probabilities (see forward_core). */
double FN(loglik_probs)(int l, const uint8_t *read, const double *eps, const double *tmi,
                        const double *tmd, const double *gcp, const double *tmm, int k,
                        const uint8_t *hap, double log2C, int rescale, int *status)
{
    *status = -1;
    if (l < 1 || k < 1)
        return NAN;
    real *w = widen(l, eps, tmi, tmd, gcp, tmm);
    if (!w)
        return NAN;
    double r = forward_core(l, read, w, w + l, w + 2 * l, w + 3 * l, w + 4 * l, k, hap, log2C,
                            rescale, status, NULL, NULL);
    free(w);
    return r;
}

/* As loglik_probs, also returning the final stored sum S (Eq. 4, before log10) and the
 * accumulated rescaling exponent E, so that L * C = S * 2^E. */
double FN(forward_raw)(int l, const uint8_t *read, const double *eps, const double *tmi,
                       const double *tmd, const double *gcp, const double *tmm, int k,
                       const uint8_t *hap, double log2C, int rescale, int *status, double *S,
                       long *E)
{
    *status = -1;
    if (l < 1 || k < 1)
        return NAN;
    real *w = widen(l, eps, tmi, tmd, gcp, tmm);
    if (!w)
        return NAN;
    double r = forward_core(l, read, w, w + l, w + 2 * l, w + 3 * l, w + 4 * l, k, hap, log2C,
                            rescale, status, S, E);
    free(w);
    return r;
}

/* Phred qualities -> per-row probabilities in REAL precision, then forward_core.
 * Any quality above 93 -> status -1. */
double FN(loglik_phred)(int l, const uint8_t *read, const uint8_t *bq, const uint8_t *iq,
                        const uint8_t *dq, const uint8_t *gq, int k, const uint8_t *hap,
                        double log2C, int rescale, int *status)
{
    *status = -1;
    if (l < 1 || k < 1)
        return NAN;
    real *buf = malloc(sizeof(real) * 5 * (size_t)l);
    if (!buf)
        return NAN;
    real *eps = buf, *tmi = buf + l, *tmd = buf + 2 * l, *g = buf + 3 * l, *tmm = buf + 4 * l;
    double r = NAN;
    for (int i = 0; i < l; i++) {
        if (bq[i] > 93 || iq[i] > 93 || dq[i] > 93 || gq[i] > 93)
            goto done;
        eps[i] = FN(q_phred)(bq[i]);
        tmi[i] = FN(q_phred)(iq[i]);
        tmd[i] = FN(q_phred)(dq[i]);
        g[i] = FN(q_phred)(gq[i]);
        tmm[i] = (real)1 - tmi[i] - tmd[i];
    }
    r = forward_core(l, read, eps, tmi, tmd, g, tmm, k, hap, log2C, rescale, status, NULL, NULL);
done:
    free(buf);
    return r;
}

/*
 * Batch over pairs in the library's input layout (reads and haplotypes concatenated,
 * offsets of n+1 entries, one (read, haplotype) index per pair), on n_threads POSIX
 * threads taking pairs from a shared counter.  out[p] = log10 L of pair p, or NaN on
 * invalid input.  Returns the number of invalid pairs.
 */
typedef struct {
    const uint8_t *rb, *bq, *iq, *dq, *gq, *hb;
    const uint64_t *roff, *hoff;
    const uint32_t *pr, *ph;
    uint32_t n_pairs;
    double log2C;
    int rescale;
    double *out;
    long next;
    long bad;
    pthread_mutex_t mu;
} batch_job;

static void *batch_worker(void *arg)
{
    batch_job *J = arg;
    for (;;) {
        long p;
        pthread_mutex_lock(&J->mu);
        p = J->next++;
        pthread_mutex_unlock(&J->mu);
        if (p >= (long)J->n_pairs)
            break;
        uint32_t r = J->pr[p], h = J->ph[p];
        uint64_t r0 = J->roff[r], r1 = J->roff[r + 1], h0 = J->hoff[h], h1 = J->hoff[h + 1];
        int st;
        double v = FN(loglik_phred)((int)(r1 - r0), J->rb + r0, J->bq + r0, J->iq + r0,
                                    J->dq + r0, J->gq + r0, (int)(h1 - h0), J->hb + h0,
                                    J->log2C, J->rescale, &st);
        if (st != 0) {
            v = NAN;
            pthread_mutex_lock(&J->mu);
            J->bad++;
            pthread_mutex_unlock(&J->mu);
        }
        J->out[p] = v;
    }
    return NULL;
}

long FN(batch)(const uint8_t *read_bases, const uint64_t *read_off, const uint8_t *base_q,
               const uint8_t *ins_q, const uint8_t *del_q, const uint8_t *gcp_q,
               const uint8_t *hap_bases, const uint64_t *hap_off, uint32_t n_pairs,
               const uint32_t *pair_read, const uint32_t *pair_hap, double log2C, int rescale,
               int n_threads, double *out)
{
    batch_job J = {read_bases, base_q, ins_q, del_q, gcp_q, hap_bases, read_off, hap_off,
                   pair_read, pair_hap, n_pairs, log2C, rescale, out, 0, 0,
                   PTHREAD_MUTEX_INITIALIZER};
    if (n_threads < 1)
        n_threads = 1;
    pthread_t *t = malloc(sizeof(pthread_t) * (size_t)n_threads);
    if (!t)
        return -1;
    int started = 0;
    for (int i = 0; i < n_threads; i++)
        if (pthread_create(&t[i], NULL, batch_worker, &J) == 0)
            started++;
        else
            break;
    if (started == 0)
        batch_worker(&J);
    for (int i = 0; i < started; i++)
        pthread_join(t[i], NULL);
    free(t);
    return J.bad;
}
