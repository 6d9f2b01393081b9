/*
 * FP64 CPU oracle for multichannel FIR / IIR filter chains.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may call, link or
 * execute this file; only the test suite, the smoke check and the CPU-baseline
 * leg of the benchmark use it.  It shares no code, header, table or constant
 * with the CUDA library.
 *
 * What it computes (TorchFX, arXiv 2504.08624):
 *   - Sec. 3: each filter applies a user-supplied (b, a) difference equation to
 *     every channel of a [channels x samples] signal ("lfilter" semantics), and
 *     filters compose left to right through the pipe operator / nn.Sequential.
 *   - Sec. 4 (Tables 2-4): the workloads are FIR filters, IIR filters, and a
 *     chain of IIR filters over multichannel white noise.
 * The IIR filters are given as cascades of second-order sections.  Each is the
 * literal direct-form-I difference equation with zero initial conditions:
 *     a0*y[n] = b0*x[n] + b1*x[n-1] + b2*x[n-2] - a1*y[n-1] - a2*y[n-2],
 * x[n<0] = y[n<0] = 0, applied section after section in array order.
 * The FIR filter is the causal direct convolution of length N:
 *     y[n] = sum_{k=0}^{min(n, L-1)} h[k] * x[n-k].
 * A chain applies its stages in list order.  All arithmetic is in double.
 *
 * Planted mistakes: compiling with -DORACLE_PLANT=k (k = 1..8) introduces one
 * deliberate error so that the test suite can show its pins catch it.  The
 * default build (ORACLE_PLANT undefined or 0) is the oracle.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#ifndef ORACLE_PLANT
#define ORACLE_PLANT 0
#endif

#define ORACLE_OK 0
#define ORACLE_ERR_INVALID (-1)
#define ORACLE_ERR_NOMEM (-2)

/* One second-order section on one channel, DF-I literal difference equation. */
static void sos_section(const double *x, double *y, int64_t N, const double *row)
{
    double b0 = row[0], b1 = row[1], b2 = row[2];
    double a0 = row[3], a1 = row[4], a2 = row[5];
#if ORACLE_PLANT == 2
    a1 = -a1; /* planted: wrong sign on the first feedback coefficient */
#endif
    double x1 = 0.0, x2 = 0.0, y1 = 0.0, y2 = 0.0;
    for (int64_t n = 0; n < N; ++n) {
        double xn = x[n];
#if ORACLE_PLANT == 1
        double acc = b0 * xn + b1 * x1 - a1 * y1 - a2 * y2; /* planted: b2 dropped */
#elif ORACLE_PLANT == 6
        double acc = b0 * xn + b1 * x1 + b2 * x2 - a2 * y1 - a1 * y2; /* planted: a1/a2 swapped */
#else
        double acc = b0 * xn + b1 * x1 + b2 * x2 - a1 * y1 - a2 * y2;
#endif
#if ORACLE_PLANT == 4
        double yn = acc; /* planted: no division by a0 */
        (void)a0;
#else
        double yn = acc / a0;
#endif
        x2 = x1;
        x1 = xn;
        y2 = y1;
        y1 = yn;
        y[n] = yn;
    }
}

/* Causal direct convolution of one channel, output length N. */
static void fir_channel(const double *x, double *y, int64_t N, const double *h, int32_t L)
{
    for (int64_t n = 0; n < N; ++n) {
        double acc = 0.0;
        int64_t kmax = n < (int64_t)(L - 1) ? n : (int64_t)(L - 1);
#if ORACLE_PLANT == 3
        /* planted: input index off by one */
        for (int64_t k = 0; k <= kmax; ++k)
            acc += h[k] * (n - k - 1 >= 0 ? x[n - k - 1] : 0.0);
#else
        for (int64_t k = 0; k <= kmax; ++k)
            acc += h[k] * x[n - k];
#endif
        y[n] = acc;
    }
}

/*
 * The causal direct convolution of one channel at chosen output positions
 * only: out[i] = sum_{k=0}^{min(n, L-1)} h[k] * x[n-k] with n = idx[i]
 * (0 <= n < N).  For long signals and long filters, where the whole output
 * would take too long, a sample of it can still be checked one by one.
 */
int oracle_fir_at(const double *x, int64_t N, const double *h, int32_t L,
                  const int64_t *idx, int64_t n_idx, double *out)
{
    if (N < 0 || L < 1 || !h || n_idx < 0 || (n_idx > 0 && (!idx || !out || !x)))
        return ORACLE_ERR_INVALID;
    for (int64_t i = 0; i < n_idx; ++i)
        if (idx[i] < 0 || idx[i] >= N)
            return ORACLE_ERR_INVALID;
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n_idx; ++i) {
        const int64_t n = idx[i];
#if ORACLE_PLANT == 8
        /* planted: the last tap dropped */
        const int64_t kmax = n < (int64_t)(L - 2) ? n : (int64_t)(L - 2);
#else
        const int64_t kmax = n < (int64_t)(L - 1) ? n : (int64_t)(L - 1);
#endif
        double acc = 0.0;
        for (int64_t k = 0; k <= kmax; ++k)
            acc += h[k] * x[n - k];
        out[i] = acc;
    }
    return ORACLE_OK;
}

static int check_sos(const double *sos, int32_t S)
{
    if (S < 0 || (S > 0 && !sos))
        return ORACLE_ERR_INVALID;
    for (int32_t s = 0; s < S; ++s)
        if (sos[6 * s + 3] == 0.0)
            return ORACLE_ERR_INVALID;
    return ORACLE_OK;
}

/* Cascade of S sections (rows b0 b1 b2 a0 a1 a2), channel-major [C x N]. */
int oracle_sos(const double *x, double *y, int64_t C, int64_t N,
               const double *sos, int32_t S)
{
    if (C < 0 || N < 0 || (C * N > 0 && (!x || !y)))
        return ORACLE_ERR_INVALID;
    if (check_sos(sos, S) != ORACLE_OK)
        return ORACLE_ERR_INVALID;
    if (C == 0 || N == 0)
        return ORACLE_OK;
    int err = ORACLE_OK;
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t c = 0; c < C; ++c) {
        double *tmp = (double *)malloc((size_t)N * sizeof(double));
        if (!tmp) {
#pragma omp atomic write
            err = ORACLE_ERR_NOMEM;
            continue;
        }
        memcpy(tmp, x + c * N, (size_t)N * sizeof(double));
        for (int32_t s = 0; s < S; ++s) {
            sos_section(tmp, y + c * N, N, sos + 6 * s);
            memcpy(tmp, y + c * N, (size_t)N * sizeof(double));
        }
        memcpy(y + c * N, tmp, (size_t)N * sizeof(double));
        free(tmp);
    }
    return err;
}

int oracle_fir(const double *x, double *y, int64_t C, int64_t N,
               const double *h, int32_t L)
{
    if (C < 0 || N < 0 || L < 1 || !h || (C * N > 0 && (!x || !y)))
        return ORACLE_ERR_INVALID;
    if (C == 0 || N == 0)
        return ORACLE_OK;
    int err = ORACLE_OK;
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t c = 0; c < C; ++c) {
        if (x == y) {
            /* in place: convolve from a copy of the channel */
            double *tmp = (double *)malloc((size_t)N * sizeof(double));
            if (!tmp) {
#pragma omp atomic write
                err = ORACLE_ERR_NOMEM;
                continue;
            }
            memcpy(tmp, x + c * N, (size_t)N * sizeof(double));
            fir_channel(tmp, y + c * N, N, h, L);
            free(tmp);
        } else {
            fir_channel(x + c * N, y + c * N, N, h, L);
        }
    }
    return err;
}

/*
 * Chain of stages in list order: kinds[i] is 0 for FIR (counts[i] taps) and 1
 * for an SOS cascade (counts[i] sections, 6 doubles per row); coefs[i] points
 * at the stage's coefficients.
 */
int oracle_chain(const double *x, double *y, int64_t C, int64_t N,
                 const int32_t *kinds, const int32_t *counts,
                 const double *const *coefs, int32_t nst)
{
    if (C < 0 || N < 0 || nst < 0 || (nst > 0 && (!kinds || !counts || !coefs)))
        return ORACLE_ERR_INVALID;
    if (C * N > 0 && (!x || !y))
        return ORACLE_ERR_INVALID;
    for (int32_t i = 0; i < nst; ++i) {
        if (kinds[i] == 0) {
            if (counts[i] < 1 || !coefs[i])
                return ORACLE_ERR_INVALID;
        } else if (kinds[i] == 1) {
            if (check_sos(coefs[i], counts[i]) != ORACLE_OK)
                return ORACLE_ERR_INVALID;
        } else {
            return ORACLE_ERR_INVALID;
        }
    }
    if (C == 0 || N == 0)
        return ORACLE_OK;
    size_t bytes = (size_t)C * (size_t)N * sizeof(double);
    double *cur = (double *)malloc(bytes);
    double *nxt = (double *)malloc(bytes);
    if (!cur || !nxt) {
        free(cur);
        free(nxt);
        return ORACLE_ERR_NOMEM;
    }
    memcpy(cur, x, bytes);
    int err = ORACLE_OK;
#if ORACLE_PLANT == 5
    for (int32_t i = 0; i + 1 < nst && err == ORACLE_OK; ++i) { /* planted: last stage dropped */
#else
    for (int32_t i = 0; i < nst && err == ORACLE_OK; ++i) {
#endif
        if (kinds[i] == 0)
            err = oracle_fir(cur, nxt, C, N, coefs[i], counts[i]);
        else
            err = oracle_sos(cur, nxt, C, N, coefs[i], counts[i]);
        double *t = cur;
        cur = nxt;
        nxt = t;
    }
    if (err == ORACLE_OK)
        memcpy(y, cur, bytes);
    free(cur);
    free(nxt);
    return err;
}

/* Number of host threads the oracle's parallel loops use. */
int oracle_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

void oracle_set_num_threads(int n)
{
#ifdef _OPENMP
    if (n > 0)
        omp_set_num_threads(n);
#else
    (void)n;
#endif
}

int oracle_plant(void) { return ORACLE_PLANT; }

/*
 * Vector-Jacobian product of a chain: for an upstream gradient g = dL/dy,
 * returns dL/dx and dL/d(coefficients).  Computed from definitions, not by
 * the adjoint method:
 *   - dL/dx[m] = sum_n g[n] dy[n]/dx[m] = sum_n g[n] h_chain[n-m], with the
 *     chain's impulse response h_chain obtained by running the chain on a
 *     unit impulse (the chain is linear and time invariant in x);
 *   - coefficient derivatives by forward-mode sensitivity: differentiating a
 *     section's difference equation a0 y[n] = sum b_k u[n-k] - a1 y[n-1] -
 *     a2 y[n-2] gives, for each coefficient p, the recursion
 *       a0 s[n] = d(rhs)/dp - a1 s[n-1] - a2 s[n-2]   (s = dy/dp, s[<0] = 0),
 *     with d(rhs)/db_k = u[n-k], d(rhs)/da_k = -y[n-k] (k = 1, 2) and
 *     d(rhs)/da0 = -y[n]; the sensitivity then passes through the remaining
 *     stages (linear in their input) and dL/dp = sum_n g[n] * (that signal);
 *     for an FIR tap dy[n]/dh_k = u[n-k].
 * coef_grads: one block per stage, FIR: L doubles; SOS: 6 doubles per row.
 * Gradients are summed over channels.  O(N^2) for dx: small inputs only.
 */
static void chain_tail(const double *in, double *out, int64_t N, const int32_t *kinds, const int32_t *counts,
                       const double *const *coefs, int32_t from, int32_t nst, double *tmp)
{
    memcpy(out, in, (size_t)N * sizeof(double));
    for (int32_t i = from; i < nst; ++i) {
        if (kinds[i] == 0) {
            fir_channel(out, tmp, N, coefs[i], counts[i]);
        } else {
            for (int32_t s = 0; s < counts[i]; ++s) {
                sos_section(out, tmp, N, coefs[i] + 6 * s);
                memcpy(out, tmp, (size_t)N * sizeof(double));
            }
            continue;
        }
        memcpy(out, tmp, (size_t)N * sizeof(double));
    }
}

int oracle_chain_vjp(const double *x, const double *g, double *dx, double *coef_grads, int64_t C, int64_t N,
                     const int32_t *kinds, const int32_t *counts, const double *const *coefs, int32_t nst)
{
    if (C < 0 || N < 0 || nst < 0 || (C * N > 0 && (!x || !g)))
        return ORACLE_ERR_INVALID;
    int64_t ncoef = 0;
    for (int32_t i = 0; i < nst; ++i)
        ncoef += kinds[i] == 0 ? counts[i] : 6 * counts[i];
    if (ncoef > 0 && !coef_grads)
        return ORACLE_ERR_INVALID;
    for (int64_t k = 0; k < ncoef; ++k)
        coef_grads[k] = 0.0;
    if (C == 0 || N == 0)
        return ORACLE_OK;
    double *hc = NULL;
    if (dx) { /* the chain's impulse response, for dx */
        double *imp = (double *)calloc((size_t)N, sizeof(double));
        double *tmp = (double *)malloc((size_t)N * sizeof(double));
        hc = (double *)malloc((size_t)N * sizeof(double));
        if (!imp || !tmp || !hc) {
            free(imp); free(tmp); free(hc);
            return ORACLE_ERR_NOMEM;
        }
        imp[0] = 1.0;
        chain_tail(imp, hc, N, kinds, counts, coefs, 0, nst, tmp);
        free(imp); free(tmp);
    }
    /* per-channel gradient rows, summed in channel order afterwards */
    double *rows = (double *)calloc((size_t)(C * (ncoef > 0 ? ncoef : 1)), sizeof(double));
    if (!rows) {
        free(hc);
        return ORACLE_ERR_NOMEM;
    }
    int err = 0;
#pragma omp parallel
    {
        double *a = (double *)malloc((size_t)N * sizeof(double));
        double *b = (double *)malloc((size_t)N * sizeof(double));
        double *s = (double *)malloc((size_t)N * sizeof(double));
        double *t = (double *)malloc((size_t)N * sizeof(double));
        double *tmp = (double *)malloc((size_t)N * sizeof(double));
        const int ok = a && b && s && t && tmp;
        if (!ok) {
#pragma omp atomic write
            err = 1;
        }
#pragma omp for schedule(dynamic, 1)
        for (int64_t c = 0; c < C; ++c) {
            if (!ok)
                continue;
            const double *xc = x + c * N, *gc = g + c * N;
            double *gr = rows + c * ncoef;
            if (dx) {
                double *dxc = dx + c * N;
                for (int64_t m = 0; m < N; ++m) {
                    double acc = 0.0;
                    for (int64_t n = m; n < N; ++n)
                        acc += gc[n] * hc[n - m];
                    dxc[m] = acc;
                }
            }
            /* walk the stages, keeping the current stage input in a */
            memcpy(a, xc, (size_t)N * sizeof(double));
            int64_t off = 0;
            for (int32_t i = 0; i < nst; ++i) {
                if (kinds[i] == 0) {
                    const int32_t L = counts[i];
                    for (int32_t k = 0; k < L; ++k) {
                        /* sensitivity dy/dh_k = a[n-k], then the remaining stages */
                        for (int64_t n = 0; n < N; ++n)
                            s[n] = n - k >= 0 ? a[n - k] : 0.0;
                        chain_tail(s, t, N, kinds, counts, coefs, i + 1, nst, tmp);
                        double acc = 0.0;
                        for (int64_t n = 0; n < N; ++n)
                            acc += gc[n] * t[n];
                        gr[off + k] += acc;
                    }
                    fir_channel(a, b, N, coefs[i], L);
                    memcpy(a, b, (size_t)N * sizeof(double));
                    off += L;
                } else {
                    for (int32_t r = 0; r < counts[i]; ++r) {
                        const double *row = coefs[i] + 6 * r;
                        sos_section(a, b, N, row); /* b = section output y */
                        const double a0 = row[3], a1 = row[4], a2 = row[5];
                        for (int p = 0; p < 6; ++p) {
                            for (int64_t n = 0; n < N; ++n) {
                                double d;
                                if (p < 3)
                                    d = n - p >= 0 ? a[n - p] : 0.0;
                                else if (p == 3)
                                    d = -b[n];
                                else
                                    d = n - (p - 3) >= 0 ? -b[n - (p - 3)] : 0.0;
#if ORACLE_PLANT == 7
                                if (p == 4) d = -d; /* planted: wrong sign of the a1 sensitivity source */
#endif
                                const double s1 = n >= 1 ? s[n - 1] : 0.0, s2 = n >= 2 ? s[n - 2] : 0.0;
                                s[n] = (d - a1 * s1 - a2 * s2) / a0;
                            }
                            /* through the remaining sections of this stage, then later stages */
                            for (int32_t q = r + 1; q < counts[i]; ++q) {
                                sos_section(s, tmp, N, coefs[i] + 6 * q);
                                memcpy(s, tmp, (size_t)N * sizeof(double));
                            }
                            chain_tail(s, t, N, kinds, counts, coefs, i + 1, nst, tmp);
                            double acc = 0.0;
                            for (int64_t n = 0; n < N; ++n)
                                acc += gc[n] * t[n];
                            gr[off + 6 * r + p] += acc;
                        }
                        memcpy(a, b, (size_t)N * sizeof(double));
                    }
                    off += 6 * counts[i];
                }
            }
        }
        free(a); free(b); free(s); free(t); free(tmp);
    }
    if (!err)
        for (int64_t c = 0; c < C; ++c)
            for (int64_t k = 0; k < ncoef; ++k)
                coef_grads[k] += rows[c * ncoef + k];
    free(rows);
    free(hc);
    return err ? ORACLE_ERR_NOMEM : ORACLE_OK;
}
