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
 * Planted mistakes: compiling with -DORACLE_PLANT=k (k = 1..6) introduces one
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
