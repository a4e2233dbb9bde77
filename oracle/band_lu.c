/*
 * Oracle (test infrastructure only): plain FP64 complex band and dense LU.
 *
 * This is the CPU reference for the linear solves T(z_i)^{-1} U of Algorithm 2,
 * Step 2 (the paper leaves the solver to the host software; a partial-pivoting
 * LU of the banded T(z_i) is its direct-solver form).  It is written for
 * clarity, not speed: unblocked, column by column, no reordering of the work.
 *
 * Band storage (LAPACK general-band layout): column-major array ab with leading
 * dimension ldab >= 2*kl + ku + 1; A(i, j) lives at ab[(kv + i - j) + j*ldab]
 * with kv = kl + ku.  Rows 0..kl-1 of ab hold the fill that row interchanges
 * create and must be zero on entry.  Complex values are interleaved (re, im).
 *
 * Pivoting: partial pivoting by cabs1(x) = |re x| + |im x|; on ties the lowest
 * row wins.  A zero pivot records the first such column (1-based) in the return
 * value and leaves that column unscaled, as LAPACK does.
 */
#include <complex.h>
#include <math.h>
#include <stdint.h>

typedef double complex zc;

static double cabs1(zc x) { return fabs(creal(x)) + fabs(cimag(x)); }

#define AB(i, j) ab[(kv + (i) - (j)) + (int64_t)(j) * ldab]

static int64_t imin(int64_t a, int64_t b) { return a < b ? a : b; }
static int64_t imax(int64_t a, int64_t b) { return a > b ? a : b; }

int64_t orc_zgbtrf(int64_t n, int64_t kl, int64_t ku, zc* ab, int64_t ldab, int32_t* ipiv)
{
    const int64_t kv = kl + ku;
    int64_t info = 0;
    for (int64_t j = 0; j < n; ++j) {
        const int64_t last_row = imin(j + kl, n - 1);   /* column j's band ends here */
        const int64_t last_col = imin(j + kv, n - 1);   /* U row j may fill up to here */
        int64_t p = j;
        double best = cabs1(AB(j, j));
        for (int64_t i = j + 1; i <= last_row; ++i) {
            double v = cabs1(AB(i, j));
            if (v > best) { best = v; p = i; }
        }
        ipiv[j] = (int32_t)p;
        if (AB(p, j) == 0.0) {
            if (info == 0) info = j + 1;
            continue;
        }
        if (p != j) {
            for (int64_t c = j; c <= last_col; ++c) {
                zc t = AB(j, c); AB(j, c) = AB(p, c); AB(p, c) = t;
            }
        }
        const zc r = 1.0 / AB(j, j);
        for (int64_t i = j + 1; i <= last_row; ++i) AB(i, j) *= r;
        for (int64_t c = j + 1; c <= last_col; ++c) {
            const zc u = AB(j, c);
            if (u == 0.0) continue;
            for (int64_t i = j + 1; i <= last_row; ++i) AB(i, c) -= AB(i, j) * u;
        }
    }
    return info;
}

/* Solve A X = B with the factors of orc_zgbtrf; B is n x nrhs column-major (ldb). */
void orc_zgbtrs(int64_t n, int64_t kl, int64_t ku, int64_t nrhs, const zc* ab, int64_t ldab,
                const int32_t* ipiv, zc* b, int64_t ldb)
{
    const int64_t kv = kl + ku;
    for (int64_t r = 0; r < nrhs; ++r) {
        zc* x = b + r * ldb;
        for (int64_t j = 0; j < n; ++j) {           /* L y = P b */
            const int64_t p = ipiv[j];
            if (p != j) { zc t = x[j]; x[j] = x[p]; x[p] = t; }
            const int64_t last_row = imin(j + kl, n - 1);
            for (int64_t i = j + 1; i <= last_row; ++i) x[i] -= AB(i, j) * x[j];
        }
        for (int64_t j = n - 1; j >= 0; --j) {      /* U x = y */
            x[j] /= AB(j, j);
            const int64_t first_row = imax(0, j - kv);
            for (int64_t i = first_row; i < j; ++i) x[i] -= AB(i, j) * x[j];
        }
    }
}

#undef AB
#define A(i, j) a[(i) + (int64_t)(j) * lda]

/* Dense LU with the same pivot rule (for problems with no usable band). */
int64_t orc_zgetrf(int64_t n, zc* a, int64_t lda, int32_t* ipiv)
{
    int64_t info = 0;
    for (int64_t j = 0; j < n; ++j) {
        int64_t p = j;
        double best = cabs1(A(j, j));
        for (int64_t i = j + 1; i < n; ++i) {
            double v = cabs1(A(i, j));
            if (v > best) { best = v; p = i; }
        }
        ipiv[j] = (int32_t)p;
        if (A(p, j) == 0.0) { if (info == 0) info = j + 1; continue; }
        /* interchange only the active columns j..n-1 (the multipliers already stored in
           columns < j stay in place), so the solve applies each interchange just before
           the elimination step that follows it, as in the band solve */
        if (p != j)
            for (int64_t c = j; c < n; ++c) { zc t = A(j, c); A(j, c) = A(p, c); A(p, c) = t; }
        const zc r = 1.0 / A(j, j);
        for (int64_t i = j + 1; i < n; ++i) A(i, j) *= r;
        for (int64_t c = j + 1; c < n; ++c) {
            const zc u = A(j, c);
            if (u == 0.0) continue;
            for (int64_t i = j + 1; i < n; ++i) A(i, c) -= A(i, j) * u;
        }
    }
    return info;
}

void orc_zgetrs(int64_t n, int64_t nrhs, const zc* a, int64_t lda, const int32_t* ipiv,
                zc* b, int64_t ldb)
{
    for (int64_t r = 0; r < nrhs; ++r) {
        zc* x = b + r * ldb;
        for (int64_t j = 0; j < n; ++j) {
            const int64_t p = ipiv[j];
            if (p != j) { zc t = x[j]; x[j] = x[p]; x[p] = t; }
            for (int64_t i = j + 1; i < n; ++i) x[i] -= A(i, j) * x[j];
        }
        for (int64_t j = n - 1; j >= 0; --j) {
            x[j] /= A(j, j);
            for (int64_t i = 0; i < j; ++i) x[i] -= A(i, j) * x[j];
        }
    }
}
