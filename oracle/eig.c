/* Eigenvalues of a real general matrix (oracle, FP64, serial).
 *
 * TEST INFRASTRUCTURE ONLY: called from oracle/eig.py by the tests, the smoke
 * check and the CPU baseline of the benchmark; never by the product library.
 *
 * Section II-B-2 classifies a scenario as unstable when an eigenvalue of the
 * linearised state matrix has a non-negative real part.  The paper calls an
 * external tool; this file is the textbook route written out plainly:
 *   1. balancing by powers of two (Parlett and Reinsch), an exact similarity;
 *   2. Householder reduction to upper Hessenberg form;
 *   3. implicit Francis double-shift QR iteration on the unreduced trailing
 *      block, eigenvalues only (Golub and Van Loan, "Matrix Computations",
 *      Sections 7.4-7.5), with deflation when a subdiagonal entry is
 *      negligible (at most eps times the sum of its two diagonal neighbours,
 *      or eps times the largest entry of the Hessenberg matrix when both are
 *      zero) and ad hoc exceptional shifts after 10 and 20 iterations without
 *      deflation.  Householder vectors follow the textbook house(): the norm
 *      below the leading entry is summed directly.
 * No LAPACK.  Pinned in tests/test_oracle_eig.py against 2x2 swing-equation
 * closed forms, companion matrices with known roots, planted spectra
 * V diag V^-1, trace identities and (test-only) numpy.linalg.eigvals.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

#define A_(i, j) a[(size_t)(i) * n + (j)]

/* Balance rows/columns of the n x n row-major matrix in place. */
static void balance(int n, double* a)
{
    const double radix = 2.0, sqrdx = 4.0;
    int done = 0, sweeps = 0;
    while (!done && sweeps < 100) {            /* converges in a few sweeps; capped */
        done = 1;
        ++sweeps;
        for (int i = 0; i < n; ++i) {
            double c = 0.0, r = 0.0;
            for (int j = 0; j < n; ++j) {
                if (j == i) continue;
                c += fabs(A_(j, i));
                r += fabs(A_(i, j));
            }
            if (c == 0.0 || r == 0.0 || !isfinite(c) || !isfinite(r)) continue;
            double g = r / radix, f = 1.0, s = c + r;
            while (c < g) { f *= radix; c *= sqrdx; }
            g = r * radix;
            while (c > g) { f /= radix; c /= sqrdx; }
            if ((c + r) / f < 0.95 * s) {
                done = 0;
                double ginv = 1.0 / f;
                for (int j = 0; j < n; ++j) A_(i, j) *= ginv;
                for (int j = 0; j < n; ++j) A_(j, i) *= f;
            }
        }
    }
}

/* Householder reduction to upper Hessenberg form, in place. */
static void hessenberg(int n, double* a, double* v)
{
    for (int k = 0; k + 2 < n; ++k) {
        double tail = 0.0;                       /* squared norm below the subdiagonal */
        for (int i = k + 2; i < n; ++i) tail += A_(i, k) * A_(i, k);
        if (tail == 0.0) continue;               /* already zero below the subdiagonal */
        double x0 = A_(k + 1, k);
        double nrm2 = x0 * x0 + tail;
        double alpha = (x0 >= 0.0) ? -sqrt(nrm2) : sqrt(nrm2);
        int m = n - k - 1;
        v[0] = x0 - alpha;
        for (int i = 1; i < m; ++i) v[i] = A_(k + 1 + i, k);
        double vtv = v[0] * v[0] + tail;
        double beta = 2.0 / vtv;
        /* left: rows k+1.., columns k.. */
        for (int j = k; j < n; ++j) {
            double s = 0.0;
            for (int i = 0; i < m; ++i) s += v[i] * A_(k + 1 + i, j);
            s *= beta;
            for (int i = 0; i < m; ++i) A_(k + 1 + i, j) -= s * v[i];
        }
        /* right: all rows, columns k+1.. */
        for (int i = 0; i < n; ++i) {
            double s = 0.0;
            for (int j = 0; j < m; ++j) s += A_(i, k + 1 + j) * v[j];
            s *= beta;
            for (int j = 0; j < m; ++j) A_(i, k + 1 + j) -= s * v[j];
        }
        A_(k + 1, k) = alpha;
        for (int i = k + 2; i < n; ++i) A_(i, k) = 0.0;
    }
}

/* Eigenvalues of the 2x2 block [[p, q], [r, s]]. */
static void eig2(double p, double q, double r, double s, double* re, double* im)
{
    double hm = 0.5 * (p - s);
    double disc = hm * hm + q * r;
    double mean = 0.5 * (p + s);
    if (disc >= 0.0) {
        double root = sqrt(disc);
        double big = mean + (hm >= 0.0 ? root : -root);
        /* the other root from the determinant when the sum cancels */
        double det = p * s - q * r;
        double other = (big != 0.0) ? det / big : mean - (hm >= 0.0 ? root : -root);
        re[0] = big; im[0] = 0.0;
        re[1] = other; im[1] = 0.0;
    } else {
        double root = sqrt(-disc);
        re[0] = mean; im[0] = root;
        re[1] = mean; im[1] = -root;
    }
}

/* Reflector for a 2- or 3-vector: (I - beta u u^T) x = alpha e1, u[0] = x0 - alpha.
 * Returns 0 when x is already a multiple of e1 (no transformation). */
static int house3(int len, const double* x, double* u, double* beta)
{
    double t2 = 0.0;
    for (int i = 1; i < len; ++i) t2 += x[i] * x[i];
    if (t2 == 0.0) return 0;
    double nrm = sqrt(x[0] * x[0] + t2);
    double alpha = (x[0] >= 0.0) ? -nrm : nrm;
    u[0] = x[0] - alpha;
    for (int i = 1; i < len; ++i) u[i] = x[i];
    *beta = 2.0 / (u[0] * u[0] + t2);
    return 1;
}

/* Francis double-shift QR on the upper Hessenberg matrix, eigenvalues only.
 * Returns 0 on success, -1 if an eigenvalue needed more than 30*n sweeps. */
static int hqr(int n, double* a, double* wr, double* wi, int* sweeps_out)
{
    const double eps = 2.220446049250313e-16;
    /* scale for the deflation test when both diagonal neighbours are zero */
    double hmax = 0.0;
    for (int i = 0; i < n; ++i)
        for (int j = (i > 0 ? i - 1 : 0); j < n; ++j)
            if (fabs(A_(i, j)) > hmax) hmax = fabs(A_(i, j));
    int hi = n - 1;
    int its = 0, total = 0;
    while (hi >= 0) {
        /* locate the top of the unreduced block ending at hi */
        int lo = hi;
        while (lo > 0) {
            double s = fabs(A_(lo - 1, lo - 1)) + fabs(A_(lo, lo));
            if (s == 0.0) s = hmax;
            if (fabs(A_(lo, lo - 1)) <= eps * s) { A_(lo, lo - 1) = 0.0; break; }
            --lo;
        }
        if (lo == hi) {                       /* one real eigenvalue */
            wr[hi] = A_(hi, hi); wi[hi] = 0.0;
            --hi; its = 0;
            continue;
        }
        if (lo == hi - 1) {                   /* a 2x2 block */
            double re[2], im[2];
            eig2(A_(hi - 1, hi - 1), A_(hi - 1, hi), A_(hi, hi - 1), A_(hi, hi), re, im);
            wr[hi - 1] = re[0]; wi[hi - 1] = im[0];
            wr[hi] = re[1]; wi[hi] = im[1];
            hi -= 2; its = 0;
            continue;
        }
        if (its >= 30 * n) return -1;
        ++its; ++total;
        /* shifts: the eigenvalues of the trailing 2x2, through their sum and product */
        double s, t;
        if (its == 10 || its == 20) {
            double w = fabs(A_(hi, hi - 1)) + fabs(A_(hi - 1, hi - 2));
            s = 1.5 * w;
            t = w * w;
        } else {
            s = A_(hi - 1, hi - 1) + A_(hi, hi);
            t = A_(hi - 1, hi - 1) * A_(hi, hi) - A_(hi - 1, hi) * A_(hi, hi - 1);
        }
        /* first column of (H - s1 I)(H - s2 I) restricted to the block */
        double h00 = A_(lo, lo), h01 = A_(lo, lo + 1), h10 = A_(lo + 1, lo);
        double h11 = A_(lo + 1, lo + 1), h21 = A_(lo + 2, lo + 1);
        double x[3], u[3], beta;
        x[0] = h00 * h00 + h01 * h10 - s * h00 + t;
        x[1] = h10 * (h00 + h11 - s);
        x[2] = h10 * h21;
        for (int k = lo; k <= hi - 1; ++k) {
            int len = (k + 2 <= hi) ? 3 : 2;
            if (house3(len, x, u, &beta)) {
                int c0 = (k > lo) ? k - 1 : lo;
                for (int j = c0; j <= hi; ++j) {      /* rows k..k+len-1 */
                    double d = 0.0;
                    for (int i = 0; i < len; ++i) d += u[i] * A_(k + i, j);
                    d *= beta;
                    for (int i = 0; i < len; ++i) A_(k + i, j) -= d * u[i];
                }
                int r1 = (k + 3 < hi) ? k + 3 : hi;
                for (int i = lo; i <= r1; ++i) {       /* columns k..k+len-1 */
                    double d = 0.0;
                    for (int j = 0; j < len; ++j) d += A_(i, k + j) * u[j];
                    d *= beta;
                    for (int j = 0; j < len; ++j) A_(i, k + j) -= d * u[j];
                }
            }
            if (k + 1 <= hi - 1) {
                x[0] = A_(k + 1, k);
                x[1] = A_(k + 2, k);
                x[2] = (k + 3 <= hi) ? A_(k + 3, k) : 0.0;
            }
        }
        /* clean the bulge remnants below the subdiagonal inside the block */
        for (int i = lo + 2; i <= hi; ++i) {
            A_(i, i - 2) = 0.0;
            if (i >= lo + 3) A_(i, i - 3) = 0.0;
        }
    }
    if (sweeps_out) *sweeps_out = total;
    return 0;
}

/* Public entry: eigenvalues of the n x n row-major matrix a (overwritten).
 * wr, wi receive real and imaginary parts.  Returns 0, or -1 on QR failure. */
int oracle_eigvals(int n, double* a, double* wr, double* wi, int do_balance, int* sweeps)
{
    if (n <= 0) return 0;
    double* v = (double*)malloc(sizeof(double) * (size_t)n);
    if (!v) return -2;
    if (do_balance) balance(n, a);
    hessenberg(n, a, v);
    int rc = hqr(n, a, wr, wi, sweeps);
    free(v);
    return rc;
}

/* Exposed for tests: balance then Hessenberg form (a overwritten). */
int oracle_hessenberg(int n, double* a, int do_balance)
{
    double* v = (double*)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
    if (!v) return -2;
    if (do_balance) balance(n, a);
    hessenberg(n, a, v);
    free(v);
    return 0;
}
