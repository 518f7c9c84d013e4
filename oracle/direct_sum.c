/*
 * Oracle (test infrastructure only): direct O(n^2) kernel sums in FP64.
 *
 * Computes, for each requested row r,
 *     out[r, c] = sum_{j != r} K(x_r - x_j) * V[j, c]
 * which is (W V)_r for the weight matrix of Sec. 2 (w(x_i,x_j) = K(x_i - x_j)
 * for i != j, zero diagonal because self-edges are excluded) with one of the
 * two radial kernels named in Sec. 4:
 *     kernel 0 (Gaussian)   K(y) = exp(-||y||^2 / sigma^2)
 *     kernel 1 (Laplacian)  K(y) = exp(-||y|| / sigma)
 * Points X are n x d row-major, V is n x b
 * row-major, out is nrows x b row-major.  rows == NULL means all rows.
 *
 * The sum over j runs in index order, as the definition reads (in FP64 its
 * rounding error, at most about n ulp, stays far below every tolerance the
 * tests use).  OpenMP parallelises over rows; nthreads <= 0 uses the runtime
 * default.
 * Returns 0 on success, -1 on bad arguments.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORACLE_MAXB 64

int oracle_kernel_rows(const double *X, int64_t n, int d, double sigma, int kernel, const double *V, int b,
                       const int64_t *rows, int64_t nrows, double *out, int nthreads)
{
    if (!X || !V || !out || n <= 0 || d < 1 || b < 1 || b > ORACLE_MAXB || !(sigma > 0) ||
        (kernel != 0 && kernel != 1))
        return -1;
    if (rows == NULL) nrows = n;
    const double inv_s2 = 1.0 / (sigma * sigma);
    const double inv_s = 1.0 / sigma;
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 4)
#endif
    for (int64_t rr = 0; rr < nrows; ++rr) {
        const int64_t r = rows ? rows[rr] : rr;
        double total[ORACLE_MAXB];
        for (int c = 0; c < b; ++c) total[c] = 0.0;
        if (r < 0 || r >= n) {
            for (int c = 0; c < b; ++c) out[rr * b + c] = NAN;
            continue;
        }
        const double *xr = X + r * d;
        for (int64_t j = 0; j < n; ++j) {
            if (j == r) continue;
            const double *xj = X + j * d;
            double r2 = 0.0;
            for (int a = 0; a < d; ++a) {
                const double t = xr[a] - xj[a];
                r2 += t * t;
            }
            const double w = kernel == 0 ? exp(-r2 * inv_s2) : exp(-sqrt(r2) * inv_s);
            const double *vj = V + j * b;
            for (int c = 0; c < b; ++c) total[c] += w * vj[c];
        }
        for (int c = 0; c < b; ++c) out[rr * b + c] = total[c];
    }
    return 0;
}

int oracle_gauss_rows(const double *X, int64_t n, int d, double sigma, const double *V, int b,
                      const int64_t *rows, int64_t nrows, double *out, int nthreads)
{
    return oracle_kernel_rows(X, n, d, sigma, 0, V, b, rows, nrows, out, nthreads);
}

/* Number of threads OpenMP would use (for the baseline's core count). */
int oracle_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
