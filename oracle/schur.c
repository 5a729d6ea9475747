/* Dense Schur complement of the quasi-definite KKT matrix of the ADMM linear
 * step (paper Section 3.2, eq. (kkt)) after the constraint block is
 * eliminated:
 *
 *     S = P + sigma I + A' R A,   R = diag(r)   (n x n, dense, row-major)
 *
 * which is the matrix of the reduced system eq. (kkt_red_sc).  TEST
 * INFRASTRUCTURE of the FP64 CPU oracle (oracle/dense.py); the GPU path never
 * forms S.
 *
 * Each constraint row j adds r_j a_j a_j' (a_j its nonzeros) to S.  The rows
 * of S are split into bands, one per thread; a thread visits every row of A
 * in order and adds only the products that land in its band, so each entry
 * of S is summed by one thread in the order of the rows of A: the result
 * does not depend on the number of threads. */
#include <stdint.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

void schur_form(int32_t n, int32_t m, const int64_t *Ap, const int32_t *Ai, const double *Ax, const double *r,
                const int64_t *Pp, const int32_t *Pi, const double *Px, double sigma, double *S) {
    memset(S, 0, sizeof(double) * (size_t)n * (size_t)n);
#pragma omp parallel
    {
        int t = 0, nt = 1;
#ifdef _OPENMP
        t = omp_get_thread_num();
        nt = omp_get_num_threads();
#endif
        const int32_t lo = (int32_t)((int64_t)n * t / nt);
        const int32_t hi = (int32_t)((int64_t)n * (t + 1) / nt);
        for (int32_t j = 0; j < m; ++j) {
            const int64_t b = Ap[j], e = Ap[j + 1];
            for (int64_t p = b; p < e; ++p) {
                const int32_t i = Ai[p];
                if (i < lo || i >= hi) continue;
                const double ra = r[j] * Ax[p];
                double *row = S + (size_t)i * (size_t)n;
                for (int64_t q = b; q < e; ++q) row[Ai[q]] += ra * Ax[q];
            }
        }
        for (int32_t i = lo; i < hi; ++i) {
            double *row = S + (size_t)i * (size_t)n;
            for (int64_t p = Pp[i]; p < Pp[i + 1]; ++p) row[Pi[p]] += Px[p];
            row[i] += sigma;
        }
    }
}
