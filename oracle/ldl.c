/*
 * Sparse LDL' factorization and solve for the oracle (test infrastructure).
 *
 * ORACLE / TEST INFRASTRUCTURE ONLY.  Nothing on the GPU solver's path may
 * link, load or call this file; only the tests, the oracle module and the
 * CPU-baseline leg of the benchmark use it.
 *
 * What it computes: the factorization K = L D L' of a symmetric matrix K
 * (here the quasi-definite KKT matrix [[P + sigma I, A'], [A, -R^{-1}]] of
 * the ADMM linear-system step, paper Section 3.2, "Solving the KKT System"),
 * with L unit lower triangular and D diagonal, in the order the caller has
 * already permuted K into.  Quasi-definite matrices have such a factorization
 * for every symmetric permutation (the paper cites George & Ikramov for
 * this), so no pivoting is done; a zero or non-finite pivot is reported.
 *
 * Method: the up-looking sparse LDL' of T. A. Davis ("Algorithm 849: a
 * concise sparse Cholesky factorization package", ACM TOMS 2005), written
 * from its description:
 *   1. symbolic: the elimination tree of K and the number of entries in each
 *      column of L, found by walking, for every entry K(i,k) with i < k, from
 *      i up the tree until a node already visited for row k;
 *   2. numeric: row k of L is the solution of a sparse triangular system
 *      L(0:k,0:k) D y = K(0:k,k); its pattern is the set of tree nodes met in
 *      the same walks, visited in topological order.
 * The input is the upper triangle of K (diagonal included) in compressed
 * sparse column form: column k holds the entries K(i,k) with i <= k.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* Symbolic pass: parent[] (elimination tree, -1 = root) and colcount[] (the
 * number of strictly-lower entries in each column of L). */
void ldl_symbolic(int32_t n, const int64_t *Kp, const int32_t *Ki, int32_t *parent,
                  int64_t *colcount) {
    int32_t *mark = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
    for (int32_t k = 0; k < n; k++) {
        parent[k] = -1;
        mark[k] = k;
        colcount[k] = 0;
        for (int64_t p = Kp[k]; p < Kp[k + 1]; p++) {
            int32_t i = Ki[p];
            if (i >= k) continue;
            /* walk from i towards the root, stopping at nodes seen for row k */
            while (mark[i] != k) {
                if (parent[i] == -1) parent[i] = k;
                colcount[i]++; /* L(k,i) is an entry */
                mark[i] = k;
                i = parent[i];
            }
        }
    }
    free(mark);
}

/* Numeric pass.  Lp must hold the column starts (prefix sums of colcount);
 * Li/Lx receive the row indices and values of L, Dg the diagonal of D.
 * Returns n on success or the index of the first zero / non-finite pivot. */
int32_t ldl_numeric(int32_t n, const int64_t *Kp, const int32_t *Ki, const double *Kx,
                    const int64_t *Lp, const int32_t *parent, int32_t *Li, double *Lx,
                    double *Dg) {
    double *y = (double *)calloc((size_t)(n > 0 ? n : 1), sizeof(double));
    int32_t *pattern = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
    int32_t *mark = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
    int64_t *fill = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
    int32_t result = n;
    for (int32_t k = 0; k < n; k++) {
        /* scatter column k of the upper triangle into y; find the pattern
         * of row k of L (tree nodes reached from each i), stacked so that
         * pattern[top..n) is in topological order */
        int32_t top = n;
        mark[k] = k;
        fill[k] = 0;
        for (int64_t p = Kp[k]; p < Kp[k + 1]; p++) {
            int32_t i = Ki[p];
            if (i > k) continue;
            y[i] += Kx[p];
            int32_t len = 0;
            while (mark[i] != k) {
                pattern[len++] = i; /* temporarily at the front */
                mark[i] = k;
                i = parent[i];
            }
            while (len > 0) pattern[--top] = pattern[--len];
        }
        double dk = y[k];
        y[k] = 0.0;
        for (; top < n; top++) {
            int32_t i = pattern[top];
            double yi = y[i];
            y[i] = 0.0;
            int64_t p2 = Lp[i] + fill[i];
            for (int64_t p = Lp[i]; p < p2; p++) y[Li[p]] -= Lx[p] * yi;
            double lki = yi / Dg[i];
            dk -= lki * yi;
            Li[p2] = k;
            Lx[p2] = lki;
            fill[i]++;
        }
        Dg[k] = dk;
        if (dk == 0.0 || !isfinite(dk)) {
            result = k;
            break;
        }
    }
    free(y);
    free(pattern);
    free(mark);
    free(fill);
    return result;
}

/* Solve L D L' x = b in place (b becomes x). */
void ldl_solve(int32_t n, const int64_t *Lp, const int32_t *Li, const double *Lx,
               const double *Dg, double *b) {
    for (int32_t j = 0; j < n; j++) {
        double bj = b[j];
        for (int64_t p = Lp[j]; p < Lp[j + 1]; p++) b[Li[p]] -= Lx[p] * bj;
    }
    for (int32_t j = 0; j < n; j++) b[j] /= Dg[j];
    for (int32_t j = n - 1; j >= 0; j--) {
        double bj = b[j];
        for (int64_t p = Lp[j]; p < Lp[j + 1]; p++) bj -= Lx[p] * b[Li[p]];
        b[j] = bj;
    }
}
