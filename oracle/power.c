/*
 * O1 in C: the Power Method S_{t+1} = (c P^T S_t P) v I from S_0 = I (Sec. 2.2,
 * "Other Related Work"), FP64, OpenMP over rows, for graphs of up to a few 10^4 nodes.
 *
 * TEST INFRASTRUCTURE ONLY.  Loaded by oracle/power.py (power_method_c) for tests/.
 * The CUDA library never links or includes this file.
 *
 * P is the reverse transition matrix: P(a, i) = mult(a -> i) / din(i) for a in I(i)
 * (a repeated in-edge counts once per copy).  One iteration, written entry by entry:
 *   T(i, :)  = (1/din(i)) sum_{a in I(i)} S_t(a, :)          T = P^T S_t (0 if din(i) = 0)
 *   M(i, j)  = (1/din(j)) sum_{b in I(j)} T(i, b)            M = T P     (0 if din(j) = 0)
 *   S_{t+1}(i, j) = c M(i, j) off the diagonal, 1 on it.
 * The off-diagonal entries c M stay below 1 and the diagonal of c M below 1, so the
 * element-wise maximum with I is exactly this.  After t iterations the error is at
 * most c^(t+1).  S is n x n row-major, owned by the caller; a second n x n buffer is
 * allocated here for T.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

int oracle_power_method(int64_t n, const int64_t* rp, const int32_t* col, double c, int32_t iterations,
                        double* S) {
    if (n < 1 || !rp || !S || iterations < 0) return -1;
    double* T = (double*)malloc(sizeof(double) * (size_t)n * (size_t)n);
    if (!T) return -2;
    memset(S, 0, sizeof(double) * (size_t)n * (size_t)n);
    for (int64_t i = 0; i < n; ++i) S[i * n + i] = 1.0;
    for (int32_t it = 0; it < iterations; ++it) {
#pragma omp parallel for schedule(dynamic, 16)
        for (int64_t i = 0; i < n; ++i) {
            double* Ti = T + i * n;
            memset(Ti, 0, sizeof(double) * (size_t)n);
            const int64_t b = rp[i], e = rp[i + 1];
            if (e == b) continue;
            for (int64_t p = b; p < e; ++p) {
                const double* Sa = S + (int64_t)col[p] * n;
                for (int64_t j = 0; j < n; ++j) Ti[j] += Sa[j];
            }
            const double inv = 1.0 / (double)(e - b);
            for (int64_t j = 0; j < n; ++j) Ti[j] *= inv;
        }
#pragma omp parallel for schedule(dynamic, 16)
        for (int64_t i = 0; i < n; ++i) {
            const double* Ti = T + i * n;
            double* Si = S + i * n;
            for (int64_t j = 0; j < n; ++j) {
                const int64_t b = rp[j], e = rp[j + 1];
                double sum = 0.0;
                for (int64_t p = b; p < e; ++p) sum += Ti[col[p]];
                Si[j] = e > b ? c * (sum / (double)(e - b)) : 0.0;
            }
            Si[i] = 1.0;
        }
    }
    free(T);
    return 0;
}
