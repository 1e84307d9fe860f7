/*
 * FP64 reference oracle for SALS / CDTF (Shin & Kang, "Distributed Methods for
 * High-dimensional and Large-scale Tensor Factorization", arXiv 1410.5209).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product library links, includes or
 * calls this file; only the tests, the smoke check and the CPU-baseline leg of the
 * benchmark load it.  It shares no code, header, table or helper with the CUDA path.
 *
 * Every routine is a plain, serial, double-precision restatement of the paper:
 *   - Definition 1 / Eq. (1)  loss over the observed set Omega plus lambda * sum ||A||_F^2
 *   - Algorithm 1             serial SALS outer iteration (splits, R-hat, T_in x N modes x rows, R update)
 *   - Eq. (4) + Theorem 1     row update (B + lambda I_C)^{-1} c, solved by Cholesky (Section 3.1)
 *   - Eq. (5)                 residual refresh after a split
 *   - Eq. (2)                 ALS row solve, used here for the fold-in of a new row
 *   - Algorithm 3             greedy row assignment (with the row cap and both tie-breaks)
 * No blocking, fusion or reordering is applied beyond what those statements give.
 * Compiled plain (serial) for the tests; the CPU baseline of the benchmark also compiles
 * it with -fopenmp, which runs the rows of a mode and the per-entry R-hat / R updates in
 * parallel without changing any row's or entry's arithmetic.
 *
 * Readings where the paper is silent (each one is also listed in the design notes):
 *   - Omega_i^(n) is visited in lexicographic order of the coordinate tuple taken
 *     cyclically from mode n: (i_n, i_{n+1}, ..., i_N, i_1, ..., i_{n-1}).  With no
 *     duplicate coordinates this is a total order.
 *   - Weighted lambda (Section 5.1.3) multiplies lambda by |Omega_i^(n)| for row i of
 *     mode n; it is off unless ORC_WEIGHTED is passed.  The loss then uses the same
 *     per-row weights.
 *   - A Cholesky pivot <= 0 (singular B + lambda I, e.g. an empty row with lambda = 0)
 *     leaves the row unchanged and is counted.
 *   - When C does not divide K the last split holds the remaining K mod C columns.
 *   - Alg. 3 ties left after both stated tie-breaks go to the lowest machine index;
 *     rows of equal |Omega_i| are taken in increasing row index.
 *
 * Conventions: 0-based indices; coords are row-major [nnz][N] int32; factor matrix
 * A[n] is row-major [I_n][K]; all arithmetic in double.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

enum { ORC_OK = 0, ORC_EINVAL = 1, ORC_ERANGE = 2, ORC_EDUP = 3, ORC_ENOMEM = 4 };
enum { ORC_WEIGHTED = 1 };

/* ------------------------------------------------------------------------- */
/* Grouping: Omega^(n)_{i_n} (table of symbols, Section 2.1)                  */
/* ------------------------------------------------------------------------- */

/* qsort has no context argument; the comparator reads these. Not re-entrant. */
static const int32_t *g_coords;
static int g_N, g_mode;

static int cmp_cyclic(const void *pa, const void *pb) {
    int64_t a = *(const int64_t *)pa, b = *(const int64_t *)pb;
    for (int t = 0; t < g_N; ++t) {
        int m = (g_mode + t) % g_N;
        int32_t ka = g_coords[a * g_N + m], kb = g_coords[b * g_N + m];
        if (ka != kb) return ka < kb ? -1 : 1;
    }
    return (a > b) - (a < b); /* only reached for duplicate coordinates */
}

/* perm[j] = canonical index of the j-th entry of mode-n order; off[i]..off[i+1]
 * is the range of Omega^(n)_i inside perm. */
int orc_group(int N, const int64_t *dims, int64_t nnz, const int32_t *coords, int n,
              int64_t *off, int64_t *perm) {
    if (N < 1 || n < 0 || n >= N || nnz < 0) return ORC_EINVAL;
    for (int64_t e = 0; e < nnz; ++e) perm[e] = e;
    g_coords = coords; g_N = N; g_mode = n;
    qsort(perm, (size_t)nnz, sizeof(int64_t), cmp_cyclic);
    for (int64_t i = 0; i <= dims[n]; ++i) off[i] = 0;
    for (int64_t e = 0; e < nnz; ++e) off[coords[e * N + n] + 1] += 1;
    for (int64_t i = 0; i < dims[n]; ++i) off[i + 1] += off[i];
    return ORC_OK;
}

/* Omega is a set (table of symbols): reject coordinates out of range or repeated. */
int orc_validate(int N, const int64_t *dims, int64_t nnz, const int32_t *coords) {
    if (N < 1 || nnz < 0) return ORC_EINVAL;
    for (int64_t e = 0; e < nnz; ++e)
        for (int n = 0; n < N; ++n)
            if (coords[e * N + n] < 0 || coords[e * N + n] >= dims[n]) return ORC_ERANGE;
    if (nnz < 2) return ORC_OK;
    int64_t *perm = (int64_t *)malloc(sizeof(int64_t) * (size_t)nnz);
    int64_t *off = (int64_t *)malloc(sizeof(int64_t) * (size_t)(dims[0] + 1));
    if (!perm || !off) { free(perm); free(off); return ORC_ENOMEM; }
    orc_group(N, dims, nnz, coords, 0, off, perm);
    int st = ORC_OK;
    for (int64_t j = 1; j < nnz && st == ORC_OK; ++j) {
        int same = 1;
        for (int n = 0; n < N; ++n)
            if (coords[perm[j] * N + n] != coords[perm[j - 1] * N + n]) { same = 0; break; }
        if (same) st = ORC_EDUP;
    }
    free(perm); free(off);
    return st;
}

/* ------------------------------------------------------------------------- */
/* Definition 1, Eq. (1): residual and loss                                   */
/* ------------------------------------------------------------------------- */

/* r_e = x_e - sum_k prod_n a^(n)_{i_n k}  (residual tensor R, Section 3.1) */
int orc_residual(int N, int64_t nnz, const int32_t *coords, const double *x, int K,
                 const double *const *A, double *r) {
    for (int64_t e = 0; e < nnz; ++e) {
        double s = 0.0;
        for (int k = 0; k < K; ++k) {
            double p = 1.0;
            for (int n = 0; n < N; ++n) p *= A[n][(int64_t)coords[e * N + n] * K + k];
            s += p;
        }
        r[e] = x[e] - s;
    }
    return ORC_OK;
}

/* loss = sum_Omega r^2 + lambda * sum_n ||A^(n)||_F^2 (Eq. 1); with ORC_WEIGHTED the
 * squared norm of row i of mode n is weighted by |Omega_i^(n)| (row_nnz[n][i]).
 * rmse = sqrt(sum r^2 / |Omega|). */
int orc_loss(int N, const int64_t *dims, int64_t nnz, const double *r, int K,
             const double *const *A, double lambda, int flags,
             const int64_t *const *row_nnz, double *loss, double *rmse) {
    double sr = 0.0;
    for (int64_t e = 0; e < nnz; ++e) sr += r[e] * r[e];
    double reg = 0.0;
    for (int n = 0; n < N; ++n)
        for (int64_t i = 0; i < dims[n]; ++i) {
            double w = (flags & ORC_WEIGHTED) ? (double)row_nnz[n][i] : 1.0;
            double s = 0.0;
            for (int k = 0; k < K; ++k) s += A[n][i * K + k] * A[n][i * K + k];
            reg += w * s;
        }
    *loss = sr + lambda * reg;
    *rmse = nnz > 0 ? sqrt(sr / (double)nnz) : 0.0;
    return ORC_OK;
}

/* ------------------------------------------------------------------------- */
/* Cholesky solve of the symmetric positive definite system (Section 3.1)     */
/* ------------------------------------------------------------------------- */

/* Solves M a = c in place (M is m x m row-major, overwritten by its factor L).
 * Returns 0 on success, 1 when a pivot is <= 0. */
static int cholesky_solve(int m, double *M, const double *c, double *a) {
    for (int j = 0; j < m; ++j) {
        double d = M[j * m + j];
        for (int k = 0; k < j; ++k) d -= M[j * m + k] * M[j * m + k];
        if (!(d > 0.0)) return 1;
        double ljj = sqrt(d);
        M[j * m + j] = ljj;
        for (int i = j + 1; i < m; ++i) {
            double s = M[i * m + j];
            for (int k = 0; k < j; ++k) s -= M[i * m + k] * M[j * m + k];
            M[i * m + j] = s / ljj;
        }
    }
    /* L y = c */
    for (int i = 0; i < m; ++i) {
        double s = c[i];
        for (int k = 0; k < i; ++k) s -= M[i * m + k] * a[k];
        a[i] = s / M[i * m + i];
    }
    /* L^T a = y */
    for (int i = m - 1; i >= 0; --i) {
        double s = a[i];
        for (int k = i + 1; k < m; ++k) s -= M[k * m + i] * a[k];
        a[i] = s / M[i * m + i];
    }
    return 0;
}

/* ------------------------------------------------------------------------- */
/* Eq. (4): update of the C parameters of one row                             */
/* ------------------------------------------------------------------------- */

/* Builds B (C x C) and c (C) of Eq. (4) for row i of mode n over Omega_i^(n) (the
 * entries perm[off[i]..off[i+1]) ), with h_c = prod_{l != n} a^(l)_{i_l k_c} and the
 * right-hand side weighted by rhat_e; adds lambda_i I_C and solves by Cholesky.
 * On success writes A[n][i, S] and returns 0; returns 1 (row unchanged) on a
 * non-positive pivot. */
int orc_row_update(int N, int n, int64_t i, const int32_t *coords, const double *rhat,
                   int K, double *const *A, const int32_t *S, int C, double lambda, int flags,
                   const int64_t *off, const int64_t *perm) {
    double *B = (double *)calloc((size_t)C * C, sizeof(double));
    double *c = (double *)calloc((size_t)C, sizeof(double));
    double *h = (double *)malloc(sizeof(double) * (size_t)C);
    double *a = (double *)malloc(sizeof(double) * (size_t)C);
    if (!B || !c || !h || !a) { free(B); free(c); free(h); free(a); return -1; }
    for (int64_t j = off[i]; j < off[i + 1]; ++j) {
        int64_t e = perm[j];
        for (int q = 0; q < C; ++q) {
            double p = 1.0;
            for (int l = 0; l < N; ++l)
                if (l != n) p *= A[l][(int64_t)coords[e * N + l] * K + S[q]];
            h[q] = p;
        }
        for (int q1 = 0; q1 < C; ++q1) {
            for (int q2 = 0; q2 < C; ++q2) B[q1 * C + q2] += h[q1] * h[q2];
            c[q1] += rhat[e] * h[q1];
        }
    }
    double lam = lambda;
    if (flags & ORC_WEIGHTED) lam *= (double)(off[i + 1] - off[i]);
    for (int q = 0; q < C; ++q) B[q * C + q] += lam;
    int st = cholesky_solve(C, B, c, a);
    if (st == 0)
        for (int q = 0; q < C; ++q) A[n][i * K + S[q]] = a[q];
    free(B); free(c); free(h); free(a);
    return st;
}

/* sum_{c in S} prod_n a^(n)_{i_n k_c}: the part of the model carried by columns S. */
static double model_part(int N, const int32_t *ce, int K, double *const *A, const int32_t *S,
                         int C) {
    double s = 0.0;
    for (int q = 0; q < C; ++q) {
        double p = 1.0;
        for (int n = 0; n < N; ++n) p *= A[n][(int64_t)ce[n] * K + S[q]];
        s += p;
    }
    return s;
}

/* ------------------------------------------------------------------------- */
/* Algorithm 1: one outer iteration of serial SALS                            */
/* ------------------------------------------------------------------------- */

/* stats[0] += rows left unchanged because of a non-positive pivot. */
int orc_sals_sweep(int N, const int64_t *dims, int64_t nnz, const int32_t *coords, int K,
                   double *const *A, double *r, int C, double lambda, int T_in, int flags,
                   const int32_t *col_order, const int64_t *const *off,
                   const int64_t *const *perm, int64_t *stats) {
    if (C < 1 || C > K || T_in < 1) return ORC_EINVAL;
    double *rhat = (double *)malloc(sizeof(double) * (size_t)(nnz > 0 ? nnz : 1));
    if (!rhat) return ORC_ENOMEM;
    int nsplit = (K + C - 1) / C;
    for (int s = 0; s < nsplit; ++s) {
        const int32_t *S = col_order + (int64_t)s * C;
        int Cs = (s == nsplit - 1) ? K - s * C : C;
        /* R-hat: r_hat = r + sum_{c in S} prod_n a (Algorithm 1, "compute R-hat") */
#pragma omp parallel for schedule(static)
        for (int64_t e = 0; e < nnz; ++e)
            rhat[e] = r[e] + model_part(N, coords + e * N, K, A, S, Cs);
        /* T_in x (modes x rows), Eq. (4).  The rows of one mode are independent given the
         * other modes (Section 3.3), so the OpenMP build of this file (the CPU baseline)
         * updates them in parallel; each row's arithmetic is the serial one. */
        for (int t = 0; t < T_in; ++t)
            for (int n = 0; n < N; ++n) {
                int64_t bad = 0;
                int oom = 0;
#pragma omp parallel for schedule(dynamic, 16) reduction(+ : bad) reduction(| : oom)
                for (int64_t i = 0; i < dims[n]; ++i) {
                    int st = orc_row_update(N, n, i, coords, rhat, K, A, S, Cs, lambda, flags,
                                            off[n], perm[n]);
                    if (st < 0) oom = 1;
                    if (st == 1) bad += 1;
                }
                if (oom) { free(rhat); return ORC_ENOMEM; }
                if (stats) stats[0] += bad;
            }
        /* Eq. (5): r = r_hat - sum_{c in S} prod_n a */
#pragma omp parallel for schedule(static)
        for (int64_t e = 0; e < nnz; ++e)
            r[e] = rhat[e] - model_part(N, coords + e * N, K, A, S, Cs);
    }
    free(rhat);
    return ORC_OK;
}

/* ------------------------------------------------------------------------- */
/* Eq. (2): ALS row solve against frozen factors (fold-in of a new row)       */
/* ------------------------------------------------------------------------- */

/* A new row of mode `mode` observed at m entries: other[j*(N-1) + t] is the index of
 * the t-th other mode (modes in increasing order, skipping `mode`), x[j] its value.
 * out = (B + lambda I_K)^{-1} c with B, c of Eq. (2).  Returns 1 on a bad pivot. */
int orc_foldin(int N, int K, const double *const *A, int mode, int64_t m,
               const int32_t *other, const double *x, double lambda, double *out) {
    double *B = (double *)calloc((size_t)K * K, sizeof(double));
    double *c = (double *)calloc((size_t)K, sizeof(double));
    double *h = (double *)malloc(sizeof(double) * (size_t)K);
    if (!B || !c || !h) { free(B); free(c); free(h); return ORC_ENOMEM; }
    for (int64_t j = 0; j < m; ++j) {
        for (int k = 0; k < K; ++k) {
            double p = 1.0;
            int t = 0;
            for (int l = 0; l < N; ++l) {
                if (l == mode) continue;
                p *= A[l][(int64_t)other[j * (N - 1) + t] * K + k];
                ++t;
            }
            h[k] = p;
        }
        for (int k1 = 0; k1 < K; ++k1) {
            for (int k2 = 0; k2 < K; ++k2) B[k1 * K + k2] += h[k1] * h[k2];
            c[k1] += x[j] * h[k1];
        }
    }
    for (int k = 0; k < K; ++k) B[k * K + k] += lambda;
    int st = cholesky_solve(K, B, c, out);
    free(B); free(c); free(h);
    return st;
}

/* ------------------------------------------------------------------------- */
/* Algorithm 3: greedy row assignment                                         */
/* ------------------------------------------------------------------------- */

static const int64_t *g_rownnz;
static int cmp_rows_desc(const void *pa, const void *pb) {
    int64_t a = *(const int64_t *)pa, b = *(const int64_t *)pb;
    if (g_rownnz[a] != g_rownnz[b]) return g_rownnz[a] > g_rownnz[b] ? -1 : 1;
    return (a > b) - (a < b);
}

/* row_nnz[n][i] = |Omega_i^(n)|; assign[n][i] receives the machine of row i of mode n. */
int orc_greedy_assign(int N, const int64_t *dims, const int64_t *const *row_nnz, int M,
                      int32_t *const *assign) {
    if (M < 1) return ORC_EINVAL;
    int64_t *omega_all = (int64_t *)calloc((size_t)M, sizeof(int64_t)); /* |_m Omega| */
    int64_t *omega_n = (int64_t *)malloc(sizeof(int64_t) * (size_t)M);  /* |_m Omega^(n)| */
    int64_t *rows_n = (int64_t *)malloc(sizeof(int64_t) * (size_t)M);   /* |_m S_n| */
    if (!omega_all || !omega_n || !rows_n) {
        free(omega_all); free(omega_n); free(rows_n); return ORC_ENOMEM;
    }
    for (int n = 0; n < N; ++n) {
        int64_t In = dims[n];
        int64_t cap = (In + M - 1) / M;
        for (int m = 0; m < M; ++m) { omega_n[m] = 0; rows_n[m] = 0; }
        int64_t *order = (int64_t *)malloc(sizeof(int64_t) * (size_t)(In > 0 ? In : 1));
        if (!order) { free(omega_all); free(omega_n); free(rows_n); return ORC_ENOMEM; }
        for (int64_t i = 0; i < In; ++i) order[i] = i;
        g_rownnz = row_nnz[n];
        qsort(order, (size_t)In, sizeof(int64_t), cmp_rows_desc);
        for (int64_t t = 0; t < In; ++t) {
            int64_t i = order[t];
            int best = -1;
            for (int m = 0; m < M; ++m) {
                if (rows_n[m] >= cap) continue;
                if (best < 0 || omega_n[m] < omega_n[best] ||
                    (omega_n[m] == omega_n[best] &&
                     (rows_n[m] < rows_n[best] ||
                      (rows_n[m] == rows_n[best] && omega_all[m] < omega_all[best]))))
                    best = m;
            }
            assign[n][i] = best;
            rows_n[best] += 1;
            omega_n[best] += row_nnz[n][i];
            omega_all[best] += row_nnz[n][i];
        }
        free(order);
    }
    free(omega_all); free(omega_n); free(rows_n);
    return ORC_OK;
}
