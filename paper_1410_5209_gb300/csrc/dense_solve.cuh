// One warp solves (B + lam I) x = c for a C x C symmetric positive definite system held
// in shared memory (Section 3.1's Cholesky row solve, for systems too wide for the
// per-thread register version): B as a packed lower triangle P[i (i + 1) / 2 + j],
// factored in place by a right-looking Cholesky; c is overwritten by x.  Returns false
// (P and c then meaningless) when a pivot is not positive.  Every lane calls it.
#pragma once

namespace tfs {

__host__ __device__ constexpr int ptri(int i, int j) { return i * (i + 1) / 2 + j; }

template <class T>
__device__ __forceinline__ T warp_allsum(T v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xFFFFFFFFu, v, o);
    return v;
}

template <class T>
__device__ bool warp_chol_solve(T *P, T *c, int C, T lam, int lane) {
    for (int i = lane; i < C; i += 32) P[ptri(i, i)] += lam;
    __syncwarp();
    bool ok = true;
    for (int j = 0; j < C; ++j) {
        const T d = P[ptri(j, j)];
        ok = ok && (d > T(0));
        const T ljj = sqrt(d > T(0) ? d : T(1));
        __syncwarp();
        if (lane == 0) P[ptri(j, j)] = ljj;
        for (int i = j + 1 + lane; i < C; i += 32) P[ptri(i, j)] /= ljj;
        __syncwarp();
        // trailing update of the lower triangle: rows i > j, columns j < k <= i
        for (int i = j + 1; i < C; ++i) {
            const T lij = P[ptri(i, j)];
            T *row = P + ptri(i, 0);
            for (int k = j + 1 + lane; k <= i; k += 32) row[k] -= lij * P[ptri(k, j)];
        }
        __syncwarp();
    }
    // L y = c, then L^T x = y
    for (int i = 0; i < C; ++i) {
        T s = T(0);
        for (int k = lane; k < i; k += 32) s += P[ptri(i, k)] * c[k];
        s = warp_allsum(s);
        if (lane == 0) c[i] = (c[i] - s) / P[ptri(i, i)];
        __syncwarp();
    }
    for (int i = C - 1; i >= 0; --i) {
        T s = T(0);
        for (int k = i + 1 + lane; k < C; k += 32) s += P[ptri(k, i)] * c[k];
        s = warp_allsum(s);
        if (lane == 0) c[i] = (c[i] - s) / P[ptri(i, i)];
        __syncwarp();
    }
    return ok;
}

}  // namespace tfs
