// One warp solves (B + lam I) x = c for a C x C symmetric positive definite system held
// in shared memory (Section 3.1's Cholesky row solve, for systems too wide for the
// per-thread register version): B as a packed lower triangle P[i (i + 1) / 2 + j],
// factored in place by a left-looking Cholesky (lanes over rows, dot products with the
// pivot row); c is overwritten by x.  Returns false
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

// Factor of B + lam I in place (left-looking: column j from the finished columns 0..j-1,
// lanes over the rows below the diagonal, each a dot product with the broadcast row j).
// *min_ratio (if given) receives the smallest pivot ratio d_j / (B_jj + lam).
template <class T>
__device__ bool warp_chol_factor(T *P, int C, T lam, int lane, T *min_ratio = nullptr) {
    bool ok = true;
    T ratio = T(1);
    for (int j = 0; j < C; ++j) {
        const T *rj = P + ptri(j, 0);
        T s = T(0);
        for (int k = lane; k < j; k += 32) s += rj[k] * rj[k];
        s = warp_allsum(s);
        const T a_jj = P[ptri(j, j)] + lam;
        const T d = a_jj - s;
        ok = ok && (d > T(0));
        if (a_jj > T(0)) ratio = d / a_jj < ratio ? d / a_jj : ratio;
        const T ljj = sqrt(d > T(0) ? d : T(1));
        for (int i = j + 1 + lane; i < C; i += 32) {
            const T *ri = P + ptri(i, 0);
            T t0 = T(0), t1 = T(0), t2 = T(0), t3 = T(0);  // four independent chains
            int k = 0;
            for (; k + 4 <= j; k += 4) {
                t0 += ri[k] * rj[k];
                t1 += ri[k + 1] * rj[k + 1];
                t2 += ri[k + 2] * rj[k + 2];
                t3 += ri[k + 3] * rj[k + 3];
            }
            for (; k < j; ++k) t0 += ri[k] * rj[k];
            P[ptri(i, j)] = (ri[j] - ((t0 + t1) + (t2 + t3))) / ljj;
        }
        __syncwarp();
        if (lane == 0) P[ptri(j, j)] = ljj;
        __syncwarp();
    }
    if (min_ratio) *min_ratio = ratio;
    return ok;
}

// c <- (L L^T)^-1 c with the factor of warp_chol_factor: L y = c, then L^T x = y.
template <class T>
__device__ void warp_chol_apply(const T *P, T *c, int C, int lane) {
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
}

template <class T>
__device__ bool warp_chol_solve(T *P, T *c, int C, T lam, int lane) {
    const bool ok = warp_chol_factor<T>(P, C, lam, lane);
    warp_chol_apply<T>(P, c, C, lane);
    return ok;
}

}  // namespace tfs
