// The fused mode pass of a SALS split (Algorithm 1, inner loop over rows; Eq. (4)).
//
// One warp works through the items of one bin.  For an item (a row, or a chunk of a
// row split across bins) its 32 lanes stride over the row's entries in mode-n order;
// each lane, per entry:
//   1. reads the N-1 other-mode indices and the residual copy (coalesced streams),
//   2. gathers the packed slice rows of the other modes (C-wide, L1/L2 resident),
//   3. forms h = prod_{l != n} a^(l)_{i_l, S} (the Hadamard product of Eq. (4)),
//   4. on the split's first inner iteration refreshes the residual copy to this
//      split's R-hat (Algorithm 1) and writes it back,
//   5. accumulates B += h h^T (lower triangle) and c += r_hat h in registers.
// The warp then sums B and c with butterfly shuffles.  A whole row is solved right
// there: B + lambda I_C (lambda * |Omega_i| when weighted) by a register Cholesky
// (Section 3.1), and the new C parameters go to the packed slice and to A^(n).  A chunk
// writes its partial (B, c) to its slot instead; k_combine sums the slots of each
// split row in slot order (deterministic) and solves.
#pragma once

#include <algorithm>

#include "sweep.cuh"

namespace tfs {

__host__ __device__ constexpr int tri(int i, int j) { return i * (i + 1) / 2 + j; }

template <class T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xFFFFFFFFu, v, o);
    return v;
}

// Solves (B + lam I) x = c for the leading C x C block of a CM x CM packed lower
// triangle; rows/columns >= C are replaced by the identity (their x is 0).
// Returns false when a pivot is <= 0 (x is then meaningless).
template <class T, int CM>
__device__ __forceinline__ bool chol_solve(T (&B)[CM * (CM + 1) / 2], const T (&c)[CM], int C,
                                           T lam, T (&x)[CM]) {
#pragma unroll
    for (int i = 0; i < CM; ++i) {
#pragma unroll
        for (int j = 0; j <= i; ++j) {
            T v = B[tri(i, j)];
            if (i >= C || j >= C)
                v = (i == j) ? T(1) : T(0);
            else if (i == j)
                v += lam;
            B[tri(i, j)] = v;
        }
    }
    bool ok = true;
#pragma unroll
    for (int j = 0; j < CM; ++j) {
        T d = B[tri(j, j)];
#pragma unroll
        for (int k = 0; k < j; ++k) d -= B[tri(j, k)] * B[tri(j, k)];
        ok = ok && (d > T(0));
        const T ljj = sqrt(d > T(0) ? d : T(1));
        B[tri(j, j)] = ljj;
#pragma unroll
        for (int i = j + 1; i < CM; ++i) {
            T s = B[tri(i, j)];
#pragma unroll
            for (int k = 0; k < j; ++k) s -= B[tri(i, k)] * B[tri(j, k)];
            B[tri(i, j)] = s / ljj;
        }
    }
    T y[CM];
#pragma unroll
    for (int i = 0; i < CM; ++i) {
        T s = (i < C) ? c[i] : T(0);
#pragma unroll
        for (int k = 0; k < i; ++k) s -= B[tri(i, k)] * y[k];
        y[i] = s / B[tri(i, i)];
    }
#pragma unroll
    for (int i = CM - 1; i >= 0; --i) {
        T s = y[i];
#pragma unroll
        for (int k = i + 1; k < CM; ++k) s -= B[tri(k, i)] * x[k];
        x[i] = s / B[tri(i, i)];
    }
    return ok;
}

template <class T, int CM>
__device__ __forceinline__ void write_row(const PassArgs<T> &a, int row, const T (&x)[CM]) {
    T *z = a.Zn + (int64_t)row * a.W;
    T *Ar = a.A_n + (int64_t)row * a.K;
#pragma unroll
    for (int c = 0; c < CM; ++c) {
        if (c < a.C) {
            z[c] = x[c];
            Ar[a.S[c]] = x[c];
        }
    }
}

template <class T, int CM>
__global__ void __launch_bounds__(kPassThreads) k_mode_pass(const PassArgs<T> a) {
    constexpr int NT = CM * (CM + 1) / 2;
    const int lane = threadIdx.x & 31;
    const int C = a.C, Cq = a.Cq, first = a.first;
    // Bins are fetched dynamically (one ticket per fetch): which warp runs a bin does
    // not change any result, only the load balance.
    for (;;) {
    unsigned long long tk = 0;
    if (lane == 0) tk = atomicAdd(a.ticket, 1ull) - a.ticket_base;
    tk = __shfl_sync(0xFFFFFFFFu, tk, 0);
    if (tk >= (unsigned long long)a.P) break;
    const int bin = (int)tk;
    const int64_t it_end = a.bin_ptr[bin + 1];
    for (int64_t it = a.bin_ptr[bin]; it < it_end; ++it) {
        const tf_item item = a.items[it];
        const T *zown = a.Zn + (int64_t)item.row * a.W;
        T own_old[CM], own_prev[CM];
#pragma unroll
        for (int c = 0; c < CM; ++c) {
            own_old[c] = (first && c < C) ? zown[a.off_old + c] : T(0);
            own_prev[c] = (first && c < Cq) ? zown[a.off_prev + c] : T(0);
        }
        T Bacc[NT], cacc[CM];
#pragma unroll
        for (int v = 0; v < NT; ++v) Bacc[v] = T(0);
#pragma unroll
        for (int c = 0; c < CM; ++c) cacc[c] = T(0);

        const int64_t jend = item.begin + item.len;
        for (int64_t j = item.begin + lane; j < jend; j += kWarp) {
            T h[CM], qo[CM], qp[CM];
#pragma unroll
            for (int c = 0; c < CM; ++c) h[c] = qo[c] = qp[c] = T(1);
            for (int t = 0; t < a.N - 1; ++t) {
                const T *z = a.Zo[t] + (int64_t)a.oidx[t][j] * a.W;
#pragma unroll
                for (int c = 0; c < CM; ++c) {
                    if (c < C) {
                        h[c] *= z[c];
                        if (first) qo[c] *= z[a.off_old + c];
                    }
                    if (first && c < Cq) qp[c] *= z[a.off_prev + c];
                }
            }
            T v = a.res[j];
            if (first) {
                T po = T(0), pp = T(0);
#pragma unroll
                for (int c = 0; c < CM; ++c) {
                    po += own_old[c] * qo[c];
                    pp += own_prev[c] * qp[c];
                }
                v = v - pp + po;
                a.res[j] = v;
            }
#pragma unroll
            for (int c1 = 0; c1 < CM; ++c1) {
                cacc[c1] += v * h[c1];
#pragma unroll
                for (int c2 = 0; c2 <= c1; ++c2) Bacc[tri(c1, c2)] += h[c1] * h[c2];
            }
        }
#pragma unroll
        for (int v = 0; v < NT; ++v) Bacc[v] = warp_sum(Bacc[v]);
#pragma unroll
        for (int c = 0; c < CM; ++c) cacc[c] = warp_sum(cacc[c]);

        if (lane == 0) {
            if (item.slot >= 0) {
                T *p = a.partials + (int64_t)item.slot * (NT + CM);
#pragma unroll
                for (int v = 0; v < NT; ++v) p[v] = Bacc[v];
#pragma unroll
                for (int c = 0; c < CM; ++c) p[NT + c] = cacc[c];
            } else {
                const T lam = a.weighted ? a.lambda * (T)item.len : a.lambda;
                T x[CM];
                if (chol_solve<T, CM>(Bacc, cacc, C, lam, x))
                    write_row<T, CM>(a, item.row, x);
                else
                    atomicAdd(&a.stat->singular_rows, 1ull);
            }
        }
        __syncwarp();
    }
    }
}

template <class T, int CM>
__global__ void __launch_bounds__(kCombineThreads) k_combine(const PassArgs<T> a,
                                                             const SplitRow *rows) {
    constexpr int NT = CM * (CM + 1) / 2, NB = NT + CM;
    constexpr int G = kCombineThreads / NB;
    __shared__ T red[G * NB];
    __shared__ T tot[NB];
    const SplitRow sr = rows[blockIdx.x];
    const int t = threadIdx.x, g = t / NB, v = t - g * NB;
    if (g < G) {
        T s = T(0);
        for (int k = g; k < sr.n_slots; k += G)
            s += a.partials[(int64_t)(sr.first_slot + k) * NB + v];
        red[t] = s;
    }
    __syncthreads();
    if (t < NB) {
        T s = T(0);
        for (int gg = 0; gg < G; ++gg) s += red[gg * NB + t];
        tot[t] = s;
    }
    __syncthreads();
    if (t == 0) {
        T B[NT], c[CM], x[CM];
#pragma unroll
        for (int q = 0; q < NT; ++q) B[q] = tot[q];
#pragma unroll
        for (int q = 0; q < CM; ++q) c[q] = tot[NT + q];
        const T lam = a.weighted ? a.lambda * (T)sr.len : a.lambda;
        if (chol_solve<T, CM>(B, c, a.C, lam, x))
            write_row<T, CM>(a, sr.row, x);
        else
            atomicAdd(&a.stat->singular_rows, 1ull);
    }
}

template <class T, int CM>
int mode_pass_grid_cm(int P, int num_sms) {
    int per_sm = 0;
    TFS_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_mode_pass<T, CM>,
                                                           kPassThreads, 0));
    return std::max(1, std::min(pass_blocks(P), std::max(per_sm, 1) * num_sms));
}

template <class T, int CM>
void launch_mode_pass_cm(const PassArgs<T> &a, int grid, cudaStream_t st) {
    k_mode_pass<T, CM><<<grid, kPassThreads, 0, st>>>(a);
    TFS_CUDA(cudaGetLastError());
}

template <class T, int CM>
void launch_combine_cm(const PassArgs<T> &a, const SplitRow *rows, int n_rows, cudaStream_t st) {
    if (n_rows <= 0) return;
    k_combine<T, CM><<<n_rows, kCombineThreads, 0, st>>>(a, rows);
    TFS_CUDA(cudaGetLastError());
}

#define TFS_FOR_EACH_CM(X) X(1) X(2) X(4) X(6) X(8) X(10) X(12) X(16)

template <class T>
void launch_mode_pass_impl(const PassArgs<T> &a, int CM, int grid, cudaStream_t st) {
    switch (CM) {
#define TFS_CASE(cm)                                 \
    case cm:                                         \
        launch_mode_pass_cm<T, cm>(a, grid, st);     \
        return;
        TFS_FOR_EACH_CM(TFS_CASE)
#undef TFS_CASE
        default:
            throw ApiError{TF_EINVAL, "no mode-pass instance for this C"};
    }
}

template <class T>
int mode_pass_grid_impl(int CM, int P, int num_sms) {
    switch (CM) {
#define TFS_CASE(cm) \
    case cm:         \
        return mode_pass_grid_cm<T, cm>(P, num_sms);
        TFS_FOR_EACH_CM(TFS_CASE)
#undef TFS_CASE
        default:
            throw ApiError{TF_EINVAL, "no mode-pass instance for this C"};
    }
}

template <class T>
void launch_combine_impl(const PassArgs<T> &a, int CM, const SplitRow *rows, int n_rows,
                         cudaStream_t st) {
    switch (CM) {
#define TFS_CASE(cm)                                        \
    case cm:                                                \
        launch_combine_cm<T, cm>(a, rows, n_rows, st);      \
        return;
        TFS_FOR_EACH_CM(TFS_CASE)
#undef TFS_CASE
        default:
            throw ApiError{TF_EINVAL, "no combine instance for this C"};
    }
}

}  // namespace tfs
