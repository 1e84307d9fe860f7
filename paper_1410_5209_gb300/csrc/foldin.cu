// Fold-in of a new row against frozen factors: the ALS row solve of Eq. (2),
// a = (B + lambda I_K)^{-1} c with B = sum_e h_e h_e^T, c = sum_e x_e h_e and
// h_e,k = prod_{l != mode} a^(l)_{i_l k}, over the request's m entries.
// Float contexts (K < 128) refine every solve once: the residual of the normal equations
// is formed from the entries in FP64 and the correction solved with the FP32 factor,
// which takes the row to FP32 accuracy whatever the rounding of the FP32 Gram sums.
//
// One CTA per request.  Entries are taken in tiles of kTileE: the tile's H rows are
// built in shared memory, then each thread adds the tile's contribution to its own
// entries of the lower triangle of B (kept in shared memory) and of c.  The K x K
// system is factored in place by a right-looking Cholesky (one column per step), and
// warp 0 does the two triangular solves.
#include <algorithm>

#include "dense_solve.cuh"
#include "sweep.cuh"

namespace tfs {
namespace {

constexpr int kFoldThreads = 256;
constexpr int kTileE = 32;

template <class T>
__global__ void __launch_bounds__(kFoldThreads) k_foldin(const FoldArgs<T> a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int K = a.K;
    T *B = reinterpret_cast<T *>(smem_raw);  // K*K, lower triangle used
    T *cv = B + (size_t)K * K;                // K (c, then y, then x)
    T *H = cv + K;                            // kTileE*K
    T *xs = H + (size_t)kTileE * K;           // kTileE
    __shared__ int bad;
    const int tid = threadIdx.x;
    if (tid == 0) bad = 0;
    for (int q = tid; q < K * K; q += blockDim.x) B[q] = T(0);
    for (int q = tid; q < K; q += blockDim.x) cv[q] = T(0);
    __syncthreads();

    for (int64_t e0 = 0; e0 < a.m; e0 += kTileE) {
        const int ne = (int)(a.m - e0 < kTileE ? a.m - e0 : kTileE);
        for (int q = tid; q < ne * K; q += blockDim.x) {
            const int e = q / K, k = q - e * K;
            T p = T(1);
            int t = 0;
            for (int l = 0; l < a.N; ++l) {
                if (l == a.mode) continue;
                const int32_t idx = a.other[(e0 + e) * (a.N - 1) + t];
                ++t;
                if (idx < 0 || idx >= a.I[l]) {
                    bad = 1;
                    p = T(0);
                } else {
                    p *= a.A[l][(int64_t)idx * K + k];
                }
            }
            H[e * K + k] = p;
        }
        for (int q = tid; q < ne; q += blockDim.x) xs[q] = a.x[e0 + q];
        __syncthreads();
        for (int q = tid; q < K * K; q += blockDim.x) {
            const int i = q / K, j = q - i * K;
            if (j > i) continue;
            T s = T(0);
            for (int e = 0; e < ne; ++e) s += H[e * K + i] * H[e * K + j];
            B[q] += s;
        }
        for (int q = tid; q < K; q += blockDim.x) {
            T s = T(0);
            for (int e = 0; e < ne; ++e) s += H[e * K + q] * xs[e];
            cv[q] += s;
        }
        __syncthreads();
    }
    for (int q = tid; q < K; q += blockDim.x) B[q * K + q] += a.lambda;
    __syncthreads();

    // right-looking Cholesky, lower triangle
    __shared__ int pivot_bad;
    if (tid == 0) pivot_bad = 0;
    for (int j = 0; j < K; ++j) {
        __syncthreads();
        if (tid == 0) {
            T d = B[j * K + j];
            if (!(d > T(0))) {
                pivot_bad = 1;
                d = T(1);
            }
            B[j * K + j] = sqrt(d);
        }
        __syncthreads();
        const T ljj = B[j * K + j];
        for (int i = j + 1 + tid; i < K; i += blockDim.x) B[i * K + j] /= ljj;
        __syncthreads();
        const int rem = K - j - 1;
        for (int q = tid; q < rem * rem; q += blockDim.x) {
            const int i = j + 1 + q / rem, k = j + 1 + q % rem;
            if (k <= i) B[i * K + k] -= B[i * K + j] * B[k * K + j];
        }
    }
    __syncthreads();
    if (tid < kWarp) {
        const int lane = tid;
        for (int i = 0; i < K; ++i) {  // L y = c (y overwrites c)
            T s = T(0);
            for (int k = lane; k < i; k += kWarp) s += B[i * K + k] * cv[k];
            for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xFFFFFFFFu, s, o);
            if (lane == 0) cv[i] = (cv[i] - s) / B[i * K + i];
            __syncwarp();
        }
        for (int i = K - 1; i >= 0; --i) {  // L^T x = y (x overwrites y)
            T s = T(0);
            for (int k = i + 1 + lane; k < K; k += kWarp) s += B[k * K + i] * cv[k];
            for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xFFFFFFFFu, s, o);
            if (lane == 0) cv[i] = (cv[i] - s) / B[i * K + i];
            __syncwarp();
        }
    }
    __syncthreads();
    if (tid == 0) {
        if (bad) atomicOr(&a.stat->bits, kStatFoldRange);
        if (pivot_bad) atomicOr(&a.stat->bits, kStatFoldPivot);
    }
    if (!bad && !pivot_bad)
        for (int q = tid; q < K; q += blockDim.x) a.out[q] = cv[q];
}

// Tiled fold-in for K < 128, any number of requests in one launch: block b takes the
// entries blk_range[2b] .. blk_range[2b + 1] of request blk_req[b] (at most 256); tiles
// of 32 entries build H' = [H | x] in shared memory (8 threads per entry, columns
// strided by 8, one round of independent row loads), and a 16 x 16 grid of register
// tiles accumulates the lower triangle of H'^T H' (B and, in row K, c).  Each block
// writes its partial; k_fold_solve (one warp per request) sums the request's partials
// in block order and solves.  Bad indices and non-positive pivots are flagged per
// request in req_status (1 and 2).
constexpr int kFoldTile = 32;
constexpr int kFoldGramThreads = 256;

template <class T, int CW>
__global__ void __launch_bounds__(kFoldGramThreads) k_fold_gram(const FoldArgs<T> a) {
    constexpr int R = CW / 16, HS = CW + 4;
    __shared__ __align__(16) T H[kFoldTile * HS];
    __shared__ int bad;
    const int tid = threadIdx.x, ty = tid >> 4, tx = tid & 15;
    const int K = a.K;
    const bool active = ty >= tx;
    if (tid == 0) bad = 0;
    T acc[R][R];
#pragma unroll
    for (int i = 0; i < R; ++i)
#pragma unroll
        for (int j = 0; j < R; ++j) acc[i][j] = T(0);
    const int64_t b0 = a.blk_range[2 * blockIdx.x], b1 = a.blk_range[2 * blockIdx.x + 1];
    for (int64_t e0 = b0; e0 < b1; e0 += kFoldTile) {
        const int ne = (int)(b1 - e0 < kFoldTile ? b1 - e0 : kFoldTile);
        __syncthreads();
        {
            const int e = tid >> 3, g = tid & 7;
            const bool valid = e < ne;
            T *h = H + e * HS;
            const T *rows[kMaxModes];
            int t = 0;
            bool ok = valid;
            for (int l = 0; l < a.N; ++l) {
                if (l == a.mode) continue;
                const int32_t idx = valid ? a.other[(e0 + e) * (a.N - 1) + t] : 0;
                const bool in = idx >= 0 && idx < a.I[l];
                ok = ok && in;
                rows[t++] = a.A[l] + (int64_t)(in ? idx : 0) * K;
            }
            if (valid && !ok) bad = 1;
#pragma unroll
            for (int k = 0; k < CW / 8; ++k) {
                const int c = g + 8 * k;
                T hv = T(0);
                if (ok && c < K) {
                    hv = T(1);
                    for (int u = 0; u < a.N - 1; ++u) hv *= rows[u][c];
                }
                h[c] = hv;
            }
            __syncwarp();
            if (g == 0) h[K] = ok ? a.x[e0 + e] : T(0);
        }
        __syncthreads();
        if (active) {
#pragma unroll 4
            for (int e = 0; e < ne; ++e) {
                const T *h = H + e * HS;
                T x[R], y[R];
#pragma unroll
                for (int i = 0; i < R; ++i) x[i] = h[ty * R + i];
#pragma unroll
                for (int j = 0; j < R; ++j) y[j] = h[tx * R + j];
#pragma unroll
                for (int i = 0; i < R; ++i)
#pragma unroll
                    for (int j = 0; j < R; ++j) acc[i][j] += x[i] * y[j];
            }
        }
    }
    __syncthreads();
    if (tid == 0 && bad) atomicOr(&a.req_status[a.blk_req[blockIdx.x]], 1);
    const int NT = K * (K + 1) / 2;
    T *p = a.part + (int64_t)blockIdx.x * (NT + K);
    if (active) {
#pragma unroll
        for (int i = 0; i < R; ++i)
#pragma unroll
            for (int j = 0; j < R; ++j) {
                const int r = ty * R + i, cc = tx * R + j;
                if (r < K && cc <= r) p[r * (r + 1) / 2 + cc] = acc[i][j];
                if (r == K && cc < K) p[NT + cc] = acc[i][j];
            }
    }
}

template <class T>
__global__ void __launch_bounds__(32) k_fold_solve(const FoldArgs<T> a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int K = a.K, lane = threadIdx.x, r = blockIdx.x;
    const int NT = K * (K + 1) / 2, NB = NT + K;
    T *P = reinterpret_cast<T *>(smem_raw);
    T *cv = P + NT;
    const int bb = a.req_blk[r], be = a.req_blk[r + 1];
    for (int q = lane; q < NB; q += 32) {
        T s = T(0);
        for (int b = bb; b < be; ++b) s += a.part[(int64_t)b * NB + q];
        P[q] = s;  // cv follows P: q >= NT lands in cv[q - NT]
    }
    __syncwarp();
    const bool ok = warp_chol_solve<T>(P, cv, K, a.lambda, lane);
    if (!ok) {
        if (lane == 0) atomicOr(&a.req_status[r], 2);
        return;
    }
    for (int q = lane; q < K; q += 32) a.out[(int64_t)r * K + q] = cv[q];
    if (a.refine)
        for (int q = lane; q < NT; q += 32) a.fac[(int64_t)r * NT + q] = P[q];
}

// Refinement, first half: per block of entries (the Gram's block table), the FP64 sum
// over its entries of h_e (x_e - h_e . x0), x0 the request's first solution.  One warp
// per entry at a time (lanes over k, coalesced row reads); h_e,k is a product of FP32
// factor values formed in FP64, so the entry residual x_e - h_e . x0 carries no
// cancellation error of the working precision.  The block's warps add their sums in
// warp order.
constexpr int kFoldResThreads = 256;

template <class T>
__global__ void __launch_bounds__(kFoldResThreads) k_fold_resid(const FoldArgs<T> a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    double *wsum = reinterpret_cast<double *>(smem_raw);  // [8][K]
    const int K = a.K, lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    constexpr int NW = kFoldResThreads / 32;
    const int req = a.blk_req[blockIdx.x];
    const int64_t b0 = a.blk_range[2 * blockIdx.x], b1 = a.blk_range[2 * blockIdx.x + 1];
    double *acc = wsum + (size_t)w * K;
    for (int k = lane; k < K; k += 32) acc[k] = 0.0;
    const bool skip = a.req_status[req] != 0;  // bad index or pivot: no refinement
    const T *x0 = a.out + (int64_t)req * K;
    if (!skip) {
        for (int64_t e = b0 + w; e < b1; e += NW) {
            const T *rows[kMaxModes];
            int t = 0;
            for (int l = 0; l < a.N; ++l) {
                if (l == a.mode) continue;
                const int32_t idx = a.other[e * (a.N - 1) + t];  // checked by k_fold_gram
                rows[t] = a.A[l] + (int64_t)idx * K;
                ++t;
            }
            double dot = 0.0;
            for (int k = lane; k < K; k += 32) {
                double h = 1.0;
                for (int u = 0; u < a.N - 1; ++u) h *= (double)rows[u][k];
                dot += h * (double)x0[k];
            }
            dot = warp_sum_d(dot);
            const double rho = (double)a.x[e] - dot;
            for (int k = lane; k < K; k += 32) {
                double h = 1.0;
                for (int u = 0; u < a.N - 1; ++u) h *= (double)rows[u][k];
                acc[k] += h * rho;
            }
        }
    }
    __syncthreads();
    for (int k = threadIdx.x; k < K; k += blockDim.x) {
        double s = 0.0;
        for (int ww = 0; ww < NW; ++ww) s += wsum[(size_t)ww * K + k];
        a.rpart[(int64_t)blockIdx.x * K + k] = s;
    }
}

// Refinement, second half: one warp per request sums its blocks' partials in block
// order, subtracts lambda x0 (FP64), solves for the correction with the stored factor
// and adds it to x0.
template <class T>
__global__ void __launch_bounds__(32) k_fold_refine(const FoldArgs<T> a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int K = a.K, lane = threadIdx.x, r = blockIdx.x;
    const int NT = K * (K + 1) / 2;
    T *L = reinterpret_cast<T *>(smem_raw);
    T *d = L + NT;
    if (a.req_status[r] != 0) return;
    const int bb = a.req_blk[r], be = a.req_blk[r + 1];
    T *x = a.out + (int64_t)r * K;
    for (int q = lane; q < NT; q += 32) L[q] = a.fac[(int64_t)r * NT + q];
    for (int k = lane; k < K; k += 32) {
        double s = 0.0;
        for (int b = bb; b < be; ++b) s += a.rpart[(int64_t)b * K + k];
        d[k] = (T)(s - (double)a.lambda * (double)x[k]);
    }
    __syncwarp();
    warp_chol_apply<T>(L, d, K, lane);
    for (int k = lane; k < K; k += 32) x[k] += d[k];
}

}  // namespace

bool foldin_tiled_ok(int K) { return K + 1 <= 128; }

int foldin_plan_blocks(const int64_t *offsets, int n_req, std::vector<int64_t> &blk_range,
                       std::vector<int32_t> &blk_req, std::vector<int32_t> &req_blk) {
    blk_range.clear();
    blk_req.clear();
    req_blk.assign((size_t)n_req + 1, 0);
    for (int r = 0; r < n_req; ++r) {
        req_blk[r] = (int32_t)blk_req.size();
        for (int64_t b = offsets[r]; b < offsets[r + 1]; b += 256) {
            blk_range.push_back(b);
            blk_range.push_back(std::min<int64_t>(b + 256, offsets[r + 1]));
            blk_req.push_back(r);
        }
    }
    req_blk[n_req] = (int32_t)blk_req.size();
    return (int)blk_req.size();
}

size_t foldin_part_elems(int K, int blocks) {
    return (size_t)std::max(blocks, 1) * ((size_t)K * (K + 1) / 2 + K);
}

template <class T>
void launch_foldin_tiled(const FoldArgs<T> &a, int blocks, int n_req, cudaStream_t st) {
    const int cw = a.K + 1 <= 32 ? 32 : (a.K + 1 <= 64 ? 64 : 128);
    if (blocks > 0) {
        if (cw == 32)
            k_fold_gram<T, 32><<<blocks, kFoldGramThreads, 0, st>>>(a);
        else if (cw == 64)
            k_fold_gram<T, 64><<<blocks, kFoldGramThreads, 0, st>>>(a);
        else
            k_fold_gram<T, 128><<<blocks, kFoldGramThreads, 0, st>>>(a);
        TFS_CUDA(cudaGetLastError());
    }
    const size_t smem = sizeof(T) * ((size_t)a.K * (a.K + 1) / 2 + a.K);
    TFS_CUDA(raise_smem_limit((const void *)k_fold_solve<T>, (int)smem));
    k_fold_solve<T><<<n_req, 32, smem, st>>>(a);
    TFS_CUDA(cudaGetLastError());
    if (a.refine && blocks > 0) {
        const size_t rs = sizeof(double) * (kFoldResThreads / 32) * (size_t)a.K;
        TFS_CUDA(raise_smem_limit((const void *)k_fold_resid<T>, (int)rs));
        k_fold_resid<T><<<blocks, kFoldResThreads, rs, st>>>(a);
        TFS_CUDA(cudaGetLastError());
        TFS_CUDA(raise_smem_limit((const void *)k_fold_refine<T>, (int)smem));
        k_fold_refine<T><<<n_req, 32, smem, st>>>(a);
        TFS_CUDA(cudaGetLastError());
    }
}

size_t foldin_refine_elems(int K, int blocks, int n_req, size_t *fac_elems) {
    *fac_elems = (size_t)std::max(n_req, 1) * ((size_t)K * (K + 1) / 2);
    return (size_t)std::max(blocks, 1) * (size_t)K;
}

template <class T>
size_t foldin_smem_bytes(int K) {
    return sizeof(T) * ((size_t)K * K + K + (size_t)kTileE * K + kTileE);
}

template <class T>
void launch_foldin(const FoldArgs<T> &a, cudaStream_t st) {
    const size_t smem = foldin_smem_bytes<T>(a.K);
    TFS_CUDA(raise_smem_limit((const void *)k_foldin<T>, (int)smem));
    k_foldin<T><<<1, kFoldThreads, smem, st>>>(a);
    TFS_CUDA(cudaGetLastError());
}

template size_t foldin_smem_bytes<float>(int);
template size_t foldin_smem_bytes<double>(int);
template void launch_foldin<float>(const FoldArgs<float> &, cudaStream_t);
template void launch_foldin<double>(const FoldArgs<double> &, cudaStream_t);
template void launch_foldin_tiled<float>(const FoldArgs<float> &, int, int, cudaStream_t);
template void launch_foldin_tiled<double>(const FoldArgs<double> &, int, int, cudaStream_t);

}  // namespace tfs
