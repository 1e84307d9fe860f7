// Fold-in of a new row against frozen factors: the ALS row solve of Eq. (2),
// a = (B + lambda I_K)^{-1} c with B = sum_e h_e h_e^T, c = sum_e x_e h_e and
// h_e,k = prod_{l != mode} a^(l)_{i_l k}, over the request's m entries.
//
// One CTA per request.  Entries are taken in tiles of kTileE: the tile's H rows are
// built in shared memory, then each thread adds the tile's contribution to its own
// entries of the lower triangle of B (kept in shared memory) and of c.  The K x K
// system is factored in place by a right-looking Cholesky (one column per step), and
// warp 0 does the two triangular solves.
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

}  // namespace

template <class T>
size_t foldin_smem_bytes(int K) {
    return sizeof(T) * ((size_t)K * K + K + (size_t)kTileE * K + kTileE);
}

template <class T>
void launch_foldin(const FoldArgs<T> &a, cudaStream_t st) {
    const size_t smem = foldin_smem_bytes<T>(a.K);
    TFS_CUDA(cudaFuncSetAttribute(k_foldin<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)smem));
    k_foldin<T><<<1, kFoldThreads, smem, st>>>(a);
    TFS_CUDA(cudaGetLastError());
}

template size_t foldin_smem_bytes<float>(int);
template size_t foldin_smem_bytes<double>(int);
template void launch_foldin<float>(const FoldArgs<float> &, cudaStream_t);
template void launch_foldin<double>(const FoldArgs<double> &, cudaStream_t);

}  // namespace tfs
