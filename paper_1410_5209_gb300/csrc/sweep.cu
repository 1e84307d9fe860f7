// Per-split and per-sweep helper kernels: slice packing (the C columns of a split,
// Theorem 3's "only C columns need to be resident"), residual reconstruction and
// loss reduction (Eq. 1, accumulated in double in a fixed order), residual
// initialisation (Section 3.1) and the default factor initialisation (Algorithm 1).
#include <math.h>

#include <map>
#include <mutex>

#include <type_traits>

#include "sweep.cuh"

namespace tfs {

cudaError_t raise_smem_limit(const void *kern, int bytes) {
    static std::mutex mu;
    static std::map<std::pair<int, const void *>, int> limit;  // (device, kernel) -> bytes
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    std::lock_guard<std::mutex> g(mu);
    int &cur = limit[{dev, kern}];
    if (bytes <= cur) return cudaSuccess;
    e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (e == cudaSuccess) cur = bytes;
    return e;
}

int pick_cm(int C) {
    static const int cms[] = {1, 2, 4, 6, 8, 10, 12, 16};
    for (int cm : cms)
        if (C <= cm) return cm;
    if (wide_tile_width(C) > 0) return (C + 3) / 4 * 4;
    return 0;
}

namespace {

constexpr int kResThreads = 256;

template <class T>
__global__ void k_pack(const PackArgs<T> a) {
    const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= a.row_base[a.N]) return;
    int l = 0;
    while (r >= a.row_base[l + 1]) ++l;
    const int64_t i = r - a.row_base[l];  // slice row (rank)
    const T *Ar = a.A[l] + (int64_t)a.id_of[l][i] * a.K;
    T *z = a.Z[l] + i * a.W;
    // regions are CM = off_prev wide; columns beyond C (cur, old) and Cq (prev) are
    // zero, so products over a full region need no column mask
    const int CM = a.off_prev;
    for (int c = 0; c < CM; ++c) {
        const T v = c < a.C ? Ar[a.S[c]] : T(0);
        z[c] = v;
        z[a.off_old + c] = v;
        z[a.off_prev + c] = c < a.Cq ? Ar[a.Q[c]] : T(0);
    }
}

template <class T>
__global__ void __launch_bounds__(kResThreads) k_init_res(const InitArgs<T> a) {
    const int lane = threadIdx.x & 31;
    const int bin = (int)(((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5);
    if (bin >= a.P) return;
    for (int64_t it = a.bin_ptr[bin]; it < a.bin_ptr[bin + 1]; ++it) {
        const tf_item item = a.items[it];
        const T *An = a.An + (int64_t)item.row * a.K;
        const int64_t jend = item.begin + item.len;
        for (int64_t j = item.begin + lane; j < jend; j += kWarp) {
            T model = T(0);
            if (!a.model_zero) {
                for (int k = 0; k < a.K; ++k) {
                    T q = An[k];
                    for (int t = 0; t < a.N - 1; ++t)
                        q *= a.Ao[t][(int64_t)a.id_o[t][a.oidx[t][j]] * a.K + k];
                    model += q;
                }
            }
            a.res[j] = a.x[a.perm[j]] - model;
        }
    }
}

template <class T>
__global__ void __launch_bounds__(kResThreads) k_reg(const T *A, int64_t I, int K,
                                                     const int64_t *off, double *block_out) {
    __shared__ double wsum[kResThreads / kWarp];
    double acc = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < I;
         i += (int64_t)gridDim.x * blockDim.x) {
        double s = 0.0;
        for (int k = 0; k < K; ++k) {
            const double v = (double)A[i * K + k];
            s += v * v;
        }
        acc += off ? s * (double)(off[i + 1] - off[i]) : s;
    }
    acc = warp_sum_d(acc);
    if ((threadIdx.x & 31) == 0) wsum[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int w = 0; w < kResThreads / kWarp; ++w) s += wsum[w];
        block_out[blockIdx.x] = s;
    }
}

__global__ void k_sum_blocks(const double *in, int n, double *out) {
    __shared__ double sh[256];
    double s = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) s += in[i];
    sh[threadIdx.x] = s;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) *out = sh[0];
}

__device__ __forceinline__ uint64_t mix64(uint64_t z) {
    z += 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

// Box-Muller from two counter-based uniforms per element.  Float factors take 24-bit
// uniforms and float arithmetic (FP64 transcendentals run at a small fraction of the
// FP32 rate on this GPU and made the draw a millisecond per 1e7 values).
template <class T>
__global__ void k_init_normal(T *A, int64_t count, uint64_t key, double std) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= count) return;
    if constexpr (std::is_same<T, float>::value) {
        const float u1 = (float)(mix64(key + 2 * (uint64_t)i) >> 40) * 0x1.0p-24f;
        const float u2 = (float)(mix64(key + 2 * (uint64_t)i + 1) >> 40) * 0x1.0p-24f;
        A[i] = (float)std * sqrtf(-2.0f * log1pf(-u1)) * cospif(2.0f * u2);
    } else {
        const double u1 = (double)(mix64(key + 2 * (uint64_t)i) >> 11) * 0x1.0p-53;
        const double u2 = (double)(mix64(key + 2 * (uint64_t)i + 1) >> 11) * 0x1.0p-53;
        A[i] = (T)(std * sqrt(-2.0 * log1p(-u1)) * cospi(2.0 * u2));
    }
}

// One warp per coordinate, lanes over the K columns (coalesced factor rows), FP64 sum.
template <class T>
__global__ void __launch_bounds__(256) k_predict(const PredictArgs<T> a) {
    const int lane = threadIdx.x & 31;
    const int64_t e = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (e >= a.m) return;
    const int32_t *c = a.coords + e * a.N;
    bool ok = true;
    for (int n = 0; n < a.N; ++n) ok = ok && c[n] >= 0 && c[n] < a.I[n];
    double s = 0.0;
    if (ok)
        for (int k = lane; k < a.K; k += 32) {
            double p = 1.0;
            for (int n = 0; n < a.N; ++n) p *= (double)a.A[n][(int64_t)c[n] * a.K + k];
            s += p;
        }
    s = warp_sum_d(s);
    if (lane == 0) {
        a.out[e] = ok ? (T)s : T(0);
        if (!ok) atomicOr(&a.stat->bits, kStatPredictRange);
    }
}

inline unsigned blocks_for(int64_t n, int threads) {
    return (unsigned)((n > 0 ? n : 1) + threads - 1) / threads;
}

}  // namespace

template <class T>
void launch_pack(const PackArgs<T> &a, cudaStream_t st) {
    const int64_t rows = a.row_base[a.N];
    if (rows <= 0) return;
    k_pack<T><<<blocks_for(rows, 256), 256, 0, st>>>(a);
    TFS_CUDA(cudaGetLastError());
}

template <class T>
void launch_init_res(const InitArgs<T> &a, cudaStream_t st) {
    k_init_res<T><<<(unsigned)((a.P * kWarp + kResThreads - 1) / kResThreads), kResThreads, 0, st>>>(a);
    TFS_CUDA(cudaGetLastError());
}

template <class T>
void launch_reg(const T *A, int64_t I, int K, const int64_t *off, double *block_out, int blocks,
                cudaStream_t st) {
    k_reg<T><<<blocks, kResThreads, 0, st>>>(A, I, K, off, block_out);
    TFS_CUDA(cudaGetLastError());
}

void launch_sum_blocks(const double *in, int n, double *out, cudaStream_t st) {
    k_sum_blocks<<<1, 256, 0, st>>>(in, n, out);
    TFS_CUDA(cudaGetLastError());
}

template <class T>
void launch_predict(const PredictArgs<T> &a, cudaStream_t st) {
    if (a.m <= 0) return;
    k_predict<T><<<blocks_for(a.m * 32, 256), 256, 0, st>>>(a);
    TFS_CUDA(cudaGetLastError());
}

// Bfloat16 copy of a slice's columns, two values per thread (round to nearest even).
__global__ void k_slice_bf16(const float *__restrict__ Z, uint32_t *__restrict__ Zb, int64_t rows,
                             int W, int Wb, int col0, int npairs) {
    const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= rows * npairs) return;
    const int64_t i = q / npairs;
    const int c = col0 + 2 * (int)(q - i * npairs);
    const float2 v = *reinterpret_cast<const float2 *>(Z + i * W + c);
    uint32_t packed;
    asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(packed) : "f"(v.y), "f"(v.x));
    Zb[(i * Wb + c) / 2] = packed;
}

void launch_slice_bf16(const float *Z, uint16_t *Zb, int64_t rows, int W, int Wb, int col0,
                       int ncols, cudaStream_t st) {
    if (rows <= 0 || ncols <= 0) return;
    if ((col0 | ncols | W | Wb) & 1) throw ApiError{TF_EINVAL, "bfloat16 slice copy: odd column"};
    const int npairs = ncols / 2;
    k_slice_bf16<<<blocks_for(rows * npairs, 256), 256, 0, st>>>(
        Z, reinterpret_cast<uint32_t *>(Zb), rows, W, Wb, col0, npairs);
    TFS_CUDA(cudaGetLastError());
}

template <class T>
void launch_init_normal(T *A, int64_t count, uint64_t seed, uint64_t stream_id, double std,
                        cudaStream_t st) {
    if (count <= 0) return;
    const uint64_t key = mix64_host(seed ^ mix64_host(stream_id + 0x51A5ull));
    k_init_normal<T><<<blocks_for(count, 256), 256, 0, st>>>(A, count, key, std);
    TFS_CUDA(cudaGetLastError());
}

#define TFS_INST(T)                                                                        \
    template void launch_pack<T>(const PackArgs<T> &, cudaStream_t);                       \
    template void launch_init_res<T>(const InitArgs<T> &, cudaStream_t);                   \
    template void launch_reg<T>(const T *, int64_t, int, const int64_t *, double *, int,   \
                                cudaStream_t);                                             \
    template void launch_init_normal<T>(T *, int64_t, uint64_t, uint64_t, double, cudaStream_t); \
    template void launch_predict<T>(const PredictArgs<T> &, cudaStream_t);
TFS_INST(float)
TFS_INST(double)
#undef TFS_INST

}  // namespace tfs
