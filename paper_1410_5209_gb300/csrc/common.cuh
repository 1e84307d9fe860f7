// Shared definitions of the SALS / CDTF CUDA library (sm_103a).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/tf_sals.h"

namespace tfs {

constexpr int kMaxModes = 8;
constexpr int kWarp = 32;

// Bits of the device status word (OR-ed by kernels, read back by synchronising calls).
enum : int {
    kStatRange = 1,      // coordinate out of range
    kStatDup = 2,        // duplicate coordinate
    kStatFoldRange = 4,  // fold-in index out of range
    kStatFoldPivot = 8,  // fold-in Cholesky pivot <= 0
    kStatTimeout = 16,   // a bounded wait on the device gave up
    kStatPredictRange = 32,  // tf_predict coordinate out of range
    kStatPlan = 64,          // a gather plan outgrew its bound (internal error)
};

struct DeviceStatus {
    int bits;
    int pad;
    unsigned long long singular_rows;  // rows left unchanged by a pivot <= 0
    unsigned long long fp64_rows;      // float rows re-solved in FP64 (ill-conditioned)
};

// ------------------------------------------------------------------ error plumbing

struct CudaError {
    cudaError_t err;
    const char *what;
};

#define TFS_CUDA(call)                                                    \
    do {                                                                  \
        cudaError_t e_ = (call);                                          \
        if (e_ != cudaSuccess) throw ::tfs::CudaError{e_, #call};         \
    } while (0)

struct ApiError {
    tf_status status;
    std::string msg;
};

inline uint64_t mix64_host(uint64_t z) {  // splitmix64 (Steele, Lea, Flood 2014)
    z += 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

#ifdef __CUDACC__
__device__ __forceinline__ double warp_sum_d(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xFFFFFFFFu, v, o);
    return v;
}
#endif

inline int ceil_log2_u64(uint64_t v) {  // bits needed to represent v - 1 (v >= 1)
    int b = 0;
    while (b < 63 && (uint64_t(1) << b) < v) ++b;
    return b;
}

template <class T>
inline T ceil_div(T a, T b) {
    return (a + b - 1) / b;
}

// ------------------------------------------------------------------ sort (sort.cu)

// Workspace-allocating stable LSD radix sort of (key, value) pairs on 32-bit keys,
// `bits` low-order bits significant.  Result lands in keys/vals (in place).
struct SortWorkspace {
    uint32_t *keys_alt = nullptr;
    int32_t *vals_alt = nullptr;
    uint32_t *hist = nullptr;
    uint32_t *scan_tmp = nullptr;
    size_t cap_items = 0, cap_hist = 0, cap_scan = 0;
    void reserve(int64_t n, cudaStream_t st);  // stream-ordered allocations on st
    void release(cudaStream_t st);
};

// Raises a kernel's dynamic shared-memory limit on the current device to at least `bytes`
// and never lowers it.  The limit is one per kernel for the whole process, and contexts
// driven from other host threads may launch the same kernel with other sizes meanwhile:
// lowering it between another thread's set and launch would fail that launch.
cudaError_t raise_smem_limit(const void *kern, int bytes);

size_t sort_workspace_bytes(int64_t n);  // device bytes SortWorkspace::reserve(n) holds

// The library's stream-ordered memory pool on the current device, created on first use.
// Freed blocks stay in it for later contexts (no unmapping when a context is destroyed,
// none of the mapping cost when the next one is created) until tf_pool_trim; the pool
// inserts no cross-stream dependencies to reuse a block (a context never waits for
// another context's stream).  nullptr when no pool can be created.
cudaMemPool_t library_pool();

// Stream-ordered allocation from library_pool() (the device's default pool as a fallback).
inline cudaError_t pool_alloc(void **p, size_t bytes, cudaStream_t st) {
    cudaMemPool_t pool = library_pool();
    return pool ? cudaMallocFromPoolAsync(p, bytes, pool, st) : cudaMallocAsync(p, bytes, st);
}

void radix_sort_pairs(uint32_t *keys, int32_t *vals, int64_t n, int bits, SortWorkspace &ws,
                      cudaStream_t st);

// Exclusive scan of n uint32 values (out may alias in).  tmp: scan_temp_elems(n) words.
size_t scan_temp_elems(int64_t n);
void scan_exclusive_u32(const uint32_t *in, uint32_t *out, int64_t n, uint32_t *tmp,
                        cudaStream_t st);

// Builds the layout pieces used by the context (see sort.cu for the contracts).
void launch_transpose_check(const int32_t *coords_rowmajor, int N, int64_t nnz,
                            const int64_t *dims_dev, int32_t *coords_soa, DeviceStatus *stat,
                            cudaStream_t st);
void launch_iota(int32_t *p, int64_t n, cudaStream_t st);
void launch_gather_keys(const int32_t *col, const int32_t *perm, uint32_t *keys, int64_t n,
                        cudaStream_t st);
// out[i] = rank[col[perm[i]]]
void launch_gather_rank(const int32_t *col, const int32_t *perm, const int32_t *rank, int32_t *out,
                        int64_t n, cudaStream_t st);
void launch_offsets(const uint32_t *sorted_keys, int64_t n, int64_t I, int64_t *off,
                    cudaStream_t st);
void launch_dup_check(const int32_t *coords_soa, int N, int64_t nnz, const int32_t *perm,
                      DeviceStatus *stat, cudaStream_t st);

// ------------------------------------------------------------------ scheduling (sched.cpp)

// Row ids in decreasing order of count, equal counts in increasing id (host).
std::vector<int64_t> rows_by_degree(const std::vector<int64_t> &count);
tf_status plan_mode(const int64_t *off, int64_t I, int P, int64_t cap, tf_sched_policy policy,
                    uint64_t seed, std::vector<tf_item> &items, int64_t &n_slots,
                    std::vector<int64_t> &bin_ptr);

}  // namespace tfs
