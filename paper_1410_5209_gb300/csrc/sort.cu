// Device construction of the per-mode sorted layout: the slices Omega_i^(n) of the
// paper's table of symbols, with bit-exact row offsets.
//
// Each mode n gets the permutation of the observed entries that orders them
// lexicographically by (i_n, i_{n+1}, ..., i_N, i_1, ..., i_{n-1}); with no duplicate
// coordinates this order is total, so the permutation is unique.  The first mode's is
// produced by stable least-significant-digit radix sorts (8-bit digits) over the modes
// from the least to the most significant, with the entry permutation as payload; every
// other mode's by one stable sort by its own index of the following mode's permutation
// (the layout build in api.cu).  Every pass
// is "count per tile -> one exclusive scan over (digit, tile) -> stable scatter", the
// stable in-tile rank coming from warp match/popc over 32 consecutive keys at a time.
#include "common.cuh"

namespace tfs {
namespace {

constexpr int kSortThreads = 256;
constexpr int kSortItems = 16;  // keys per thread per tile
constexpr int kTile = kSortThreads * kSortItems;
constexpr int kDigits = 256;
constexpr int kDigitBits = 8;
constexpr int kScanThreads = 1024;
constexpr int kScanItems = 4;
constexpr int kScanTile = kScanThreads * kScanItems;

__global__ void __launch_bounds__(kSortThreads) k_radix_hist(const uint32_t *__restrict__ kin,
                                                             int64_t n, int shift,
                                                             uint32_t *__restrict__ hist,
                                                             int64_t ntiles) {
    __shared__ uint32_t cnt[kDigits];
    cnt[threadIdx.x] = 0;
    __syncthreads();
    const int64_t base = (int64_t)blockIdx.x * kTile;
    for (int i = threadIdx.x; i < kTile; i += kSortThreads) {
        int64_t idx = base + i;
        if (idx < n) atomicAdd(&cnt[(kin[idx] >> shift) & (kDigits - 1)], 1u);
    }
    __syncthreads();
    hist[(int64_t)threadIdx.x * ntiles + blockIdx.x] = cnt[threadIdx.x];
}

__global__ void __launch_bounds__(kSortThreads) k_radix_scatter(
    const uint32_t *__restrict__ kin, const int32_t *__restrict__ vin,
    uint32_t *__restrict__ kout, int32_t *__restrict__ vout, int64_t n, int shift,
    const uint32_t *__restrict__ hist_scanned, int64_t ntiles) {
    constexpr int kWarps = kSortThreads / kWarp;
    __shared__ uint32_t wcnt[kWarps][kDigits];
    __shared__ uint32_t gbase[kDigits];
    __shared__ uint32_t tstart[kDigits];   // tile-local start of each digit's run
    __shared__ uint32_t wsum[kWarps];
    __shared__ uint32_t skey[kTile];
    __shared__ int32_t sval[kTile];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int w = 0; w < kWarps; ++w) wcnt[w][threadIdx.x] = 0;
    gbase[threadIdx.x] = hist_scanned[(int64_t)threadIdx.x * ntiles + blockIdx.x];
    __syncthreads();

    const uint32_t lt_mask = (1u << lane) - 1u;
    const int64_t tile0 = (int64_t)blockIdx.x * kTile;
    const int64_t base = tile0 + (int64_t)warp * (kTile / kWarps);
    uint32_t key[kSortItems], loc[kSortItems];
    int32_t val[kSortItems];
#pragma unroll
    for (int r = 0; r < kSortItems; ++r) {
        const int64_t idx = base + r * kWarp + lane;
        const bool valid = idx < n;
        key[r] = valid ? kin[idx] : 0u;
        val[r] = valid ? vin[idx] : 0;
        const uint32_t d = valid ? ((key[r] >> shift) & (kDigits - 1)) : 0xFFFFFFFFu;
        const uint32_t peers = __match_any_sync(0xFFFFFFFFu, d);
        const uint32_t rank = __popc(peers & lt_mask);
        loc[r] = valid ? wcnt[warp][valid ? d : 0u] + rank : 0u;
        __syncwarp();
        if (valid && rank == 0) wcnt[warp][d] += __popc(peers);
        __syncwarp();
    }
    __syncthreads();
    uint32_t total;
    {  // exclusive prefix over warps, per digit (thread = digit)
        uint32_t run = 0;
        for (int w = 0; w < kWarps; ++w) {
            uint32_t t = wcnt[w][threadIdx.x];
            wcnt[w][threadIdx.x] = run;
            run += t;
        }
        total = run;
    }
    {  // exclusive prefix over digits of the tile's counts
        uint32_t incl = total;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t t = __shfl_up_sync(0xFFFFFFFFu, incl, o);
            if (lane >= o) incl += t;
        }
        if (lane == 31) wsum[warp] = incl;
        __syncthreads();
        uint32_t before = 0;
        for (int w = 0; w < warp; ++w) before += wsum[w];
        tstart[threadIdx.x] = before + incl - total;
    }
    __syncthreads();
    // local order: keys grouped by digit inside the tile (stable), then written out in
    // that order, so consecutive threads write consecutive positions of a digit's run
#pragma unroll
    for (int r = 0; r < kSortItems; ++r) {
        const int64_t idx = base + r * kWarp + lane;
        if (idx < n) {
            const uint32_t d = (key[r] >> shift) & (kDigits - 1);
            const uint32_t lp = tstart[d] + wcnt[warp][d] + loc[r];
            skey[lp] = key[r];
            sval[lp] = val[r];
        }
    }
    __syncthreads();
    const int tile_n = (int)(n - tile0 < kTile ? n - tile0 : kTile);
    for (int i = threadIdx.x; i < tile_n; i += kSortThreads) {
        const uint32_t k = skey[i];
        const uint32_t d = (k >> shift) & (kDigits - 1);
        const uint32_t dst = gbase[d] + (uint32_t)i - tstart[d];
        kout[dst] = k;
        vout[dst] = sval[i];
    }
}

// Exclusive scan of one tile per block; writes the tile total to sums[blockIdx.x].
__global__ void __launch_bounds__(kScanThreads) k_scan_tile(const uint32_t *in, uint32_t *out,
                                                            int64_t n, uint32_t *sums) {
    __shared__ uint32_t warp_tot[kScanThreads / kWarp];
    const int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanItems;
    uint32_t v[kScanItems];
    uint32_t tsum = 0;
#pragma unroll
    for (int i = 0; i < kScanItems; ++i) {
        v[i] = (base + i < n) ? in[base + i] : 0u;
        tsum += v[i];
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t incl = tsum;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        uint32_t t = __shfl_up_sync(0xFFFFFFFFu, incl, o);
        if (lane >= o) incl += t;
    }
    if (lane == 31) warp_tot[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        uint32_t w = (lane < kScanThreads / kWarp) ? warp_tot[lane] : 0u;
        uint32_t wi = w;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            uint32_t t = __shfl_up_sync(0xFFFFFFFFu, wi, o);
            if (lane >= o) wi += t;
        }
        if (lane < kScanThreads / kWarp) warp_tot[lane] = wi - w;  // exclusive
        if (lane == kScanThreads / kWarp - 1 && sums) sums[blockIdx.x] = wi;
    }
    __syncthreads();
    uint32_t run = warp_tot[warp] + incl - tsum;
#pragma unroll
    for (int i = 0; i < kScanItems; ++i) {
        if (base + i < n) out[base + i] = run;
        run += v[i];
    }
}

__global__ void k_scan_add(uint32_t *out, int64_t n, const uint32_t *offs) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] += offs[i / kScanTile];
}

__global__ void k_transpose_check(const int32_t *__restrict__ coords, int N, int64_t nnz,
                                  const int64_t *__restrict__ dims, int32_t *__restrict__ soa,
                                  DeviceStatus *stat) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= nnz) return;
    int bad = 0;
    for (int m = 0; m < N; ++m) {
        int32_t v = coords[e * N + m];
        if (v < 0 || (int64_t)v >= dims[m]) {
            bad = 1;
            v = 0;
        }
        soa[(int64_t)m * nnz + e] = v;
    }
    if (bad) atomicOr(&stat->bits, kStatRange);
}

__global__ void k_iota(int32_t *p, int64_t n) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) p[i] = (int32_t)i;
}

__global__ void k_gather_keys(const int32_t *__restrict__ col, const int32_t *__restrict__ perm,
                              uint32_t *__restrict__ keys, int64_t n) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) keys[i] = (uint32_t)col[perm[i]];
}

__global__ void k_gather_rank(const int32_t *__restrict__ col, const int32_t *__restrict__ perm,
                              const int32_t *__restrict__ rank, int32_t *__restrict__ out,
                              int64_t n) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = rank[col[perm[i]]];
}

// off[i] = first sorted position whose key is >= i, for i in 0..I (so off[I] = n).
__global__ void k_offsets(const uint32_t *__restrict__ keys, int64_t n, int64_t I,
                          int64_t *__restrict__ off) {
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j > n) return;
    const int64_t kprev = (j == 0) ? -1 : (int64_t)keys[j - 1];
    const int64_t kcur = (j == n) ? I : (int64_t)keys[j];
    for (int64_t i = kprev + 1; i <= kcur; ++i) off[i] = j;
}

__global__ void k_dup_check(const int32_t *__restrict__ soa, int N, int64_t nnz,
                            const int32_t *__restrict__ perm, DeviceStatus *stat) {
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x + 1;
    if (j >= nnz) return;
    const int32_t a = perm[j], b = perm[j - 1];
    for (int m = 0; m < N; ++m)
        if (soa[(int64_t)m * nnz + a] != soa[(int64_t)m * nnz + b]) return;
    atomicOr(&stat->bits, kStatDup);
}

inline unsigned grid_for(int64_t n, int threads) {
    return (unsigned)ceil_div<int64_t>(n > 0 ? n : 1, threads);
}

}  // namespace

size_t scan_temp_elems(int64_t n) {
    size_t total = 0;
    while (n > 1) {
        n = ceil_div<int64_t>(n, kScanTile);
        total += (size_t)n + 32;
    }
    return total + 32;
}

void scan_exclusive_u32(const uint32_t *in, uint32_t *out, int64_t n, uint32_t *tmp,
                        cudaStream_t st) {
    if (n <= 0) return;
    const int64_t nb = ceil_div<int64_t>(n, kScanTile);
    k_scan_tile<<<(unsigned)nb, kScanThreads, 0, st>>>(in, out, n, nb > 1 ? tmp : nullptr);
    TFS_CUDA(cudaGetLastError());
    if (nb > 1) {
        scan_exclusive_u32(tmp, tmp, nb, tmp + nb + 32, st);
        k_scan_add<<<grid_for(n, 256), 256, 0, st>>>(out, n, tmp);
        TFS_CUDA(cudaGetLastError());
    }
}

void SortWorkspace::reserve(int64_t n, cudaStream_t st) {
    const size_t items = (size_t)(n > 0 ? n : 1);
    const size_t ntiles = (size_t)ceil_div<int64_t>(n > 0 ? n : 1, kTile);
    const size_t hist = ntiles * kDigits;
    const size_t scan = scan_temp_elems((int64_t)hist);
    auto regrow = [&](auto *&p, size_t &cap, size_t want) {
        if (want <= cap) return;
        if (p) cudaFreeAsync(p, st);
        p = nullptr;
        cap = 0;
        TFS_CUDA(pool_alloc(reinterpret_cast<void **>(&p), want * sizeof(*p), st));
        cap = want;
    };
    size_t cap_vals = cap_items;
    regrow(keys_alt, cap_items, items);
    regrow(vals_alt, cap_vals, items);
    regrow(this->hist, cap_hist, hist);
    regrow(scan_tmp, cap_scan, scan);
}

size_t sort_workspace_bytes(int64_t n) {
    const size_t items = (size_t)(n > 0 ? n : 1);
    const size_t hist = (size_t)ceil_div<int64_t>(n > 0 ? n : 1, kTile) * kDigits;
    return items * (sizeof(uint32_t) + sizeof(int32_t)) +
           (hist + scan_temp_elems((int64_t)hist)) * sizeof(uint32_t);
}

void SortWorkspace::release(cudaStream_t st) {
    if (keys_alt) cudaFreeAsync(keys_alt, st);
    if (vals_alt) cudaFreeAsync(vals_alt, st);
    if (hist) cudaFreeAsync(hist, st);
    if (scan_tmp) cudaFreeAsync(scan_tmp, st);
    keys_alt = nullptr;
    vals_alt = nullptr;
    hist = nullptr;
    scan_tmp = nullptr;
    cap_items = cap_hist = cap_scan = 0;
}

void radix_sort_pairs(uint32_t *keys, int32_t *vals, int64_t n, int bits, SortWorkspace &ws,
                      cudaStream_t st) {
    if (n <= 1 || bits <= 0) return;
    ws.reserve(n, st);
    const int64_t ntiles = ceil_div<int64_t>(n, kTile);
    uint32_t *kin = keys, *kout = ws.keys_alt;
    int32_t *vin = vals, *vout = ws.vals_alt;
    int passes = 0;
    for (int shift = 0; shift < bits; shift += kDigitBits, ++passes) {
        k_radix_hist<<<(unsigned)ntiles, kSortThreads, 0, st>>>(kin, n, shift, ws.hist, ntiles);
        TFS_CUDA(cudaGetLastError());
        scan_exclusive_u32(ws.hist, ws.hist, ntiles * kDigits, ws.scan_tmp, st);
        k_radix_scatter<<<(unsigned)ntiles, kSortThreads, 0, st>>>(kin, vin, kout, vout, n, shift,
                                                                   ws.hist, ntiles);
        TFS_CUDA(cudaGetLastError());
        std::swap(kin, kout);
        std::swap(vin, vout);
    }
    if (passes & 1) {  // result sits in the workspace: copy back
        TFS_CUDA(cudaMemcpyAsync(keys, kin, n * sizeof(uint32_t), cudaMemcpyDeviceToDevice, st));
        TFS_CUDA(cudaMemcpyAsync(vals, vin, n * sizeof(int32_t), cudaMemcpyDeviceToDevice, st));
    }
}

void launch_transpose_check(const int32_t *coords, int N, int64_t nnz, const int64_t *dims_dev,
                            int32_t *soa, DeviceStatus *stat, cudaStream_t st) {
    if (nnz <= 0) return;
    k_transpose_check<<<grid_for(nnz, 256), 256, 0, st>>>(coords, N, nnz, dims_dev, soa, stat);
    TFS_CUDA(cudaGetLastError());
}

void launch_iota(int32_t *p, int64_t n, cudaStream_t st) {
    if (n <= 0) return;
    k_iota<<<grid_for(n, 256), 256, 0, st>>>(p, n);
    TFS_CUDA(cudaGetLastError());
}

void launch_gather_keys(const int32_t *col, const int32_t *perm, uint32_t *keys, int64_t n,
                        cudaStream_t st) {
    if (n <= 0) return;
    k_gather_keys<<<grid_for(n, 256), 256, 0, st>>>(col, perm, keys, n);
    TFS_CUDA(cudaGetLastError());
}

void launch_gather_rank(const int32_t *col, const int32_t *perm, const int32_t *rank, int32_t *out,
                        int64_t n, cudaStream_t st) {
    if (n <= 0) return;
    k_gather_rank<<<grid_for(n, 256), 256, 0, st>>>(col, perm, rank, out, n);
    TFS_CUDA(cudaGetLastError());
}

void launch_offsets(const uint32_t *keys, int64_t n, int64_t I, int64_t *off, cudaStream_t st) {
    k_offsets<<<grid_for(n + 1, 256), 256, 0, st>>>(keys, n, I, off);
    TFS_CUDA(cudaGetLastError());
}

void launch_dup_check(const int32_t *soa, int N, int64_t nnz, const int32_t *perm,
                      DeviceStatus *stat, cudaStream_t st) {
    if (nnz <= 1) return;
    k_dup_check<<<grid_for(nnz - 1, 256), 256, 0, st>>>(soa, N, nnz, perm, stat);
    TFS_CUDA(cudaGetLastError());
}

}  // namespace tfs
