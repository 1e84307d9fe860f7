// Packed-key construction of the per-mode sorted layout (the slices Omega_i^(n) of the
// paper's table of symbols) for tensors whose coordinates fit one 64-bit word together:
// sum over modes of ceil(log2 I_m) <= 64.
//
// Every entry's coordinates are packed once into a key, mode 0 in the most significant
// bits, mode N-1 in the least.  Mode 0's order, lexicographic in (i_0, ..., i_{N-1}),
// is one stable LSD radix sort of the whole key; mode n's order, lexicographic in
// (i_n, i_{n+1}, ..., i_{n-1}), is one stable sort by the field i_n of mode n+1's
// sorted keys (equal i_n keep mode n+1's order, which is the rest of mode n's key).
// The keys travel with the entry permutation through the passes, so no pass gathers a
// coordinate by the permutation, the duplicate check compares neighbouring keys, and
// the other modes' indices of every sorted position come from its own key.  The row
// counts of every mode are taken in the packing pass, before any sort, so the host can
// rank rows by degree and schedule them while the device sorts.
#include "common.cuh"
#include "layout.cuh"

namespace tfs {
namespace {

// ------------------------------------------------------------------ pack + count

constexpr int kPackThreads = 512;
constexpr int kPackItems = 16;
constexpr int kPackTile = kPackThreads * kPackItems;
constexpr int kHashBits = 13;
constexpr int kHash = 1 << kHashBits;  // shared-memory count slots per block and mode
constexpr int kHashProbes = 16;

__device__ __forceinline__ int32_t key_field(uint64_t key, int shift, int bits) {
    return (int32_t)((key >> shift) & ((uint64_t(1) << bits) - 1));
}

// One tile of entries per block: range check and key of every entry (coordinates out
// of range count as 0 and set kStatRange), then, mode by mode, the tile's row counts
// summed in shared memory and added to the global counts.  Rows of a mode with at
// most kHash rows index the shared array directly; longer modes go through an
// open-addressing table (linear probing, bounded), whose misses add to the global
// count directly.  A hot row (the skewed modes' heaviest rows hold a tenth of the
// entries) so costs one global atomic per block instead of one per entry.
__global__ void __launch_bounds__(kPackThreads) k_pack_count(const int32_t *__restrict__ coords,
                                                             int64_t e0, int64_t ne,
                                                             const KeyFields f,
                                                             uint64_t *__restrict__ keys,
                                                             uint32_t *__restrict__ counts,
                                                             DeviceStatus *stat) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    int32_t *hkey = reinterpret_cast<int32_t *>(smem_raw);
    uint32_t *hcnt = reinterpret_cast<uint32_t *>(hkey + kHash);
    const int64_t tile0 = (int64_t)blockIdx.x * kPackTile;
    uint64_t key[kPackItems];
    int bad = 0;
#pragma unroll
    for (int r = 0; r < kPackItems; ++r) {
        const int64_t e = tile0 + (int64_t)r * kPackThreads + threadIdx.x;
        uint64_t k = 0;
        if (e < ne) {
            for (int m = 0; m < f.N; ++m) {
                int32_t v = coords[e * f.N + m];
                if (v < 0 || (int64_t)v >= f.dims[m]) {
                    bad = 1;
                    v = 0;
                }
                k |= (uint64_t)(uint32_t)v << f.shift[m];
            }
            keys[e0 + e] = k;
        }
        key[r] = k;
    }
    if (bad) atomicOr(&stat->bits, kStatRange);

    for (int m = 0; m < f.N; ++m) {
        const bool direct = f.dims[m] <= kHash;
        const int slots = direct ? (int)f.dims[m] : kHash;
        uint32_t *gcnt = counts + f.cnt_off[m];
        for (int s = threadIdx.x; s < slots; s += kPackThreads) {
            hkey[s] = -1;
            hcnt[s] = 0;
        }
        __syncthreads();
#pragma unroll
        for (int r = 0; r < kPackItems; ++r) {
            const int64_t e = tile0 + (int64_t)r * kPackThreads + threadIdx.x;
            if (e >= ne) continue;
            const int32_t row = key_field(key[r], f.shift[m], f.bits[m]);
            if (direct) {
                atomicAdd(&hcnt[row], 1u);
                continue;
            }
            uint32_t h = ((uint32_t)row * 2654435761u) >> (32 - kHashBits);
            bool done = false;
            for (int p = 0; p < kHashProbes && !done; ++p) {
                int32_t k = reinterpret_cast<volatile int32_t *>(hkey)[h];
                if (k == -1) k = atomicCAS(&hkey[h], -1, row);
                if (k == -1 || k == row) {
                    atomicAdd(&hcnt[h], 1u);
                    done = true;
                }
                h = (h + 1) & (kHash - 1);
            }
            if (!done) atomicAdd(&gcnt[row], 1u);
        }
        __syncthreads();
        for (int s = threadIdx.x; s < slots; s += kPackThreads) {
            const uint32_t c = hcnt[s];
            if (c != 0) atomicAdd(&gcnt[direct ? s : hkey[s]], c);
        }
        __syncthreads();
    }
}

// ------------------------------------------------------------------ 64-bit key sort

constexpr int kSortThreads = 512;
constexpr int kSortItems = 8;
constexpr int kTile = kSortThreads * kSortItems;  // keys per tile
constexpr int kSortWarps = kSortThreads / kWarp;
constexpr int kMaxDigitBits = 10;

// Per-tile digit counts, hist[d * ntiles + tile] (digit-major, so one exclusive scan
// gives every (digit, tile) its first output position).  A block counts kHistTiles
// consecutive tiles, so each digit's counts of those tiles go out as one run of
// consecutive words (whole 32-byte sectors instead of one partial sector per count).
constexpr int kHistTiles = 8;

template <int DB>
__global__ void __launch_bounds__(kSortThreads) k_hist64(const uint64_t *__restrict__ kin,
                                                         int64_t n, int shift, int width,
                                                         uint32_t *__restrict__ hist,
                                                         int64_t ntiles) {
    __shared__ uint32_t cnt[kHistTiles << DB];  // [tile][digit]
    const int nb = 1 << width;
    for (int i = threadIdx.x; i < (kHistTiles << DB); i += kSortThreads) cnt[i] = 0;
    __syncthreads();
    const int64_t t0 = (int64_t)blockIdx.x * kHistTiles;
    const int nt = (int)(ntiles - t0 < kHistTiles ? ntiles - t0 : kHistTiles);
    for (int t = 0; t < nt; ++t) {
        const int64_t base = (t0 + t) * kTile;
        uint32_t *c = cnt + (t << DB);
#pragma unroll
        for (int r = 0; r < kSortItems; ++r) {
            const int64_t idx = base + (int64_t)r * kSortThreads + threadIdx.x;
            if (idx < n) atomicAdd(&c[(kin[idx] >> shift) & (uint64_t)(nb - 1)], 1u);
        }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < nb * kHistTiles; i += kSortThreads) {
        const int d = i / kHistTiles, t = i - d * kHistTiles;
        if (t < nt) hist[(int64_t)d * ntiles + t0 + t] = cnt[(t << DB) + d];
    }
}

// Second payload carried with the keys: none, 4-byte or 8-byte words.
template <int XB>
struct XWord {
    using type = uint32_t;
};
template <>
struct XWord<8> {
    using type = uint64_t;
};

// Shared memory of one scatter block: the warps' 16-bit digit counters, later reused as
// the tile's staging area (keys, permutation, payload), then the tile's digit bases.
template <int DB, int XB>
struct ScatterLayout {
    static constexpr bool kRecords = XB == 4;  // staged as one 16-byte record per key
    static constexpr int kCounters = kSortWarps * (1 << DB) * 2;
    static constexpr int kStaging = kRecords ? kTile * 16 : kTile * (8 + 4 + XB);
    static constexpr int kRegion = kCounters > kStaging ? kCounters : kStaging;
    static constexpr int kBytes = kRegion + 2 * (1 << DB) * 4 + kSortWarps * 4;
};

// Stable scatter of one tile of 4096 keys.  Each warp ranks its 256 consecutive keys
// 32 at a time (match of equal digits, 16-bit per-warp counters), a per-digit prefix over
// the warps and a block scan over the digits give every key its place in the tile
// regrouped by digit, the tile is staged in that order (over the counters, no longer
// needed) and written out run by run at the digit's global base.  vin == nullptr stands
// for the identity permutation; XB > 0 carries xin along.
template <int DB, int XB>
__global__ void __launch_bounds__(kSortThreads, 2) k_scatter64(
    const uint64_t *__restrict__ kin, const int32_t *__restrict__ vin,
    const typename XWord<XB>::type *__restrict__ xin, uint64_t *__restrict__ kout,
    int32_t *__restrict__ vout, typename XWord<XB>::type *__restrict__ xout, int64_t n,
    int shift, int width, const uint32_t *__restrict__ hist_scanned, int64_t ntiles) {
    using XT = typename XWord<XB>::type;
    using L = ScatterLayout<DB, XB>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    uint16_t *wcnt = reinterpret_cast<uint16_t *>(smem_raw);  // [warp][digit]
    uint64_t *skey = reinterpret_cast<uint64_t *>(smem_raw);
    int32_t *sval = reinterpret_cast<int32_t *>(skey + kTile);
    XT *sx = reinterpret_cast<XT *>(sval + kTile);
    uint32_t *gbase = reinterpret_cast<uint32_t *>(smem_raw + L::kRegion);
    uint32_t *tstart = gbase + (1 << DB);
    uint32_t *wsum = tstart + (1 << DB);

    const int nb = 1 << width;
    const uint64_t dmask = (uint64_t)(nb - 1);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int i = threadIdx.x; i < kSortWarps * nb; i += kSortThreads) wcnt[i] = 0;
    for (int d = threadIdx.x; d < nb; d += kSortThreads)
        gbase[d] = hist_scanned[(int64_t)d * ntiles + blockIdx.x];

    const int64_t tile0 = (int64_t)blockIdx.x * kTile;
    const int64_t base = tile0 + (int64_t)warp * (kTile / kSortWarps);
    uint64_t key[kSortItems];
    int32_t val[kSortItems];
    XT xv[kSortItems];
    uint32_t loc[kSortItems];
#pragma unroll
    for (int r = 0; r < kSortItems; ++r) {
        const int64_t idx = base + r * kWarp + lane;
        const bool valid = idx < n;
        key[r] = valid ? kin[idx] : 0ull;
        val[r] = valid ? (vin ? vin[idx] : (int32_t)idx) : 0;
        if (XB > 0) xv[r] = valid ? xin[idx] : XT(0);
    }
    __syncthreads();
    const uint32_t lt_mask = (1u << lane) - 1u;
    uint16_t *mycnt = wcnt + warp * nb;
#pragma unroll
    for (int r = 0; r < kSortItems; ++r) {
        const bool valid = base + r * kWarp + lane < n;
        const int32_t d = valid ? (int32_t)((key[r] >> shift) & dmask) : -1;
        const uint32_t peers = __match_any_sync(0xFFFFFFFFu, d);
        const uint32_t rank = __popc(peers & lt_mask);
        loc[r] = valid ? (uint32_t)mycnt[d] + rank : 0u;
        __syncwarp();
        if (valid && rank == 0) mycnt[d] = (uint16_t)(mycnt[d] + __popc(peers));
        __syncwarp();
    }
    __syncthreads();
    // per digit: the warps' exclusive offsets and the tile total; each thread takes a
    // contiguous range of digits, then a block scan of the ranges' totals
    const int per = (nb + kSortThreads - 1) / kSortThreads;
    const int d0 = threadIdx.x * per;
    uint32_t mine = 0;
    for (int d = d0; d < d0 + per && d < nb; ++d) {
        uint32_t run = 0;
        for (int w = 0; w < kSortWarps; ++w) {
            const uint32_t t = wcnt[w * nb + d];
            wcnt[w * nb + d] = (uint16_t)run;
            run += t;
        }
        tstart[d] = run;  // the digit's total for now
        mine += run;
    }
    uint32_t incl = mine;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t t = __shfl_up_sync(0xFFFFFFFFu, incl, o);
        if (lane >= o) incl += t;
    }
    if (lane == 31) wsum[warp] = incl;
    __syncthreads();
    uint32_t before = 0;
    for (int w = 0; w < warp; ++w) before += wsum[w];
    uint32_t at = before + incl - mine;
    for (int d = d0; d < d0 + per && d < nb; ++d) {
        const uint32_t tot = tstart[d];
        tstart[d] = at;
        at += tot;
    }
    __syncthreads();
#pragma unroll
    for (int r = 0; r < kSortItems; ++r) {
        const uint32_t d = (uint32_t)((key[r] >> shift) & dmask);
        if (base + r * kWarp + lane < n) loc[r] += tstart[d] + mycnt[d];
    }
    __syncthreads();  // the counters are dead: the staging area takes their place
    // one base per digit from here on: the output position of tile position i is
    // gbase[d] - tstart[d] + i (modulo 2^32)
    for (int d = threadIdx.x; d < nb; d += kSortThreads) gbase[d] -= tstart[d];
    const unsigned stage_s = (unsigned)__cvta_generic_to_shared(smem_raw);
#pragma unroll
    for (int r = 0; r < kSortItems; ++r) {
        if (base + r * kWarp + lane < n) {
            if constexpr (L::kRecords) {
                const uint32_t xw = XB > 0 ? (uint32_t)xv[r] : 0u;
                asm volatile("st.shared.v4.b32 [%0], {%1, %2, %3, %4};" ::"r"(stage_s + 16u * loc[r]),
                             "r"((uint32_t)key[r]), "r"((uint32_t)(key[r] >> 32)),
                             "r"((uint32_t)val[r]), "r"(xw)
                             : "memory");
            } else {
                skey[loc[r]] = key[r];
                sval[loc[r]] = val[r];
                if constexpr (XB > 0) sx[loc[r]] = xv[r];
            }
        }
    }
    __syncthreads();
    const int tile_n = (int)(n - tile0 < kTile ? n - tile0 : kTile);
    for (int i = threadIdx.x; i < tile_n; i += kSortThreads) {
        uint64_t k;
        int32_t v;
        XT xw = XT(0);
        if constexpr (L::kRecords) {
            uint32_t w0, w1, w2, w3;
            asm volatile("ld.shared.v4.b32 {%0, %1, %2, %3}, [%4];"
                         : "=r"(w0), "=r"(w1), "=r"(w2), "=r"(w3)
                         : "r"(stage_s + 16u * (unsigned)i));
            k = (uint64_t)w0 | ((uint64_t)w1 << 32);
            v = (int32_t)w2;
            xw = (XT)w3;
        } else {
            k = skey[i];
            v = sval[i];
            if constexpr (XB > 0) xw = sx[i];
        }
        const uint32_t d = (uint32_t)((k >> shift) & dmask);
        const uint32_t dst = gbase[d] + (uint32_t)i;
        kout[dst] = k;
        vout[dst] = v;
        if (XB > 0) xout[dst] = xw;
    }
}

__global__ void k_iota32(int32_t *p, int64_t n) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) p[i] = (int32_t)i;
}

// ------------------------------------------------------------------ extraction

// Mode n's other-mode slice rows from its sorted keys, for the first mode the
// duplicate check (equal neighbouring keys), and where the values did not travel with
// the keys, the residual copy res[j] = x[perm[j]] (R = X at the start).
template <class XT>
__global__ void k_extract(const uint64_t *__restrict__ keys, int64_t nnz, const ExtractArgs a,
                          DeviceStatus *stat) {
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= nnz) return;
    const uint64_t key = keys[j];
    if (a.x) static_cast<XT *>(a.res)[j] = static_cast<const XT *>(a.x)[a.perm[j]];
    for (int t = 0; t < a.n_other; ++t)
        a.oidx[t][j] = a.rank[t][key_field(key, a.shift[t], a.bits[t])];
    if (a.check_dup && j > 0 && keys[j - 1] == key) atomicOr(&stat->bits, kStatDup);
}

inline unsigned grid_for(int64_t n, int threads) {
    return (unsigned)ceil_div<int64_t>(n > 0 ? n : 1, threads);
}

template <int DB, int XB>
void sort_pass(const uint64_t *kin, const int32_t *vin, const void *xin, uint64_t *kout,
               int32_t *vout, void *xout, int64_t n, int shift, int width, KeySortWorkspace &ws,
               cudaStream_t st) {
    using XT = typename XWord<XB>::type;
    const int64_t ntiles = ceil_div<int64_t>(n, kTile);
    const int64_t hn = ntiles << width;
    k_hist64<DB><<<(unsigned)ceil_div<int64_t>(ntiles, kHistTiles), kSortThreads, 0, st>>>(
        kin, n, shift, width, ws.hist, ntiles);
    TFS_CUDA(cudaGetLastError());
    scan_exclusive_u32(ws.hist, ws.hist, hn, ws.scan_tmp, st);
    const int smem = ScatterLayout<DB, XB>::kBytes;
    TFS_CUDA(raise_smem_limit((const void *)k_scatter64<DB, XB>, smem));
    k_scatter64<DB, XB><<<(unsigned)ntiles, kSortThreads, smem, st>>>(
        kin, vin, static_cast<const XT *>(xin), kout, vout, static_cast<XT *>(xout), n, shift,
        width, ws.hist, ntiles);
    TFS_CUDA(cudaGetLastError());
}

template <int XB>
void sort_pass_w(const uint64_t *kin, const int32_t *vin, const void *xin, uint64_t *kout,
                 int32_t *vout, void *xout, int64_t n, int shift, int width, KeySortWorkspace &ws,
                 cudaStream_t st) {
    if (width <= 8)
        sort_pass<8, XB>(kin, vin, xin, kout, vout, xout, n, shift, width, ws, st);
    else
        sort_pass<kMaxDigitBits, XB>(kin, vin, xin, kout, vout, xout, n, shift, width, ws, st);
}

}  // namespace

int packed_key_bits(const int64_t *dims, int N) {
    int b = 0;
    for (int m = 0; m < N; ++m) b += ceil_log2_u64((uint64_t)dims[m]);
    return b;
}

KeyFields key_fields(const int64_t *dims, int N) {
    KeyFields f{};
    f.N = N;
    int shift = 0;
    int64_t off = 0;
    for (int m = N - 1; m >= 0; --m) {
        f.bits[m] = ceil_log2_u64((uint64_t)dims[m]);
        f.shift[m] = shift;
        shift += f.bits[m];
    }
    for (int m = 0; m < N; ++m) {
        f.dims[m] = dims[m];
        f.cnt_off[m] = off;
        off += dims[m];
    }
    return f;
}

void KeySortWorkspace::reserve(int64_t n, cudaStream_t st) {
    const size_t hist_n = (size_t)ceil_div<int64_t>(n > 0 ? n : 1, kTile) << kMaxDigitBits;
    const size_t scan_n = scan_temp_elems((int64_t)hist_n);
    if (hist_n > cap_hist) {
        if (hist) cudaFreeAsync(hist, st);
        hist = nullptr;
        cap_hist = 0;
        TFS_CUDA(pool_alloc(reinterpret_cast<void **>(&hist), hist_n * sizeof(uint32_t), st));
        cap_hist = hist_n;
    }
    if (scan_n > cap_scan) {
        if (scan_tmp) cudaFreeAsync(scan_tmp, st);
        scan_tmp = nullptr;
        cap_scan = 0;
        TFS_CUDA(pool_alloc(reinterpret_cast<void **>(&scan_tmp), scan_n * sizeof(uint32_t), st));
        cap_scan = scan_n;
    }
}

void KeySortWorkspace::release(cudaStream_t st) {
    if (hist) cudaFreeAsync(hist, st);
    if (scan_tmp) cudaFreeAsync(scan_tmp, st);
    hist = nullptr;
    scan_tmp = nullptr;
    cap_hist = cap_scan = 0;
}

size_t key_sort_workspace_bytes(int64_t n) {
    const size_t hist_n = (size_t)ceil_div<int64_t>(n > 0 ? n : 1, kTile) << kMaxDigitBits;
    return (hist_n + scan_temp_elems((int64_t)hist_n)) * sizeof(uint32_t);
}

int64_t pack_count_tile() { return kPackTile; }

void launch_pack_count(const int32_t *coords, int64_t e0, int64_t ne, const KeyFields &f,
                       uint64_t *keys, uint32_t *counts, DeviceStatus *stat, cudaStream_t st) {
    if (ne <= 0) return;
    const int smem = kHash * (int)(sizeof(int32_t) + sizeof(uint32_t));
    TFS_CUDA(raise_smem_limit((const void *)k_pack_count, smem));
    k_pack_count<<<grid_for(ne, kPackTile), kPackThreads, smem, st>>>(coords, e0, ne, f, keys,
                                                                     counts, stat);
    TFS_CUDA(cudaGetLastError());
}

void radix_sort_keys64(const uint64_t *kin, const int32_t *vin, const void *xin, uint64_t *kout,
                       int32_t *vout, void *xout, uint64_t *kalt, int32_t *valt, void *xalt,
                       int xbytes, int64_t n, int lo_bit, int hi_bit, KeySortWorkspace &ws,
                       cudaStream_t st) {
    if (n <= 0) return;
    if (xbytes != 0 && xbytes != 4 && xbytes != 8)
        throw ApiError{TF_EINVAL, "sort payload must be 0, 4 or 8 bytes"};
    const int bits = hi_bit - lo_bit;
    if (bits <= 0 || n == 1) {  // nothing to order: the input as it is
        TFS_CUDA(cudaMemcpyAsync(kout, kin, n * sizeof(uint64_t), cudaMemcpyDeviceToDevice, st));
        if (vin)
            TFS_CUDA(cudaMemcpyAsync(vout, vin, n * sizeof(int32_t), cudaMemcpyDeviceToDevice, st));
        else {
            k_iota32<<<grid_for(n, 256), 256, 0, st>>>(vout, n);
            TFS_CUDA(cudaGetLastError());
        }
        if (xbytes)
            TFS_CUDA(cudaMemcpyAsync(xout, xin, (size_t)n * xbytes, cudaMemcpyDeviceToDevice, st));
        return;
    }
    ws.reserve(n, st);
    const int passes = ceil_div(bits, kMaxDigitBits);
    // pass p writes the outputs when (passes - 1 - p) is even, the alternate buffers
    // otherwise, so the last pass lands in the outputs and no pass writes the input
    const uint64_t *ki = kin;
    const int32_t *vi = vin;
    const void *xi = xin;
    int lo = lo_bit;
    for (int p = 0; p < passes; ++p) {
        const int width = (bits - (lo - lo_bit) + (passes - p) - 1) / (passes - p);
        const bool to_out = ((passes - 1 - p) & 1) == 0;
        uint64_t *ko = to_out ? kout : kalt;
        int32_t *vo = to_out ? vout : valt;
        void *xo = to_out ? xout : xalt;
        if (xbytes == 0)
            sort_pass_w<0>(ki, vi, nullptr, ko, vo, nullptr, n, lo, width, ws, st);
        else if (xbytes == 4)
            sort_pass_w<4>(ki, vi, xi, ko, vo, xo, n, lo, width, ws, st);
        else
            sort_pass_w<8>(ki, vi, xi, ko, vo, xo, n, lo, width, ws, st);
        ki = ko;
        vi = vo;
        xi = xo;
        lo += width;
    }
}

void launch_extract(const uint64_t *keys, int64_t nnz, const ExtractArgs &a, DeviceStatus *stat,
                    cudaStream_t st) {
    if (nnz <= 0) return;
    if (a.x && a.xbytes == 8)
        k_extract<uint64_t><<<grid_for(nnz, 256), 256, 0, st>>>(keys, nnz, a, stat);
    else
        k_extract<uint32_t><<<grid_for(nnz, 256), 256, 0, st>>>(keys, nnz, a, stat);
    TFS_CUDA(cudaGetLastError());
}

}  // namespace tfs
