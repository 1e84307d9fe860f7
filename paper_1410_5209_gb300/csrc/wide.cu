// Mode pass, row solves and residual reductions for wide column subsets (16 < C < 128),
// where per-lane Gram accumulators no longer fit in registers.
//
// Mode pass (Eq. 4 with the lazy R-hat refresh of Algorithm 1): one block per bin
// (bins come from the same ticket counter as the narrow passes).  An item's entries
// are taken 32 at a time; each warp builds the rows of H' = [H | r_hat] for its
// entries in shared memory (lanes over columns, so the slice rows are read with
// coalesced loads), then the block adds H'^T H' to a 16 x 16 grid of register tiles:
// the C x C Gram matrix B and, in row C, the right-hand side c = H^T r_hat.  At the
// end of an item the lower triangle of B and c go to the item's partial slot, in the
// packed layout the narrow kernels use.
//
// Row solve: one warp per row sums the row's slots in slot order, factors B + lambda I
// (right-looking Cholesky in shared memory, Section 3.1) and writes the row.  A
// non-positive pivot leaves the row unchanged and is counted.
#include <algorithm>

#include "dense_solve.cuh"
#include "sweep.cuh"

namespace tfs {
namespace {

constexpr int kWideThreads = 256;
constexpr int kWideTile = 32;        // entries per tile
constexpr int kSolveWarps = 4;        // rows per solve block

template <class T>
__device__ __forceinline__ T wsum(T v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xFFFFFFFFu, v, o);
    return v;
}

// 16-byte vector of slice values (4 floats or 2 doubles).
template <class T>
struct Vec16;
template <>
struct Vec16<float> {
    using type = float4;
    static constexpr int n = 4;
    __device__ static void unpack(const float4 &v, float (&x)[4]) {
        x[0] = v.x, x[1] = v.y, x[2] = v.z, x[3] = v.w;
    }
};
template <>
struct Vec16<double> {
    using type = double2;
    static constexpr int n = 2;
    __device__ static void unpack(const double2 &v, double (&x)[2]) { x[0] = v.x, x[1] = v.y; }
};

// Columns of one entry's H' row taken by lane g of its 8 lanes: h_c for c < C, and on the
// first inner iteration the R-hat refresh products po (c < C) and pp (c < Cq).  Three-mode
// tensors (two other rows): lane g takes 16-byte vectors of columns VW g + 8 VW k .. + VW - 1
// (VW = 4 floats or 2 doubles), so each row region is read with whole-vector loads, all
// issued together; regions start at multiples of CM, a multiple of VW on this path, and
// the packed slices hold zeros past C (cur, old) and past Cq (prev).  Other orders take
// columns g, g + 8, ... one value at a time.
template <class T, int CW, bool FIRST, class Store>
__device__ __forceinline__ void wide_entry_columns(const T *const *rows, int no, int n_lo, int C,
                                                   int Cq, int CM, const T *own, bool valid,
                                                   int g, T &pp, T &po, Store store) {
    if (no == 2) {
        using V = typename Vec16<T>::type;
        constexpr int VW = Vec16<T>::n;
#pragma unroll
        for (int k = 0; k < CW / (8 * VW); ++k) {
            const int c0 = VW * g + 8 * VW * k;
            T x0[VW], x1[VW], o0[VW], o1[VW], p0[VW], p1[VW];
#pragma unroll
            for (int u = 0; u < VW; ++u) x0[u] = x1[u] = o0[u] = o1[u] = p0[u] = p1[u] = T(0);
            if (valid && c0 < CM) {
                Vec16<T>::unpack(*reinterpret_cast<const V *>(rows[0] + c0), x0);
                Vec16<T>::unpack(*reinterpret_cast<const V *>(rows[1] + c0), x1);
                if (FIRST) {
                    if (n_lo > 0)
                        Vec16<T>::unpack(*reinterpret_cast<const V *>(rows[0] + 2 * CM + c0), o0);
                    if (n_lo > 1)
                        Vec16<T>::unpack(*reinterpret_cast<const V *>(rows[1] + 2 * CM + c0), o1);
                    if (c0 < Cq) {
                        Vec16<T>::unpack(*reinterpret_cast<const V *>(rows[0] + CM + c0), p0);
                        Vec16<T>::unpack(*reinterpret_cast<const V *>(rows[1] + CM + c0), p1);
                    }
                }
            }
#pragma unroll
            for (int u = 0; u < VW; ++u) {
                const int c = c0 + u;
                T hv = T(0);
                if (valid && c < C) {
                    hv = x0[u] * x1[u];
                    if (FIRST) {
                        const T a0 = n_lo > 0 ? o0[u] : x0[u];
                        const T a1 = n_lo > 1 ? o1[u] : x1[u];
                        po += own[CM + c] * (a0 * a1);
                    }
                }
                if (FIRST && valid && c < Cq) pp += own[c] * (p0[u] * p1[u]);
                store(c, hv);
            }
        }
        return;
    }
#pragma unroll
    for (int k = 0; k < CW / 8; ++k) {
        const int c = g + 8 * k;
        T hv = T(0);
        if (valid && c < C) {
            hv = T(1);
            for (int t = 0; t < no; ++t) hv *= rows[t][c];
            if (FIRST) {
                T o = own[CM + c];
                for (int t = 0; t < no; ++t) o *= (t < n_lo ? rows[t][2 * CM + c] : rows[t][c]);
                po += o;
            }
        }
        if (FIRST && valid && c < Cq) {
            T p = own[c];
            for (int t = 0; t < no; ++t) p *= rows[t][CM + c];
            pp += p;
        }
        store(c, hv);
    }
}

// CW: Gram tile width (32, 64 or 128), at least C + 1 (column C holds r_hat) and at least
// CM (the previous subset's columns are read through the same loop).
template <class T, int CW, bool FIRST>
__global__ void __launch_bounds__(kWideThreads) k_pass_wide(const PassArgs<T> a, int CM, int W) {
    constexpr int R = CW / 16;       // register tile edge
    constexpr int HS = CW + 4;       // H row stride (elements)
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T *H = reinterpret_cast<T *>(smem_raw);           // [kWideTile][HS]
    T *own = H + kWideTile * HS;                       // prev | old of the own row (2 CM)
    T *s_res2 = own + 2 * CM;                          // [2][kWideTile]
    int32_t *s_idx2 = reinterpret_cast<int32_t *>(s_res2 + 2 * kWideTile);  // [2][no][kWideTile]
    __shared__ unsigned long long s_tk;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int ty = tid >> 4, tx = tid & 15;
    const int no = a.N - 1, n_lo = a.n, C = a.C, Cq = a.Cq;
    const bool active = ty >= tx;  // lower block triangle only
    T acc[R][R];
#pragma unroll
    for (int i = 0; i < R; ++i)
#pragma unroll
        for (int j = 0; j < R; ++j) acc[i][j] = T(0);

    for (;;) {
        if (tid == 0) s_tk = atomicAdd(a.ticket, 1ull) - a.ticket_base;
        __syncthreads();
        const unsigned long long tk = s_tk;
        __syncthreads();
        if (tk >= (unsigned long long)a.P) break;
        for (int64_t it = a.bin_ptr[tk]; it < a.bin_ptr[tk + 1]; ++it) {
            const tf_item item = a.items[it];
            if (FIRST) {
                const T *z = a.Zn + (int64_t)a.rank_n[item.row] * W;
                for (int q = tid; q < 2 * CM; q += kWideThreads) own[q] = z[CM + q];
            }
            int buf = 0;
            for (int64_t j0 = item.begin; j0 < item.begin + item.len; j0 += kWideTile) {
                const int64_t left = item.begin + item.len - j0;
                const int ne = left < kWideTile ? (int)left : kWideTile;
                __syncthreads();  // H and own are free; this tile's indices are staged
                int32_t *s_idx = s_idx2 + buf * (kMaxModes - 1) * kWideTile;
                T *s_res = s_res2 + buf * kWideTile;
                if (j0 == item.begin) {  // the item's first tile: its indices now
                    if (tid < kWideTile * (no + 1)) {
                        const int t = tid / kWideTile, e = tid - t * kWideTile;
                        if (e < ne) {
                            if (t < no)
                                s_idx[t * kWideTile + e] = a.oidx[t][j0 + e];
                            else
                                s_res[e] = a.res[j0 + e];
                        }
                    }
                    __syncthreads();
                }
                // the next tile's indices and residuals: loaded now, stored after this
                // tile's Gram, so their latency hides behind the work on this tile
                const int64_t j1 = j0 + kWideTile, left1 = item.begin + item.len - j1;
                const int ne1 = left1 <= 0 ? 0 : (left1 < kWideTile ? (int)left1 : kWideTile);
                const int pq_t = tid / kWideTile, pq_e = tid - pq_t * kWideTile;
                const bool pre = tid < kWideTile * (no + 1) && pq_e < ne1;
                int32_t pre_i = 0;
                T pre_r = T(0);
                if (pre) {
                    if (pq_t < no)
                        pre_i = a.oidx[pq_t][j1 + pq_e];
                    else
                        pre_r = a.res[j1 + pq_e];
                }
                {   // 8 lanes per entry, columns g, g + 8, ...: one round of independent loads
                    const int e = tid >> 3, g = tid & 7;
                    const bool valid = e < ne;
                    T *h = H + e * HS;
                    const T *rows[kMaxModes - 1];
                    for (int t = 0; t < no; ++t)
                        rows[t] = a.Zo[t] + (int64_t)(valid ? s_idx[t * kWideTile + e] : 0) * W;
                    T pp = T(0), po = T(0);
                    // columns of S (< C <= CW - 1) and of the previous subset Q (< Cq <= CM
                    // <= CW)
                    wide_entry_columns<T, CW, FIRST>(rows, no, n_lo, C, Cq, CM, own, valid, g, pp,
                                                     po, [&](int c, T hv) { h[c] = hv; });
#pragma unroll
                    for (int o = 4; o > 0; o >>= 1) {
                        pp += __shfl_xor_sync(0xFFFFFFFFu, pp, o);
                        po += __shfl_xor_sync(0xFFFFFFFFu, po, o);
                    }
                    __syncwarp();
                    if (valid && g == 0) {
                        T v = s_res[e];
                        if (FIRST) {
                            v = v - pp + po;
                            a.res[j0 + e] = v;
                        }
                        h[C] = v;
                    }
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
                if (pre) {
                    if (pq_t < no)
                        s_idx2[(buf ^ 1) * (kMaxModes - 1) * kWideTile + pq_t * kWideTile + pq_e] = pre_i;
                    else
                        s_res2[(buf ^ 1) * kWideTile + pq_e] = pre_r;
                }
                buf ^= 1;
            }
            // item end: lower triangle of B (rows/cols < C) and c = row C of H'^T H'
            T *p = a.partials + (int64_t)item.slot * (CM * (CM + 1) / 2 + CM);
            const int NT = CM * (CM + 1) / 2;
            if (active) {
#pragma unroll
                for (int i = 0; i < R; ++i)
#pragma unroll
                    for (int j = 0; j < R; ++j) {
                        const int r = ty * R + i, cc = tx * R + j;
                        if (r < CM && cc <= r) p[r * (r + 1) / 2 + cc] = r < C ? acc[i][j] : T(0);
                        if (r == C && cc < CM) p[NT + cc] = cc < C ? acc[i][j] : T(0);
                        acc[i][j] = T(0);
                    }
            }
            if (C < CM)  // columns C..CM-1 of c (row C covers c only up to CW)
                for (int q = C + tid; q < CM; q += kWideThreads) p[NT + q] = T(0);
        }
    }
}

// ---------------------------------------------------------------- tensor-core Gram
// Float contexts: the same pass with H'^T H' on the 5th-generation tensor cores.  The
// tile's H' is stored transposed in shared memory (columns of H' as M rows, entries as
// K, no swizzle: 8-row x 16-byte core matrices, K-adjacent ones 128 bytes apart, 8-row
// groups kTcSbo bytes apart), split into a TF32 high part and a TF32 remainder; three
// tcgen05.mma kind::tf32 per 8 entries (hi.hi + hi.lo + lo.hi) accumulate the Gram in a
// 128 x CW fp32 tile of tensor memory, which keeps FP32-level accuracy.  One thread
// issues the MMAs and commits them to the mbarrier of the operand stage; a stage is
// rewritten only after its commit arrived (bounded waits).  At the end of an item warps 0-3 read
// the tile back (tcgen05.ld, one row per thread) and store the item's partial.

constexpr int kTcM = 128;                          // MMA rows (H' columns, padded)
constexpr int kTcSbo = (kWideTile / 4) * 128;      // bytes between 8-row groups
constexpr int kTcBuf = (kTcM / 8) * kTcSbo;        // one operand copy: 16 KB
constexpr long long kTcSpin = 1ll << 24;
// Operand stages.  Two let the next tile be built while the MMAs run, but cost a block
// per SM; the tile build (row gathers) dominates and measured faster with one.
constexpr int kTcStages = 1;

__device__ __forceinline__ unsigned tc_saddr(const void *p) {
    return (unsigned)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ uint64_t tc_desc(const void *p) {
    const uint64_t a = tc_saddr(p);
    return ((a >> 4) & 0x3FFFull) | ((uint64_t)(128 >> 4) << 16) |
           ((uint64_t)(kTcSbo >> 4) << 32) | (1ull << 46);
}
__device__ __forceinline__ uint32_t tf32_bits(float x) {
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return r;
}
__device__ __forceinline__ bool tc_wait(uint64_t *bar, unsigned parity) {
    for (long long i = 0; i < kTcSpin; ++i) {
        uint32_t ok;
        asm volatile(
            "{ .reg .pred p; mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2; selp.u32 %0, 1, "
            "0, p; }"
            : "=r"(ok)
            : "r"(tc_saddr(bar)), "r"(parity)
            : "memory");
        if (ok) return true;
    }
    return false;
}
__device__ __forceinline__ void tc_ld32(uint32_t taddr, uint32_t (&r)[32]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,"
        "%14,%15,%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
          "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
          "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]),
          "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]),
          "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr)
        : "memory");
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

// SPLIT: three TF32 products per term (FP32-level accuracy); without it one TF32
// product (about 1e-3 relative error in B and c, the reduced-precision form).  64- and
// 128-wide tiles are held to three blocks per SM (about 80 registers): at 1e8 entries that
// took the C = 50 and C = 100 sweeps from 170 and 166 ms to 146 and 144 ms.
template <int CW, bool FIRST, bool SPLIT>
__global__ void __launch_bounds__(kWideThreads, CW >= 64 ? 3 : 1)
    k_pass_wide_tc(const PassArgs<float> a, int CM, int W) {
    using T = float;
    constexpr int kTcCols = CW;  // tensor-memory columns: the accumulator is 128 x CW fp32
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    // kTcStages operand stages (hi and lo copies each)
    unsigned char *stage0 = smem_raw;
    T *own = reinterpret_cast<T *>(smem_raw + 2 * kTcStages * kTcBuf);  // prev | old (2 CM)
    T *s_res2 = own + 2 * CM;                                  // [2][kWideTile]
    int32_t *s_idx2 = reinterpret_cast<int32_t *>(s_res2 + 2 * kWideTile);  // [2][no][kWideTile]
    __shared__ __align__(8) uint64_t mbar[2];
    __shared__ uint32_t s_taddr;
    __shared__ unsigned long long s_tk;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int no = a.N - 1, n_lo = a.n, C = a.C, Cq = a.Cq;
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         tc_saddr(&s_taddr)),
                     "r"(kTcCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(tc_saddr(&mbar[0])) : "memory");
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(tc_saddr(&mbar[1])) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t taddr = s_taddr;
    const uint32_t idesc = (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(CW >> 3) << 17) |
                           ((uint32_t)(kTcM >> 4) << 24);
    // per stage: the parity the next wait expects, and whether a commit is outstanding
    // (every thread tracks the same values)
    unsigned phase[2] = {0u, 0u};
    bool pending[2] = {false, false};
    bool timed_out = false;
    unsigned tiles = 0;
    auto drain = [&](int st) {
        if (!pending[st]) return true;
        const bool ok = tc_wait(&mbar[st], phase[st]);
        phase[st] ^= 1u;
        pending[st] = false;
        return ok;
    };

    for (;;) {
        if (tid == 0) s_tk = atomicAdd(a.ticket, 1ull) - a.ticket_base;
        __syncthreads();
        const unsigned long long tk = s_tk;
        __syncthreads();
        if (tk >= (unsigned long long)a.P) break;
        for (int64_t it = a.bin_ptr[tk]; it < a.bin_ptr[tk + 1] && !timed_out; ++it) {
            const tf_item item = a.items[it];
            if (FIRST) {
                const T *z = a.Zn + (int64_t)a.rank_n[item.row] * W;
                for (int q = tid; q < 2 * CM; q += kWideThreads) own[q] = z[CM + q];
            }
            bool first_tile = true;
            int buf = 0;
            for (int64_t j0 = item.begin; j0 < item.begin + item.len; j0 += kWideTile) {
                const int64_t left = item.begin + item.len - j0;
                const int ne = left < kWideTile ? (int)left : kWideTile;
                const int st = kTcStages == 1 ? 0 : (int)(tiles & 1u);
                unsigned char *ahi = stage0 + st * 2 * kTcBuf, *alo = ahi + kTcBuf;
                // the stage's previous MMAs must be done before its operands change
                const bool ok = drain(st);
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                if (__syncthreads_or(!ok)) {
                    timed_out = true;
                    break;
                }
                int32_t *s_idx = s_idx2 + buf * (kMaxModes - 1) * kWideTile;
                T *s_res = s_res2 + buf * kWideTile;
                if (j0 == item.begin) {  // the item's first tile: its indices now
                    if (tid < kWideTile * (no + 1)) {
                        const int t = tid / kWideTile, e = tid - t * kWideTile;
                        if (e < ne) {
                            if (t < no)
                                s_idx[t * kWideTile + e] = a.oidx[t][j0 + e];
                            else
                                s_res[e] = a.res[j0 + e];
                        }
                    }
                    __syncthreads();
                }
                // the next tile's indices and residuals: loaded now, stored after this
                // tile's Gram, so their latency hides behind the work on this tile
                const int64_t j1 = j0 + kWideTile, left1 = item.begin + item.len - j1;
                const int ne1 = left1 <= 0 ? 0 : (left1 < kWideTile ? (int)left1 : kWideTile);
                const int pq_t = tid / kWideTile, pq_e = tid - pq_t * kWideTile;
                const bool pre = tid < kWideTile * (no + 1) && pq_e < ne1;
                int32_t pre_i = 0;
                T pre_r = T(0);
                if (pre) {
                    if (pq_t < no)
                        pre_i = a.oidx[pq_t][j1 + pq_e];
                    else
                        pre_r = a.res[j1 + pq_e];
                }
                {
                    const int e = tid >> 3, g = tid & 7;
                    const bool valid = e < ne;
                    const T *rows[kMaxModes - 1];
                    for (int t = 0; t < no; ++t)
                        rows[t] = a.Zo[t] + (int64_t)(valid ? s_idx[t * kWideTile + e] : 0) * W;
                    T pp = T(0), po = T(0);
                    const int eoff = (e >> 2) * 128 + (e & 3) * 4;
                    wide_entry_columns<T, CW, FIRST>(
                        rows, no, n_lo, C, Cq, CM, own, valid, g, pp, po, [&](int c, T hv) {
                            if (c == C) return;
                            const int off = (c >> 3) * kTcSbo + eoff + (c & 7) * 16;
                            const uint32_t hb = tf32_bits(hv);
                            *reinterpret_cast<uint32_t *>(ahi + off) = hb;
                            if (SPLIT)
                                *reinterpret_cast<uint32_t *>(alo + off) = tf32_bits(hv - __uint_as_float(hb));
                        });
#pragma unroll
                    for (int o = 4; o > 0; o >>= 1) {
                        pp += __shfl_xor_sync(0xFFFFFFFFu, pp, o);
                        po += __shfl_xor_sync(0xFFFFFFFFu, po, o);
                    }
                    if (g == 0) {
                        T v = valid ? s_res[e] : T(0);
                        if (FIRST && valid) {
                            v = v - pp + po;
                            a.res[j0 + e] = v;
                        }
                        const int off = (C >> 3) * kTcSbo + eoff + (C & 7) * 16;
                        const uint32_t hb = tf32_bits(v);
                        *reinterpret_cast<uint32_t *>(ahi + off) = hb;
                        if (SPLIT)
                            *reinterpret_cast<uint32_t *>(alo + off) = tf32_bits(v - __uint_as_float(hb));
                    }
                }
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
                __syncthreads();
                if (tid == 0) {
                    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                    for (int k = 0; k < kWideTile / 8; ++k) {
                        const uint64_t dh = tc_desc(ahi + k * 256), dl = tc_desc(alo + k * 256);
                        const uint64_t A[3] = {dh, dh, dl}, B[3] = {dh, dl, dh};
#pragma unroll
                        for (int u = 0; u < (SPLIT ? 3 : 1); ++u) {
                            const uint32_t acc = (first_tile && k == 0 && u == 0) ? 0u : 1u;
                            asm volatile(
                                "{ .reg .pred p; setp.ne.b32 p, %4, 0; "
                                "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p; }" ::"r"(taddr),
                                "l"(A[u]), "l"(B[u]), "r"(idesc), "r"(acc)
                                : "memory");
                        }
                    }
                    asm volatile(
                        "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                            tc_saddr(&mbar[st]))
                        : "memory");
                }
                if (pre) {
                    if (pq_t < no)
                        s_idx2[(buf ^ 1) * (kMaxModes - 1) * kWideTile + pq_t * kWideTile + pq_e] = pre_i;
                    else
                        s_res2[(buf ^ 1) * kWideTile + pq_e] = pre_r;
                }
                buf ^= 1;
                pending[st] = true;
                ++tiles;
                first_tile = false;
            }
            if (timed_out) break;
            // item end: wait for its MMAs, then rows of the Gram tile -> lower triangle
            // of B and c = row C
            {
                const bool ok0 = drain(0), ok1 = drain(1);
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                if (__syncthreads_or(!(ok0 && ok1))) {
                    timed_out = true;
                    break;
                }
            }
            T *p = a.partials + (int64_t)item.slot * (CM * (CM + 1) / 2 + CM);
            const int NT = CM * (CM + 1) / 2;
            if (warp < 4) {
                const int r = warp * 32 + lane;
                for (int cc = 0; cc < CW; cc += 32) {
                    uint32_t v[32];
                    if (!first_tile) {
                        tc_ld32(taddr + ((uint32_t)(warp * 32) << 16) + (uint32_t)cc, v);
                    } else {
#pragma unroll
                        for (int q = 0; q < 32; ++q) v[q] = 0u;  // empty item: B = 0, c = 0
                    }
#pragma unroll
                    for (int q = 0; q < 32; ++q) {
                        const int j = cc + q;
                        const T val = __uint_as_float(v[q]);
                        if (r < CM && j <= r) p[r * (r + 1) / 2 + j] = (r < C && j < C) ? val : T(0);
                        if (r == C && j < CM) p[NT + j] = j < C ? val : T(0);
                    }
                }
            }
            if (C < CM)
                for (int q = C + tid; q < CM; q += kWideThreads) p[NT + q] = T(0);
            asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
            __syncthreads();
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        }
        if (timed_out) break;
    }
    {   // MMAs still in flight (after a timeout) finish before the tensor memory goes
        const bool ok0 = drain(0), ok1 = drain(1);
        if ((timed_out || !ok0 || !ok1) && tid == 0) atomicOr(&a.stat->bits, kStatTimeout);
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(kTcCols)
                     : "memory");
}

// Shared memory of one warp of k_solve_wide: the system (packed triangle and rhs) and,
// for float contexts that refine or may fall back to FP64, a copy of the sums and a double
// copy for the FP64 solve.
template <class T>
__host__ __device__ inline size_t wide_solve_warp_bytes(int C, bool refine, bool fallback) {
    const size_t nb = (size_t)C * (C + 1) / 2 + C;
    size_t b = nb * sizeof(T);
    if (sizeof(T) == 4 && (refine || fallback)) b += nb * sizeof(T);
    b = (b + 15) / 16 * 16;
    if (sizeof(T) == 4 && fallback) b += nb * sizeof(double);
    return b;
}

// One warp per row (kSolveWarps rows per block): sums the row's slots in slot order
// into a packed lower triangle in shared memory, solves (B + lambda I) x = c and writes
// x to A_n[row][S[c]] and to the cur region of the own slice row.  Float contexts refine
// the solve or solve ill-conditioned rows again in FP64 as PassArgs::refine / cond_limit
// say (the narrow row_solve does the same per thread).
template <class T>
__global__ void __launch_bounds__(kSolveWarps * 32) k_solve_wide(const PassArgs<T> a,
                                                                 const SplitRow *rows, int n_rows,
                                                                 int CM, int W) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int C = a.C;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int r = blockIdx.x * (int)(blockDim.x >> 5) + warp;
    if (r >= n_rows) return;
    const int NT = CM * (CM + 1) / 2, NB = NT + CM;
    const bool refine = sizeof(T) == 4 && a.refine;
    const bool fallback = sizeof(T) == 4 && a.cond_limit > 0.f;
    const size_t nt = (size_t)C * (C + 1) / 2;
    unsigned char *wbase = smem_raw + warp * wide_solve_warp_bytes<T>(C, refine, fallback);
    T *P = reinterpret_cast<T *>(wbase);
    T *cv = P + nt;
    T *P0 = cv + C;  // the sums as accumulated (refine / fallback)
    T *c0 = P0 + nt;
    const SplitRow sr = rows[r];
    // rows with more than kSlotGroup slots hold their group sums at every kSlotGroup-th slot
    const int step = sr.n_slots > kSlotGroup ? kSlotGroup : 1;
    const int ntc = C * (C + 1) / 2;
    if (sr.n_slots == 1) {
        // a row held by one item: its slot is the system; eight loads in flight per lane
        // (the first C rows of the packed CM-triangle are the packed C-triangle)
        const T *src = a.partials + (int64_t)sr.first_slot * NB;
        for (int q0 = lane; q0 < ntc + C; q0 += 32 * 8) {
            T v[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const int q = q0 + 32 * u;
                v[u] = q < ntc ? src[q] : (q < ntc + C ? src[NT + (q - ntc)] : T(0));
            }
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const int q = q0 + 32 * u;
                if (q < ntc + C) {  // cv follows P in shared memory, and c0 follows P0
                    P[q] = v[u];
                    if (refine || fallback) P0[q] = v[u];
                }
            }
        }
    } else {
        for (int q = lane; q < ntc; q += 32) {
            T s = T(0);
            for (int k = 0; k < sr.n_slots; k += step)
                s += a.partials[(int64_t)(sr.first_slot + k) * NB + q];
            P[q] = s;
            if (refine || fallback) P0[q] = s;
        }
        for (int q = lane; q < C; q += 32) {
            T s = T(0);
            for (int k = 0; k < sr.n_slots; k += step)
                s += a.partials[(int64_t)(sr.first_slot + k) * NB + NT + q];
            cv[q] = s;
            if (refine || fallback) c0[q] = s;
        }
    }
    __syncwarp();
    const T lam = a.weighted ? a.lambda * (T)sr.len : a.lambda;
    T ratio = T(1);
    bool ok = warp_chol_factor<T>(P, C, lam, lane, &ratio);
    if (fallback && (!ok || ratio * (T)a.cond_limit < T(1))) {
        double *Pd = reinterpret_cast<double *>(
            wbase + ((2 * (nt + C) * sizeof(T) + 15) / 16) * 16);
        double *cd = Pd + nt;
        for (int q = lane; q < (int)nt; q += 32) Pd[q] = (double)P0[q];
        for (int q = lane; q < C; q += 32) cd[q] = (double)c0[q];
        __syncwarp();
        ok = warp_chol_factor<double>(Pd, C, (double)lam, lane);
        if (ok) {
            warp_chol_apply<double>(Pd, cd, C, lane);
            for (int q = lane; q < C; q += 32) cv[q] = (T)cd[q];
            if (lane == 0) atomicAdd(&a.stat->fp64_rows, 1ull);
        }
        __syncwarp();
    } else if (ok) {
        warp_chol_apply<T>(P, cv, C, lane);
        if (refine) {
            // residual of the system as accumulated, in FP64: c - (B + lam I) x, into c0
            for (int i = lane; i < C; i += 32) {
                double s = (double)c0[i] - (double)lam * (double)cv[i];
                for (int j = 0; j < C; ++j) {
                    const T b = j <= i ? P0[ptri(i, j)] : P0[ptri(j, i)];
                    s -= (double)b * (double)cv[j];
                }
                c0[i] = (T)s;
            }
            __syncwarp();
            warp_chol_apply<T>(P, c0, C, lane);
            for (int q = lane; q < C; q += 32) cv[q] += c0[q];
            __syncwarp();
        }
    }
    if (!ok) {
        if (lane == 0) atomicAdd(&a.stat->singular_rows, 1ull);
        return;
    }
    T *z = a.Zn + (int64_t)a.rank_n[sr.row] * W;
    T *Ar = a.A_n + (int64_t)sr.row * a.K;
    for (int q = lane; q < C; q += 32) {
        z[q] = cv[q];
        Ar[a.S[q]] = cv[q];
    }
}

// One block per group of consecutive slots of a split row: the group's elementwise sum,
// in slot order, into its first slot.
template <class T>
__global__ void __launch_bounds__(256) k_sum_slot_groups(T *partials, int NB,
                                                         const int32_t *groups) {
    const int64_t first = groups[2 * blockIdx.x];
    const int cnt = groups[2 * blockIdx.x + 1];
    T *base = partials + first * NB;
    for (int q = threadIdx.x; q < NB; q += blockDim.x) {
        T s = base[q];
        for (int k = 1; k < cnt; ++k) s += base[(int64_t)k * NB + q];
        base[q] = s;
    }
}

// Residual of copy n against the cur region of the slices: one warp per bin, lanes
// over columns; what = 0 sums r^2 per block (fixed order), 1 scatters r to canonical
// order, 2 writes r back to the copy.
template <class T>
__global__ void __launch_bounds__(kWideThreads) k_res_wide(const ResArgs<T> a, int W) {
    __shared__ double wsum_d[kWideThreads / 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int bin = blockIdx.x * (kWideThreads / 32) + warp;
    const int no = a.N - 1;
    double acc = 0.0;
    if (bin < a.P) {
        for (int64_t it = a.bin_ptr[bin]; it < a.bin_ptr[bin + 1]; ++it) {
            const tf_item item = a.items[it];
            const T *own = a.Zn + (int64_t)a.rank_n[item.row] * W;
            for (int64_t j = item.begin; j < item.begin + item.len; ++j) {
                T p = T(0);
                for (int c = lane; c < a.Cq; c += 32) {
                    T q = own[c];
                    for (int t = 0; t < no; ++t) q *= a.Zo[t][(int64_t)a.oidx[t][j] * W + c];
                    p += q;
                }
                p = wsum(p);
                const T r = a.res[j] - p;
                if (lane == 0) {
                    if (a.what == 0)
                        acc += (double)r * (double)r;
                    else if (a.what == 1)
                        a.out[a.perm[j]] = r;
                    else
                        a.res[j] = r;
                }
            }
        }
    }
    if (a.what != 0) return;
    if (lane == 0) wsum_d[warp] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int w = 0; w < kWideThreads / 32; ++w) s += wsum_d[w];
        a.block_out[blockIdx.x] = s;
    }
}

// Shared memory per tensor-core block that keeps residency at most 512 / CW blocks per SM
// (the SM's shared memory, 228 KB, over one more block than that, plus a margin).
size_t tc_min_smem(int CW) {
    const int max_blocks = 512 / CW;
    return (size_t)(228 * 1024) / (size_t)(max_blocks + 1) + 1024;
}

template <int CW>
void launch_pass_wide_tc_cw(const PassArgs<float> &a, int CM, int W, int grid, bool split,
                            cudaStream_t st) {
    // enough shared memory per block that at most 512 / CW blocks (each holding CW of the
    // SM's 512 tensor-memory columns) fit on an SM, so no allocation ever waits
    size_t smem = 2 * kTcStages * (size_t)kTcBuf + sizeof(float) * (2 * (size_t)CM + 2 * kWideTile) +
                  sizeof(int32_t) * 2 * (size_t)kWideTile * (kMaxModes - 1);
    smem = std::max<size_t>(smem, tc_min_smem(CW));
    auto kern = split ? (a.first ? k_pass_wide_tc<CW, true, true> : k_pass_wide_tc<CW, false, true>)
                      : (a.first ? k_pass_wide_tc<CW, true, false> : k_pass_wide_tc<CW, false, false>);
    TFS_CUDA(raise_smem_limit((const void *)kern, (int)smem));
    kern<<<grid, kWideThreads, smem, st>>>(a, CM, W);
    TFS_CUDA(cudaGetLastError());
}

template <class T, int CW>
void launch_pass_wide_cw(const PassArgs<T> &a, int CM, int W, int grid, cudaStream_t st) {
    const size_t smem = sizeof(T) * ((size_t)kWideTile * (CW + 4) + 2 * (size_t)CM + 2 * kWideTile) +
                        sizeof(int32_t) * 2 * (size_t)kWideTile * (kMaxModes - 1);
    auto kern = a.first ? k_pass_wide<T, CW, true> : k_pass_wide<T, CW, false>;
    TFS_CUDA(raise_smem_limit((const void *)kern, (int)smem));
    kern<<<grid, kWideThreads, smem, st>>>(a, CM, W);
    TFS_CUDA(cudaGetLastError());
}

}  // namespace

int wide_tile_width(int C) { return C + 1 <= 32 ? 32 : (C + 1 <= 64 ? 64 : (C + 1 <= 128 ? 128 : 0)); }

// Tile width of a split: H' needs C + 1 columns, and the R-hat refresh reads the previous
// subset's Cq <= CM columns through the same column loop.
int wide_split_width(int C, int CM) {
    const int need = std::max(C + 1, CM);
    return need <= 32 ? 32 : (need <= 64 ? 64 : (need <= 128 ? 128 : 0));
}

// Blocks of a wide pass: every block that can be resident (the SIMT variant's few
// registers allow up to 8 per SM; the tensor-core one is held to 4 by its shared memory,
// 4 x 128 tensor-memory columns).
template <class T>
int pass_wide_grid(int num_sms, int P, int C, int CM, bool tensor_cores, bool first) {
    int per_sm = 4;
    if (sizeof(T) == 4 && tensor_cores) {
        const int cw = wide_split_width(C, CM);
        const size_t smem = std::max<size_t>(
            2 * kTcStages * (size_t)kTcBuf + sizeof(float) * (2 * (size_t)CM + 2 * kWideTile) +
                sizeof(int32_t) * 2 * (size_t)kWideTile * (kMaxModes - 1),
            tc_min_smem(cw));
        per_sm = std::max(1, std::min(512 / cw, (int)((228 * 1024) / (smem + 1024))));
    } else {
        const int cw = wide_split_width(C, CM);
        const size_t smem = sizeof(T) * ((size_t)kWideTile * (cw + 4) + 2 * (size_t)CM + 2 * kWideTile) +
                            sizeof(int32_t) * 2 * (size_t)kWideTile * (kMaxModes - 1);
        const void *kern = nullptr;
        if (cw == 32)
            kern = first ? (const void *)k_pass_wide<T, 32, true> : (const void *)k_pass_wide<T, 32, false>;
        else if (cw == 64)
            kern = first ? (const void *)k_pass_wide<T, 64, true> : (const void *)k_pass_wide<T, 64, false>;
        else
            kern = first ? (const void *)k_pass_wide<T, 128, true> : (const void *)k_pass_wide<T, 128, false>;
        TFS_CUDA(raise_smem_limit((const void *)kern, (int)smem));
        TFS_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kWideThreads, smem));
        per_sm = std::max(1, std::min(per_sm, 8));
    }
    return std::max(1, std::min(P, num_sms * per_sm));
}

template <class T>
void launch_pass_wide(const PassArgs<T> &a, int CM, int W, int grid, bool tensor_cores, bool split,
                      cudaStream_t st) {
    if constexpr (sizeof(T) == 4) {
        if (tensor_cores) {
            switch (wide_split_width(a.C, CM)) {
                case 32:
                    launch_pass_wide_tc_cw<32>(a, CM, W, grid, split, st);
                    return;
                case 64:
                    launch_pass_wide_tc_cw<64>(a, CM, W, grid, split, st);
                    return;
                case 128:
                    launch_pass_wide_tc_cw<128>(a, CM, W, grid, split, st);
                    return;
                default:
                    throw ApiError{TF_EINVAL, "C >= 128 is not supported"};
            }
        }
    }
    switch (wide_split_width(a.C, CM)) {
        case 32:
            launch_pass_wide_cw<T, 32>(a, CM, W, grid, st);
            return;
        case 64:
            launch_pass_wide_cw<T, 64>(a, CM, W, grid, st);
            return;
        case 128:
            launch_pass_wide_cw<T, 128>(a, CM, W, grid, st);
            return;
        default:
            throw ApiError{TF_EINVAL, "C >= 128 is not supported"};
    }
}

template <class T>
void launch_solve_wide(const PassArgs<T> &a, const SplitRow *rows, int n_rows, int CM, int W,
                       cudaStream_t st) {
    if (n_rows <= 0) return;
    int dev = 0, smem_blk = 0, smem_sm = 0;
    TFS_CUDA(cudaGetDevice(&dev));
    TFS_CUDA(cudaDeviceGetAttribute(&smem_blk, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
    TFS_CUDA(cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev));
    const size_t per_warp =
        wide_solve_warp_bytes<T>(a.C, a.refine != 0, a.cond_limit > 0.f);
    // warps per block: the most resident warps per SM (each warp holds one system in
    // shared memory, so the block size decides how well the SM's shared memory is used)
    int wpb = 1, best = 0;
    for (int w = 1; w <= kSolveWarps; ++w) {
        if ((size_t)w * per_warp > (size_t)smem_blk) break;
        const int blocks = std::min<int>(32, (int)((size_t)smem_sm / ((size_t)w * per_warp + 1024)));
        if (blocks * w >= best) {
            best = blocks * w;
            wpb = w;
        }
    }
    const size_t smem = per_warp * wpb;
    TFS_CUDA(raise_smem_limit((const void *)k_solve_wide<T>, (int)smem));
    k_solve_wide<T><<<(n_rows + wpb - 1) / wpb, wpb * 32, smem, st>>>(a, rows, n_rows, CM, W);
    TFS_CUDA(cudaGetLastError());
}

int res_wide_blocks(int P) { return (P + kWideThreads / 32 - 1) / (kWideThreads / 32); }

template <class T>
void launch_sum_slot_groups(T *partials, int NB, const int32_t *groups, int n_groups,
                            cudaStream_t st) {
    if (n_groups <= 0) return;
    k_sum_slot_groups<T><<<n_groups, 256, 0, st>>>(partials, NB, groups);
    TFS_CUDA(cudaGetLastError());
}

template <class T>
void launch_res_wide(const ResArgs<T> &a, int W, cudaStream_t st) {
    k_res_wide<T><<<res_wide_blocks(a.P), kWideThreads, 0, st>>>(a, W);
    TFS_CUDA(cudaGetLastError());
}

#define TFS_INST(T)                                                                           \
    template int pass_wide_grid<T>(int, int, int, int, bool, bool);                           \
    template void launch_pass_wide<T>(const PassArgs<T> &, int, int, int, bool, bool,          \
                                      cudaStream_t);                                          \
    template void launch_solve_wide<T>(const PassArgs<T> &, const SplitRow *, int, int, int,  \
                                       cudaStream_t);                                         \
    template void launch_res_wide<T>(const ResArgs<T> &, int, cudaStream_t);                \
    template void launch_sum_slot_groups<T>(T *, int, const int32_t *, int, cudaStream_t);
TFS_INST(float)
TFS_INST(double)
#undef TFS_INST

}  // namespace tfs
