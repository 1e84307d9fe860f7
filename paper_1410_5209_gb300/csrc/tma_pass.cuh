// Mode pass fed by the Tensor Memory Accelerator (float, three modes, C <= 10).
//
// Same arithmetic as k_mode_pass (Eq. 4 Gram / rhs and the lazy R-hat refresh of
// Algorithm 1), different data movement.  One block per SM, W warps, each warp working
// through bins taken from the ticket counter with a ring of shared-memory slots filled
// by TMA, one mbarrier per slot (no ordering between slots):
//   2 steps ahead: one lane issues 1D bulk copies of the step's index windows of both
//                  other modes, its residual window and (first step of an item) the own
//                  slice row;
//   1 step ahead:  the warp finds the step's distinct slice rows that are not cached
//                  (consecutive entries of a row share their leading other-mode index
//                  in long runs), lists them, and up to 16 lanes each issue one
//                  tile::gather4 of 4 listed rows into the step's row slot;
//   now:           wait for the slot, compute, release it.
// Row cache: at launch the block copies the first H[t] rows of each other mode's slice
// (in degree-rank order: the rows with the most entries) into shared memory; a small
// mode is held whole.  Entries whose row is cached read it there and are never
// gathered.
// Gathered rows land densely at the box width; boxes are 8, 24 or 40 floats (a multiple
// of 8 floats keeps every 4-row destination 128-byte aligned; a row of 2 mod 4 16-byte
// vectors limits lane-per-row vector reads to 2-way bank conflicts).  Box columns past
// the slice row are zero-filled by the TMA.  Every wait is bounded: on expiry the
// kernel records kStatTimeout, drains what it issued (bounded again) and returns.
#pragma once

#include <cuda.h>

#include "mode_pass.cuh"

namespace tfs {

constexpr int kTmaLeadRows = 1, kTmaLeadIdx = 2;
constexpr int kTmaRowSlots = kTmaLeadRows + 1, kTmaIdxSlots = kTmaLeadIdx + 1;
constexpr int kTmaWin = 36;               // window entries: 32 + alignment slack (4)
constexpr int kTmaMaxWarps = 12;          // warps per block (one block per SM)
constexpr long long kTmaSpinLimit = 1ll << 25;

// Box width (floats) for `need` leading floats of a slice row.
__host__ __device__ constexpr int tma_box(int need) {
    return need <= 8 ? 8 : (need <= 24 ? 24 : (need <= 40 ? 40 : 56));
}

// Byte layout of one warp's ring (every piece 128-byte aligned, sizes set at launch).
struct TmaWarpLayout {
    static constexpr unsigned kIdxSlot = 2 * kTmaWin * 4 + kTmaWin * 4 + 128 + 32;  // 592
    static constexpr unsigned kListBytes = 2 * 32 * 4;
    static constexpr unsigned kItemBytes = 32 * sizeof(tf_item) + 32 * 4;
    unsigned row_slot;   // bytes of one row slot (the staged other modes)
    unsigned mode1_off;  // offset of mode t = 1 inside a row slot
    unsigned bytes;      // whole ring, a multiple of 128
};

inline TmaWarpLayout tma_warp_layout(int box0, int box1, bool stage0, bool stage1) {
    TmaWarpLayout L;
    L.mode1_off = stage0 ? 32u * box0 * 4u : 0u;
    L.row_slot = L.mode1_off + (stage1 ? 32u * box1 * 4u : 0u);
    const unsigned b = kTmaRowSlots * L.row_slot + kTmaIdxSlots * TmaWarpLayout::kIdxSlot +
                       TmaWarpLayout::kListBytes + TmaWarpLayout::kItemBytes + 128 /*own*/ +
                       (kTmaRowSlots + kTmaIdxSlots) * 8;
    L.bytes = (b + 127) / 128 * 128;
    return L;
}

struct TmaPassArgs {
    PassArgs<float> p;
    CUtensorMap tm[2];   // other modes' slices, box widths box[t]
    int box[2];          // gather box (floats) per other mode
    int hot[2];          // rows [0, hot[t]) of other mode t are cached in shared memory
    int cs[2];           // cached row stride (floats, an odd number of 16-byte vectors)
    int cv[2];           // 16-byte vectors copied per cached row
    unsigned cache_off1; // byte offset of mode 1's cache; rings start at cache_bytes
    unsigned cache_bytes;
    TmaWarpLayout L;
};

__device__ __forceinline__ void mbar_init(void *bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count)
                 : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(void *bar, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)),
                 "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(void *bar, unsigned parity) {
    unsigned done;
    asm volatile(
        "{ .reg .pred p; mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2; selp.u32 %0, 1, 0, "
        "p; }"
        : "=r"(done)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return done != 0;
}
__device__ __forceinline__ bool mbar_wait_bounded(void *bar, unsigned parity) {
    for (long long i = 0; i < kTmaSpinLimit; ++i)
        if (mbar_try_wait(bar, parity)) return true;
    return false;
}
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, unsigned bytes, void *bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::
            "r"(smem_addr(dst)),
        "l"(src), "r"(bytes), "r"(smem_addr(bar))
        : "memory");
}
__device__ __forceinline__ void gather4_g2s(void *dst, const CUtensorMap *tm, int x, int y0, int y1,
                                            int y2, int y3, void *bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile::gather4.mbarrier::complete_tx::bytes "
        "[%0], [%1, {%2, %3, %4, %5, %6}], [%7];" ::"r"(smem_addr(dst)),
        "l"(tm), "r"(x), "r"(y0), "r"(y1), "r"(y2), "r"(y3), "r"(smem_addr(bar))
        : "memory");
}

// Run heads of one step and one other mode: lanes holding a valid entry whose row is
// not cached and differs from the previous lane's (consecutive equal rows share one
// gathered copy).
__device__ __forceinline__ unsigned tma_heads(int rank, int hot, int nvalid, int lane) {
    const int before = __shfl_up_sync(0xFFFFFFFFu, rank, 1);
    return __ballot_sync(0xFFFFFFFFu,
                         lane < nvalid && rank >= hot && (lane == 0 || rank != before));
}

template <int CM, bool FIRST>
__global__ void __launch_bounds__(kTmaMaxWarps * kWarp, 1)
    k_mode_pass_tma(const __grid_constant__ TmaPassArgs ta) {
    using T = float;
    using G = Geo<T, CM>;
    constexpr int NT = G::NT;
    const PassArgs<T> &a = ta.p;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    // 128-byte aligned base (the launch reserves 128 extra bytes)
    unsigned char *aligned = reinterpret_cast<unsigned char *>(
        (reinterpret_cast<uintptr_t>(smem_raw) + 127) & ~static_cast<uintptr_t>(127));
    const T *cache[2] = {reinterpret_cast<const T *>(aligned),
                         reinterpret_cast<const T *>(aligned + ta.cache_off1)};

    // block-wide: the hottest rows of both other modes (ranks [0, hot[t]))
#pragma unroll
    for (int t = 0; t < 2; ++t) {
        const int nv = ta.cv[t], cs = ta.cs[t];
        float4 *dst = reinterpret_cast<float4 *>(const_cast<T *>(cache[t]));
        const float4 *src = reinterpret_cast<const float4 *>(a.Zo[t]);
        const int total = ta.hot[t] * nv;
        for (int q = threadIdx.x; q < total; q += blockDim.x) {
            const int r = q / nv, v = q - r * nv;
            dst[r * (cs / 4) + v] = src[r * (G::W / 4) + v];
        }
    }
    __syncthreads();

    const TmaWarpLayout &L = ta.L;
    unsigned char *base = aligned + ta.cache_bytes + warp * L.bytes;
    unsigned char *rows0 = base;
    unsigned char *idx0 = rows0 + kTmaRowSlots * L.row_slot;
    int32_t *list = reinterpret_cast<int32_t *>(idx0 + kTmaIdxSlots * TmaWarpLayout::kIdxSlot);
    tf_item *ib_items = reinterpret_cast<tf_item *>(reinterpret_cast<unsigned char *>(list) +
                                                    TmaWarpLayout::kListBytes);
    int32_t *ib_rank = reinterpret_cast<int32_t *>(ib_items + 32);
    T *own = reinterpret_cast<T *>(ib_rank + 32);
    uint64_t *rbar = reinterpret_cast<uint64_t *>(reinterpret_cast<unsigned char *>(own) + 128);
    uint64_t *ibar = rbar + kTmaRowSlots;
    if (lane == 0) {
        for (int i = 0; i < kTmaRowSlots + kTmaIdxSlots; ++i) mbar_init(rbar + i, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncwarp();
    auto islot = [&](int r) { return idx0 + r * TmaWarpLayout::kIdxSlot; };
    auto rslot = [&](int b) { return rows0 + b * L.row_slot; };
    const int n_lo = a.n, C = a.C, Cq = a.Cq;
    unsigned rpar = 0, ipar = 0;   // expected phase per slot
    unsigned rout = 0, iout = 0;   // slots with copies issued and not yet waited
    bool timed_out = false;

    T Bacc[NT], cacc[CM];
#pragma unroll
    for (int v = 0; v < NT; ++v) Bacc[v] = T(0);
#pragma unroll
    for (int c = 0; c < CM; ++c) cacc[c] = T(0);

    // Item descriptors of the current bin, 32 at a time (and the own rows' slice ranks):
    // a reload keeps the four items before the requested one, which steps still in the
    // ring may belong to.
    int64_t ib_base = 0, it0 = 0, it1 = 0;
    auto item_at = [&](int64_t it) -> const tf_item & {
        if (it < ib_base || it >= ib_base + 32) {
            ib_base = it - 4 > it0 ? it - 4 : it0;
            __syncwarp();
            const int64_t k = ib_base + lane;
            if (k < it1) {
                const tf_item x = a.items[k];
                ib_items[lane] = x;
                if (FIRST) ib_rank[lane] = a.rank_n[x.row];
            }
            __syncwarp();
        }
        return ib_items[it - ib_base];
    };
    auto step_at = [&](int64_t it) {
        Step s;
        s.it = (int32_t)it;
        if (it >= it1) {
            s.j0 = s.jend = 0;
            s.flags = 0;
            return s;
        }
        const tf_item &x = item_at(it);
        s.j0 = (int32_t)x.begin;
        s.jend = (int32_t)(x.begin + x.len);
        s.flags = 1 | 2 | ((x.len <= kWarp) ? 4 : 0);
        return s;
    };
    auto step_after = [&](const Step &s) {
        if (!(s.flags & 1)) return s;
        if (s.j0 + kWarp < s.jend) {
            Step n = s;
            n.j0 += kWarp;
            n.flags = 1 | ((n.j0 + kWarp >= n.jend) ? 4 : 0);
            return n;
        }
        return step_at((int64_t)s.it + 1);
    };

    // stage A of step s into idx slot r: index windows, residual window, own row
    auto issue_idx = [&](const Step &s, int r) {
        if (!(s.flags & 1)) return;
        const bool own_row = FIRST && (s.flags & 2);
        const int orank = own_row ? ib_rank[s.it - ib_base] : 0;
        if (lane == 0) {
            const int w0 = s.j0 & ~3;
            unsigned bytes = 3u * kTmaWin * 4u + (own_row ? 128u : 0u);
            unsigned char *d = islot(r);
            mbar_expect_tx(ibar + r, bytes);
            bulk_g2s(d, a.oidx[0] + w0, kTmaWin * 4, ibar + r);
            bulk_g2s(d + kTmaWin * 4, a.oidx[1] + w0, kTmaWin * 4, ibar + r);
            bulk_g2s(d + 2 * kTmaWin * 4, a.res + w0, kTmaWin * 4, ibar + r);
            if (own_row) bulk_g2s(d + 3 * kTmaWin * 4, a.Zn + (int64_t)orank * G::W, 128, ibar + r);
        }
        iout |= 1u << r;
    };
    // bounded wait, decided for the whole warp (every lane polls, all must succeed)
    auto wait_slot = [&](uint64_t *bar, unsigned &par, unsigned &out, int r) {
        if (timed_out) return;
        const bool ok = __all_sync(0xFFFFFFFFu, mbar_wait_bounded(bar, (par >> r) & 1u));
        if (!ok) {
            timed_out = true;
            return;
        }
        par ^= 1u << r;
        out &= ~(1u << r);
    };
    auto wait_idx = [&](int r) { wait_slot(ibar + r, ipar, iout, r); };
    // stage B of step s (its idx slot r complete) into row slot b: the step's distinct
    // uncached rows of each other mode, listed in lane order, gathered 4 at a time
    auto issue_rows = [&](const Step &s, int r, int b) {
        if (!(s.flags & 1)) return;
        const int sh = s.j0 & 3, nvalid = min(s.jend - s.j0, kWarp);
        int cnt[2];
        unsigned bytes = 0;
#pragma unroll
        for (int t = 0; t < 2; ++t) {
            const int32_t *win = reinterpret_cast<const int32_t *>(islot(r)) + t * kTmaWin;
            const int rank = win[sh + lane];
            const unsigned hm = tma_heads(rank, ta.hot[t], nvalid, lane);
            if ((hm >> lane) & 1u) list[t * 32 + __popc(hm & ((1u << lane) - 1u))] = rank;
            cnt[t] = __popc(hm);
            bytes += (unsigned)((cnt[t] + 3) >> 2) * 16u * (unsigned)ta.box[t];
        }
        __syncwarp();
        if (lane == 0) mbar_expect_tx(rbar + b, bytes);
        __syncwarp();
        if (lane < 16) {
            const int t = lane >> 3, g = lane & 7;
            const int n = t ? cnt[1] : cnt[0];
            if (4 * g < n) {
                const int32_t *li = list + t * 32;
                int y[4];
#pragma unroll
                for (int q = 0; q < 4; ++q) y[q] = li[4 * g + q < n ? 4 * g + q : 0];
                unsigned char *dst =
                    rslot(b) + (t ? L.mode1_off : 0u) + (unsigned)g * 16u * (unsigned)ta.box[t];
                gather4_g2s(dst, &ta.tm[t], 0, y[0], y[1], y[2], y[3], rbar + b);
            }
        }
        rout |= 1u << b;
    };
    auto wait_rows = [&](int b) { wait_slot(rbar + b, rpar, rout, b); };

    for (;;) {
        unsigned long long tk = 0;
        if (lane == 0) tk = atomicAdd(a.ticket, 1ull) - a.ticket_base;
        tk = __shfl_sync(0xFFFFFFFFu, tk, 0);
        if (tk >= (unsigned long long)a.P || timed_out) break;
        it0 = a.bin_ptr[tk];
        it1 = a.bin_ptr[tk + 1];
        ib_base = it0 - 64;  // forces a load at the first lookup
        // step ring (registers): steps s .. s+kTmaLeadIdx
        Step st[kTmaLeadIdx + 1];
        st[0] = step_at(it0);
#pragma unroll
        for (int k = 1; k <= kTmaLeadIdx; ++k) st[k] = step_after(st[k - 1]);
#pragma unroll
        for (int k = 0; k < kTmaLeadIdx; ++k) issue_idx(st[k], k);
#pragma unroll
        for (int k = 0; k < kTmaLeadRows; ++k) {
            if (st[k].flags & 1) {
                wait_idx(k);
                issue_rows(st[k], k, k);
            }
        }
        int is = 0, rs = 0;
        while ((st[0].flags & 1) && !timed_out) {
            {   // rows of step +kTmaLeadRows, indices of step +kTmaLeadIdx
                const Step &sb = st[kTmaLeadRows];
                const int ib = (is + kTmaLeadRows) % kTmaIdxSlots;
                const int rb = (rs + kTmaLeadRows) % kTmaRowSlots;
                if (sb.flags & 1) {
                    wait_idx(ib);
                    if (timed_out) break;
                    issue_rows(sb, ib, rb);
                }
                issue_idx(st[kTmaLeadIdx], (is + kTmaLeadIdx) % kTmaIdxSlots);
            }
            wait_rows(rs);
            if (timed_out) break;
            const Step cur = st[0];
            const unsigned char *ib = islot(is);
            if (FIRST && (cur.flags & 2)) {
                own[lane] = reinterpret_cast<const T *>(ib + 3 * kTmaWin * 4)[lane];
                __syncwarp();
            }
            const int sh = cur.j0 & 3, nvalid = min(cur.jend - cur.j0, kWarp);
            const T *rowp[2];
#pragma unroll
            for (int t = 0; t < 2; ++t) {
                const int rank = reinterpret_cast<const int32_t *>(ib)[t * kTmaWin + sh + lane];
                const unsigned hm = tma_heads(rank, ta.hot[t], nvalid, lane);
                const int pos = __popc(hm & (0xFFFFFFFFu >> (31 - lane))) - 1;
                rowp[t] = rank < ta.hot[t]
                              ? cache[t] + rank * ta.cs[t]
                              : reinterpret_cast<const T *>(rslot(rs) + (t ? L.mode1_off : 0u)) +
                                    pos * ta.box[t];
            }
            const int j = cur.j0 + lane;
            if (lane < nvalid) {
                T h[CM], po = T(0), pp = T(0);
                // own = the own slice row: prev at CM, old at 2 CM
                entry_products<T, CM, 2, FIRST, CM, 2 * CM>(rowp, own, 2, n_lo, C, Cq, h, po, pp);
                T v = reinterpret_cast<const T *>(ib + 2 * kTmaWin * 4)[sh + lane];
                if (FIRST) {
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
            if (cur.flags & 4) {
                constexpr int NB = NT + CM;
                T *p = a.partials + (int64_t)item_at(cur.it).slot * NB;
#pragma unroll
                for (int v = 0; v < NT; ++v) {
                    const T tot = warp_sum(Bacc[v]);
                    if ((v & 31) == lane) p[v] = tot;
                    Bacc[v] = T(0);
                }
#pragma unroll
                for (int c = 0; c < CM; ++c) {
                    const T tot = warp_sum(cacc[c]);
                    if (((NT + c) & 31) == lane) p[NT + c] = tot;
                    cacc[c] = T(0);
                }
            }
            __syncwarp();
#pragma unroll
            for (int k = 0; k < kTmaLeadIdx; ++k) st[k] = st[k + 1];
            st[kTmaLeadIdx] = step_after(st[kTmaLeadIdx - 1]);
            is = (is + 1) % kTmaIdxSlots;
            rs = (rs + 1) % kTmaRowSlots;
        }
        if (timed_out) break;
    }
    if (timed_out) {
        // drain what was issued (bounded) before the shared memory goes away
        for (int r = 0; r < kTmaIdxSlots; ++r)
            if (iout & (1u << r)) mbar_wait_bounded(ibar + r, (ipar >> r) & 1u);
        for (int b = 0; b < kTmaRowSlots; ++b)
            if (rout & (1u << b)) mbar_wait_bounded(rbar + b, (rpar >> b) & 1u);
        if (lane == 0) atomicOr(&a.stat->bits, kStatTimeout);
    }
}

}  // namespace tfs
