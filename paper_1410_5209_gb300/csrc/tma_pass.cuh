// Mode pass fed by the Tensor Memory Accelerator (float, three modes, C <= 10).
//
// Same arithmetic as k_mode_pass (Eq. 4 Gram / rhs and the lazy R-hat refresh of
// Algorithm 1), different data movement: every warp keeps a ring of shared-memory
// slots filled by TMA, with one mbarrier per slot (no ordering between slots):
//   4 steps ahead: one lane issues 1D bulk copies of the step's index windows of both
//                  other modes, its residual window and (first step of an item) the own
//                  slice row;
//   2 steps ahead: 16 lanes each issue one tile::gather4 (4 slice rows of one other
//                  mode, selected by index) into the step's row slot;
//   now:           wait for the slot, compute, release it.
// Rows land densely at the box width; boxes are 8, 24 or 40 floats (a multiple of
// 8 floats keeps every 4-row destination 128-byte aligned; a row of 2 mod 4 16-byte
// vectors limits lane-per-row vector reads to 2-way bank conflicts).  Box columns past
// the slice row are zero-filled by the TMA.  Every wait is bounded: on expiry the
// kernel records kStatTimeout, drains what it issued (bounded again) and returns.
#pragma once

#include <cuda.h>

#include "mode_pass.cuh"

namespace tfs {

constexpr int kTmaLeadRows = 2, kTmaLeadIdx = 4;
constexpr int kTmaRowSlots = kTmaLeadRows + 1, kTmaIdxSlots = kTmaLeadIdx + 1;
constexpr int kTmaWin = 36;               // window entries: 32 + alignment slack (4)
constexpr int kTmaThreads = 64;           // two warps per block
constexpr long long kTmaSpinLimit = 1ll << 25;

// Box width (floats) for `need` leading floats of a slice row.
__host__ __device__ constexpr int tma_box(int need) {
    return need <= 8 ? 8 : (need <= 24 ? 24 : (need <= 40 ? 40 : 56));
}

struct TmaPassArgs {
    PassArgs<float> p;
    CUtensorMap tm[2];  // other modes' slices, box widths box[t]
    int box[2];
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

// Byte layout of one warp's ring (128-byte aligned pieces).
struct TmaLayout {
    unsigned row_slot;   // bytes of one row slot (both other modes)
    unsigned mode1_off;  // offset of mode t = 1 inside a row slot
    static constexpr unsigned kIdxSlot = 2 * kTmaWin * 4 + kTmaWin * 4 + 128 + 32;  // 592
    __host__ __device__ TmaLayout(int box0, int box1) {
        mode1_off = 32u * box0 * 4u;
        row_slot = mode1_off + 32u * box1 * 4u;
    }
    __host__ __device__ unsigned warp_bytes() const {  // a multiple of 128
        const unsigned b = kTmaRowSlots * row_slot + kTmaIdxSlots * kIdxSlot + 128 /*own*/ +
                           (kTmaRowSlots + kTmaIdxSlots) * 8;
        return (b + 127) / 128 * 128;
    }
};

template <int CM, bool FIRST>
__global__ void __launch_bounds__(kTmaThreads, 5) k_mode_pass_tma(const __grid_constant__ TmaPassArgs ta) {
    using T = float;
    using G = Geo<T, CM>;
    constexpr int NT = G::NT;
    const PassArgs<T> &a = ta.p;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const TmaLayout L(ta.box[0], ta.box[1]);
    // 128-byte aligned base (the launch reserves 128 extra bytes)
    unsigned char *aligned = reinterpret_cast<unsigned char *>(
        (reinterpret_cast<uintptr_t>(smem_raw) + 127) & ~static_cast<uintptr_t>(127));
    unsigned char *base = aligned + warp * L.warp_bytes();
    unsigned char *rows0 = base;
    unsigned char *idx0 = rows0 + kTmaRowSlots * L.row_slot;
    T *own = reinterpret_cast<T *>(idx0 + kTmaIdxSlots * TmaLayout::kIdxSlot);
    uint64_t *rbar = reinterpret_cast<uint64_t *>(reinterpret_cast<unsigned char *>(own) + 128);
    uint64_t *ibar = rbar + kTmaRowSlots;
    if (lane == 0) {
        for (int i = 0; i < kTmaRowSlots + kTmaIdxSlots; ++i) mbar_init(rbar + i, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncwarp();
    auto islot = [&](int r) { return idx0 + r * TmaLayout::kIdxSlot; };
    auto rslot = [&](int b) { return rows0 + b * L.row_slot; };
    const int n_lo = a.n, C = a.C, Cq = a.Cq;
    const unsigned row_bytes = 8u * 4u * (unsigned)(ta.box[0] + ta.box[1]) * 4u;
    unsigned rpar = 0, ipar = 0;   // expected phase per slot
    unsigned rout = 0, iout = 0;   // slots with copies issued and not yet waited
    bool timed_out = false;

    T Bacc[NT], cacc[CM];
#pragma unroll
    for (int v = 0; v < NT; ++v) Bacc[v] = T(0);
#pragma unroll
    for (int c = 0; c < CM; ++c) cacc[c] = T(0);

    // stage A of step s into idx slot r: index windows, residual window, own row
    auto issue_idx = [&](const Step &s, int r) {
        if (!(s.flags & 1)) return;
        if (lane == 0) {
            const int w0 = s.j0 & ~3;
            const bool own_row = FIRST && (s.flags & 2);
            unsigned bytes = 3u * kTmaWin * 4u + (own_row ? 128u : 0u);
            unsigned char *d = islot(r);
            mbar_expect_tx(ibar + r, bytes);
            bulk_g2s(d, a.oidx[0] + w0, kTmaWin * 4, ibar + r);
            bulk_g2s(d + kTmaWin * 4, a.oidx[1] + w0, kTmaWin * 4, ibar + r);
            bulk_g2s(d + 2 * kTmaWin * 4, a.res + w0, kTmaWin * 4, ibar + r);
            if (own_row)
                bulk_g2s(d + 3 * kTmaWin * 4, a.Zn + (int64_t)a.rank_n[a.items[s.it].row] * G::W,
                         128, ibar + r);
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
    // stage B of step s (its idx slot r complete) into row slot b
    auto issue_rows = [&](const Step &s, int r, int b) {
        if (!(s.flags & 1)) return;
        if (lane == 0) mbar_expect_tx(rbar + b, row_bytes);
        __syncwarp();
        if (lane < 16) {
            const int t = lane >> 3, g = lane & 7;
            const int32_t *win = reinterpret_cast<const int32_t *>(islot(r)) + t * kTmaWin;
            const int sh = s.j0 & 3, nvalid = min(s.jend - s.j0, kWarp);
            int y[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int e = 4 * g + q;
                y[q] = e < nvalid ? win[sh + e] : 0;
            }
            unsigned char *dst = rslot(b) + (t ? L.mode1_off : 0u) + g * 4u * ta.box[t] * 4u;
            gather4_g2s(dst, &ta.tm[t], 0, y[0], y[1], y[2], y[3], rbar + b);
        }
        rout |= 1u << b;
    };
    auto wait_rows = [&](int b) { wait_slot(rbar + b, rpar, rout, b); };

    for (;;) {
        unsigned long long tk = 0;
        if (lane == 0) tk = atomicAdd(a.ticket, 1ull) - a.ticket_base;
        tk = __shfl_sync(0xFFFFFFFFu, tk, 0);
        if (tk >= (unsigned long long)a.P || timed_out) break;
        const int64_t it0 = a.bin_ptr[tk], it1 = a.bin_ptr[tk + 1];
        // step ring (registers): steps s .. s+kTmaLeadIdx
        Step st[kTmaLeadIdx + 1];
        st[0] = step_at_item(a.items, it0, it1);
#pragma unroll
        for (int k = 1; k <= kTmaLeadIdx; ++k) st[k] = step_next(st[k - 1], a.items, it1);
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
            {   // rows of step +2 (its indices are 2 steps old), indices of step +4
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
            const int j = cur.j0 + lane;
            if (j < cur.jend) {
                const int sh = cur.j0 & 3;
                const T *rb = reinterpret_cast<const T *>(rslot(rs));
                const T *rowp[2] = {rb + lane * ta.box[0],
                                    reinterpret_cast<const T *>(rslot(rs) + L.mode1_off) +
                                        lane * ta.box[1]};
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
            if (cur.flags & 4) finish_item<T, CM>(a, cur, Bacc, cacc, lane);
            __syncwarp();
#pragma unroll
            for (int k = 0; k < kTmaLeadIdx; ++k) st[k] = st[k + 1];
            st[kTmaLeadIdx] = step_next(st[kTmaLeadIdx - 1], a.items, it1);
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
