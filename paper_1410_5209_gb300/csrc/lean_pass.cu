// Mode pass of a SALS split for float three-way tensors (Algorithm 1's inner loop over the
// rows of mode n, Eq. 4 per row, with the R-hat / R updates of Section 3.1 fused as in the
// cp.async pass): the same arithmetic per entry, organised to move fewer bytes through the
// SM's load/store pipe and to issue fewer instructions.
//
//   * Hot slice rows stay in shared memory.  Slices are stored in decreasing order of their
//     rows' entry counts, so the first R rows of an other mode's slice are the rows that
//     most entries gather; a block copies them once per launch and every entry whose row
//     is among them reads it there (no global load, no staging copy).  The host picks R
//     per other mode from the modes' degree sums so that the cached rows cover the most
//     entries that fit.
//   * Rows outside the cache are staged one step ahead through a per-warp ring: the warp
//     lists the step's distinct cold rows (consecutive equal indices are one row) and
//     copies them with 16-byte cp.async, a fixed group of lanes per row.  A step with more
//     distinct cold rows than the ring holds reads the rest straight from global memory.
//   * Index and residual streams are loaded into registers two steps ahead; the item's own
//     row (its previous / old columns for the R-hat refresh) is staged with its first step.
//   * The Gram matrix, right-hand side and refresh products use packed two-wide FP32
//     instructions (fma.rn.f32x2): a lane accumulates B in 2 x 2 blocks of the lower
//     triangle.  At the end of an item the 32 lanes' sums are combined by a reduce-scatter
//     (halving exchanges, fixed order) and written to the item's partial slot.
#include <algorithm>
#include <numeric>

#include "sweep.cuh"

namespace tfs {
namespace {

constexpr int kLeanWarps = 12;
constexpr int kLeanThreads = kLeanWarps * kWarp;

typedef unsigned long long u64;

__device__ __forceinline__ u64 pk(float lo, float hi) {
    u64 r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
    return r;
}
__device__ __forceinline__ void upk(u64 v, float &lo, float &hi) {
    asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(v));
}
__device__ __forceinline__ u64 swp(u64 v) {
    float lo, hi;
    upk(v, lo, hi);
    return pk(hi, lo);
}
__device__ __forceinline__ u64 fma2(u64 a, u64 b, u64 c) {
    u64 d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}
__device__ __forceinline__ u64 mul2(u64 a, u64 b) {
    u64 d;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ float hsum(u64 v) {
    float lo, hi;
    upk(v, lo, hi);
    return lo + hi;
}
__device__ __forceinline__ unsigned saddr(const void *p) {
    return (unsigned)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void lds2(unsigned a, u64 &x, u64 &y) {
    asm volatile("ld.shared.v2.b64 {%0, %1}, [%2];" : "=l"(x), "=l"(y) : "r"(a));
}
__device__ __forceinline__ void ldg2(const float *p, u64 &x, u64 &y) {
    asm volatile("ld.global.v2.b64 {%0, %1}, [%2];" : "=l"(x), "=l"(y) : "l"(p));
}
__device__ __forceinline__ u64 lds1(unsigned a) {
    u64 x;
    asm volatile("ld.shared.b64 %0, [%1];" : "=l"(x) : "r"(a));
    return x;
}
__device__ __forceinline__ void cp16(unsigned dst, const void *src) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 16;\n" ::"r"(dst), "l"(src) : "memory");
}
__device__ __forceinline__ void cp4(unsigned dst, const void *src) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(dst), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_wait() {
    asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

// Compile-time geometry for register width CM (even) and the refresh flavour.
//   NLO other modes precede mode n (updated earlier in this split: their rows carry the
//   cur | prev | old regions); the others carry cur | prev (FIRST) or cur only.  RUN is
//   the other mode whose index forms runs along a row's entries (the first key of the
//   row's sort order), VAR the one that varies from entry to entry.
template <int CM, bool FIRST, int NLO, int RUN>
struct LG {
    static constexpr int H = CM / 2;                          // pairs per region
    static constexpr int W = slice_stride_elems(CM, 4);       // floats per slice row
    static constexpr int V_CUR = (CM + 3) / 4, V_CP = (2 * CM + 3) / 4, V_ALL = (3 * CM + 3) / 4;
    static constexpr bool lo(int t) { return FIRST && t < NLO; }
    static constexpr int nv(int t) { return FIRST ? (lo(t) ? V_ALL : V_CP) : V_CUR; }
    static constexpr int cs(int t) { return (nv(t) | 1) * 4; }  // staged row stride, floats
    static constexpr int VAR = 1 - RUN;
    static constexpr int NBLK = H * (H + 1) / 2;                  // 2 x 2 blocks of B
    static constexpr int NACC = 2 * NBLK + H;                     // packed accumulators
    static constexpr int NT = CM * (CM + 1) / 2;
};

constexpr int kLeanSlots = 3;  // ring slots: cold rows are staged two steps ahead

template <int CM, bool FIRST, int NLO, int RUN>
__global__ void __launch_bounds__(kLeanThreads, 1)
    k_lean_pass(const PassArgs<float> a, const LeanParams lp) {
    using G = LG<CM, FIRST, NLO, RUN>;
    constexpr int H = G::H, W = G::W, NACC = G::NACC, VAR = G::VAR;
    constexpr int NVR = G::nv(RUN), NVV = G::nv(VAR), CSR = G::cs(RUN), CSV = G::cs(VAR);
    constexpr bool LOR = G::lo(RUN), LOV = G::lo(VAR);
    extern __shared__ __align__(16) float sm[];
    __shared__ short tgt[2 * NACC];  // partial-slot index of each accumulator float
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const uint32_t lt_mask = (1u << lane) - 1u, le_mask = lt_mask | (1u << lane);
    const float *ZR = a.Zo[RUN], *ZV = a.Zo[VAR];
    const int32_t *ixR = a.oidx[RUN], *ixV = a.oidx[VAR];

    // accumulator layout -> partial slot index (B lower triangle, then c); -1 = unused
    for (int q = threadIdx.x; q < 2 * NACC; q += blockDim.x) {
        const int k = q >> 1, hi = q & 1;
        int v = -1;
        if (k < 2 * G::NBLK) {
            const int b = k >> 1, anti = k & 1;
            int I = 0;
            while ((I + 1) * (I + 2) / 2 <= b) ++I;
            const int J = b - I * (I + 1) / 2;
            const int i = 2 * I + hi, j = anti ? 2 * J + 1 - hi : 2 * J + hi;
            if (j <= i) v = i * (i + 1) / 2 + j;
        } else {
            v = G::NT + 2 * (k - 2 * G::NBLK) + hi;
        }
        tgt[q] = (short)v;
    }
    // hot rows of the other modes' slices -> shared memory
    {
        constexpr int NV0 = G::nv(0), NV1 = G::nv(1), CS0 = G::cs(0), CS1 = G::cs(1);
        float *c0 = sm + lp.cache_off[0], *c1 = sm + lp.cache_off[1];
        const float *Z0 = a.Zo[0], *Z1 = a.Zo[1];
        const int n0 = lp.R[0] * NV0, n1 = lp.R[1] * NV1;
        for (int q = threadIdx.x; q < n0 + n1; q += blockDim.x) {
            if (q < n0) {
                const int r = q / NV0, v = q - r * NV0;
                cp16(saddr(c0 + r * CS0 + 4 * v), Z0 + (int64_t)r * W + 4 * v);
            } else {
                const int qq = q - n0, r = qq / NV1, v = qq - r * NV1;
                cp16(saddr(c1 + r * CS1 + 4 * v), Z1 + (int64_t)r * W + 4 * v);
            }
        }
        cp_commit();
        cp_wait<0>();
        __syncthreads();
    }
    const unsigned cacheR = saddr(sm + lp.cache_off[RUN]), cacheV = saddr(sm + lp.cache_off[VAR]);
    float *ring = sm + lp.ring_off + warp * lp.ring_floats;
    int32_t *list = reinterpret_cast<int32_t *>(ring + lp.list_off);  // [2][32]
    const int RR = lp.R[RUN], RV = lp.R[VAR], capR = lp.cap[RUN], capV = lp.cap[VAR];
    const int run_off = capV * CSV;  // run-mode rows follow the varying mode's in a slot

    u64 acc[NACC];
#pragma unroll
    for (int k = 0; k < NACC; ++k) acc[k] = 0ull;
    // Per lane, products of the run-mode row (and the own row) that stay fixed while the
    // lane's run index does: wc = cur, wp = own prev * prev, wo = own old * old.
    u64 wc[H], wp[H], wo[H];
#pragma unroll
    for (int k = 0; k < H; ++k) wc[k] = wp[k] = wo[k] = 0ull;

    // The bin's items, one per lane (item wbase + lane), reloaded every 32 items.
    int64_t wbase = 0;
    int w_j0 = 0, w_len = 0, w_slot = 0, w_rank = 0;
    auto load_window = [&](int64_t base, int64_t it_end) {
        wbase = base;
        w_j0 = w_len = w_slot = w_rank = 0;
        if (base + lane < it_end) {
            const tf_item x = a.items[base + lane];
            w_j0 = (int)x.begin;
            w_len = x.len;
            w_slot = x.slot;
            if (FIRST) w_rank = a.rank_n[x.row];
        }
    };
    // Step: entries [j0, jend) of item `it`; meta: bit 0 valid, 1 first, 2 last step.
    struct St {
        int j0, jend, it, meta, slot, rank;
    };
    auto step_at = [&](int64_t it, int64_t it_end) {
        St s;
        s.it = (int)it;
        if (it >= it_end) {
            s.j0 = s.jend = s.meta = s.slot = s.rank = 0;
            return s;
        }
        if (it - wbase >= 32) load_window(it, it_end);
        const int src = (int)(it - wbase);
        s.j0 = __shfl_sync(0xFFFFFFFFu, w_j0, src);
        const int len = __shfl_sync(0xFFFFFFFFu, w_len, src);
        s.slot = __shfl_sync(0xFFFFFFFFu, w_slot, src);
        s.rank = FIRST ? __shfl_sync(0xFFFFFFFFu, w_rank, src) : 0;
        s.jend = s.j0 + len;
        s.meta = 1 | 2 | (len <= kWarp ? 4 : 0);
        return s;
    };
    auto step_next = [&](const St &s, int64_t it_end) {
        if (!(s.meta & 1)) return s;
        if (s.j0 + kWarp < s.jend) {
            St n = s;
            n.j0 += kWarp;
            n.meta = 1 | (n.j0 + kWarp >= n.jend ? 4 : 0);
            return n;
        }
        return step_at((int64_t)s.it + 1, it_end);
    };
    struct Sr {
        int iR, iV;
        float rv;
    };
    auto load_streams = [&](const St &s) {
        Sr r;
        r.iR = r.iV = -1;
        r.rv = 0.f;
        const int j = s.j0 + lane;
        if ((s.meta & 1) && j < s.jend) {
            r.iR = __ldg(ixR + j);
            r.iV = __ldg(ixV + j);
            r.rv = a.res[j];
        }
        return r;
    };
    // Step s (streams r; rp = the streams of the step before it): which lanes recompute
    // their run-mode products (nx), and the distinct cold rows that must be staged --
    // every cold varying row, and the cold run rows of lanes that recompute -- listed and
    // copied into ring slot `slot` (16-byte cp.async, a fixed lane group per row); on an
    // item's first step also the own row's prev | old regions.  hV / hR: head masks.
    struct Sm {
        uint32_t hV, hR, nx;
    };
    auto fetch = [&](const St &s, const Sr &r, const Sr &rp, int slot) {
        Sm m;
        m.hV = m.hR = m.nx = 0u;
        if (!(s.meta & 1)) return m;
        const bool valid = s.j0 + lane < s.jend;
        float *rows = ring + slot * lp.slot_floats;
        {
            const int p = __shfl_up_sync(0xFFFFFFFFu, r.iV, 1);
            const bool cold = valid && r.iV >= RV;
            m.hV = __ballot_sync(0xFFFFFFFFu, cold && (lane == 0 || p != r.iV));
            const int k = __popc(m.hV & lt_mask);
            if (((m.hV >> lane) & 1u) && k < capV) list[k] = r.iV;
        }
        {
            const bool nx = valid && ((s.meta & 2) || r.iR != rp.iR);
            m.nx = __ballot_sync(0xFFFFFFFFu, nx);
            const bool key = nx && r.iR >= RR;
            const int p = __shfl_up_sync(0xFFFFFFFFu, r.iR, 1);
            const uint32_t keys = __ballot_sync(0xFFFFFFFFu, key);
            const bool pkey = lane > 0 && ((keys >> (lane - 1)) & 1u);
            m.hR = __ballot_sync(0xFFFFFFFFu, key && (!pkey || p != r.iR));
            const int k = __popc(m.hR & lt_mask);
            if (((m.hR >> lane) & 1u) && k < capR) list[32 + k] = r.iR;
        }
        __syncwarp();
        {
            constexpr int RPR = 32 / NVV;
            const int n = min(__popc(m.hV), capV);
            const int sub = lane / NVV, part = lane - sub * NVV;
            for (int k0 = 0; k0 < n; k0 += RPR) {
                const int k = k0 + sub;
                if (sub < RPR && k < n)
                    cp16(saddr(rows + k * CSV + 4 * part), ZV + (int64_t)list[k] * W + 4 * part);
            }
        }
        {
            constexpr int RPR = 32 / NVR;
            const int n = min(__popc(m.hR), capR);
            const int sub = lane / NVR, part = lane - sub * NVR;
            for (int k0 = 0; k0 < n; k0 += RPR) {
                const int k = k0 + sub;
                if (sub < RPR && k < n)
                    cp16(saddr(rows + run_off + k * CSR + 4 * part),
                         ZR + (int64_t)list[32 + k] * W + 4 * part);
            }
        }
        if (FIRST && (s.meta & 2) && lane < 2 * CM)
            cp4(saddr(ring + lp.own_off + (s.it & 3) * 2 * CM + lane),
                a.Zn + (int64_t)s.rank * W + CM + lane);
        __syncwarp();  // the list is rewritten by the next fetch
        return m;
    };

    unsigned long long tk_next = 0;
    if (lane == 0) tk_next = atomicAdd(a.ticket, 1ull) - a.ticket_base;
    tk_next = __shfl_sync(0xFFFFFFFFu, tk_next, 0);
    for (;;) {
        const unsigned long long tk = tk_next;
        if (tk >= (unsigned long long)a.P) break;
        const int64_t it0 = a.bin_ptr[tk], it1 = a.bin_ptr[tk + 1];
        if (lane == 0) tk_next = atomicAdd(a.ticket, 1ull) - a.ticket_base;
        tk_next = __shfl_sync(0xFFFFFFFFu, tk_next, 0);
        load_window(it0, it1);

        St s0 = step_at(it0, it1);
        St s1 = step_next(s0, it1);
        St s2 = step_next(s1, it1);
        Sr r0 = load_streams(s0), r1 = load_streams(s1), r2 = load_streams(s2);
        Sm m0 = fetch(s0, r0, r0, 0);
        cp_commit();
        Sm m1 = fetch(s1, r1, r0, 1);
        cp_commit();
        int slot = 0;
        while (s0.meta & 1) {
            const St s3 = step_next(s2, it1);
            const Sr r3 = load_streams(s3);
            const int slot2 = slot + 2 >= kLeanSlots ? slot + 2 - kLeanSlots : slot + 2;
            const Sm m2 = fetch(s2, r2, r1, slot2);
            cp_commit();
            cp_wait<kLeanSlots - 1>();
            __syncwarp();
            // ---------------------------------------------------------- compute step s0
            const float *rows = ring + slot * lp.slot_floats;
            const int j = s0.j0 + lane;
            if (j < s0.jend) {
                if ((m0.nx >> lane) & 1u) {
                    u64 xr[2 * NVR];
                    const int k = __popc(m0.hR & le_mask) - 1;
                    if (r0.iR < RR) {
                        const unsigned p = cacheR + 4u * (unsigned)(r0.iR * CSR);
#pragma unroll
                        for (int v = 0; v < NVR; ++v) lds2(p + 16 * v, xr[2 * v], xr[2 * v + 1]);
                    } else if (k < capR) {
                        const unsigned p = saddr(rows + run_off) + 4u * (unsigned)(k * CSR);
#pragma unroll
                        for (int v = 0; v < NVR; ++v) lds2(p + 16 * v, xr[2 * v], xr[2 * v + 1]);
                    } else {
                        const float *p = ZR + (int64_t)r0.iR * W;
#pragma unroll
                        for (int v = 0; v < NVR; ++v) ldg2(p + 4 * v, xr[2 * v], xr[2 * v + 1]);
                    }
#pragma unroll
                    for (int q = 0; q < H; ++q) wc[q] = xr[q];
                    if constexpr (FIRST) {
                        const unsigned o = saddr(ring + lp.own_off + (s0.it & 3) * 2 * CM);
#pragma unroll
                        for (int q = 0; q < H; ++q) {
                            wp[q] = mul2(lds1(o + 8 * q), xr[H + q]);
                            wo[q] = mul2(lds1(o + 8 * (H + q)), LOR ? xr[(LOR ? 2 * H : 0) + q] : xr[q]);
                        }
                    }
                }
                u64 y[2 * NVV];
                {
                    const int k = __popc(m0.hV & le_mask) - 1;
                    if (r0.iV < RV) {
                        const unsigned p = cacheV + 4u * (unsigned)(r0.iV * CSV);
#pragma unroll
                        for (int v = 0; v < NVV; ++v) lds2(p + 16 * v, y[2 * v], y[2 * v + 1]);
                    } else if (k < capV) {
                        const unsigned p = saddr(rows) + 4u * (unsigned)(k * CSV);
#pragma unroll
                        for (int v = 0; v < NVV; ++v) lds2(p + 16 * v, y[2 * v], y[2 * v + 1]);
                    } else {
                        const float *p = ZV + (int64_t)r0.iV * W;
#pragma unroll
                        for (int v = 0; v < NVV; ++v) ldg2(p + 4 * v, y[2 * v], y[2 * v + 1]);
                    }
                }
                u64 h[H];
#pragma unroll
                for (int q = 0; q < H; ++q) h[q] = mul2(wc[q], y[q]);
                float v = r0.rv;
                if constexpr (FIRST) {
                    // R-hat of this split from the copy's R-hat of the previous one:
                    // v - sum_Q prod prev + sum_S prod old (Algorithm 1, Eq. 5); modes
                    // after n still hold their old columns in cur
                    u64 pp = 0ull, po = 0ull;
#pragma unroll
                    for (int q = 0; q < H; ++q) {
                        pp = fma2(wp[q], y[H + q], pp);
                        po = fma2(wo[q], LOV ? y[(LOV ? 2 * H : 0) + q] : y[q], po);
                    }
                    v = v - hsum(pp) + hsum(po);
                    a.res[j] = v;
                }
                const u64 vv = pk(v, v);
#pragma unroll
                for (int J = 0; J < H; ++J) {
                    const u64 hs = swp(h[J]);
#pragma unroll
                    for (int I = J; I < H; ++I) {
                        const int b = I * (I + 1) / 2 + J;
                        acc[2 * b] = fma2(h[I], h[J], acc[2 * b]);
                        acc[2 * b + 1] = fma2(h[I], hs, acc[2 * b + 1]);
                    }
                }
#pragma unroll
                for (int I = 0; I < H; ++I)
                    acc[2 * G::NBLK + I] = fma2(h[I], vv, acc[2 * G::NBLK + I]);
            }
            if (s0.meta & 4) {
                // ------------------------------------------------------ end of item
                // reduce-scatter of the 2 NACC floats over the warp (halving exchanges);
                // the lane's segment of the sums is [base, base + cnt), in f[0 .. cnt)
                float f[2 * NACC];
#pragma unroll
                for (int k = 0; k < NACC; ++k) upk(acc[k], f[2 * k], f[2 * k + 1]);
                int base = 0, cnt = 2 * NACC;
                constexpr int L0 = 2 * NACC, L1 = (L0 + 1) / 2, L2 = (L1 + 1) / 2,
                              L3 = (L2 + 1) / 2, L4 = (L3 + 1) / 2, L5 = (L4 + 1) / 2;
                auto level = [&](auto nconst, auto hconst, int o) {
                    constexpr int n = decltype(nconst)::value, hh = decltype(hconst)::value;
                    const bool up = (lane & o) != 0;
#pragma unroll
                    for (int k = 0; k < hh; ++k) {
                        const float lo = f[k], hi = (k + hh < n) ? f[k + hh] : 0.f;
                        const float send = up ? lo : hi, keep = up ? hi : lo;
                        f[k] = keep + __shfl_xor_sync(0xFFFFFFFFu, send, o);
                    }
                    if (up) {
                        base += hh;
                        cnt = cnt > hh ? cnt - hh : 0;
                    } else {
                        cnt = cnt < hh ? cnt : hh;
                    }
                };
                level(std::integral_constant<int, L0>{}, std::integral_constant<int, L1>{}, 16);
                level(std::integral_constant<int, L1>{}, std::integral_constant<int, L2>{}, 8);
                level(std::integral_constant<int, L2>{}, std::integral_constant<int, L3>{}, 4);
                level(std::integral_constant<int, L3>{}, std::integral_constant<int, L4>{}, 2);
                level(std::integral_constant<int, L4>{}, std::integral_constant<int, L5>{}, 1);
                float *p = a.partials + (int64_t)s0.slot * (G::NT + CM);
#pragma unroll
                for (int k = 0; k < L5; ++k) {
                    if (k < cnt) {
                        const int t = tgt[base + k];
                        if (t >= 0) p[t] = f[k];
                    }
                }
#pragma unroll
                for (int k = 0; k < NACC; ++k) acc[k] = 0ull;
            }
            __syncwarp();
            s0 = s1;
            s1 = s2;
            s2 = s3;
            r0 = r1;
            r1 = r2;
            r2 = r3;
            m0 = m1;
            m1 = m2;
            slot = slot + 1 >= kLeanSlots ? 0 : slot + 1;
        }
        cp_wait<0>();
        __syncwarp();
    }
}

}  // namespace

bool lean_pass_supported(int CM, int N) {
    return N == 3 && (CM == 2 || CM == 4 || CM == 6 || CM == 8 || CM == 10 || CM == 12);
}

// Row geometry of other mode t (0 or 1) of mode n's pass: vectors fetched, staged stride.
static void lean_geo(int CM, bool first, int n, int t, int &nv, int &cs) {
    const int vc = (CM + 3) / 4, vcp = (2 * CM + 3) / 4, vall = (3 * CM + 3) / 4;
    nv = first ? (t < n ? vall : vcp) : vc;
    cs = (nv | 1) * 4;
}

// The other mode whose index forms runs along mode n's rows: entries of a row are sorted
// by (i_{n+1}, i_{n+2}) (mode numbers mod 3), and other mode t = 0 / 1 is the lower /
// higher of the two mode numbers.
static int lean_run_mode(int n) { return n == 1 ? 1 : 0; }

LeanPlan lean_pass_plan(int CM, bool first, int n, const int64_t *dims_o,
                        const std::vector<int64_t> *deg_cum[2], int64_t nnz, int num_sms, int P,
                        int max_cache_rows, int ring_cap) {
    int dev = 0, smem_blk = 0;
    TFS_CUDA(cudaGetDevice(&dev));
    TFS_CUDA(cudaDeviceGetAttribute(&smem_blk, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
    LeanPlan pl;
    LeanParams &lp = pl.p;
    int nv[2], cs[2];
    for (int t = 0; t < 2; ++t) lean_geo(CM, first, n, t, nv[t], cs[t]);
    const int run = lean_run_mode(n), var = 1 - run;
    // staged rows per step: the varying mode's cold rows every step, the run mode's only
    // where a lane's run index changes
    lp.cap[var] = ring_cap;
    lp.cap[run] = std::max(1, ring_cap / 3);
    lp.slot_floats = lp.cap[var] * cs[var] + lp.cap[run] * cs[run];
    lp.own_off = kLeanSlots * lp.slot_floats;
    lp.list_off = lp.own_off + 4 * 2 * CM;
    lp.ring_floats = (lp.list_off + 64 + 3) / 4 * 4;
    pl.warps = kLeanWarps;
    const size_t kStatic = 2048;  // the kernel's static shared memory (target table) + slack
    const size_t ring_bytes = (size_t)pl.warps * lp.ring_floats * 4;
    const size_t avail =
        (size_t)smem_blk > ring_bytes + kStatic ? smem_blk - ring_bytes - kStatic : 0;
    // cache rows: greedy in chunks of 32 rows by entries covered per byte
    int R[2] = {0, 0};
    size_t used = 0;
    int64_t lim[2];
    for (int t = 0; t < 2; ++t)
        lim[t] = std::min<int64_t>(dims_o[t], max_cache_rows < 0 ? INT32_MAX : max_cache_rows);
    for (;;) {
        int best = -1, best_rows = 0;
        double best_gain = 0.0;
        for (int t = 0; t < 2; ++t) {
            if (R[t] >= lim[t]) continue;
            const int rows = (int)std::min<int64_t>(32, lim[t] - R[t]);
            const size_t bytes = (size_t)rows * cs[t] * 4;
            if (used + bytes > avail) continue;
            const std::vector<int64_t> &dc = *deg_cum[t];
            const double gain = (double)(dc[R[t] + rows] - dc[R[t]]) / (double)bytes;
            if (best < 0 || gain > best_gain) {
                best = t;
                best_gain = gain;
                best_rows = rows;
            }
        }
        if (best < 0) break;
        R[best] += best_rows;
        used += (size_t)best_rows * cs[best] * 4;
    }
    (void)nnz;
    lp.R[0] = R[0];
    lp.R[1] = R[1];
    lp.cache_off[0] = 0;
    lp.cache_off[1] = R[0] * cs[0];
    lp.ring_off = (lp.cache_off[1] + R[1] * cs[1] + 3) / 4 * 4;
    pl.smem = (size_t)(lp.ring_off + pl.warps * lp.ring_floats) * 4;
    pl.grid = std::max(1, std::min(num_sms, (P + pl.warps - 1) / pl.warps));
    return pl;
}

template <int CM, bool FIRST, int NLO, int RUN>
static void launch_lean_t(const PassArgs<float> &a, const LeanPlan &pl, cudaStream_t st) {
    auto kern = k_lean_pass<CM, FIRST, NLO, RUN>;
    TFS_CUDA(raise_smem_limit((const void *)kern, (int)pl.smem));
    kern<<<pl.grid, kLeanThreads, pl.smem, st>>>(a, pl.p);
    TFS_CUDA(cudaGetLastError());
}

template <int CM>
static void launch_lean_cm(const PassArgs<float> &a, const LeanPlan &pl, cudaStream_t st) {
    if (!a.first) {
        if (a.n == 1)
            launch_lean_t<CM, false, 0, 1>(a, pl, st);
        else
            launch_lean_t<CM, false, 0, 0>(a, pl, st);
        return;
    }
    switch (a.n) {
        case 0: launch_lean_t<CM, true, 0, 0>(a, pl, st); return;
        case 1: launch_lean_t<CM, true, 1, 1>(a, pl, st); return;
        default: launch_lean_t<CM, true, 2, 0>(a, pl, st); return;
    }
}

void launch_lean_pass(const PassArgs<float> &a, int CM, const LeanPlan &pl, cudaStream_t st) {
    switch (CM) {
        case 2: launch_lean_cm<2>(a, pl, st); return;
        case 4: launch_lean_cm<4>(a, pl, st); return;
        case 6: launch_lean_cm<6>(a, pl, st); return;
        case 8: launch_lean_cm<8>(a, pl, st); return;
        case 10: launch_lean_cm<10>(a, pl, st); return;
        case 12: launch_lean_cm<12>(a, pl, st); return;
        default: throw ApiError{TF_EINVAL, "no lean mode-pass instance for this C"};
    }
}

}  // namespace tfs
