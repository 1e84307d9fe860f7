// Mode pass of a SALS split for float three-way tensors (Algorithm 1's inner loop over the
// rows of mode n, Eq. 4 per row, with the R-hat / R updates of Section 3.1 fused as in the
// cp.async pass), split into a planning kernel that runs once per row schedule and slice
// width, and the pass itself, which runs every split.
//
// The index streams of a tensor never change after it is built, so where each entry's
// other-mode rows will be in shared memory can be decided once:
//   * Hot slice rows stay in shared memory.  Slices are stored in decreasing order of their
//     rows' entry counts, so the first R rows of an other mode's slice are the rows that
//     most entries gather; each pass copies them once per block.  The host picks R per
//     other mode from the modes' degree sums so that the cached rows cover the most
//     entries that fit.
//   * The plan (k_gather_plan, gather_plan.cu) cuts each item (a row or row chunk) into
//     steps of up to 32 consecutive entries, short enough that a step's distinct cold rows
//     (rows outside the caches; consecutive equal indices are one row) fit a warp's staging
//     pool, lists those rows per step, and gives every entry one 32-bit word: where its
//     varying-mode row is (cache row or pool position) and where its run-mode row is, or
//     that the lane already holds the products of that row (the same run index as the
//     lane's previous entry).
//   * The pass (k_lean_pass) walks a bin's steps: it loads the entries' words and residuals
//     and the steps' cold-row lists three steps ahead, stages the listed rows one step
//     ahead with 16-byte cp.async (a fixed group of lanes per row), and computes: per lane,
//     products of the run-mode row with the own row's previous / old columns that stay in
//     registers while the run index holds, the Hadamard product h, the R-hat refresh, and
//     the Gram matrix, right-hand side with packed two-wide FP32 instructions
//     (fma.rn.f32x2; 2 x 2 blocks of the lower triangle).  At the end of an item the 32
//     lanes' sums are combined by a reduce-scatter (halving exchanges, fixed order) and
//     written to the item's partial slot.
#include <algorithm>
#include <numeric>

#include "gather_plan.cuh"
#include "sweep.cuh"

namespace tfs {
namespace {

// Warps per block at most: the packed-FMA Gram's per-lane accumulators grow as CM^2 and
// set the register budget (12 warps at CM = 10 and 12); the tensor-core Gram holds 8 sums
// per lane.
__host__ __device__ constexpr int lean_max_warps(int CM, int GK) {
    return (GK == 1 || GK == 3) ? 16 : (CM <= 4 ? 20 : (CM <= 8 ? 16 : 12));
}

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
__device__ __forceinline__ uint32_t to_tf32(float x) {
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return r;
}
__device__ __forceinline__ void ldsm4(unsigned addr, uint32_t &r0, uint32_t &r1, uint32_t &r2,
                                      uint32_t &r3) {
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0, %1, %2, %3}, [%4];"
                 : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3)
                 : "r"(addr));
}
// D (16 x 8, FP32) += A (16 x 8, TF32, row-major) * B (8 x 8, TF32, column-major)
__device__ __forceinline__ void mma_tf32(float (&d)[4], uint32_t a0, uint32_t a1, uint32_t a2,
                                         uint32_t a3, uint32_t b0, uint32_t b1) {
    asm volatile(
        "mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0, %1, %2, %3}, {%4, %5, %6, %7}, "
        "{%8, %9}, {%0, %1, %2, %3};"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}
__device__ __forceinline__ void sts32(unsigned a, uint32_t v) {
    asm volatile("st.shared.b32 [%0], %1;" ::"r"(a), "r"(v) : "memory");
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
//   VB = 1: the varying mode's rows come from a bfloat16 copy of its slice (16-byte
//   vectors of 8 values, widened to FP32 in registers); VB = 2: both other modes' rows;
//   the own row, products, sums and residuals stay FP32.
template <int CM, bool FIRST, int NLO, int RUN, int VB = 0>
struct LG {
    static constexpr int H = CM / 2;                          // pairs per region
    static constexpr int W = slice_stride_elems(CM, 4);       // floats per slice row
    static constexpr int V_CUR = (CM + 3) / 4, V_CP = (2 * CM + 3) / 4, V_ALL = (3 * CM + 3) / 4;
    static constexpr int VAR = 1 - RUN;
    static constexpr bool lo(int t) { return FIRST && t < NLO; }
    static constexpr bool half(int t) { return VB == 2 || (VB == 1 && t == VAR); }
    static constexpr int ncols(int t) { return FIRST ? (lo(t) ? 3 * CM : 2 * CM) : CM; }
    // 16-byte vectors fetched per row: 4 floats, or 8 bfloat16 values
    static constexpr int nv(int t) {
        return half(t) ? (ncols(t) + 7) / 8 : (FIRST ? (lo(t) ? V_ALL : V_CP) : V_CUR);
    }
    static constexpr int cs(int t) { return (nv(t) | 1) * 4; }  // staged row stride, floats
    static constexpr int NBLK = H * (H + 1) / 2;                  // 2 x 2 blocks of B
    static constexpr int NACC = 2 * NBLK + H;                     // packed accumulators
    static constexpr int NT = CM * (CM + 1) / 2;
};

constexpr int kLeanSlots = 2;        // pool slots: cold rows are staged one step ahead

// ---------------------------------------------------------------------------- the pass
// GK: how the Gram matrix and right-hand side are accumulated.  2: not at all: the loss
// pass (plain geometry, mode 0): per entry r = r_hat - <own row, h> over the slices'
// current columns, r^2 summed in FP64 per item into a.loss_out[the item's slot].  0: per
// lane, packed
// two-wide FP32 FMAs (a lane sums its own entries; the warp's sums are combined at the
// end of an item).  1 / 3: on the tensor cores (mma.sync m16n8k8, TF32 operands, FP32
// accumulation): the warp writes the step's H' = [h | r_hat] (columns 0 .. CM-1 and 15)
// transposed into shared memory, loads it as A fragments, and since the product is
// H'^T H' the B fragments are the same registers; the 16 x 16 sums are spread over the
// warp, 8 per lane, so no end-of-item reduction is needed.  1: one TF32 product per term;
// 3: three (h = hi + lo, hi hi + hi lo + lo hi), FP32-level.
constexpr int kLeanStageStride = 36;  // floats per staged H' row (conflict-free)

template <int CM, bool FIRST, int NLO, int RUN, int GK, int VB>
__global__ void __launch_bounds__(lean_max_warps(CM, GK) * kWarp, 1)
    k_lean_pass(const PassArgs<float> a, const LeanParams lp, const GStep *__restrict__ steps,
                const int32_t *__restrict__ srank, const uint32_t *__restrict__ step_range,
                const int32_t *__restrict__ list, const uint32_t *__restrict__ word) {
    using G = LG<CM, FIRST, NLO, RUN, VB>;
    constexpr int H = G::H, W = G::W, NACC = G::NACC, VAR = G::VAR;
    constexpr int NVR = G::nv(RUN), NVV = G::nv(VAR), CSR = G::cs(RUN), CSV = G::cs(VAR);
    constexpr int CSP = CSR > CSV ? CSR : CSV;  // pool row stride
    constexpr bool LOR = G::lo(RUN), LOV = G::lo(VAR);
    extern __shared__ __align__(16) float sm[];
    __shared__ short tgt[2 * NACC];  // partial-slot index of each accumulator float
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const float *ZR = a.Zo[RUN], *ZV = a.Zo[VAR];
    const uint16_t *ZVb = a.Zob[VAR], *ZRb = a.Zob[RUN];  // bfloat16 slice copies (VB)

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
                cp16(saddr(c0 + r * CS0 + 4 * v),
                     G::half(0) ? (const void *)(a.Zob[0] + (int64_t)r * a.Wb + 8 * v)
                                : (const void *)(Z0 + (int64_t)r * W + 4 * v));
            } else {
                const int qq = q - n0, r = qq / NV1, v = qq - r * NV1;
                cp16(saddr(c1 + r * CS1 + 4 * v),
                     G::half(1) ? (const void *)(a.Zob[1] + (int64_t)r * a.Wb + 8 * v)
                                : (const void *)(Z1 + (int64_t)r * W + 4 * v));
            }
        }
        cp_commit();
        cp_wait<0>();
        __syncthreads();
    }
    const unsigned cacheR = saddr(sm + lp.cache_off[RUN]), cacheV = saddr(sm + lp.cache_off[VAR]);
    const unsigned ring_s = saddr(sm + lp.ring_off + warp * lp.ring_floats);
    const unsigned str_s = ring_s + 4u * (unsigned)lp.str_off;

    u64 acc[GK == 0 ? NACC : 1];
#pragma unroll
    for (int k = 0; k < (GK == 0 ? NACC : 1); ++k) acc[k] = 0ull;
    float dg[2][4];  // tensor-core sums: columns 0-7 and 8-15 of H'^T H'
#pragma unroll
    for (int q = 0; q < 4; ++q) dg[0][q] = dg[1][q] = 0.f;
    const unsigned stage_hi = ring_s + 4u * (unsigned)lp.list_off;
    const unsigned stage_lo = stage_hi + 4u * 16u * kLeanStageStride;
    if (GK == 1 || GK == 3) {  // staged H' rows CM .. 14 stay zero
        for (int q = lane; q < 16 * kLeanStageStride * (GK == 3 ? 2 : 1); q += 32)
            sts32(stage_hi + 4u * (unsigned)q, 0u);
        __syncwarp();
    }
    // Per lane, products of the run-mode row (and the own row) that stay fixed while the
    // lane's run index does: wc = cur, wp = own prev * prev, wo = own old * old.
    u64 wc[H], wp[H], wo[H];
#pragma unroll
    for (int k = 0; k < H; ++k) wc[k] = wp[k] = wo[k] = 0ull;
    double lacc = 0.0;  // loss pass: this lane's sum of r^2

    unsigned long long tk_next = 0;
    if (lane == 0) tk_next = atomicAdd(a.ticket, 1ull) - a.ticket_base;
    tk_next = __shfl_sync(0xFFFFFFFFu, tk_next, 0);
    for (;;) {
        const unsigned long long tk = tk_next;
        if (tk >= (unsigned long long)a.P) break;
        const int s_begin = (int)step_range[2 * tk], s_end = (int)step_range[2 * tk + 1];
        if (lane == 0) tk_next = atomicAdd(a.ticket, 1ull) - a.ticket_base;
        tk_next = __shfl_sync(0xFFFFFFFFu, tk_next, 0);
        // the bin's step records, one per lane (steps wb + lane), reloaded as needed
        int wb = s_begin;
        GStep rec;
        int rrank = 0;
        auto window = [&](int base) {
            wb = base;
            rec.j0 = rec.slot = 0;
            rec.list_off = 0u;
            rec.info = 0u;
            rrank = 0;
            if (base + lane < s_end) {
                rec = steps[base + lane];
                if (FIRST || GK == 2) rrank = srank[base + lane];
            }
        };
        window(s_begin);
        // per step in flight: info (uniform), the lane's word and residual, the lane's entry
        // of the step's cold-row list
        auto info_of = [&](int s) -> uint32_t {
            return s < s_end ? __shfl_sync(0xFFFFFFFFu, rec.info, s - wb) : 0u;
        };
        // Streams in the warp's shared-memory ring (slot = step mod 4: word [32],
        // residual [32], list entries [32]), copied in with 4-byte cp.async so that no
        // register waits on a load before its step comes up.
        auto str_at = [&](int s, int arr) -> unsigned {
            return str_s + 4u * (unsigned)(((s & 3) * 3 + arr) * 32 + lane);
        };
        auto load_words = [&](int s) {
            if (s >= s_end) return;
            const uint32_t inf = __shfl_sync(0xFFFFFFFFu, rec.info, s - wb);
            const int j0 = __shfl_sync(0xFFFFFFFFu, rec.j0, s - wb);
            const int hi = (int)(inf & 63u), lo = (int)((inf >> 22) & 31u);
            if (lane >= lo && lane < hi) {
                cp4(str_at(s, 0), word + j0 + lane);
                cp4(str_at(s, 1), a.res + j0 + lane);
            }
        };
        auto load_list = [&](int s) {
            if (s >= s_end) return;
            const uint32_t inf = __shfl_sync(0xFFFFFFFFu, rec.info, s - wb);
            const uint32_t loff = __shfl_sync(0xFFFFFFFFu, rec.list_off, s - wb);
            const int nlist = (int)((inf >> 10) & 63u) + (int)((inf >> 16) & 63u);
            if (lane < nlist) cp4(str_at(s, 2), list + (size_t)loff + lane);
        };
        // stages step s's cold rows (list entries held by its lanes) into pool slot `slot`,
        // and on an item's first step the own row's prev | old regions
        auto stage = [&](int s, int slot) {
            if (s >= s_end) return;
            int li = 0;
            asm volatile("ld.shared.b32 %0, [%1];" : "=r"(li) : "r"(str_at(s, 2)));
            const uint32_t inf = __shfl_sync(0xFFFFFFFFu, rec.info, s - wb);
            const int nV = (int)((inf >> 10) & 63u), nR = (int)((inf >> 16) & 63u);
            const unsigned pool = ring_s + 4u * (unsigned)(slot * lp.slot_floats);
            {
                constexpr int RPR = 32 / NVV;
                const int sub = lane / NVV, part = lane - sub * NVV;
                for (int k0 = 0; k0 < nV; k0 += RPR) {
                    const int k = k0 + sub;
                    const int row = __shfl_sync(0xFFFFFFFFu, li, k & 31);
                    if (sub < RPR && k < nV)
                        cp16(pool + 4u * (unsigned)(k * CSP + 4 * part),
                             G::half(VAR) ? (const void *)(ZVb + (int64_t)row * a.Wb + 8 * part)
                                          : (const void *)(ZV + (int64_t)row * W + 4 * part));
                }
            }
            {
                constexpr int RPR = 32 / NVR;
                const int sub = lane / NVR, part = lane - sub * NVR;
                for (int k0 = 0; k0 < nR; k0 += RPR) {
                    const int k = nV + k0 + sub;
                    const int row = __shfl_sync(0xFFFFFFFFu, li, k & 31);
                    if (sub < RPR && k0 + sub < nR)
                        cp16(pool + 4u * (unsigned)(k * CSP + 4 * part),
                             G::half(RUN) ? (const void *)(ZRb + (int64_t)row * a.Wb + 8 * part)
                                          : (const void *)(ZR + (int64_t)row * W + 4 * part));
                }
            }
            if (FIRST && (inf & 64u)) {
                const int rk = __shfl_sync(0xFFFFFFFFu, rrank, s - wb);
                if (lane < 2 * CM)
                    cp4(ring_s + 4u * (unsigned)(lp.own_off + (int)((inf >> 8) & 3u) * 2 * CM + lane),
                        a.Zn + (int64_t)rk * W + CM + lane);
            }
            if (GK == 2 && (inf & 64u)) {  // the own row's current columns
                const int rk = __shfl_sync(0xFFFFFFFFu, rrank, s - wb);
                if (lane < CM)
                    cp4(ring_s + 4u * (unsigned)(lp.own_off + (int)((inf >> 8) & 3u) * 2 * CM + lane),
                        a.Zn + (int64_t)rk * W + lane);
            }
        };

        // Pipeline (two cp.async groups per step, the rows of the next step first, then the
        // streams): words and residuals three steps ahead, list entries four ahead, rows
        // one ahead.  At the top of step s every group but the newest is complete: the
        // rows of s (committed at step s - 1), its words (s - 3) and the list of s + 1.
        load_words(s_begin);
        load_list(s_begin);
        load_list(s_begin + 1);
        load_list(s_begin + 2);
        load_list(s_begin + 3);
        cp_commit();
        cp_wait<0>();
        __syncwarp();
        stage(s_begin, 0);
        cp_commit();
        load_words(s_begin + 1);
        load_words(s_begin + 2);
        cp_commit();
        int slot = 0;
        for (int s = s_begin; s < s_end; ++s) {
            if (s + 4 - wb >= 32) window(s);
            cp_wait<1>();
            __syncwarp();
            stage(s + 1, slot ^ 1);
            cp_commit();
            load_words(s + 3);
            load_list(s + 4);
            cp_commit();
            uint32_t w0;
            float v0;
            asm volatile("ld.shared.b32 %0, [%1];" : "=r"(w0) : "r"(str_at(s, 0)));
            asm volatile("ld.shared.f32 %0, [%1];" : "=f"(v0) : "r"(str_at(s, 1)));
            // ---------------------------------------------------------- compute step s
            const uint32_t inf = info_of(s);
            const int j0 = __shfl_sync(0xFFFFFFFFu, rec.j0, s - wb);
            const unsigned pool = ring_s + 4u * (unsigned)(slot * lp.slot_floats);
            u64 h[H];
#pragma unroll
            for (int q = 0; q < H; ++q) h[q] = 0ull;
            float v = 0.f;
            const bool act = lane >= (int)((inf >> 22) & 31u) && lane < (int)(inf & 63u);
            if (act) {
                const uint32_t locR = w0 >> 16, locV = w0 & 0xFFFFu;
                if (locR != kKeep) {
                    u64 xr[G::half(RUN) ? 4 * NVR : 2 * NVR];
                    const unsigned p = (locR & kPoolBit) ? pool + 4u * (unsigned)((locR & 0x7FFFu) * CSP)
                                                         : cacheR + 4u * (unsigned)(locR * CSR);
                    if constexpr (G::half(RUN)) {
#pragma unroll
                        for (int v = 0; v < NVR; ++v) {
                            uint32_t w[4];
                            asm volatile("ld.shared.v4.b32 {%0, %1, %2, %3}, [%4];"
                                         : "=r"(w[0]), "=r"(w[1]), "=r"(w[2]), "=r"(w[3])
                                         : "r"(p + 16 * v));
#pragma unroll
                            for (int k = 0; k < 4; ++k)
                                xr[4 * v + k] = pk(__uint_as_float(w[k] << 16),
                                                   __uint_as_float(w[k] & 0xFFFF0000u));
                        }
                    } else {
#pragma unroll
                        for (int v = 0; v < NVR; ++v) lds2(p + 16 * v, xr[2 * v], xr[2 * v + 1]);
                    }
#pragma unroll
                    for (int q = 0; q < H; ++q) wc[q] = xr[q];
                    if constexpr (FIRST) {
                        const unsigned o = ring_s + 4u * (unsigned)(lp.own_off + (int)((inf >> 8) & 3u) * 2 * CM);
#pragma unroll
                        for (int q = 0; q < H; ++q) {
                            wp[q] = mul2(lds1(o + 8 * q), xr[H + q]);
                            wo[q] = mul2(lds1(o + 8 * (H + q)), xr[(LOR ? 2 * H : 0) + q]);
                        }
                    }
                }
                u64 y[G::half(VAR) ? 4 * NVV : 2 * NVV];
                {
                    const unsigned p = (locV & kPoolBit) ? pool + 4u * (unsigned)((locV & 0x7FFFu) * CSP)
                                                         : cacheV + 4u * (unsigned)(locV * CSV);
                    if constexpr (G::half(VAR)) {
                        // 8 bfloat16 values per vector; a bfloat16 is the top half of the
                        // float it widens to
#pragma unroll
                        for (int v = 0; v < NVV; ++v) {
                            uint32_t w[4];
                            asm volatile("ld.shared.v4.b32 {%0, %1, %2, %3}, [%4];"
                                         : "=r"(w[0]), "=r"(w[1]), "=r"(w[2]), "=r"(w[3])
                                         : "r"(p + 16 * v));
#pragma unroll
                            for (int k = 0; k < 4; ++k)
                                y[4 * v + k] = pk(__uint_as_float(w[k] << 16),
                                                  __uint_as_float(w[k] & 0xFFFF0000u));
                        }
                    } else {
#pragma unroll
                        for (int v = 0; v < NVV; ++v) lds2(p + 16 * v, y[2 * v], y[2 * v + 1]);
                    }
                }
#pragma unroll
                for (int q = 0; q < H; ++q) h[q] = mul2(wc[q], y[q]);
                v = v0;
                if constexpr (FIRST) {
                    // R-hat of this split from the copy's R-hat of the previous one:
                    // v - sum_Q prod prev + sum_S prod old (Algorithm 1, Eq. 5); modes
                    // after n still hold their old columns in cur
                    u64 pp0 = 0ull, po0 = 0ull, pp1 = 0ull, po1 = 0ull;
#pragma unroll
                    for (int q = 0; q < H; q += 2) {
                        pp0 = fma2(wp[q], y[H + q], pp0);
                        po0 = fma2(wo[q], y[(LOV ? 2 * H : 0) + q], po0);
                        if (q + 1 < H) {
                            pp1 = fma2(wp[q + 1], y[H + q + 1], pp1);
                            po1 = fma2(wo[q + 1], y[(LOV ? 2 * H : 0) + q + 1], po1);
                        }
                    }
                    v = v - (hsum(pp0) + hsum(pp1)) + (hsum(po0) + hsum(po1));
                    a.res[j0 + lane] = v;
                }
                if constexpr (GK == 2) {
                    // R of this entry: the copy's r_hat less the products of the columns
                    // in the slices (beyond C they are zero)
                    const unsigned o = ring_s + 4u * (unsigned)(lp.own_off + (int)((inf >> 8) & 3u) * 2 * CM);
                    u64 pa = 0ull, pb = 0ull;
#pragma unroll
                    for (int q = 0; q < H; q += 2) {
                        pa = fma2(lds1(o + 8 * q), h[q], pa);
                        if (q + 1 < H) pb = fma2(lds1(o + 8 * (q + 1)), h[q + 1], pb);
                    }
                    const float r = v - (hsum(pa) + hsum(pb));
                    lacc += (double)r * (double)r;
                }
                if constexpr (GK == 0) {
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
            }
            if constexpr (GK == 1 || GK == 3) {
                // H' of the step (idle lanes: zeros), transposed: row f holds feature f of
                // the 32 entries; then per 8 entries one A-fragment load and two MMAs
                // (three products each for GK 3)
                {
                    float hf[2 * H];
#pragma unroll
                    for (int q = 0; q < H; ++q) upk(h[q], hf[2 * q], hf[2 * q + 1]);
#pragma unroll
                    for (int f = 0; f <= CM; ++f) {
                        const float x = f < CM ? hf[f < CM ? f : 0] : v;
                        const int row = f < CM ? f : 15;
                        const uint32_t hi = to_tf32(x);
                        sts32(stage_hi + 4u * (unsigned)(row * kLeanStageStride + lane), hi);
                        if (GK == 3)
                            sts32(stage_lo + 4u * (unsigned)(row * kLeanStageStride + lane),
                                  to_tf32(x - __uint_as_float(hi)));
                    }
                }
                __syncwarp();
                const int t = lane >> 3, r = lane & 7;
                const unsigned tile = 4u * (unsigned)((r + 8 * (t & 1)) * kLeanStageStride + 4 * (t >> 1));
#pragma unroll
                for (int kb = 0; kb < 4; ++kb) {
                    uint32_t a0, a1, a2, a3;
                    ldsm4(stage_hi + tile + 32u * kb, a0, a1, a2, a3);
                    mma_tf32(dg[0], a0, a1, a2, a3, a0, a2);
                    mma_tf32(dg[1], a0, a1, a2, a3, a1, a3);
                    if constexpr (GK == 3) {
                        uint32_t c0, c1, c2, c3;
                        ldsm4(stage_lo + tile + 32u * kb, c0, c1, c2, c3);
                        mma_tf32(dg[0], a0, a1, a2, a3, c0, c2);
                        mma_tf32(dg[1], a0, a1, a2, a3, c1, c3);
                        mma_tf32(dg[0], c0, c1, c2, c3, a0, a2);
                        mma_tf32(dg[1], c0, c1, c2, c3, a1, a3);
                    }
                }
                __syncwarp();  // the staging buffer is rewritten by the next step
            }
            if ((GK == 1 || GK == 3) && (inf & 128u)) {
                // end of item: each sum is held by one lane (the C-fragment layout)
                const int pslot = __shfl_sync(0xFFFFFFFFu, rec.slot, s - wb);
                float *p = a.partials + (int64_t)pslot * (G::NT + CM);
                const int g = lane >> 2, tg = lane & 3;
#pragma unroll
                for (int nb = 0; nb < 2; ++nb)
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        const int i = g + 8 * (q >> 1), jj = 2 * tg + (q & 1) + 8 * nb;
                        if (i < CM) {
                            if (jj == 15)
                                p[G::NT + i] = dg[nb][q];
                            else if (jj <= i)
                                p[i * (i + 1) / 2 + jj] = dg[nb][q];
                        }
                        dg[nb][q] = 0.f;
                    }
            }
            if (GK == 2 && (inf & 128u)) {
                // end of item: its sum of r^2 (butterfly: every lane holds the same value)
                // to the item's slot, so the total does not depend on which warp took it
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) lacc += __shfl_xor_sync(0xFFFFFFFFu, lacc, o);
                const int pslot = __shfl_sync(0xFFFFFFFFu, rec.slot, s - wb);
                if (lane == 0) a.loss_out[pslot] = lacc;
                lacc = 0.0;
            }
            if (GK == 0 && (inf & 128u)) {
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
                const int pslot = __shfl_sync(0xFFFFFFFFu, rec.slot, s - wb);
                float *p = a.partials + (int64_t)pslot * (G::NT + CM);
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
            slot ^= 1;
        }
        cp_wait<0>();
        __syncwarp();
    }
}

}  // namespace

bool lean_pass_supported(int CM, int N) {
    return N == 3 && (CM == 2 || CM == 4 || CM == 6 || CM == 8 || CM == 10 || CM == 12);
}

// The other mode whose index forms runs along mode n's rows: entries of a row are sorted
// by (i_{n+1}, i_{n+2}) (mode numbers mod 3), and other mode t = 0 / 1 is the lower /
// higher of the two mode numbers.
int lean_run_mode(int n) { return n == 1 ? 1 : 0; }

// Row geometry of other mode t (0 or 1) of mode n's pass: 16-byte vectors fetched, staged
// stride in floats (the kernel's LG); vb: bfloat16 rows of the varying mode (1) or of both
// other modes (2).
static void lean_geo(int CM, bool first, int n, int t, int vb, int &nv, int &cs) {
    const int cols = first ? (t < n ? 3 * CM : 2 * CM) : CM;
    const bool half = vb == 2 || (vb == 1 && t == 1 - lean_run_mode(n));
    nv = half ? (cols + 7) / 8 : (cols + 3) / 4;
    cs = (nv | 1) * 4;
}

LeanPlan lean_pass_plan(int CM, bool first, int n, const int64_t *dims_o,
                        const std::vector<int64_t> *deg_cum[2], int64_t nnz, int num_sms, int P,
                        int max_cache_rows, int pool_rows, int warps, int gk, int vb) {
    int dev = 0, smem_blk = 0;
    TFS_CUDA(cudaGetDevice(&dev));
    TFS_CUDA(cudaDeviceGetAttribute(&smem_blk, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
    LeanPlan pl;
    LeanParams &lp = pl.p;
    // row counts and pool positions are planned for the refreshing pass's rows (the widest),
    // so the plain inner iterations (narrower rows in the same counts) share its plan
    int nv[2], cs[2], nvw[2], csw[2];
    for (int t = 0; t < 2; ++t) {
        lean_geo(CM, first, n, t, vb, nv[t], cs[t]);
        lean_geo(CM, true, n, t, vb, nvw[t], csw[t]);
    }
    const int csp = std::max(cs[0], cs[1]);
    lp.cap[0] = lp.cap[1] = pool_rows;
    pl.gk = gk;
    pl.vb = vb;
    const int stage = (gk == 1 || gk == 3) ? 16 * kLeanStageStride * (gk == 3 ? 2 : 1) : 0;
    lp.slot_floats = pool_rows * csp;
    lp.own_off = kLeanSlots * lp.slot_floats;
    lp.list_off = (lp.own_off + 4 * 2 * CM + 3) / 4 * 4;  // the tensor-core staging follows
    lp.str_off = lp.list_off + stage;  // stream ring: 4 slots x (words, residuals, lists)
    lp.ring_floats = lp.str_off + 4 * 3 * 32;
    const size_t kStatic = 2048;  // the kernel's static shared memory (target table) + slack
    const int cspw = std::max(csw[0], csw[1]);
    const size_t warp_bytes =
        ((((size_t)kLeanSlots * pool_rows * cspw + 8 * CM + 3) / 4 * 4) + stage + 4 * 3 * 32) * 4;
    // as many warps as asked for (default: the most the registers allow) whose rings fit,
    // never more than the kernel's launch bound
    const int max_warps = lean_max_warps(CM, gk);
    const int fit = (int)std::min<size_t>(max_warps, ((size_t)smem_blk - kStatic) / warp_bytes);
    if (fit < 1) throw ApiError{TF_EINVAL, "lean mode pass: staging pool does not fit"};
    pl.warps = std::max(1, std::min(warps > 0 ? warps : max_warps, fit));
    const size_t ring_bytes = (size_t)pl.warps * warp_bytes;
    const size_t avail =
        (size_t)smem_blk > ring_bytes + kStatic ? smem_blk - ring_bytes - kStatic : 0;
    // cache rows: greedy in chunks of 32 rows by entries covered per byte, the run mode's
    // counted at half (its rows are read only where a lane's run index changes; at 1e8
    // entries this split of the cache took the three passes from 60.0 to 59.6 ms a sweep)
    int R[2] = {0, 0};
    size_t used = 0;
    int64_t lim[2];
    for (int t = 0; t < 2; ++t)
        lim[t] = std::min<int64_t>(std::min<int64_t>(dims_o[t], 0x7FFF),
                                   max_cache_rows < 0 ? INT32_MAX : max_cache_rows);
    for (;;) {
        int best = -1, best_rows = 0;
        double best_gain = 0.0;
        for (int t = 0; t < 2; ++t) {
            if (R[t] >= lim[t]) continue;
            const int rows = (int)std::min<int64_t>(32, lim[t] - R[t]);
            const size_t bytes = (size_t)rows * csw[t] * 4;
            if (used + bytes > avail) continue;
            const std::vector<int64_t> &dc = *deg_cum[t];
            const double gain = (double)(dc[R[t] + rows] - dc[R[t]]) / (double)bytes *
                                (t == lean_run_mode(n) ? 0.5 : 1.0);
            if (best < 0 || gain > best_gain) {
                best = t;
                best_gain = gain;
                best_rows = rows;
            }
        }
        if (best < 0) break;
        R[best] += best_rows;
        used += (size_t)best_rows * csw[best] * 4;
    }
    {
        const int var = 1 - lean_run_mode(n);
        const std::vector<int64_t> &dc = *deg_cum[var];
        pl.coverage = nnz > 0 ? (double)dc[R[var]] / (double)nnz : 1.0;
    }
    lp.R[0] = R[0];
    lp.R[1] = R[1];
    lp.cache_off[0] = 0;
    lp.cache_off[1] = R[0] * cs[0];
    lp.ring_off = (lp.cache_off[1] + R[1] * cs[1] + 3) / 4 * 4;
    pl.smem = (size_t)(lp.ring_off + pl.warps * lp.ring_floats) * 4;
    pl.grid = std::max(1, std::min(num_sms, (P + pl.warps - 1) / pl.warps));
    return pl;
}

template <int CM, bool FIRST, int NLO, int RUN, int GK, int VB>
static void launch_lean_t(const PassArgs<float> &a, const LeanPlan &pl, const GatherPlanDev &gp,
                          cudaStream_t st) {
    auto kern = k_lean_pass<CM, FIRST, NLO, RUN, GK, VB>;
    TFS_CUDA(raise_smem_limit((const void *)kern, (int)pl.smem));
    kern<<<pl.grid, pl.warps * kWarp, pl.smem, st>>>(
        a, pl.p, static_cast<const GStep *>(gp.steps), gp.rank, gp.step_range, gp.list, gp.word);
    TFS_CUDA(cudaGetLastError());
}

template <int CM, int GK, int VB>
static void launch_lean_cm(const PassArgs<float> &a, const LeanPlan &pl, const GatherPlanDev &gp,
                           cudaStream_t st) {
    if constexpr (GK == 2) {  // the loss pass: mode 0, plain geometry
        if (a.first || a.n != 0) throw ApiError{TF_EINVAL, "the lean loss pass runs mode 0's plain pass"};
        launch_lean_t<CM, false, 0, 0, 2, 0>(a, pl, gp, st);
        return;
    }
    if (!a.first) {
        if (a.n == 1)
            launch_lean_t<CM, false, 0, 1, GK, VB>(a, pl, gp, st);
        else
            launch_lean_t<CM, false, 0, 0, GK, VB>(a, pl, gp, st);
        return;
    }
    switch (a.n) {
        case 0: launch_lean_t<CM, true, 0, 0, GK, VB>(a, pl, gp, st); return;
        case 1: launch_lean_t<CM, true, 1, 1, GK, VB>(a, pl, gp, st); return;
        default: launch_lean_t<CM, true, 2, 0, GK, VB>(a, pl, gp, st); return;
    }
}

template <int CM>
static void launch_lean_gk(const PassArgs<float> &a, const LeanPlan &pl, const GatherPlanDev &gp,
                           cudaStream_t st) {
    if (pl.vb) {
        if (pl.gk != 0) throw ApiError{TF_EINVAL, "bfloat16 rows take the packed FMA Gram"};
        if (pl.vb == 2)
            launch_lean_cm<CM, 0, 2>(a, pl, gp, st);
        else
            launch_lean_cm<CM, 0, 1>(a, pl, gp, st);
        return;
    }
    switch (pl.gk) {
        case 1: launch_lean_cm<CM, 1, 0>(a, pl, gp, st); return;
        case 2: launch_lean_cm<CM, 2, 0>(a, pl, gp, st); return;
        case 3: launch_lean_cm<CM, 3, 0>(a, pl, gp, st); return;
        default: launch_lean_cm<CM, 0, 0>(a, pl, gp, st); return;
    }
}

void launch_lean_pass(const PassArgs<float> &a, int CM, const LeanPlan &pl,
                      const GatherPlanDev &gp, cudaStream_t st) {
    switch (CM) {
        case 2: launch_lean_gk<2>(a, pl, gp, st); return;
        case 4: launch_lean_gk<4>(a, pl, gp, st); return;
        case 6: launch_lean_gk<6>(a, pl, gp, st); return;
        case 8: launch_lean_gk<8>(a, pl, gp, st); return;
        case 10: launch_lean_gk<10>(a, pl, gp, st); return;
        case 12: launch_lean_gk<12>(a, pl, gp, st); return;
        default: throw ApiError{TF_EINVAL, "no lean mode-pass instance for this C"};
    }
}

}  // namespace tfs
