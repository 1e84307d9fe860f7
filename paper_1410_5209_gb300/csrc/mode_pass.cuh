// The fused mode pass of a SALS split (Algorithm 1, inner loop over rows; Eq. (4)),
// and the residual / loss pass that shares its gather machinery.
//
// One warp works through the items of one bin.  For an item (a row, or a chunk of a
// row split across bins) the warp walks the row's entries 32 at a time:
//   1. each lane reads its entry's N-1 other-mode indices and its residual-copy value
//      (coalesced streams);
//   2. the warp stages the 32 entries' packed slice rows of every other mode into
//      shared memory cooperatively: 16-byte vector loads, consecutive lanes covering
//      one row, so each gathered row costs one L1 wavefront instead of one per element;
//   3. each lane forms h = prod_{l != n} a^(l)_{i_l, S} (the Hadamard product of Eq. 4)
//      from shared memory, refreshes its residual copy to this split's R-hat on the
//      first inner iteration (Algorithm 1; done lazily per copy, see PassArgs) and
//      accumulates B += h h^T (lower triangle) and c += r_hat h in registers.
// The warp then sums B and c with butterfly shuffles.  A whole row is solved right
// there: B + lambda I_C (lambda * |Omega_i| when weighted) by a register Cholesky
// (Section 3.1), and the new C parameters go to the packed slice and to A^(n).  A chunk
// writes its partial (B, c) to its slot instead; k_combine sums the slots of each
// split row in slot order (deterministic) and solves.
#pragma once

#include <algorithm>

#include "sweep.cuh"

namespace tfs {

__host__ __device__ constexpr int tri(int i, int j) { return i * (i + 1) / 2 + j; }

template <class T>
struct Vec16;
template <>
struct Vec16<float> {
    using type = float4;
};
template <>
struct Vec16<double> {
    using type = double2;
};

// Compile-time geometry of the packed slices and of the shared-memory staging.
template <class T, int CM>
struct Geo {
    static constexpr int V = 16 / (int)sizeof(T);               // elements per 16-byte vector
    static constexpr int W = slice_stride_elems(CM, sizeof(T));  // slice row stride
    static constexpr int NV = W / V;                             // vectors per row (power of 2)
    static constexpr int RS = W + V;                             // staged row stride: odd in
                                                                 // vectors -> conflict-free
    static constexpr int NV_CUR = (CM + V - 1) / V;              // vectors covering cur
    static constexpr int NV_CP = (2 * CM + V - 1) / V;           // cur|prev
    static constexpr int NV_ALL = (3 * CM + V - 1) / V;          // cur|prev|old
    static constexpr int OFF_PREV = CM, OFF_OLD = 2 * CM;
    static constexpr int NT = CM * (CM + 1) / 2;
    static_assert((NV & (NV - 1)) == 0 && NV <= 32, "slice rows must be 2^k vectors");
};

// Reads elements [OFF, OFF + CNT) of a 16-byte aligned shared-memory row with vector
// loads (the covering vectors; all offsets are compile-time).
template <class T, int OFF, int CNT>
__device__ __forceinline__ void lds_range(T (&r)[CNT], const T *row) {
    constexpr int V = 16 / (int)sizeof(T);
    constexpr int v0 = OFF / V, v1 = (OFF + CNT - 1) / V;
    T tmp[(v1 - v0 + 1) * V];
#pragma unroll
    for (int k = v0; k <= v1; ++k) {
        if constexpr (sizeof(T) == 4) {
            const float4 v = reinterpret_cast<const float4 *>(row)[k];
            tmp[(k - v0) * 4 + 0] = v.x;
            tmp[(k - v0) * 4 + 1] = v.y;
            tmp[(k - v0) * 4 + 2] = v.z;
            tmp[(k - v0) * 4 + 3] = v.w;
        } else {
            const double2 v = reinterpret_cast<const double2 *>(row)[k];
            tmp[(k - v0) * 2 + 0] = v.x;
            tmp[(k - v0) * 2 + 1] = v.y;
        }
    }
#pragma unroll
    for (int e = 0; e < CNT; ++e) r[e] = tmp[OFF - v0 * V + e];
}

template <class T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xFFFFFFFFu, v, o);
    return v;
}

// Cholesky factor, in place, of B + lam I for the leading C x C block of a CM x CM packed
// lower triangle; rows/columns >= C are replaced by the identity.  min_ratio receives the
// smallest pivot ratio d_j / (B_jj + lam) over the leading block (1 when perfectly
// conditioned, near 0 when a column is nearly a combination of the earlier ones).
// Returns false when a pivot is <= 0.
template <class T, int CM>
__device__ __forceinline__ bool chol_factor(T (&B)[CM * (CM + 1) / 2], int C, T lam,
                                            T &min_ratio) {
#pragma unroll
    for (int i = 0; i < CM; ++i) {
#pragma unroll
        for (int j = 0; j <= i; ++j) {
            T v = B[tri(i, j)];
            if (i >= C || j >= C)
                v = (i == j) ? T(1) : T(0);
            else if (i == j)
                v += lam;
            B[tri(i, j)] = v;
        }
    }
    bool ok = true;
    min_ratio = T(1);
#pragma unroll
    for (int j = 0; j < CM; ++j) {
        const T a_jj = B[tri(j, j)];
        T d = a_jj;
#pragma unroll
        for (int k = 0; k < j; ++k) d -= B[tri(j, k)] * B[tri(j, k)];
        ok = ok && (d > T(0));
        if (a_jj > T(0)) min_ratio = fmin(min_ratio, d / a_jj);
        const T ljj = sqrt(d > T(0) ? d : T(1));
        B[tri(j, j)] = ljj;
#pragma unroll
        for (int i = j + 1; i < CM; ++i) {
            T s = B[tri(i, j)];
#pragma unroll
            for (int k = 0; k < j; ++k) s -= B[tri(i, k)] * B[tri(j, k)];
            B[tri(i, j)] = s / ljj;
        }
    }
    return ok;
}

// x = (L L^T)^-1 r with the factor of chol_factor (r beyond C is ignored).
template <class T, int CM>
__device__ __forceinline__ void chol_apply(const T (&L)[CM * (CM + 1) / 2], const T (&r)[CM],
                                           int C, T (&x)[CM]) {
    T y[CM];
#pragma unroll
    for (int i = 0; i < CM; ++i) {
        T s = (i < C) ? r[i] : T(0);
#pragma unroll
        for (int k = 0; k < i; ++k) s -= L[tri(i, k)] * y[k];
        y[i] = s / L[tri(i, i)];
    }
#pragma unroll
    for (int i = CM - 1; i >= 0; --i) {
        T s = y[i];
#pragma unroll
        for (int k = i + 1; k < CM; ++k) s -= L[tri(k, i)] * x[k];
        x[i] = s / L[tri(i, i)];
    }
}

// Solves (B + lam I) x = c for the leading C x C block of a CM x CM packed lower
// triangle; rows/columns >= C are replaced by the identity (their x is 0).  B is
// overwritten by its factor.  Returns false when a pivot is <= 0 (x is then meaningless).
template <class T, int CM>
__device__ __forceinline__ bool chol_solve(T (&B)[CM * (CM + 1) / 2], const T (&c)[CM], int C,
                                           T lam, T (&x)[CM]) {
    T ratio;
    const bool ok = chol_factor<T, CM>(B, C, lam, ratio);
    chol_apply<T, CM>(B, c, C, x);
    return ok;
}

// The row solve of the mode passes (Eq. 4).  Double contexts: the Cholesky above.  Float
// contexts with a.cond_limit > 0: a row whose smallest pivot ratio is below 1 / cond_limit
// (or that has a non-positive pivot) is solved again in FP64 from the same sums; with
// a.refine: one step of iterative refinement, x += (L L^T)^-1 (c - (B + lam I) x) with the
// residual formed in FP64.  B and c are the row's sums as accumulated; B is not modified.
template <class T, int CM>
__device__ __forceinline__ bool row_solve(const PassArgs<T> &a, const T (&B)[CM * (CM + 1) / 2],
                                          const T (&c)[CM], T lam, T (&x)[CM]) {
    constexpr int NT = CM * (CM + 1) / 2;
    const int C = a.C;
    T L[NT];
#pragma unroll
    for (int q = 0; q < NT; ++q) L[q] = B[q];
    T ratio;
    bool ok = chol_factor<T, CM>(L, C, lam, ratio);
    if constexpr (sizeof(T) == 4) {
        if (a.cond_limit > 0.f && (!ok || ratio * a.cond_limit < 1.f)) {
            double Bd[NT], cd[CM], xd[CM];
#pragma unroll
            for (int q = 0; q < NT; ++q) Bd[q] = (double)B[q];
#pragma unroll
            for (int q = 0; q < CM; ++q) cd[q] = (double)c[q];
            if (!chol_solve<double, CM>(Bd, cd, C, (double)lam, xd)) return false;
#pragma unroll
            for (int q = 0; q < CM; ++q) x[q] = (T)xd[q];
            atomicAdd(&a.stat->fp64_rows, 1ull);
            return true;
        }
        if (!ok) return false;
        chol_apply<T, CM>(L, c, C, x);
        if (a.refine) {
            T r[CM], dx[CM];
#pragma unroll
            for (int i = 0; i < CM; ++i) {
                double s = (i < C) ? (double)c[i] - (double)lam * (double)x[i] : 0.0;
#pragma unroll
                for (int j = 0; j < CM; ++j) {
                    const T b = j <= i ? B[tri(i, j)] : B[tri(j, i)];
                    if (i < C && j < C) s -= (double)b * (double)x[j];
                }
                r[i] = (T)s;
            }
            chol_apply<T, CM>(L, r, C, dx);
#pragma unroll
            for (int i = 0; i < CM; ++i) x[i] += dx[i];
        }
        return true;
    } else {
        if (ok) chol_apply<T, CM>(L, c, C, x);
        return ok;
    }
}

template <class T, int CM>
__device__ __forceinline__ void write_row(const PassArgs<T> &a, int row, const T (&x)[CM]) {
    T *z = a.Zn + (int64_t)a.rank_n[row] * Geo<T, CM>::W;
    T *Ar = a.A_n + (int64_t)row * a.K;
#pragma unroll
    for (int c = 0; c < CM; ++c) {
        if (c < a.C) {
            z[c] = x[c];
            Ar[a.S[c]] = x[c];
        }
    }
}

// ----------------------------------------------------------------- warp pipeline
//
// Per warp, steps of up to 32 entries (one item, i.e. one row or row chunk, per step)
// flow through a ring in shared memory:
//   lead kLeadIdx: the other-mode indices, residual values and (first step of an item)
//                  the own row are copied in with 4/8-byte cp.async;
//   lead kLeadRows: the slice rows of the other modes are gathered with 16-byte
//                  cp.async, one fixed vector column per lane, skipping rows equal to
//                  the previous entry's (entries are sorted, so equal indices form runs);
//   lead 0: the step is computed.
// One commit group per iteration; since kLeadIdx >= 2 kLeadRows, waiting for all but
// the newest kLeadRows - 1 groups makes both this step's rows and the indices of the
// step whose rows are issued next available.
// The ring is kept shallow (rows one step ahead): the shared memory it leaves is the
// SM's L1, which serves the gathers of the hot (high-degree) slice rows; deeper rings
// and explicit row caches measured slower on Zipf-skewed tensors.

constexpr int kLeadRows = 1;
constexpr int kLeadIdx = 2;
constexpr int kRowSlots = kLeadRows + 1;
constexpr int kIdxSlots = kLeadIdx + 1;

__device__ __forceinline__ unsigned smem_addr(const void *p) {
    return (unsigned)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void cp_async16(void *dst, const void *src) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 16;\n" ::"r"(smem_addr(dst)), "l"(src)
                 : "memory");
}
template <int BYTES>
__device__ __forceinline__ void cp_async_small(void *dst, const void *src) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], %2;\n" ::"r"(smem_addr(dst)), "l"(src),
                 "n"(BYTES)
                 : "memory");
}
__device__ __forceinline__ void cp_async_commit() {
    asm volatile("cp.async.commit_group;\n" ::: "memory");
}
template <int N>
__device__ __forceinline__ void cp_async_wait() {
    asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

__host__ __device__ constexpr size_t align16(size_t b) { return (b + 15) / 16 * 16; }
__host__ __device__ constexpr int odd_up(int v) { return v | 1; }

struct Step {  // nnz < 2^31, so entry positions fit in 32 bits
    int32_t j0, jend;
    int32_t it;
    int32_t flags;  // 1 valid, 2 first step of its item, 4 last step of its item
};

__device__ __forceinline__ Step step_at_item(const tf_item *items, int64_t it, int64_t it_end) {
    Step s;
    s.it = (int32_t)it;
    if (it >= it_end) {
        s.j0 = s.jend = 0;
        s.flags = 0;
        return s;
    }
    const tf_item x = items[it];
    s.j0 = (int32_t)x.begin;
    s.jend = (int32_t)(x.begin + x.len);
    s.flags = 1 | 2 | ((x.len <= kWarp) ? 4 : 0);
    return s;
}

__device__ __forceinline__ Step step_next(const Step &s, const tf_item *items, int64_t it_end) {
    if (!(s.flags & 1)) return s;
    if (s.j0 + kWarp < s.jend) {
        Step n = s;
        n.j0 += kWarp;
        n.flags = 1 | ((n.j0 + kWarp >= n.jend) ? 4 : 0);
        return n;
    }
    return step_at_item(items, (int64_t)s.it + 1, it_end);
}

// Geometry of one pipeline flavour: NV_LO / NV_HI vectors fetched for other modes before
// / after mode n (n_lo of them are "before"); staged row strides are odd numbers of
// vectors, so 32 lanes reading one vector each of their own rows never conflict.
template <class T, int CM, int NV_LO, int NV_HI>
struct PipeGeo {
    static constexpr int V = 16 / (int)sizeof(T);
    static constexpr int RS_LO = odd_up(NV_LO) * V;
    static constexpr int RS_HI = odd_up(NV_HI) * V;
    static __host__ __device__ int lo_count(int no, int n_lo) { return no < n_lo ? no : n_lo; }
    static __host__ __device__ size_t slot_elems(int no, int n_lo) {
        const int nl = lo_count(no, n_lo);
        return (size_t)32 * (nl * RS_LO + (no - nl) * RS_HI);
    }
    static __host__ __device__ size_t mode_off(int t, int n_lo) {  // elements within a slot
        const int nl = t < n_lo ? t : n_lo;
        return (size_t)32 * (nl * RS_LO + (t - nl) * RS_HI);
    }
    static __host__ __device__ size_t rows_bytes(int no, int n_lo) {
        return align16(slot_elems(no > 0 ? no : 1, n_lo) * sizeof(T));
    }
    static __host__ __device__ size_t ridx_bytes(int no) {
        return align16((size_t)(no > 0 ? no : 1) * 32 * 4);
    }
    static constexpr size_t RV_BYTES = align16(32 * sizeof(T));
    static constexpr size_t OWN_BYTES = align16(2 * CM * sizeof(T));
    static __host__ __device__ size_t heads_bytes(int no) {
        return align16((size_t)(no > 0 ? no : 1) * 4);
    }
    static __host__ __device__ size_t warp_bytes(int no, int n_lo) {
        return kRowSlots * (rows_bytes(no, n_lo) + heads_bytes(no)) +
               kIdxSlots * (ridx_bytes(no) + RV_BYTES + OWN_BYTES + sizeof(Step)) + OWN_BYTES;
    }
};

// Warp-private views of the ring (slot pointers are computed, not stored in arrays).
template <class T, int CM, int NV_LO, int NV_HI>
struct PipeSmem {
    using PG = PipeGeo<T, CM, NV_LO, NV_HI>;
    unsigned char *rows0, *heads0, *ridx0, *rv0, *ownr0, *steps0;
    unsigned rows_b, heads_b, ridx_b;
    T *own;
    __device__ PipeSmem(unsigned char *base, int no, int n_lo) {
        rows_b = (unsigned)PG::rows_bytes(no, n_lo);
        heads_b = (unsigned)PG::heads_bytes(no);
        ridx_b = (unsigned)PG::ridx_bytes(no);
        rows0 = base;
        heads0 = rows0 + kRowSlots * rows_b;
        ridx0 = heads0 + kRowSlots * heads_b;
        rv0 = ridx0 + kIdxSlots * ridx_b;
        ownr0 = rv0 + kIdxSlots * PG::RV_BYTES;
        own = reinterpret_cast<T *>(ownr0 + kIdxSlots * PG::OWN_BYTES);
        steps0 = reinterpret_cast<unsigned char *>(own) + PG::OWN_BYTES;
    }
    __device__ __forceinline__ T *rows(int b) const {
        return reinterpret_cast<T *>(rows0 + b * rows_b);
    }
    __device__ __forceinline__ uint32_t *heads(int b) const {
        return reinterpret_cast<uint32_t *>(heads0 + b * heads_b);
    }
    __device__ __forceinline__ int32_t *ridx(int r) const {
        return reinterpret_cast<int32_t *>(ridx0 + r * ridx_b);
    }
    __device__ __forceinline__ T *rv(int r) const {
        return reinterpret_cast<T *>(rv0 + r * PG::RV_BYTES);
    }
    __device__ __forceinline__ T *ownring(int r) const {
        return reinterpret_cast<T *>(ownr0 + r * PG::OWN_BYTES);
    }
    __device__ __forceinline__ Step *step(int r) const {
        return reinterpret_cast<Step *>(steps0) + r;
    }
};

// Where the other modes' index streams and slices are: read from the kernel
// parameters when the number of other modes is a compile-time constant (every index
// is then a constant), from a shared-memory table otherwise (no local-memory copy of
// the parameter arrays).
template <class T, int NO>
struct OtherModes {
    const int32_t *const *oidx;
    const T *const *Zo;
    int no;
    __device__ __forceinline__ int count() const { return NO > 0 ? NO : no; }
};

// Indices, residual values, and (first step of an item) the own row's elements
// [own_off, own_off + own_len) of the own slice.
template <class T, int CM, int NO>
__device__ __forceinline__ void issue_idx(const Step &s, int32_t *ridx, T *rv, T *ownring,
                                          const OtherModes<T, NO> &om, const T *res,
                                          const tf_item *items, const T *Zn, const int32_t *rank_n,
                                          int own_off, int own_len, int lane) {
    if (!(s.flags & 1)) return;
    const int j = s.j0 + lane;
    if (j < s.jend) {
        const int no = om.count();
#pragma unroll(NO > 0 ? NO : 1)
        for (int t = 0; t < no; ++t) cp_async_small<4>(ridx + t * 32 + lane, om.oidx[t] + j);
        cp_async_small<sizeof(T)>(rv + lane, res + j);
    }
    if ((s.flags & 2) && lane < own_len) {
        const int64_t row = rank_n[items[s.it].row];
        cp_async_small<sizeof(T)>(ownring + lane, Zn + row * Geo<T, CM>::W + own_off + lane);
    }
}

// The slice rows of a step: for each other mode, entry r's row unless it equals entry
// r-1's (then entry r reads the run head's staged row).  Records the run heads.
template <class T, int CM, int NV_LO, int NV_HI, int NO>
__device__ __forceinline__ void issue_rows(const Step &s, T *rows, uint32_t *heads,
                                           const int32_t *ridx, const OtherModes<T, NO> &om,
                                           int n_lo, int lane) {
    using G = Geo<T, CM>;
    using PG = PipeGeo<T, CM, NV_LO, NV_HI>;
    constexpr int RPR = 32 / G::NV;  // rows per round
    if (!(s.flags & 1)) return;
    const int nvalid = min(s.jend - s.j0, kWarp);
    const int no = om.count();
    const int part = lane & (G::NV - 1), rsub = lane / G::NV;
#pragma unroll(NO > 0 ? NO : 1)
    for (int t = 0; t < no; ++t) {
        const int32_t *ri = ridx + t * 32;
        const int mine = ri[lane], before = lane > 0 ? ri[lane - 1] : -1;
        const uint32_t hm =
            __ballot_sync(0xFFFFFFFFu, lane < nvalid && (lane == 0 || mine != before));
        if (lane == 0) heads[t] = hm;
        const bool lo = t < n_lo;
        const int need = lo ? NV_LO : NV_HI, rs = lo ? PG::RS_LO : PG::RS_HI;
        if (part >= need) continue;
        T *dst = rows + PG::mode_off(t, n_lo) + rsub * rs + part * G::V;
        const T *Z = om.Zo[t] + part * G::V;
#pragma unroll
        for (int k = 0; k < G::NV; ++k) {
            const int row = k * RPR + rsub;
            if ((hm >> row) & 1u)
                cp_async16(dst + k * RPR * rs, Z + (int64_t)ri[row] * G::W);
        }
    }
}

// Staged row of other mode t that entry `lane` reads: the head of its run.
__device__ __forceinline__ int run_head(uint32_t heads, int lane) {
    const uint32_t upto = heads & (0xFFFFFFFFu >> (31 - lane));
    return 31 - __clz(upto);
}

// End of an item: warp-sum (B, c) with butterflies and store them in the item's
// partial slot (the solves run afterwards, all rows in parallel: k_solve_rows /
// k_combine).  Lane k stores values k, k + 32, ...; the summation order is fixed.
template <class T, int CM>
__device__ __forceinline__ void finish_item(const PassArgs<T> &a, const Step &s,
                                            T (&Bacc)[CM * (CM + 1) / 2], T (&cacc)[CM],
                                            int lane) {
    constexpr int NT = CM * (CM + 1) / 2, NB = NT + CM;
    T *p = a.partials + (int64_t)a.items[s.it].slot * NB;
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

// Per-entry arithmetic of the mode pass on staged rows.  rowp[t] points at the staged
// row of other mode t that this entry reads.  Returns h (zero beyond C) and, on the
// first inner iteration, the products that refresh R-hat: po = sum_{c<C} prod_l old_l[c]
// (own old included) and pp = sum_{c<Cq} prod_l prev_l[c].  Other modes t >= n_lo come
// after mode n and have not been updated in this split: their "old" is their "cur".
// own is 16-byte aligned; its prev / old regions start at OWN_PREV / OWN_OLD.
template <class T, int CM, int NO, bool FIRST, int OWN_PREV = 0, int OWN_OLD = CM>
__device__ __forceinline__ void entry_products(const T *const (&rowp)[(NO > 0 ? NO : kMaxModes - 1)],
                                               const T *own, int no, int n_lo, int C, int Cq,
                                               T (&h)[CM], T &po, T &pp) {
    using G = Geo<T, CM>;
    constexpr int OP = G::OFF_PREV, OO = G::OFF_OLD;
    if constexpr (NO == 2) {
        const T *r0 = rowp[0], *r1 = rowp[1];
        {
            T x[CM], y[CM];
            lds_range<T, 0, CM>(x, r0);
            lds_range<T, 0, CM>(y, r1);
#pragma unroll
            for (int c = 0; c < CM; ++c) h[c] = (c < C) ? x[c] * y[c] : T(0);
        }
        if constexpr (FIRST) {
            {
                T x[CM], y[CM], o[CM];
                lds_range<T, OP, CM>(x, r0);
                lds_range<T, OP, CM>(y, r1);
                lds_range<T, OWN_PREV, CM>(o, own);
                pp = T(0);
#pragma unroll
                for (int c = 0; c < CM; ++c)
                    if (c < Cq) pp += o[c] * (x[c] * y[c]);
            }
            {
                T o[CM];
                lds_range<T, OWN_OLD, CM>(o, own);
                po = T(0);
                if (n_lo == 0) {  // both other modes after n: old == cur, so po = own_old . h
#pragma unroll
                    for (int c = 0; c < CM; ++c) po += o[c] * h[c];
                } else {
                    T x[CM], y[CM];
                    lds_range<T, OO, CM>(x, r0);
                    if (n_lo > 1)
                        lds_range<T, OO, CM>(y, r1);
                    else
                        lds_range<T, 0, CM>(y, r1);
#pragma unroll
                    for (int c = 0; c < CM; ++c)
                        if (c < C) po += o[c] * (x[c] * y[c]);
                }
            }
        }
    } else {
        T x[CM];
#pragma unroll
        for (int c = 0; c < CM; ++c) h[c] = T(1);
#pragma unroll(NO > 0 ? NO : 1)
        for (int t = 0; t < (NO > 0 ? NO : no); ++t) {
            lds_range<T, 0, CM>(x, rowp[t]);
#pragma unroll
            for (int c = 0; c < CM; ++c) h[c] *= x[c];
        }
#pragma unroll
        for (int c = 0; c < CM; ++c)
            if (c >= C) h[c] = T(0);
        if constexpr (FIRST) {
            T q[CM];
            lds_range<T, OWN_PREV, CM>(q, own);  // own prev
#pragma unroll(NO > 0 ? NO : 1)
            for (int t = 0; t < (NO > 0 ? NO : no); ++t) {
                lds_range<T, OP, CM>(x, rowp[t]);
#pragma unroll
                for (int c = 0; c < CM; ++c) q[c] *= x[c];
            }
            pp = T(0);
#pragma unroll
            for (int c = 0; c < CM; ++c)
                if (c < Cq) pp += q[c];
            lds_range<T, OWN_OLD, CM>(q, own);  // own old
#pragma unroll(NO > 0 ? NO : 1)
            for (int t = 0; t < (NO > 0 ? NO : no); ++t) {
                if (t < n_lo)
                    lds_range<T, OO, CM>(x, rowp[t]);
                else
                    lds_range<T, 0, CM>(x, rowp[t]);
#pragma unroll
                for (int c = 0; c < CM; ++c) q[c] *= x[c];
            }
            po = T(0);
#pragma unroll
            for (int c = 0; c < CM; ++c)
                if (c < C) po += q[c];
        }
    }
}

// Drives one bin through the ring; Consumer does the per-step work:
//   c.item_begin(sm, step, idx_slot)   first step of an item (own row is in the ring)
//   c.entry(sm, step, row_slot, idx_slot, lane)
//   c.item_end(step)                   last step of an item
template <class T, int CM, int NV_LO, int NV_HI, int NO, class Consumer>
__device__ __forceinline__ void run_bin(const tf_item *items, int64_t it0, int64_t it1,
                                        const OtherModes<T, NO> &om, const T *res, const T *Zn,
                                        const int32_t *rank_n, int n_lo, int own_off, int own_len,
                                        bool fetch_rows,
                                        PipeSmem<T, CM, NV_LO, NV_HI> &sm, Consumer &cons,
                                        int lane) {
    // prologue: steps 0 .. kLeadIdx-1 (indices), then rows of steps 0 .. kLeadRows-1
    Step gen = step_at_item(items, it0, it1);
#pragma unroll
    for (int k = 0; k < kLeadIdx; ++k) {
        if (lane == 0) *sm.step(k) = gen;
        issue_idx<T, CM, NO>(gen, sm.ridx(k), sm.rv(k), sm.ownring(k), om, res, items, Zn, rank_n,
                             own_off, own_len, lane);
        gen = step_next(gen, items, it1);
    }
    cp_async_commit();
    cp_async_wait<0>();
    __syncwarp();
#pragma unroll
    for (int k = 0; k < kLeadRows; ++k) {
        if (fetch_rows) {
            const Step sk = *sm.step(k);
            issue_rows<T, CM, NV_LO, NV_HI, NO>(sk, sm.rows(k), sm.heads(k), sm.ridx(k), om, n_lo,
                                                lane);
        }
        cp_async_commit();
    }
    int is = 0, rs = 0;  // ring slots of the step computed now
    for (;;) {
        cp_async_wait<kLeadRows - 1>();
        __syncwarp();
        const Step cur = *sm.step(is);
        if (!(cur.flags & 1)) break;
        // rows of step +kLeadRows, indices of step +kLeadIdx
        {
            const int ib = (is + kLeadRows) % kIdxSlots, rb = (rs + kLeadRows) % kRowSlots;
            if (fetch_rows) {
                const Step sb = *sm.step(ib);
                issue_rows<T, CM, NV_LO, NV_HI, NO>(sb, sm.rows(rb), sm.heads(rb), sm.ridx(ib), om,
                                                    n_lo, lane);
            }
            const int ia = (is + kLeadIdx) % kIdxSlots;
            __syncwarp();  // everyone has read slot ia's step before it is replaced
            if (lane == 0) *sm.step(ia) = gen;
            issue_idx<T, CM, NO>(gen, sm.ridx(ia), sm.rv(ia), sm.ownring(ia), om, res, items, Zn,
                                 rank_n, own_off, own_len, lane);
            gen = step_next(gen, items, it1);
            cp_async_commit();
        }
        if (cur.flags & 2) cons.item_begin(sm, cur, is, lane);
        cons.entry(sm, cur, rs, is, lane);
        if (cur.flags & 4) cons.item_end(cur, lane);
        __syncwarp();
        is = (is + 1) % kIdxSlots;
        rs = (rs + 1) % kRowSlots;
    }
    cp_async_wait<0>();
    __syncwarp();
}

template <class T, int CM, int NO, bool FIRST>
struct PassConsumer {
    using G = Geo<T, CM>;
    static constexpr int NV_LO = FIRST ? G::NV_ALL : G::NV_CUR;  // cur|prev|old
    static constexpr int NV_HI = FIRST ? G::NV_CP : G::NV_CUR;   // cur|prev
    using PG = PipeGeo<T, CM, NV_LO, NV_HI>;
    using SM = PipeSmem<T, CM, NV_LO, NV_HI>;
    const PassArgs<T> &a;
    int no, n_lo;
    T Bacc[G::NT], cacc[CM];
    __device__ PassConsumer(const PassArgs<T> &a_, int no_, int n_lo_) : a(a_), no(no_), n_lo(n_lo_) {
#pragma unroll
        for (int v = 0; v < G::NT; ++v) Bacc[v] = T(0);
#pragma unroll
        for (int c = 0; c < CM; ++c) cacc[c] = T(0);
    }
    __device__ __forceinline__ void item_begin(const SM &sm, const Step &, int is, int lane) {
        if (FIRST) {
            if (lane < 2 * CM) sm.own[lane] = sm.ownring(is)[lane];
            __syncwarp();
        }
    }
    __device__ __forceinline__ void entry(const SM &sm, const Step &st, int rs, int is, int lane) {
        const int j = st.j0 + lane;
        if (j >= st.jend) return;
        const T *slot = sm.rows(rs);
        const uint32_t *hd = sm.heads(rs);
        constexpr int NP = NO > 0 ? NO : kMaxModes - 1;
        const T *rowp[NP];
#pragma unroll
        for (int t = 0; t < NP; ++t) {
            if (t < no) {
                const int rsz = t < n_lo ? PG::RS_LO : PG::RS_HI;
                rowp[t] = slot + PG::mode_off(t, n_lo) + run_head(hd[t], lane) * rsz;
            } else {
                rowp[t] = slot;
            }
        }
        T h[CM], po = T(0), pp = T(0);
        entry_products<T, CM, NO, FIRST>(rowp, sm.own, no, n_lo, a.C, a.Cq, h, po, pp);
        T v = sm.rv(is)[lane];
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
    __device__ __forceinline__ void item_end(const Step &st, int lane) {
        finish_item<T, CM>(a, st, Bacc, cacc, lane);
    }
};

template <class T, int NO>
__device__ __forceinline__ OtherModes<T, NO> other_modes(const int32_t *const *p_oidx,
                                                         const T *const *p_Zo, int N,
                                                         const int32_t **s_oidx,
                                                         const T **s_Zo) {
    OtherModes<T, NO> om;
    om.no = N - 1;
    if constexpr (NO > 0) {
        om.oidx = p_oidx;
        om.Zo = p_Zo;
    } else {
        if (threadIdx.x < kMaxModes - 1) {
            s_oidx[threadIdx.x] = p_oidx[threadIdx.x];
            s_Zo[threadIdx.x] = p_Zo[threadIdx.x];
        }
        __syncthreads();
        om.oidx = s_oidx;
        om.Zo = s_Zo;
    }
    return om;
}

// Bytes of one warp's ring for a mode pass of mode n (n_lo = n other modes before it).
template <class T, int CM, bool FIRST>
__host__ __device__ size_t pass_warp_bytes(int N, int n) {
    using G = Geo<T, CM>;
    using PG = PipeGeo<T, CM, FIRST ? G::NV_ALL : G::NV_CUR, FIRST ? G::NV_CP : G::NV_CUR>;
    return PG::warp_bytes(N - 1, n);
}

// Warps per block of the mode pass (one block per SM): as many as the registers of the
// per-lane Gram accumulators allow without spilling (the accumulators grow as CM^2).
template <class T, int CM>
constexpr int pass_max_warps() {
    return sizeof(T) == 4 ? (CM <= 2 ? 24 : (CM <= 4 ? 20 : (CM <= 8 ? 16 : 12))) : (CM <= 4 ? 12 : 8);
}

// NO: number of other modes (N - 1) when specialised, 0 for any N (runtime loops).
// FIRST: the split's first inner iteration (R-hat refresh) or a later one.
// One block per SM (the staging rings are small, so most of the SM's shared memory
// stays L1 cache: the hottest slice rows are served from there).
template <class T, int CM, int NO, bool FIRST>
__global__ void __launch_bounds__(pass_max_warps<T, CM>() * kWarp, 1)
    k_mode_pass(const PassArgs<T> a) {
    using Cons = PassConsumer<T, CM, NO, FIRST>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ const int32_t *s_oidx[kMaxModes - 1];
    __shared__ const T *s_Zo[kMaxModes - 1];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const OtherModes<T, NO> om = other_modes<T, NO>(a.oidx, a.Zo, a.N, s_oidx, s_Zo);
    const int no = a.N - 1, n_lo = a.n;
    typename Cons::SM sm(smem_raw + warp * pass_warp_bytes<T, CM, FIRST>(a.N, a.n), no, n_lo);
    Cons cons(a, no, n_lo);
    // own row: prev|old regions, [CM, 3 CM) of the own slice row (first iteration only)
    const int own_len = FIRST ? 2 * CM : 0;
    // Bins are fetched dynamically (one ticket per fetch): which warp runs a bin does
    // not change any result, only the load balance.
    for (;;) {
        unsigned long long tk = 0;
        if (lane == 0) tk = atomicAdd(a.ticket, 1ull) - a.ticket_base;
        tk = __shfl_sync(0xFFFFFFFFu, tk, 0);
        if (tk >= (unsigned long long)a.P) break;
        const int bin = (int)tk;
        run_bin<T, CM, Cons::NV_LO, Cons::NV_HI, NO>(a.items, a.bin_ptr[bin], a.bin_ptr[bin + 1],
                                                     om, a.res, a.Zn, a.rank_n, n_lo, CM, own_len,
                                                     true, sm, cons, lane);
    }
}

// Rows held by a single item: one thread per row reads its slot and solves
// (B + lambda I) a = c (Eq. 4) by the register Cholesky of Section 3.1.
// XS: the solve options of float contexts (refinement / FP64 fallback) are on; the plain
// Cholesky otherwise, so that the default kernels carry none of their registers.
template <class T, int CM, bool XS>
__global__ void __launch_bounds__(128) k_solve_rows(const PassArgs<T> a, const SplitRow *rows,
                                                    int n_rows) {
    constexpr int NT = CM * (CM + 1) / 2, NB = NT + CM;
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= n_rows) return;
    const SplitRow sr = rows[r];
    const T *p = a.partials + (int64_t)sr.first_slot * NB;
    T B[NT], c[CM], x[CM];
#pragma unroll
    for (int q = 0; q < NT; ++q) B[q] = p[q];
#pragma unroll
    for (int q = 0; q < CM; ++q) c[q] = p[NT + q];
    const T lam = a.weighted ? a.lambda * (T)sr.len : a.lambda;
    if (XS ? row_solve<T, CM>(a, B, c, lam, x) : chol_solve<T, CM>(B, c, a.C, lam, x))
        write_row<T, CM>(a, sr.row, x);
    else
        atomicAdd(&a.stat->singular_rows, 1ull);
}

template <class T, int CM, bool XS>
__global__ void __launch_bounds__(kCombineThreads) k_combine(const PassArgs<T> a,
                                                             const SplitRow *rows) {
    constexpr int NT = CM * (CM + 1) / 2, NB = NT + CM;
    constexpr int G = kCombineThreads / NB;
    __shared__ T red[G * NB];
    __shared__ T tot[NB];
    const SplitRow sr = rows[blockIdx.x];
    const int t = threadIdx.x, g = t / NB, v = t - g * NB;
    if (g < G) {
        T s = T(0);
        for (int k = g; k < sr.n_slots; k += G)
            s += a.partials[(int64_t)(sr.first_slot + k) * NB + v];
        red[t] = s;
    }
    __syncthreads();
    if (t < NB) {
        T s = T(0);
        for (int gg = 0; gg < G; ++gg) s += red[gg * NB + t];
        tot[t] = s;
    }
    __syncthreads();
    if (t == 0) {
        T B[NT], c[CM], x[CM];
#pragma unroll
        for (int q = 0; q < NT; ++q) B[q] = tot[q];
#pragma unroll
        for (int q = 0; q < CM; ++q) c[q] = tot[NT + q];
        const T lam = a.weighted ? a.lambda * (T)sr.len : a.lambda;
        if (XS ? row_solve<T, CM>(a, B, c, lam, x) : chol_solve<T, CM>(B, c, a.C, lam, x))
            write_row<T, CM>(a, sr.row, x);
        else
            atomicAdd(&a.stat->singular_rows, 1ull);
    }
}

// Residual of copy n against the columns held in the slices' "cur" region (the last
// split's final values): r = res - sum_{c < Cq} prod_l Z_l[i_l, c].  One warp per bin,
// every bin launched (the per-block double sums are then in a fixed order); the same
// warp pipeline as the mode pass feeds it.
template <class T, int CM>
struct ResConsumer {
    using G = Geo<T, CM>;
    static constexpr int NV_LO = G::NV_CUR, NV_HI = G::NV_CUR;
    using PG = PipeGeo<T, CM, NV_LO, NV_HI>;
    using SM = PipeSmem<T, CM, NV_LO, NV_HI>;
    const ResArgs<T> &a;
    int no;
    double acc = 0.0;
    __device__ ResConsumer(const ResArgs<T> &a_, int no_) : a(a_), no(no_) {}
    __device__ __forceinline__ void item_begin(const SM &sm, const Step &, int is, int lane) {
        if (a.Cq > 0) {
            if (lane < CM) sm.own[lane] = sm.ownring(is)[lane];
            __syncwarp();
        }
    }
    __device__ __forceinline__ void entry(const SM &sm, const Step &st, int rs, int is, int lane) {
        const int j = st.j0 + lane;
        if (j >= st.jend) return;
        T p = T(0);
        if (a.Cq > 0) {
            const T *slot = sm.rows(rs);
            const uint32_t *hd = sm.heads(rs);
            T q[CM], x[CM];
            lds_range<T, 0, CM>(q, sm.own);
            for (int t = 0; t < no; ++t) {
                lds_range<T, 0, CM>(x, slot + PG::mode_off(t, no) + run_head(hd[t], lane) * PG::RS_LO);
#pragma unroll
                for (int c = 0; c < CM; ++c) q[c] *= x[c];
            }
#pragma unroll
            for (int c = 0; c < CM; ++c)
                if (c < a.Cq) p += q[c];
        }
        const T r = sm.rv(is)[lane] - p;
        if (a.what == 0)
            acc += (double)r * (double)r;
        else if (a.what == 1)
            a.out[a.perm[j]] = r;
        else
            a.res[j] = r;
    }
    __device__ __forceinline__ void item_end(const Step &, int) {}
};

template <class T, int CM>
__host__ __device__ size_t res_warp_bytes(int N) {
    using G = Geo<T, CM>;
    return PipeGeo<T, CM, G::NV_CUR, G::NV_CUR>::warp_bytes(N - 1, N - 1);
}

template <class T, int CM>
__global__ void __launch_bounds__(kPassThreads) k_res(const ResArgs<T> a) {
    using Cons = ResConsumer<T, CM>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ double wsum[kPassThreads / kWarp];
    __shared__ const int32_t *s_oidx[kMaxModes - 1];
    __shared__ const T *s_Zo[kMaxModes - 1];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int no = a.N - 1;
    const OtherModes<T, 0> om = other_modes<T, 0>(a.oidx, a.Zo, a.N, s_oidx, s_Zo);
    typename Cons::SM sm(smem_raw + warp * res_warp_bytes<T, CM>(a.N), no, no);
    Cons cons(a, no);
    const int bin = (int)(((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5);
    if (bin < a.P)
        run_bin<T, CM, Cons::NV_LO, Cons::NV_HI, 0>(a.items, a.bin_ptr[bin], a.bin_ptr[bin + 1], om,
                                                    a.res, a.Zn, a.rank_n, no, 0, a.Cq > 0 ? CM : 0,
                                                    a.Cq > 0, sm, cons, lane);
    if (a.what != 0) return;
    const double acc = warp_sum_d(cons.acc);
    if (lane == 0) wsum[warp] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int w = 0; w < (int)(blockDim.x / kWarp); ++w) s += wsum[w];
        a.block_out[blockIdx.x] = s;
    }
}

// Warps per block of the pipelined kernels: the count (1, 2 or 4) that puts the most
// warps on an SM given the per-warp ring size (at least one).
inline int best_warps_per_block(size_t warp_bytes) {
    int dev = 0, smem_sm = 0, smem_blk = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
    cudaDeviceGetAttribute(&smem_blk, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    int best = 1, best_total = 0;
    for (int w = kPassThreads / kWarp; w >= 1; w /= 2) {
        const size_t blk = w * warp_bytes + 1024;  // + static shared memory / reserve
        if (blk > (size_t)smem_blk) continue;
        const int total = w * std::min(32 / w, (int)(smem_sm / blk));
        if (total > best_total) {
            best_total = total;
            best = w;
        }
    }
    return best;
}

// Three- and five-way tensors get the number of other modes as a compile-time constant
// (fully unrolled mode loops); other orders run the generic kernel.
template <class T, int CM>
auto mode_pass_kernel(int N, bool first) {
    if (N == 3) return first ? k_mode_pass<T, CM, 2, true> : k_mode_pass<T, CM, 2, false>;
    if constexpr (sizeof(T) == 4)
        if (N == 5) return first ? k_mode_pass<T, CM, 4, true> : k_mode_pass<T, CM, 4, false>;
    return first ? k_mode_pass<T, CM, 0, true> : k_mode_pass<T, CM, 0, false>;
}

// Plan of a mode-n pass: one block per SM with as many warps as fit (up to
// pass_max_warps); the shared memory the rings leave is L1 cache.
template <class T, int CM, bool FIRST>
PassPlan mode_pass_plan_cm(int N, int n, int num_sms, int P) {
    constexpr size_t kReserve = 1024;  // static shared memory of the kernel
    int dev = 0, smem_blk = 0;
    TFS_CUDA(cudaGetDevice(&dev));
    TFS_CUDA(cudaDeviceGetAttribute(&smem_blk, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
    const size_t ring = pass_warp_bytes<T, CM, FIRST>(N, n);
    PassPlan plan;
    plan.warps = (int)std::min<size_t>(pass_max_warps<T, CM>(), ((size_t)smem_blk - kReserve) / ring);
    if (plan.warps < 1) throw ApiError{TF_EINVAL, "mode pass does not fit in shared memory"};
    plan.smem = (size_t)plan.warps * ring;
    plan.grid = std::max(1, std::min(num_sms, (P + plan.warps - 1) / plan.warps));
    return plan;
}

template <class T, int CM>
void launch_mode_pass_cm(const PassArgs<T> &a, const PassPlan &plan, cudaStream_t st) {
    auto kern = mode_pass_kernel<T, CM>(a.N, a.first != 0);
    TFS_CUDA(raise_smem_limit((const void *)kern, (int)plan.smem));
    kern<<<plan.grid, plan.warps * kWarp, plan.smem, st>>>(a);
    TFS_CUDA(cudaGetLastError());
}

template <class T, int CM>
void launch_combine_cm(const PassArgs<T> &a, const SplitRow *rows, int n_rows, cudaStream_t st) {
    if (n_rows <= 0) return;
    if (sizeof(T) == 4 && (a.refine || a.cond_limit > 0.f))
        k_combine<T, CM, true><<<n_rows, kCombineThreads, 0, st>>>(a, rows);
    else
        k_combine<T, CM, false><<<n_rows, kCombineThreads, 0, st>>>(a, rows);
    TFS_CUDA(cudaGetLastError());
}

template <class T, int CM>
void launch_solve_rows_cm(const PassArgs<T> &a, const SplitRow *rows, int n_rows,
                          cudaStream_t st) {
    if (n_rows <= 0) return;
    if (sizeof(T) == 4 && (a.refine || a.cond_limit > 0.f))
        k_solve_rows<T, CM, true><<<(n_rows + 127) / 128, 128, 0, st>>>(a, rows, n_rows);
    else
        k_solve_rows<T, CM, false><<<(n_rows + 127) / 128, 128, 0, st>>>(a, rows, n_rows);
    TFS_CUDA(cudaGetLastError());
}

template <class T, int CM>
int res_warps(int N) {
    return best_warps_per_block(res_warp_bytes<T, CM>(N));
}

template <class T, int CM>
void launch_res_cm(const ResArgs<T> &a, cudaStream_t st) {
    const int wpb = res_warps<T, CM>(a.N);
    const size_t smem = wpb * res_warp_bytes<T, CM>(a.N);
    TFS_CUDA(raise_smem_limit((const void *)k_res<T, CM>, (int)smem));
    k_res<T, CM><<<res_blocks(a.P, wpb), wpb * kWarp, smem, st>>>(a);
    TFS_CUDA(cudaGetLastError());
}

template <class T, int CM>
int res_blocks_cm(int P, int N) {
    return res_blocks(P, res_warps<T, CM>(N));
}

#define TFS_FOR_EACH_CM(X) X(1) X(2) X(4) X(6) X(8) X(10) X(12) X(16)

template <class T>
void launch_mode_pass_impl(const PassArgs<T> &a, int CM, const PassPlan &plan, cudaStream_t st) {
    switch (CM) {
#define TFS_CASE(cm)                             \
    case cm:                                     \
        launch_mode_pass_cm<T, cm>(a, plan, st); \
        return;
        TFS_FOR_EACH_CM(TFS_CASE)
#undef TFS_CASE
        default:
            throw ApiError{TF_EINVAL, "no mode-pass instance for this C"};
    }
}

template <class T>
PassPlan mode_pass_plan_impl(int CM, int N, int n, bool first, int num_sms, int P) {
    switch (CM) {
#define TFS_CASE(cm)                                                       \
    case cm:                                                               \
        return first ? mode_pass_plan_cm<T, cm, true>(N, n, num_sms, P)    \
                     : mode_pass_plan_cm<T, cm, false>(N, n, num_sms, P);
        TFS_FOR_EACH_CM(TFS_CASE)
#undef TFS_CASE
        default:
            throw ApiError{TF_EINVAL, "no mode-pass instance for this C"};
    }
}

template <class T>
void launch_combine_impl(const PassArgs<T> &a, int CM, const SplitRow *rows, int n_rows,
                         cudaStream_t st) {
    switch (CM) {
#define TFS_CASE(cm)                                   \
    case cm:                                           \
        launch_combine_cm<T, cm>(a, rows, n_rows, st); \
        return;
        TFS_FOR_EACH_CM(TFS_CASE)
#undef TFS_CASE
        default:
            throw ApiError{TF_EINVAL, "no combine instance for this C"};
    }
}

template <class T>
void launch_solve_rows_impl(const PassArgs<T> &a, int CM, const SplitRow *rows, int n_rows,
                            cudaStream_t st) {
    switch (CM) {
#define TFS_CASE(cm)                                       \
    case cm:                                               \
        launch_solve_rows_cm<T, cm>(a, rows, n_rows, st);  \
        return;
        TFS_FOR_EACH_CM(TFS_CASE)
#undef TFS_CASE
        default:
            throw ApiError{TF_EINVAL, "no solve instance for this C"};
    }
}

template <class T>
void launch_res_impl(const ResArgs<T> &a, int CM, cudaStream_t st) {
    switch (CM) {
#define TFS_CASE(cm)                 \
    case cm:                         \
        launch_res_cm<T, cm>(a, st); \
        return;
        TFS_FOR_EACH_CM(TFS_CASE)
#undef TFS_CASE
        default:
            if (CM > 16) {
                launch_res_wide<T>(a, slice_stride_elems(CM, (int)sizeof(T)), st);
                return;
            }
            throw ApiError{TF_EINVAL, "no residual instance for this C"};
    }
}

template <class T>
int res_blocks_impl(int CM, int P, int N) {
    switch (CM) {
#define TFS_CASE(cm) \
    case cm:         \
        return res_blocks_cm<T, cm>(P, N);
        TFS_FOR_EACH_CM(TFS_CASE)
#undef TFS_CASE
        default:
            if (CM > 16) return res_wide_blocks(P);
            throw ApiError{TF_EINVAL, "no residual instance for this C"};
    }
}

}  // namespace tfs
