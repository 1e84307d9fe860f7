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
// Row solve: one block per row sums the row's slots in slot order, factors B + lambda I
// (right-looking Cholesky in shared memory, Section 3.1) and writes the row.  A
// non-positive pivot leaves the row unchanged and is counted.
#include <algorithm>

#include "sweep.cuh"

namespace tfs {
namespace {

constexpr int kWideThreads = 256;
constexpr int kWideTile = 32;        // entries per tile
constexpr int kSolveThreads = 128;

template <class T>
__device__ __forceinline__ T wsum(T v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xFFFFFFFFu, v, o);
    return v;
}

// CW: Gram tile width (32, 64 or 128), at least C + 1 (column C holds r_hat).
template <class T, int CW, bool FIRST>
__global__ void __launch_bounds__(kWideThreads) k_pass_wide(const PassArgs<T> a, int CM, int W) {
    constexpr int R = CW / 16;       // register tile edge
    constexpr int HS = CW + 4;       // H row stride (elements)
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T *H = reinterpret_cast<T *>(smem_raw);           // [kWideTile][HS]
    T *own = H + kWideTile * HS;                       // prev | old of the own row (2 CM)
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
            for (int64_t j0 = item.begin; j0 < item.begin + item.len; j0 += kWideTile) {
                const int64_t left = item.begin + item.len - j0;
                const int ne = left < kWideTile ? (int)left : kWideTile;
                __syncthreads();  // H and own are ready to be (over)written / read
                for (int e = warp; e < kWideTile; e += kWideThreads / 32) {
                    T *h = H + e * HS;
                    if (e >= ne) {
                        for (int c = lane; c < CW; c += 32) h[c] = T(0);
                        continue;
                    }
                    const int64_t jj = j0 + e;
                    const T *rows[kMaxModes - 1];
                    for (int t = 0; t < no; ++t) rows[t] = a.Zo[t] + (int64_t)a.oidx[t][jj] * W;
                    T pp = T(0), po = T(0);
                    // columns of S (< C <= CW - 1) and of the previous subset Q (< Cq <= CM)
                    const int cmax = CW > CM ? CW : CM;
                    for (int c = lane; c < cmax; c += 32) {
                        T hv = T(0);
                        if (c < C) {
                            hv = T(1);
                            for (int t = 0; t < no; ++t) hv *= rows[t][c];
                            if (FIRST) {
                                T o = own[CM + c];
                                for (int t = 0; t < no; ++t) o *= (t < n_lo ? rows[t][2 * CM + c] : rows[t][c]);
                                po += o;
                            }
                        }
                        if (FIRST && c < Cq) {
                            T p = own[c];
                            for (int t = 0; t < no; ++t) p *= rows[t][CM + c];
                            pp += p;
                        }
                        if (c < CW) h[c] = hv;
                    }
                    T v = a.res[jj];
                    if (FIRST) {
                        pp = wsum(pp);
                        po = wsum(po);
                        v = v - pp + po;
                        if (lane == 0) a.res[jj] = v;
                    }
                    __syncwarp();
                    if (lane == 0) h[C] = v;
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

// One block per row: (B + lambda I) x = c for the C x C system summed over the row's
// slots; writes x to A_n[row][S[c]] and to the cur region of the own slice row.
template <class T>
__global__ void __launch_bounds__(kSolveThreads) k_solve_wide(const PassArgs<T> a,
                                                              const SplitRow *rows, int CM, int W) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int C = a.C;
    T *B = reinterpret_cast<T *>(smem_raw);  // C x C, lower triangle used
    T *cv = B + (size_t)C * C;
    __shared__ int bad;
    const SplitRow sr = rows[blockIdx.x];
    const int tid = threadIdx.x;
    const int NT = CM * (CM + 1) / 2, NB = NT + CM;
    if (tid == 0) bad = 0;
    for (int q = tid; q < C * C; q += blockDim.x) {
        const int i = q / C, j = q - i * C;
        if (j > i) continue;
        T s = T(0);
        for (int k = 0; k < sr.n_slots; ++k)
            s += a.partials[(int64_t)(sr.first_slot + k) * NB + i * (i + 1) / 2 + j];
        B[q] = s;
    }
    for (int q = tid; q < C; q += blockDim.x) {
        T s = T(0);
        for (int k = 0; k < sr.n_slots; ++k) s += a.partials[(int64_t)(sr.first_slot + k) * NB + NT + q];
        cv[q] = s;
    }
    __syncthreads();
    const T lam = a.weighted ? a.lambda * (T)sr.len : a.lambda;
    for (int q = tid; q < C; q += blockDim.x) B[q * C + q] += lam;
    for (int j = 0; j < C; ++j) {
        __syncthreads();
        if (tid == 0) {
            T d = B[j * C + j];
            if (!(d > T(0))) {
                bad = 1;
                d = T(1);
            }
            B[j * C + j] = sqrt(d);
        }
        __syncthreads();
        const T ljj = B[j * C + j];
        for (int i = j + 1 + tid; i < C; i += blockDim.x) B[i * C + j] /= ljj;
        __syncthreads();
        const int rem = C - j - 1;
        for (int q = tid; q < rem * rem; q += blockDim.x) {
            const int i = j + 1 + q / rem, k = j + 1 + q % rem;
            if (k <= i) B[i * C + k] -= B[i * C + j] * B[k * C + j];
        }
    }
    __syncthreads();
    if (tid < 32) {
        const int lane = tid;
        for (int i = 0; i < C; ++i) {  // L y = c
            T s = T(0);
            for (int k = lane; k < i; k += 32) s += B[i * C + k] * cv[k];
            s = wsum(s);
            if (lane == 0) cv[i] = (cv[i] - s) / B[i * C + i];
            __syncwarp();
        }
        for (int i = C - 1; i >= 0; --i) {  // L^T x = y
            T s = T(0);
            for (int k = i + 1 + lane; k < C; k += 32) s += B[k * C + i] * cv[k];
            s = wsum(s);
            if (lane == 0) cv[i] = (cv[i] - s) / B[i * C + i];
            __syncwarp();
        }
    }
    __syncthreads();
    if (bad) {
        if (tid == 0) atomicAdd(&a.stat->singular_rows, 1ull);
        return;
    }
    T *z = a.Zn + (int64_t)a.rank_n[sr.row] * W;
    T *Ar = a.A_n + (int64_t)sr.row * a.K;
    for (int q = tid; q < C; q += blockDim.x) {
        z[q] = cv[q];
        Ar[a.S[q]] = cv[q];
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

template <class T, int CW>
void launch_pass_wide_cw(const PassArgs<T> &a, int CM, int W, int grid, cudaStream_t st) {
    const size_t smem = sizeof(T) * ((size_t)kWideTile * (CW + 4) + 2 * (size_t)CM);
    auto kern = a.first ? k_pass_wide<T, CW, true> : k_pass_wide<T, CW, false>;
    TFS_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    kern<<<grid, kWideThreads, smem, st>>>(a, CM, W);
    TFS_CUDA(cudaGetLastError());
}

}  // namespace

int wide_tile_width(int C) { return C + 1 <= 32 ? 32 : (C + 1 <= 64 ? 64 : (C + 1 <= 128 ? 128 : 0)); }

template <class T>
int pass_wide_grid(int num_sms, int P) {
    return std::max(1, std::min(P, num_sms * 4));
}

template <class T>
void launch_pass_wide(const PassArgs<T> &a, int CM, int W, int grid, cudaStream_t st) {
    switch (wide_tile_width(a.C)) {
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
    const size_t smem = sizeof(T) * ((size_t)a.C * a.C + a.C);
    TFS_CUDA(cudaFuncSetAttribute(k_solve_wide<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)smem));
    k_solve_wide<T><<<n_rows, kSolveThreads, smem, st>>>(a, rows, CM, W);
    TFS_CUDA(cudaGetLastError());
}

int res_wide_blocks(int P) { return (P + kWideThreads / 32 - 1) / (kWideThreads / 32); }

template <class T>
void launch_res_wide(const ResArgs<T> &a, int W, cudaStream_t st) {
    k_res_wide<T><<<res_wide_blocks(a.P), kWideThreads, 0, st>>>(a, W);
    TFS_CUDA(cudaGetLastError());
}

#define TFS_INST(T)                                                                           \
    template int pass_wide_grid<T>(int, int);                                                 \
    template void launch_pass_wide<T>(const PassArgs<T> &, int, int, int, cudaStream_t);      \
    template void launch_solve_wide<T>(const PassArgs<T> &, const SplitRow *, int, int, int,  \
                                       cudaStream_t);                                         \
    template void launch_res_wide<T>(const ResArgs<T> &, int, cudaStream_t);
TFS_INST(float)
TFS_INST(double)
#undef TFS_INST

}  // namespace tfs
