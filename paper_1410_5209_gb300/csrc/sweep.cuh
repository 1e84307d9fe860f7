// Kernel interfaces of one SALS sweep (sweep.cu) and of the fold-in (foldin.cu).
#pragma once

#include <vector>

#include "common.cuh"

namespace tfs {

// A row and its partial slots [first_slot, first_slot + n_slots) (one slot for a row
// held by a single item; consecutive slots in entry order for a row split across bins).
struct SplitRow {
    int32_t row;
    int32_t first_slot;
    int32_t n_slots;
    int32_t pad;
    int64_t len;  // |Omega_i^(n)| (for weighted lambda)
};

// Packed slice layout, one row of W = slice_stride_elems(CM) elements per factor row i
// of mode l, stored at the row's degree rank in that mode (rows with the most entries
// first; the other-mode index streams hold ranks), where CM >= C is the register width
// the sweep was compiled for:
//   [0, C)            "cur":  a^(l)_{i,S} as updated in this split
//   [CM, CM + Cq)     "prev": a^(l)_{i,Q}, the previous split's columns (final values)
//   [2CM, 2CM + C)    "old":  a^(l)_{i,S} at the start of the split
// Residual copy n holds, for its entries in mode-n order, R-hat of the split during
// which it was last refreshed (columns Q); its first pass of a new split turns it into
// this split's R-hat: r_hat_S = r_hat_Q - sum_{c in Q} prod_l prev + sum_{c in S} prod_l old
// (Eq. 5 followed by the R-hat step of Algorithm 1, fused and done lazily per copy).
template <class T>
struct PassArgs {
    const tf_item *items;
    const int64_t *bin_ptr;
    int P;
    int N, n;       // number of modes, mode being updated
    int C, Cq;      // |S| of this split, |Q| of the previous one (Cq <= CM)
    int first;      // first inner iteration of the split: refresh R-hat
    int weighted;   // weighted lambda
    T lambda;
    const int32_t *oidx[kMaxModes - 1];  // other-mode indices, mode-n order
    const T *Zo[kMaxModes - 1];          // packed slices of those modes
    const uint16_t *Zob[kMaxModes - 1];  // their bfloat16 copies (lean pass, precision 2)
    int Wb;                              // values per row of the bfloat16 copies
    T *Zn;                               // packed slice of mode n (rows in rank order)
    const int32_t *rank_n;               // row id of mode n -> slice row (degree rank)
    T *res;                              // residual copy of mode n
    T *A_n;                              // factor matrix of mode n [I_n][K]
    int K;
    const int32_t *S;                    // the split's columns (device)
    T *partials;                         // [slots][CM(CM+1)/2 + CM]
    DeviceStatus *stat;
    unsigned long long *ticket;          // monotone bin counter shared by all passes
    unsigned long long ticket_base;      // its value when this launch starts
    // float contexts: one step of iterative refinement of every row solve (residual of the
    // system in FP64), and a new solve in FP64 of rows whose smallest pivot ratio
    // d_j / (B_jj + lambda) of the Cholesky is below 1 / cond_limit (0: never)
    int refine;
    float cond_limit;
    double *loss_out;  // lean loss pass: per-item (slot) sums of r^2 (other passes: unused)
};

template <class T>
struct PackArgs {
    int N;
    T *Z[kMaxModes];
    const T *A[kMaxModes];
    int64_t row_base[kMaxModes + 1];
    int K, W, C, Cq, off_old, off_prev;
    const int32_t *S, *Q;
    const int32_t *id_of[kMaxModes];  // slice row (rank) -> row id, per mode
};

// Residual of copy n against the columns held in the slices' "cur" region:
//   r_e = res_e - sum_{c < Cq} prod_l Z_l[i_l, c]
// what = 0: accumulate sum r^2 (double) per block; 1: out[perm[j]] = r; 2: res_e = r.
template <class T>
struct ResArgs {
    const tf_item *items;
    const int64_t *bin_ptr;
    int P;
    int N, n, Cq, what;
    const int32_t *oidx[kMaxModes - 1];
    const T *Zo[kMaxModes - 1];
    const T *Zn;
    const int32_t *rank_n;
    T *res;
    double *block_out;
    const int32_t *perm;
    T *out;
};

// res_e = x[perm[j]] - sum_k prod_l A_l[i_l, k]  (Section 3.1's residual), per copy.
template <class T>
struct InitArgs {
    const tf_item *items;
    const int64_t *bin_ptr;
    int P;
    int N, n, K, model_zero;
    const int32_t *oidx[kMaxModes - 1];   // ranks of the other modes' rows
    const int32_t *id_o[kMaxModes - 1];   // rank -> row id of those modes
    const T *Ao[kMaxModes - 1];
    const T *An;
    const T *x;
    const int32_t *perm;
    T *res;
};

template <class T>
struct FoldArgs {
    int N, K, mode;
    const T *A[kMaxModes];
    int64_t I[kMaxModes];
    int64_t m;
    const int32_t *other;
    const T *x;
    T lambda;
    T *out;
    DeviceStatus *stat;
    T *part;      // [blocks][K (K + 1) / 2 + K] partial Gram / rhs of the tiled fold-in
    // tiled fold-in of a batch: per block its entry range and request, per request its
    // first block (n_req + 1), per request a status word (1 bad index, 2 bad pivot);
    // out is then [n_req][K]
    const int64_t *blk_range;
    const int32_t *blk_req;
    const int32_t *req_blk;
    int32_t *req_status;
    // float contexts: one step of iterative refinement of every request's solve.  The
    // solve keeps its Cholesky factor in fac [n_req][K (K + 1) / 2]; a second pass over
    // the request's entries forms the residual of the normal equations,
    // c - (B + lambda I) x0 = sum_e h_e (x_e - h_e . x0) - lambda x0, in FP64 (per-block
    // partials in rpart [blocks][K]); the correction solved with the factor is added.
    int refine;
    T *fac;
    double *rpart;
};

constexpr int kPassThreads = 128;
constexpr int kCombineThreads = 512;

int pick_cm(int C);  // smallest instantiated register width >= C (0 if none); C > 16
                     // takes the wide path (wide.cu) with CM = C rounded up to 4

__host__ __device__ constexpr int next_pow2(int v) {
    int p = 1;
    while (p < v) p *= 2;
    return p;
}

// Row stride (elements) of a packed slice for register width CM: three regions of CM
// elements, padded to a power-of-two number of 16-byte vectors (so that a fixed group
// of lanes can move one row with one vector each).
__host__ __device__ constexpr int slice_stride_elems(int CM, int elem_bytes) {
    return CM <= 16 ? (16 / elem_bytes) * next_pow2((3 * CM + 16 / elem_bytes - 1) / (16 / elem_bytes))
                    : (16 / elem_bytes) * ((3 * CM + 16 / elem_bytes - 1) / (16 / elem_bytes));
}
inline int partial_stride(int CM) { return CM * (CM + 1) / 2 + CM; }

// Wide column subsets, 16 < C < 128 (wide.cu): block-per-bin mode pass with a tiled
// Gram update, block-per-row Cholesky solves, warp-per-bin residual reductions.
int wide_tile_width(int C);
int wide_split_width(int C, int CM);
template <class T>
int pass_wide_grid(int num_sms, int P, int C, int CM, bool tensor_cores, bool first);
// tensor_cores: float contexts only (tcgen05 Gram; split = three TF32 products per term,
// else one); otherwise SIMT FMAs.
template <class T>
void launch_pass_wide(const PassArgs<T> &a, int CM, int W, int grid, bool tensor_cores, bool split,
                      cudaStream_t st);
template <class T>
void launch_solve_wide(const PassArgs<T> &a, const SplitRow *rows, int n_rows, int CM, int W,
                       cudaStream_t st);
int res_wide_blocks(int P);
// Split rows of wide subsets with more than kSlotGroup partial slots: their slots are
// first summed in groups of kSlotGroup consecutive slots, one block per group, each sum
// stored in the group's first slot (groups [2 g] = first slot, [2 g + 1] = count);
// k_solve_wide then adds the group sums in order.  A partial of a wide subset holds
// C(C+1)/2 + C values, and a row split into thousands of chunks would otherwise be
// summed by one warp.
constexpr int kSlotGroup = 64;
template <class T>
void launch_sum_slot_groups(T *partials, int NB, const int32_t *groups, int n_groups,
                            cudaStream_t st);
template <class T>
void launch_res_wide(const ResArgs<T> &a, int W, cudaStream_t st);

// Launch plan of one cp.async mode pass: one block per SM, warps per block.
struct PassPlan {
    int warps = 0, grid = 0;
    size_t smem = 0;
};
template <class T>
PassPlan mode_pass_plan(int CM, int N, int n, bool first, int num_sms, int P);
template <class T>
void launch_mode_pass(const PassArgs<T> &a, int CM, const PassPlan &plan, cudaStream_t st);
template <class T>
void launch_combine(const PassArgs<T> &a, int CM, const SplitRow *rows, int n_rows,
                    cudaStream_t st);
template <class T>
void launch_solve_rows(const PassArgs<T> &a, int CM, const SplitRow *rows, int n_rows,
                       cudaStream_t st);
template <class T>
void launch_pack(const PackArgs<T> &a, cudaStream_t st);
template <class T>
void launch_res(const ResArgs<T> &a, int CM, cudaStream_t st);
// Blocks of a residual / loss launch (one warp per bin, every bin launched).
template <class T>
int res_grid(int CM, int P, int N);
// Default bins of a mode's schedule per SM.  With up to 12 warps per SM taking bins from
// a counter, 128 bins per SM (about 10 per warp, heavy rows split into chunks of at most
// |Omega| / P entries) balance the skewed workloads: measured on 1e8 Zipf entries at
// C = 10, 96.5 ms per sweep at 32 per SM, 87.1 at 128, 86.1 at 192, 87.2 at 256.
constexpr int kBinsPerSM = 128;

// Default bin count of a schedule: kBinsPerSM per SM, fewer for small tensors so that a
// bin averages at least 64 entries (at least 4 bins per SM), a multiple of the SM count.
// On 1e5 entries 128 per SM split nearly every row into chunks whose combine step
// dominated the sweep (FP64: 2.2 ms per sweep against 1.1 ms at 32 per SM).
inline int default_bins(int num_sms, int64_t nnz) {
    const int64_t hi = (int64_t)num_sms * kBinsPerSM, lo = (int64_t)num_sms * 4;
    int64_t p = nnz / 64;
    p = p < lo ? lo : (p > hi ? hi : p);
    return (int)((p + num_sms - 1) / num_sms * num_sms);
}

inline int res_blocks(int P, int warps_per_block) {
    return (P + warps_per_block - 1) / warps_per_block;
}
template <class T>
void launch_init_res(const InitArgs<T> &a, cudaStream_t st);
template <class T>
void launch_reg(const T *A, int64_t I, int K, const int64_t *off, double *block_out, int blocks,
                cudaStream_t st);
void launch_sum_blocks(const double *in, int n, double *out, cudaStream_t st);
template <class T>
void launch_init_normal(T *A, int64_t count, uint64_t seed, uint64_t stream_id, double std,
                        cudaStream_t st);
template <class T>
void launch_foldin(const FoldArgs<T> &a, cudaStream_t st);

// Model values x_hat_e = sum_k prod_n A^(n)[i_n, k] (the CP model of Eq. 1) at m
// coordinates [m][N]; an out-of-range coordinate sets kStatPredictRange (its value 0).
template <class T>
struct PredictArgs {
    int N, K;
    const T *A[kMaxModes];
    int64_t I[kMaxModes];
    int64_t m;
    const int32_t *coords;
    T *out;
    DeviceStatus *stat;
};
template <class T>
void launch_predict(const PredictArgs<T> &a, cudaStream_t st);
// Tiled fold-in (K < 128): block table of a batch of requests (offsets[n_req + 1] into
// the concatenated entries; 256 entries per block), partial buffer length, launch.
bool foldin_tiled_ok(int K);
int foldin_plan_blocks(const int64_t *offsets, int n_req, std::vector<int64_t> &blk_range,
                       std::vector<int32_t> &blk_req, std::vector<int32_t> &req_blk);
size_t foldin_part_elems(int K, int blocks);
// Refinement buffers of a tiled fold-in: returns the FP64 partial residual elements
// (blocks x K); *fac_elems receives the factor store's elements (n_req x K(K+1)/2).
size_t foldin_refine_elems(int K, int blocks, int n_req, size_t *fac_elems);
template <class T>
void launch_foldin_tiled(const FoldArgs<T> &a, int blocks, int n_req, cudaStream_t st);
template <class T>
size_t foldin_smem_bytes(int K);


// Per-launch parameters of the lean pass (host plan -> kernel).
struct LeanParams {
    int R[2];          // cached rows of each other mode (slice rows 0 .. R-1)
    int cap[2];        // staging pool rows per step (both modes together: cap[0])
    int cache_off[2];  // float offsets of the caches in dynamic shared memory
    int ring_off;      // float offset of warp 0's ring
    int ring_floats;   // floats per warp ring (pool slots, own-row buffers)
    int slot_floats;   // floats of one pool slot
    int own_off;       // float offset of the own-row buffers within a warp ring
    int list_off;      // end of the own-row buffers within a warp ring (tensor-core staging)
    int str_off;       // stream ring (words, residuals, list entries) within a warp ring
};

struct LeanPlan {
    LeanParams p;
    int warps = 0, grid = 0;
    int gk = 0;  // Gram: 0 packed FP32 FMAs, 1 one TF32 MMA product, 3 three (FP32-level)
    int vb = 0;  // bfloat16 slice rows: 1 of the varying mode, 2 of both other modes
    size_t smem = 0;
    double coverage = 0;  // entries whose varying-mode row is cached, fraction of all
};

// Device arrays of a gather plan (gather_plan.cu): per bin its records step_range[2b] ..
// step_range[2b + 1] - 1 (16-byte records), the own-row rank of each record, the records'
// cold-row lists and one location word per entry.
struct GatherPlanDev {
    const void *steps = nullptr;
    const int32_t *rank = nullptr;
    const uint32_t *step_range = nullptr;
    const int32_t *list = nullptr;
    const uint32_t *word = nullptr;
};

// Lean float pass (lean_pass.cu): three-way tensors, even register widths up to 12.
bool lean_pass_supported(int CM, int N);
int lean_run_mode(int n);  // the other mode (0 / 1) whose index forms runs in mode n's rows
// Plan of mode n's lean pass: cached rows of the two other modes chosen by entries covered
// (deg_cum[t][R] = entries whose mode-t row is among that slice's first R rows), at most
// max_cache_rows each (< 0: no limit), pool_rows staged cold rows per step, warps per block
// (0: default), gk the Gram flavour (LeanPlan::gk), vb the varying rows' type (LeanPlan::vb).
LeanPlan lean_pass_plan(int CM, bool first, int n, const int64_t *dims_o,
                        const std::vector<int64_t> *deg_cum[2], int64_t nnz, int num_sms, int P,
                        int max_cache_rows, int pool_rows, int warps, int gk, int vb);
// Values per row of a slice's bfloat16 copy (all three regions, 16-byte rows).
inline int slice_bf16_stride(int CM) { return (3 * CM + 7) / 8 * 8; }
// Zb[i][col0 .. col0 + ncols) = Z[i][same columns] rounded to bfloat16 (nearest even), i < rows.
void launch_slice_bf16(const float *Z, uint16_t *Zb, int64_t rows, int W, int Wb, int col0,
                       int ncols, cudaStream_t st);
size_t gather_plan_step_bytes();  // bytes per step record (+ its own-row rank)
// The plan of one mode in one launch.  base[b] (b <= P) counts the step units of the bins
// before b (an item of len entries has max(1, ceil(len / 32))), base[P + 1 + b] their
// entries; bin b's records go to [rmax * base[b], rmax * base[b + 1]) of steps / rank and
// its lists to [2 base[P + 1 + b], 2 base[P + 2 + b]) of list, rmax =
// plan_records_per_step(cap); range[2b], range[2b + 1] receive the bin's first and end
// record.  Overrunning a region (which the bounds exclude) sets kStatPlan.
void launch_gather_plan(const tf_item *items, const int64_t *bin_ptr, int P, const int32_t *ixR,
                        const int32_t *ixV, const int32_t *rank_n, int RR, int RV, int cap,
                        int first, const uint32_t *base, uint32_t *range, void *steps,
                        int32_t *rank, int32_t *list, uint32_t *word, DeviceStatus *stat,
                        cudaStream_t st);
void launch_lean_pass(const PassArgs<float> &a, int CM, const LeanPlan &pl,
                      const GatherPlanDev &gp, cudaStream_t st);

// TMA-fed mode pass (float, N = 3, CM <= 10; tma_pass.cuh).  A plan fixes the gather
// box width per other mode, the rows of each other mode's slice held in the block's
// shared-memory cache, and the warps per block (one block per SM).
bool tma_pass_supported(int CM, int N);
struct TmaPlan {
    int warps = 0, grid = 0;
    int box[2] = {0, 0};
    int hot[2] = {0, 0};
    bool whole[2] = {false, false};  // cached whole: never gathered, no row-slot space
    size_t smem = 0;
};
TmaPlan tma_pass_plan(int CM, bool first, const bool before_n[2], const int64_t dims_o[2],
                      int num_sms, int P);
// tmaps points at two CUtensorMap objects (the other modes' slices, box widths plan.box).
void launch_mode_pass_tma(const PassArgs<float> &a, const void *tmaps, const TmaPlan &plan,
                          int CM, bool first, const bool before_n[2], cudaStream_t st);

}  // namespace tfs
