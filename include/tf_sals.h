/*
 * tf_sals.h -- C ABI of the GB300 SALS / CDTF library.
 *
 * The library factorises a partially observed N-way tensor X (observed set Omega)
 * into factor matrices A^(1..N) (each I_n x K) by Subset Alternating Least Squares
 * (SALS) and its C = 1 special case CDTF, after Shin & Kang, "Distributed Methods
 * for High-dimensional and Large-scale Tensor Factorization" (arXiv 1410.5209):
 *   loss  L = sum_{Omega} (x - sum_k prod_n a^(n)_{i_n k})^2 + lambda sum_n ||A^(n)||_F^2   (Eq. 1)
 * One call of tf_sals_sweep is one outer iteration of Algorithm 1.
 *
 * Conventions shared by every entry point
 *   - Indices are 0-based.  Coordinates are int32, row-major [nnz][N].
 *   - Factor matrices are row-major [I_n][K] in the context's dtype (float or double).
 *   - Every call returns a tf_status and never aborts, traps or exits.  Errors found
 *     on the device are recorded in a device status word that the next synchronising
 *     call (tf_loss, tf_get_*, tf_sync) reads back.  tf_last_error() describes the
 *     most recent failure in words.
 *   - Inputs are copied: the caller keeps ownership of every buffer it passes, and
 *     owns every output buffer.  All device memory belongs to the context and is
 *     released by tf_destroy.  The tensor's layout is allocated by tf_create; scratch
 *     that grows with later calls (Gram partials, loss reduction, fold-in and predict
 *     staging) is allocated in stream order on the context's stream, so that growing
 *     it waits for no other stream of the device.
 *   - Calls on one context are ordered on the context's CUDA stream.  A context is
 *     not thread-safe; distinct contexts are independent.
 *   - Host-only entry points (tf_assign_rows, tf_plan_mode, tf_version, and
 *     tf_estimate_bytes given num_sms > 0) need no GPU.
 */
#ifndef TF_SALS_H
#define TF_SALS_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct tf_ctx tf_ctx;

typedef enum {
    TF_OK = 0,
    TF_EINVAL = 1,   /* an argument is out of its documented range */
    TF_ERANGE = 2,   /* a coordinate is negative or >= its mode length */
    TF_EDUP = 3,     /* two observed entries share a coordinate (Omega is a set) */
    TF_ENOMEM = 4,   /* a device or host allocation failed */
    TF_ECUDA = 5,    /* a CUDA runtime call failed (no device, launch error, ...) */
    TF_ETIMEOUT = 6, /* a bounded wait on the device gave up */
    TF_EBUSY = 7     /* the context is in a state that forbids the call */
} tf_status;

typedef enum { TF_F32 = 0, TF_F64 = 1 } tf_dtype;

/* tf_create flags */
#define TF_INPUT_DEVICE 1u  /* coords and values are device pointers (same device) */
#define TF_LAYOUT_FIELD_SORTS 2u  /* build the layout by per-mode sorts of gathered
                                     coordinates even where one 64-bit key holds them
                                     all (same layout, slower; for comparison) */
#define TF_KEEP_DEFAULT_INIT 0u

/* per-sweep flags (tf_sals_sweep_ex) */
#define TF_WEIGHTED_LAMBDA 1u /* lambda * |Omega_i^(n)| per row (weighted-lambda, Sec. 5.1.3) */

/* row scheduling policies (tf_assign_rows / tf_plan_mode / tf_set_schedule) */
typedef enum {
    TF_SCHED_LPT = 0,    /* longest first to the least-loaded bin, no row cap (default) */
    TF_SCHED_GREEDY = 1, /* Algorithm 3: row cap ceil(I_n/M), tie-breaks on rows, totals */
    TF_SCHED_SEQ = 2,    /* contiguous row ranges (the paper's SEQ baseline, Sec. 5.5) */
    TF_SCHED_RAN = 3     /* seeded random bin per row (the paper's RAN baseline) */
} tf_sched_policy;

/* One unit of device work: entries [begin, begin + len) of a mode's sorted order, all
 * in row `row`.  The item writes its Gram matrix and right-hand side (Eq. 4) over those
 * entries to partial slot `slot`; a row is either one item or, when longer than the
 * cap, several chunks whose slots are consecutive in entry order.  The row's system is
 * the sum of its slots, in slot order. */
typedef struct {
    int64_t begin;
    int32_t len;
    int32_t row;
    int32_t slot;
    int32_t bin;
} tf_item;

/* ------------------------------------------------------------------ lifecycle */

/* Creates a context holding the tensor X and the factor matrices.
 *   coords  [nnz][N] int32, 0-based (host, or device with TF_INPUT_DEVICE)
 *   values  [nnz] float (dtype TF_F32) or double (TF_F64), same residency as coords
 *   dims    [N] mode lengths I_n, 1 <= I_n <= 2^31 - 1 (host)
 *   N       1..8;  nnz 0..2^31 - 1;  K >= 1
 *   seed    seeds the default initialisation and the default column orders
 *   stream  cudaStream_t to order all work on (NULL = the legacy default stream); it must
 *           stay valid until tf_destroy, which frees the context's memory on it (or until
 *           tf_set_stream moves the context to another stream)
 * Builds, on the device, the per-mode sorted layout (Omega_i^(n) of the table of
 * symbols, entries of a row in lexicographic order of the remaining coordinates taken
 * cyclically from mode n), with bit-exact row offsets; validates coordinates
 * (TF_ERANGE) and the set property (TF_EDUP); schedules rows onto bins (LPT).  Where
 * the modes' index widths, ceil(log2 I_n), sum to at most 64, every entry's coordinates
 * travel as one 64-bit key through the sorts; otherwise (or with TF_LAYOUT_FIELD_SORTS)
 * each sort gathers one mode's indices through the permutation so far.  Both give the
 * same layout.  flags: TF_INPUT_DEVICE, TF_LAYOUT_FIELD_SORTS; other bits TF_EINVAL.
 * Initialises the factors as Algorithm 1 does: A^(1) = 0 and A^(n>1) i.i.d. normal
 * with std K^(-1/(2N)) from `seed`, so that R = X.  *out is NULL on failure. */
tf_status tf_create(const int32_t *coords, const void *values, tf_dtype dtype,
                    const int64_t *dims, int N, int64_t nnz, int K, uint64_t seed,
                    void *stream, uint32_t flags, tf_ctx **out);

/* Releases every resource of ctx (NULL is a no-op). */
void tf_destroy(tf_ctx *ctx);

/* Text of the last failure on ctx (or of the last failed tf_create when ctx is NULL).
 * The pointer stays valid until the next call on the same context. */
const char *tf_last_error(const tf_ctx *ctx);

/* Waits for the context's stream and reports any device-side error. */
tf_status tf_sync(tf_ctx *ctx);

/* Row solves of float contexts (Eq. 4; the paper solves in the precision of its data).
 * refine = 1: every C x C solve takes one step of iterative refinement, x += (L L^T)^-1
 * (c - (B + lambda I) x) with the residual formed in FP64 from the sums as accumulated,
 * which removes the FP32 Cholesky's error on ill-conditioned rows.  cond_limit > 0: a row
 * whose smallest Cholesky pivot ratio d_j / (B_jj + lambda) is below 1 / cond_limit (or
 * that meets a non-positive pivot) is solved again, entirely in FP64, from the same sums;
 * such rows are counted (tf_solve_info).  Defaults 0, 0.  No effect on double contexts.
 * The Gram sums themselves keep the precision of the pass (tf_set_precision). */
tf_status tf_set_solve(tf_ctx *ctx, int refine, double cond_limit);

/* Float rows re-solved in FP64 so far (synchronises). */
tf_status tf_solve_info(tf_ctx *ctx, int64_t *fp64_rows);

/* enable = 1: sweeps run as CUDA graphs.  The launches of a sweep (pack, mode passes,
 * solves, for every split) depend only on C, T_in, lambda, flags, the columns left from
 * the previous sweep and the context's settings; the second sweep with a given such key is
 * captured into a graph and every later one replays it -- one launch per sweep.  Results
 * are bit-identical to eager sweeps.  Up to 8 graphs are kept per context (least recently
 * used dropped).  Not used while profiling (tf_profile) or on the legacy default stream.
 * enable = 0 (the default) drops the graphs.  The paper has no counterpart. */
tf_status tf_set_graphs(tf_ctx *ctx, int enable);

/* Picks the fastest (P, C) pair for this tensor by measurement: for every bin count
 * P_list[i] (0 = the default of tf_set_schedule; it sets how many rows' work one warp takes, the
 * rows-per-CTA knob of the mode passes) and every subset size C_list[j], one sweep
 * (lambda, T_in, flags as tf_sals_sweep_ex, default column order) is timed on the device
 * after an untimed sweep from the same state.  The state before the call (factors,
 * residuals, the previous subset's columns, the sweep counter) is restored bit for bit
 * after every trial and at the end, so later sweeps give what they would have given
 * without the call -- on the schedule of *best_P, which the context keeps.  Times go to
 * ms[i * n_C + j] (may be NULL).  Needs device memory for one copy of the factors and
 * residuals.  Speed only: a C that converges per sweep more slowly is not penalised.
 * The paper picks C by hand from its experiments (Section 5); it has no autotuner. */
tf_status tf_autotune(tf_ctx *ctx, const int32_t *C_list, int n_C, const int32_t *P_list,
                      int n_P, double lambda, int T_in, uint32_t flags, int32_t *best_C,
                      int32_t *best_P, float *ms);

/* Sweeps run from a graph so far, and graphs held. */
tf_status tf_graph_info(tf_ctx *ctx, int64_t *replays, int64_t *cached);

/* The context's mode count, rank and dtype (any output may be NULL). */
tf_status tf_get_shape(tf_ctx *ctx, int *N, int *K, tf_dtype *dtype);

/* The stream the context's work is ordered on. */
tf_status tf_get_stream(tf_ctx *ctx, void **stream);

/* Orders all later work of ctx on `stream` (a cudaStream_t of the same device; NULL = the
 * legacy default stream), after waiting for the work already queued on the old one.  A
 * serving context can so move to a high-priority stream, whose kernels the GPU starts
 * first when other contexts' kernels share it. */
tf_status tf_set_stream(tf_ctx *ctx, void *stream);

/* ------------------------------------------------------------------ factors */

/* Copies factor matrix n ([I_n][K], host, context dtype) into the context and marks
 * the residual for recomputation (R = X - model, Section 3.1) before the next use. */
tf_status tf_set_factors(tf_ctx *ctx, int n, const void *host_A);

/* Copies factor matrix n to host_A ([I_n][K], context dtype).  Synchronises. */
tf_status tf_get_factors(tf_ctx *ctx, int n, void *host_A);

/* ------------------------------------------------------------------ the sweep */

/* One outer iteration of Algorithm 1: ceil(K/C) splits; for each, R-hat (Algorithm 1),
 * then T_in passes over modes 1..N updating every row's C parameters by Eq. (4)
 * (Cholesky, Section 3.1; C = 1 is CDTF's closed form), then the R update of Eq. (5).
 * The last split holds K mod C columns when C does not divide K.
 * Column order: a seeded permutation per sweep for C > 1 (chosen without replacement,
 * Algorithm 1), the identity for C = 1 (CDTF keeps a fixed order, Section 3.1).
 *   C in 1..min(K, 127) (C <= 16: per-lane register Gram; 16 < C < 128: block-tiled
 *   Gram and shared-memory Cholesky), lambda >= 0 (double; converted to the context
 *   dtype), T_in >= 1.  C = K is the ALS row update of Eq. (2).  Asynchronous: returns
 *   once the work is queued on the stream.
 * A row whose B + lambda I has a non-positive Cholesky pivot (e.g. an empty row with
 * lambda = 0) is left unchanged and counted (tf_get_counters). */
tf_status tf_sals_sweep(tf_ctx *ctx, int C, double lambda, int T_in);

/* As tf_sals_sweep with an explicit column order col_order[K] (a permutation of
 * 0..K-1, host); split s takes col_order[s*C .. min((s+1)*C, K)).  NULL = default. */
tf_status tf_sals_sweep_order(tf_ctx *ctx, int C, double lambda, int T_in,
                              const int32_t *col_order);

/* As tf_sals_sweep_order with flags (TF_WEIGHTED_LAMBDA). */
tf_status tf_sals_sweep_ex(tf_ctx *ctx, int C, double lambda, int T_in,
                           const int32_t *col_order, uint32_t flags);

/* Writes the default column order of sweep number `sweep` (0-based) for this C. */
tf_status tf_default_order(const tf_ctx *ctx, int sweep, int C, int32_t *col_order);

/* ------------------------------------------------------------------ loss */

/* loss = sum_Omega r^2 + lambda * sum_n ||A^(n)||_F^2 (Eq. 1; with TF_WEIGHTED_LAMBDA
 * each row's squared norm is weighted by |Omega_i^(n)|), train_rmse =
 * sqrt(sum r^2 / |Omega|).  Accumulated in double on the device, in a fixed order
 * (bit-reproducible).  Synchronises.  Either output pointer may be NULL. */
tf_status tf_loss(tf_ctx *ctx, double lambda, uint32_t flags, double *loss,
                  double *train_rmse);

/* The loss of tf_loss, computed without allocating device memory; the paper has no
 * counterpart (it is an interface for callers, not part of the method).
 * Meant for callers that cannot call cudaMalloc at this point: a process whose device
 * memory is already reserved by another allocator (a caching allocator or a serving
 * engine that holds the free memory as its own pool), so that a new allocation fails
 * or fragments that pool, and latency-bound loops that must not take the device-wide
 * synchronisation a cudaMalloc or cudaFree may cause.  tf_loss keeps its reduction
 * buffer in the context and allocates it on first use; this entry point instead uses a
 * fixed device array of 24,576 doubles (192 KiB) built into the library, one per
 * device, and calls no allocating routine.
 *   Arguments, result and synchronisation as tf_loss; the result is bit-identical to
 *   tf_loss's on the same state.
 *   Limit: the reduction needs 2 + B + 256 N doubles, B = the residual kernel's block
 *   count (at most P, the schedule's bin count).  Beyond 24,576 the call returns
 *   TF_EINVAL, says so in tf_last_error, and launches nothing.  The default schedule
 *   (at most 128 bins per SM) fits for every N <= 8 on GPUs of up to 175 SMs; a
 *   schedule set with tf_set_schedule fits while P + 256 N <= 24,574.
 *   Device: the call must be made with the context's device current (the device that
 *   was current at tf_create); otherwise it returns TF_EINVAL and launches nothing.
 *   Set-up: the first call on each device (the device current at the call) looks up
 *   the array's device address with cudaGetSymbolAddress; make that first call before
 *   any stream capture begins.
 *   Sharing: every call on a device uses the same array, which keeps the previous
 *   call's contents.  Each call writes every element it reads before reading it, so
 *   nothing needs clearing.  Calls that overlap on the GPU (from several host threads,
 *   or several contexts, on one device) race on the array: serialise them. */
tf_status tf_loss_noalloc(tf_ctx *ctx, double lambda, uint32_t flags, double *loss,
                          double *train_rmse);

/* ------------------------------------------------------------------ fold-in */

/* Least-squares row for a new slice of mode `mode` against the frozen factors: the
 * ALS row solve of Eq. (2), a = (B + lambda I_K)^{-1} c, B = sum h h^T, c = sum x h,
 * h_k = prod_{l != mode} a^(l)_{i_l k}, over the request's m entries.
 *   other  [m][N-1] int32 (host): indices of the other modes in increasing mode order
 *   values [m] context dtype (host);  out_row [K] context dtype (host)
 * Synchronises.  TF_ERANGE if an index is out of range.  A non-positive pivot gives
 * TF_EINVAL with out_row untouched. */
tf_status tf_foldin(tf_ctx *ctx, int mode, const int32_t *other, const void *values,
                    int64_t m, double lambda, void *out_row);

/* ------------------------------------------------------------------ prediction */

/* Model values x_hat_e = sum_k prod_n a^(n)_{i_n k} (the CP model of Eq. 1) at m
 * coordinates, e.g. held-out entries for a test RMSE.
 *   coords [m][N] int32, 0-based; out [m] context dtype.  Both host buffers, or both
 *   device buffers on the context's device with flags = TF_INPUT_DEVICE.
 * Products and the sum over k in double on the device.  Synchronises.  TF_ERANGE if a
 * coordinate is out of range (out is then unspecified). */
tf_status tf_predict(tf_ctx *ctx, const int32_t *coords, int64_t m, void *out, uint32_t flags);

/* Many fold-in requests of one mode in one batch (one launch of the tiled Gram over all
 * of their entries, one warp-level solve per request): request r has the entries
 * offsets[r] .. offsets[r + 1] - 1 of the concatenated other [total][N-1] and values
 * [total] (host; offsets[n_req + 1] int64 with offsets[0] = 0, non-decreasing).
 * out_rows [n_req][K] (host, context dtype); status [n_req] (host): 0 ok, 1 an index
 * out of range, 2 a non-positive pivot — the row of a failed request is left untouched
 * and the others are still solved.  Synchronises.  Results equal tf_foldin's per
 * request (same blocks, same summation order). */
tf_status tf_foldin_batch(tf_ctx *ctx, int mode, int n_req, const int64_t *offsets,
                          const int32_t *other, const void *values, double lambda, void *out_rows,
                          int32_t *status);

/* ------------------------------------------------------------------ inspection */

/* Row offsets off[I_n + 1] (int64) and, if perm != NULL, the canonical entry index of
 * every position of mode n's sorted order, perm[nnz] (int64).  Synchronises. */
tf_status tf_get_grouping(tf_ctx *ctx, int n, int64_t *off, int64_t *perm);

/* The residual r_e = x_e - sum_k prod_n a^(n)_{i_n k} (Section 3.1) of every entry in
 * canonical (input) order, host [nnz], context dtype.  Synchronises. */
tf_status tf_get_residual(tf_ctx *ctx, void *host_r);

/* counters[0] = rows left unchanged by a non-positive pivot since creation,
 * counters[1] = sweeps run, counters[2] = kernels launched by the last sweep,
 * counters[3] = work items of all modes, counters[4] = rows split across bins,
 * counters[5] = bins P of the schedule, counters[6] = kernels launched by the last
 * tf_loss, counters[7] = mode-pass data paths the last sweep used (bit 0: SIMT pass,
 * bit 1: TMA gather pass, bit 2: tensor-core Gram pass of wide subsets; 0 = no sweep). */
tf_status tf_get_counters(tf_ctx *ctx, int64_t counters[8]);

/* Re-plans the row schedule of every mode (policy, P bins; P = 0 picks the default
 * for this GPU and tensor: 128 bins per SM, fewer for small tensors so that a bin holds
 * 64 entries on average, at least 4 per SM).  The schedule changes only the order in which a row's
 * partial sums are added (heavy rows are split into chunks of at most |Omega| / P
 * entries), so results agree to rounding. */
tf_status tf_set_schedule(tf_ctx *ctx, tf_sched_policy policy, int P);

/* Data path of the mode pass: 0 = automatic (C <= 16: for float three-way tensors and
 * C <= 12 the lean pass (hot slice rows resident in shared memory, packed two-wide FP32
 * Gram), else the cp.async SIMT pass; 16 < C < 128: for float contexts the Gram on the
 * tensor cores (tcgen05, three TF32 products per term, FP32 accumulation) for C >= 32,
 * where it measures faster, SIMT FMAs below and for double), 1 = the cp.async SIMT pass
 * and the SIMT wide Gram everywhere, 2 = the TMA tile::gather4 pass with its shared-memory row cache for
 * C <= 10 (float, N = 3; TF_EINVAL from the next sweep where it does not apply) and the
 * tensor-core Gram for every wide C, 3 = the lean pass (TF_EINVAL from the next sweep
 * where it does not apply; wide C as path 0).  The cp.async and TMA passes give
 * bit-identical results; the lean pass sums each row's terms in another order and the
 * tensor-core Gram rounds its products differently, both agreeing to FP32 rounding. */
tf_status tf_set_kernel_path(tf_ctx *ctx, int path);

/* Blocks of this context's persistent mode passes (each holds an SM for the whole pass):
 * at most `sms` (0 = one per SM, the default).  A serving process gives its factorisation
 * jobs a limit below the SM count so that kernels on other streams (fold-ins) find SMs
 * free at any time instead of waiting for a pass to end.  Results do not depend on it.
 * TF_EINVAL for sms < 0.  No counterpart in the paper. */
tf_status tf_set_sm_limit(tf_ctx *ctx, int sms);

/* Shared-memory layout of the lean pass (kernel path 0 or 3): at most max_rows rows of
 * each other mode's slice are held in shared memory per launch (< 0: as many as fit, the
 * rows with the most entries first; 0: none); the distinct rows outside that cache that a
 * step of 32 entries needs are staged one step ahead in one of two per-warp pool slots of
 * pool_rows rows each (2..32; a step's lanes are split over several rounds where its rows
 * would not fit); warps per block 1..16 (0: the most that fit the registers and shared memory, at
 * most 12 with the packed-FMA Gram, 16 with the tensor-core Gram).  The lean pass plans, once per row schedule and setting, where
 * each entry's rows will be; no setting changes any result (bit-identical).  TF_EINVAL
 * for values outside these ranges.  No counterpart in the paper. */
tf_status tf_set_pass_cache(tf_ctx *ctx, int max_rows, int pool_rows, int warps);

/* Reduced-precision forms of the sweep in float contexts (no counterpart in the paper):
 *   0 = FP32-level (default; on the tensor cores three TF32 products per Gram term);
 *   1 = one TF32 product per Gram term on the tensor cores, for wide subsets (16 < C < 128)
 *       and for the lean pass (three-way tensors, C <= 12): B and c carry about 1e-3
 *       relative error, so a row update differs from the FP32 one by about
 *       cond(B + lambda I) * 1e-3;
 *   2 = the lean pass reads the varying mode's slice rows (one of the two per-entry
 *       gathers) from bfloat16 copies of the slices (8 significand bits, rounded to nearest
 *       even from the FP32 slices after every pack and every mode's solve); run-mode and
 *       own rows, products, sums and residuals stay FP32.  Other passes run FP32-level.
 *       Adds sum_n I_n * ceil(3 C_max / 8) * 16 bytes of copies;
 *   3 = as 2 for both other modes' rows (the R-hat refresh products then carry two
 *       rounded factors: the training RMSE moved by up to 2e-3 relative on a low-noise
 *       test tensor, by 6e-6 on the skewed 1e8-entry workload).
 * In forms 1 and 2 the training RMSE after a few sweeps stays within 1e-3 of the FP64
 * oracle's on the tested workloads.  TF_EINVAL for a mode other than 0 on a double
 * context, or outside 0..2. */
tf_status tf_set_precision(tf_ctx *ctx, int mode);

/* ------------------------------------------------------------------ timing */

/* Measured peaks of the current device's units that bind the narrow mode passes (not of
 * the method): FP32 FMA throughput in TFLOP/s, plain (fp32_tflops) and with packed two-wide
 * FMAs (fp32x2_tflops), and shared-memory load bandwidth in TB/s (16-byte loads without
 * bank conflicts; smem_tbytes).  Each is timed with CUDA events over five launches of a
 * microbenchmark kernel after one warm-up, on a stream of its own; it allocates and frees
 * a small device buffer (cudaMalloc / cudaFree, which synchronise the device).  Any
 * output may be NULL.  TF_ECUDA on a CUDA failure. */
tf_status tf_device_peaks(double *fp32_tflops, double *fp32x2_tflops, double *smem_tbytes);


/* Kernel kinds reported by tf_get_profile. */
typedef enum {
    TF_KIND_PACK = 0,      /* slice packing of a split (Theorem 3's C resident columns) */
    TF_KIND_MODE_PASS = 1, /* fused R-hat / Gram / rhs pass over one mode (Eq. 4)        */
    TF_KIND_COMBINE = 2,   /* sum of split rows' partial Gram/rhs + Cholesky solve      */
    TF_KIND_LOSS = 3,      /* loss / residual reductions (Eq. 1)                        */
    TF_KIND_OTHER = 4,     /* residual rebuilds and flushes                             */
    TF_KIND_SOLVE = 5,     /* Cholesky solves of the rows held by one item (Sec. 3.1)   */
    TF_KIND_COUNT = 6
} tf_kernel_kind;

/* enable != 0: from now on bracket every kernel launch of this context with CUDA
 * events on its stream and accumulate the device time per kind; enable == 0 stops
 * and clears.  Off by default. */
tf_status tf_profile(tf_ctx *ctx, int enable);

/* Launch counts and summed device milliseconds per kind since profiling was enabled
 * (arrays of TF_KIND_COUNT).  Synchronises. */
tf_status tf_get_profile(tf_ctx *ctx, int64_t *launches, double *ms);

/* Per-launch trace since profiling was enabled: up to cap records of (kind, mode,
 * milliseconds) in launch order; *n receives the number available.  mode is the
 * tensor mode the launch worked on (-1 when it spans all modes).  Synchronises. */
tf_status tf_get_launch_trace(tf_ctx *ctx, int64_t cap, int64_t *n, int32_t *kinds,
                              int32_t *modes, float *ms);

/* ------------------------------------------------------------------ host-only */

/* Row-to-bin assignment of every mode (no splitting) for M bins, as the paper's
 * Algorithm 3 does for machines with TF_SCHED_GREEDY (row cap ceil(I_n/M); ties to
 * fewer rows, then to the smaller total over earlier modes, then to the lower index;
 * equal rows in increasing index).  TF_SCHED_LPT drops the cap; SEQ and RAN are the
 * baselines of Section 5.5.  row_nnz[n][I_n], assign[n][I_n] (host).  No GPU. */
tf_status tf_assign_rows(tf_sched_policy policy, int N, const int64_t *dims,
                         const int64_t *const *row_nnz, int M, uint64_t seed,
                         int32_t *const *assign);

/* Work items of one mode for P bins: rows longer than cap entries are split into
 * ceil(len / cap) near-equal chunks (cap = 0: ceil(nnz / P)); rows and chunks are
 * placed longest first on the least-loaded bin (TF_SCHED_LPT) or by another policy.
 * off[I + 1] are the row offsets (host).  items (capacity max_items) come out grouped
 * by bin, bins in increasing order; bin_ptr[P + 1] indexes them.  *n_items and
 * *n_slots receive the counts (every item has its own slot, so they are equal).  TF_ENOMEM if max_items is too small.  No GPU. */
tf_status tf_plan_mode(const int64_t *off, int64_t I, int P, int64_t cap,
                       tf_sched_policy policy, uint64_t seed, tf_item *items,
                       int64_t max_items, int64_t *n_items, int64_t *n_slots,
                       int64_t *bin_ptr);

/* ------------------------------------------------------------------ memory */

/* Upper bound, in bytes, of the device memory a context holds at any time from tf_create
 * through sweeps with C <= C_max and tf_loss (the peak of the layout build or of the
 * sweeps, whichever is larger), counting the stream-ordered pool's rounding.  Fold-in and
 * predict staging are not included (they grow with the requests).  No counterpart in the
 * paper: a serving process admits jobs against free device memory with it.
 *   dims [N], N, nnz, K, dtype, flags   as for tf_create (TF_INPUT_DEVICE,
 *                                       TF_LAYOUT_FIELD_SORTS)
 *   C_max    largest C of the sweeps to come, 1..min(K, 127)
 *   num_sms  the device's SM count (> 0: no device needed), <= 0: asked of the device
 * TF_EINVAL for arguments tf_create or tf_sals_sweep would refuse. */
tf_status tf_estimate_bytes(const int64_t *dims, int N, int64_t nnz, int K, int C_max,
                            tf_dtype dtype, uint32_t flags, int num_sms, int64_t *bytes);

/* The library's stream-ordered memory pool on the current device, which holds every
 * context's device memory: bytes in use, their high-water mark, and bytes the pool holds
 * (in use, or freed by destroyed contexts and kept for later ones); reset_high != 0
 * restarts the high-water mark at the current use.  Any output pointer may be NULL.  The
 * pool keeps freed memory (creating a context after destroying one maps nothing new) and
 * never makes one context's stream wait for another's to reuse a block. */
tf_status tf_pool_usage(int64_t *used, int64_t *used_high, int64_t *reserved, int reset_high);

/* Returns the pool's unused memory to the device, keeping at most keep_bytes held
 * (synchronises the device first). */
tf_status tf_pool_trim(int64_t keep_bytes);

/* Library version string. */
const char *tf_version(void);

#ifdef __cplusplus
}
#endif

#endif /* TF_SALS_H */
