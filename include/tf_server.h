/* Serving loop of the SALS / CDTF library: one process, one GPU, a persistent host
 * scheduler that takes two kinds of requests and keeps their work on the device.
 *
 *   - Factorisation jobs (a tensor, K, C, lambda, T_in and a number of outer sweeps of
 *     Algorithm 1).  A job is admitted when its device footprint (tf_estimate_bytes) fits
 *     the free device memory (with what the library's pool holds unused, less the reserve
 *     and the footprints of admitted jobs still building their layout), and the job budget
 *     when one is set; each admitted job runs in its own context on its own low-priority
 *     stream from its own host thread, so the kernels of several jobs overlap on the
 *     device.  Its factors and residuals stay on the
 *     device until the caller releases it.
 *   - Fold-in requests: a new slice of one mode solved against the frozen factors of a
 *     model context (the ALS row update of Eq. 2 for that slice).  Requests that arrive
 *     while a batch is on the GPU wait and form the next batch (continuous batching):
 *     one tf_foldin_batch per batch on the server's high-priority stream.
 *
 * The paper has no serving layer; this is built around its kernels.  Results do not
 * depend on what else runs: a job gives the factors it gives alone, bit for bit (contexts
 * share no device state), and a fold-in gives the row it gives alone (a request's partial
 * Gram matrices are summed in its own fixed block order whatever batch it lands in).
 *
 * Threading: every tf_server_* call is thread-safe (a job's factors may be read while
 * another thread releases it: the release waits).  While a server exists, its model
 * context belongs to the server: the caller makes no call on it until tf_server_destroy.
 * Inputs are copied at submission; the caller keeps ownership of every buffer.
 */
#ifndef TF_SERVER_H
#define TF_SERVER_H

#include <stdint.h>

#include "tf_sals.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct tf_server tf_server;

typedef struct {
    int64_t hbm_budget;  /* bytes the admitted jobs may hold together (their estimates);
                            0 = no budget beyond free device memory */
    int64_t hbm_reserve; /* bytes left free on the device at every admission; 0 = 1 GiB */
    int max_running;     /* jobs admitted at once, 1..256; 0 = 8 */
    int max_batch;       /* fold-in requests per batch, 1..65536; 0 = 256 */
    int max_bypass;      /* times a queued job may be passed by later jobs that fit when it
                            does not (first fit in arrival order); then admission waits for
                            it.  0 = 8, < 0 = never pass (strict arrival order) */
    int reserve_sms;     /* SMs the jobs' persistent mode passes leave free (tf_set_sm_limit)
                            so that fold-in kernels start without waiting for a pass to end;
                            0 = 8 when a model is served (none otherwise), < 0 = none */
} tf_server_config;

typedef struct {
    const int32_t *coords;      /* [nnz][N] int32, host */
    const void *values;         /* [nnz] float (TF_F32) or double (TF_F64), host */
    const int64_t *dims;        /* [N] */
    int N;
    int64_t nnz;
    int K;
    tf_dtype dtype;
    uint64_t seed;              /* as tf_create: initial factors and default orders */
    int C;                      /* columns per subset, 1..min(K, 127) */
    double lambda;
    int T_in;
    int sweeps;                 /* outer iterations of Algorithm 1, >= 1 */
    uint32_t sweep_flags;       /* TF_WEIGHTED_LAMBDA or 0 */
    const int32_t *col_orders;  /* [sweeps][K] column orders, or NULL for the defaults */
} tf_job_desc;

typedef enum {
    TF_JOB_QUEUED = 0,
    TF_JOB_RUNNING = 1,
    TF_JOB_DONE = 2,
    TF_JOB_FAILED = 3
} tf_job_state;

typedef struct {
    tf_job_state state;
    tf_status status;   /* why it failed (TF_JOB_FAILED); TF_OK otherwise */
    int sweeps_done;
    double loss, rmse;  /* tf_loss after the last sweep (TF_JOB_DONE) */
    int64_t bytes;      /* the footprint it was admitted with (tf_estimate_bytes) */
    double queued_s, started_s, finished_s; /* seconds since tf_server_create; -1 = not yet */
} tf_job_info;

typedef struct {
    int64_t jobs_queued, jobs_running, jobs_done, jobs_failed;
    int64_t foldins_done, foldin_batches, foldin_max_batch;
    int64_t bytes_admitted;      /* sum of the estimates of the jobs holding memory */
    int64_t bytes_admitted_peak;
    int64_t running_peak;        /* most jobs running at once */
} tf_server_stats;

/* Starts the admission and batching threads on the current device.  model (may be NULL:
 * no fold-ins) is moved to a stream of the device's highest priority for the server's life
 * and back to its own stream by tf_server_destroy.  *out is NULL on failure. */
tf_status tf_server_create(const tf_server_config *cfg, tf_ctx *model, tf_server **out);

/* Stops the server: queued jobs and fold-ins fail with TF_EBUSY, running jobs stop after
 * their current sweep (TF_EBUSY), every job context is destroyed, threads are joined.
 * NULL is a no-op. */
void tf_server_destroy(tf_server *srv);

/* Text of the last failure of a call on srv (or of the last failed tf_server_create
 * when srv is NULL). */
const char *tf_server_last_error(const tf_server *srv);

/* Queues a job.  TF_EINVAL for arguments tf_create or tf_sals_sweep would refuse;
 * TF_ENOMEM when its footprint exceeds the budget or the device's total memory less the
 * reserve, so that it could never be admitted. */
tf_status tf_server_submit_job(tf_server *srv, const tf_job_desc *job, int64_t *job_id);

/* State of a job (any state until released). */
tf_status tf_server_job_info(tf_server *srv, int64_t job_id, tf_job_info *info);

/* Waits up to timeout_s seconds for the job to be done or failed; TF_ETIMEOUT if it is
 * still queued or running then.  info may be NULL. */
tf_status tf_server_wait_job(tf_server *srv, int64_t job_id, double timeout_s,
                             tf_job_info *info);

/* Copies factor matrix n [I_n][K] (job's dtype) of a done job to host memory. */
tf_status tf_server_job_factors(tf_server *srv, int64_t job_id, int n, void *host_A);

/* Destroys a done or failed job's context (its device memory goes back to the pool and
 * its admission bytes to the budget) and forgets the job.  TF_EBUSY while it is queued
 * or running. */
tf_status tf_server_release_job(tf_server *srv, int64_t job_id);

/* Queues a fold-in request: m entries of a new slice of `mode`, their other-mode
 * indices other [m][N-1] (modes in increasing order, `mode` left out) and values
 * [m] in the model's dtype.  TF_EINVAL without a model or for a bad mode / lambda. */
tf_status tf_server_submit_foldin(tf_server *srv, int mode, const int32_t *other,
                                  const void *vals, int64_t m, double lambda,
                                  int64_t *req_id);

/* Waits up to timeout_s seconds for a fold-in; then writes its row [K] (model dtype)
 * to out_row, its status (0 ok, 1 index out of range, 2 non-positive pivot, or a
 * tf_status + 16 when the batch failed as a whole) to req_status, and the seconds from
 * submission to completion to latency_s (may be NULL), and forgets the request.
 * TF_ETIMEOUT if not done yet (the request stays queued). */
tf_status tf_server_wait_foldin(tf_server *srv, int64_t req_id, double timeout_s,
                                void *out_row, int32_t *req_status, double *latency_s);

tf_status tf_server_get_stats(tf_server *srv, tf_server_stats *stats);

/* Which queued jobs to admit, as the scheduler decides it (host only, no GPU): jobs
 * 0..n-1 in arrival order with footprints need[n] and pass counts bypassed[n] (updated
 * in place), `room` bytes of device memory available, `budget_left` bytes of budget (< 0 =
 * no budget), `slots` jobs that may still start, max_bypass as in tf_server_config (already
 * defaulted).  Sets admit[j] = 1 for each job to start; returns the number admitted. */
int tf_server_plan_admission(int n, const int64_t *need, int32_t *bypassed, int64_t room,
                             int64_t budget_left, int slots, int max_bypass, int32_t *admit);

#ifdef __cplusplus
}
#endif

#endif /* TF_SERVER_H */
