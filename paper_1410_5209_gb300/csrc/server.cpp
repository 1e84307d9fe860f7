// Serving loop: threads that admit factorisation jobs against free device memory and
// batch fold-in requests continuously, built on the public C ABI of the library (every
// step of the method runs in the library's kernels).
//
// Threads: an admission thread starts jobs; a batching thread owns the model context and
// runs the fold-in batches on a stream of the device's highest priority (neither holds
// the lock while it calls into CUDA); each admitted job has a worker thread that
// creates the job's context on its own stream of the lowest priority, runs its sweeps
// and its loss, and leaves the context for the caller to read and release.  All shared
// state sits behind one mutex; condition variables wake the admission thread (new jobs,
// freed memory), the batching thread (new fold-ins) and the callers waiting for a
// finished job or fold-in.
#include <string.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <new>
#include <string>
#include <thread>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/tf_server.h"

namespace {

using Clock = std::chrono::steady_clock;

thread_local std::string g_server_create_err;

struct Job {
    int64_t id = 0;
    tf_job_desc d{};
    std::vector<int32_t> coords, orders;
    std::vector<char> values;
    std::vector<int64_t> dims;
    tf_job_info info{};
    int32_t bypassed = 0;
    bool first_sweep_done = false;  // its allocations have reached their steady size
    tf_ctx *ctx = nullptr;
    cudaStream_t stream = nullptr;
    std::thread worker;
    std::mutex use;  // calls on ctx after the worker is done (factors, release)
};

struct Foldin {
    int64_t id = 0;
    int mode = 0;
    double lambda = 0;
    std::vector<int32_t> other;
    std::vector<char> vals;
    int64_t m = 0;
    Clock::time_point submitted, done_at;
    bool done = false;
    int32_t status = 0;
    std::vector<char> row;
};

double secs(Clock::time_point a, Clock::time_point b) {
    return std::chrono::duration<double>(b - a).count();
}

}  // namespace

struct tf_server {
    tf_server_config cfg{};
    int device = 0;
    tf_ctx *model = nullptr;
    void *model_old_stream = nullptr;
    cudaStream_t hi = nullptr;
    int model_N = 0, model_K = 0;
    tf_dtype model_dtype = TF_F32;
    int64_t device_total = 0;
    Clock::time_point t0;

    std::mutex mu;
    std::condition_variable cv_work, cv_fold, cv_done;
    bool stop = false;
    std::string err;

    int64_t next_id = 1;
    std::deque<std::shared_ptr<Job>> queue;             // arrival order
    std::map<int64_t, std::shared_ptr<Job>> jobs;       // every job not yet released
    std::deque<std::shared_ptr<Foldin>> fq;             // fold-ins waiting for a batch
    std::map<int64_t, std::shared_ptr<Foldin>> foldins; // every fold-in not yet collected
    int64_t running = 0, admitted_bytes = 0;
    tf_server_stats st{};
    std::thread sched, batcher;

    double now() const { return secs(t0, Clock::now()); }
    void run_scheduler();
    void run_batcher();
    void run_job(std::shared_ptr<Job> j);
    void admit_locked(int64_t free_b, int64_t pool_unused);
    void batch_foldins(std::unique_lock<std::mutex> &lk);
};

namespace {

size_t elem_bytes(tf_dtype t) { return t == TF_F64 ? 8 : 4; }

}  // namespace

// Admission: scan the queue in arrival order and start every job that fits (first fit);
// a job that does not fit while a later one starts is passed once more; a job passed
// max_bypass times blocks everything behind it until it fits.
// free_b: the device's free memory; pool_unused: memory the library's pool holds but no
// context uses (free for new jobs too) -- both read by the caller without the lock.
void tf_server::admit_locked(int64_t free_b, int64_t pool_unused) {
    if (queue.empty()) return;
    const int slots = (int)std::max<int64_t>(0, cfg.max_running - running);
    if (slots == 0) return;
    // memory that admitted jobs have yet to allocate: a job's whole estimate until its
    // first sweep has run
    int64_t pending = 0;
    for (auto &kv : jobs)
        if (kv.second->info.state == TF_JOB_RUNNING && !kv.second->first_sweep_done)
            pending += kv.second->info.bytes;
    const int64_t room = free_b + pool_unused - cfg.hbm_reserve - pending;
    const int64_t budget_left = cfg.hbm_budget > 0 ? cfg.hbm_budget - admitted_bytes : -1;
    const int n = (int)queue.size();
    std::vector<int64_t> need(n);
    std::vector<int32_t> byp(n), admit(n, 0);
    for (int i = 0; i < n; ++i) {
        need[i] = queue[i]->info.bytes;
        byp[i] = queue[i]->bypassed;
    }
    tf_server_plan_admission(n, need.data(), byp.data(), room, budget_left, slots,
                             cfg.max_bypass, admit.data());
    std::deque<std::shared_ptr<Job>> rest;
    for (int i = 0; i < n; ++i) {
        auto &j = queue[i];
        j->bypassed = byp[i];
        if (!admit[i]) {
            rest.push_back(j);
            continue;
        }
        j->info.state = TF_JOB_RUNNING;
        j->info.started_s = now();
        admitted_bytes += j->info.bytes;
        ++running;
        st.running_peak = std::max(st.running_peak, running);
        st.bytes_admitted_peak = std::max(st.bytes_admitted_peak, admitted_bytes);
        try {
            j->worker = std::thread(&tf_server::run_job, this, j);
        } catch (...) {  // no thread for it: the job fails, its admission is undone
            admitted_bytes -= j->info.bytes;
            --running;
            j->info.state = TF_JOB_FAILED;
            j->info.status = TF_ENOMEM;
            j->info.started_s = -1;
            j->info.finished_s = now();
            ++st.jobs_failed;
            cv_done.notify_all();
        }
    }
    queue.swap(rest);
}

void tf_server::run_job(std::shared_ptr<Job> j) {
    tf_status s = TF_OK;
    int done = 0;
    double loss = 0, rmse = 0;
    int lo = 0, hi_p = 0;
    cudaSetDevice(device);
    cudaDeviceGetStreamPriorityRange(&lo, &hi_p);  // lo = least urgent
    if (cudaStreamCreateWithPriority(&j->stream, cudaStreamNonBlocking, lo) != cudaSuccess) {
        cudaGetLastError();
        j->stream = nullptr;
        s = TF_ECUDA;
    }
    tf_ctx *ctx = nullptr;
    if (s == TF_OK)
        s = tf_create(j->coords.data(), j->values.data(), j->d.dtype, j->dims.data(), j->d.N,
                      j->d.nnz, j->d.K, j->d.seed, j->stream, 0, &ctx);
    if (s == TF_OK && cfg.reserve_sms > 0) {  // SMs left free for the fold-ins
        int sms = 0;
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
        s = tf_set_sm_limit(ctx, std::max(1, sms - cfg.reserve_sms));
    }
    // the host copies of the inputs are no longer needed
    std::vector<int32_t>().swap(j->coords);
    std::vector<char>().swap(j->values);
    for (int t = 0; s == TF_OK && t < j->d.sweeps; ++t) {
        {
            std::lock_guard<std::mutex> g(mu);
            if (stop) {
                s = TF_EBUSY;
                break;
            }
        }
        const int32_t *ord = j->orders.empty() ? nullptr : j->orders.data() + (size_t)t * j->d.K;
        s = tf_sals_sweep_ex(ctx, j->d.C, j->d.lambda, j->d.T_in, ord, j->d.sweep_flags);
        if (s == TF_OK && t == 0) s = tf_sync(ctx);
        if (s == TF_OK) {
            ++done;
            std::lock_guard<std::mutex> g(mu);
            j->info.sweeps_done = done;
            if (!j->first_sweep_done) {
                j->first_sweep_done = true;
                cv_work.notify_all();  // its memory is now allocated: admission may go on
            }
        }
    }
    if (s == TF_OK) s = tf_loss(ctx, j->d.lambda, j->d.sweep_flags, &loss, &rmse);
    std::lock_guard<std::mutex> g(mu);
    j->ctx = ctx;
    if (s == TF_OK) {
        j->info.state = TF_JOB_DONE;
        j->info.loss = loss;
        j->info.rmse = rmse;
        ++st.jobs_done;
    } else {
        j->info.state = TF_JOB_FAILED;
        j->info.status = s;
        ++st.jobs_failed;
    }
    j->first_sweep_done = true;
    j->info.finished_s = now();
    --running;
    cv_done.notify_all();
    cv_work.notify_all();
}

// One batch: the oldest waiting request and every later one with the same mode and
// lambda, up to max_batch, solved by one tf_foldin_batch call (lock released meanwhile).
void tf_server::batch_foldins(std::unique_lock<std::mutex> &lk) {
    std::vector<std::shared_ptr<Foldin>> b;
    const int mode = fq.front()->mode;
    const double lam = fq.front()->lambda;
    std::deque<std::shared_ptr<Foldin>> rest;
    for (auto &r : fq) {
        if ((int)b.size() < cfg.max_batch && r->mode == mode && r->lambda == lam)
            b.push_back(r);
        else
            rest.push_back(r);
    }
    fq.swap(rest);
    lk.unlock();
    const int n = (int)b.size();
    const size_t eb = elem_bytes(model_dtype);
    std::vector<char> rows;
    std::vector<int32_t> status;
    tf_status s = TF_OK;
    try {  // host staging of the batch; a failed allocation fails the batch
        std::vector<int64_t> off((size_t)n + 1, 0);
        for (int r = 0; r < n; ++r) off[r + 1] = off[r] + b[r]->m;
        std::vector<int32_t> other((size_t)std::max<int64_t>(off[n], 1) *
                                   std::max(model_N - 1, 1));
        std::vector<char> vals((size_t)std::max<int64_t>(off[n], 1) * eb);
        for (int r = 0; r < n; ++r) {
            memcpy(other.data() + off[r] * (model_N - 1), b[r]->other.data(),
                   b[r]->other.size() * sizeof(int32_t));
            memcpy(vals.data() + off[r] * eb, b[r]->vals.data(), b[r]->vals.size());
        }
        rows.assign((size_t)n * model_K * eb, 0);
        status.assign((size_t)n, 0);
        s = tf_foldin_batch(model, mode, n, off.data(), other.data(), vals.data(), lam,
                            rows.data(), status.data());
    } catch (...) {
        s = TF_ENOMEM;
    }
    const auto t = Clock::now();
    lk.lock();
    for (int r = 0; r < n; ++r) {
        auto &q = *b[r];
        if (s == TF_OK)
            q.row.assign(rows.begin() + (size_t)r * model_K * eb,
                         rows.begin() + (size_t)(r + 1) * model_K * eb);
        q.status = s == TF_OK ? status[r] : 16 + (int32_t)s;
        q.done = true;
        q.done_at = t;
        std::vector<int32_t>().swap(q.other);
        std::vector<char>().swap(q.vals);
    }
    st.foldins_done += n;
    ++st.foldin_batches;
    st.foldin_max_batch = std::max<int64_t>(st.foldin_max_batch, n);
    cv_done.notify_all();
}

// Admission thread.  Device-memory queries can wait for the driver while other threads
// allocate; they run without the lock, so submissions and fold-in batches never wait
// for them.
void tf_server::run_scheduler() {
    cudaSetDevice(device);
    std::unique_lock<std::mutex> lk(mu);
    while (!stop) {
        if (!queue.empty() && running < cfg.max_running) {
            lk.unlock();
            size_t free_b = 0, total_b = 0;
            int64_t used = 0, held = 0;
            const bool ok = cudaMemGetInfo(&free_b, &total_b) == cudaSuccess;
            if (!ok) cudaGetLastError();
            if (tf_pool_usage(&used, nullptr, &held, 0) != TF_OK) used = held = 0;
            lk.lock();
            if (ok && !stop) admit_locked((int64_t)free_b, std::max<int64_t>(0, held - used));
        }
        // wake for new jobs or freed memory; poll now and then, since device memory can
        // also be freed by other users of the GPU
        cv_work.wait_for(lk, std::chrono::milliseconds(50));
    }
}

// Fold-in thread: a batch whenever requests wait (continuous batching).
void tf_server::run_batcher() {
    cudaSetDevice(device);
    std::unique_lock<std::mutex> lk(mu);
    while (!stop) {
        if (!fq.empty()) {
            batch_foldins(lk);
            continue;
        }
        cv_fold.wait(lk, [&] { return stop || !fq.empty(); });
    }
}

extern "C" {

int tf_server_plan_admission(int n, const int64_t *need, int32_t *bypassed, int64_t room,
                             int64_t budget_left, int slots, int max_bypass, int32_t *admit) {
    int started = 0;
    for (int i = 0; i < n; ++i) admit[i] = 0;
    for (int i = 0; i < n && started < slots; ++i) {
        const bool fits = need[i] <= room && (budget_left < 0 || need[i] <= budget_left);
        if (fits) {
            admit[i] = 1;
            ++started;
            room -= need[i];
            if (budget_left >= 0) budget_left -= need[i];
            // every earlier job still waiting has been passed once more
            for (int k = 0; k < i; ++k)
                if (!admit[k]) ++bypassed[k];
            continue;
        }
        // a job that may be passed no more holds everything behind it
        if (max_bypass < 0 || bypassed[i] >= max_bypass) break;
    }
    return started;
}

tf_status tf_server_create(const tf_server_config *cfg, tf_ctx *model, tf_server **out) {
    if (!out) return TF_EINVAL;
    *out = nullptr;
    tf_server_config c = cfg ? *cfg : tf_server_config{};
    if (c.hbm_budget < 0 || c.hbm_reserve < 0 || c.max_running < 0 || c.max_running > 256 ||
        c.max_batch < 0 || c.max_batch > 65536) {
        g_server_create_err = "server configuration out of range";
        return TF_EINVAL;
    }
    if (c.hbm_reserve == 0) c.hbm_reserve = (int64_t)1 << 30;
    if (c.max_running == 0) c.max_running = 8;
    if (c.max_batch == 0) c.max_batch = 256;
    if (c.max_bypass == 0) c.max_bypass = 8;
    if (c.reserve_sms == 0) c.reserve_sms = model ? 8 : -1;
    auto s = std::make_unique<tf_server>();
    s->cfg = c;
    s->t0 = Clock::now();
    size_t fb = 0, tb = 0;
    if (cudaGetDevice(&s->device) != cudaSuccess || cudaMemGetInfo(&fb, &tb) != cudaSuccess) {
        cudaGetLastError();
        g_server_create_err = "no CUDA device";
        return TF_ECUDA;
    }
    s->device_total = (int64_t)tb;
    if (model) {
        int N = 0, K = 0;
        tf_dtype dt = TF_F32;
        tf_status r = tf_get_shape(model, &N, &K, &dt);
        if (r == TF_OK) r = tf_get_stream(model, &s->model_old_stream);
        if (r != TF_OK) {
            g_server_create_err = "model context unusable";
            return r;
        }
        int lo = 0, hi = 0;
        cudaDeviceGetStreamPriorityRange(&lo, &hi);
        if (cudaStreamCreateWithPriority(&s->hi, cudaStreamNonBlocking, hi) != cudaSuccess) {
            cudaGetLastError();
            g_server_create_err = "stream creation failed";
            return TF_ECUDA;
        }
        r = tf_set_stream(model, s->hi);
        if (r != TF_OK) {
            cudaStreamDestroy(s->hi);
            g_server_create_err = "could not move the model to the server's stream";
            return r;
        }
        s->model = model;
        s->model_N = N;
        s->model_K = K;
        s->model_dtype = dt;
    }
    try {
        s->sched = std::thread(&tf_server::run_scheduler, s.get());
        s->batcher = std::thread(&tf_server::run_batcher, s.get());
    } catch (...) {
        {
            std::lock_guard<std::mutex> g(s->mu);
            s->stop = true;
        }
        s->cv_work.notify_all();
        s->cv_fold.notify_all();
        if (s->sched.joinable()) s->sched.join();
        if (s->batcher.joinable()) s->batcher.join();
        if (s->model) {
            tf_set_stream(s->model, s->model_old_stream);
            cudaStreamDestroy(s->hi);
        }
        g_server_create_err = "could not start the server's threads";
        return TF_ENOMEM;
    }
    *out = s.release();
    return TF_OK;
}

void tf_server_destroy(tf_server *srv) {
    if (!srv) return;
    std::vector<std::shared_ptr<Job>> all;
    {
        std::lock_guard<std::mutex> g(srv->mu);
        srv->stop = true;
        for (auto &j : srv->queue) {
            j->info.state = TF_JOB_FAILED;
            j->info.status = TF_EBUSY;
            ++srv->st.jobs_failed;
        }
        srv->queue.clear();
        for (auto &q : srv->fq) {
            q->done = true;
            q->status = 16 + TF_EBUSY;
            q->done_at = Clock::now();
        }
        srv->fq.clear();
        for (auto &kv : srv->jobs) all.push_back(kv.second);
        srv->cv_work.notify_all();
        srv->cv_fold.notify_all();
        srv->cv_done.notify_all();
    }
    srv->sched.join();
    srv->batcher.join();
    for (auto &j : all) {
        if (j->worker.joinable()) j->worker.join();
        std::lock_guard<std::mutex> u(j->use);
        tf_destroy(j->ctx);
        j->ctx = nullptr;
        if (j->stream) cudaStreamDestroy(j->stream);
        j->stream = nullptr;
    }
    if (srv->model) {
        tf_set_stream(srv->model, srv->model_old_stream);
        cudaStreamDestroy(srv->hi);
    }
    delete srv;
}

const char *tf_server_last_error(const tf_server *srv) {
    return srv ? srv->err.c_str() : g_server_create_err.c_str();
}

tf_status tf_server_submit_job(tf_server *srv, const tf_job_desc *d, int64_t *job_id) {
    if (!srv || !d || !job_id) return TF_EINVAL;
    auto fail = [&](tf_status s, const char *why) {
        std::lock_guard<std::mutex> g(srv->mu);
        srv->err = why;
        return s;
    };
    if (!d->coords || !d->values || !d->dims || d->N < 1 || d->nnz < 0 || d->K < 1 ||
        d->C < 1 || d->C > d->K || d->T_in < 1 || d->sweeps < 1 || !(d->lambda >= 0.0) ||
        (d->dtype != TF_F32 && d->dtype != TF_F64) || (d->sweep_flags & ~TF_WEIGHTED_LAMBDA))
        return fail(TF_EINVAL, "job description out of range");
    int64_t need = 0;
    tf_status s = tf_estimate_bytes(d->dims, d->N, d->nnz, d->K, d->C, d->dtype, 0, 0, &need);
    if (s != TF_OK) return fail(s, "job shape refused (tf_estimate_bytes)");
    const int64_t cap = srv->cfg.hbm_budget > 0
                            ? std::min(srv->cfg.hbm_budget, srv->device_total - srv->cfg.hbm_reserve)
                            : srv->device_total - srv->cfg.hbm_reserve;
    if (need > cap) return fail(TF_ENOMEM, "job can never fit the device memory or budget");
    if (d->col_orders)
        for (int t = 0; t < d->sweeps; ++t) {
            std::vector<char> seen((size_t)d->K, 0);
            for (int k = 0; k < d->K; ++k) {
                const int32_t c = d->col_orders[(size_t)t * d->K + k];
                if (c < 0 || c >= d->K || seen[c]) return fail(TF_EINVAL, "col_orders row is not a permutation");
                seen[c] = 1;
            }
        }
    std::shared_ptr<Job> j;
    try {  // the host copy of the inputs
        j = std::make_shared<Job>();
        j->d = *d;
        j->dims.assign(d->dims, d->dims + d->N);
        j->coords.assign(d->coords, d->coords + (size_t)d->nnz * d->N);
        const char *v = static_cast<const char *>(d->values);
        j->values.assign(v, v + (size_t)d->nnz * elem_bytes(d->dtype));
        if (d->col_orders)
            j->orders.assign(d->col_orders, d->col_orders + (size_t)d->sweeps * d->K);
    } catch (...) {
        return fail(TF_ENOMEM, "host copy of the job's inputs failed");
    }
    j->d.coords = nullptr;
    j->d.values = nullptr;
    j->d.dims = nullptr;
    j->d.col_orders = nullptr;
    j->info.state = TF_JOB_QUEUED;
    j->info.status = TF_OK;
    j->info.bytes = need;
    j->info.started_s = j->info.finished_s = -1;
    std::lock_guard<std::mutex> g(srv->mu);
    if (srv->stop) return TF_EBUSY;
    j->id = srv->next_id++;
    j->info.queued_s = srv->now();
    srv->jobs[j->id] = j;
    srv->queue.push_back(j);
    *job_id = j->id;
    srv->cv_work.notify_all();
    return TF_OK;
}

tf_status tf_server_job_info(tf_server *srv, int64_t id, tf_job_info *info) {
    if (!srv || !info) return TF_EINVAL;
    std::lock_guard<std::mutex> g(srv->mu);
    auto it = srv->jobs.find(id);
    if (it == srv->jobs.end()) return TF_EINVAL;
    *info = it->second->info;
    return TF_OK;
}

tf_status tf_server_wait_job(tf_server *srv, int64_t id, double timeout_s, tf_job_info *info) {
    if (!srv || !(timeout_s >= 0)) return TF_EINVAL;
    std::unique_lock<std::mutex> lk(srv->mu);
    auto it = srv->jobs.find(id);
    if (it == srv->jobs.end()) return TF_EINVAL;
    auto j = it->second;
    const auto until = Clock::now() + std::chrono::duration_cast<Clock::duration>(
                                          std::chrono::duration<double>(std::min(timeout_s, 1e7)));
    const bool fin = srv->cv_done.wait_until(lk, until, [&] {
        return j->info.state == TF_JOB_DONE || j->info.state == TF_JOB_FAILED;
    });
    if (info) *info = j->info;
    return fin ? TF_OK : TF_ETIMEOUT;
}

tf_status tf_server_job_factors(tf_server *srv, int64_t id, int n, void *host_A) {
    if (!srv || !host_A) return TF_EINVAL;
    std::shared_ptr<Job> j;
    {
        std::lock_guard<std::mutex> g(srv->mu);
        auto it = srv->jobs.find(id);
        if (it == srv->jobs.end()) return TF_EINVAL;
        if (it->second->info.state != TF_JOB_DONE) return TF_EBUSY;
        j = it->second;
    }
    std::lock_guard<std::mutex> u(j->use);  // a concurrent release waits for this copy
    if (!j->ctx) return TF_EINVAL;           // released in the meantime
    return tf_get_factors(j->ctx, n, host_A);
}

tf_status tf_server_release_job(tf_server *srv, int64_t id) {
    if (!srv) return TF_EINVAL;
    std::shared_ptr<Job> j;
    {
        std::lock_guard<std::mutex> g(srv->mu);
        auto it = srv->jobs.find(id);
        if (it == srv->jobs.end()) return TF_EINVAL;
        j = it->second;
        if (j->info.state != TF_JOB_DONE && j->info.state != TF_JOB_FAILED) return TF_EBUSY;
        srv->jobs.erase(it);
    }
    if (j->worker.joinable()) j->worker.join();
    {
        std::lock_guard<std::mutex> u(j->use);
        tf_destroy(j->ctx);  // stream-ordered frees: no wait on other streams
        j->ctx = nullptr;
        if (j->stream) cudaStreamDestroy(j->stream);
        j->stream = nullptr;
    }
    std::lock_guard<std::mutex> g(srv->mu);
    if (j->info.started_s >= 0) srv->admitted_bytes -= j->info.bytes;
    srv->cv_work.notify_all();
    return TF_OK;
}

tf_status tf_server_submit_foldin(tf_server *srv, int mode, const int32_t *other,
                                  const void *vals, int64_t m, double lambda, int64_t *req_id) {
    if (!srv || !req_id || m < 0 || (m > 0 && (!other || !vals))) return TF_EINVAL;
    if (!srv->model || mode < 0 || mode >= srv->model_N || !(lambda >= 0.0)) return TF_EINVAL;
    std::shared_ptr<Foldin> q;
    try {  // the host copy of the request
        q = std::make_shared<Foldin>();
        q->mode = mode;
        q->lambda = lambda;
        q->m = m;
        q->other.assign(other, other + (size_t)m * (srv->model_N - 1));
        const char *v = static_cast<const char *>(vals);
        q->vals.assign(v, v + (size_t)m * elem_bytes(srv->model_dtype));
    } catch (...) {
        return TF_ENOMEM;
    }
    q->submitted = Clock::now();
    std::lock_guard<std::mutex> g(srv->mu);
    if (srv->stop) return TF_EBUSY;
    q->id = srv->next_id++;
    srv->foldins[q->id] = q;
    srv->fq.push_back(q);
    *req_id = q->id;
    srv->cv_fold.notify_one();
    return TF_OK;
}

tf_status tf_server_wait_foldin(tf_server *srv, int64_t id, double timeout_s, void *out_row,
                                int32_t *req_status, double *latency_s) {
    if (!srv || !(timeout_s >= 0)) return TF_EINVAL;
    std::unique_lock<std::mutex> lk(srv->mu);
    auto it = srv->foldins.find(id);
    if (it == srv->foldins.end()) return TF_EINVAL;
    auto q = it->second;
    const auto until = Clock::now() + std::chrono::duration_cast<Clock::duration>(
                                          std::chrono::duration<double>(std::min(timeout_s, 1e7)));
    if (!srv->cv_done.wait_until(lk, until, [&] { return q->done; })) return TF_ETIMEOUT;
    if (out_row && !q->row.empty()) memcpy(out_row, q->row.data(), q->row.size());
    if (req_status) *req_status = q->status;
    if (latency_s) *latency_s = secs(q->submitted, q->done_at);
    srv->foldins.erase(it);
    return TF_OK;
}

tf_status tf_server_get_stats(tf_server *srv, tf_server_stats *out) {
    if (!srv || !out) return TF_EINVAL;
    std::lock_guard<std::mutex> g(srv->mu);
    *out = srv->st;
    out->jobs_queued = (int64_t)srv->queue.size();
    out->jobs_running = srv->running;
    out->bytes_admitted = srv->admitted_bytes;
    return TF_OK;
}

}  // extern "C"
