// C ABI of the SALS / CDTF library: context lifecycle, layout construction and the
// sweep driver.  Everything the method computes runs in the kernels of this library;
// the host only validates arguments, plans the row schedule once per tensor, and
// queues kernels on the context's stream.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <exception>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <type_traits>
#include <thread>
#include <vector>

#include <cuda.h>

#include "gather_plan.cuh"
#include "layout.cuh"
#include "sweep.cuh"

namespace tfs {

// Device buffer owned by a context, allocated and freed in the order of the context's
// stream (from the library's pool / cudaFreeAsync).  cudaFree waits for every stream of the device,
// so a context built or destroyed beside running work (a serving process admitting and
// retiring jobs) would stall all other work on the GPU; stream-ordered calls wait for
// nothing but the context's own stream.  `s` is the stream the buffer is freed on; it
// follows the context when tf_set_stream moves it.
template <class T>
struct Buf {
    T *p = nullptr;
    size_t n = 0;
    cudaStream_t s = nullptr;
    Buf() = default;
    Buf(const Buf &) = delete;
    Buf &operator=(const Buf &) = delete;
    ~Buf() { reset(); }
    void reset() {
        if (p) cudaFreeAsync(p, s);
        p = nullptr;
        n = 0;
    }
    void alloc(size_t count, cudaStream_t st) {
        reset();
        if (count == 0) count = 1;
        s = st;
        cudaError_t e = pool_alloc(reinterpret_cast<void **>(&p), count * sizeof(T), st);
        if (e != cudaSuccess) {
            p = nullptr;
            cudaGetLastError();
            throw ApiError{TF_ENOMEM, "device allocation of " + std::to_string(count * sizeof(T)) +
                                          " bytes failed"};
        }
        n = count;
    }
    // Growable scratch: capacity grows by at least half each time.
    void ensure(size_t count, cudaStream_t st) {
        if (count > n) alloc(std::max(count, n + n / 2), st);
    }
};

// Page-locked host blocks reused across contexts.  cudaFreeHost waits for the whole
// device, so a destroyed context returns its staging block to this list instead; blocks
// live as long as the process.  Sizes are rounded up to powers of two (>= 4 KiB).
class PinnedCache {
  public:
    void *get(size_t bytes) {
        const size_t sz = round(bytes);
        {
            std::lock_guard<std::mutex> g(m_);
            auto it = free_.find(sz);
            if (it != free_.end() && !it->second.empty()) {
                void *q = it->second.back();
                it->second.pop_back();
                return q;
            }
        }
        void *q = nullptr;
        if (cudaMallocHost(&q, sz) != cudaSuccess) {
            cudaGetLastError();
            throw ApiError{TF_ENOMEM, "page-locked allocation failed"};
        }
        return q;
    }
    void put(void *q, size_t bytes) {
        if (!q) return;
        std::lock_guard<std::mutex> g(m_);
        free_[round(bytes)].push_back(q);
    }

  private:
    static size_t round(size_t b) {
        size_t sz = 4096;
        while (sz < b) sz <<= 1;
        return sz;
    }
    std::mutex m_;
    std::map<size_t, std::vector<void *>> free_;
};

PinnedCache &pinned_cache() {
    static PinnedCache c;
    return c;
}

// Page-locked staging of host-to-device copies queued on a stream.  cudaMemcpyAsync from
// pageable memory returns only once the stream has reached the copy, which would hold
// the host behind all device work queued before it; from page-locked memory it returns at
// once.  The blocks go back to the cache after the stream has passed the last copy out of
// them (also when the caller fails part way).
struct PinnedStage {
    std::vector<std::pair<void *, size_t>> blocks;
    cudaEvent_t done = nullptr;
    char *arena = nullptr;  // one block taken up front, handed out in 16-byte steps
    size_t arena_bytes = 0, used = 0;
    // Takes the block before any device work is queued: a first page-locked allocation
    // is not stream-ordered and would otherwise wait on the work queued before it.
    void reserve(size_t bytes) {
        arena = static_cast<char *>(pinned_cache().get(bytes));
        blocks.emplace_back(arena, bytes);
        arena_bytes = bytes;
    }
    void copy(void *dst, const void *src, size_t bytes, cudaStream_t st) {
        if (bytes == 0) return;
        void *p = nullptr;
        const size_t at = (used + 15) / 16 * 16;
        if (arena && at + bytes <= arena_bytes) {
            p = arena + at;
            used = at + bytes;
        } else {
            p = pinned_cache().get(bytes);
            blocks.emplace_back(p, bytes);
        }
        memcpy(p, src, bytes);
        if (!done) TFS_CUDA(cudaEventCreateWithFlags(&done, cudaEventDisableTiming));
        TFS_CUDA(cudaMemcpyAsync(dst, p, bytes, cudaMemcpyHostToDevice, st));
        TFS_CUDA(cudaEventRecord(done, st));
    }
    PinnedStage() = default;
    PinnedStage(const PinnedStage &) = delete;
    PinnedStage &operator=(const PinnedStage &) = delete;
    ~PinnedStage() {
        if (done) cudaEventSynchronize(done);
        for (auto &b : blocks) pinned_cache().put(b.first, b.second);
        if (done) cudaEventDestroy(done);
    }
};

cudaMemPool_t library_pool() {
    static std::mutex mu;
    static std::map<int, cudaMemPool_t> pools;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    std::lock_guard<std::mutex> g(mu);
    auto it = pools.find(dev);
    if (it != pools.end()) return it->second;
    cudaMemPoolProps props{};
    props.allocType = cudaMemAllocationTypePinned;
    props.handleTypes = cudaMemHandleTypeNone;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = dev;
    cudaMemPool_t pool = nullptr;
    if (cudaMemPoolCreate(&pool, &props) != cudaSuccess) {
        cudaGetLastError();
        pools[dev] = nullptr;
        return nullptr;
    }
    uint64_t keep = UINT64_MAX;
    int no = 0;
    cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
    cudaMemPoolSetAttribute(pool, cudaMemPoolReuseAllowInternalDependencies, &no);
    cudaGetLastError();
    pools[dev] = pool;
    return pool;
}

struct ModeLayout {
    int64_t I = 0;
    Buf<int64_t> off;       // [I + 1]
    Buf<int32_t> perm;      // [nnz] canonical index per sorted position
    Buf<int32_t> oidx;      // [(N-1) * nnz] other-mode indices, mode order
    Buf<tf_item> items;
    Buf<int64_t> bin_ptr;   // [P + 1]
    Buf<SplitRow> split;    // rows held by several items (chunks)
    Buf<SplitRow> single;   // rows held by one item
    int64_t n_items = 0, n_slots = 0;
    int n_split = 0, n_single = 0;
    int64_t ostride = 0;    // elements between two other-mode index arrays
    Buf<int32_t> rank_of;   // row id -> degree rank (slice row)
    Buf<int32_t> id_of;     // degree rank -> row id
    Buf<int32_t> groups;    // slot groups of split rows (first slot, count), wide subsets
    int n_groups = 0;
    std::vector<int64_t> deg_cum;  // host: entries of the first R rows in degree-rank order
    // per bin, the step units and entries of the bins before it (gather-plan regions)
    Buf<uint32_t> plan_base;  // [2 (P + 1)]
    int64_t plan_units = 0;   // step units of all bins
    int P = 0;
    int omode[kMaxModes - 1];
    template <class F>
    void each_buf(F f) {
        f(off), f(perm), f(oidx), f(items), f(bin_ptr), f(split), f(single), f(rank_of),
            f(id_of), f(groups), f(plan_base);
    }
};

// The packed-key layout build applies when one 64-bit key holds every coordinate.
inline bool packed_layout_applies(const int64_t *dims, int N, int64_t nnz, uint32_t flags) {
    return !(flags & TF_LAYOUT_FIELD_SORTS) && nnz > 0 && packed_key_bits(dims, N) <= 64;
}

struct CtxBase {
    std::string err;
    tf_dtype dtype;
    int device = 0;  // ordinal of the device current when the context was created
    virtual ~CtxBase() = default;
};

template <class T>
struct Impl : CtxBase {
    int N = 0, K = 0;
    int64_t nnz = 0;
    std::vector<int64_t> dims;
    cudaStream_t st = nullptr;
    uint64_t seed = 0;
    int num_sms = 0;
    int sm_limit = 0;  // blocks of the persistent mode passes (0: one per SM)
    int pass_sms() const { return sm_limit > 0 && sm_limit < num_sms ? sm_limit : num_sms; }
    tf_sched_policy policy = TF_SCHED_LPT;
    int P = 0;

    Buf<T> x;                      // canonical values
    Buf<T> A[kMaxModes];           // factor matrices
    Buf<T> res[kMaxModes];         // residual copies, mode-n order
    Buf<T> Z[kMaxModes];           // packed slices
    ModeLayout mode[kMaxModes];
    Buf<T> partials;
    Buf<int32_t> d_order, d_Q;
    Buf<DeviceStatus> stat;
    Buf<unsigned long long> ticket;  // bin counter of the mode passes
    unsigned long long ticket_base = 0;
    Buf<double> red;               // reduction scratch
    Buf<int64_t> d_dims;
    Buf<int32_t> f_other;          // fold-in scratch
    Buf<T> f_x, f_out, f_part, f_fac;
    Buf<double> f_rpart;           // fold-in refinement: factors and FP64 partial residuals
    Buf<int64_t> f_meta;           // tiled fold-in block table / request offsets / status
    Buf<int32_t> p_coords;         // tf_predict staging
    Buf<T> p_out;
    int32_t *h_order = nullptr;    // pinned staging of the column order
    cudaEvent_t order_ev = nullptr;
    bool order_pending = false;

    // kernel timing (tf_profile): event pairs per launch, folded in at tf_get_profile
    bool prof_on = false;
    std::vector<std::pair<cudaEvent_t, cudaEvent_t>> prof_pending;
    std::vector<int> prof_kind, prof_mode;
    std::vector<int32_t> trace_kind, trace_mode;
    std::vector<float> trace_ms;
    int64_t prof_launches[TF_KIND_COUNT] = {0};
    double prof_ms[TF_KIND_COUNT] = {0};

    int path = 0;                  // 0 auto, 1 cp.async SIMT pass, 2 TMA pass when supported,
                                   // 3 lean float pass (three-way tensors), 4 the lean pass
                                   // with its Gram on the tensor cores
    int lean_cache_rows = -1;      // lean pass: cached rows per other mode (< 0: as fit)
    int lean_ring_cap = 32;        // lean pass: staged cold rows per step (both modes)
    int lean_warps = 0;            // lean pass: warps per block (0: default)
    // Gather plans of the lean pass, built once per (mode, cache rows, pool, refresh
    // flavour, row schedule) and reused by every later split and sweep.
    struct GatherPlan {
        int n = -1, RR = 0, RV = 0, cap = 0, first = 0;
        int64_t layout_gen = -1;
        Buf<unsigned char> steps;  // GStep records then the per-record own-row ranks
        Buf<uint32_t> step_range, word;
        Buf<int32_t> list;
        int64_t nsteps = 0;
        uint64_t used = 0;  // last use (LRU)
    };
    std::vector<std::unique_ptr<GatherPlan>> gplans;
    uint64_t gplan_clock = 0;
    int precision = 0;             // 0 FP32-level, 1 single-TF32 tensor-core Gram, 2 / 3
                                   // bfloat16 varying-mode / other-mode rows in the lean pass
    Buf<uint16_t> Zb[kMaxModes];   // bfloat16 copies of the slices (precision 2)
    int solve_refine = 0;          // float: one refinement step of every row solve
    float solve_cond = 0.f;        // float: FP64 solve of rows with pivot ratio < 1 / this
    CUtensorMap tmaps[kMaxModes][3];  // per mode: slice maps with boxes 8, 24, 40 floats
    const void *tmaps_for_Z[kMaxModes] = {nullptr};
    int Cq = 0, CM_last = 1;       // columns Q held by the copies' R-hat; register width
                                   // (and so slice layout) of the sweep that left them
    bool dirty = false;            // residual copies must be rebuilt from the factors
    bool a0_zero = true;           // A^(1) known to be zero (R = X)
    int64_t sweeps = 0, last_launches = 0, loss_launches = 0;
    int64_t last_path = 0;  // mode-pass paths of the last sweep: bit 0 cp.async, bit 1 TMA
    int64_t launches = 0;
    int64_t layout_gen = 0;  // bumped whenever the row schedule is rebuilt

    // Every device buffer of the context (tf_set_stream moves their frees to the new stream).
    template <class F>
    void each_buf(F f) {
        f(x), f(partials), f(d_order), f(d_Q), f(stat), f(ticket), f(red), f(d_dims);
        f(f_other), f(f_x), f(f_out), f(f_part), f(f_fac), f(f_rpart), f(f_meta), f(p_coords),
            f(p_out);
        for (int n = 0; n < kMaxModes; ++n) {
            f(A[n]), f(res[n]), f(Z[n]), f(Zb[n]);
            mode[n].each_buf(f);
        }
        for (auto &g : gplans) f(g->steps), f(g->step_range), f(g->word), f(g->list);
    }

    ~Impl() override {
        drop_graphs();
        // device buffers go back to the pool behind the last work on st (their destructors)
        if (order_pending) cudaEventSynchronize(order_ev);  // the last copy out of h_order
        if (h_order) pinned_cache().put(h_order, sizeof(int32_t) * (size_t)K);
        if (order_ev) cudaEventDestroy(order_ev);
        for (auto &pr : prof_pending) {
            cudaEventDestroy(pr.first);
            cudaEventDestroy(pr.second);
        }
    }

    // Brackets one launch with events when profiling is on.
    int cur_mode = -1;  // mode recorded with the next timed launches

    template <class F>
    void timed(int kind, F &&launch) {
        if (!prof_on) {
            launch();
            return;
        }
        cudaEvent_t a, b;
        TFS_CUDA(cudaEventCreate(&a));
        TFS_CUDA(cudaEventCreate(&b));
        TFS_CUDA(cudaEventRecord(a, st));
        launch();
        TFS_CUDA(cudaEventRecord(b, st));
        prof_pending.push_back({a, b});
        prof_kind.push_back(kind);
        prof_mode.push_back(cur_mode);
    }

    void profile(int enable) {
        TFS_CUDA(cudaStreamSynchronize(st));
        for (auto &pr : prof_pending) {
            cudaEventDestroy(pr.first);
            cudaEventDestroy(pr.second);
        }
        prof_pending.clear();
        prof_kind.clear();
        prof_mode.clear();
        trace_kind.clear();
        trace_mode.clear();
        trace_ms.clear();
        for (int k = 0; k < TF_KIND_COUNT; ++k) {
            prof_launches[k] = 0;
            prof_ms[k] = 0.0;
        }
        prof_on = enable != 0;
    }

    void get_profile(int64_t *launches_out, double *ms_out) {
        TFS_CUDA(cudaStreamSynchronize(st));
        for (size_t i = 0; i < prof_pending.size(); ++i) {
            float ms = 0.f;
            TFS_CUDA(cudaEventElapsedTime(&ms, prof_pending[i].first, prof_pending[i].second));
            prof_launches[prof_kind[i]] += 1;
            prof_ms[prof_kind[i]] += ms;
            trace_kind.push_back(prof_kind[i]);
            trace_mode.push_back(prof_mode[i]);
            trace_ms.push_back(ms);
            cudaEventDestroy(prof_pending[i].first);
            cudaEventDestroy(prof_pending[i].second);
        }
        prof_pending.clear();
        prof_kind.clear();
        prof_mode.clear();
        for (int k = 0; k < TF_KIND_COUNT; ++k) {
            if (launches_out) launches_out[k] = prof_launches[k];
            if (ms_out) ms_out[k] = prof_ms[k];
        }
    }

    // A mode's row schedule on the host (items grouped by bin, split and single rows).
    struct PlanHost {
        std::vector<tf_item> items;
        std::vector<int64_t> bin_ptr;
        std::vector<SplitRow> split, single;
        std::vector<int32_t> groups;  // slot groups of rows with many chunks (wide subsets)
        int64_t n_slots = 0;
        // gather-plan regions: step units (max(1, ceil(len / 32)) per item) and entries
        // of the bins before each bin, [P + 1] each
        std::vector<uint32_t> plan_base;
        int64_t plan_units = 0;
    };

    // Host vectors whose device copies are queued on st during the build: they live
    // until create synchronises.
    struct BuildHost {
        std::vector<PlanHost> plans;
        std::vector<std::vector<int64_t>> offs;
        std::vector<std::vector<int32_t>> ids, ranks;
        PinnedStage stage;  // declared last: destroyed first, once its copies have run
    };

    // ------------------------------------------------------------ construction
    void create(const int32_t *coords, const void *values, const int64_t *dims_in, int N_,
                int64_t nnz_, int K_, uint64_t seed_, cudaStream_t st_, uint32_t flags) {
        N = N_;
        K = K_;
        nnz = nnz_;
        seed = seed_;
        st = st_;
        dims.assign(dims_in, dims_in + N);
        int dev = 0;
        TFS_CUDA(cudaGetDevice(&dev));
        device = dev;
        TFS_CUDA(cudaDeviceGetAttribute(&num_sms, cudaDevAttrMultiProcessorCount, dev));
        P = default_bins(num_sms, nnz);
        stat.alloc(1, st);
        TFS_CUDA(cudaMemsetAsync(stat.p, 0, sizeof(DeviceStatus), st));
        ticket.alloc(1, st);
        TFS_CUDA(cudaMemsetAsync(ticket.p, 0, sizeof(unsigned long long), st));
        ticket_base = 0;
        red.ensure(4096, st);
        d_dims.alloc(N, st);
        TFS_CUDA(cudaMemcpyAsync(d_dims.p, dims.data(), N * sizeof(int64_t),
                                 cudaMemcpyHostToDevice, st));
        h_order = static_cast<int32_t *>(pinned_cache().get(sizeof(int32_t) * (size_t)K));
        TFS_CUDA(cudaEventCreateWithFlags(&order_ev, cudaEventDisableTiming));
        d_order.alloc(K, st);
        d_Q.alloc(K, st);

        const bool on_dev = flags & TF_INPUT_DEVICE;
        const cudaMemcpyKind kind = on_dev ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
        x.alloc(nnz, st);
        const bool packed = packed_layout_applies(dims.data(), N, nnz, flags);
        BuildHost bh;
        {
            // staged host-to-device bytes of the build at most: per mode its row offsets and
            // degree tables, and its schedule (items at most rows + bins, bin offsets, row
            // lists, slot groups, plan regions)
            size_t b = 0;
            for (int n = 0; n < N; ++n) {
                const size_t I = (size_t)dims[n], it = I + (size_t)P + 1;
                b += 16 * I + 8 + sizeof(tf_item) * it + 8 * ((size_t)P + 1) + sizeof(SplitRow) * I +
                     8 * it + 8 * ((size_t)P + 1) + 12 * 16;
            }
            bh.stage.reserve(b);
            // and the landing block of the packed build's row counts, cached now for the
            // same reason
            if (packed) {
                int64_t sum_I = 0;
                for (int n = 0; n < N; ++n) sum_I += dims[n];
                const size_t cb = (size_t)sum_I * sizeof(uint32_t);
                pinned_cache().put(pinned_cache().get(cb), cb);
            }
        }
        if (packed) {
            build_packed(coords, values, on_dev, bh);
        } else {
            if (nnz > 0) TFS_CUDA(cudaMemcpyAsync(x.p, values, nnz * sizeof(T), kind, st));
            build_general(coords, on_dev, bh);
        }
        for (int n = 0; n < N; ++n) plan_upload(n, bh.plans[n], bh.stage);

        // Algorithm 1 initialisation: A^(1) = 0, the other modes random, so R = X.
        const double std = pow((double)K, -1.0 / (2.0 * N));
        for (int n = 0; n < N; ++n) {
            A[n].alloc((size_t)dims[n] * K, st);
            if (n == 0)
                TFS_CUDA(cudaMemsetAsync(A[n].p, 0, (size_t)dims[n] * K * sizeof(T), st));
            else
                launch_init_normal<T>(A[n].p, dims[n] * K, seed, (uint64_t)n, std, st);
        }
        a0_zero = true;
        if (packed) {  // the sorts carried X into every residual copy (R = X)
            Cq = 0;
            dirty = false;
        } else {
            for (int n = 0; n < N; ++n) {
                res[n].alloc(nnz + 64, st);
                TFS_CUDA(cudaMemsetAsync(res[n].p, 0, (nnz + 64) * sizeof(T), st));
            }
            rebuild_residuals();
        }
        TFS_CUDA(cudaStreamSynchronize(st));  // host copies of the schedules and tables read
        if (packed) {
            const DeviceStatus s = read_status();
            if (s.bits & kStatRange)
                throw ApiError{TF_ERANGE, "a coordinate is negative or not below its mode length"};
            if (s.bits & kStatDup)
                throw ApiError{TF_EDUP, "two observed entries share a coordinate"};
        }
    }

    // The other-mode index arrays are written entry by entry (positions below nnz); only
    // their padding after nnz is zeroed here (all of it where no other mode exists).
    void zero_oidx_padding(ModeLayout &L) {
        if (N < 2) {
            TFS_CUDA(cudaMemsetAsync(L.oidx.p, 0, (size_t)L.ostride * sizeof(int32_t), st));
            return;
        }
        for (int t = 0; t < N - 1; ++t)
            TFS_CUDA(cudaMemsetAsync(L.oidx.p + (size_t)t * L.ostride + nnz, 0,
                                     (size_t)(L.ostride - nnz) * sizeof(int32_t), st));
    }

    // Per-mode sorted layout by key sorts of gathered coordinates: mode 0's order by N
    // stable sorts of one mode's indices each (least significant mode first), every other
    // mode's by one stable sort of the next mode's order; used where the coordinates do
    // not fit one 64-bit key (or on request, TF_LAYOUT_FIELD_SORTS).
    void build_general(const int32_t *coords, bool on_dev, BuildHost &bh) {
        // canonical coordinates -> SoA with range check
        Buf<int32_t> soa;
        soa.alloc((size_t)N * nnz, st);
        {
            Buf<int32_t> rowmajor;
            const int32_t *src = coords;
            if (!on_dev && nnz > 0) {
                rowmajor.alloc((size_t)N * nnz, st);
                TFS_CUDA(cudaMemcpyAsync(rowmajor.p, coords, (size_t)N * nnz * sizeof(int32_t),
                                         cudaMemcpyHostToDevice, st));
                src = rowmajor.p;
            }
            launch_transpose_check(src, N, nnz, d_dims.p, soa.p, stat.p, st);
            DeviceStatus s = read_status();
            if (s.bits & kStatRange)
                throw ApiError{TF_ERANGE, "a coordinate is negative or not below its mode length"};
        }

        // per-mode sorted layout
        std::vector<std::vector<int64_t>> offs;
        std::vector<PlanHost> plans;
        SortWorkspace ws;
        Buf<uint32_t> keys;
        keys.alloc(nnz, st);
        try {
            // Mode 0's order, lexicographic in (i_0, i_1, ..., i_{N-1}), by N stable key sorts
            // (least significant mode first).  Then, for n = N-1 down to 1, mode n's order
            // (i_n, i_{n+1}, ..., i_{n-1}) is one stable sort by i_n of mode n+1's order:
            // equal i_n keep (i_{n+1}, ..., i_{n-1}, i_n), which is the rest of mode n's key.
            // 2N - 1 key sorts instead of N^2; the orders are total, so the same.
            auto sorted_by = [&](ModeLayout &L, int m) {
                launch_gather_keys(soa.p + (size_t)m * nnz, L.perm.p, keys.p, nnz, st);
                radix_sort_pairs(keys.p, L.perm.p, nnz, ceil_log2_u64((uint64_t)dims[m]), ws, st);
            };
            for (int n = 0; n < N; ++n) {
                mode[n].I = dims[n];
                mode[n].perm.alloc(nnz, st);
                mode[n].off.alloc(mode[n].I + 1, st);
            }
            launch_iota(mode[0].perm.p, nnz, st);
            for (int m = N - 1; m >= 0; --m) sorted_by(mode[0], m);
            launch_offsets(keys.p, nnz, mode[0].I, mode[0].off.p, st);
            launch_dup_check(soa.p, N, nnz, mode[0].perm.p, stat.p, st);
            {
                DeviceStatus s = read_status();
                if (s.bits & kStatDup)
                    throw ApiError{TF_EDUP, "two observed entries share a coordinate"};
            }
            for (int n = N - 1; n >= 1; --n) {
                ModeLayout &L = mode[n];
                const ModeLayout &next = mode[(n + 1) % N];
                TFS_CUDA(cudaMemcpyAsync(L.perm.p, next.perm.p, (size_t)nnz * sizeof(int32_t),
                                         cudaMemcpyDeviceToDevice, st));
                sorted_by(L, n);
                launch_offsets(keys.p, nnz, L.I, L.off.p, st);
            }
            // degree ranks: slices are stored with each mode's rows in decreasing order of
            // their entry counts (equal counts by row id); one host thread per mode
            offs = download_offsets();
            std::vector<std::vector<int32_t>> &ids = bh.ids, &ranks = bh.ranks;
            ids.assign((size_t)N, {});
            ranks.assign((size_t)N, {});
            run_per_mode([&](int n) {
                const int64_t I = mode[n].I;
                std::vector<int64_t> cnt((size_t)I);
                for (int64_t i = 0; i < I; ++i) cnt[i] = offs[n][i + 1] - offs[n][i];
                degree_order(n, cnt, ids[n], ranks[n]);
            });
            for (int n = 0; n < N; ++n) {
                ModeLayout &L = mode[n];
                L.id_of.alloc(L.I, st);
                L.rank_of.alloc(L.I, st);
                TFS_CUDA(cudaMemcpyAsync(L.id_of.p, ids[n].data(), L.I * sizeof(int32_t),
                                         cudaMemcpyHostToDevice, st));
                TFS_CUDA(cudaMemcpyAsync(L.rank_of.p, ranks[n].data(), L.I * sizeof(int32_t),
                                         cudaMemcpyHostToDevice, st));
            }
            for (int n = 0; n < N; ++n) {
                ModeLayout &L = mode[n];
                // index arrays start 256-byte aligned and end in 64 padding entries
                // (bulk copies read fixed windows past a step's last entry)
                L.ostride = (nnz + 64 + 63) / 64 * 64;
                L.oidx.alloc((size_t)std::max(N - 1, 1) * L.ostride, st);
                zero_oidx_padding(L);
                int t = 0;
                for (int l = 0; l < N; ++l) {
                    if (l == n) continue;
                    L.omode[t] = l;
                    launch_gather_rank(soa.p + (size_t)l * nnz, L.perm.p, mode[l].rank_of.p,
                                       L.oidx.p + (size_t)t * L.ostride, nnz, st);
                    ++t;
                }
            }
            // the row schedules, on the host while the device gathers the index streams
            plans = plan_all_host(offs);
        } catch (...) {
            ws.release(st);
            throw;
        }
        ws.release(st);
        keys.reset();
        soa.reset();

        bh.plans = std::move(plans);
        bh.offs = std::move(offs);
    }

    // Per-mode sorted layout from packed 64-bit keys (layout.cu).  The row counts come
    // from the packing pass; while the device sorts mode 0's keys the host turns them
    // into row offsets and degree ranks (one thread per mode), then schedules the rows
    // while the device sorts the other modes and extracts every mode's arrays.
    void build_packed(const int32_t *coords, const void *values, bool on_dev, BuildHost &bh) {
        const KeyFields f = key_fields(dims.data(), N);
        const int total_bits = packed_key_bits(dims.data(), N);
        int64_t sum_I = 0;
        for (int n = 0; n < N; ++n) sum_I += dims[n];
        Buf<uint64_t> kb[3];
        Buf<uint32_t> cnt;
        kb[0].alloc(nnz, st);
        cnt.alloc(sum_I, st);
        TFS_CUDA(cudaMemsetAsync(cnt.p, 0, sum_I * sizeof(uint32_t), st));
        Buf<int32_t> rowmajor;
        // Host inputs: the coordinates go up in chunks on a side stream and each chunk is
        // packed on st as soon as it has landed; the values go up behind them and are
        // first needed by mode 0's extraction, after mode 0's sort.  The side stream is
        // drained before anything it writes is freed (also when the build fails).
        struct Side {
            cudaStream_t s = nullptr;
            std::vector<cudaEvent_t> ev;
            cudaEvent_t make() {
                cudaEvent_t e = nullptr;
                TFS_CUDA(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
                ev.push_back(e);
                return e;
            }
            ~Side() {
                if (s) cudaStreamSynchronize(s);
                for (cudaEvent_t e : ev) cudaEventDestroy(e);
                if (s) cudaStreamDestroy(s);
            }
        } side;
        cudaEvent_t x_ready = nullptr;
        if (on_dev) {
            TFS_CUDA(cudaMemcpyAsync(x.p, values, nnz * sizeof(T), cudaMemcpyDeviceToDevice, st));
            launch_pack_count(coords, 0, nnz, f, kb[0].p, cnt.p, stat.p, st);
        } else {
            rowmajor.alloc((size_t)N * nnz, st);
            TFS_CUDA(cudaStreamCreateWithFlags(&side.s, cudaStreamNonBlocking));
            cudaEvent_t allocated = side.make();
            TFS_CUDA(cudaEventRecord(allocated, st));  // x and rowmajor exist from here on
            TFS_CUDA(cudaStreamWaitEvent(side.s, allocated, 0));
            constexpr int64_t kChunks = 16;
            const int64_t tile = pack_count_tile();
            const int64_t chunk = std::max<int64_t>(tile, ceil_div(ceil_div(nnz, kChunks), tile) * tile);
            for (int64_t e0 = 0; e0 < nnz; e0 += chunk) {
                const int64_t ne = std::min(chunk, nnz - e0);
                TFS_CUDA(cudaMemcpyAsync(rowmajor.p + (size_t)e0 * N, coords + (size_t)e0 * N,
                                         (size_t)ne * N * sizeof(int32_t), cudaMemcpyHostToDevice,
                                         side.s));
                cudaEvent_t landed = side.make();
                TFS_CUDA(cudaEventRecord(landed, side.s));
                TFS_CUDA(cudaStreamWaitEvent(st, landed, 0));
                launch_pack_count(rowmajor.p + (size_t)e0 * N, e0, ne, f, kb[0].p, cnt.p, stat.p, st);
            }
            TFS_CUDA(cudaMemcpyAsync(x.p, values, nnz * sizeof(T), cudaMemcpyHostToDevice, side.s));
            x_ready = side.make();
            TFS_CUDA(cudaEventRecord(x_ready, side.s));
        }
        rowmajor.reset();  // st has waited for every chunk
        // page-locked landing block of the counts; it goes back to the cache only after
        // the copy into it has completed (also when the build fails)
        struct CountsHost {
            uint32_t *p = nullptr;
            size_t bytes = 0;
            cudaEvent_t done = nullptr;
            ~CountsHost() {
                if (done) cudaEventSynchronize(done);
                if (p) pinned_cache().put(p, bytes);
                if (done) cudaEventDestroy(done);
            }
        } hc;
        TFS_CUDA(cudaEventCreateWithFlags(&hc.done, cudaEventDisableTiming));
        hc.bytes = (size_t)sum_I * sizeof(uint32_t);
        hc.p = static_cast<uint32_t *>(pinned_cache().get(hc.bytes));
        uint32_t *h_cnt = hc.p;
        cudaEvent_t counted = hc.done;
        TFS_CUDA(cudaMemcpyAsync(h_cnt, cnt.p, sum_I * sizeof(uint32_t), cudaMemcpyDeviceToHost, st));
        TFS_CUDA(cudaEventRecord(counted, st));

        Buf<int32_t> valt;
        Buf<T> xalt;
        KeySortWorkspace ws;
        struct WsBack {
            KeySortWorkspace &w;
            cudaStream_t s;
            ~WsBack() { w.release(s); }
        } ws_back{ws, st};
        for (int n = 0; n < N; ++n) {
            mode[n].I = dims[n];
            mode[n].perm.alloc(nnz, st);
            // residual copies: R = X at the start (A^(1) = 0): mode 0's gathered, the others'
            // carried with the keys from the previous mode's copy; 64 zero entries after them
            res[n].alloc(nnz + 64, st);
            TFS_CUDA(cudaMemsetAsync(res[n].p + nnz, 0, 64 * sizeof(T), st));
        }
        kb[1].alloc(nnz, st);
        kb[2].alloc(nnz, st);
        valt.alloc(nnz, st);
        xalt.alloc(nnz, st);
        // mode 0: the whole key, most significant field i_0
        radix_sort_keys64(kb[0].p, nullptr, nullptr, kb[1].p, mode[0].perm.p, nullptr, kb[2].p,
                          valt.p, nullptr, 0, nnz, 0, total_bits, ws, st);

        // row offsets and degree ranks on the host while the sort runs
        TFS_CUDA(cudaEventSynchronize(counted));
        bh.offs.assign((size_t)N, {});
        bh.ids.assign((size_t)N, {});
        bh.ranks.assign((size_t)N, {});
        run_per_mode([&](int n) {
            const int64_t I = dims[n];
            const uint32_t *c = h_cnt + f.cnt_off[n];
            std::vector<int64_t> count((size_t)I);
            std::vector<int64_t> &off = bh.offs[n];
            off.assign((size_t)I + 1, 0);
            for (int64_t i = 0; i < I; ++i) {
                count[i] = c[i];
                off[i + 1] = off[i] + c[i];
            }
            degree_order(n, count, bh.ids[n], bh.ranks[n]);
        });
        // page-locked staging: the copies queue behind mode 0's sort without holding the host
        for (int n = 0; n < N; ++n) {
            ModeLayout &L = mode[n];
            L.off.alloc(L.I + 1, st);
            L.id_of.alloc(L.I, st);
            L.rank_of.alloc(L.I, st);
            bh.stage.copy(L.off.p, bh.offs[n].data(), (L.I + 1) * sizeof(int64_t), st);
            bh.stage.copy(L.id_of.p, bh.ids[n].data(), L.I * sizeof(int32_t), st);
            bh.stage.copy(L.rank_of.p, bh.ranks[n].data(), L.I * sizeof(int32_t), st);
        }
        // the schedules on host threads while the device continues
        bh.plans.assign((size_t)N, {});
        std::vector<std::exception_ptr> plan_err((size_t)N);
        std::vector<std::thread> planners;
        struct Joiner {
            std::vector<std::thread> &t;
            ~Joiner() {
                for (auto &x : t)
                    if (x.joinable()) x.join();
            }
        } join_planners{planners};
        for (int n = 0; n < N; ++n)
            planners.emplace_back([&, n] {
                try {
                    bh.plans[n] = plan_host(bh.offs[n], dims[n]);
                } catch (...) {
                    plan_err[n] = std::current_exception();
                }
            });

        for (int n = 0; n < N; ++n) {
            ModeLayout &L = mode[n];
            L.ostride = (nnz + 64 + 63) / 64 * 64;
            L.oidx.alloc((size_t)std::max(N - 1, 1) * L.ostride, st);
            zero_oidx_padding(L);
            int t = 0;
            for (int l = 0; l < N; ++l)
                if (l != n) L.omode[t++] = l;
        }
        auto extract = [&](int n, const uint64_t *keys) {
            const ModeLayout &L = mode[n];
            ExtractArgs a{};
            a.n_other = N - 1;
            a.check_dup = n == 0 ? 1 : 0;
            for (int t = 0; t < N - 1; ++t) {
                const int l = L.omode[t];
                a.shift[t] = f.shift[l];
                a.bits[t] = f.bits[l];
                a.oidx[t] = L.oidx.p + (size_t)t * L.ostride;
                a.rank[t] = mode[l].rank_of.p;
            }
            if (n == 0) {  // R = X into mode 0's order; later modes' values come with their keys
                a.perm = L.perm.p;
                a.x = x.p;
                a.res = res[0].p;
                a.xbytes = (int)sizeof(T);
            }
            launch_extract(keys, nnz, a, stat.p, st);
        };
        if (x_ready) TFS_CUDA(cudaStreamWaitEvent(st, x_ready, 0));
        int cur = 1;
        extract(0, kb[cur].p);
        // mode n from mode n+1: a stable sort by the field i_n
        for (int n = N - 1; n >= 1; --n) {
            const int out = cur == 0 ? 1 : 0, alt = 3 - cur - out;
            radix_sort_keys64(kb[cur].p, mode[(n + 1) % N].perm.p, res[(n + 1) % N].p, kb[out].p,
                              mode[n].perm.p, res[n].p, kb[alt].p, valt.p, xalt.p, (int)sizeof(T),
                              nnz, f.shift[n], f.shift[n] + f.bits[n], ws, st);
            cur = out;
            extract(n, kb[cur].p);
        }
        for (auto &t : planners) t.join();
        for (auto &e : plan_err)
            if (e) std::rethrow_exception(e);
        // the range and duplicate flags are read once create has synchronised
    }

    // Rows of mode n in decreasing order of entry count, equal counts by row id: ids[r]
    // is the row at degree rank r, ranks its inverse; also the mode's cumulative counts
    // in that order (deg_cum).
    void degree_order(int n, const std::vector<int64_t> &count, std::vector<int32_t> &ids,
                      std::vector<int32_t> &ranks) {
        const int64_t I = (int64_t)count.size();
        const std::vector<int64_t> order = rows_by_degree(count);
        ids.resize((size_t)I);
        ranks.resize((size_t)I);
        std::vector<int64_t> &dc = mode[n].deg_cum;
        dc.assign((size_t)I + 1, 0);
        for (int64_t r = 0; r < I; ++r) {
            ids[r] = (int32_t)order[r];
            ranks[order[r]] = (int32_t)r;
            dc[r + 1] = dc[r] + count[order[r]];
        }
    }

    // f(n) for every mode on its own host thread; the first exception is rethrown.
    template <class F>
    void run_per_mode(F &&f) {
        std::vector<std::exception_ptr> errs((size_t)N);
        std::vector<std::thread> th;
        for (int n = 0; n < N; ++n)
            th.emplace_back([&, n] {
                try {
                    f(n);
                } catch (...) {
                    errs[n] = std::current_exception();
                }
            });
        for (auto &t : th) t.join();
        for (auto &e : errs)
            if (e) std::rethrow_exception(e);
    }

    // Row schedule of one mode, computed on the host from its row offsets (no device call,
    // so the modes' schedules can be computed in parallel threads).
    PlanHost plan_host(const std::vector<int64_t> &off, int64_t I) const {
        PlanHost h;
        tf_status s = plan_mode(off.data(), I, P, 0, policy, seed, h.items, h.n_slots, h.bin_ptr);
        if (s != TF_OK) throw ApiError{s, "row scheduling failed"};
        // rows and their slots (a row's slots are consecutive, in entry order):
        // single-item rows are solved by k_solve_rows, split rows by k_combine
        std::vector<int32_t> item_of_slot((size_t)h.n_slots, -1);
        for (size_t i = 0; i < h.items.size(); ++i) item_of_slot[(size_t)h.items[i].slot] = (int32_t)i;
        for (int64_t q = 0; q < h.n_slots;) {
            const tf_item &first = h.items[(size_t)item_of_slot[(size_t)q]];
            int64_t q2 = q + 1;
            while (q2 < h.n_slots && h.items[(size_t)item_of_slot[(size_t)q2]].row == first.row) ++q2;
            const int64_t r = first.row;
            const SplitRow sr{first.row, first.slot, (int32_t)(q2 - q), 0, off[r + 1] - off[r]};
            (q2 - q > 1 ? h.split : h.single).push_back(sr);
            q = q2;
        }
        for (const SplitRow &sr : h.split)
            if (sr.n_slots > kSlotGroup)
                for (int g = 0; g < sr.n_slots; g += kSlotGroup) {
                    h.groups.push_back(sr.first_slot + g);
                    h.groups.push_back(std::min(kSlotGroup, sr.n_slots - g));
                }
        {
            const int Pn = (int)h.bin_ptr.size() - 1;
            h.plan_base.assign((size_t)2 * (Pn + 1), 0u);
            uint64_t su = 0, se = 0;
            for (int b = 0; b < Pn; ++b) {
                h.plan_base[b] = (uint32_t)su;
                h.plan_base[Pn + 1 + b] = (uint32_t)se;
                for (int64_t it = h.bin_ptr[b]; it < h.bin_ptr[b + 1]; ++it) {
                    const int64_t len = h.items[it].len;
                    su += (uint64_t)std::max<int64_t>(1, (len + 31) / 32);
                    se += (uint64_t)len;
                }
            }
            h.plan_base[Pn] = (uint32_t)su;
            h.plan_base[2 * Pn + 1] = (uint32_t)se;
            if (su > 0xFFFFFFFFull || se > 0x7FFFFFFFull)
                throw ApiError{TF_EINVAL, "too many entries for the gather plan's 32-bit offsets"};
            h.plan_units = (int64_t)su;
        }
        return h;
    }

    // Device copies of a schedule, queued on st through page-locked staging.
    void plan_upload(int n, const PlanHost &h, PinnedStage &stage) {
        ModeLayout &L = mode[n];
        ++layout_gen;
        L.P = P;
        L.n_items = (int64_t)h.items.size();
        L.n_slots = h.n_slots;
        L.n_split = (int)h.split.size();
        L.n_single = (int)h.single.size();
        L.items.alloc(h.items.size(), st);
        L.bin_ptr.alloc(h.bin_ptr.size(), st);
        L.split.alloc(h.split.size(), st);
        L.single.alloc(h.single.size(), st);
        L.n_groups = (int)(h.groups.size() / 2);
        L.groups.alloc(std::max<size_t>(h.groups.size(), 2), st);
        L.plan_base.alloc(h.plan_base.size(), st);
        L.plan_units = h.plan_units;
        stage.copy(L.groups.p, h.groups.data(), h.groups.size() * sizeof(int32_t), st);
        stage.copy(L.single.p, h.single.data(), h.single.size() * sizeof(SplitRow), st);
        stage.copy(L.items.p, h.items.data(), h.items.size() * sizeof(tf_item), st);
        stage.copy(L.bin_ptr.p, h.bin_ptr.data(), h.bin_ptr.size() * sizeof(int64_t), st);
        stage.copy(L.split.p, h.split.data(), h.split.size() * sizeof(SplitRow), st);
        stage.copy(L.plan_base.p, h.plan_base.data(), h.plan_base.size() * sizeof(uint32_t), st);
    }

    // Schedules of every mode from their row offsets on the host: one thread per mode.
    std::vector<PlanHost> plan_all_host(const std::vector<std::vector<int64_t>> &offs) const {
        std::vector<PlanHost> hs((size_t)N);
        std::vector<std::exception_ptr> errs((size_t)N);
        std::vector<std::thread> th;
        for (int n = 0; n < N; ++n)
            th.emplace_back([&, n] {
                try {
                    hs[n] = plan_host(offs[n], dims[n]);
                } catch (...) {
                    errs[n] = std::current_exception();
                }
            });
        for (auto &t : th) t.join();
        for (auto &e : errs)
            if (e) std::rethrow_exception(e);
        return hs;
    }

    std::vector<std::vector<int64_t>> download_offsets() {
        std::vector<std::vector<int64_t>> offs((size_t)N);
        for (int n = 0; n < N; ++n) {
            offs[n].resize((size_t)mode[n].I + 1);
            TFS_CUDA(cudaMemcpyAsync(offs[n].data(), mode[n].off.p, offs[n].size() * sizeof(int64_t),
                                     cudaMemcpyDeviceToHost, st));
        }
        TFS_CUDA(cudaStreamSynchronize(st));
        return offs;
    }

    void plan_all() {
        const auto offs = download_offsets();
        const auto hs = plan_all_host(offs);
        PinnedStage stage;
        for (int n = 0; n < N; ++n) plan_upload(n, hs[n], stage);
        TFS_CUDA(cudaStreamSynchronize(st));
    }

    DeviceStatus read_status() {
        DeviceStatus s;
        TFS_CUDA(cudaMemcpyAsync(&s, stat.p, sizeof(s), cudaMemcpyDeviceToHost, st));
        TFS_CUDA(cudaStreamSynchronize(st));
        return s;
    }

    // ------------------------------------------------------------ residual copies
    void rebuild_residuals() {
        for (int n = 0; n < N; ++n) {
            InitArgs<T> a{};
            const ModeLayout &L = mode[n];
            a.items = L.items.p;
            a.bin_ptr = L.bin_ptr.p;
            a.P = L.P;
            a.N = N;
            a.n = n;
            a.K = K;
            a.model_zero = a0_zero ? 1 : 0;
            for (int t = 0; t < N - 1; ++t) {
                a.oidx[t] = L.oidx.p + (size_t)t * L.ostride;
                a.id_o[t] = mode[L.omode[t]].id_of.p;
                a.Ao[t] = A[L.omode[t]].p;
            }
            a.An = A[n].p;
            a.x = x.p;
            a.perm = L.perm.p;
            a.res = res[n].p;
            timed(TF_KIND_OTHER, [&] { launch_init_res<T>(a, st); });
        }
        Cq = 0;
        dirty = false;
    }

    template <class Args>
    void fill_other(Args &a, int n, const ModeLayout &L) {
        (void)n;
        for (int t = 0; t < N - 1; ++t) {
            a.oidx[t] = L.oidx.p + (size_t)t * L.ostride;
            a.Zo[t] = Z[L.omode[t]].p;
        }
    }

    // copies: R-hat of columns Q  ->  true residual (subtract Q's part)
    void flush_q() {
        if (Cq == 0) return;
        for (int n = 0; n < N; ++n) {
            ResArgs<T> a{};
            const ModeLayout &L = mode[n];
            a.items = L.items.p;
            a.bin_ptr = L.bin_ptr.p;
            a.P = L.P;
            a.N = N;
            a.n = n;
            a.Cq = Cq;
            a.what = 2;
            fill_other(a, n, L);
            a.Zn = Z[n].p;
            a.rank_n = L.rank_of.p;
            a.res = res[n].p;
            timed(TF_KIND_OTHER, [&] { launch_res<T>(a, CM_last, st); });
        }
        Cq = 0;
    }

    void launch_trace(int64_t cap, int64_t *n, int32_t *kinds, int32_t *modes, float *ms) {
        get_profile(nullptr, nullptr);
        *n = (int64_t)trace_ms.size();
        for (int64_t i = 0; i < std::min<int64_t>(cap, *n); ++i) {
            if (kinds) kinds[i] = trace_kind[i];
            if (modes) modes[i] = trace_mode[i];
            if (ms) ms[i] = trace_ms[i];
        }
    }

    // ------------------------------------------------------------ lean-pass gather plans
    // The plan of mode n's lean pass for cache rows (RR, RV) of its run / varying modes
    // and a pool of cap rows: built on the device in one pass (gather_plan.cu) the first
    // time a split needs it, then kept (one per mode) until the row schedule or the cache
    // sizes change.  The refreshing and the plain inner iterations share it: their cache
    // sizes are both planned for the refreshing pass's wider rows.
    // The plan of mode n for these cache sizes if one is kept (nothing is built).
    const GatherPlan *find_gather_plan(int n, int RR, int RV, int cap) const {
        for (auto &g : gplans)
            if (g->n == n && g->RR == RR && g->RV == RV && g->cap == cap && g->layout_gen == layout_gen)
                return g.get();
        return nullptr;
    }

    GatherPlanDev gather_plan(int n, int RR, int RV, int cap) {
        const int first = 1;
        const ModeLayout &L = mode[n];
        auto dev_of = [](const GatherPlan &g) {
            GatherPlanDev d;
            d.steps = g.steps.p;
            d.rank = reinterpret_cast<const int32_t *>(g.steps.p + (size_t)g.nsteps * sizeof(GStep));
            d.step_range = g.step_range.p;
            d.list = g.list.p;
            d.word = g.word.p;
            return d;
        };
        for (auto &g : gplans)
            if (g->n == n && g->RR == RR && g->RV == RV && g->cap == cap &&
                g->layout_gen == layout_gen) {
                g->used = ++gplan_clock;
                return dev_of(*g);
            }
        // drop plans of an old schedule and this mode's plan for other cache sizes; sweep
        // graphs captured with a dropped plan go too (they hold its addresses)
        const size_t before = gplans.size();
        gplans.erase(std::remove_if(gplans.begin(), gplans.end(),
                                    [&](const std::unique_ptr<GatherPlan> &g) {
                                        return g->layout_gen != layout_gen || g->n == n;
                                    }),
                     gplans.end());
        if (gplans.size() != before) drop_graphs();
        auto g = std::make_unique<GatherPlan>();
        g->n = n, g->RR = RR, g->RV = RV, g->cap = cap, g->first = first;
        g->layout_gen = layout_gen;
        const int Pn = L.P;
        const int run = lean_run_mode(n), var = 1 - run;
        const int32_t *ixR = L.oidx.p + (size_t)run * L.ostride, *ixV = L.oidx.p + (size_t)var * L.ostride;
        // regions from the schedule: plan_records_per_step(cap) records per step unit, two
        // list entries per entry
        const int64_t cap_steps = (int64_t)plan_records_per_step(cap) * L.plan_units;
        if (cap_steps > INT32_MAX)
            throw ApiError{TF_EINVAL, "gather plan: too many records for this pool size"};
        g->nsteps = std::max<int64_t>(cap_steps, 1);
        g->steps.alloc((size_t)g->nsteps * gather_plan_step_bytes(), st);
        g->step_range.alloc((size_t)2 * std::max(Pn, 1), st);
        g->list.alloc((size_t)std::max<int64_t>(2 * nnz, 1), st);
        g->word.alloc((size_t)std::max<int64_t>(nnz, 1), st);
        GatherPlanDev d = dev_of(*g);
        launch_gather_plan(L.items.p, L.bin_ptr.p, Pn, ixR, ixV, L.rank_of.p, RR, RV, cap, first,
                           L.plan_base.p, g->step_range.p, g->steps.p,
                           const_cast<int32_t *>(d.rank), g->list.p, g->word.p, stat.p, st);
        g->used = ++gplan_clock;
        gplans.push_back(std::move(g));
        return d;
    }

    // ------------------------------------------------------------ the sweep
    void sweep(int C, double lambda, int T_in, const int32_t *order, uint32_t flags) {
        if (C < 1 || C > K) throw ApiError{TF_EINVAL, "C must be in 1..K"};
        if (T_in < 1) throw ApiError{TF_EINVAL, "T_in must be >= 1"};
        if (!(lambda >= 0.0) || !isfinite(lambda)) throw ApiError{TF_EINVAL, "lambda must be >= 0"};
        const int CM = pick_cm(C);
        if (CM == 0) throw ApiError{TF_EINVAL, "C >= 128 is not supported (the widest Gram tile is 128 columns)"};
        const bool wide = CM > 16;
        int64_t launches0 = launches;
        if (dirty) {
            rebuild_residuals();
            launches += N;
        }
        if (Cq > CM) {
            flush_q();
            launches += N;
        }
        // column order -> device
        if (order_pending) {
            TFS_CUDA(cudaEventSynchronize(order_ev));
            order_pending = false;
        }
        if (order) {
            std::vector<char> seen(K, 0);
            for (int k = 0; k < K; ++k) {
                if (order[k] < 0 || order[k] >= K || seen[order[k]])
                    throw ApiError{TF_EINVAL, "col_order is not a permutation of 0..K-1"};
                seen[order[k]] = 1;
            }
            memcpy(h_order, order, sizeof(int32_t) * K);
        } else {
            default_order((int)sweeps, C, h_order);
        }
        TFS_CUDA(cudaMemcpyAsync(d_order.p, h_order, sizeof(int32_t) * K, cudaMemcpyHostToDevice,
                                 st));
        TFS_CUDA(cudaEventRecord(order_ev, st));
        order_pending = true;

        const int W = slice_stride_elems(CM, (int)sizeof(T));
        const int off_prev = CM, off_old = 2 * CM;
        int64_t max_slots = 0;
        for (int n = 0; n < N; ++n) {
            if (Z[n].n < (size_t)dims[n] * W) {
                Z[n].alloc((size_t)dims[n] * W, st);
                TFS_CUDA(cudaMemsetAsync(Z[n].p, 0, Z[n].n * sizeof(T), st));
            }
            max_slots = std::max(max_slots, mode[n].n_slots);
        }
        partials.ensure((size_t)std::max<int64_t>(max_slots, 1) * partial_stride(CM), st);

        bool use_tma = false;
        if constexpr (sizeof(T) == 4) {
            // the TMA pass only on request: the cp.async pass reads hot slice rows from
            // L1, which TMA loads bypass, and measures faster on skewed tensors
            if (path == 2 && tma_pass_supported(CM, N)) {
                bool ok = true;
                for (int l = 0; l < N; ++l) ok = ok && tmaps_for_Z[l] == (const void *)Z[l].p;
                use_tma = ok || build_tmaps(W);
            }
        }
        if (path == 2 && !use_tma && !(wide && sizeof(T) == 4))
            throw ApiError{TF_EINVAL, "TMA mode pass not available here"};
        // the lean float pass wherever it exists (three-way tensors, even widths <= 12)
        const bool use_lean = sizeof(T) == 4 && !wide && (path == 0 || path >= 3) &&
                              lean_pass_supported(CM, N);
        if (path >= 3 && !use_lean && !wide)
            throw ApiError{TF_EINVAL, "lean mode pass not available here"};
        // precision 2 / 3: the lean pass reads the varying mode's / both other modes' rows
        // from bfloat16 copies of the slices, refreshed after every pack and every solve
        const bool bf16_rows = use_lean && precision >= 2;
        const int Wb = slice_bf16_stride(CM);
        if (bf16_rows)
            for (int l = 0; l < N; ++l)
                if (Zb[l].n < (size_t)dims[l] * Wb) {
                    Zb[l].alloc((size_t)dims[l] * Wb, st);
                    TFS_CUDA(cudaMemsetAsync(Zb[l].p, 0, Zb[l].n * sizeof(uint16_t), st));
                }
        last_path = 0;
        const int nsplit = (K + C - 1) / C;
        // every launch of the splits (pack, mode passes, solves) and the copy of the last
        // split's columns into Q; returns |Q|
        auto run_splits = [&]() {
            int cq = Cq;
            const int32_t *Qp = d_Q.p;
            for (int s = 0; s < nsplit; ++s) {
                const int Cs = (s == nsplit - 1) ? K - s * C : C;
                const int32_t *Sp = d_order.p + (size_t)s * C;
                PackArgs<T> pk{};
                pk.N = N;
                pk.row_base[0] = 0;
                for (int l = 0; l < N; ++l) {
                    pk.Z[l] = Z[l].p;
                    pk.A[l] = A[l].p;
                    pk.id_of[l] = mode[l].id_of.p;
                    pk.row_base[l + 1] = pk.row_base[l] + dims[l];
                }
                pk.K = K;
                pk.W = W;
                pk.C = Cs;
                pk.Cq = cq;
                pk.off_old = off_old;
                pk.off_prev = off_prev;
                pk.S = Sp;
                pk.Q = Qp;
                timed(TF_KIND_PACK, [&] { launch_pack<T>(pk, st); });
                ++launches;
                if (bf16_rows) {
                    for (int l = 0; l < N; ++l)
                        timed(TF_KIND_PACK, [&] {
                            launch_slice_bf16((const float *)Z[l].p, Zb[l].p, dims[l], W, Wb, 0,
                                              3 * CM, st);
                        });
                    launches += N;
                }
                for (int t = 0; t < T_in; ++t) {
                    for (int n = 0; n < N; ++n) {
                        const ModeLayout &L = mode[n];
                        cur_mode = n;
                        PassArgs<T> a{};
                        a.items = L.items.p;
                        a.bin_ptr = L.bin_ptr.p;
                        a.P = L.P;
                        a.N = N;
                        a.n = n;
                        a.C = Cs;
                        a.Cq = cq;
                        a.first = (t == 0);
                        a.weighted = (flags & TF_WEIGHTED_LAMBDA) ? 1 : 0;
                        a.lambda = (T)lambda;
                        a.refine = solve_refine;
                        a.cond_limit = solve_cond;
                        for (int u = 0; u < N - 1; ++u) {
                            a.oidx[u] = L.oidx.p + (size_t)u * L.ostride;
                            a.Zo[u] = Z[L.omode[u]].p;
                            a.Zob[u] = Zb[L.omode[u]].p;
                        }
                        a.Wb = Wb;
                        a.Zn = Z[n].p;
                        a.rank_n = L.rank_of.p;
                        a.res = res[n].p;
                        a.A_n = A[n].p;
                        a.K = K;
                        a.S = Sp;
                        a.partials = partials.p;
                        a.stat = stat.p;
                        a.ticket = ticket.p;
                        a.ticket_base = ticket_base;
                        if (wide) {
                            // float: the Gram on the tensor cores for 64- and 128-wide tiles
                            // (C >= 32: faster than the SIMT Gram at 1e8 entries) or when
                            // requested (path 2, precision 1); SIMT for 32-wide tiles and
                            // on path 1
                            const bool tc = sizeof(T) == 4 && path != 1 &&
                                            (path == 2 || precision == 1 ||
                                             wide_split_width(Cs, CM) >= 64);
                            const int wgrid = pass_wide_grid<T>(pass_sms(), L.P, Cs, CM, tc, t == 0);
                            // every block takes one ticket past the last bin
                            ticket_base += (unsigned long long)L.P + (unsigned long long)wgrid;
                            timed(TF_KIND_MODE_PASS,
                                  [&] { launch_pass_wide<T>(a, CM, W, wgrid, tc, precision != 1, st); });
                            last_path |= tc ? 4 : 1;
                            ++launches;
                            if (L.n_single > 0) {
                                timed(TF_KIND_SOLVE, [&] {
                                    launch_solve_wide<T>(a, L.single.p, L.n_single, CM, W, st);
                                });
                                ++launches;
                            }
                            if (L.n_split > 0) {
                                if (L.n_groups > 0) {
                                    timed(TF_KIND_COMBINE, [&] {
                                        launch_sum_slot_groups<T>(partials.p,
                                                                  partial_stride(CM),
                                                                  L.groups.p, L.n_groups, st);
                                    });
                                    ++launches;
                                }
                                timed(TF_KIND_COMBINE, [&] {
                                    launch_solve_wide<T>(a, L.split.p, L.n_split, CM, W, st);
                                });
                                ++launches;
                            }
                            continue;
                        }
                        if constexpr (sizeof(T) == 4) {
                            // the lean pass where its shared-memory cache serves at
                            // least a quarter of the varying mode's gathers (measured
                            // slower than the cp.async pass on tensors without hot rows:
                            // a batch of 4,096 small tensors, uniform 1e5^3)
                            const std::vector<int64_t> *dc[2] = {&mode[L.omode[0]].deg_cum,
                                                                 &mode[L.omode[1]].deg_cum};
                            const int64_t dims_o[2] = {dims[L.omode[0]], dims[L.omode[1]]};
                            // Gram flavour: TF32 x 1 on the tensor cores for the
                            // reduced-precision form; FP32-level otherwise (packed FMAs,
                            // or three TF32 products on the tensor cores on path 4)
                            const int gk = bf16_rows ? 0 : precision == 1 ? 1 : (path == 4 ? 3 : 0);
                            LeanPlan plan{};
                            bool lean_here = use_lean;
                            if (lean_here) {
                                plan = lean_pass_plan(CM, t == 0, n, dims_o, dc, nnz, pass_sms(), L.P,
                                                      lean_cache_rows, lean_ring_cap, lean_warps, gk,
                                                      bf16_rows ? precision - 1 : 0);
                                lean_here = path != 0 || plan.coverage >= 0.25;
                            }
                            if (lean_here) {
                                const int run = lean_run_mode(n);
                                const GatherPlanDev gp =
                                    gather_plan(n, plan.p.R[run], plan.p.R[1 - run],
                                                plan.p.cap[0]);
                                ticket_base += (unsigned long long)L.P +
                                               (unsigned long long)plan.grid * plan.warps;
                                timed(TF_KIND_MODE_PASS, [&] {
                                    launch_lean_pass((const PassArgs<float> &)a, CM, plan, gp, st);
                                });
                                last_path |= 8;
                                ++launches;
                                goto solved;
                            }
                            if (use_tma) {
                                const bool before[2] = {L.omode[0] < n, L.omode[1] < n};
                                const int64_t dims_o[2] = {dims[L.omode[0]], dims[L.omode[1]]};
                                const TmaPlan plan =
                                    tma_pass_plan(CM, t == 0, before, dims_o, pass_sms(), L.P);

                                const int bidx[2] = {
                                    plan.box[0] == 8 ? 0 : (plan.box[0] == 24 ? 1 : 2),
                                    plan.box[1] == 8 ? 0 : (plan.box[1] == 24 ? 1 : 2)};
                                CUtensorMap tm2[2] = {tmaps[L.omode[0]][bidx[0]],
                                                      tmaps[L.omode[1]][bidx[1]]};
                                ticket_base += (unsigned long long)L.P +
                                               (unsigned long long)plan.grid * plan.warps;
                                timed(TF_KIND_MODE_PASS, [&] {
                                    launch_mode_pass_tma(a, tm2, plan, CM, t == 0, before, st);
                                });
                                last_path |= 2;
                                ++launches;
                                goto solved;
                            }
                        }
                    {
                        const PassPlan plan = mode_pass_plan<T>(CM, N, n, t == 0, pass_sms(), L.P);
                        // every launched warp takes one ticket past the last bin
                        ticket_base += (unsigned long long)L.P +
                                       (unsigned long long)plan.grid * plan.warps;
                        timed(TF_KIND_MODE_PASS, [&] { launch_mode_pass<T>(a, CM, plan, st); });
                        last_path |= 1;
                    }
                        ++launches;
                    solved:
                        if (L.n_single > 0) {
                            timed(TF_KIND_SOLVE,
                                  [&] { launch_solve_rows<T>(a, CM, L.single.p, L.n_single, st); });
                            ++launches;
                        }
                        if (L.n_split > 0) {
                            timed(TF_KIND_COMBINE,
                                  [&] { launch_combine<T>(a, CM, L.split.p, L.n_split, st); });
                            ++launches;
                        }
                        if (bf16_rows) {  // the rows just solved, into the bfloat16 copy
                            timed(TF_KIND_PACK, [&] {
                                launch_slice_bf16((const float *)Z[n].p, Zb[n].p, dims[n], W, Wb,
                                                  0, CM, st);
                            });
                            ++launches;
                        }
                    }
                }
                cq = Cs;
                Qp = Sp;
                cur_mode = -1;
            }
            // the copies now hold R-hat of the last split's columns
            TFS_CUDA(cudaMemcpyAsync(d_Q.p, Qp, sizeof(int32_t) * cq, cudaMemcpyDeviceToDevice,
                                     st));
            return cq;
        };
        int cq_end;
        if (!graphs_on || prof_on || st == nullptr) {
            cq_end = run_splits();
        } else {
            GraphKey gk{};
            gk.C = C, gk.T_in = T_in, gk.CM = CM, gk.Cq = Cq, gk.path = path;
            gk.precision = precision, gk.use_tma = use_tma, gk.flags = flags;
            gk.refine = solve_refine, gk.cond = solve_cond;
            gk.lambda = lambda, gk.layout_gen = layout_gen, gk.partials = partials.p;
            for (int l = 0; l < N; ++l) {
                gk.Z[l] = Z[l].p;
                gk.Zb[l] = Zb[l].p;
            }
            cq_end = run_splits_graph(gk, run_splits);
        }
        Cq = cq_end;
        CM_last = CM;
        ++sweeps;
        last_launches = launches - launches0;
    }

    // ------------------------------------------------------------ sweeps as CUDA graphs
    // The launches of a sweep depend only on the key below; the column order reaches the
    // kernels through d_order, copied before the graph runs.  A key's first sweep runs
    // eagerly (kernel attributes and plans settle), its second is captured into a graph
    // and launched, later ones replay the graph: one launch per sweep instead of one per
    // kernel.  The graph resets the bin counter itself (the mode passes' ticket bases
    // are baked in as seen from zero).
    struct GraphKey {
        int C, T_in, CM, Cq, path, precision, refine;
        float cond;
        bool use_tma;
        uint32_t flags;
        double lambda;
        int64_t layout_gen;
        const void *partials;
        const void *Z[kMaxModes];
        const void *Zb[kMaxModes];
        bool operator==(const GraphKey &o) const {
            if (C != o.C || T_in != o.T_in || CM != o.CM || Cq != o.Cq || path != o.path ||
                precision != o.precision || refine != o.refine || cond != o.cond ||
                use_tma != o.use_tma || flags != o.flags ||
                lambda != o.lambda || layout_gen != o.layout_gen || partials != o.partials)
                return false;
            for (int l = 0; l < kMaxModes; ++l)
                if (Z[l] != o.Z[l] || Zb[l] != o.Zb[l]) return false;
            return true;
        }
    };
    struct SweepGraph {
        GraphKey key;
        cudaGraphExec_t exec;
        int64_t launches;               // kernels in the graph
        unsigned long long ticket_end;  // bin counter after the graph
        int64_t path_bits;
        int cq_end;
    };
    static constexpr size_t kMaxGraphs = 8;
    bool graphs_on = false;
    std::vector<SweepGraph> graphs;  // least recently used first
    GraphKey last_eager{};
    bool have_last_eager = false;
    int64_t graph_replays = 0;

    template <class F>
    int run_splits_graph(const GraphKey &gk, F &run_splits) {
        for (size_t i = 0; i < graphs.size(); ++i) {
            if (!(graphs[i].key == gk)) continue;
            SweepGraph g = graphs[i];
            graphs.erase(graphs.begin() + (long)i);
            graphs.push_back(g);
            TFS_CUDA(cudaGraphLaunch(g.exec, st));
            launches += g.launches;
            ticket_base = g.ticket_end;
            last_path = g.path_bits;
            ++graph_replays;
            return g.cq_end;
        }
        if (!(have_last_eager && last_eager == gk)) {
            last_eager = gk;
            have_last_eager = true;
            return run_splits();
        }
        const int64_t l0 = launches;
        cudaGraph_t graph = nullptr;
        int cq_end = 0;
        TFS_CUDA(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
        try {
            TFS_CUDA(cudaMemsetAsync(ticket.p, 0, sizeof(unsigned long long), st));
            ticket_base = 0;
            cq_end = run_splits();
        } catch (...) {
            cudaStreamEndCapture(st, &graph);
            if (graph) cudaGraphDestroy(graph);
            cudaGetLastError();
            throw;
        }
        TFS_CUDA(cudaStreamEndCapture(st, &graph));
        cudaGraphExec_t exec = nullptr;
        const cudaError_t e = cudaGraphInstantiate(&exec, graph, 0);
        cudaGraphDestroy(graph);
        TFS_CUDA(e);
        if (graphs.size() >= kMaxGraphs) {
            TFS_CUDA(cudaStreamSynchronize(st));
            cudaGraphExecDestroy(graphs.front().exec);
            graphs.erase(graphs.begin());
        }
        graphs.push_back({gk, exec, launches - l0, ticket_base, last_path, cq_end});
        TFS_CUDA(cudaGraphLaunch(exec, st));
        ++graph_replays;
        return cq_end;
    }

    void drop_graphs() {
        if (!graphs.empty()) cudaStreamSynchronize(st);
        for (auto &g : graphs) cudaGraphExecDestroy(g.exec);
        graphs.clear();
        have_last_eager = false;
    }

    // Tensor maps of every mode's packed slice (float, W = 32): boxes of 8, 24, 40 floats,
    // one row high (tile::gather4 loads), no swizzle, zero fill beyond the row.
    bool build_tmaps(int W) {
        typedef CUresult (*EncodeTiled)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *,
                                        const cuuint64_t *, const cuuint64_t *, const cuuint32_t *,
                                        const cuuint32_t *, CUtensorMapInterleave,
                                        CUtensorMapSwizzle, CUtensorMapL2promotion,
                                        CUtensorMapFloatOOBfill);
        static EncodeTiled enc = nullptr;
        if (!enc) {
            void *fp = nullptr;
            cudaDriverEntryPointQueryResult q;
            if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fp, 12000,
                                                 cudaEnableDefault, &q) != cudaSuccess ||
                q != cudaDriverEntryPointSuccess || !fp) {
                cudaGetLastError();
                return false;
            }
            enc = (EncodeTiled)fp;
        }
        static const cuuint32_t boxes[3] = {8, 24, 40};
        for (int l = 0; l < N; ++l) {
            const cuuint64_t gdim[2] = {(cuuint64_t)W, (cuuint64_t)dims[l]};
            const cuuint64_t gstride[1] = {(cuuint64_t)W * sizeof(float)};
            const cuuint32_t es[2] = {1, 1};
            for (int b = 0; b < 3; ++b) {
                const cuuint32_t box[2] = {boxes[b], 1};
                if (enc(&tmaps[l][b], CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, (void *)Z[l].p, gdim,
                        gstride, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                        CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                        CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
                    return false;
            }
            tmaps_for_Z[l] = Z[l].p;
        }
        return true;
    }

    void default_order(int sweep_idx, int C, int32_t *out) const {
        for (int k = 0; k < K; ++k) out[k] = k;
        if (C == 1) return;  // CDTF keeps a fixed column order (Section 3.1)
        // Fisher-Yates driven by splitmix64 of (seed, sweep)
        uint64_t s = mix64_host(seed ^ mix64_host(0xC01D0000ull + (uint64_t)sweep_idx));
        for (int k = K - 1; k > 0; --k) {
            s = mix64_host(s);
            const int j = (int)(s % (uint64_t)(k + 1));
            std::swap(out[k], out[j]);
        }
    }

    // ------------------------------------------------------------ loss
    void loss(double lambda, uint32_t flags, double *loss_out, double *rmse_out) {
        red.ensure(loss_scratch_need(), st);
        loss_into(lambda, flags, loss_out, rmse_out, red.p, red.n);
    }

    // Doubles of reduction scratch the loss needs: two totals, one partial per block of
    // the residual kernel and 256 per mode of the regularisation sums.
    static constexpr int kRegBlocks = 256;
    size_t loss_scratch_need() const {
        return 2 + (size_t)res_grid<T>(CM_last, mode[0].P, N) + (size_t)N * kRegBlocks;
    }

    // The loss with its block partials and two sums in `scratch` (cap doubles of device
    // memory): tf_loss passes the context's reduction buffer, tf_loss_noalloc the
    // library's static array; the kernels and their order are the same, so the results
    // are bit-identical.
    void loss_into(double lambda, uint32_t flags, double *loss_out, double *rmse_out,
                   double *scratch, size_t cap) {
        const ModeLayout &L = mode[0];
        const int blocks = res_grid<T>(CM_last, L.P, N);
        const size_t need = loss_scratch_need();
        if (need > cap)
            throw ApiError{TF_EINVAL, "loss reduction needs " + std::to_string(need) +
                                          " scratch doubles; the static array holds " +
                                          std::to_string(cap) + " (lower P in tf_set_schedule)"};
        if (dirty) rebuild_residuals();
        ResArgs<T> a{};
        a.items = L.items.p;
        a.bin_ptr = L.bin_ptr.p;
        a.P = L.P;
        a.N = N;
        a.n = 0;
        a.Cq = Cq;
        a.what = 0;
        for (int t = 0; t < N - 1; ++t) {
            a.oidx[t] = L.oidx.p + (size_t)t * L.ostride;
            a.Zo[t] = Z[L.omode[t]].p;
        }
        a.Zn = Z[0].p;
        a.rank_n = L.rank_of.p;
        a.res = res[0].p;
        a.block_out = scratch + 2;
        double *regp = scratch + 2 + blocks;
        // float three-way contexts whose last sweep ran mode 0's lean pass in its default
        // form: the loss from that pass's plan and caches (the plain pass with the sums of
        // r^2 in place of the Gram); otherwise the pipelined residual kernel
        LeanPlan lplan{};
        GatherPlanDev lgp{};
        bool lean_loss = false;
        if constexpr (sizeof(T) == 4) {
            if (N == 3 && Cq > 0 && precision == 0 && (path == 0 || path == 3) &&
                lean_pass_supported(CM_last, N)) {
                const std::vector<int64_t> *dc[2] = {&mode[L.omode[0]].deg_cum,
                                                     &mode[L.omode[1]].deg_cum};
                const int64_t dims_o[2] = {dims[L.omode[0]], dims[L.omode[1]]};
                // the sweep's plan (packed Gram, same cache, pool and warps): the same gather plan
                lplan = lean_pass_plan(CM_last, false, 0, dims_o, dc, nnz, pass_sms(), L.P,
                                       lean_cache_rows, lean_ring_cap, lean_warps, 0, 0);
                // the per-item sums go to the partials buffer (a sweep has sized it for
                // every slot, at two floats or more per slot); the sweep's gather plan must
                // be kept (the loss builds and allocates nothing)
                const int run0 = lean_run_mode(0);
                lean_loss = (path != 0 || lplan.coverage >= 0.25) && partials.p != nullptr &&
                            partials.n >= (size_t)2 * (size_t)std::max<int64_t>(L.n_slots, 1) &&
                            find_gather_plan(0, lplan.p.R[run0], lplan.p.R[1 - run0],
                                             lplan.p.cap[0]) != nullptr;
                if (lean_loss) {
                    const int run = lean_run_mode(0);
                    lgp = gather_plan(0, lplan.p.R[run], lplan.p.R[1 - run], lplan.p.cap[0]);
                    lplan.gk = 2;
                }
            }
        }
        double *item_sums = lean_loss ? reinterpret_cast<double *>(partials.p) : nullptr;
        timed(TF_KIND_LOSS, [&] {
            if constexpr (sizeof(T) == 4) {
                if (lean_loss) {
                    PassArgs<float> pa{};
                    pa.items = L.items.p;
                    pa.bin_ptr = L.bin_ptr.p;
                    pa.P = L.P;
                    pa.N = N;
                    pa.n = 0;
                    pa.C = CM_last;
                    pa.Cq = Cq;
                    pa.first = 0;
                    for (int u = 0; u < N - 1; ++u) {
                        pa.oidx[u] = L.oidx.p + (size_t)u * L.ostride;
                        pa.Zo[u] = reinterpret_cast<const float *>(Z[L.omode[u]].p);
                        pa.Zob[u] = Zb[L.omode[u]].p;
                    }
                    pa.Zn = reinterpret_cast<float *>(Z[0].p);
                    pa.rank_n = L.rank_of.p;
                    pa.res = reinterpret_cast<float *>(res[0].p);
                    pa.K = K;
                    pa.stat = stat.p;
                    pa.ticket = ticket.p;
                    pa.ticket_base = ticket_base;
                    pa.loss_out = item_sums;
                    launch_lean_pass(pa, CM_last, lplan, lgp, st);
                    ticket_base += (unsigned long long)L.P +
                                   (unsigned long long)lplan.grid * lplan.warps;
                    // the items' sums in slot order
                    launch_sum_blocks(item_sums, (int)L.n_slots, scratch + 0, st);
                }
            }
            if (!lean_loss) {
                launch_res<T>(a, CM_last, st);
                launch_sum_blocks(scratch + 2, blocks, scratch + 0, st);
            }
            for (int n = 0; n < N; ++n)
                launch_reg<T>(A[n].p, dims[n], K,
                              (flags & TF_WEIGHTED_LAMBDA) ? mode[n].off.p : nullptr,
                              regp + (size_t)n * kRegBlocks, kRegBlocks, st);
            launch_sum_blocks(regp, N * kRegBlocks, scratch + 1, st);
        });
        loss_launches = 3 + N;
        double h[2];
        TFS_CUDA(cudaMemcpyAsync(h, scratch, 2 * sizeof(double), cudaMemcpyDeviceToHost, st));
        TFS_CUDA(cudaStreamSynchronize(st));
        check_errors();
        if (loss_out) *loss_out = h[0] + lambda * h[1];
        if (rmse_out) *rmse_out = nnz > 0 ? sqrt(h[0] / (double)nnz) : 0.0;
    }

    void get_residual(T *host_r) {
        if (dirty) rebuild_residuals();
        Buf<T> out;
        out.alloc(nnz, st);
        const ModeLayout &L = mode[0];
        ResArgs<T> a{};
        a.items = L.items.p;
        a.bin_ptr = L.bin_ptr.p;
        a.P = L.P;
        a.N = N;
        a.n = 0;
        a.Cq = Cq;
        a.what = 1;
        for (int t = 0; t < N - 1; ++t) {
            a.oidx[t] = L.oidx.p + (size_t)t * L.ostride;
            a.Zo[t] = Z[L.omode[t]].p;
        }
        a.Zn = Z[0].p;
        a.rank_n = L.rank_of.p;
        a.res = res[0].p;
        a.perm = L.perm.p;
        a.out = out.p;
        launch_res<T>(a, CM_last, st);
        if (nnz > 0)
            TFS_CUDA(cudaMemcpyAsync(host_r, out.p, nnz * sizeof(T), cudaMemcpyDeviceToHost, st));
        TFS_CUDA(cudaStreamSynchronize(st));
        check_errors();
    }

    void check_errors() {
        DeviceStatus s = read_status();
        if (s.bits & kStatTimeout) {
            TFS_CUDA(cudaMemsetAsync(&stat.p->bits, 0, sizeof(int), st));
            TFS_CUDA(cudaStreamSynchronize(st));
            throw ApiError{TF_ETIMEOUT, "a bounded wait in a kernel gave up; results are invalid"};
        }
        if (s.bits & kStatPlan) {
            TFS_CUDA(cudaMemsetAsync(&stat.p->bits, 0, sizeof(int), st));
            TFS_CUDA(cudaStreamSynchronize(st));
            throw ApiError{TF_ECUDA, "a gather plan outgrew its bound; results are invalid"};
        }
        if (s.bits & (kStatRange | kStatDup)) throw ApiError{TF_ECUDA, "device status corrupt"};
    }

    // ------------------------------------------------------------ factors
    void set_factors(int n, const T *host_A) {
        if (n < 0 || n >= N) throw ApiError{TF_EINVAL, "mode out of range"};
        const size_t cnt = (size_t)dims[n] * K;
        TFS_CUDA(cudaMemcpyAsync(A[n].p, host_A, cnt * sizeof(T), cudaMemcpyHostToDevice, st));
        if (n == 0) {
            bool zero = true;
            for (size_t i = 0; i < cnt && zero; ++i) zero = (host_A[i] == T(0));
            a0_zero = zero;
        }
        TFS_CUDA(cudaStreamSynchronize(st));
        dirty = true;
        Cq = 0;
    }

    void get_factors(int n, T *host_A) {
        if (n < 0 || n >= N) throw ApiError{TF_EINVAL, "mode out of range"};
        TFS_CUDA(cudaMemcpyAsync(host_A, A[n].p, (size_t)dims[n] * K * sizeof(T),
                                 cudaMemcpyDeviceToHost, st));
        TFS_CUDA(cudaStreamSynchronize(st));
        check_errors();
    }

    // ------------------------------------------------------------ prediction
    void predict(const int32_t *coords, int64_t m, T *out, uint32_t flags) {
        if (m < 0) throw ApiError{TF_EINVAL, "m must be >= 0"};
        if (m == 0) return;
        const bool dev = (flags & TF_INPUT_DEVICE) != 0;
        const int32_t *dc = coords;
        T *dout = out;
        if (!dev) {
            p_coords.ensure((size_t)m * N, st);
            p_out.ensure((size_t)m, st);
            TFS_CUDA(cudaMemcpyAsync(p_coords.p, coords, (size_t)m * N * sizeof(int32_t),
                                     cudaMemcpyHostToDevice, st));
            dc = p_coords.p;
            dout = p_out.p;
        }
        PredictArgs<T> a{};
        a.N = N;
        a.K = K;
        for (int l = 0; l < N; ++l) {
            a.A[l] = A[l].p;
            a.I[l] = dims[l];
        }
        a.m = m;
        a.coords = dc;
        a.out = dout;
        a.stat = stat.p;
        launch_predict<T>(a, st);
        DeviceStatus s = read_status();
        if (s.bits & kStatPredictRange) {
            TFS_CUDA(cudaMemsetAsync(&stat.p->bits, 0, sizeof(int), st));
            TFS_CUDA(cudaStreamSynchronize(st));
            throw ApiError{TF_ERANGE, "prediction coordinate out of range"};
        }
        if (!dev) {
            TFS_CUDA(cudaMemcpyAsync(out, dout, (size_t)m * sizeof(T), cudaMemcpyDeviceToHost, st));
            TFS_CUDA(cudaStreamSynchronize(st));
        }
    }

    // ------------------------------------------------------------ fold-in
    // Requests r = 0..n_req-1 with entries offsets[r] .. offsets[r + 1] of the
    // concatenated (other, vals); out [n_req][K]; status[r] = 0 ok, 1 index out of range,
    // 2 non-positive pivot (out row then untouched).
    void foldin_batch(int md, int n_req, const int64_t *offsets, const int32_t *other,
                      const T *vals, double lambda, T *out, int32_t *status) {
        if (md < 0 || md >= N) throw ApiError{TF_EINVAL, "mode out of range"};
        if (n_req < 0) throw ApiError{TF_EINVAL, "n_req must be >= 0"};
        if (!(lambda >= 0.0) || !isfinite(lambda)) throw ApiError{TF_EINVAL, "lambda must be >= 0"};
        if (n_req == 0) return;
        if (offsets[0] != 0) throw ApiError{TF_EINVAL, "offsets[0] must be 0"};
        for (int r = 0; r < n_req; ++r)
            if (offsets[r + 1] < offsets[r]) throw ApiError{TF_EINVAL, "offsets must not decrease"};
        const int64_t m = offsets[n_req];
        if (!foldin_tiled_ok(K)) {  // one block per request
            for (int r = 0; r < n_req; ++r) {
                status[r] = 0;
                try {
                    foldin_one(md, other + offsets[r] * (N - 1), vals + offsets[r],
                               offsets[r + 1] - offsets[r], lambda, out + (int64_t)r * K);
                } catch (const ApiError &e) {
                    if (e.status == TF_ERANGE || e.status == TF_EINVAL)
                        status[r] = e.status == TF_ERANGE ? 1 : 2;
                    else
                        throw;
                }
            }
            return;
        }
        std::vector<int64_t> blk_range;
        std::vector<int32_t> blk_req, req_blk;
        const int blocks = foldin_plan_blocks(offsets, n_req, blk_range, blk_req, req_blk);
        f_other.ensure((size_t)std::max<int64_t>(m, 1) * std::max(N - 1, 1), st);
        f_x.ensure((size_t)std::max<int64_t>(m, 1), st);
        f_out.ensure((size_t)n_req * K, st);
        f_part.ensure(foldin_part_elems(K, blocks), st);
        const bool refine = sizeof(T) == 4;
        if (refine) {
            size_t fac_elems = 0;
            f_rpart.ensure(foldin_refine_elems(K, blocks, n_req, &fac_elems), st);
            f_fac.ensure(fac_elems, st);
        }
        // one int64 staging buffer: block entry ranges [2B], then as int32 the blocks'
        // requests [B], the requests' first blocks [n_req + 1] and their status [n_req]
        const size_t B = (size_t)std::max(blocks, 1);
        const size_t n32 = B + 2 * (size_t)n_req + 1;
        const size_t n64 = 2 * B + (n32 + 1) / 2;
        f_meta.ensure(n64, st);
        std::vector<int64_t> meta(n64, 0);
        std::copy(blk_range.begin(), blk_range.end(), meta.begin());
        int32_t *m32 = reinterpret_cast<int32_t *>(meta.data() + 2 * B);
        std::copy(blk_req.begin(), blk_req.end(), m32);
        std::copy(req_blk.begin(), req_blk.end(), m32 + B);
        int32_t *st_host = m32 + B + n_req + 1;
        std::fill(st_host, st_host + n_req, 0);
        if (m > 0) {
            TFS_CUDA(cudaMemcpyAsync(f_other.p, other, (size_t)m * (N - 1) * sizeof(int32_t),
                                     cudaMemcpyHostToDevice, st));
            TFS_CUDA(cudaMemcpyAsync(f_x.p, vals, (size_t)m * sizeof(T), cudaMemcpyHostToDevice, st));
        }
        TFS_CUDA(cudaMemcpyAsync(f_meta.p, meta.data(), meta.size() * sizeof(int64_t),
                                 cudaMemcpyHostToDevice, st));
        const int32_t *d32 = reinterpret_cast<const int32_t *>(f_meta.p + 2 * B);
        FoldArgs<T> a{};
        a.N = N;
        a.K = K;
        a.mode = md;
        for (int l = 0; l < N; ++l) {
            a.A[l] = A[l].p;
            a.I[l] = dims[l];
        }
        a.m = m;
        a.other = f_other.p;
        a.x = f_x.p;
        a.lambda = (T)lambda;
        a.out = f_out.p;
        a.stat = stat.p;
        a.part = f_part.p;
        a.blk_range = f_meta.p;
        a.blk_req = d32;
        a.req_blk = d32 + B;
        a.req_status = const_cast<int32_t *>(d32 + B + n_req + 1);
        a.refine = refine ? 1 : 0;
        a.fac = refine ? f_fac.p : nullptr;
        a.rpart = refine ? f_rpart.p : nullptr;
        launch_foldin_tiled<T>(a, blocks, n_req, st);
        std::vector<T> rows((size_t)n_req * K);
        TFS_CUDA(cudaMemcpyAsync(status, a.req_status, (size_t)n_req * sizeof(int32_t),
                                 cudaMemcpyDeviceToHost, st));
        TFS_CUDA(cudaMemcpyAsync(rows.data(), f_out.p, rows.size() * sizeof(T),
                                 cudaMemcpyDeviceToHost, st));
        TFS_CUDA(cudaStreamSynchronize(st));
        check_errors();
        // rows of requests that failed stay untouched
        for (int r = 0; r < n_req; ++r)
            if (status[r] == 0) std::copy(rows.begin() + (size_t)r * K, rows.begin() + (size_t)(r + 1) * K,
                                          out + (size_t)r * K);
    }

    void foldin(int md, const int32_t *other, const T *vals, int64_t m, double lambda, T *out) {
        if (m < 0) throw ApiError{TF_EINVAL, "m must be >= 0"};
        if (!foldin_tiled_ok(K) || m == 0) {
            foldin_one(md, other, vals, m, lambda, out);
            return;
        }
        const int64_t offs[2] = {0, m};
        int32_t status = 0;
        foldin_batch(md, 1, offs, other, vals, lambda, out, &status);
        if (status & 1) throw ApiError{TF_ERANGE, "fold-in index out of range"};
        if (status & 2) throw ApiError{TF_EINVAL, "fold-in system is not positive definite"};
    }

    // one request, one block (any K that fits the block's shared memory)
    void foldin_one(int md, const int32_t *other, const T *vals, int64_t m, double lambda, T *out) {
        if (md < 0 || md >= N) throw ApiError{TF_EINVAL, "mode out of range"};
        if (m < 0) throw ApiError{TF_EINVAL, "m must be >= 0"};
        if (!(lambda >= 0.0) || !isfinite(lambda)) throw ApiError{TF_EINVAL, "lambda must be >= 0"};
        int dev = 0, maxsm = 0;
        TFS_CUDA(cudaGetDevice(&dev));
        TFS_CUDA(cudaDeviceGetAttribute(&maxsm, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
        if (foldin_smem_bytes<T>(K) + 1024 > (size_t)maxsm)
            throw ApiError{TF_EINVAL, "K too large for the fold-in kernel"};
        f_other.ensure((size_t)std::max<int64_t>(m, 1) * std::max(N - 1, 1), st);
        f_x.ensure((size_t)std::max<int64_t>(m, 1), st);
        f_out.ensure((size_t)K, st);
        if (m > 0) {
            TFS_CUDA(cudaMemcpyAsync(f_other.p, other, (size_t)m * (N - 1) * sizeof(int32_t),
                                     cudaMemcpyHostToDevice, st));
            TFS_CUDA(cudaMemcpyAsync(f_x.p, vals, (size_t)m * sizeof(T), cudaMemcpyHostToDevice, st));
        }
        FoldArgs<T> a{};
        a.N = N;
        a.K = K;
        a.mode = md;
        for (int l = 0; l < N; ++l) {
            a.A[l] = A[l].p;
            a.I[l] = dims[l];
        }
        a.m = m;
        a.other = f_other.p;
        a.x = f_x.p;
        a.lambda = (T)lambda;
        a.out = f_out.p;
        a.stat = stat.p;
        launch_foldin<T>(a, st);
        DeviceStatus s = read_status();
        const int fbits = s.bits & (kStatFoldRange | kStatFoldPivot);
        if (fbits) {
            TFS_CUDA(cudaMemsetAsync(&stat.p->bits, 0, sizeof(int), st));
            TFS_CUDA(cudaStreamSynchronize(st));
            if (fbits & kStatFoldRange) throw ApiError{TF_ERANGE, "fold-in index out of range"};
            throw ApiError{TF_EINVAL, "fold-in system is not positive definite"};
        }
        TFS_CUDA(cudaMemcpyAsync(out, f_out.p, K * sizeof(T), cudaMemcpyDeviceToHost, st));
        TFS_CUDA(cudaStreamSynchronize(st));
    }

    void grouping(int n, int64_t *off, int64_t *perm) {
        if (n < 0 || n >= N) throw ApiError{TF_EINVAL, "mode out of range"};
        const ModeLayout &L = mode[n];
        TFS_CUDA(cudaMemcpyAsync(off, L.off.p, (L.I + 1) * sizeof(int64_t), cudaMemcpyDeviceToHost,
                                 st));
        std::vector<int32_t> p32;
        if (perm && nnz > 0) {
            p32.resize(nnz);
            TFS_CUDA(cudaMemcpyAsync(p32.data(), L.perm.p, nnz * sizeof(int32_t),
                                     cudaMemcpyDeviceToHost, st));
        }
        TFS_CUDA(cudaStreamSynchronize(st));
        if (perm)
            for (int64_t j = 0; j < nnz; ++j) perm[j] = p32[j];
    }

    void counters(int64_t *c) {
        DeviceStatus s = read_status();
        c[0] = (int64_t)s.singular_rows;
        c[1] = sweeps;
        c[2] = last_launches;
        int64_t items = 0, split = 0;
        for (int n = 0; n < N; ++n) {
            items += mode[n].n_items;
            split += mode[n].n_split;
        }
        c[3] = items;
        c[4] = split;
        c[5] = P;
        c[6] = loss_launches;
        c[7] = last_path;
    }

    // ------------------------------------------------------------ autotuning
    // Times one sweep per (P, C) candidate pair from the current state and restores that
    // state bit for bit after each trial (factors, residual copies, the columns Q, the
    // sweep counter that seeds the default orders); leaves the fastest pair's schedule.
    // Each trial is preceded by an untimed sweep from the same state (first-launch costs).
    void autotune(const int *C_list, int n_C, const int *P_list, int n_P, double lambda,
                  int T_in, uint32_t flags, int *best_C, int *best_P, float *ms_out) {
        if (n_C < 1 || n_P < 1 || !C_list || !P_list || !best_C || !best_P)
            throw ApiError{TF_EINVAL, "empty candidate list"};
        for (int i = 0; i < n_C; ++i)
            if (C_list[i] < 1 || C_list[i] > K || pick_cm(C_list[i]) == 0)
                throw ApiError{TF_EINVAL, "C candidate out of range"};
        for (int i = 0; i < n_P; ++i)
            if (P_list[i] < 0) throw ApiError{TF_EINVAL, "P candidate must be >= 0"};
        if (prof_on) throw ApiError{TF_EBUSY, "autotuning while profiling"};
        TFS_CUDA(cudaStreamSynchronize(st));
        // saved state
        std::vector<std::unique_ptr<Buf<T>>> sA, sR;
        for (int n = 0; n < N; ++n) {
            sA.emplace_back(new Buf<T>());
            sR.emplace_back(new Buf<T>());
            sA[n]->alloc(A[n].n, st);
            sR[n]->alloc(res[n].n, st);
            TFS_CUDA(cudaMemcpyAsync(sA[n]->p, A[n].p, A[n].n * sizeof(T), cudaMemcpyDeviceToDevice, st));
            TFS_CUDA(cudaMemcpyAsync(sR[n]->p, res[n].p, res[n].n * sizeof(T), cudaMemcpyDeviceToDevice, st));
        }
        Buf<int32_t> sQ;
        sQ.alloc(K, st);
        TFS_CUDA(cudaMemcpyAsync(sQ.p, d_Q.p, K * sizeof(int32_t), cudaMemcpyDeviceToDevice, st));
        const int Cq0 = Cq, CMl0 = CM_last;
        const bool dirty0 = dirty, a00 = a0_zero;
        const int64_t sweeps0 = sweeps, launches0 = launches, last0 = last_launches;
        const int64_t path0 = last_path;
        const int P0 = P;
        auto restore = [&] {
            for (int n = 0; n < N; ++n) {
                TFS_CUDA(cudaMemcpyAsync(A[n].p, sA[n]->p, A[n].n * sizeof(T), cudaMemcpyDeviceToDevice, st));
                TFS_CUDA(cudaMemcpyAsync(res[n].p, sR[n]->p, res[n].n * sizeof(T), cudaMemcpyDeviceToDevice, st));
            }
            TFS_CUDA(cudaMemcpyAsync(d_Q.p, sQ.p, K * sizeof(int32_t), cudaMemcpyDeviceToDevice, st));
            Cq = Cq0, CM_last = CMl0, dirty = dirty0, a0_zero = a00, sweeps = sweeps0;
        };
        const bool graphs0 = graphs_on;
        graphs_on = false;  // a capture's host time would show up as device idle time
        cudaEvent_t e0 = nullptr, e1 = nullptr;
        TFS_CUDA(cudaEventCreate(&e0));
        TFS_CUDA(cudaEventCreate(&e1));
        float best = -1.f;
        try {
            for (int ip = 0; ip < n_P; ++ip) {
                set_schedule(policy, P_list[ip]);
                for (int ic = 0; ic < n_C; ++ic) {
                    restore();
                    sweep(C_list[ic], lambda, T_in, nullptr, flags);
                    restore();
                    TFS_CUDA(cudaEventRecord(e0, st));
                    sweep(C_list[ic], lambda, T_in, nullptr, flags);
                    TFS_CUDA(cudaEventRecord(e1, st));
                    TFS_CUDA(cudaEventSynchronize(e1));
                    float ms = 0.f;
                    TFS_CUDA(cudaEventElapsedTime(&ms, e0, e1));
                    if (ms_out) ms_out[(size_t)ip * n_C + ic] = ms;
                    if (best < 0.f || ms < best) {
                        best = ms;
                        *best_C = C_list[ic];
                        *best_P = P_list[ip];
                    }
                }
            }
        } catch (...) {
            cudaEventDestroy(e0);
            cudaEventDestroy(e1);
            restore();
            graphs_on = graphs0;
            set_schedule(policy, P0 == default_bins(num_sms, nnz) ? 0 : P0);
            throw;
        }
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        graphs_on = graphs0;
        restore();
        set_schedule(policy, *best_P);
        launches = launches0, last_launches = last0, last_path = path0;
        TFS_CUDA(cudaStreamSynchronize(st));
        check_errors();
    }

    void set_schedule(tf_sched_policy pol, int P_) {
        if (pol < TF_SCHED_LPT || pol > TF_SCHED_RAN) throw ApiError{TF_EINVAL, "bad policy"};
        if (P_ < 0) throw ApiError{TF_EINVAL, "P must be >= 0"};
        TFS_CUDA(cudaStreamSynchronize(st));
        policy = pol;
        P = P_ > 0 ? P_ : default_bins(num_sms, nnz);
        plan_all();
    }
};

}  // namespace tfs

struct tf_ctx {
    std::unique_ptr<tfs::CtxBase> impl;
    std::string err;
};

// ------------------------------------------------------------ loss without allocation
// Scratch of tf_loss_noalloc: the per-block partial sums of the loss reductions and the
// two totals, in a fixed device array instead of memory the context allocates.  One
// array per device, shared by every call on that device.  Sized for the default
// schedule of a 152-SM GPU in the worst case: 2 totals + 19,456 residual blocks (one
// warp per bin, 128 bins per SM, one warp per block when a warp's ring is large) +
// 256 regularisation blocks for each of up to 8 modes = 21,506 doubles.
static constexpr size_t kLossScratchDoubles = 24576;  // 192 KiB
static __device__ __align__(256) double g_loss_scratch[kLossScratchDoubles];

namespace {

// Device address of g_loss_scratch on `dev`, which must be the current device; looked
// up once per device (the first call on a device does the lookup, later calls reuse it).
double *loss_scratch_on(int dev) {
    int cur = 0;
    TFS_CUDA(cudaGetDevice(&cur));
    if (cur != dev)
        throw tfs::ApiError{TF_EINVAL, "tf_loss_noalloc: the current device (" +
                                           std::to_string(cur) +
                                           ") is not the context's device (" +
                                           std::to_string(dev) + ")"};
    static std::mutex mu;
    static std::vector<double *> addr;  // by device ordinal
    std::lock_guard<std::mutex> lock(mu);
    if ((size_t)dev >= addr.size()) addr.resize((size_t)dev + 1, nullptr);
    if (!addr[dev]) {
        void *p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_loss_scratch);
        if (e != cudaSuccess || !p) {
            cudaGetLastError();
            throw tfs::ApiError{TF_ECUDA, std::string("cudaGetSymbolAddress of the loss scratch "
                                                      "array failed: ") +
                                              cudaGetErrorString(e)};
        }
        addr[dev] = static_cast<double *>(p);
    }
    return addr[dev];
}

}  // namespace

namespace {

thread_local std::string g_create_err;

template <class F>
tf_status guarded(tf_ctx *ctx, F &&f) {
    try {
        f();
        return TF_OK;
    } catch (const tfs::ApiError &e) {
        if (ctx) ctx->err = e.msg;
        return e.status;
    } catch (const tfs::CudaError &e) {
        if (ctx) ctx->err = std::string(e.what) + ": " + cudaGetErrorString(e.err);
        cudaGetLastError();
        return e.err == cudaErrorMemoryAllocation ? TF_ENOMEM : TF_ECUDA;
    } catch (const std::bad_alloc &) {
        if (ctx) ctx->err = "host allocation failed";
        return TF_ENOMEM;
    } catch (...) {
        if (ctx) ctx->err = "unexpected error";
        return TF_ECUDA;
    }
}

template <class F>
tf_status dispatch(tf_ctx *ctx, F &&f) {
    if (!ctx || !ctx->impl) return TF_EINVAL;
    return guarded(ctx, [&] {
        if (ctx->impl->dtype == TF_F32)
            f(static_cast<tfs::Impl<float> &>(*ctx->impl));
        else
            f(static_cast<tfs::Impl<double> &>(*ctx->impl));
    });
}

}  // namespace

extern "C" {

tf_status tf_create(const int32_t *coords, const void *values, tf_dtype dtype, const int64_t *dims,
                    int N, int64_t nnz, int K, uint64_t seed, void *stream, uint32_t flags,
                    tf_ctx **out) {
    if (!out) return TF_EINVAL;
    *out = nullptr;
    g_create_err.clear();
    if (N < 1 || N > tfs::kMaxModes || nnz < 0 || nnz > INT32_MAX || K < 1 || !dims ||
        (nnz > 0 && (!coords || !values)) || (dtype != TF_F32 && dtype != TF_F64) ||
        (flags & ~(TF_INPUT_DEVICE | TF_LAYOUT_FIELD_SORTS))) {
        g_create_err = "invalid argument (N in 1..8, 0 <= nnz < 2^31, K >= 1, buffers non-NULL, "
                       "known flags)";
        return TF_EINVAL;
    }
    for (int n = 0; n < N; ++n)
        if (dims[n] < 1 || dims[n] > INT32_MAX) {
            g_create_err = "mode lengths must be in 1..2^31-1";
            return TF_EINVAL;
        }
    tf_ctx *ctx = new (std::nothrow) tf_ctx;
    if (!ctx) return TF_ENOMEM;
    tf_status s = guarded(ctx, [&] {
        if (dtype == TF_F32) {
            auto *p = new tfs::Impl<float>();
            p->dtype = dtype;
            ctx->impl.reset(p);
            p->create(coords, values, dims, N, nnz, K, seed, (cudaStream_t)stream, flags);
        } else {
            auto *p = new tfs::Impl<double>();
            p->dtype = dtype;
            ctx->impl.reset(p);
            p->create(coords, values, dims, N, nnz, K, seed, (cudaStream_t)stream, flags);
        }
    });
    if (s != TF_OK) {
        g_create_err = ctx->err;
        delete ctx;
        return s;
    }
    *out = ctx;
    return TF_OK;
}

void tf_destroy(tf_ctx *ctx) {
    if (!ctx) return;
    if (ctx->impl) {
        cudaStream_t st = ctx->impl->dtype == TF_F32
                              ? static_cast<tfs::Impl<float> &>(*ctx->impl).st
                              : static_cast<tfs::Impl<double> &>(*ctx->impl).st;
        cudaStreamSynchronize(st);
    }
    delete ctx;
}

const char *tf_last_error(const tf_ctx *ctx) {
    return ctx ? ctx->err.c_str() : g_create_err.c_str();
}

tf_status tf_sync(tf_ctx *ctx) {
    return dispatch(ctx, [&](auto &c) {
        TFS_CUDA(cudaStreamSynchronize(c.st));
        c.check_errors();
    });
}

tf_status tf_set_factors(tf_ctx *ctx, int n, const void *host_A) {
    if (!host_A) return TF_EINVAL;
    return dispatch(ctx, [&](auto &c) {
        using T = typename std::remove_reference<decltype(*c.x.p)>::type;
        c.set_factors(n, static_cast<const T *>(host_A));
    });
}

tf_status tf_get_factors(tf_ctx *ctx, int n, void *host_A) {
    if (!host_A) return TF_EINVAL;
    return dispatch(ctx, [&](auto &c) {
        using T = typename std::remove_reference<decltype(*c.x.p)>::type;
        c.get_factors(n, static_cast<T *>(host_A));
    });
}

tf_status tf_sals_sweep_ex(tf_ctx *ctx, int C, double lambda, int T_in, const int32_t *col_order,
                           uint32_t flags) {
    return dispatch(ctx, [&](auto &c) { c.sweep(C, lambda, T_in, col_order, flags); });
}

tf_status tf_sals_sweep_order(tf_ctx *ctx, int C, double lambda, int T_in,
                              const int32_t *col_order) {
    return tf_sals_sweep_ex(ctx, C, lambda, T_in, col_order, 0u);
}

tf_status tf_sals_sweep(tf_ctx *ctx, int C, double lambda, int T_in) {
    return tf_sals_sweep_ex(ctx, C, lambda, T_in, nullptr, 0u);
}

tf_status tf_default_order(const tf_ctx *ctx, int sweep, int C, int32_t *col_order) {
    if (!ctx || !ctx->impl || !col_order || sweep < 0 || C < 1) return TF_EINVAL;
    if (ctx->impl->dtype == TF_F32)
        static_cast<const tfs::Impl<float> &>(*ctx->impl).default_order(sweep, C, col_order);
    else
        static_cast<const tfs::Impl<double> &>(*ctx->impl).default_order(sweep, C, col_order);
    return TF_OK;
}

tf_status tf_loss(tf_ctx *ctx, double lambda, uint32_t flags, double *loss, double *train_rmse) {
    return dispatch(ctx, [&](auto &c) { c.loss(lambda, flags, loss, train_rmse); });
}

tf_status tf_loss_noalloc(tf_ctx *ctx, double lambda, uint32_t flags, double *loss,
                          double *train_rmse) {
    return dispatch(ctx, [&](auto &c) {
        c.loss_into(lambda, flags, loss, train_rmse, loss_scratch_on(c.device),
                    kLossScratchDoubles);
    });
}

tf_status tf_foldin(tf_ctx *ctx, int mode, const int32_t *other, const void *values, int64_t m,
                    double lambda, void *out_row) {
    if (!out_row || (m > 0 && (!other || !values))) return TF_EINVAL;
    return dispatch(ctx, [&](auto &c) {
        using T = typename std::remove_reference<decltype(*c.x.p)>::type;
        c.foldin(mode, other, static_cast<const T *>(values), m, lambda, static_cast<T *>(out_row));
    });
}

tf_status tf_foldin_batch(tf_ctx *ctx, int mode, int n_req, const int64_t *offsets,
                          const int32_t *other, const void *values, double lambda, void *out_rows,
                          int32_t *status) {
    if (n_req < 0 || (n_req > 0 && (!offsets || !out_rows || !status))) return TF_EINVAL;
    if (n_req > 0 && offsets[n_req] > 0 && (!other || !values)) return TF_EINVAL;
    return dispatch(ctx, [&](auto &c) {
        using T = typename std::remove_reference<decltype(*c.x.p)>::type;
        c.foldin_batch(mode, n_req, offsets, other, static_cast<const T *>(values), lambda,
                       static_cast<T *>(out_rows), status);
    });
}

tf_status tf_predict(tf_ctx *ctx, const int32_t *coords, int64_t m, void *out, uint32_t flags) {
    if (m > 0 && (!coords || !out)) return TF_EINVAL;
    return dispatch(ctx, [&](auto &c) {
        using T = typename std::remove_reference<decltype(*c.x.p)>::type;
        c.predict(coords, m, static_cast<T *>(out), flags);
    });
}

tf_status tf_get_grouping(tf_ctx *ctx, int n, int64_t *off, int64_t *perm) {
    if (!off) return TF_EINVAL;
    return dispatch(ctx, [&](auto &c) { c.grouping(n, off, perm); });
}

tf_status tf_get_residual(tf_ctx *ctx, void *host_r) {
    if (!host_r) return TF_EINVAL;
    return dispatch(ctx, [&](auto &c) {
        using T = typename std::remove_reference<decltype(*c.x.p)>::type;
        c.get_residual(static_cast<T *>(host_r));
    });
}

tf_status tf_get_counters(tf_ctx *ctx, int64_t counters[8]) {
    if (!counters) return TF_EINVAL;
    return dispatch(ctx, [&](auto &c) { c.counters(counters); });
}

tf_status tf_profile(tf_ctx *ctx, int enable) {
    return dispatch(ctx, [&](auto &c) { c.profile(enable); });
}

tf_status tf_get_profile(tf_ctx *ctx, int64_t *launches, double *ms) {
    return dispatch(ctx, [&](auto &c) { c.get_profile(launches, ms); });
}

tf_status tf_get_launch_trace(tf_ctx *ctx, int64_t cap, int64_t *n, int32_t *kinds,
                              int32_t *modes, float *ms) {
    if (!n || cap < 0) return TF_EINVAL;
    return dispatch(ctx, [&](auto &c) { c.launch_trace(cap, n, kinds, modes, ms); });
}

tf_status tf_estimate_bytes(const int64_t *dims, int N, int64_t nnz, int K, int C_max,
                            tf_dtype dtype, uint32_t flags, int num_sms, int64_t *bytes) {
    if (!dims || !bytes || N < 1 || N > tfs::kMaxModes || nnz < 0 || K < 1 || C_max < 1 ||
        C_max > K || (dtype != TF_F32 && dtype != TF_F64))
        return TF_EINVAL;
    for (int n = 0; n < N; ++n)
        if (dims[n] < 1) return TF_EINVAL;
    const int CM = tfs::pick_cm(C_max);
    if (CM == 0) return TF_EINVAL;
    if (num_sms <= 0) {
        int dev = 0;
        if (cudaGetDevice(&dev) != cudaSuccess ||
            cudaDeviceGetAttribute(&num_sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
            cudaGetLastError();
            return TF_ECUDA;
        }
    }
    // the same sizes tf_create and the sweeps allocate (see Impl::create / Impl::sweep)
    const double T = dtype == TF_F32 ? 4.0 : 8.0;
    const double P = (double)tfs::default_bins(num_sms, nnz);
    const double e = (double)nnz, ostride = (double)((nnz + 64 + 63) / 64 * 64);
    const int W = tfs::slice_stride_elems(CM, (int)T);
    double layout = 0, plan = 0, factors = 0, maxI = 0;
    for (int n = 0; n < N; ++n) {
        const double I = (double)dims[n];
        layout += e * 4 + (I + 1) * 8 + I * 8 + std::max(N - 1, 1) * ostride * 4;
        plan += (I + P) * sizeof(tf_item) + (P + 1) * 8 + I * sizeof(tfs::SplitRow);
        factors += I * K * T + (e + 64) * T + I * W * T;
        maxI = std::max(maxI, I);
    }
    const double base = 4096.0 * 8 + 2.0 * K * 4 + N * 8 + 1024;
    const double x = e * T, soa = (double)N * e * 4;
    const double host_copy = (flags & TF_INPUT_DEVICE) ? 0.0 : (double)N * e * 4;
    double transpose, sorting;
    if (tfs::packed_layout_applies(dims, N, nnz, flags)) {
        // packing: the values, the row-major copy, the keys and the row counts; sorting
        // and extraction: three key buffers, the spare permutation and values, the sort
        // scratch, the layout and the residual copies
        double sum_I = 0, res = 0;
        for (int n = 0; n < N; ++n) {
            sum_I += (double)dims[n];
            res += (e + 64) * T;
        }
        transpose = x + host_copy + e * 8 + sum_I * 4;
        sorting = x + 3 * e * 8 + e * 4 + e * T + (double)tfs::key_sort_workspace_bytes(nnz) +
                  sum_I * 4 + layout + res;
    } else {
        transpose = x + soa + host_copy;
        sorting = x + soa + e * 4 + (double)tfs::sort_workspace_bytes(nnz) + layout;
    }
    const double partials = (maxI + P) * tfs::partial_stride(CM) * T;
    // gather plans of the lean float pass (three-way tensors), one per mode, in the regions
    // they are built into: a location word and two list entries per entry, and at the
    // default pool of 32 rows three records per step unit (max(1, ceil(len / 32)) of each
    // item, at most len / 32 + 1; items are at most the rows plus one chunk per bin)
    double gplans = 0;
    if (dtype == TF_F32 && N == 3)
        for (int n = 0; n < N; ++n)
            gplans += e * 4 + e * 8 +
                      tfs::plan_records_per_step(32) * (e / 32 + (double)dims[n] + P) *
                          tfs::gather_plan_step_bytes() +
                      (P + 1) * 4 * 4;
    const double steady = x + layout + plan + factors + partials + gplans;
    // stream-ordered pool rounding: large buffers round up to the pool's 2 MiB mapping
    // granularity (at most 2 MiB each), small ones share chunks
    const double raw = base + std::max(transpose, std::max(sorting, steady));
    const double mib2 = 2.0 * 1024 * 1024;
    const double rounding = std::min(0.05 * raw, (16.0 + 12.0 * N) * mib2) + mib2;
    *bytes = (int64_t)(raw + rounding);
    return TF_OK;
}

tf_status tf_pool_usage(int64_t *used, int64_t *used_high, int64_t *reserved, int reset_high) {
    cudaMemPool_t pool = tfs::library_pool();
    if (!pool) return TF_ECUDA;
    uint64_t a = 0, b = 0, c = 0;
    if (cudaMemPoolGetAttribute(pool, cudaMemPoolAttrUsedMemCurrent, &a) != cudaSuccess ||
        cudaMemPoolGetAttribute(pool, cudaMemPoolAttrUsedMemHigh, &b) != cudaSuccess ||
        cudaMemPoolGetAttribute(pool, cudaMemPoolAttrReservedMemCurrent, &c) != cudaSuccess) {
        cudaGetLastError();
        return TF_ECUDA;
    }
    if (used) *used = (int64_t)a;
    if (used_high) *used_high = (int64_t)b;
    if (reserved) *reserved = (int64_t)c;
    if (reset_high) {
        uint64_t zero = 0;
        if (cudaMemPoolSetAttribute(pool, cudaMemPoolAttrUsedMemHigh, &zero) != cudaSuccess) {
            cudaGetLastError();
            return TF_ECUDA;
        }
    }
    return TF_OK;
}

tf_status tf_pool_trim(int64_t keep_bytes) {
    if (keep_bytes < 0) return TF_EINVAL;
    cudaMemPool_t pool = tfs::library_pool();
    if (!pool) return TF_ECUDA;
    if (cudaDeviceSynchronize() != cudaSuccess || cudaMemPoolTrimTo(pool, (size_t)keep_bytes) != cudaSuccess) {
        cudaGetLastError();
        return TF_ECUDA;
    }
    return TF_OK;
}

tf_status tf_get_shape(tf_ctx *ctx, int *N, int *K, tf_dtype *dtype) {
    return dispatch(ctx, [&](auto &c) {
        if (N) *N = c.N;
        if (K) *K = c.K;
        if (dtype) *dtype = sizeof(*c.x.p) == 4 ? TF_F32 : TF_F64;
    });
}

tf_status tf_get_stream(tf_ctx *ctx, void **stream) {
    if (!stream) return TF_EINVAL;
    return dispatch(ctx, [&](auto &c) { *stream = (void *)c.st; });
}

tf_status tf_set_stream(tf_ctx *ctx, void *stream) {
    return dispatch(ctx, [&](auto &c) {
        TFS_CUDA(cudaStreamSynchronize(c.st));
        c.st = (cudaStream_t)stream;
        c.each_buf([&](auto &b) { b.s = c.st; });
    });
}

tf_status tf_set_precision(tf_ctx *ctx, int mode) {
    if (mode < 0 || mode > 3) return TF_EINVAL;
    return dispatch(ctx, [&](auto &c) {
        if (mode != 0 && sizeof(*c.x.p) != 4)
            throw tfs::ApiError{TF_EINVAL, "the reduced-precision forms need a float context"};
        c.precision = mode;
    });
}

tf_status tf_set_graphs(tf_ctx *ctx, int enable) {
    if (enable < 0 || enable > 1) return TF_EINVAL;
    return dispatch(ctx, [&](auto &c) {
        if (!enable) c.drop_graphs();
        c.graphs_on = enable != 0;
    });
}

tf_status tf_autotune(tf_ctx *ctx, const int32_t *C_list, int n_C, const int32_t *P_list,
                      int n_P, double lambda, int T_in, uint32_t flags, int32_t *best_C,
                      int32_t *best_P, float *ms) {
    if (!C_list || !P_list || !best_C || !best_P || n_C < 1 || n_P < 1) return TF_EINVAL;
    return dispatch(ctx, [&](auto &c) {
        int bc = 0, bp = 0;
        std::vector<int> cl(C_list, C_list + std::max(n_C, 0)), pl(P_list, P_list + std::max(n_P, 0));
        c.autotune(cl.data(), n_C, pl.data(), n_P, lambda, T_in, flags, &bc, &bp, ms);
        *best_C = bc;
        *best_P = bp;
    });
}

tf_status tf_graph_info(tf_ctx *ctx, int64_t *replays, int64_t *cached) {
    return dispatch(ctx, [&](auto &c) {
        if (replays) *replays = c.graph_replays;
        if (cached) *cached = (int64_t)c.graphs.size();
    });
}

tf_status tf_set_solve(tf_ctx *ctx, int refine, double cond_limit) {
    if (refine < 0 || refine > 1 || !(cond_limit >= 0.0) || !isfinite(cond_limit))
        return TF_EINVAL;
    return dispatch(ctx, [&](auto &c) {
        c.solve_refine = refine;
        c.solve_cond = (float)cond_limit;
    });
}

tf_status tf_solve_info(tf_ctx *ctx, int64_t *fp64_rows) {
    if (!fp64_rows) return TF_EINVAL;
    return dispatch(ctx, [&](auto &c) { *fp64_rows = (int64_t)c.read_status().fp64_rows; });
}

tf_status tf_set_kernel_path(tf_ctx *ctx, int path) {
    if (path < 0 || path > 4) return TF_EINVAL;
    return dispatch(ctx, [&](auto &c) {
        c.path = path;
        c.drop_graphs();
    });
}

tf_status tf_set_sm_limit(tf_ctx *ctx, int sms) {
    if (sms < 0) return TF_EINVAL;
    return dispatch(ctx, [&](auto &c) {
        c.sm_limit = sms;
        c.drop_graphs();
    });
}

tf_status tf_set_pass_cache(tf_ctx *ctx, int max_rows, int pool_rows, int warps) {
    if (pool_rows < 2 || pool_rows > 32 || warps < 0 || warps > 16) return TF_EINVAL;
    return dispatch(ctx, [&](auto &c) {
        c.lean_cache_rows = max_rows;
        c.lean_ring_cap = pool_rows;
        c.lean_warps = warps;
        c.drop_graphs();
    });
}

tf_status tf_set_schedule(tf_ctx *ctx, tf_sched_policy policy, int P) {
    return dispatch(ctx, [&](auto &c) { c.set_schedule(policy, P); });
}

}  // extern "C"
