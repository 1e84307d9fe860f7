// Host-side row scheduling: the GPU counterpart of the paper's greedy row assignment
// (Algorithm 3, Section 3.3).  The paper balances |mOmega^(n)| (entries per machine)
// because the slowest machine sets each step's time; here the "machines" are bins of
// warps on the GPU.  The default policy is LPT without the paper's row cap (the cap
// only bounded the parameter broadcast of the MapReduce design) and with rows longer
// than a cap split into chunks whose partial Gram/rhs are summed before the solve.
// The paper's own policy (row cap and both tie-breaks) and its SEQ / RAN baselines
// (Section 5.5) are kept for comparison.
#include <stdint.h>

#include <algorithm>
#include <numeric>
#include <queue>
#include <tuple>
#include <vector>

#include "../../include/tf_sals.h"

namespace tfs {
namespace {

uint64_t splitmix(uint64_t z) {
    z += 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

// Bin key in the order the paper's Algorithm 3 prefers machines: fewest entries of
// this mode, then fewest rows of this mode, then fewest entries over all modes so far,
// then the lowest index.
struct BinKey {
    int64_t load, rows, total;
    int32_t bin;
    bool operator>(const BinKey &o) const {
        return std::tie(load, rows, total, bin) > std::tie(o.load, o.rows, o.total, o.bin);
    }
};
using MinHeap = std::priority_queue<BinKey, std::vector<BinKey>, std::greater<BinKey>>;

// Rows in decreasing length, equal lengths in increasing index.  Short lengths take one
// counting sort; otherwise a least-significant-digit radix sort of the complemented
// lengths (11-bit digits, stable, so equal lengths stay in index order), skipping digits
// that every key shares.  Lengths beyond 32 bits take a comparison sort.
std::vector<int64_t> rows_by_length(const int64_t *len, int64_t I) {
    std::vector<int64_t> order(I);
    int64_t max_len = 0;
    bool nonneg = true;
    for (int64_t i = 0; i < I; ++i) {
        max_len = std::max(max_len, len[i]);
        nonneg = nonneg && len[i] >= 0;
    }
    if (nonneg && max_len <= 4 * I + 1024) {
        std::vector<int64_t> start((size_t)max_len + 2, 0);
        for (int64_t i = 0; i < I; ++i) start[(size_t)(max_len - len[i]) + 1] += 1;
        for (int64_t v = 0; v <= max_len; ++v) start[v + 1] += start[v];
        for (int64_t i = 0; i < I; ++i) order[(size_t)start[(size_t)(max_len - len[i])]++] = i;
        return order;
    }
    if (!nonneg || max_len > (int64_t)UINT32_MAX || I > (int64_t)UINT32_MAX) {
        std::iota(order.begin(), order.end(), 0);
        std::stable_sort(order.begin(), order.end(),
                         [&](int64_t a, int64_t b) { return len[a] > len[b]; });
        return order;
    }
    constexpr int kBits = 11, kBuckets = 1 << kBits;
    std::vector<uint32_t> key((size_t)I), key2((size_t)I), idx((size_t)I), idx2((size_t)I);
    for (int64_t i = 0; i < I; ++i) {
        key[i] = (uint32_t)(UINT32_MAX - (uint64_t)len[i]);
        idx[i] = (uint32_t)i;
    }
    std::vector<int64_t> cnt(kBuckets + 1);
    for (int shift = 0; shift < 32; shift += kBits) {
        std::fill(cnt.begin(), cnt.end(), 0);
        for (int64_t i = 0; i < I; ++i) cnt[((key[i] >> shift) & (kBuckets - 1)) + 1] += 1;
        bool one_bucket = false;
        for (int d = 0; d < kBuckets; ++d) one_bucket = one_bucket || cnt[d + 1] == I;
        if (one_bucket) continue;
        for (int d = 0; d < kBuckets; ++d) cnt[d + 1] += cnt[d];
        for (int64_t i = 0; i < I; ++i) {
            const int64_t at = cnt[(key[i] >> shift) & (kBuckets - 1)]++;
            key2[(size_t)at] = key[i];
            idx2[(size_t)at] = idx[i];
        }
        key.swap(key2);
        idx.swap(idx2);
    }
    for (int64_t i = 0; i < I; ++i) order[i] = (int64_t)idx[i];
    return order;
}

// LPT: every job, longest first, to the bin with the least load (lowest index on ties).
// A job's load is its entries plus kItemCost: every item has a fixed cost in the mode
// pass (its first step, its partial write), so the many short or empty rows of a tensor
// spread over the bins instead of piling into whichever bin is least loaded last.  A
// min-heap of packed keys (load in the high bits, bin in the low 21 bits).
constexpr int64_t kItemCost = 32;
void lpt_bins(const std::vector<int64_t> &job_len, const std::vector<int64_t> &order, int M,
              std::vector<int32_t> &bin_of_job) {
    // a 4-ary heap: half the levels of a binary one, the four children in one cache line
    std::vector<uint64_t> heap((size_t)M);
    for (int m = 0; m < M; ++m) heap[m] = (uint64_t)m;  // already a min-heap
    bin_of_job.assign(job_len.size(), -1);
    auto sift_down = [&](size_t i) {
        const size_t n = heap.size();
        const uint64_t v = heap[i];
        for (;;) {
            const size_t c0 = 4 * i + 1;
            if (c0 >= n) break;
            size_t c = c0;
            const size_t cend = std::min(c0 + 4, n);
            for (size_t k = c0 + 1; k < cend; ++k)
                if (heap[k] < heap[c]) c = k;
            if (heap[c] >= v) break;
            heap[i] = heap[c];
            i = c;
        }
        heap[i] = v;
    };
    for (int64_t j : order) {
        const uint64_t top = heap[0];
        const int32_t m = (int32_t)(top & ((1u << 21) - 1));
        bin_of_job[j] = m;
        heap[0] = top + ((uint64_t)(job_len[j] + kItemCost) << 21);  // load grows, bin stays
        sift_down(0);
    }
}

// Greedy assignment of one mode's jobs to M bins.  cap_rows < 0 means no row cap.
// totals (size M) carries |mOmega| across modes and is updated.
void greedy_bins(const std::vector<int64_t> &job_len, const std::vector<int64_t> &order, int M,
                 int64_t cap_rows, std::vector<int64_t> &totals, std::vector<int32_t> &bin_of_job) {
    std::vector<int64_t> load(M, 0), rows(M, 0);
    MinHeap heap;
    for (int m = 0; m < M; ++m) heap.push({0, 0, totals[m], m});
    bin_of_job.assign(job_len.size(), -1);
    for (int64_t j : order) {
        BinKey k = heap.top();
        heap.pop();
        const int m = k.bin;
        bin_of_job[j] = m;
        load[m] += job_len[j];
        rows[m] += 1;
        totals[m] += job_len[j];
        if (cap_rows < 0 || rows[m] < cap_rows) heap.push({load[m], rows[m], totals[m], m});
    }
}

}  // namespace

tf_status assign_rows_impl(tf_sched_policy policy, int N, const int64_t *dims,
                           const int64_t *const *row_nnz, int M, uint64_t seed,
                           int32_t *const *assign) {
    if (N < 1 || M < 1 || !dims || !row_nnz || !assign) return TF_EINVAL;
    std::vector<int64_t> totals(M, 0);
    for (int n = 0; n < N; ++n) {
        const int64_t I = dims[n];
        if (I < 0) return TF_EINVAL;
        switch (policy) {
            case TF_SCHED_GREEDY:
            case TF_SCHED_LPT: {
                std::vector<int64_t> len(row_nnz[n], row_nnz[n] + I);
                std::vector<int64_t> order = rows_by_length(len.data(), I);
                std::vector<int32_t> bin;
                const int64_t cap = policy == TF_SCHED_GREEDY ? (I + M - 1) / M : -1;
                greedy_bins(len, order, M, cap, totals, bin);
                for (int64_t i = 0; i < I; ++i) assign[n][i] = bin[i];
                break;
            }
            case TF_SCHED_SEQ:
                // m-th range: I*m/M <= i < I*(m+1)/M (0-based form of the paper's SEQ)
                for (int m = 0; m < M; ++m)
                    for (int64_t i = I * m / M; i < I * (m + 1) / M; ++i) assign[n][i] = m;
                break;
            case TF_SCHED_RAN:
                for (int64_t i = 0; i < I; ++i)
                    assign[n][i] = (int32_t)(splitmix(seed ^ splitmix((uint64_t)n << 40 ^ i)) % M);
                break;
            default:
                return TF_EINVAL;
        }
    }
    return TF_OK;
}

std::vector<int64_t> rows_by_degree(const std::vector<int64_t> &count) {
    return rows_by_length(count.data(), (int64_t)count.size());
}

tf_status plan_mode(const int64_t *off, int64_t I, int P, int64_t cap, tf_sched_policy policy,
                    uint64_t seed, std::vector<tf_item> &items, int64_t &n_slots,
                    std::vector<int64_t> &bin_ptr) {
    if (I < 0 || P < 1 || cap < 0) return TF_EINVAL;
    const int64_t nnz = I > 0 ? off[I] : 0;
    if (cap == 0) cap = std::max<int64_t>(1, (nnz + P - 1) / P);

    // jobs: whole rows, or chunks of rows longer than cap (LPT only)
    std::vector<tf_item> jobs;
    jobs.reserve((size_t)I + (size_t)P + 16);
    n_slots = 0;
    for (int64_t i = 0; i < I; ++i) {
        const int64_t len = off[i + 1] - off[i];
        if (policy != TF_SCHED_LPT || len <= cap) {
            if (len > INT32_MAX) return TF_EINVAL;
            jobs.push_back({off[i], (int32_t)len, (int32_t)i, (int32_t)n_slots++, -1});
            continue;
        }
        const int64_t k = (len + cap - 1) / cap;
        const int64_t base = len / k, rem = len % k;
        int64_t b = off[i];
        for (int64_t c = 0; c < k; ++c) {
            const int64_t l = base + (c < rem ? 1 : 0);
            jobs.push_back({b, (int32_t)l, (int32_t)i, (int32_t)n_slots++, -1});
            b += l;
        }
    }

    std::vector<int32_t> bin(jobs.size(), 0);
    switch (policy) {
        case TF_SCHED_LPT:
        case TF_SCHED_GREEDY: {
            std::vector<int64_t> len(jobs.size());
            for (size_t j = 0; j < jobs.size(); ++j) len[j] = jobs[j].len;
            std::vector<int64_t> order = rows_by_length(len.data(), (int64_t)len.size());
            if (policy == TF_SCHED_LPT && P < (1 << 21)) {
                lpt_bins(len, order, P, bin);
            } else {
                std::vector<int64_t> totals(P, 0);
                const int64_t cap_rows = policy == TF_SCHED_GREEDY ? (I + P - 1) / P : -1;
                greedy_bins(len, order, P, cap_rows, totals, bin);
            }
            // bins receive jobs longest first: keep that order inside each bin (grouped
            // by bin in the same pass)
            bin_ptr.assign((size_t)P + 1, 0);
            for (size_t j = 0; j < jobs.size(); ++j) bin_ptr[bin[j] + 1] += 1;
            for (int p = 0; p < P; ++p) bin_ptr[p + 1] += bin_ptr[p];
            std::vector<int64_t> fill(bin_ptr.begin(), bin_ptr.end() - 1);
            items.resize(jobs.size());
            for (int64_t j : order) {
                tf_item it = jobs[j];
                it.bin = bin[j];
                items[(size_t)fill[it.bin]++] = it;
            }
            return TF_OK;
        }
        case TF_SCHED_SEQ:
            for (auto &it : jobs) it.bin = (int32_t)(((int64_t)it.row * P) / std::max<int64_t>(I, 1));
            break;
        case TF_SCHED_RAN:
            for (auto &it : jobs) it.bin = (int32_t)(splitmix(seed ^ (uint64_t)it.row) % P);
            break;
        default:
            return TF_EINVAL;
    }
    // group by bin, keeping the assignment order within a bin (a counting sort)
    bin_ptr.assign((size_t)P + 1, 0);
    for (const auto &it : jobs) bin_ptr[it.bin + 1] += 1;
    for (int p = 0; p < P; ++p) bin_ptr[p + 1] += bin_ptr[p];
    std::vector<int64_t> fill(bin_ptr.begin(), bin_ptr.end() - 1);
    items.resize(jobs.size());
    for (const auto &it : jobs) items[(size_t)fill[it.bin]++] = it;
    return TF_OK;
}

}  // namespace tfs

extern "C" {

tf_status tf_assign_rows(tf_sched_policy policy, int N, const int64_t *dims,
                         const int64_t *const *row_nnz, int M, uint64_t seed,
                         int32_t *const *assign) {
    try {
        return tfs::assign_rows_impl(policy, N, dims, row_nnz, M, seed, assign);
    } catch (...) {
        return TF_ENOMEM;
    }
}

tf_status tf_plan_mode(const int64_t *off, int64_t I, int P, int64_t cap,
                       tf_sched_policy policy, uint64_t seed, tf_item *items,
                       int64_t max_items, int64_t *n_items, int64_t *n_slots,
                       int64_t *bin_ptr) {
    if (!off || !n_items || !n_slots) return TF_EINVAL;
    try {
        std::vector<tf_item> v;
        std::vector<int64_t> bp;
        int64_t slots = 0;
        tf_status st = tfs::plan_mode(off, I, P, cap, policy, seed, v, slots, bp);
        if (st != TF_OK) return st;
        *n_items = (int64_t)v.size();
        *n_slots = slots;
        if ((int64_t)v.size() > max_items || !items) return TF_ENOMEM;
        std::copy(v.begin(), v.end(), items);
        if (bin_ptr) std::copy(bp.begin(), bp.end(), bin_ptr);
        return TF_OK;
    } catch (...) {
        return TF_ENOMEM;
    }
}

const char *tf_version(void) { return "sals-gb300 0.1"; }

}  // extern "C"
