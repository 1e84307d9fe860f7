// Gather plans of the lean float pass (the pass that walks them is lean_pass.cu).
//
// A plan cuts each item (a row or row chunk) of a bin into steps of up to 32 consecutive
// entries, splits a step into records where its distinct cold rows (rows outside the
// shared-memory caches; consecutive equal indices are one row) would overflow a warp's
// staging pool, lists those rows per record, and gives every entry one 32-bit location
// word.  It is built in one pass: a bin's records and lists go to regions whose sizes
// follow from the schedule alone (plan_records_per_step records per step of each item,
// two list entries per entry), so no counting pass, scan or host round trip comes first;
// each bin then records where its records end.
#include "gather_plan.cuh"
#include "sweep.cuh"

namespace tfs {
namespace {

struct GPlanArgs {
    const tf_item *items;
    const int64_t *bin_ptr;
    int P;
    const int32_t *ixR, *ixV;  // run / varying mode index streams (slice ranks)
    const int32_t *rank_n;     // own row -> slice rank
    int RR, RV, cap, first, rmax;
    const uint32_t *base;  // [P + 1] step units before bin b, then [P + 1] entries before it
    uint32_t *range;       // [2P]: bin b's records are range[2b] .. range[2b + 1] - 1
    GStep *steps;
    int32_t *rank;   // own slice rank per record (first records of items)
    int32_t *list;
    uint32_t *word;  // per entry: varying location | run location << 16
    DeviceStatus *stat;
};

// One warp per bin.  The bin's steps in order, the next step's index pair (and the next
// item's record and own rank) loaded before the current step is worked on, so a warp keeps
// two steps' loads in flight instead of waiting on each.
__global__ void __launch_bounds__(256) k_gather_plan(const GPlanArgs g) {
    const int lane = threadIdx.x & 31;
    const int b = (int)(((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5);
    if (b >= g.P) return;
    const uint32_t lt = (1u << lane) - 1u, le = lt | (1u << lane);
    const uint32_t s0 = (uint32_t)g.rmax * g.base[b];
    const uint32_t s_cap = (uint32_t)g.rmax * g.base[b + 1] - s0;
    const uint32_t l0 = 2u * g.base[g.P + 1 + b];
    const uint32_t l_cap = 2u * g.base[g.P + 2 + b] - l0;
    uint32_t ns = 0, nl = 0;
    bool over = false;  // the bounds above would be exceeded (cannot happen; checked anyway)
    const int64_t it0 = g.bin_ptr[b], it1 = g.bin_ptr[b + 1];
    if (it0 < it1) {
        int64_t it = it0;
        tf_item x = g.items[it];
        tf_item xn = it + 1 < it1 ? g.items[it + 1] : x;
        int own = g.first ? g.rank_n[x.row] : 0;
        int own_n = g.first && it + 1 < it1 ? g.rank_n[xn.row] : 0;
        int j = (int)x.begin, jend = (int)(x.begin + x.len);
        int prevR = -1;  // run index of this lane's previous entry in the item
        bool first = true;
        int cV, cR;  // the current step's indices (-1 past its end)
        {
            const bool v = lane < min(kWarp, jend - j);
            cV = v ? g.ixV[j + lane] : -1;
            cR = v ? g.ixR[j + lane] : -1;
        }
        for (;;) {
            const int cmax = min(kWarp, jend - j);
            const bool valid = lane < cmax;
            const bool more_in_item = j + cmax < jend;
            const bool more = more_in_item || it + 1 < it1;
            // the next step: this item's next 32 entries, or the next item's first
            int nV = -1, nR = -1;
            if (more) {
                const int jn = more_in_item ? j + cmax : (int)xn.begin;
                const int jnend = more_in_item ? jend : (int)(xn.begin + xn.len);
                if (lane < min(kWarp, jnend - jn)) {
                    nV = g.ixV[jn + lane];
                    nR = g.ixR[jn + lane];
                }
            }
            const int iV = cV, iR = cR;
            const int pV = __shfl_up_sync(0xFFFFFFFFu, iV, 1), pR = __shfl_up_sync(0xFFFFFFFFu, iR, 1);
            const bool coldV = valid && iV >= g.RV;
            const bool need = valid && (first || iR != prevR);
            const bool coldR = need && iR >= g.RR;
            const uint32_t mV = __ballot_sync(0xFFFFFFFFu, coldV);
            const uint32_t mR = __ballot_sync(0xFFFFFFFFu, coldR);
            // records of this step: lanes [lo, hi), the most whose distinct cold rows fit
            int lo = 0;
            do {
                // heads relative to the record's first lane
                const bool pcV = lane > lo && ((mV >> (lane - 1)) & 1u);
                const bool pcR = lane > lo && ((mR >> (lane - 1)) & 1u);
                const uint32_t from = lo >= 32 ? 0u : ~((1u << lo) - 1u);
                const uint32_t hV = __ballot_sync(0xFFFFFFFFu, coldV && (!pcV || pV != iV)) & from;
                const uint32_t hR = __ballot_sync(0xFFFFFFFFu, coldR && (!pcR || pR != iR)) & from;
                // usually every remaining cold row fits: one record to the step's end (the
                // same lanes the general count below would take)
                int hi = cmax;
                if (__popc(hV) + __popc(hR) > g.cap) {
                    const int upto = __popc(hV & le) + __popc(hR & le);
                    hi = lo + __popc(__ballot_sync(0xFFFFFFFFu, valid && lane >= lo && upto <= g.cap));
                }
                const uint32_t keep = (hi >= 32 ? 0xFFFFFFFFu : ((1u << hi) - 1u)) & from;
                const int nVr = __popc(hV & keep), nRr = __popc(hR & keep);
                over = over || ns >= s_cap || nl + (uint32_t)(nVr + nRr) > l_cap;
                if (lane >= lo && lane < hi) {
                    const uint32_t locV =
                        coldV ? (kPoolBit | (uint32_t)(__popc(hV & le) - 1)) : (uint32_t)iV;
                    const uint32_t locR = !need   ? kKeep
                                          : coldR ? (kPoolBit | (uint32_t)(nVr + __popc(hR & le) - 1))
                                                  : (uint32_t)iR;
                    g.word[j + lane] = locV | (locR << 16);
                    if (!over) {
                        if ((hV >> lane) & 1u) g.list[l0 + nl + __popc(hV & lt)] = iV;
                        if ((hR >> lane) & 1u) g.list[l0 + nl + nVr + __popc(hR & lt)] = iR;
                    }
                }
                if (lane == 0 && !over) {
                    GStep st;
                    st.j0 = j;
                    st.list_off = l0 + nl;
                    const bool last = hi >= cmax && !more_in_item;
                    st.info = (uint32_t)hi | (first && lo == 0 ? 64u : 0u) | (last ? 128u : 0u) |
                              ((uint32_t)((it - it0) & 3) << 8) | ((uint32_t)nVr << 10) |
                              ((uint32_t)nRr << 16) | ((uint32_t)lo << 22);
                    st.slot = x.slot;
                    g.steps[s0 + ns] = st;
                    g.rank[s0 + ns] = own;
                }
                if (!over) {
                    ++ns;
                    nl += (uint32_t)(nVr + nRr);
                }
                lo = hi;
            } while (lo < cmax);
            if (!more) break;
            cV = nV;
            cR = nR;
            if (more_in_item) {
                if (valid) prevR = iR;
                j += cmax;
                first = false;
            } else {
                ++it;
                x = xn;
                own = own_n;
                if (it + 1 < it1) {
                    xn = g.items[it + 1];
                    own_n = g.first ? g.rank_n[xn.row] : 0;
                }
                j = (int)x.begin;
                jend = (int)(x.begin + x.len);
                prevR = -1;
                first = true;
            }
        }
    }
    if (lane == 0) {
        g.range[2 * b] = s0;
        g.range[2 * b + 1] = s0 + ns;
        if (over) atomicOr(&g.stat->bits, kStatPlan);
    }
}

}  // namespace

size_t gather_plan_step_bytes() { return sizeof(GStep) + sizeof(int32_t); }

void launch_gather_plan(const tf_item *items, const int64_t *bin_ptr, int P, const int32_t *ixR,
                        const int32_t *ixV, const int32_t *rank_n, int RR, int RV, int cap,
                        int first, const uint32_t *base, uint32_t *range, void *steps,
                        int32_t *rank, int32_t *list, uint32_t *word, DeviceStatus *stat,
                        cudaStream_t st) {
    GPlanArgs g{};
    g.items = items;
    g.bin_ptr = bin_ptr;
    g.P = P;
    g.ixR = ixR;
    g.ixV = ixV;
    g.rank_n = rank_n;
    g.RR = RR;
    g.RV = RV;
    g.cap = cap;
    g.first = first;
    g.rmax = plan_records_per_step(cap);
    g.base = base;
    g.range = range;
    g.steps = static_cast<GStep *>(steps);
    g.rank = rank;
    g.list = list;
    g.word = word;
    g.stat = stat;
    const int threads = 256;
    const int blocks = (int)(((int64_t)P * 32 + threads - 1) / threads);
    k_gather_plan<<<blocks, threads, 0, st>>>(g);
    TFS_CUDA(cudaGetLastError());
}

}  // namespace tfs
