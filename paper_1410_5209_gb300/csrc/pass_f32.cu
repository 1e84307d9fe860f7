// Instantiation of the mode-pass and combine kernels for float (one translation unit
// per element type, so the two compile in parallel).
#include <string.h>

#include "tma_pass.cuh"

namespace tfs {

template <>
void launch_mode_pass<float>(const PassArgs<float> &a, int CM, const PassPlan &plan, cudaStream_t st) {
    launch_mode_pass_impl<float>(a, CM, plan, st);
}

template <>
PassPlan mode_pass_plan<float>(int CM, int N, int n, bool first, int num_sms, int P) {
    return mode_pass_plan_impl<float>(CM, N, n, first, num_sms, P);
}

template <>
int res_grid<float>(int CM, int P, int N) {
    return res_blocks_impl<float>(CM, P, N);
}

template <>
void launch_combine<float>(const PassArgs<float> &a, int CM, const SplitRow *rows, int n_rows,
                          cudaStream_t st) {
    launch_combine_impl<float>(a, CM, rows, n_rows, st);
}

template <>
void launch_res<float>(const ResArgs<float> &a, int CM, cudaStream_t st) {
    launch_res_impl<float>(a, CM, st);
}

template <>
void launch_solve_rows<float>(const PassArgs<float> &a, int CM, const SplitRow *rows, int n_rows,
                            cudaStream_t st) {
    launch_solve_rows_impl<float>(a, CM, rows, n_rows, st);
}

bool tma_pass_supported(int CM, int N) {
    return N == 3 && CM <= 10 && slice_stride_elems(CM, 4) == 32;
}

namespace {

template <int CM>
auto tma_kernel(bool first) {
    return first ? k_mode_pass_tma<CM, true> : k_mode_pass_tma<CM, false>;
}

size_t align128(size_t b) { return (b + 127) / 128 * 128; }

struct TmaGeom {
    int need[2], box[2], cv[2], cs[2];
};

TmaGeom tma_geom(int CM, bool first, const bool before_n[2]) {
    TmaGeom g;
    for (int t = 0; t < 2; ++t) {
        g.need[t] = !first ? CM : (before_n[t] ? 3 * CM : 2 * CM);
        g.box[t] = tma_box(g.need[t]);
        g.cv[t] = (g.need[t] + 3) / 4;
        g.cs[t] = (g.cv[t] | 1) * 4;
    }
    return g;
}

#define TFS_FOR_EACH_TMA_CM(X) X(1) X(2) X(4) X(6) X(8) X(10)

}  // namespace

// Warps and cache of one pass: a mode whose whole slice takes at most kWholeCache bytes
// is cached whole (its rows are never gathered) when that still leaves room for at
// least kMinWarps warps; then as many warps as fit (up to kTmaMaxWarps); what shared
// memory is left goes to the highest-ranked rows of the gathered modes.
TmaPlan tma_pass_plan(int CM, bool first, const bool before_n[2], const int64_t dims_o[2],
                      int num_sms, int P) {
    constexpr size_t kWholeCache = 112 * 1024;
    constexpr int kMinWarps = 8;
    int dev = 0, smem_blk = 0;
    TFS_CUDA(cudaGetDevice(&dev));
    TFS_CUDA(cudaDeviceGetAttribute(&smem_blk, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
    const size_t budget = (size_t)smem_blk - 128;  // alignment slack of the launch
    const TmaGeom g = tma_geom(CM, first, before_n);
    size_t row_b[2], whole[2];
    for (int t = 0; t < 2; ++t) {
        row_b[t] = (size_t)g.cs[t] * 4;
        whole[t] = align128((size_t)dims_o[t] * row_b[t]);
    }
    bool cached[2] = {false, false};
    size_t cache = 0;
    const int order[2] = {whole[0] <= whole[1] ? 0 : 1, whole[0] <= whole[1] ? 1 : 0};
    for (int k = 0; k < 2; ++k) {
        const int t = order[k];
        if (whole[t] > kWholeCache) continue;
        const bool st0 = !(cached[0] || t == 0), st1 = !(cached[1] || t == 1);
        const TmaWarpLayout L = tma_warp_layout(g.box[0], g.box[1], st0, st1);
        if (cache + whole[t] + (size_t)kMinWarps * L.bytes <= budget) {
            cached[t] = true;
            cache += whole[t];
        }
    }
    const TmaWarpLayout L = tma_warp_layout(g.box[0], g.box[1], !cached[0], !cached[1]);
    TmaPlan plan;
    plan.warps = (int)std::min<size_t>(kTmaMaxWarps, (budget - cache) / L.bytes);
    if (plan.warps < 1) throw ApiError{TF_EINVAL, "TMA mode pass does not fit in shared memory"};
    size_t left = budget - cache - (size_t)plan.warps * L.bytes;
    const int n_staged = (cached[0] ? 0 : 1) + (cached[1] ? 0 : 1);
    for (int t = 0; t < 2; ++t) {
        plan.box[t] = g.box[t];
        plan.whole[t] = cached[t];
        if (cached[t]) {
            plan.hot[t] = (int)dims_o[t];
        } else {
            const size_t share = left / (size_t)n_staged;
            const int64_t rows = (int64_t)((share >= 128 ? share - 128 : 0) / row_b[t]) & ~7ll;
            plan.hot[t] = (int)std::min<int64_t>(dims_o[t], rows);
        }
    }
    size_t used = 0;
    for (int t = 0; t < 2; ++t) used += align128((size_t)plan.hot[t] * row_b[t]);
    plan.smem = used + (size_t)plan.warps * L.bytes + 128;
    plan.grid = std::max(1, std::min(num_sms, (P + plan.warps - 1) / plan.warps));
    return plan;
}

namespace {

template <int CM>
void tma_launch_cm(const TmaPassArgs &ta, const TmaPlan &plan, bool first, cudaStream_t st) {
    auto kern = tma_kernel<CM>(first);
    TFS_CUDA(raise_smem_limit((const void *)kern, (int)plan.smem));
    kern<<<plan.grid, plan.warps * kWarp, plan.smem, st>>>(ta);
    TFS_CUDA(cudaGetLastError());
}

}  // namespace

void launch_mode_pass_tma(const PassArgs<float> &a, const void *tmaps, const TmaPlan &plan,
                          int CM, bool first, const bool before_n[2], cudaStream_t st) {
    const TmaGeom g = tma_geom(CM, first, before_n);
    TmaPassArgs ta;
    ta.p = a;
    memcpy(&ta.tm[0], tmaps, 2 * sizeof(CUtensorMap));
    size_t off = 0;
    for (int t = 0; t < 2; ++t) {
        if (plan.box[t] != g.box[t]) throw ApiError{TF_EINVAL, "TMA plan does not match the pass"};
        ta.box[t] = g.box[t];
        ta.hot[t] = plan.hot[t];
        ta.cs[t] = g.cs[t];
        ta.cv[t] = g.cv[t];
        if (t == 1) ta.cache_off1 = (unsigned)off;
        off += align128((size_t)plan.hot[t] * g.cs[t] * 4);
    }
    ta.cache_bytes = (unsigned)off;
    // a mode is left out of the row slots only when it is cached whole
    ta.L = tma_warp_layout(g.box[0], g.box[1], !plan.whole[0], !plan.whole[1]);
    switch (CM) {
#define TFS_CASE(cm)                               \
    case cm:                                       \
        tma_launch_cm<cm>(ta, plan, first, st);    \
        return;
        TFS_FOR_EACH_TMA_CM(TFS_CASE)
#undef TFS_CASE
        default:
            throw ApiError{TF_EINVAL, "no TMA mode-pass instance for this C"};
    }
}

}  // namespace tfs
