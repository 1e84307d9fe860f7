// Instantiation of the mode-pass and combine kernels for float (one translation unit
// per element type, so the two compile in parallel).
#include <string.h>

#include "tma_pass.cuh"

namespace tfs {

template <>
void launch_mode_pass<float>(const PassArgs<float> &a, int CM, int grid, cudaStream_t st) {
    launch_mode_pass_impl<float>(a, CM, grid, st);
}

template <>
int mode_pass_grid<float>(int CM, int P, int num_sms, int N) {
    return mode_pass_grid_impl<float>(CM, P, num_sms, N);
}

template <>
int mode_pass_warps<float>(int CM, int N) {
    return mode_pass_warps_impl<float>(CM, N);
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

int tma_box_for(int CM, bool first, bool before_n) {
    const int need = !first ? CM : (before_n ? 3 * CM : 2 * CM);
    return tma_box(need);
}

int tma_pass_warps() { return kTmaThreads / kWarp; }

namespace {

template <int CM>
auto tma_kernel(bool first) {
    return first ? k_mode_pass_tma<CM, true> : k_mode_pass_tma<CM, false>;
}

size_t tma_smem(const int box[2]) {
    return (size_t)TmaLayout(box[0], box[1]).warp_bytes() * tma_pass_warps() + 128;
}

template <int CM>
int tma_grid_cm(int P, int num_sms, bool first, const int box[2]) {
    const size_t smem = tma_smem(box);
    auto kern = tma_kernel<CM>(first);
    TFS_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int per_sm = 0;
    TFS_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kTmaThreads, smem));
    const int need = (P + tma_pass_warps() - 1) / tma_pass_warps();
    return std::max(1, std::min(need, std::max(per_sm, 1) * num_sms));
}

template <int CM>
void tma_launch_cm(const TmaPassArgs &ta, int grid, cudaStream_t st) {
    auto kern = tma_kernel<CM>(ta.p.first != 0);
    kern<<<grid, kTmaThreads, tma_smem(ta.box), st>>>(ta);
    TFS_CUDA(cudaGetLastError());
}

#define TFS_FOR_EACH_TMA_CM(X) X(1) X(2) X(4) X(6) X(8) X(10)

}  // namespace

int tma_pass_grid(int CM, int P, int num_sms, bool first, const int box[2]) {
    switch (CM) {
#define TFS_CASE(cm) \
    case cm:         \
        return tma_grid_cm<cm>(P, num_sms, first, box);
        TFS_FOR_EACH_TMA_CM(TFS_CASE)
#undef TFS_CASE
        default:
            throw ApiError{TF_EINVAL, "no TMA mode-pass instance for this C"};
    }
}

void launch_mode_pass_tma(const PassArgs<float> &a, const void *tmaps, const int box[2], int CM,
                          int grid, cudaStream_t st) {
    TmaPassArgs ta;
    ta.p = a;
    memcpy(&ta.tm[0], tmaps, 2 * sizeof(CUtensorMap));
    ta.box[0] = box[0];
    ta.box[1] = box[1];
    switch (CM) {
#define TFS_CASE(cm)                        \
    case cm:                                \
        tma_launch_cm<cm>(ta, grid, st);    \
        return;
        TFS_FOR_EACH_TMA_CM(TFS_CASE)
#undef TFS_CASE
        default:
            throw ApiError{TF_EINVAL, "no TMA mode-pass instance for this C"};
    }
}

}  // namespace tfs
