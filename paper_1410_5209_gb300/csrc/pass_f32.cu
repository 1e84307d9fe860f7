// Instantiation of the mode-pass and combine kernels for float (one translation unit
// per element type, so the two compile in parallel).
#include "mode_pass.cuh"

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

}  // namespace tfs
