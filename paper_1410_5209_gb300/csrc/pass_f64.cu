// Instantiation of the mode-pass and combine kernels for double (one translation unit
// per element type, so the two compile in parallel).
#include "mode_pass.cuh"

namespace tfs {

template <>
void launch_mode_pass<double>(const PassArgs<double> &a, int CM, int grid, cudaStream_t st) {
    launch_mode_pass_impl<double>(a, CM, grid, st);
}

template <>
int mode_pass_grid<double>(int CM, int P, int num_sms) {
    return mode_pass_grid_impl<double>(CM, P, num_sms);
}

template <>
void launch_combine<double>(const PassArgs<double> &a, int CM, const SplitRow *rows, int n_rows,
                          cudaStream_t st) {
    launch_combine_impl<double>(a, CM, rows, n_rows, st);
}

}  // namespace tfs
