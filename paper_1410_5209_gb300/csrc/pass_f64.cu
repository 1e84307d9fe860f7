// Instantiation of the mode-pass and combine kernels for double (one translation unit
// per element type, so the two compile in parallel).
#include "mode_pass.cuh"

namespace tfs {

template <>
void launch_mode_pass<double>(const PassArgs<double> &a, int CM, const PassPlan &plan, cudaStream_t st) {
    launch_mode_pass_impl<double>(a, CM, plan, st);
}

template <>
PassPlan mode_pass_plan<double>(int CM, int N, int n, bool first, int num_sms, int P) {
    return mode_pass_plan_impl<double>(CM, N, n, first, num_sms, P);
}

template <>
int res_grid<double>(int CM, int P, int N) {
    return res_blocks_impl<double>(CM, P, N);
}

template <>
void launch_combine<double>(const PassArgs<double> &a, int CM, const SplitRow *rows, int n_rows,
                          cudaStream_t st) {
    launch_combine_impl<double>(a, CM, rows, n_rows, st);
}

template <>
void launch_res<double>(const ResArgs<double> &a, int CM, cudaStream_t st) {
    launch_res_impl<double>(a, CM, st);
}

template <>
void launch_solve_rows<double>(const PassArgs<double> &a, int CM, const SplitRow *rows, int n_rows,
                            cudaStream_t st) {
    launch_solve_rows_impl<double>(a, CM, rows, n_rows, st);
}

}  // namespace tfs
