// Instantiation of the fused step with the relaxation-time extensions (SCHEME = 3: the paper's
// forcing with a density-dependent Maxwell time and a fluidity memory for tau_M) in FP64, FP32
// and BF16, both stress modes (a translation unit of its own so the library builds in parallel).
#include "lb_step_tile.cuh"

namespace lbk {
template cudaError_t launch_step_tile<double, double, 0, 3>(const StepArgs<double, double>&, int, size_t, cudaStream_t);
template cudaError_t launch_step_tile<double, double, 1, 3>(const StepArgs<double, double>&, int, size_t, cudaStream_t);
template cudaError_t launch_step_tile<float, float, 0, 3>(const StepArgs<float, float>&, int, size_t, cudaStream_t);
template cudaError_t launch_step_tile<float, float, 1, 3>(const StepArgs<float, float>&, int, size_t, cudaStream_t);
template cudaError_t launch_step_tile<__nv_bfloat16, float, 0, 3>(const StepArgs<__nv_bfloat16, float>&, int, size_t,
                                                                  cudaStream_t);
template cudaError_t launch_step_tile<__nv_bfloat16, float, 1, 3>(const StepArgs<__nv_bfloat16, float>&, int, size_t,
                                                                  cudaStream_t);
}  // namespace lbk
