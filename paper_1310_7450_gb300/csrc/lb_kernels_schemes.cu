// Instantiation of the fused step for the comparison schemes of Sec. II C (generalized Newtonian,
// SCHEME = 1; divergence of Sigma^nN as a force density, SCHEME = 2) in FP64, FP32 and BF16, stress
// mode 0 (a translation unit of its own so the library builds in parallel).
#include "lb_step_tile.cuh"

namespace lbk {
template cudaError_t launch_step_tile<double, double, 0, 1>(const StepArgs<double, double>&, int, size_t, cudaStream_t);
template cudaError_t launch_step_tile<double, double, 0, 2>(const StepArgs<double, double>&, int, size_t, cudaStream_t);
template cudaError_t launch_step_tile<float, float, 0, 1>(const StepArgs<float, float>&, int, size_t, cudaStream_t);
template cudaError_t launch_step_tile<float, float, 0, 2>(const StepArgs<float, float>&, int, size_t, cudaStream_t);
template cudaError_t launch_step_tile<__nv_bfloat16, float, 0, 1>(const StepArgs<__nv_bfloat16, float>&, int, size_t,
                                                                  cudaStream_t);
template cudaError_t launch_step_tile<__nv_bfloat16, float, 0, 2>(const StepArgs<__nv_bfloat16, float>&, int, size_t,
                                                                  cudaStream_t);
}  // namespace lbk
