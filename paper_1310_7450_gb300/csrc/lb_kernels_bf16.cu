// Instantiation of the fused step for __nv_bfloat16 storage / float arithmetic (one translation unit per
// precision so the library builds in parallel).
#include "lb_step_tile.cuh"

namespace lbk {
template cudaError_t launch_step_tile<__nv_bfloat16, float, 0>(const StepArgs<__nv_bfloat16, float>&, int, size_t, cudaStream_t);
template cudaError_t launch_step_tile<__nv_bfloat16, float, 1>(const StepArgs<__nv_bfloat16, float>&, int, size_t, cudaStream_t);
}  // namespace lbk
