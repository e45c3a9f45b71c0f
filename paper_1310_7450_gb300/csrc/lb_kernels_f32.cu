// Instantiation of the fused step for float storage / float arithmetic (one translation unit per
// precision so the library builds in parallel).
#include "lb_step_tile.cuh"

namespace lbk {
template cudaError_t launch_step_tile<float, float, 0>(const StepArgs<float, float>&, int, size_t, cudaStream_t);
template cudaError_t launch_step_tile<float, float, 1>(const StepArgs<float, float>&, int, size_t, cudaStream_t);
}  // namespace lbk
