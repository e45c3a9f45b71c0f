// Instantiation of the fused step for double storage / double arithmetic (one translation unit per
// precision so the library builds in parallel).
#include "lb_step_tile.cuh"

namespace lbk {
template cudaError_t launch_step_tile<double, double, 0>(const StepArgs<double, double>&, int, size_t, cudaStream_t);
template cudaError_t launch_step_tile<double, double, 1>(const StepArgs<double, double>&, int, size_t, cudaStream_t);
}  // namespace lbk
