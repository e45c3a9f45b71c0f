// Instantiation of the fused step for the two mixed diagnostic precisions: FP64 storage with FP32
// arithmetic, and FP32 storage with FP64 arithmetic.  They separate the error of the storage
// format from the error of the arithmetic when the FP32 path is compared with the FP64 one.
#include "lb_step_tile.cuh"

namespace lbk {
template cudaError_t launch_step_tile<double, float, 0>(const StepArgs<double, float>&, int, size_t, cudaStream_t);
template cudaError_t launch_step_tile<double, float, 1>(const StepArgs<double, float>&, int, size_t, cudaStream_t);
template cudaError_t launch_step_tile<float, double, 0>(const StepArgs<float, double>&, int, size_t, cudaStream_t);
template cudaError_t launch_step_tile<float, double, 1>(const StepArgs<float, double>&, int, size_t, cudaStream_t);
}  // namespace lbk
