// Instantiation of the row-march kernel with pressure-driven ends (and a moving wall), BND = 1,
// and with a moving wall only, BND = 2 (FP32, BF16).
#include "lb_step_march.cuh"

namespace lbk {
template cudaError_t launch_step_march<float, float, 0, 1>(const CUtensorMap&, const StepArgs<float, float>&, const MarchCtl&, int, cudaStream_t);
template cudaError_t launch_step_march<float, float, 1, 1>(const CUtensorMap&, const StepArgs<float, float>&, const MarchCtl&, int, cudaStream_t);
template cudaError_t launch_step_march<__nv_bfloat16, float, 0, 1>(const CUtensorMap&, const StepArgs<__nv_bfloat16, float>&, const MarchCtl&, int, cudaStream_t);
template cudaError_t launch_step_march<__nv_bfloat16, float, 1, 1>(const CUtensorMap&, const StepArgs<__nv_bfloat16, float>&, const MarchCtl&, int, cudaStream_t);
template cudaError_t march_occupancy<float, float, 0, 1>(int*);
template cudaError_t march_occupancy<float, float, 1, 1>(int*);
template cudaError_t march_occupancy<__nv_bfloat16, float, 0, 1>(int*);
template cudaError_t march_occupancy<__nv_bfloat16, float, 1, 1>(int*);
template cudaError_t launch_step_march<float, float, 0, 2>(const CUtensorMap&, const StepArgs<float, float>&, const MarchCtl&, int, cudaStream_t);
template cudaError_t launch_step_march<float, float, 1, 2>(const CUtensorMap&, const StepArgs<float, float>&, const MarchCtl&, int, cudaStream_t);
template cudaError_t launch_step_march<__nv_bfloat16, float, 0, 2>(const CUtensorMap&, const StepArgs<__nv_bfloat16, float>&, const MarchCtl&, int, cudaStream_t);
template cudaError_t launch_step_march<__nv_bfloat16, float, 1, 2>(const CUtensorMap&, const StepArgs<__nv_bfloat16, float>&, const MarchCtl&, int, cudaStream_t);
template cudaError_t march_occupancy<float, float, 0, 2>(int*);
template cudaError_t march_occupancy<float, float, 1, 2>(int*);
template cudaError_t march_occupancy<__nv_bfloat16, float, 0, 2>(int*);
template cudaError_t march_occupancy<__nv_bfloat16, float, 1, 2>(int*);
}  // namespace lbk
