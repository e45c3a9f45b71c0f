// Instantiation of the TMA-fed row-march step (wide single channels; FP32 and BF16 storage; the
// paper's scheme in both stress modes, the generalized-Newtonian comparison scheme and the
// relaxation-time extensions).
#include "lb_step_march.cuh"

namespace lbk {
template cudaError_t launch_step_march<float, float, 0>(const CUtensorMap&, const StepArgs<float, float>&, const MarchCtl&, int, cudaStream_t);
template cudaError_t launch_step_march<float, float, 1>(const CUtensorMap&, const StepArgs<float, float>&, const MarchCtl&, int, cudaStream_t);
template cudaError_t launch_step_march<__nv_bfloat16, float, 0>(const CUtensorMap&, const StepArgs<__nv_bfloat16, float>&, const MarchCtl&, int, cudaStream_t);
template cudaError_t launch_step_march<__nv_bfloat16, float, 1>(const CUtensorMap&, const StepArgs<__nv_bfloat16, float>&, const MarchCtl&, int, cudaStream_t);
template cudaError_t march_occupancy<float, float, 0>(int*);
template cudaError_t march_occupancy<float, float, 1>(int*);
template cudaError_t march_occupancy<__nv_bfloat16, float, 0>(int*);
template cudaError_t march_occupancy<__nv_bfloat16, float, 1>(int*);
// the generalized-Newtonian comparison scheme (stress mode A, periodic x, bounce-back walls)
template cudaError_t launch_step_march<float, float, 0, 0, 1>(const CUtensorMap&, const StepArgs<float, float>&, const MarchCtl&, int, cudaStream_t);
template cudaError_t launch_step_march<__nv_bfloat16, float, 0, 0, 1>(const CUtensorMap&, const StepArgs<__nv_bfloat16, float>&, const MarchCtl&, int, cudaStream_t);
template cudaError_t march_occupancy<float, float, 0, 0, 1>(int*);
template cudaError_t march_occupancy<__nv_bfloat16, float, 0, 0, 1>(int*);
// the relaxation-time extensions (periodic x, bounce-back walls, both stress modes)
template cudaError_t launch_step_march<float, float, 0, 0, 3>(const CUtensorMap&, const StepArgs<float, float>&, const MarchCtl&, int, cudaStream_t);
template cudaError_t launch_step_march<float, float, 1, 0, 3>(const CUtensorMap&, const StepArgs<float, float>&, const MarchCtl&, int, cudaStream_t);
template cudaError_t launch_step_march<__nv_bfloat16, float, 0, 0, 3>(const CUtensorMap&, const StepArgs<__nv_bfloat16, float>&, const MarchCtl&, int, cudaStream_t);
template cudaError_t launch_step_march<__nv_bfloat16, float, 1, 0, 3>(const CUtensorMap&, const StepArgs<__nv_bfloat16, float>&, const MarchCtl&, int, cudaStream_t);
template cudaError_t march_occupancy<float, float, 0, 0, 3>(int*);
template cudaError_t march_occupancy<float, float, 1, 0, 3>(int*);
template cudaError_t march_occupancy<__nv_bfloat16, float, 0, 0, 3>(int*);
template cudaError_t march_occupancy<__nv_bfloat16, float, 1, 0, 3>(int*);
}  // namespace lbk
