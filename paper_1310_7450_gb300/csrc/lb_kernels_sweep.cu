// Instantiation of the persistent cluster sweep (FP32 / BF16 / FP64 storage; stress mode A; any width,
// and the width 4 as a compile-time constant).
#include "lb_sweep.cuh"

namespace lbk {
#define LB_SWEEP_INST(T, C, NX)                                                                              \
    template cudaError_t launch_sweep<T, C, 128, 4, NX>(const SweepArgs<T, C>&, int, int, size_t, cudaStream_t); \
    template cudaError_t launch_sweep<T, C, 256, 4, NX>(const SweepArgs<T, C>&, int, int, size_t, cudaStream_t); \
    template cudaError_t launch_sweep_capacity<T, C, 128, 4, NX>(int, size_t, int*);                               \
    template cudaError_t launch_sweep_capacity<T, C, 256, 4, NX>(int, size_t, int*);
LB_SWEEP_INST(float, float, 0)
LB_SWEEP_INST(__nv_bfloat16, float, 0)
LB_SWEEP_INST(double, double, 0)
LB_SWEEP_INST(float, float, 4)  // the 4-column channels of the batched sweep
LB_SWEEP_INST(__nv_bfloat16, float, 4)
LB_SWEEP_INST(double, double, 4)
#undef LB_SWEEP_INST
}  // namespace lbk
