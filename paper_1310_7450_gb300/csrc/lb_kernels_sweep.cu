// Instantiation of the persistent cluster sweep (FP32 / BF16 / FP64 storage; stress mode A).
#include "lb_sweep.cuh"

namespace lbk {
#define LB_SWEEP_INST(T, C)                                                                              \
    template cudaError_t launch_sweep<T, C, 128, 4>(const SweepArgs<T, C>&, int, int, size_t, cudaStream_t); \
    template cudaError_t launch_sweep<T, C, 256, 4>(const SweepArgs<T, C>&, int, int, size_t, cudaStream_t); \
    template cudaError_t launch_sweep_capacity<T, C, 128, 4>(int, size_t, int*);                               \
    template cudaError_t launch_sweep_capacity<T, C, 256, 4>(int, size_t, int*);
LB_SWEEP_INST(float, float)
LB_SWEEP_INST(__nv_bfloat16, float)
LB_SWEEP_INST(double, double)
#undef LB_SWEEP_INST
}  // namespace lbk
