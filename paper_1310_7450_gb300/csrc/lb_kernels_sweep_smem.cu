// Instantiation of the shared-memory resident cluster sweep (FP32 / BF16 / FP64 storage; stress mode A).
#include "lb_sweep_smem.cuh"

namespace lbk {
#define LB_SWEEP_SMEM_INST(T, C)                                                                              \
    template cudaError_t launch_sweep_smem<T, C, 128, 4>(const SweepArgs<T, C>&, int, int, size_t, cudaStream_t); \
    template cudaError_t launch_sweep_smem<T, C, 256, 4>(const SweepArgs<T, C>&, int, int, size_t, cudaStream_t); \
    template cudaError_t launch_sweep_smem_capacity<T, C, 128, 4>(int, size_t, int*);                               \
    template cudaError_t launch_sweep_smem_capacity<T, C, 256, 4>(int, size_t, int*);
LB_SWEEP_SMEM_INST(float, float)
LB_SWEEP_SMEM_INST(__nv_bfloat16, float)
LB_SWEEP_SMEM_INST(double, double)
#undef LB_SWEEP_SMEM_INST
}  // namespace lbk
