// lb_api.cu -- the C ABI declared in include/lbnlm.h: handle management, state layout, launch
// sequencing of the fused step, field output, residual reduction, checkpointing.
//
// Device layout of a handle (all channels in one allocation per field):
//   every channel c owns planes of P[c] elements (P[c] >= nx*ny[c], padded to 64 elements);
//   base[c] = sum_{c'<c} P[c'] is the channel's plane offset, so a field with k planes keeps
//   plane j of channel c at  k*base[c] + j*P[c].  Populations: 9 planes (ping-pong A/B);
//   delta rho: 1 plane; carried stress (mode 1): 3 planes; stress output: 4 planes; saved
//   velocity: 2 planes.
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <type_traits>
#include <vector>

#include "lb_step_march.cuh"
#include "lb_step_tile.cuh"
#include "lb_sweep.cuh"
#include "lb_sweep_smem.cuh"
#include "lbnlm.h"

namespace lbk {
// learned warm start (lb_warmstart.cu)
struct WsChan {
    double g, G, tau0, theta, gamma_c;
};
cudaError_t launch_ws_closed_form(int n_ch, const WsChan* prm, const int* nys, const int* row_off, double* rows,
                                  double* grid, double* scale, cudaStream_t s);
cudaError_t launch_ws_decode(int n_ch, const float* pred, const float* t_mu, const float* t_sd, const double* grid,
                             const double* scale, const double* rows, const int* nys, const int* row_off,
                             const long long* node_off, int nx, double* u, double* rho, double* drho, cudaStream_t s);
template <typename F>
cudaError_t launch_ws_targets(int n_ch, const F* fu, const F* fs, const double* grid, const double* scale, const int* nys,
                              const long long* node_off, int nx, float* targets, cudaStream_t s);
extern template cudaError_t launch_step_tile<double, double, 0>(const StepArgs<double, double>&, int, size_t, cudaStream_t);
extern template cudaError_t launch_step_tile<double, double, 1>(const StepArgs<double, double>&, int, size_t, cudaStream_t);
extern template cudaError_t launch_step_tile<float, float, 0>(const StepArgs<float, float>&, int, size_t, cudaStream_t);
extern template cudaError_t launch_step_tile<float, float, 1>(const StepArgs<float, float>&, int, size_t, cudaStream_t);
extern template cudaError_t launch_step_tile<__nv_bfloat16, float, 0>(const StepArgs<__nv_bfloat16, float>&, int, size_t, cudaStream_t);
extern template cudaError_t launch_step_tile<__nv_bfloat16, float, 1>(const StepArgs<__nv_bfloat16, float>&, int, size_t, cudaStream_t);
extern template cudaError_t launch_step_tile<double, float, 0>(const StepArgs<double, float>&, int, size_t, cudaStream_t);
extern template cudaError_t launch_step_tile<double, float, 1>(const StepArgs<double, float>&, int, size_t, cudaStream_t);
extern template cudaError_t launch_step_tile<float, double, 0>(const StepArgs<float, double>&, int, size_t, cudaStream_t);
extern template cudaError_t launch_step_tile<float, double, 1>(const StepArgs<float, double>&, int, size_t, cudaStream_t);
extern template cudaError_t launch_step_tile<double, double, 0, 3>(const StepArgs<double, double>&, int, size_t, cudaStream_t);
extern template cudaError_t launch_step_tile<double, double, 1, 3>(const StepArgs<double, double>&, int, size_t, cudaStream_t);
extern template cudaError_t launch_step_tile<float, float, 0, 3>(const StepArgs<float, float>&, int, size_t, cudaStream_t);
extern template cudaError_t launch_step_tile<float, float, 1, 3>(const StepArgs<float, float>&, int, size_t, cudaStream_t);
extern template cudaError_t launch_step_tile<__nv_bfloat16, float, 0, 3>(const StepArgs<__nv_bfloat16, float>&, int, size_t,
                                                                         cudaStream_t);
extern template cudaError_t launch_step_tile<__nv_bfloat16, float, 1, 3>(const StepArgs<__nv_bfloat16, float>&, int, size_t,
                                                                         cudaStream_t);
extern template cudaError_t launch_step_tile<double, double, 0, 1>(const StepArgs<double, double>&, int, size_t, cudaStream_t);
extern template cudaError_t launch_step_tile<double, double, 0, 2>(const StepArgs<double, double>&, int, size_t, cudaStream_t);
extern template cudaError_t launch_step_tile<float, float, 0, 1>(const StepArgs<float, float>&, int, size_t, cudaStream_t);
extern template cudaError_t launch_step_tile<float, float, 0, 2>(const StepArgs<float, float>&, int, size_t, cudaStream_t);
extern template cudaError_t launch_step_tile<__nv_bfloat16, float, 0, 1>(const StepArgs<__nv_bfloat16, float>&, int, size_t,
                                                                         cudaStream_t);
extern template cudaError_t launch_step_tile<__nv_bfloat16, float, 0, 2>(const StepArgs<__nv_bfloat16, float>&, int, size_t,
                                                                         cudaStream_t);
extern template cudaError_t launch_step_march<float, float, 0>(const CUtensorMap&, const StepArgs<float, float>&, const MarchCtl&, int, cudaStream_t);
extern template cudaError_t launch_step_march<float, float, 1>(const CUtensorMap&, const StepArgs<float, float>&, const MarchCtl&, int, cudaStream_t);
extern template cudaError_t launch_step_march<__nv_bfloat16, float, 0>(const CUtensorMap&, const StepArgs<__nv_bfloat16, float>&, const MarchCtl&, int, cudaStream_t);
extern template cudaError_t launch_step_march<__nv_bfloat16, float, 1>(const CUtensorMap&, const StepArgs<__nv_bfloat16, float>&, const MarchCtl&, int, cudaStream_t);
#define LB_SWEEP_EXTERN(T, C, NX)                                                                                   \
    extern template cudaError_t launch_sweep<T, C, 128, 4, NX>(const SweepArgs<T, C>&, int, int, size_t, cudaStream_t); \
    extern template cudaError_t launch_sweep<T, C, 256, 4, NX>(const SweepArgs<T, C>&, int, int, size_t, cudaStream_t); \
    extern template cudaError_t launch_sweep_capacity<T, C, 128, 4, NX>(int, size_t, int*);                            \
    extern template cudaError_t launch_sweep_capacity<T, C, 256, 4, NX>(int, size_t, int*);
LB_SWEEP_EXTERN(float, float, 0)
LB_SWEEP_EXTERN(__nv_bfloat16, float, 0)
LB_SWEEP_EXTERN(double, double, 0)
LB_SWEEP_EXTERN(float, float, 4)
LB_SWEEP_EXTERN(__nv_bfloat16, float, 4)
LB_SWEEP_EXTERN(double, double, 4)
#undef LB_SWEEP_EXTERN
#define LB_SWEEP_SMEM_EXTERN(T, C, NX)                                                                                   \
    extern template cudaError_t launch_sweep_smem<T, C, 128, 4, NX>(const SweepArgs<T, C>&, int, int, size_t, cudaStream_t); \
    extern template cudaError_t launch_sweep_smem<T, C, 256, 4, NX>(const SweepArgs<T, C>&, int, int, size_t, cudaStream_t); \
    extern template cudaError_t launch_sweep_smem_capacity<T, C, 128, 4, NX>(int, size_t, int*);                            \
    extern template cudaError_t launch_sweep_smem_capacity<T, C, 256, 4, NX>(int, size_t, int*);
LB_SWEEP_SMEM_EXTERN(float, float, 0)
LB_SWEEP_SMEM_EXTERN(__nv_bfloat16, float, 0)
LB_SWEEP_SMEM_EXTERN(double, double, 0)
LB_SWEEP_SMEM_EXTERN(float, float, 4)
LB_SWEEP_SMEM_EXTERN(__nv_bfloat16, float, 4)
LB_SWEEP_SMEM_EXTERN(double, double, 4)
#undef LB_SWEEP_SMEM_EXTERN
extern template cudaError_t march_occupancy<float, float, 0>(int*);
extern template cudaError_t march_occupancy<float, float, 1>(int*);
extern template cudaError_t march_occupancy<__nv_bfloat16, float, 0>(int*);
extern template cudaError_t march_occupancy<__nv_bfloat16, float, 1>(int*);
extern template cudaError_t launch_step_march<float, float, 0, 0, 1>(const CUtensorMap&, const StepArgs<float, float>&, const MarchCtl&, int, cudaStream_t);
extern template cudaError_t launch_step_march<__nv_bfloat16, float, 0, 0, 1>(const CUtensorMap&, const StepArgs<__nv_bfloat16, float>&, const MarchCtl&, int, cudaStream_t);
extern template cudaError_t march_occupancy<float, float, 0, 0, 1>(int*);
extern template cudaError_t march_occupancy<__nv_bfloat16, float, 0, 0, 1>(int*);
extern template cudaError_t launch_step_march<float, float, 0, 0, 3>(const CUtensorMap&, const StepArgs<float, float>&, const MarchCtl&, int, cudaStream_t);
extern template cudaError_t launch_step_march<float, float, 1, 0, 3>(const CUtensorMap&, const StepArgs<float, float>&, const MarchCtl&, int, cudaStream_t);
extern template cudaError_t launch_step_march<__nv_bfloat16, float, 0, 0, 3>(const CUtensorMap&, const StepArgs<__nv_bfloat16, float>&, const MarchCtl&, int, cudaStream_t);
extern template cudaError_t launch_step_march<__nv_bfloat16, float, 1, 0, 3>(const CUtensorMap&, const StepArgs<__nv_bfloat16, float>&, const MarchCtl&, int, cudaStream_t);
extern template cudaError_t march_occupancy<float, float, 0, 0, 3>(int*);
extern template cudaError_t march_occupancy<float, float, 1, 0, 3>(int*);
extern template cudaError_t march_occupancy<__nv_bfloat16, float, 0, 0, 3>(int*);
extern template cudaError_t march_occupancy<__nv_bfloat16, float, 1, 0, 3>(int*);
extern template cudaError_t launch_step_march<float, float, 0, 1>(const CUtensorMap&, const StepArgs<float, float>&, const MarchCtl&, int, cudaStream_t);
extern template cudaError_t launch_step_march<float, float, 1, 1>(const CUtensorMap&, const StepArgs<float, float>&, const MarchCtl&, int, cudaStream_t);
extern template cudaError_t launch_step_march<__nv_bfloat16, float, 0, 1>(const CUtensorMap&, const StepArgs<__nv_bfloat16, float>&, const MarchCtl&, int, cudaStream_t);
extern template cudaError_t launch_step_march<__nv_bfloat16, float, 1, 1>(const CUtensorMap&, const StepArgs<__nv_bfloat16, float>&, const MarchCtl&, int, cudaStream_t);
extern template cudaError_t march_occupancy<float, float, 0, 1>(int*);
extern template cudaError_t march_occupancy<float, float, 1, 1>(int*);
extern template cudaError_t march_occupancy<__nv_bfloat16, float, 0, 1>(int*);
extern template cudaError_t march_occupancy<__nv_bfloat16, float, 1, 1>(int*);
extern template cudaError_t launch_step_march<float, float, 0, 2>(const CUtensorMap&, const StepArgs<float, float>&, const MarchCtl&, int, cudaStream_t);
extern template cudaError_t launch_step_march<float, float, 1, 2>(const CUtensorMap&, const StepArgs<float, float>&, const MarchCtl&, int, cudaStream_t);
extern template cudaError_t launch_step_march<__nv_bfloat16, float, 0, 2>(const CUtensorMap&, const StepArgs<__nv_bfloat16, float>&, const MarchCtl&, int, cudaStream_t);
extern template cudaError_t launch_step_march<__nv_bfloat16, float, 1, 2>(const CUtensorMap&, const StepArgs<__nv_bfloat16, float>&, const MarchCtl&, int, cudaStream_t);
extern template cudaError_t march_occupancy<float, float, 0, 2>(int*);
extern template cudaError_t march_occupancy<float, float, 1, 2>(int*);
extern template cudaError_t march_occupancy<__nv_bfloat16, float, 0, 2>(int*);
extern template cudaError_t march_occupancy<__nv_bfloat16, float, 1, 2>(int*);
}  // namespace lbk

using namespace lbk;

namespace {

thread_local char g_err[512] = "";

lb_status fail(lb_status s, const char* fmt, const char* detail = nullptr) {
    std::snprintf(g_err, sizeof g_err, fmt, detail ? detail : "");
    return s;
}
}  // namespace

namespace lbk {
// Lets other translation units of the library report a failure through lb_last_error().
void set_last_error(const char* msg) { std::snprintf(g_err, sizeof g_err, "%s", msg); }
}  // namespace lbk

namespace {

lb_status cuda_fail(cudaError_t e, const char* where) {
    std::snprintf(g_err, sizeof g_err, "%s: %s", where, cudaGetErrorString(e));
    return e == cudaErrorMemoryAllocation ? LB_ENOMEM : LB_ECUDA;
}
#define LB_CK(call)                                              \
    do {                                                         \
        cudaError_t e_ = (call);                                 \
        if (e_ != cudaSuccess) return cuda_fail(e_, #call);      \
    } while (0)

constexpr int kThreads = 256;        // threads per CTA of the tile kernel
constexpr double kGuard = 0.3;       // |u| above which a channel is declared unstable

// SplitMix64 (Steele, Lea & Flood 2014; 64-bit finaliser as published by Vigna): output number
// `counter` (>= 1) of the stream seeded with `seed`.
__device__ __forceinline__ uint64_t splitmix64(uint64_t seed, uint64_t counter) {
    uint64_t z = seed + counter * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

struct InitChan {
    long long base, P;
    int ny, gpbc;
    double rho0, amp;
    uint64_t seed;
    double rho_in, rho_out;  // GPBC: densities at the ghost columns x = -1 and x = nx
};

// Rest equilibrium n_i = w_i rho(r), rho = rho0 (1 + amp U(-1,1)); delta rho = 0.  Under GPBC the
// density starts on the straight line between the inlet and outlet ghost densities (the linear
// pre-initialisation of Sec. II B): rho = rho_in + (rho_out - rho_in)(x+1)/(nx+1) + rho0 amp U.
template <typename T, typename C>
__global__ void k_init(T* pop, C* drho, C* sig3, const InitChan* ch, int nx, int smode) {
    const InitChan c = ch[blockIdx.y];
    const long long n = (long long)nx * c.ny;
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n; k += (long long)gridDim.x * blockDim.x) {
        double rho = c.rho0;
        double U = 0.0;
        if (c.amp != 0.0) {
            const uint64_t z = splitmix64(c.seed, (uint64_t)k + 1ull);
            U = __dadd_rn(__dmul_rn((double)(z >> 11), 0x1p-52), -1.0);
            rho = __dmul_rn(c.rho0, __dadd_rn(1.0, __dmul_rn(c.amp, U)));
        }
        if (c.gpbc) {
            const double lin = c.rho_in + (c.rho_out - c.rho_in) * (double)(k % nx + 1) / (double)(nx + 1);
            rho = __dadd_rn(lin, __dmul_rn(c.rho0, __dmul_rn(c.amp, U)));
        }
        const double dev = rho - 1.0;
#pragma unroll
        for (int i = 0; i < 9; ++i) Store<T>::st(pop + 9 * c.base + i * c.P + k, (C)(wgt<double>(i) * dev));
        drho[c.base + k] = C(0);
        if (smode == 1)
            for (int j = 0; j < 3; ++j) sig3[3 * c.base + j * c.P + k] = C(0);
    }
}

// Populations <-> full FP64 values in plane order (host staging is compact per channel).
template <typename T, typename C>
__global__ void k_pop_from_f64(T* pop, const double* src, const long long* base, const long long* P,
                               const long long* node_off, const int* ny, int nx) {
    const int c = blockIdx.y;
    const long long n = (long long)nx * ny[c];
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n; k += (long long)gridDim.x * blockDim.x)
#pragma unroll
        for (int i = 0; i < 9; ++i)
            Store<T>::st(pop + 9 * base[c] + i * P[c] + k, (C)(src[9 * node_off[c] + i * n + k] - wgt<double>(i)));
}
template <typename T, typename C>
__global__ void k_pop_to_f64(const T* pop, double* dst, const long long* base, const long long* P,
                             const long long* node_off, const int* ny, int nx) {
    const int c = blockIdx.y;
    const long long n = (long long)nx * ny[c];
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n; k += (long long)gridDim.x * blockDim.x)
#pragma unroll
        for (int i = 0; i < 9; ++i)
            dst[9 * node_off[c] + i * n + k] = (double)Store<T>::ld(pop + 9 * base[c] + i * P[c] + k) + wgt<double>(i);
}
// k planes of a compact per-channel FP64 field <-> the padded C planes.
template <typename C>
__global__ void k_planes_from_f64(C* dst, const double* src, int kp, const long long* base, const long long* P,
                                  const long long* node_off, const int* ny, int nx) {
    const int c = blockIdx.y;
    const long long n = (long long)nx * ny[c];
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n; k += (long long)gridDim.x * blockDim.x)
        for (int j = 0; j < kp; ++j) dst[kp * base[c] + j * P[c] + k] = (C)src[kp * node_off[c] + j * n + k];
}
template <typename C>
__global__ void k_planes_to_f64(const C* src, double* dst, int kp, const long long* base, const long long* P,
                                const long long* node_off, const int* ny, int nx) {
    const int c = blockIdx.y;
    const long long n = (long long)nx * ny[c];
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n; k += (long long)gridDim.x * blockDim.x)
        for (int j = 0; j < kp; ++j) dst[kp * node_off[c] + j * n + k] = (double)src[kp * base[c] + j * P[c] + k];
}

// Warm start: equilibrium of (rho, u - f/(2 rho)) so that j = sum c n + f/2 = rho u (Eq. rhoj).
template <typename T, typename C>
__global__ void k_set_fields(T* pop, C* drho, C* sig3, const double* u, const double* rho, const double* dr,
                             const long long* base, const long long* P, const long long* node_off, const int* ny,
                             const double* gx, int nx, int smode, int gpbc) {
    const int c = blockIdx.y;
    const double g = gpbc ? 0.0 : gx[c];  // no body force in a pressure-driven channel
    const long long n = (long long)nx * ny[c];
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n; k += (long long)gridDim.x * blockDim.x) {
        const long long node = node_off[c] + k;
        const double r = rho[node];
        const double ux = u[2 * node] - 0.5 * g / r, uy = u[2 * node + 1];
        const double usq = ux * ux + uy * uy;
#pragma unroll
        for (int i = 0; i < 9; ++i) {
            const double cu = cx(i) * ux + cy(i) * uy;
            const double w = wgt<double>(i);
            const double dev = w * ((r - 1.0) + r * (3.0 * cu + 4.5 * cu * cu - 1.5 * usq));
            Store<T>::st(pop + 9 * base[c] + i * P[c] + k, (C)dev);
        }
        drho[base[c] + k] = (dr && !gpbc) ? (C)dr[node] : C(0);
        if (smode == 1)
            for (int j = 0; j < 3; ++j) sig3[3 * base[c] + j * P[c] + k] = C(0);
    }
}

// Apply the per-channel body forces (staged[0..n_ch)) and moving-wall velocities
// (staged[n_ch..2 n_ch)), read straight from the pinned host staging slot (mapped), and keep a
// device copy in gx for the kernels that read the drive there.
template <typename C>
__global__ void k_apply_gx(ChanParams<C>* chan, double* gx, const double* staged, int n_ch, int nx) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= n_ch) return;
    const double g = staged[c], uw = staged[n_ch + c];
    gx[c] = g;
    gx[n_ch + c] = uw;
    chan[c].u_wall = (C)uw;  // staged after the forces: the moving-wall velocities
    if (chan[c].gpbc) {  // pressure-driven: g sets the ghost densities, there is no body force
        const double half = 1.5 * g * (double)(nx + 1);
        chan[c].rho_in = (C)((double)chan[c].rho0_m1 + half);
        chan[c].rho_out = (C)((double)chan[c].rho0_m1 - half);
    } else {
        chan[c].gx = (C)g;
    }
}

// Copy n doubles from device memory to mapped pinned host memory (the monitor's way back: a
// kernel's stores reach the host without a copy-engine transfer in the stream).
__global__ void k_copy_to_host(const double* src, double* dst, int n) {
    for (int k = threadIdx.x; k < n; k += blockDim.x) dst[k] = src[k];
}

// Per-channel reduction of the step's block partials, one warp per channel in a fixed order
// (deterministic; the row-march kernel forms the same values itself, see monitor_reduce_warp).
// with_residual = 0: the partials hold flux and max |u| only (F_MON); the residual slot reads -1
__global__ void k_reduce_residual(const double* partials, const int* item_begin, const int* status, double* mon,
                                  int nx, long long state_index, int with_residual) {
    const int c = blockIdx.x;
    monitor_reduce_warp(partials, item_begin[c], item_begin[c + 1], status[c], mon + 4 * c, nx, state_index,
                        with_residual, threadIdx.x);
}

template <typename A, typename B>
__global__ void k_convert(const A* src, B* dst, long long n) {
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n; k += (long long)gridDim.x * blockDim.x)
        dst[k] = (B)src[k];
}

int grid_for(long long n) {
    long long b = (n + 255) / 256;
    return (int)(b < 1 ? 1 : (b > 4096 ? 4096 : b));
}

// Storage type T and arithmetic type C of a precision mode.
template <typename X> struct Tag { using type = X; };
template <typename F>
auto with_types(int prec, F&& f) {
    switch (prec) {
        case LB_PREC_F64: return f(Tag<double>{}, Tag<double>{});
        case LB_PREC_F32: return f(Tag<float>{}, Tag<float>{});
        case LB_PREC_BF16: return f(Tag<__nv_bfloat16>{}, Tag<float>{});
        case LB_PREC_F64S_F32M: return f(Tag<double>{}, Tag<float>{});
        default: return f(Tag<float>{}, Tag<double>{});
    }
}
#define LB_TYPES(tt, tc)                          \
    using T = typename decltype(tt)::type;        \
    using C = typename decltype(tc)::type;

}  // namespace

// Channels of one width class in the batched sweep and the configuration they run with.
struct SweepGroup {
    int cls = 0;                    // floor(log2 ny)
    int begin = 0, count = 0;       // range in the widest-first channel order
    int ny_min = 0, ny_max = 0;
    int var = 0, nt = 0, cl = 0;    // 0: state through L2, 1: state in shared memory; nt == 0: not tuned
    double tune_ms = 0.0;
};

constexpr int kDriveRing = 8;  // pinned staging slots of the drive (body force, wall velocity)

// NVTX range over a public call, so that profiler timelines (Nsight Systems / Compute) group the
// launches of one lb_step or sweep; a no-op unless a tool is attached.
struct NvtxRange {
    explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange&) = delete;
    NvtxRange& operator=(const NvtxRange&) = delete;
};

struct lb_handle {
    int dev = 0;
    cudaStream_t stream = nullptr;
    int n_ch = 0, nx = 0, prec = 0, smode = 0, flags = 0;
    std::vector<int> ny;
    std::vector<long long> P, base, node_off;
    long long planes = 0;  // sum of P
    long long nodes = 0;
    std::vector<lb_params> params;
    size_t tsize = 0, csize = 0;  // storage / arithmetic element sizes
    // device state
    void *popA = nullptr, *popB = nullptr, *drho = nullptr, *sig3 = nullptr, *sig4 = nullptr, *uprev = nullptr;
    void* snn = nullptr;  // stress-divergence scheme: Sigma^nN of the current step [3 planes]
    void* phi = nullptr;  // relaxation-time extensions: fluidity 1/tau_M per node [plane]
    int scheme = 0;       // 0: the paper's forcing; 1: generalized Newtonian; 2: div Sigma^nN force;
                          // 3: the paper's forcing with the relaxation-time extensions
    std::vector<double> beta_rho, rho_ref, tau_f;  // scheme 3, per channel
    // learned warm start: per-channel closed-form parameters, row offsets, closed form on the rows
    // [row][3] and on the network grid [channel][3][256], scales [channel][3]
    void *ws_prm = nullptr, *ws_row_off = nullptr, *ws_rows = nullptr, *ws_grid = nullptr, *ws_scale = nullptr;
    void* chan = nullptr;
    WorkItem* items_d = nullptr;
    int* item_begin_d = nullptr;
    double* partials = nullptr;
    double* mon_d = nullptr;
    int* status_d = nullptr;
    long long *base_d = nullptr, *P_d = nullptr, *node_off_d = nullptr;
    int* ny_d = nullptr;
    double* gx_d = nullptr;
    void* fields = nullptr;    // staging for lb_get_fields, 7 values per node in C type
    void* fconv = nullptr;     // staging for converted fields, 7 values per node
    void* hstage = nullptr;    // device staging for FP64 host transfers
    size_t hstage_bytes = 0;
    // launch plan
    std::vector<WorkItem> items;
    std::vector<int> item_begin;
    size_t smem = 0;
    // bookkeeping
    long step = 0;
    long uprev_state = -10;    // state index whose velocity u_prev holds
    long mon_state = -1;       // state index of the last monitor evaluation (-1: none)
    bool mon_resid = false;    // the last monitor evaluation includes the residual
    int monitor_mode = 0;      // LB_MONITOR_RESIDUAL or LB_MONITOR_FLUX_MAX
    int* status_h = nullptr;   // pinned, mapped (row march: the kernel's status mirror)
    int* status_hd = nullptr;  // its device address
    double* gx_h = nullptr;              // pinned staging of the drive: kDriveRing slots of 2 n_ch
    double* gx_hd = nullptr;             // its device address (mapped)
    double* mon_h = nullptr;             // mapped pinned copy of the monitor for lb_monitor
    double* mon_hd = nullptr;
    cudaEvent_t gx_ev[kDriveRing] = {};  // values, each reused once its previous copy has run
    bool gx_pending[kDriveRing] = {};
    int gx_slot = 0;
    cudaEvent_t status_ev = nullptr;
    bool status_pending = false;
    bool any_unstable = false;
    bool any_timeout = false;
    unsigned long long wait_ns = 2000000000ull;  // limit of the row-march kernel's mbarrier waits
    // row-march kernel (wide single channels, FP32 / BF16 storage)
    bool march = false;
    CUtensorMap mapA, mapB;    // tensor maps of the two population buffers ...
    const void* mapA_buf = nullptr;  // ... and the buffers they describe (the pointers swap)
    const void* mapB_buf = nullptr;
    // persistent cluster sweep
    long long* sweep_steps_d = nullptr;
    double* sweep_res_d = nullptr;
    int* sweep_order_d = nullptr;
    std::vector<SweepGroup> sweep_groups;  // width classes of the active channels and their configurations
    std::vector<cudaStream_t> gstreams;     // forked streams of the class launches
    std::vector<cudaEvent_t> gevents;
    cudaEvent_t fork_ev = nullptr;
    bool sweep_fixed = false;               // configuration set by lb_sweep_set_config
    cudaGraphExec_t sweep_gexec = nullptr;  // the class launches captured as one graph ...
    std::vector<double> sweep_key;          // ... for these arguments and configurations
    MarchItem* march_items_d = nullptr;
    int* march_item_begin_d = nullptr;  // {0, n_march_items}: the residual reduction's item range
    int n_march_items = 0, march_grid = 0;
    // CUDA graphs of kGraphSteps plain tile-kernel steps, one per input buffer (an even count of
    // steps leaves the buffers where they were, so each graph starts from the buffer it names)
    cudaGraphExec_t gexec[2] = {nullptr, nullptr};
    const void* gexec_pin[2] = {nullptr, nullptr};
    cudaStream_t cap_stream = nullptr;
    long graph_replays = 0;
    // generalized periodic boundaries (x_mode LB_X_GPBC)
    bool gpbc = false;
    void* gcol = nullptr;  // boundary-column moments and means (see StepArgs::gcol)
    double* gpart = nullptr;    // per-block partial sums of the column kernel
    unsigned* gcount = nullptr; // per-column block counters (zero between launches)
    unsigned* done_count_d = nullptr;  // row-march CTAs done with the launch (zero between launches)
    int gpbc_max_ny = 0;
    int gny = 0;           // sum of ny over the channels
    std::vector<int> row_off;
    // planar Couette flow (walls LB_WALLS_COUETTE): Zou-He moving wall on the last row
    bool moving = false;
    std::vector<double> u_wall;
};

namespace {

template <typename C>
std::vector<ChanParams<C>> make_chan(const lb_handle* h) {
    std::vector<ChanParams<C>> v(h->n_ch);
    for (int c = 0; c < h->n_ch; ++c) {
        const lb_params& p = h->params[c];
        ChanParams<C> q{};
        q.base = h->base[c];
        q.P = h->P[c];
        q.node_off = h->node_off[c];
        q.ny = h->ny[c];
        q.omega = (C)(1.0 / p.tau_lb);
        q.k1 = (C)(-9.0 / (2.0 * p.tau_lb));
        q.k2 = (C)(1.0 - 1.0 / (2.0 * p.tau_lb));
        q.gx = (C)p.g_x;
        q.G = (C)p.G_inf;
        q.tau = (C)(p.theta * p.tau0);
        q.inv_gc = std::isinf(p.gamma_c) ? C(0) : (C)(1.0 / p.gamma_c);
        q.cD = (C)(p.G_inf * p.tau0 - p.rho0 * (p.tau_lb - 0.5) / 3.0);
        q.kdr = C(1);
        q.rho0_m1 = (C)(p.rho0 - 1.0);
        q.moving = h->moving ? 1 : 0;
        q.u_wall = (C)h->u_wall[c];
        q.scheme = h->scheme;
        q.rho_ref = C(1);
        if (h->scheme == 3) {
            q.beta_rho = (C)h->beta_rho[c];
            q.rho_ref = (C)h->rho_ref[c];
            q.tau_f = (C)h->tau_f[c];
        }
        if (h->scheme == 1 || h->scheme == 2) {
            // the comparison schemes of Sec. II C: no stress line and no flow-induced density
            q.k1 = C(0);
            q.kdr = C(0);
            q.gn_a = (C)(3.0 * p.G_inf / p.rho0);
            q.gn_b = (C)(0.5 + 3.0 * p.G_inf * p.tau0 / p.rho0);
        }
        if (h->gpbc) {
            // GPBC (Sec. II B): the pressure gradient replaces the body force, p_+ - p_- = g (nx+1)
            // between the ghost columns; no flow-induced density, Eq. (bodyforce) first line only
            q.gpbc = 1;
            q.row_off = h->row_off[c];
            q.kdr = C(0);
            q.gx = C(0);
            q.rho_in = (C)((p.rho0 - 1.0) + 1.5 * p.g_x * (double)(h->nx + 1));
            q.rho_out = (C)((p.rho0 - 1.0) - 1.5 * p.g_x * (double)(h->nx + 1));
        }
        v[c] = q;
    }
    return v;
}

// Tile plan: narrow channels (nx <= 64) use full-width tiles of at most kThreads/nx (>= 4) rows;
// wide ones 32 x 8 tiles.  Row tiles are balanced: with ny >= 3 and a row target >= 4 every tile
// gets between 2 and the target rows (one-sided differences at a wall need the two rows next to
// it inside the tile or its halo), so a tile never holds more nodes than the CTA has threads.
void plan_tiles(lb_handle* h) {
    h->items.clear();
    h->item_begin.assign(h->n_ch + 1, 0);
    int maxEX = 0, maxEY = 0;
    for (int c = 0; c < h->n_ch; ++c) {
        h->item_begin[c] = (int)h->items.size();
        const int ny = h->ny[c];
        int nxt, nyt_target;
        if (h->nx <= kThreads / 4) { nxt = h->nx; nyt_target = kThreads / h->nx; }
        else { nxt = 32; nyt_target = kThreads / 32; }
        const int ntx = (h->nx + nxt - 1) / nxt;
        const int nty = (ny + nyt_target - 1) / nyt_target;
        for (int ty = 0; ty < nty; ++ty) {
            const int y0 = (int)((long long)ny * ty / nty), y1 = (int)((long long)ny * (ty + 1) / nty);
            for (int tx = 0; tx < ntx; ++tx) {
                WorkItem w{};
                w.ch = c;
                w.x0 = tx * nxt;
                w.nxt = (tx == ntx - 1) ? h->nx - w.x0 : nxt;
                if (ntx == 1) w.nxt = h->nx;
                w.y0 = y0;
                w.nyt = y1 - y0;
                h->items.push_back(w);
                const int EX = (w.nxt == h->nx) ? h->nx : w.nxt + 2;
                if (EX > maxEX) maxEX = EX;
                if (w.nyt + 2 > maxEY) maxEY = w.nyt + 2;
            }
        }
    }
    h->item_begin[h->n_ch] = (int)h->items.size();
    h->smem = (size_t)maxEX * maxEY * 2 * h->csize;
}

// cuTensorMapEncodeTiled through the runtime's driver entry point (no link against libcuda).
typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_fn() {
    static EncodeTiledFn fn = nullptr;
    static bool tried = false;
    if (!tried) {
        tried = true;
        void* f = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (EncodeTiledFn)f;
    }
    return fn;
}

// 3-D map over the 9 population planes of channel 0: dims (nx, ny, 9), box (W + 2 HP, 1, 9).
bool make_pop_map(const lb_handle* h, void* base, CUtensorMap* map) {
    EncodeTiledFn enc = encode_fn();
    if (!enc) return false;
    const bool bf = h->prec == LB_PREC_BF16;
    const cuuint64_t es = bf ? 2 : 4;
    const cuuint32_t hp = (cuuint32_t)(16 / es);
    cuuint64_t dims[3] = {(cuuint64_t)h->nx, (cuuint64_t)h->ny[0], 9};
    cuuint64_t strides[2] = {(cuuint64_t)h->nx * es, (cuuint64_t)h->P[0] * es};
    cuuint32_t box[3] = {(cuuint32_t)kMarchW + 2 * hp, 1, 9};
    cuuint32_t estr[3] = {1, 1, 1};
    CUresult r = enc(map, bf ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, base, dims, strides,
                     box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                     CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS;
}

// Row-march work items: strips of kMarchW columns cut into row ranges, at most one item per
// resident CTA (one wave: a partial second wave would double the kernel time for a few CTAs).
// Items are not equally long, because CTAs are not equally fast: the warp schedulers favour older
// warps, so the CTAs that arrive later on an SM take longer for the same rows (measured at
// 4096 x 4096 with equal items, per CTA rank on its SM: FP32 five ranks 246 ... 275 us; BF16
// eight ranks 182 ... 219 us), and an edge strip costs more per row than an interior one (its
// halo columns are patched from the other end; with pressure-driven ends it also applies the
// crossing corrections).  The model: block b, of rank k = b / n_sm (blocks fill the SMs rank by
// rank), runs at speed 1 + skew (R-1-k)/(R-1) for R CTAs per SM; strip j costs f_j per row (f for
// the two edge strips, 1 inside).  A bisection finds the smallest common duration T whose dealing
// needs at most R n_sm blocks; rows are then split in proportion to the blocks' speeds.  Two
// dealings:
//  - strip-major: each strip takes consecutive blocks until their speeds cover ny f_j / T;
//  - chunk-major: the edge strips first, the same way, then the interior strips share their row
//    boundaries -- row chunk c of every interior strip on consecutive blocks, T times the speed of
//    the slowest of them in rows -- so neighbouring strips march the same rows at the same time
//    and read each other's halo columns from L2 (with boundaries that differ between strips, BF16
//    re-reads 9 DRAM bytes per node of halo).  Both precisions are dealt chunk-major; strip-major
//    serves grids of one or two strips.
// Items keep at least 8 rows on average (at most ny / 8 per strip).
struct MarchModel {
    double skew, fedge;
    bool chunk_major;
};

// Constants measured at 4096 x 4096 (GLUPS of the whole step; repeated runs on one GPU):
//   FP32 (HBM-bound): chunk-major skew 0.12: 60.5 (0.08: 60.1, 0.16: 60.4, 0.2: 59.4, 0.3: 58.6)
//     against strip-major skew 0: 59.1 (strip-major with skew loses: 0.12 -> 55.5, the halo
//     re-reads); f = 1.2; pressure-driven ends f = 1.5 with the edge strips first 53.6 (last: 50.3;
//     strip-major 53.0); moving wall 59.1 (57.7); 8192 x 2048 58.2 (57.2); 2048 x 2048 52.6 (51.9).
//   BF16 (issue-bound): chunk-major skew 0.3: 75.4 (0.45: 75.1, 0.6: 74.0; with the edge strips on
//     the last blocks 74.0) against strip-major skew 0.3: 74.6-74.7 (strip-major skew 0 / 0.12 / 0.2 /
//     0.28 / 0.36 / 0.45 -> 73.7 / 75.2 / 75.6 / 75.9 / 76.1 / 73.6 on another GPU); f = 1.15;
//     pressure-driven ends f = 1.5 (65.55; strip-major 65.45; f = 1.3 / 1.6 / 1.9 strip-major ->
//     62.2 / 64.8 / 63.6).
static MarchModel march_model(int prec, bool gpbc) {
    if (prec == LB_PREC_BF16) return {0.30, gpbc ? 1.5 : 1.15, true};
    return {0.12, gpbc ? 1.5 : 1.2, true};
}

static std::vector<MarchItem> march_plan(int nx, int ny, int R, int nsm, MarchModel m) {
    const int strips = nx / kMarchW;
    const int slots = R * nsm;
    const int maxn = std::max(1, ny / 8);
    auto speed = [&](int b) {
        const int k = std::min(b / nsm, R - 1);
        return 1.0 + (R > 1 ? m.skew * (R - 1 - k) / (R - 1) : 0.0);
    };
    auto cost = [&](int s) { return (s == 0 || s == strips - 1) ? m.fedge : 1.0; };
    // the rows [0, ny) of one strip split in proportion to the weights w
    auto split = [&](std::vector<MarchItem>& out, int x0, const std::vector<double>& w) {
        double tot = 0.0;
        for (double v : w) tot += v;
        double cum = 0.0;
        int y = 0;
        for (size_t k = 0; k < w.size(); ++k) {
            cum += w[k];
            const int y1 = k + 1 == w.size() ? ny : (int)std::llround(ny * cum / tot);
            MarchItem it{};
            it.x0 = x0;
            it.y0 = y;
            it.y1 = y1;
            out.push_back(it);
            y = y1;
        }
    };
    // blocks from b on until their speeds cover ny f / T (at most maxn)
    auto take = [&](double T, int b, double f) {
        double acc = 0.0;
        int n = 0;
        while (n < maxn && acc < ny * f / T) acc += speed(b + n++);
        return n;
    };
    const bool cm = m.chunk_major && strips >= 3 && strips < slots;
    const int I = strips - 2;
    // blocks per strip (strip-major) or [edge 0, edge 1, chunks] (chunk-major) at duration T
    auto deal = [&](double T, std::vector<int>* out) {
        int b = 0;
        if (!cm) {
            for (int s = 0; s < strips; ++s) {
                const int n = strips >= slots ? 1 : take(T, b, cost(s));
                if (out) out->push_back(n);
                b += n;
            }
            return b;
        }
        for (int e = 0; e < 2; ++e) {
            const int n = take(T, b, m.fedge);
            if (out) out->push_back(n);
            b += n;
        }
        int C = 0;
        double acc = 0.0;
        while (C < maxn && acc < ny) acc += T * speed(b + (++C) * I - 1);
        if (out) out->push_back(C);
        return b + C * I;
    };
    double lo = 1e-9, hi = 4.0 * ny * std::max(1.0, m.fedge);  // deal(hi): one block per strip
    if (strips >= slots || deal(lo, nullptr) <= slots) {
        hi = strips >= slots ? hi : lo;
    } else {
        for (int it = 0; it < 100; ++it) {
            const double mid = 0.5 * (lo + hi);
            if (deal(mid, nullptr) <= slots) hi = mid;
            else lo = mid;
        }
    }
    std::vector<int> n;
    deal(hi, &n);
    std::vector<MarchItem> items;
    int b = 0;
    auto strip_items = [&](int s, int cnt) {
        std::vector<double> w(cnt);
        for (int k = 0; k < cnt; ++k) w[k] = speed(b + k);
        split(items, s * kMarchW, w);
        b += cnt;
    };
    if (!cm) {
        for (int s = 0; s < strips; ++s) strip_items(s, n[s]);
        return items;
    }
    strip_items(0, n[0]);
    strip_items(strips - 1, n[1]);
    const int C = n[2];
    std::vector<double> wc(C);
    for (int c = 0; c < C; ++c) wc[c] = speed(b + (c + 1) * I - 1);
    std::vector<MarchItem> chunk;
    split(chunk, 0, wc);
    for (int c = 0; c < C; ++c)
        for (int s = 1; s <= I; ++s) {
            MarchItem it = chunk[c];
            it.x0 = s * kMarchW;
            items.push_back(it);
        }
    return items;
}

lb_status plan_march(lb_handle* h) {
    h->march = false;
    if (h->n_ch != 1 || (h->prec != LB_PREC_F32 && h->prec != LB_PREC_BF16) || h->nx % kMarchW != 0 ||
        h->ny[0] < 16 || (h->flags & LB_GRID_TILE_ONLY) || h->scheme == 2 ||
        (h->scheme == 3 && (h->gpbc || h->moving)))
        return LB_OK;
    if (!make_pop_map(h, h->popA, &h->mapA) || !make_pop_map(h, h->popB, &h->mapB)) return LB_OK;
    h->mapA_buf = h->popA;
    h->mapB_buf = h->popB;
    int bps = 0, nsm = 0;
    cudaError_t e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, h->dev);
    if (e == cudaSuccess) {
        const bool bnd = h->gpbc || h->moving;
        if (h->prec == LB_PREC_F32) {
            if (h->scheme == 1) e = march_occupancy<float, float, 0, 0, 1>(&bps);
            else if (h->scheme == 3) e = h->smode ? march_occupancy<float, float, 1, 0, 3>(&bps) : march_occupancy<float, float, 0, 0, 3>(&bps);
            else if (h->gpbc) e = h->smode ? march_occupancy<float, float, 1, 1>(&bps) : march_occupancy<float, float, 0, 1>(&bps);
            else if (bnd) e = h->smode ? march_occupancy<float, float, 1, 2>(&bps) : march_occupancy<float, float, 0, 2>(&bps);
            else e = h->smode ? march_occupancy<float, float, 1>(&bps) : march_occupancy<float, float, 0>(&bps);
        } else {
            if (h->scheme == 1) e = march_occupancy<__nv_bfloat16, float, 0, 0, 1>(&bps);
            else if (h->scheme == 3) e = h->smode ? march_occupancy<__nv_bfloat16, float, 1, 0, 3>(&bps) : march_occupancy<__nv_bfloat16, float, 0, 0, 3>(&bps);
            else if (h->gpbc) e = h->smode ? march_occupancy<__nv_bfloat16, float, 1, 1>(&bps) : march_occupancy<__nv_bfloat16, float, 0, 1>(&bps);
            else if (bnd) e = h->smode ? march_occupancy<__nv_bfloat16, float, 1, 2>(&bps) : march_occupancy<__nv_bfloat16, float, 0, 2>(&bps);
            else e = h->smode ? march_occupancy<__nv_bfloat16, float, 1>(&bps) : march_occupancy<__nv_bfloat16, float, 0>(&bps);
        }
    }
    if (e != cudaSuccess) return cuda_fail(e, "lb_create: march occupancy");
    if (bps < 1) return LB_OK;
    const int slots = bps * nsm;
    const std::vector<MarchItem> items = march_plan(h->nx, h->ny[0], bps, nsm, march_model(h->prec, h->gpbc));
    LB_CK(cudaMalloc(&h->march_items_d, sizeof(MarchItem) * items.size()));
    LB_CK(cudaMemcpy(h->march_items_d, items.data(), sizeof(MarchItem) * items.size(), cudaMemcpyHostToDevice));
    h->n_march_items = (int)items.size();
    const int ib[2] = {0, h->n_march_items};
    LB_CK(cudaMalloc(&h->march_item_begin_d, sizeof(ib)));
    LB_CK(cudaMemcpy(h->march_item_begin_d, ib, sizeof(ib), cudaMemcpyHostToDevice));
    if ((int)h->items.size() < h->n_march_items) {  // the partials buffer serves both plans
        cudaFree(h->partials);
        h->partials = nullptr;
        LB_CK(cudaMalloc(&h->partials, 4 * sizeof(double) * h->n_march_items));
    }
    h->march_grid = std::min(h->n_march_items, slots);
    h->march = true;
    return LB_OK;
}

lb_status validate(const lb_grid* g, const lb_params* p, const lb_boundary* b) {
    if (!g || !p || !b) return fail(LB_EINVAL, "lb_create: null argument%s");
    if (g->n_channels < 1 || g->nx < 1 || !g->ny) return fail(LB_EINVAL, "lb_create: need n_channels >= 1, nx >= 1, ny%s");
    if (g->precision < 0 || g->precision > 4) return fail(LB_EINVAL, "lb_create: unknown precision%s");
    if (g->stress_mode < 0 || g->stress_mode > 1) return fail(LB_EINVAL, "lb_create: unknown stress_mode%s");
    if ((b->walls != LB_WALLS_BOUNCE_BACK && b->walls != LB_WALLS_COUETTE) ||
        (b->x_mode != LB_X_PERIODIC && b->x_mode != LB_X_GPBC))
        return fail(LB_EINVAL, "lb_create: walls must be LB_WALLS_BOUNCE_BACK or LB_WALLS_COUETTE and x_mode LB_X_PERIODIC or LB_X_GPBC%s");
    const bool gn = (g->flags & LB_GRID_GENERALIZED_NEWTONIAN) != 0, dv = (g->flags & LB_GRID_STRESS_DIVERGENCE) != 0;
    const bool rx = (g->flags & LB_GRID_RELAXATION_MODEL) != 0;
    if ((int)gn + (int)dv + (int)rx > 1)
        return fail(LB_EINVAL, "lb_create: choose one comparison scheme, or the relaxation-time extensions%s");
    if (rx && g->precision != LB_PREC_F64 && g->precision != LB_PREC_F32 && g->precision != LB_PREC_BF16)
        return fail(LB_EINVAL, "lb_create: the relaxation-time extensions run in FP64, FP32 or BF16%s");
    if ((gn || dv) && (g->stress_mode != 0 || b->walls != LB_WALLS_BOUNCE_BACK || b->x_mode != LB_X_PERIODIC))
        return fail(LB_EINVAL, "lb_create: the comparison schemes run with stress mode 0, periodic x and bounce-back walls%s");
    if ((gn || dv) && g->precision != LB_PREC_F64 && g->precision != LB_PREC_F32 && g->precision != LB_PREC_BF16)
        return fail(LB_EINVAL, "lb_create: the comparison schemes run in FP64, FP32 or BF16%s");
    for (int c = 0; c < g->n_channels; ++c) {
        if (g->ny[c] < 3) return fail(LB_EINVAL, "lb_create: ny must be >= 3%s");
        if ((long long)g->ny[c] * g->nx > (1ll << 40)) return fail(LB_EINVAL, "lb_create: channel too large%s");
        const lb_params& q = p[c];
        const double v[8] = {q.tau_lb, q.g_x, q.G_inf, q.tau0, q.theta, q.rho0, q.rho_pert_amp, 0.0};
        for (double x : v)
            if (std::isnan(x) || std::isinf(x)) return fail(LB_EINVAL, "lb_create: non-finite parameter%s");
        if (!(q.tau_lb > 0.5)) return fail(LB_EINVAL, "lb_create: tau_lb must be > 1/2%s");
        if (q.G_inf < 0 || q.tau0 < 0 || q.theta < 0) return fail(LB_EINVAL, "lb_create: G_inf, tau0, theta must be >= 0%s");
        if (!(q.gamma_c > 0)) return fail(LB_EINVAL, "lb_create: gamma_c must be > 0 (inf allowed)%s");
        if (!(q.rho0 > 0) || q.rho_pert_amp < 0 || q.rho_pert_amp >= 1)
            return fail(LB_EINVAL, "lb_create: need rho0 > 0 and 0 <= rho_pert_amp < 1%s");
    }
    return LB_OK;
}

template <typename T>
void free_dev(T*& p) {
    if (p) cudaFree((void*)p);
    p = nullptr;
}

void release(lb_handle* h) {
    if (!h) return;
    if (h->stream) cudaStreamSynchronize(h->stream);
    free_dev(h->popA); free_dev(h->popB); free_dev(h->drho); free_dev(h->sig3); free_dev(h->sig4); free_dev(h->snn); free_dev(h->phi);
    free_dev(h->uprev); free_dev(h->chan); free_dev(h->items_d); free_dev(h->item_begin_d);
    free_dev(h->partials); free_dev(h->mon_d); free_dev(h->status_d); free_dev(h->base_d); free_dev(h->P_d);
    free_dev(h->node_off_d); free_dev(h->ny_d); free_dev(h->gx_d); free_dev(h->fields); free_dev(h->fconv);
    free_dev(h->hstage);
    free_dev(h->ws_prm); free_dev(h->ws_row_off); free_dev(h->ws_rows); free_dev(h->ws_grid); free_dev(h->ws_scale);
    free_dev(h->march_items_d);
    free_dev(h->march_item_begin_d);
    free_dev(h->sweep_steps_d);
    free_dev(h->sweep_res_d);
    free_dev(h->sweep_order_d);
    free_dev(h->gcol);
    free_dev(h->gpart);
    free_dev(h->gcount);
    free_dev(h->done_count_d);
    if (h->status_h) cudaFreeHost(h->status_h);
    if (h->gx_h) cudaFreeHost(h->gx_h);
    if (h->mon_h) cudaFreeHost(h->mon_h);
    if (h->status_ev) cudaEventDestroy(h->status_ev);
    for (int k = 0; k < kDriveRing; ++k)
        if (h->gx_ev[k]) cudaEventDestroy(h->gx_ev[k]);
    for (int k = 0; k < 2; ++k)
        if (h->gexec[k]) cudaGraphExecDestroy(h->gexec[k]);
    if (h->cap_stream) cudaStreamDestroy(h->cap_stream);
    for (cudaStream_t q : h->gstreams) cudaStreamDestroy(q);
    for (cudaEvent_t q : h->gevents) cudaEventDestroy(q);
    if (h->fork_ev) cudaEventDestroy(h->fork_ev);
    if (h->sweep_gexec) cudaGraphExecDestroy(h->sweep_gexec);
    delete h;
}

lb_status ensure_hstage(lb_handle* h, size_t bytes) {
    if (h->hstage_bytes >= bytes) return LB_OK;
    free_dev(h->hstage);
    h->hstage_bytes = 0;
    LB_CK(cudaMalloc(&h->hstage, bytes));
    h->hstage_bytes = bytes;
    return LB_OK;
}

// Key of the stochastic rounding for one step (SplitMix64 finaliser of the handle seed and step).
uint32_t step_key(const lb_handle* h, long long step) {
    uint64_t z = h->params[0].seed + 0x632BE59BD9B4E019ull + (uint64_t)step * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return (uint32_t)(z ^ (z >> 31));
}

template <typename T, typename C>
StepArgs<T, C> base_args(lb_handle* h) {
    StepArgs<T, C> a{};
    a.pin = (const T*)h->popA;
    a.pout = (T*)h->popB;
    a.drho = (C*)h->drho;
    a.sig3 = (C*)h->sig3;
    a.sig4 = (C*)h->sig4;
    a.uprev = (C*)h->uprev;
    a.snn = (C*)h->snn;
    a.phi = (double*)h->phi;
    a.partials = h->partials;
    a.items = h->items_d;
    a.chan = (const ChanParams<C>*)h->chan;
    a.status = h->status_d;
    a.nx = h->nx;
    a.guard = (C)kGuard;
    a.gcol = (const C*)h->gcol;
    a.gny = h->gny;
    return a;
}

// Body forces and wall velocities: host -> pinned staging (mapped) -> channel table by one small
// kernel that reads the staging slot itself, stream-ordered.  The staging is a ring of
// kDriveRing slots, and a slot is reused only after the kernel that read it ran, so a host that
// changes the drive every step runs up to kDriveRing steps ahead of the device instead of waiting
// for the step before.
lb_status push_drive(lb_handle* h) {
    const int k = h->gx_slot;
    h->gx_slot = (k + 1) % kDriveRing;
    if (h->gx_pending[k]) LB_CK(cudaEventSynchronize(h->gx_ev[k]));
    double* st = h->gx_h + (size_t)k * 2 * h->n_ch;
    for (int c = 0; c < h->n_ch; ++c) {
        st[c] = h->params[c].g_x;
        st[h->n_ch + c] = h->u_wall[c];
    }
    const double* sd = h->gx_hd + (size_t)k * 2 * h->n_ch;
    if (h->csize == 8) k_apply_gx<double><<<(h->n_ch + 255) / 256, 256, 0, h->stream>>>((ChanParams<double>*)h->chan, h->gx_d, sd, h->n_ch, h->nx);
    else k_apply_gx<float><<<(h->n_ch + 255) / 256, 256, 0, h->stream>>>((ChanParams<float>*)h->chan, h->gx_d, sd, h->n_ch, h->nx);
    LB_CK(cudaGetLastError());
    LB_CK(cudaEventRecord(h->gx_ev[k], h->stream));  // the slot is read by the kernel above
    h->gx_pending[k] = true;
    return LB_OK;
}

// Under GPBC every step kernel needs the boundary columns of its input buffer.
template <typename T, typename C>
cudaError_t gpbc_columns(lb_handle* h) {
    if (!h->gpbc) return cudaSuccess;
    return launch_gpbc_columns<T, C>((const T*)h->popA, (const ChanParams<C>*)h->chan, (C*)h->gcol, h->n_ch, h->nx,
                                     h->gny, h->gpbc_max_ny, h->gpart, h->gcount, h->stream);
}

// The comparison schemes are instantiated for the three main precisions (T and C of one type, or
// BF16 storage with FP32 arithmetic); lb_create refuses them with the mixed diagnostic ones.
template <typename T, typename C>
constexpr bool kSchemeTypes = std::is_same<T, C>::value || std::is_same<T, __nv_bfloat16>::value;

template <typename T, typename C>
cudaError_t launch(lb_handle* h, const StepArgs<T, C>& a) {
    const int n = (int)h->items.size();
    if constexpr (kSchemeTypes<T, C>) {
        if (h->scheme == 3)
            return h->smode == 0 ? launch_step_tile<T, C, 0, 3>(a, n, h->smem, h->stream)
                                 : launch_step_tile<T, C, 1, 3>(a, n, h->smem, h->stream);
        if (h->scheme == 1) return launch_step_tile<T, C, 0, 1>(a, n, h->smem, h->stream);
        if (h->scheme == 2) {
            // stress divergence: Sigma^nN of every node of this step first, then the step (or the
            // fields pass) that differentiates it
            StepArgs<T, C> s = a;
            s.flags = F_SNN;
            cudaError_t e = launch_step_tile<T, C, 0, 2>(s, n, h->smem, h->stream);
            if (e != cudaSuccess) return e;
            StepArgs<T, C> b = a;
            b.flags |= F_DIV;
            return launch_step_tile<T, C, 0, 2>(b, n, h->smem, h->stream);
        }
    } else {
        if (h->scheme != 0) return cudaErrorNotSupported;
    }
    if (h->smode == 0) return launch_step_tile<T, C, 0>(a, n, h->smem, h->stream);
    return launch_step_tile<T, C, 1>(a, n, h->smem, h->stream);
}

// The row-march kernel's last CTA mirrors the status word into mapped host memory every step and,
// on monitor steps (F_RESID / F_MON), reduces the item partials into mon_d.
void march_monitor(lb_handle* h, int flags, MarchCtl& ctl) {
    const bool mon = (flags & (F_RESID | F_MON)) != 0;
    ctl.done_count = h->done_count_d;
    ctl.status_host = h->status_hd;
    ctl.mon = mon ? (double*)h->mon_d : nullptr;
    ctl.state_index = h->step;
    ctl.with_residual = (flags & F_RESID) ? 1 : 0;
}

// The row-march kernel takes plain steps (no fields output, no residual reduction).
template <typename T, typename C>
cudaError_t launch_march(lb_handle*, const StepArgs<T, C>&) { return cudaErrorNotSupported; }
template <>
cudaError_t launch_march<float, float>(lb_handle* h, const StepArgs<float, float>& a) {
    MarchCtl ctl{h->march_items_d, h->n_march_items, h->status_d, h->P[0], h->base[0], h->wait_ns};
    march_monitor(h, a.flags, ctl);
    const CUtensorMap& m = ((const void*)a.pin == h->mapA_buf) ? h->mapA : h->mapB;
    if (h->scheme == 1) return launch_step_march<float, float, 0, 0, 1>(m, a, ctl, h->march_grid, h->stream);
    if (h->scheme == 3)
        return h->smode ? launch_step_march<float, float, 1, 0, 3>(m, a, ctl, h->march_grid, h->stream)
                        : launch_step_march<float, float, 0, 0, 3>(m, a, ctl, h->march_grid, h->stream);
    if (h->gpbc)
        return h->smode ? launch_step_march<float, float, 1, 1>(m, a, ctl, h->march_grid, h->stream)
                        : launch_step_march<float, float, 0, 1>(m, a, ctl, h->march_grid, h->stream);
    if (h->moving)
        return h->smode ? launch_step_march<float, float, 1, 2>(m, a, ctl, h->march_grid, h->stream)
                        : launch_step_march<float, float, 0, 2>(m, a, ctl, h->march_grid, h->stream);
    return h->smode ? launch_step_march<float, float, 1>(m, a, ctl, h->march_grid, h->stream)
                    : launch_step_march<float, float, 0>(m, a, ctl, h->march_grid, h->stream);
}
template <>
cudaError_t launch_march<__nv_bfloat16, float>(lb_handle* h, const StepArgs<__nv_bfloat16, float>& a) {
    MarchCtl ctl{h->march_items_d, h->n_march_items, h->status_d, h->P[0], h->base[0], h->wait_ns};
    march_monitor(h, a.flags, ctl);
    const CUtensorMap& m = ((const void*)a.pin == h->mapA_buf) ? h->mapA : h->mapB;
    if (h->scheme == 1) return launch_step_march<__nv_bfloat16, float, 0, 0, 1>(m, a, ctl, h->march_grid, h->stream);
    if (h->scheme == 3)
        return h->smode ? launch_step_march<__nv_bfloat16, float, 1, 0, 3>(m, a, ctl, h->march_grid, h->stream)
                        : launch_step_march<__nv_bfloat16, float, 0, 0, 3>(m, a, ctl, h->march_grid, h->stream);
    if (h->gpbc)
        return h->smode ? launch_step_march<__nv_bfloat16, float, 1, 1>(m, a, ctl, h->march_grid, h->stream)
                        : launch_step_march<__nv_bfloat16, float, 0, 1>(m, a, ctl, h->march_grid, h->stream);
    if (h->moving)
        return h->smode ? launch_step_march<__nv_bfloat16, float, 1, 2>(m, a, ctl, h->march_grid, h->stream)
                        : launch_step_march<__nv_bfloat16, float, 0, 2>(m, a, ctl, h->march_grid, h->stream);
    return h->smode ? launch_step_march<__nv_bfloat16, float, 1>(m, a, ctl, h->march_grid, h->stream)
                    : launch_step_march<__nv_bfloat16, float, 0>(m, a, ctl, h->march_grid, h->stream);
}

constexpr int kGraphSteps = 32;  // steps per captured graph (even)

// Capture kGraphSteps plain steps (no velocity save, no residual, no stochastic rounding) starting
// from the current input buffer on the handle's private capture stream.
template <typename T, typename C>
lb_status capture_graph(lb_handle* h, int slot) {
    if (!h->cap_stream) LB_CK(cudaStreamCreateWithFlags(&h->cap_stream, cudaStreamNonBlocking));
    if (h->gexec[slot]) {
        LB_CK(cudaGraphExecDestroy(h->gexec[slot]));
        h->gexec[slot] = nullptr;
        h->gexec_pin[slot] = nullptr;
    }
    const void* pin = h->popA;
    cudaStream_t user = h->stream;
    h->stream = h->cap_stream;
    cudaError_t e = cudaStreamBeginCapture(h->cap_stream, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) {
        h->stream = user;
        return cuda_fail(e, "graph capture begin");
    }
    for (int k = 0; k < kGraphSteps && e == cudaSuccess; ++k) {
        StepArgs<T, C> a = base_args<T, C>(h);
        a.flags = (h->flags & LB_GRID_STORE_SIGMA) ? F_STORE_SIGMA : 0;
        e = gpbc_columns<T, C>(h);
        if (e == cudaSuccess) e = launch<T, C>(h, a);
        std::swap(h->popA, h->popB);
    }
    cudaGraph_t g = nullptr;
    cudaError_t e2 = cudaStreamEndCapture(h->cap_stream, &g);
    h->stream = user;
    if (e == cudaSuccess) e = e2;
    if (e == cudaSuccess) e = cudaGraphInstantiate(&h->gexec[slot], g, 0);
    if (g) cudaGraphDestroy(g);
    if (e != cudaSuccess) {
        h->gexec[slot] = nullptr;
        return cuda_fail(e, "graph capture");
    }
    h->gexec_pin[slot] = pin;
    return LB_OK;
}

template <typename T, typename C>
lb_status run_steps(lb_handle* h, long n) {
    const bool sr = (h->flags & LB_GRID_BF16_STOCHASTIC) && h->prec == LB_PREC_BF16;
    long s = 1;
    // Runs of plain steps replay a captured graph; the last two steps of the call (velocity save,
    // residual) are always launched one by one.
    if (!h->march && !sr && !(h->flags & LB_GRID_NO_GRAPH)) {
        while (n - s + 1 >= kGraphSteps + 2) {
            int slot = h->gexec_pin[0] == h->popA ? 0 : (h->gexec_pin[1] == h->popA ? 1 : -1);
            if (slot < 0) {
                slot = h->gexec_pin[0] ? 1 : 0;
                lb_status st = capture_graph<T, C>(h, slot);
                if (st != LB_OK) return st;
            }
            LB_CK(cudaGraphLaunch(h->gexec[slot], h->stream));
            ++h->graph_replays;
            h->step += kGraphSteps;
            s += kGraphSteps;
        }
    }
    for (; s <= n; ++s) {
        StepArgs<T, C> a = base_args<T, C>(h);
        int f = 0;
        if (h->flags & LB_GRID_STORE_SIGMA) f |= F_STORE_SIGMA;
        if (sr) f |= F_SR;
        a.sr_key = step_key(h, h->step);
        bool resid = false, mon = false;
        if (h->monitor_mode == LB_MONITOR_FLUX_MAX) {
            mon = (s == n);  // flux and max |u| of the last step's state: no saved velocity
            if (mon) f |= F_MON;
        } else {
            resid = mon = (s == n) && (h->uprev_state == h->step - 1);
            if (s >= n - 1) f |= F_SAVE_U;
            if (resid) f |= F_RESID;
        }
        a.flags = f;
        LB_CK((gpbc_columns<T, C>(h)));
        if (h->march) LB_CK((launch_march<T, C>(h, a)));
        else LB_CK((launch<T, C>(h, a)));
        if (mon) {
            if (!h->march) {  // (the row-march kernel's last CTA reduces its partials itself)
                k_reduce_residual<<<h->n_ch, 32, 0, h->stream>>>(h->partials, h->item_begin_d, h->status_d, h->mon_d,
                                                                 h->nx, h->step, resid ? 1 : 0);
                LB_CK(cudaGetLastError());
            }
            h->mon_state = h->step;
            h->mon_resid = resid;
        }
        if (f & F_SAVE_U) h->uprev_state = h->step;
        std::swap(h->popA, h->popB);
        ++h->step;
    }
    return LB_OK;
}

template <typename T, typename C>
lb_status fields_pass(lb_handle* h, C* fu, C* fs, C* fr) {
    StepArgs<T, C> a = base_args<T, C>(h);
    a.flags = F_FIELDS;
    a.fu = fu;
    a.fsig = fs;
    a.frho = fr;
    LB_CK((gpbc_columns<T, C>(h)));
    LB_CK((launch<T, C>(h, a)));
    return LB_OK;
}

lb_status poll_status(lb_handle* h, bool wait) {
    if (h->march) {  // the row-march kernel stores the status word into mapped host memory itself
        const int s = *(volatile const int*)h->status_h;
        if (s & 1) h->any_unstable = true;
        if (s & 2) h->any_timeout = true;
        return LB_OK;
    }
    if (h->status_pending) {
        cudaError_t q = wait ? cudaEventSynchronize(h->status_ev) : cudaEventQuery(h->status_ev);
        if (q == cudaSuccess) {
            h->status_pending = false;
            for (int c = 0; c < h->n_ch; ++c) {
                if (h->status_h[c] & 1) h->any_unstable = true;
                if (h->status_h[c] & 2) h->any_timeout = true;
            }
        } else if (q != cudaErrorNotReady) {
            return cuda_fail(q, "status event");
        }
    }
    return LB_OK;
}

lb_status request_status(lb_handle* h) {
    LB_CK(cudaMemcpyAsync(h->status_h, h->status_d, sizeof(int) * h->n_ch, cudaMemcpyDeviceToHost, h->stream));
    LB_CK(cudaEventRecord(h->status_ev, h->stream));
    h->status_pending = true;
    return LB_OK;
}

constexpr int kSweepNPT = 4;  // nodes per thread of the sweep kernel

// Channels of one width class (floor(log2 ny)) run in their own persistent launch with their own
// tuned configuration; the classes' launches run side by side on forked streams.
int width_class(int ny) {
    int k = 0;
    while ((2 << k) <= ny) ++k;
    return k;
}
bool sweep_fits(int ny_max, int nx, int nt, int cl) {
    const int rows = (ny_max + cl - 1) / cl;
    return (long long)rows * nx <= (long long)nt * kSweepNPT;
}
size_t sweep_smem(const lb_handle* h, int ny_max, int cl) {
    const int rows = (ny_max + cl - 1) / cl + 4;
    return (size_t)rows * h->nx * 2 * h->csize;
}
// Shared-memory resident variant: every CTA owns >= 3 rows (halo rows come from the neighbours),
// and its rows, halos and velocity rows fit the 227 KB of one CTA.
size_t sweep_smem_resident(const lb_handle* h, int ny_max, int cl) {
    const int rows = (ny_max + cl - 1) / cl;
    const size_t pops = ((size_t)2 * 9 * (rows + 6) * h->nx * h->tsize + 15) / 16 * 16;
    return pops + (size_t)(rows + 4) * h->nx * 2 * h->csize;
}
bool sweep_config_fits(const lb_handle* h, const SweepGroup& g, int var, int nt, int cl) {
    if (cl < 1 || cl > 16 || (nt != 128 && nt != 256) || !sweep_fits(g.ny_max, h->nx, nt, cl)) return false;
    if (var == 0) return sweep_smem(h, g.ny_max, cl) <= 200 * 1024;
    return g.ny_min / cl >= 3 && sweep_smem_resident(h, g.ny_max, cl) <= 227 * 1024;
}

template <typename T, typename C>
cudaError_t sweep_launch(lb_handle* h, const SweepGroup& g, int var, int nt, int cl, double tol, int check,
                         long long max_steps, cudaStream_t stream) {
    SweepArgs<T, C> a{};
    a.popA = (T*)h->popA;
    a.popB = (T*)h->popB;
    a.drho = (C*)h->drho;
    a.uprev = (C*)h->uprev;
    a.chan = (const ChanParams<C>*)h->chan;
    a.status = h->status_d;
    a.order = h->sweep_order_d + g.begin;
    a.steps_out = h->sweep_steps_d;
    a.res_out = h->sweep_res_d;
    a.nx = h->nx;
    a.check = check;
    a.max_steps = max_steps;
    a.tol = tol;
    a.sr = (h->flags & LB_GRID_BF16_STOCHASTIC) && h->prec == LB_PREC_BF16;
    a.sr_key = step_key(h, h->step + 0x5bd1e995ll);
    if (var == 1) {
        const size_t smem = sweep_smem_resident(h, g.ny_max, cl);
        if (h->nx == 4) {  // the 4-column channels of the batched sweep: width known at compile time
            if (nt == 128) return launch_sweep_smem<T, C, 128, kSweepNPT, 4>(a, g.count, cl, smem, stream);
            return launch_sweep_smem<T, C, 256, kSweepNPT, 4>(a, g.count, cl, smem, stream);
        }
        if (nt == 128) return launch_sweep_smem<T, C, 128, kSweepNPT>(a, g.count, cl, smem, stream);
        return launch_sweep_smem<T, C, 256, kSweepNPT>(a, g.count, cl, smem, stream);
    }
    const size_t smem = sweep_smem(h, g.ny_max, cl);
    if (h->nx == 4) {
        if (nt == 128) return launch_sweep<T, C, 128, kSweepNPT, 4>(a, g.count, cl, smem, stream);
        return launch_sweep<T, C, 256, kSweepNPT, 4>(a, g.count, cl, smem, stream);
    }
    if (nt == 128) return launch_sweep<T, C, 128, kSweepNPT>(a, g.count, cl, smem, stream);
    return launch_sweep<T, C, 256, kSweepNPT>(a, g.count, cl, smem, stream);
}

cudaError_t sweep_launch_any(lb_handle* h, const SweepGroup& g, int var, int nt, int cl, double tol, int check,
                             long long max_steps, cudaStream_t stream) {
    return with_types(h->prec, [&](auto tt, auto tc) -> cudaError_t {
        LB_TYPES(tt, tc);
        if constexpr (std::is_same<T, double>::value != std::is_same<C, double>::value) return cudaErrorNotSupported;
        else return sweep_launch<T, C>(h, g, var, nt, cl, tol, check, max_steps, stream);
    });
}

// Clusters of this configuration the device can hold at once (0: never launched).
int sweep_capacity(lb_handle* h, const SweepGroup& g, int var, int nt, int cl) {
    int n = 0;
    const cudaError_t e = with_types(h->prec, [&](auto tt, auto tc) -> cudaError_t {
        LB_TYPES(tt, tc);
        if constexpr (std::is_same<T, double>::value != std::is_same<C, double>::value) return cudaErrorNotSupported;
        else {
            if (var == 1) {
                const size_t smem = sweep_smem_resident(h, g.ny_max, cl);
                if (h->nx == 4)
                    return nt == 128 ? launch_sweep_smem_capacity<T, C, 128, kSweepNPT, 4>(cl, smem, &n)
                                     : launch_sweep_smem_capacity<T, C, 256, kSweepNPT, 4>(cl, smem, &n);
                return nt == 128 ? launch_sweep_smem_capacity<T, C, 128, kSweepNPT>(cl, smem, &n)
                                 : launch_sweep_smem_capacity<T, C, 256, kSweepNPT>(cl, smem, &n);
            }
            const size_t smem = sweep_smem(h, g.ny_max, cl);
            if (h->nx == 4)
                return nt == 128 ? launch_sweep_capacity<T, C, 128, kSweepNPT, 4>(cl, smem, &n)
                                 : launch_sweep_capacity<T, C, 256, kSweepNPT, 4>(cl, smem, &n);
            return nt == 128 ? launch_sweep_capacity<T, C, 128, kSweepNPT>(cl, smem, &n)
                             : launch_sweep_capacity<T, C, 256, kSweepNPT>(cl, smem, &n);
        }
    });
    if (e != cudaSuccess) {
        (void)cudaGetLastError();
        return 0;
    }
    return n;
}

// Stable channels, widest first (the longest-running clusters start first), split into width
// classes; a class keeps the configuration it was tuned (or set) with.
lb_status sweep_order(lb_handle* h, int* n_active, const std::vector<char>* only = nullptr) {
    std::vector<int> st(h->n_ch);
    LB_CK(cudaMemcpyAsync(st.data(), h->status_d, sizeof(int) * h->n_ch, cudaMemcpyDeviceToHost, h->stream));
    LB_CK(cudaStreamSynchronize(h->stream));
    std::vector<int> order;
    for (int c = 0; c < h->n_ch; ++c)
        if (st[c] == 0 && (!only || (*only)[c])) order.push_back(c);
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return h->ny[a] > h->ny[b]; });
    if (!h->sweep_order_d) {
        LB_CK(cudaMalloc(&h->sweep_order_d, sizeof(int) * h->n_ch));
        LB_CK(cudaMalloc(&h->sweep_steps_d, sizeof(long long) * h->n_ch));
        LB_CK(cudaMalloc(&h->sweep_res_d, sizeof(double) * h->n_ch));
    }
    if (!order.empty())
        LB_CK(cudaMemcpy(h->sweep_order_d, order.data(), sizeof(int) * order.size(), cudaMemcpyHostToDevice));
    std::vector<SweepGroup> groups;
    for (int k = 0; k < (int)order.size(); ++k) {
        const int ny = h->ny[order[k]];
        if (groups.empty() || width_class(ny) != groups.back().cls) {
            SweepGroup g;
            g.cls = width_class(ny);
            g.begin = k;
            g.ny_max = ny;
            for (const SweepGroup& old : h->sweep_groups)
                if (old.cls == g.cls) { g.var = old.var; g.nt = old.nt; g.cl = old.cl; g.tune_ms = old.tune_ms; }
            groups.push_back(g);
        }
        groups.back().count += 1;
        groups.back().ny_min = ny;
    }
    for (SweepGroup& g : groups) {
        // a kept configuration must still fit (it does when channels only leave); a class that has
        // lost half of its channels is tuned again (few clusters: the timing becomes per-step
        // latency instead of throughput), unless the configuration was fixed by the caller
        if (g.nt && !sweep_config_fits(h, g, g.var, g.nt, g.cl)) g.nt = 0;
        for (const SweepGroup& old : h->sweep_groups)
            if (old.cls == g.cls && g.nt && !h->sweep_fixed && 2 * g.count <= old.count) g.nt = 0;
    }
    h->sweep_groups = groups;
    *n_active = (int)order.size();
    return LB_OK;
}

// Autotuner: per width class, time a short sweep of that class alone (no channel can converge:
// tol < 0) for every (kernel, threads, cluster size) that fits, from the same saved state, and
// keep the fastest.  The state is restored.
lb_status sweep_tune(lb_handle* h, bool all) {
    const size_t pop_b = 9 * h->planes * h->tsize, dr_b = h->planes * h->csize, up_b = 2 * h->planes * h->csize;
    void* save = nullptr;
    LB_CK(cudaMalloc(&save, pop_b + dr_b + up_b));
    char* sv = (char*)save;
    auto restore = [&]() -> cudaError_t {
        cudaError_t e = cudaMemcpyAsync(h->popA, sv, pop_b, cudaMemcpyDeviceToDevice, h->stream);
        if (e == cudaSuccess) e = cudaMemcpyAsync(h->drho, sv + pop_b, dr_b, cudaMemcpyDeviceToDevice, h->stream);
        if (e == cudaSuccess) e = cudaMemcpyAsync(h->uprev, sv + pop_b + dr_b, up_b, cudaMemcpyDeviceToDevice, h->stream);
        return e;
    };
    cudaError_t e = cudaMemcpyAsync(sv, h->popA, pop_b, cudaMemcpyDeviceToDevice, h->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(sv + pop_b, h->drho, dr_b, cudaMemcpyDeviceToDevice, h->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(sv + pop_b + dr_b, h->uprev, up_b, cudaMemcpyDeviceToDevice, h->stream);
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (e == cudaSuccess) e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    bool none = false;
    for (SweepGroup& g : h->sweep_groups) {
        if (e != cudaSuccess) break;
        if (g.nt && !all) continue;
        double best = 1e300;
        for (int var : {0, 1})
            for (int nt : {128, 256})
                for (int cl : {1, 2, 4, 8, 16}) {
                    if (e != cudaSuccess || !sweep_config_fits(h, g, var, nt, cl)) continue;
                    if (sweep_capacity(h, g, var, nt, cl) < 1) continue;  // cannot be co-scheduled
                    float ms = 0.f;
                    bool launched = true;
                    for (int rep = 0; rep < 2 && e == cudaSuccess && launched; ++rep) {  // first run warms up
                        e = restore();
                        if (e == cudaSuccess) e = cudaEventRecord(e0, h->stream);
                        if (e == cudaSuccess) {
                            // a cluster shape the device cannot co-schedule is refused at launch (a
                            // configuration error that leaves the context usable): skip it
                            const cudaError_t le = sweep_launch_any(h, g, var, nt, cl, -1.0, 16, 256, h->stream);
                            if (le != cudaSuccess) {
                                launched = false;
                                (void)cudaGetLastError();
                            }
                        }
                        if (e == cudaSuccess) e = cudaEventRecord(e1, h->stream);
                        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
                        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
                    }
                    if (e == cudaSuccess && launched && ms < best) {
                        best = ms;
                        g.var = var;
                        g.nt = nt;
                        g.cl = cl;
                        g.tune_ms = ms;
                    }
                }
        if (best == 1e300) none = true;
    }
    if (e == cudaSuccess) e = restore();
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaFree(save);
    if (e != cudaSuccess || none) {
        for (SweepGroup& g : h->sweep_groups) g.nt = 0;
        if (e != cudaSuccess) return cuda_fail(e, "lb_run_until_steady: autotune");
        return fail(LB_ECUDA, "lb_run_until_steady: a channel is too wide for the sweep kernels, or no configuration could be launched%s");
    }
    return LB_OK;
}

// One persistent launch per width class on forked streams, joined back: captured once as a CUDA
// graph (on the handle's private capture stream) and replayed while the arguments and the class
// configurations stay the same.
lb_status sweep_run(lb_handle* h, double tol, int check, long long max_steps) {
    const size_t G = h->sweep_groups.size();
    const uint32_t key_sr = step_key(h, h->step + 0x5bd1e995ll);
    std::vector<double> key = {tol, (double)check, (double)max_steps, (double)key_sr};
    for (const SweepGroup& g : h->sweep_groups)
        for (int v : {g.begin, g.count, g.ny_min, g.ny_max, g.var, g.nt, g.cl}) key.push_back((double)v);
    if (!h->sweep_gexec || key != h->sweep_key) {
        if (h->sweep_gexec) {
            LB_CK(cudaGraphExecDestroy(h->sweep_gexec));
            h->sweep_gexec = nullptr;
        }
        if (!h->cap_stream) LB_CK(cudaStreamCreateWithFlags(&h->cap_stream, cudaStreamNonBlocking));
        if (!h->fork_ev) LB_CK(cudaEventCreateWithFlags(&h->fork_ev, cudaEventDisableTiming));
        while (h->gstreams.size() < G) {
            cudaStream_t q = nullptr;
            cudaEvent_t ev = nullptr;
            LB_CK(cudaStreamCreateWithFlags(&q, cudaStreamNonBlocking));
            h->gstreams.push_back(q);
            LB_CK(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
            h->gevents.push_back(ev);
        }
        cudaStream_t cap = h->cap_stream;
        cudaError_t e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
        if (e != cudaSuccess) return cuda_fail(e, "lb_run_until_steady: graph capture begin");
        e = cudaEventRecord(h->fork_ev, cap);
        for (size_t k = 0; k < G && e == cudaSuccess; ++k) {
            const SweepGroup& g = h->sweep_groups[k];
            e = cudaStreamWaitEvent(h->gstreams[k], h->fork_ev, 0);  // fork
            if (e != cudaSuccess) break;
            const cudaError_t el = sweep_launch_any(h, g, g.var, g.nt, g.cl, tol, check, max_steps, h->gstreams[k]);
            // join the forked stream whatever the launch did, so that no stream stays in capture
            e = cudaEventRecord(h->gevents[k], h->gstreams[k]);
            const cudaError_t ej = cudaStreamWaitEvent(cap, h->gevents[k], 0);
            if (e == cudaSuccess) e = ej;
            if (e == cudaSuccess) e = el;
        }
        cudaGraph_t graph = nullptr;
        const cudaError_t e2 = cudaStreamEndCapture(cap, &graph);
        if (e == cudaSuccess) e = e2;
        if (e == cudaSuccess) e = cudaGraphInstantiate(&h->sweep_gexec, graph, 0);
        if (graph) cudaGraphDestroy(graph);
        if (e != cudaSuccess) {
            h->sweep_gexec = nullptr;
            return cuda_fail(e, "lb_run_until_steady: graph capture");
        }
        h->sweep_key = key;
    }
    LB_CK(cudaGraphLaunch(h->sweep_gexec, h->stream));
    return LB_OK;
}

}  // namespace

extern "C" {

const char* lb_last_error(void) { return g_err; }

lb_status lb_run_until_steady(lb_handle* h, double tol, long check_every, long max_steps, long long* steps_out,
                              double* residual_out) {
    NvtxRange range("lb_run_until_steady");
    if (!h || check_every < 2 || (check_every & 1) || max_steps < check_every || std::isnan(tol))
        return fail(LB_EINVAL, "lb_run_until_steady: need an even check_every >= 2 and max_steps >= check_every%s");
    if (h->smode != 0) return fail(LB_EINVAL, "lb_run_until_steady: the sweep kernel implements stress mode 0%s");
    if (h->gpbc || h->moving)
        return fail(LB_EINVAL, "lb_run_until_steady: the sweep kernel implements periodic x and bounce-back walls only%s");
    if (h->scheme != 0)
        return fail(LB_EINVAL, "lb_run_until_steady: the sweep kernel implements the paper's model only (step the comparison schemes and the relaxation-time extensions with lb_step)%s");
    if (h->prec == LB_PREC_F64S_F32M || h->prec == LB_PREC_F32S_F64M)
        return fail(LB_EINVAL, "lb_run_until_steady: diagnostic precision mixes are not supported%s");
    // Segments of growing length (64, 256, 1024, ... check intervals): after each one the
    // converged channels drop out and the classes that lost half of their channels are tuned
    // again, so the last, slowest channels run with the shape of lowest per-step latency.  A
    // channel's first check interval in a segment only saves its velocity.
    const long long ms = (long long)((max_steps + check_every - 1) / check_every) * check_every;
    std::vector<long long> total(h->n_ch, -3);   // -3: not run (unstable before)
    std::vector<double> res(h->n_ch, NAN);
    std::vector<char> active(h->n_ch, 1);
    std::vector<long long> seg_steps(h->n_ch);
    std::vector<double> seg_res(h->n_ch);
    long long done = 0, seg = 64LL * check_every;
    lb_status st = LB_OK;
    bool first = true;
    while (done < ms) {
        int n_active = 0;
        st = sweep_order(h, &n_active, &active);
        if (st != LB_OK) return st;
        if (n_active == 0) break;
        bool untuned = false;
        for (const SweepGroup& g : h->sweep_groups) untuned |= g.nt == 0;
        if (untuned) {
            st = sweep_tune(h, false);
            if (st != LB_OK) return st;
        }
        const long long L = std::min(seg, ms - done);
        std::vector<long long> init(h->n_ch, -3);
        LB_CK(cudaMemcpy(h->sweep_steps_d, init.data(), sizeof(long long) * h->n_ch, cudaMemcpyHostToDevice));
        st = sweep_run(h, tol, (int)check_every, L);
        if (st != LB_OK) return st;
        LB_CK(cudaMemcpyAsync(seg_steps.data(), h->sweep_steps_d, sizeof(long long) * h->n_ch, cudaMemcpyDeviceToHost, h->stream));
        LB_CK(cudaMemcpyAsync(seg_res.data(), h->sweep_res_d, sizeof(double) * h->n_ch, cudaMemcpyDeviceToHost, h->stream));
        LB_CK(cudaStreamSynchronize(h->stream));
        for (int c = 0; c < h->n_ch; ++c) {
            if (!active[c] || seg_steps[c] == -3) {
                if (first && active[c]) active[c] = 0;   // unstable before the sweep
                continue;
            }
            res[c] = seg_res[c];
            if (seg_steps[c] >= 0) {                     // converged in this segment
                total[c] = done + seg_steps[c];
                active[c] = 0;
            } else if (seg_steps[c] == -2) {             // became unstable
                total[c] = -2;
                active[c] = 0;
            } else {
                total[c] = -1;
            }
        }
        done += L;
        seg *= 4;
        first = false;
    }
    for (int c = 0; c < h->n_ch; ++c) {
        if (steps_out) steps_out[c] = total[c] == -3 ? -2 : total[c];
        if (residual_out) residual_out[c] = res[c];
    }
    h->uprev_state = -10;
    h->mon_state = -1;
    return LB_OK;
}

lb_status lb_sweep_tune(lb_handle* h) {
    NvtxRange range("lb_sweep_tune");
    if (!h) return fail(LB_EINVAL, "lb_sweep_tune: null handle%s");
    if (h->smode != 0) return fail(LB_EINVAL, "lb_sweep_tune: the sweep kernel implements stress mode 0%s");
    if (h->gpbc || h->moving)
        return fail(LB_EINVAL, "lb_sweep_tune: the sweep kernel implements periodic x and bounce-back walls only%s");
    int n_active = 0;
    lb_status st = sweep_order(h, &n_active);
    if (st != LB_OK || n_active == 0) return st;
    h->sweep_fixed = false;
    return sweep_tune(h, true);
}

int lb_sweep_variant(const lb_handle* h) {
    if (!h || h->sweep_groups.empty()) return -1;
    return h->sweep_groups[0].var;
}

int lb_sweep_groups(const lb_handle* h, int* variant, int* threads, int* cluster, int* channels, int max_groups) {
    if (!h) return -1;
    const int G = (int)h->sweep_groups.size();
    for (int k = 0; k < G && k < max_groups; ++k) {
        const SweepGroup& g = h->sweep_groups[k];
        if (variant) variant[k] = g.var;
        if (threads) threads[k] = g.nt;
        if (cluster) cluster[k] = g.cl;
        if (channels) channels[k] = g.count;
    }
    return G;
}

lb_status lb_sweep_set_config(lb_handle* h, int variant, int threads, int cluster) {
    if (!h || (variant != 0 && variant != 1) || (threads != 128 && threads != 256))
        return fail(LB_EINVAL, "lb_sweep_set_config: variant 0/1 and threads 128/256%s");
    if (h->smode != 0 || h->gpbc || h->moving) return fail(LB_EINVAL, "lb_sweep_set_config: not a sweep handle%s");
    int n_active = 0;
    lb_status st = sweep_order(h, &n_active);
    if (st != LB_OK) return st;
    for (const SweepGroup& g : h->sweep_groups)
        if (!sweep_config_fits(h, g, variant, threads, cluster) || sweep_capacity(h, g, variant, threads, cluster) < 1)
            return fail(LB_EINVAL, "lb_sweep_set_config: configuration does not fit these channels%s");
    for (SweepGroup& g : h->sweep_groups) {
        g.var = variant;
        g.nt = threads;
        g.cl = cluster;
        g.tune_ms = 0.0;
    }
    h->sweep_fixed = true;
    return LB_OK;
}

lb_status lb_sweep_config(lb_handle* h, int* threads, int* cluster, double* tune_ms) {
    if (!h) return fail(LB_EINVAL, "lb_sweep_config: null handle%s");
    const SweepGroup* g = h->sweep_groups.empty() ? nullptr : &h->sweep_groups[0];
    if (threads) *threads = g ? g->nt : 0;
    if (cluster) *cluster = g ? g->cl : 0;
    if (tune_ms) {
        double t = 0.0;
        for (const SweepGroup& q : h->sweep_groups) t += q.tune_ms;
        *tune_ms = t;
    }
    return LB_OK;
}

const char* lb_strerror(lb_status s) {
    switch (s) {
        case LB_OK: return "ok";
        case LB_EINVAL: return "invalid argument";
        case LB_ENOMEM: return "out of memory";
        case LB_ECUDA: return "CUDA error";
        case LB_EUNSTABLE: return "channel unstable";
        case LB_ETIMEOUT: return "device wait timed out";
        case LB_ESTATE: return "state not available";
    }
    return "unknown status";
}

lb_status lb_create(const lb_grid* grid, const lb_params* params, const lb_boundary* boundary, void* cuda_stream,
                    lb_handle** out) {
    if (!out) return fail(LB_EINVAL, "lb_create: out is null%s");
    *out = nullptr;
    lb_status st = validate(grid, params, boundary);
    if (st != LB_OK) return st;
    lb_handle* h = new (std::nothrow) lb_handle();
    if (!h) return fail(LB_ENOMEM, "lb_create: host allocation%s");
    auto bail = [&](lb_status s) { release(h); return s; };
    cudaGetDevice(&h->dev);
    h->stream = (cudaStream_t)cuda_stream;
    h->n_ch = grid->n_channels;
    h->nx = grid->nx;
    h->prec = grid->precision;
    h->smode = grid->stress_mode;
    h->flags = grid->flags;
    h->scheme = (grid->flags & LB_GRID_GENERALIZED_NEWTONIAN) ? 1 : ((grid->flags & LB_GRID_STRESS_DIVERGENCE) ? 2 : 0);
    if (grid->flags & LB_GRID_RELAXATION_MODEL) h->scheme = 3;
    h->tsize = with_types(h->prec, [](auto tt, auto tc) { LB_TYPES(tt, tc); (void)sizeof(C); return sizeof(T); });
    h->csize = with_types(h->prec, [](auto tt, auto tc) { LB_TYPES(tt, tc); (void)sizeof(T); return sizeof(C); });
    h->ny.assign(grid->ny, grid->ny + h->n_ch);
    h->params.assign(params, params + h->n_ch);
    h->beta_rho.assign(h->n_ch, 0.0);
    h->rho_ref.assign(h->n_ch, 1.0);
    h->tau_f.assign(h->n_ch, 0.0);
    h->P.resize(h->n_ch); h->base.resize(h->n_ch); h->node_off.resize(h->n_ch);
    long long acc = 0, nodes = 0;
    for (int c = 0; c < h->n_ch; ++c) {
        const long long n = (long long)h->nx * h->ny[c];
        h->P[c] = (n + 63) / 64 * 64;
        h->base[c] = acc;
        h->node_off[c] = nodes;
        acc += h->P[c];
        nodes += n;
    }
    h->planes = acc;
    h->nodes = nodes;
    h->gpbc = boundary->x_mode == LB_X_GPBC;
    h->moving = boundary->walls == LB_WALLS_COUETTE;
    h->u_wall.assign(h->n_ch, 0.0);
    h->row_off.resize(h->n_ch);
    for (int c = 0; c < h->n_ch; ++c) {
        h->row_off[c] = h->gny;
        h->gny += h->ny[c];
    }
    plan_tiles(h);

    auto dmalloc = [&](void** p, size_t bytes) -> cudaError_t { return cudaMalloc(p, bytes < 16 ? 16 : bytes); };
    cudaError_t e;
#define LB_ALLOC(ptr, bytes)                                                   \
    do {                                                                       \
        e = dmalloc((void**)&(ptr), (bytes));                                  \
        if (e != cudaSuccess) return bail(cuda_fail(e, "lb_create: cudaMalloc")); \
    } while (0)
    LB_ALLOC(h->popA, 9 * h->planes * h->tsize);
    LB_ALLOC(h->popB, 9 * h->planes * h->tsize);
    LB_ALLOC(h->drho, h->planes * h->csize);
    if (h->smode == 1) LB_ALLOC(h->sig3, 3 * h->planes * h->csize);
    if (h->scheme == 2) LB_ALLOC(h->snn, 3 * h->planes * h->csize);
    if (h->scheme == 3) LB_ALLOC(h->phi, h->planes * sizeof(double));  // FP64 in every precision
    if (h->flags & LB_GRID_STORE_SIGMA) LB_ALLOC(h->sig4, 4 * h->planes * h->csize);
    LB_ALLOC(h->uprev, 2 * h->planes * h->csize);
    LB_ALLOC(h->chan, h->n_ch * (h->csize == 8 ? sizeof(ChanParams<double>) : sizeof(ChanParams<float>)));
    LB_ALLOC(h->items_d, h->items.size() * sizeof(WorkItem));
    LB_ALLOC(h->item_begin_d, (h->n_ch + 1) * sizeof(int));
    LB_ALLOC(h->partials, 4 * h->items.size() * sizeof(double));
    LB_ALLOC(h->mon_d, 4 * h->n_ch * sizeof(double));
    LB_ALLOC(h->status_d, h->n_ch * sizeof(int));
    LB_ALLOC(h->base_d, h->n_ch * sizeof(long long));
    LB_ALLOC(h->P_d, h->n_ch * sizeof(long long));
    LB_ALLOC(h->node_off_d, h->n_ch * sizeof(long long));
    LB_ALLOC(h->ny_d, h->n_ch * sizeof(int));
    LB_ALLOC(h->gx_d, 2 * h->n_ch * sizeof(double));
    LB_ALLOC(h->done_count_d, sizeof(unsigned));
    if (h->gpbc) {
        for (int c = 0; c < h->n_ch; ++c) h->gpbc_max_ny = std::max(h->gpbc_max_ny, h->ny[c]);
        const size_t rb = ((size_t)h->gpbc_max_ny + 255) / 256;
        LB_ALLOC(h->gcol, (6 * (size_t)h->gny + 2 * h->n_ch) * h->csize);
        LB_ALLOC(h->gpart, 2 * h->n_ch * rb * sizeof(double));
        LB_ALLOC(h->gcount, 2 * h->n_ch * sizeof(unsigned));
    }
#undef LB_ALLOC
    e = cudaHostAlloc((void**)&h->status_h, h->n_ch * sizeof(int), cudaHostAllocMapped);
    if (e == cudaSuccess) e = cudaHostGetDevicePointer((void**)&h->status_hd, h->status_h, 0);
    if (e != cudaSuccess) return bail(cuda_fail(e, "lb_create: cudaHostAlloc (mapped)"));
    std::memset(h->status_h, 0, h->n_ch * sizeof(int));
    e = cudaHostAlloc((void**)&h->gx_h, (size_t)kDriveRing * 2 * h->n_ch * sizeof(double), cudaHostAllocMapped);
    if (e == cudaSuccess) e = cudaHostGetDevicePointer((void**)&h->gx_hd, h->gx_h, 0);
    if (e == cudaSuccess) e = cudaHostAlloc((void**)&h->mon_h, 4 * (size_t)h->n_ch * sizeof(double), cudaHostAllocMapped);
    if (e == cudaSuccess) e = cudaHostGetDevicePointer((void**)&h->mon_hd, h->mon_h, 0);
    if (e != cudaSuccess) return bail(cuda_fail(e, "lb_create: cudaHostAlloc (mapped)"));
    e = cudaEventCreateWithFlags(&h->status_ev, cudaEventDisableTiming);
    for (int k = 0; k < kDriveRing && e == cudaSuccess; ++k) e = cudaEventCreateWithFlags(&h->gx_ev[k], cudaEventDisableTiming);
    if (e != cudaSuccess) return bail(cuda_fail(e, "lb_create: cudaEventCreate"));

    // tables (synchronous copies: creation is not on the hot path)
    std::vector<double> gx(2 * h->n_ch, 0.0);
    std::vector<InitChan> ic(h->n_ch);
    for (int c = 0; c < h->n_ch; ++c) {
        gx[c] = h->params[c].g_x;
        const double half = 1.5 * h->params[c].g_x * (double)(h->nx + 1);
        ic[c] = InitChan{h->base[c], h->P[c], h->ny[c], h->gpbc ? 1 : 0, h->params[c].rho0, h->params[c].rho_pert_amp,
                         h->params[c].seed, h->params[c].rho0 + half, h->params[c].rho0 - half};
    }
    InitChan* ic_d = nullptr;
    e = cudaMalloc(&ic_d, sizeof(InitChan) * h->n_ch);
    if (e != cudaSuccess) return bail(cuda_fail(e, "lb_create: cudaMalloc"));
    bool ok = true;
    ok &= cudaMemcpy(ic_d, ic.data(), sizeof(InitChan) * h->n_ch, cudaMemcpyHostToDevice) == cudaSuccess;
    if (h->csize == 8) {
        auto v = make_chan<double>(h);
        ok &= cudaMemcpy(h->chan, v.data(), sizeof(v[0]) * v.size(), cudaMemcpyHostToDevice) == cudaSuccess;
    } else {
        auto v = make_chan<float>(h);
        ok &= cudaMemcpy(h->chan, v.data(), sizeof(v[0]) * v.size(), cudaMemcpyHostToDevice) == cudaSuccess;
    }
    ok &= cudaMemcpy(h->items_d, h->items.data(), sizeof(WorkItem) * h->items.size(), cudaMemcpyHostToDevice) == cudaSuccess;
    ok &= cudaMemcpy(h->item_begin_d, h->item_begin.data(), sizeof(int) * (h->n_ch + 1), cudaMemcpyHostToDevice) == cudaSuccess;
    ok &= cudaMemcpy(h->base_d, h->base.data(), sizeof(long long) * h->n_ch, cudaMemcpyHostToDevice) == cudaSuccess;
    ok &= cudaMemcpy(h->P_d, h->P.data(), sizeof(long long) * h->n_ch, cudaMemcpyHostToDevice) == cudaSuccess;
    ok &= cudaMemcpy(h->node_off_d, h->node_off.data(), sizeof(long long) * h->n_ch, cudaMemcpyHostToDevice) == cudaSuccess;
    ok &= cudaMemcpy(h->ny_d, h->ny.data(), sizeof(int) * h->n_ch, cudaMemcpyHostToDevice) == cudaSuccess;
    ok &= cudaMemcpy(h->gx_d, gx.data(), sizeof(double) * 2 * h->n_ch, cudaMemcpyHostToDevice) == cudaSuccess;
    ok &= cudaMemsetAsync(h->status_d, 0, sizeof(int) * h->n_ch, h->stream) == cudaSuccess;
    if (h->gcount) ok &= cudaMemsetAsync(h->gcount, 0, 2 * h->n_ch * sizeof(unsigned), h->stream) == cudaSuccess;
    ok &= cudaMemsetAsync(h->done_count_d, 0, sizeof(unsigned), h->stream) == cudaSuccess;
    ok &= cudaMemsetAsync(h->uprev, 0, 2 * h->planes * h->csize, h->stream) == cudaSuccess;
    ok &= cudaMemsetAsync(h->popB, 0, 9 * h->planes * h->tsize, h->stream) == cudaSuccess;
    if (h->sig4) ok &= cudaMemsetAsync(h->sig4, 0, 4 * h->planes * h->csize, h->stream) == cudaSuccess;
    if (h->phi) ok &= cudaMemsetAsync(h->phi, 0, h->planes * sizeof(double), h->stream) == cudaSuccess;
    if (!ok) { cudaFree(ic_d); return bail(cuda_fail(cudaGetLastError(), "lb_create: table upload")); }
    long long maxn = 0;
    for (int c = 0; c < h->n_ch; ++c) maxn = std::max(maxn, (long long)h->nx * h->ny[c]);
    dim3 g(grid_for(maxn), h->n_ch);
    with_types(h->prec, [&](auto tt, auto tc) {
        LB_TYPES(tt, tc);
        k_init<T, C><<<g, 256, 0, h->stream>>>((T*)h->popA, (C*)h->drho, (C*)h->sig3, ic_d, h->nx, h->smode);
        return 0;
    });
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    cudaFree(ic_d);
    if (e != cudaSuccess) return bail(cuda_fail(e, "lb_create: init kernel"));
    st = plan_march(h);
    if (st != LB_OK) return bail(st);
    *out = h;
    return LB_OK;
}

void lb_destroy(lb_handle* h) { release(h); }

lb_status lb_set_relaxation_model(lb_handle* h, int channel, double beta_rho, double rho_ref, double tau_f) {
    if (!h || channel < -1 || channel >= h->n_ch || !std::isfinite(beta_rho) || !std::isfinite(rho_ref) ||
        !(rho_ref > 0.0) || !std::isfinite(tau_f) || tau_f < 0.0)
        return fail(LB_EINVAL, "lb_set_relaxation_model: bad handle, channel or parameter%s");
    if (h->scheme != 3) return fail(LB_EINVAL, "lb_set_relaxation_model: the handle was created without LB_GRID_RELAXATION_MODEL%s");
    for (int c = 0; c < h->n_ch; ++c)
        if (channel < 0 || c == channel) {
            h->beta_rho[c] = beta_rho;
            h->rho_ref[c] = rho_ref;
            h->tau_f[c] = tau_f;
        }
    // the whole channel table again (its body forces and wall velocities are the host's current
    // ones), after the work already queued that reads the old table
    LB_CK(cudaStreamSynchronize(h->stream));
    if (h->csize == 8) {
        auto v = make_chan<double>(h);
        LB_CK(cudaMemcpy(h->chan, v.data(), sizeof(v[0]) * v.size(), cudaMemcpyHostToDevice));
    } else {
        auto v = make_chan<float>(h);
        LB_CK(cudaMemcpy(h->chan, v.data(), sizeof(v[0]) * v.size(), cudaMemcpyHostToDevice));
    }
    return LB_OK;
}

lb_status lb_set_wait_limit(lb_handle* h, double seconds) {
    if (!h || !(seconds >= 0.0) || seconds > 60.0) return fail(LB_EINVAL, "lb_set_wait_limit: need 0 <= seconds <= 60%s");
    h->wait_ns = (unsigned long long)(seconds * 1e9);
    return LB_OK;
}

long lb_step_count(const lb_handle* h) { return h ? h->step : -1; }
int lb_uses_row_march(const lb_handle* h) { return (h && h->march) ? 1 : 0; }

int lb_row_march_plan(int nx, int ny, int ctas_per_sm, int n_sm, int precision, int gpbc, int* items, int max_items) {
    if (nx <= 0 || nx % kMarchW != 0 || ny < 16 || ctas_per_sm < 1 || n_sm < 1 || max_items < 0 ||
        (precision != LB_PREC_F32 && precision != LB_PREC_BF16))
        return -LB_EINVAL;
    const std::vector<MarchItem> v = march_plan(nx, ny, ctas_per_sm, n_sm, march_model(precision, gpbc != 0));
    if (items) {
        if ((int)v.size() > max_items) return -LB_EINVAL;
        for (size_t i = 0; i < v.size(); ++i) {
            items[3 * i] = v[i].x0;
            items[3 * i + 1] = v[i].y0;
            items[3 * i + 2] = v[i].y1;
        }
    }
    return (int)v.size();
}
long lb_graph_replays(const lb_handle* h) { return h ? h->graph_replays : -1; }
size_t lb_num_nodes(const lb_handle* h) { return h ? (size_t)h->nodes : 0; }

lb_status lb_step(lb_handle* h, long n) {
    NvtxRange range("lb_step");
    if (!h || n < 0) return fail(LB_EINVAL, "lb_step: bad handle or n%s");
    lb_status st = poll_status(h, false);
    if (st != LB_OK) return st;
    if (h->any_timeout) return fail(LB_ETIMEOUT, "lb_step: a device-side wait timed out earlier%s");
    if (n == 0) return h->any_unstable ? LB_EUNSTABLE : LB_OK;
    st = with_types(h->prec, [&](auto tt, auto tc) { LB_TYPES(tt, tc); return run_steps<T, C>(h, n); });
    if (st != LB_OK) return st;
    if (!h->march && !h->status_pending) {
        st = request_status(h);
        if (st != LB_OK) return st;
    }
    return h->any_unstable ? LB_EUNSTABLE : LB_OK;
}

lb_status lb_get_fields(lb_handle* h, void* u, void* sigma, void* rho, int out_dtype, int on_device) {
    if (!h || (out_dtype != 0 && out_dtype != 1)) return fail(LB_EINVAL, "lb_get_fields: bad handle or dtype%s");
    if (!u && !sigma && !rho) return LB_OK;
    const long long N = h->nodes;
    if (!h->fields) LB_CK(cudaMalloc(&h->fields, 7 * N * h->csize));
    char* base = (char*)h->fields;
    void* fu = base;
    void* fs = base + 2 * N * h->csize;
    void* fr = base + 6 * N * h->csize;
    lb_status st;
    st = with_types(h->prec, [&](auto tt, auto tc) { LB_TYPES(tt, tc); return fields_pass<T, C>(h, (C*)fu, (C*)fs, (C*)fr); });
    if (st != LB_OK) return st;
    const size_t osize = out_dtype == 0 ? 8 : 4;
    const void* src = h->fields;
    if (osize != h->csize) {
        if (!h->fconv) LB_CK(cudaMalloc(&h->fconv, 7 * N * 8));
        if (h->csize == 8) k_convert<double, float><<<grid_for(7 * N), 256, 0, h->stream>>>((const double*)h->fields, (float*)h->fconv, 7 * N);
        else k_convert<float, double><<<grid_for(7 * N), 256, 0, h->stream>>>((const float*)h->fields, (double*)h->fconv, 7 * N);
        LB_CK(cudaGetLastError());
        src = h->fconv;
    }
    const cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    const char* s = (const char*)src;
    if (u) LB_CK(cudaMemcpyAsync(u, s, 2 * N * osize, kind, h->stream));
    if (sigma) LB_CK(cudaMemcpyAsync(sigma, s + 2 * N * osize, 4 * N * osize, kind, h->stream));
    if (rho) LB_CK(cudaMemcpyAsync(rho, s + 6 * N * osize, N * osize, kind, h->stream));
    if (!on_device) LB_CK(cudaStreamSynchronize(h->stream));
    return LB_OK;
}

lb_status lb_monitor(lb_handle* h, double* out) {
    if (!h || !out) return fail(LB_EINVAL, "lb_monitor: null argument%s");
    if (h->mon_state < 0) return fail(LB_ESTATE, "lb_monitor: no monitor evaluated yet (run lb_step with n >= 2)%s");
    k_copy_to_host<<<1, 128, 0, h->stream>>>(h->mon_d, h->mon_hd, 4 * h->n_ch);
    LB_CK(cudaGetLastError());
    LB_CK(cudaStreamSynchronize(h->stream));
    std::memcpy(out, h->mon_h, 4 * h->n_ch * sizeof(double));
    return LB_OK;
}

lb_status lb_monitor_async(lb_handle* h, double* out) {
    if (!h || !out) return fail(LB_EINVAL, "lb_monitor_async: null argument%s");
    if (h->mon_state < 0) return fail(LB_ESTATE, "lb_monitor_async: no monitor evaluated yet (run lb_step with n >= 2)%s");
    // pinned host memory mapped into the device's address space (what cudaHostAlloc and
    // torch's pin_memory give under unified addressing): a one-block kernel stores the values
    // there; anything else (device memory, pageable host memory) takes a stream-ordered copy
    cudaPointerAttributes at{};
    if (cudaPointerGetAttributes(&at, out) == cudaSuccess && at.type == cudaMemoryTypeHost && at.devicePointer) {
        k_copy_to_host<<<1, 128, 0, h->stream>>>(h->mon_d, (double*)at.devicePointer, 4 * h->n_ch);
        LB_CK(cudaGetLastError());
    } else {
        (void)cudaGetLastError();
        LB_CK(cudaMemcpyAsync(out, h->mon_d, 4 * h->n_ch * sizeof(double), cudaMemcpyDefault, h->stream));
    }
    return LB_OK;
}

lb_status lb_set_monitor_mode(lb_handle* h, int mode) {
    if (!h || (mode != LB_MONITOR_RESIDUAL && mode != LB_MONITOR_FLUX_MAX))
        return fail(LB_EINVAL, "lb_set_monitor_mode: bad handle or mode%s");
    h->monitor_mode = mode;
    return LB_OK;
}

lb_status lb_residual(lb_handle* h, double* r) {
    if (!h || !r) return fail(LB_EINVAL, "lb_residual: null argument%s");
    if (h->mon_state >= 0 && !h->mon_resid)
        return fail(LB_ESTATE, "lb_residual: the last monitor evaluation had no residual (LB_MONITOR_FLUX_MAX)%s");
    std::vector<double> m(4 * (size_t)h->n_ch);
    lb_status st = lb_monitor(h, m.data());
    if (st != LB_OK) return st;
    for (int c = 0; c < h->n_ch; ++c) r[c] = m[4 * c];
    return LB_OK;
}

lb_status lb_set_body_force(lb_handle* h, int channel, double g_x) {
    if (!h || channel < -1 || channel >= h->n_ch || std::isnan(g_x) || std::isinf(g_x))
        return fail(LB_EINVAL, "lb_set_body_force: bad argument%s");
    for (int c = 0; c < h->n_ch; ++c)
        if (channel < 0 || c == channel) h->params[c].g_x = g_x;
    return push_drive(h);
}

lb_status lb_set_wall_velocity(lb_handle* h, int channel, double u_wall) {
    if (!h || channel < -1 || channel >= h->n_ch || std::isnan(u_wall) || std::isinf(u_wall))
        return fail(LB_EINVAL, "lb_set_wall_velocity: bad argument%s");
    if (!h->moving) return fail(LB_EINVAL, "lb_set_wall_velocity: the handle has no moving wall%s");
    for (int c = 0; c < h->n_ch; ++c)
        if (channel < 0 || c == channel) h->u_wall[c] = u_wall;
    return push_drive(h);
}

// The start state of every channel from device fields in node order (u [node][2], rho, drho or
// nullptr): equilibrium populations of (rho, u - f/(2 rho)), delta rho, zero carried stress.
static lb_status set_fields_dev(lb_handle* h, const double* su, const double* sr, const double* sd) {
    long long maxn = 0;
    for (int c = 0; c < h->n_ch; ++c) maxn = std::max(maxn, (long long)h->nx * h->ny[c]);
    dim3 g(grid_for(maxn), h->n_ch);
    with_types(h->prec, [&](auto tt, auto tc) {
        LB_TYPES(tt, tc);
        k_set_fields<T, C><<<g, 256, 0, h->stream>>>((T*)h->popA, (C*)h->drho, (C*)h->sig3, su, sr, sd,
                                                     h->base_d, h->P_d, h->node_off_d, h->ny_d, h->gx_d, h->nx, h->smode,
                                                     h->gpbc ? 1 : 0);
        return 0;
    });
    LB_CK(cudaGetLastError());
    if (h->phi) LB_CK(cudaMemsetAsync(h->phi, 0, h->planes * sizeof(double), h->stream));  // fluidity unset
    LB_CK(cudaStreamSynchronize(h->stream));
    h->uprev_state = -10;
    return LB_OK;
}

lb_status lb_set_fields(lb_handle* h, const double* u, const double* rho, const double* drho) {
    if (!h || !u || !rho) return fail(LB_EINVAL, "lb_set_fields: null argument%s");
    const long long N = h->nodes;
    lb_status st = ensure_hstage(h, (size_t)N * 4 * sizeof(double));
    if (st != LB_OK) return st;
    double* su = (double*)h->hstage;
    double* sr = su + 2 * N;
    double* sd = su + 3 * N;
    LB_CK(cudaMemcpyAsync(su, u, 2 * N * sizeof(double), cudaMemcpyHostToDevice, h->stream));
    LB_CK(cudaMemcpyAsync(sr, rho, N * sizeof(double), cudaMemcpyHostToDevice, h->stream));
    if (drho) LB_CK(cudaMemcpyAsync(sd, drho, N * sizeof(double), cudaMemcpyHostToDevice, h->stream));
    return set_fields_dev(h, su, sr, drho ? sd : nullptr);
}

// Learned warm start: the closed-form steady profile of every channel (current parameters) on its
// rows and on the network grid, with the per-field scales.
static lb_status ws_closed_form(lb_handle* h) {
    if (!h->ws_prm) {
        LB_CK(cudaMalloc(&h->ws_prm, sizeof(WsChan) * h->n_ch));
        LB_CK(cudaMalloc(&h->ws_row_off, sizeof(int) * h->n_ch));
        LB_CK(cudaMalloc(&h->ws_rows, sizeof(double) * 3 * (size_t)h->gny));
        LB_CK(cudaMalloc(&h->ws_grid, sizeof(double) * 3 * 256 * (size_t)h->n_ch));
        LB_CK(cudaMalloc(&h->ws_scale, sizeof(double) * 3 * (size_t)h->n_ch));
        LB_CK(cudaMemcpy(h->ws_row_off, h->row_off.data(), sizeof(int) * h->n_ch, cudaMemcpyHostToDevice));
    }
    std::vector<WsChan> prm(h->n_ch);
    for (int c = 0; c < h->n_ch; ++c) {
        const lb_params& p = h->params[c];
        if (!(p.G_inf > 0.0) || !(p.tau0 > 0.0) || !(p.g_x > 0.0))
            return fail(LB_EINVAL, "lb_warmstart: every channel needs G_inf > 0, tau0 > 0 and g_x > 0 (the closed form)%s");
        prm[c] = WsChan{p.g_x, p.G_inf, p.tau0, p.theta, p.gamma_c};
    }
    LB_CK(cudaStreamSynchronize(h->stream));
    LB_CK(cudaMemcpy(h->ws_prm, prm.data(), sizeof(WsChan) * h->n_ch, cudaMemcpyHostToDevice));
    LB_CK(launch_ws_closed_form(h->n_ch, (const WsChan*)h->ws_prm, h->ny_d, (const int*)h->ws_row_off,
                                (double*)h->ws_rows, (double*)h->ws_grid, (double*)h->ws_scale, h->stream));
    return LB_OK;
}

lb_status lb_warmstart_apply(lb_handle* h, const float* pred, const float* t_mu, const float* t_sd) {
    if (!h || (!t_mu) != (!t_sd)) return fail(LB_EINVAL, "lb_warmstart_apply: null handle, or only one of t_mu, t_sd%s");
    const long long N = h->nodes;
    lb_status st = ensure_hstage(h, (size_t)N * 4 * sizeof(double));
    if (st != LB_OK) return st;
    st = ws_closed_form(h);
    if (st != LB_OK) return st;
    double* su = (double*)h->hstage;
    LB_CK(launch_ws_decode(h->n_ch, pred, t_mu, t_sd, (const double*)h->ws_grid, (const double*)h->ws_scale,
                           (const double*)h->ws_rows, h->ny_d, (const int*)h->ws_row_off, h->node_off_d, h->nx, su,
                           su + 2 * N, su + 3 * N, h->stream));
    return set_fields_dev(h, su, su + 2 * N, su + 3 * N);
}

lb_status lb_warmstart_targets(lb_handle* h, float* targets) {
    if (!h || !targets) return fail(LB_EINVAL, "lb_warmstart_targets: null argument%s");
    lb_status st = ws_closed_form(h);
    if (st != LB_OK) return st;
    const long long N = h->nodes;
    if (!h->fields) LB_CK(cudaMalloc(&h->fields, 7 * N * h->csize));
    char* base = (char*)h->fields;
    void* fu = base;
    void* fs = base + 2 * N * h->csize;
    void* fr = base + 6 * N * h->csize;
    st = with_types(h->prec, [&](auto tt, auto tc) { LB_TYPES(tt, tc); return fields_pass<T, C>(h, (C*)fu, (C*)fs, (C*)fr); });
    if (st != LB_OK) return st;
    if (h->csize == 8)
        LB_CK(launch_ws_targets<double>(h->n_ch, (const double*)fu, (const double*)fs, (const double*)h->ws_grid,
                                        (const double*)h->ws_scale, h->ny_d, h->node_off_d, h->nx, targets, h->stream));
    else
        LB_CK(launch_ws_targets<float>(h->n_ch, (const float*)fu, (const float*)fs, (const double*)h->ws_grid,
                                       (const double*)h->ws_scale, h->ny_d, h->node_off_d, h->nx, targets, h->stream));
    return LB_OK;
}

lb_status lb_set_populations(lb_handle* h, const double* n, const double* drho, const double* sig3) {
    if (!h || !n || !drho) return fail(LB_EINVAL, "lb_set_populations: null argument%s");
    const long long N = h->nodes;
    lb_status st = ensure_hstage(h, (size_t)N * 9 * sizeof(double));
    if (st != LB_OK) return st;
    long long maxn = 0;
    for (int c = 0; c < h->n_ch; ++c) maxn = std::max(maxn, (long long)h->nx * h->ny[c]);
    dim3 g(grid_for(maxn), h->n_ch);
    double* s = (double*)h->hstage;
    LB_CK(cudaMemcpyAsync(s, n, 9 * N * sizeof(double), cudaMemcpyHostToDevice, h->stream));
    with_types(h->prec, [&](auto tt, auto tc) {
        LB_TYPES(tt, tc);
        k_pop_from_f64<T, C><<<g, 256, 0, h->stream>>>((T*)h->popA, s, h->base_d, h->P_d, h->node_off_d, h->ny_d, h->nx);
        return 0;
    });
    LB_CK(cudaGetLastError());
    LB_CK(cudaMemcpyAsync(s, drho, N * sizeof(double), cudaMemcpyHostToDevice, h->stream));
    if (h->csize == 8) k_planes_from_f64<double><<<g, 256, 0, h->stream>>>((double*)h->drho, s, 1, h->base_d, h->P_d, h->node_off_d, h->ny_d, h->nx);
    else k_planes_from_f64<float><<<g, 256, 0, h->stream>>>((float*)h->drho, s, 1, h->base_d, h->P_d, h->node_off_d, h->ny_d, h->nx);
    LB_CK(cudaGetLastError());
    if (h->smode == 1) {
        if (sig3) {
            LB_CK(cudaStreamSynchronize(h->stream));
            LB_CK(cudaMemcpyAsync(s, sig3, 3 * N * sizeof(double), cudaMemcpyHostToDevice, h->stream));
            if (h->csize == 8) k_planes_from_f64<double><<<g, 256, 0, h->stream>>>((double*)h->sig3, s, 3, h->base_d, h->P_d, h->node_off_d, h->ny_d, h->nx);
            else k_planes_from_f64<float><<<g, 256, 0, h->stream>>>((float*)h->sig3, s, 3, h->base_d, h->P_d, h->node_off_d, h->ny_d, h->nx);
            LB_CK(cudaGetLastError());
        } else {
            LB_CK(cudaMemsetAsync(h->sig3, 0, 3 * h->planes * h->csize, h->stream));
        }
    }
    if (h->phi) LB_CK(cudaMemsetAsync(h->phi, 0, h->planes * sizeof(double), h->stream));  // fluidity unset
    LB_CK(cudaStreamSynchronize(h->stream));
    h->uprev_state = -10;
    return LB_OK;
}

lb_status lb_get_populations(lb_handle* h, double* n, double* drho, double* sig3) {
    if (!h || !n || !drho) return fail(LB_EINVAL, "lb_get_populations: null argument%s");
    const long long N = h->nodes;
    lb_status st = ensure_hstage(h, (size_t)N * 9 * sizeof(double));
    if (st != LB_OK) return st;
    long long maxn = 0;
    for (int c = 0; c < h->n_ch; ++c) maxn = std::max(maxn, (long long)h->nx * h->ny[c]);
    dim3 g(grid_for(maxn), h->n_ch);
    double* s = (double*)h->hstage;
    with_types(h->prec, [&](auto tt, auto tc) {
        LB_TYPES(tt, tc);
        k_pop_to_f64<T, C><<<g, 256, 0, h->stream>>>((const T*)h->popA, s, h->base_d, h->P_d, h->node_off_d, h->ny_d, h->nx);
        return 0;
    });
    LB_CK(cudaGetLastError());
    LB_CK(cudaMemcpyAsync(n, s, 9 * N * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    LB_CK(cudaStreamSynchronize(h->stream));
    if (h->csize == 8) k_planes_to_f64<double><<<g, 256, 0, h->stream>>>((const double*)h->drho, s, 1, h->base_d, h->P_d, h->node_off_d, h->ny_d, h->nx);
    else k_planes_to_f64<float><<<g, 256, 0, h->stream>>>((const float*)h->drho, s, 1, h->base_d, h->P_d, h->node_off_d, h->ny_d, h->nx);
    LB_CK(cudaGetLastError());
    LB_CK(cudaMemcpyAsync(drho, s, N * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    LB_CK(cudaStreamSynchronize(h->stream));
    if (sig3 && h->smode == 1) {
        if (h->csize == 8) k_planes_to_f64<double><<<g, 256, 0, h->stream>>>((const double*)h->sig3, s, 3, h->base_d, h->P_d, h->node_off_d, h->ny_d, h->nx);
        else k_planes_to_f64<float><<<g, 256, 0, h->stream>>>((const float*)h->sig3, s, 3, h->base_d, h->P_d, h->node_off_d, h->ny_d, h->nx);
        LB_CK(cudaGetLastError());
        LB_CK(cudaMemcpyAsync(sig3, s, 3 * N * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
        LB_CK(cudaStreamSynchronize(h->stream));
    }
    return LB_OK;
}

namespace {
struct StateHeader {
    uint64_t magic, version;
    int64_t step, planes;
    int32_t n_ch, nx, prec, smode;
    uint64_t ny_hash;  // FNV-1a of the per-channel ny list: the image's channel split
    int32_t scheme, pad_;  // the planes an image carries depend on the scheme
};
constexpr uint64_t kMagic = 0x4d4c4e2d424c6772ull;
constexpr uint64_t kStateVersion = 2;

uint64_t ny_list_hash(const std::vector<int>& ny) {
    uint64_t x = 0xcbf29ce484222325ull;  // FNV-1a, 64-bit offset basis and prime
    for (int v : ny)
        for (int b = 0; b < 4; ++b) {
            x ^= (uint64_t)(((uint32_t)v >> (8 * b)) & 0xffu);
            x *= 0x100000001b3ull;
        }
    return x;
}
}  // namespace

size_t lb_state_bytes(const lb_handle* h) {
    if (!h) return 0;
    size_t b = sizeof(StateHeader) + 9 * h->planes * h->tsize + h->planes * h->csize;
    if (h->smode == 1) b += 3 * h->planes * h->csize;
    if (h->phi) b += h->planes * sizeof(double);
    return b;
}

lb_status lb_get_state(lb_handle* h, void* buf, size_t bytes) {
    if (!h || !buf || bytes < lb_state_bytes(h)) return fail(LB_EINVAL, "lb_get_state: bad buffer%s");
    StateHeader hd{kMagic, kStateVersion, h->step, h->planes, h->n_ch, h->nx, h->prec, h->smode, ny_list_hash(h->ny),
                   h->scheme, 0};
    char* p = (char*)buf;
    std::memcpy(p, &hd, sizeof hd);
    p += sizeof hd;
    LB_CK(cudaMemcpyAsync(p, h->popA, 9 * h->planes * h->tsize, cudaMemcpyDeviceToHost, h->stream));
    p += 9 * h->planes * h->tsize;
    LB_CK(cudaMemcpyAsync(p, h->drho, h->planes * h->csize, cudaMemcpyDeviceToHost, h->stream));
    p += h->planes * h->csize;
    if (h->smode == 1) LB_CK(cudaMemcpyAsync(p, h->sig3, 3 * h->planes * h->csize, cudaMemcpyDeviceToHost, h->stream));
    if (h->smode == 1) p += 3 * h->planes * h->csize;
    if (h->phi) LB_CK(cudaMemcpyAsync(p, h->phi, h->planes * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    LB_CK(cudaStreamSynchronize(h->stream));
    return LB_OK;
}

lb_status lb_set_state(lb_handle* h, const void* buf, size_t bytes) {
    if (!h || !buf || bytes < lb_state_bytes(h)) return fail(LB_EINVAL, "lb_set_state: bad buffer%s");
    StateHeader hd;
    std::memcpy(&hd, buf, sizeof hd);
    if (hd.magic != kMagic || hd.version != kStateVersion)
        return fail(LB_EINVAL, "lb_set_state: not a state image of this library version%s");
    if (hd.planes != h->planes || hd.n_ch != h->n_ch || hd.nx != h->nx || hd.prec != h->prec || hd.scheme != h->scheme ||
        hd.smode != h->smode || hd.ny_hash != ny_list_hash(h->ny))
        return fail(LB_EINVAL, "lb_set_state: image does not match this handle's grid or channel split%s");
    const char* p = (const char*)buf + sizeof hd;
    LB_CK(cudaMemcpyAsync(h->popA, p, 9 * h->planes * h->tsize, cudaMemcpyHostToDevice, h->stream));
    p += 9 * h->planes * h->tsize;
    LB_CK(cudaMemcpyAsync(h->drho, p, h->planes * h->csize, cudaMemcpyHostToDevice, h->stream));
    p += h->planes * h->csize;
    if (h->smode == 1) LB_CK(cudaMemcpyAsync(h->sig3, p, 3 * h->planes * h->csize, cudaMemcpyHostToDevice, h->stream));
    if (h->smode == 1) p += 3 * h->planes * h->csize;
    if (h->phi) LB_CK(cudaMemcpyAsync(h->phi, p, h->planes * sizeof(double), cudaMemcpyHostToDevice, h->stream));
    // a restored state starts healthy: the per-channel status word and the sticky flags are
    // cleared, so rolling back to a good image after an instability steps every channel again
    LB_CK(cudaMemsetAsync(h->status_d, 0, sizeof(int) * h->n_ch, h->stream));
    LB_CK(cudaStreamSynchronize(h->stream));
    h->status_pending = false;
    std::memset(h->status_h, 0, h->n_ch * sizeof(int));  // (the stream is idle: no kernel writes it now)
    h->any_unstable = h->any_timeout = false;
    h->step = hd.step;
    h->uprev_state = -10;
    h->mon_state = -1;
    return LB_OK;
}

lb_status lb_channel_status(lb_handle* h, int* status) {
    if (!h || !status) return fail(LB_EINVAL, "lb_channel_status: null argument%s");
    LB_CK(cudaMemcpyAsync(status, h->status_d, sizeof(int) * h->n_ch, cudaMemcpyDeviceToHost, h->stream));
    LB_CK(cudaStreamSynchronize(h->stream));
    for (int c = 0; c < h->n_ch; ++c) {
        if (status[c] & 1) h->any_unstable = true;
        if (status[c] & 2) h->any_timeout = true;
    }
    return LB_OK;
}

}  // extern "C"
