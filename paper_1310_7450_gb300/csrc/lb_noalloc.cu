// lb_noalloc.cu -- lb_field_monitor_static: the per-channel residual / flux / max|u| reduction of
// lb_monitor, computed from two velocity fields the caller already holds on the device, with its
// scratch in a fixed array inside this library instead of any allocation.
//
// Why it exists: some callers must not allocate device memory at the moment they want these
// diagnostics -- for example a monitoring loop that cannot afford cudaMalloc's implicit device
// synchronisation in the middle of a run, or a process whose device memory is already fully
// reserved by another allocator (such as a framework's caching allocator holding the whole pool).
// Everything else in the library allocates its work buffers at lb_create time; this entry point
// allocates nothing, ever.
//
// Scratch: g_monitor_scratch below, 65536 partial records of four doubles (2 MiB).  Every GPU
// that loads the library holds this array until the process exits.  The first call on a device
// looks up the array's device address with cudaGetSymbolAddress (with that device current); make
// that first call before any stream capture.  Calls on a stream that is not capturing look the
// address up again (cheap), so a device reset or a re-created primary context does not leave a
// stale address behind; calls during a capture reuse the last address found.  All calls share the
// array: calls whose kernels overlap on the GPU (e.g. on two streams) race on it.  Each call writes
// every partial record it later reads, so no record needs clearing between calls.
//
// Non-finite fields: a NaN or Inf anywhere in a channel's u_now or u_prev makes all three of that
// channel's outputs NaN (the partial kernel marks the record's max slot with NaN and the maxima
// propagate NaN), so a diverged channel never reads as converged.
#include <cuda_runtime.h>

#include <cstdio>
#include <mutex>

#include "lbnlm.h"

namespace lbk {
void set_last_error(const char* msg);
}

namespace {

constexpr int kThreads = 256;
constexpr int kBlocksPerChannel = 64;      // partial records per channel
constexpr int kMaxRecords = 65536;         // capacity of the scratch array (records of 4 doubles)
constexpr int kMaxDevices = 64;

__device__ __align__(256) double g_monitor_scratch[4 * kMaxRecords];

double* g_scratch_addr[kMaxDevices] = {};  // host-side device addresses of the scratch, per device
std::mutex g_scratch_mu;

lb_status bad(lb_status s, const char* what) {
    char msg[256];
    std::snprintf(msg, sizeof msg, "lb_field_monitor_static: %s", what);
    lbk::set_last_error(msg);
    return s;
}

// max that keeps a NaN from either side (fmax would drop it)
__device__ __forceinline__ double max_keep_nan(double a, double b) {
    return (a != a) ? a : ((b != b) ? b : fmax(a, b));
}

template <typename F>
__global__ void k_field_partials(const F* __restrict__ u, const F* __restrict__ up, const long long* __restrict__ off,
                                 double* __restrict__ scratch) {
    const int c = blockIdx.y, b = blockIdx.x, t = threadIdx.x;
    const long long begin = off[c], end = off[c + 1];
    double s0 = 0.0, s1 = 0.0, s2 = 0.0, s3 = 0.0;
    for (long long k = begin + (long long)b * kThreads + t; k < end; k += (long long)kBlocksPerChannel * kThreads) {
        const double ux = (double)u[2 * k], uy = (double)u[2 * k + 1];
        const double px = (double)up[2 * k], py = (double)up[2 * k + 1];
        const double dx = ux - px, dy = uy - py;
        const double u2 = ux * ux + uy * uy;
        s0 += dx * dx + dy * dy;
        s1 += u2;
        s2 += ux;
        const bool finite = isfinite(ux) && isfinite(uy) && isfinite(px) && isfinite(py);
        s3 = max_keep_nan(s3, finite ? u2 : (double)NAN);
    }
    __shared__ double red[kThreads][4];
    red[t][0] = s0; red[t][1] = s1; red[t][2] = s2; red[t][3] = s3;
    __syncthreads();
    for (int h = kThreads / 2; h > 0; h >>= 1) {
        if (t < h) {
            red[t][0] += red[t + h][0];
            red[t][1] += red[t + h][1];
            red[t][2] += red[t + h][2];
            red[t][3] = max_keep_nan(red[t][3], red[t + h][3]);
        }
        __syncthreads();
    }
    if (t == 0) {
        double* o = scratch + 4 * ((long long)c * kBlocksPerChannel + b);
        o[0] = red[0][0]; o[1] = red[0][1]; o[2] = red[0][2]; o[3] = red[0][3];
    }
}

// One thread per channel sums that channel's partial records in a fixed order.
__global__ void k_field_finish(const double* __restrict__ scratch, int n_ch, int nx, double* __restrict__ out) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= n_ch) return;
    double s0 = 0.0, s1 = 0.0, s2 = 0.0, s3 = 0.0;
    for (int b = 0; b < kBlocksPerChannel; ++b) {
        const double* p = scratch + 4 * ((long long)c * kBlocksPerChannel + b);
        s0 += p[0]; s1 += p[1]; s2 += p[2]; s3 = max_keep_nan(s3, p[3]);
    }
    if (s3 != s3) {  // a non-finite value in either field of this channel
        out[3 * c + 0] = out[3 * c + 1] = out[3 * c + 2] = NAN;
        return;
    }
    out[3 * c + 0] = s1 == 0.0 ? 0.0 : sqrt(s0 / s1);  // a field at rest: 0, as lb_monitor
    out[3 * c + 1] = s2 / nx;
    out[3 * c + 2] = sqrt(s3);
}

// Device address of the scratch array for the current device.  Looked up afresh whenever the
// stream is not capturing; during a capture the last address found on this device is reused.
lb_status scratch_for_current_device(cudaStream_t s, double** ptr) {
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices)
        return bad(LB_ECUDA, "no usable current CUDA device");
    if (s) {
        int sdev = -1;
        if (cudaStreamGetDevice(s, &sdev) != cudaSuccess) return bad(LB_EINVAL, "cuda_stream is not a valid stream");
        if (sdev != dev) return bad(LB_EINVAL, "cuda_stream belongs to another device than the current one");
    }
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(s, &cap) != cudaSuccess) return bad(LB_ECUDA, "cannot query the stream's capture state");
    std::lock_guard<std::mutex> lock(g_scratch_mu);
    if (cap == cudaStreamCaptureStatusNone) {
        void* p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_monitor_scratch);
        if (e != cudaSuccess || !p) return bad(LB_ECUDA, cudaGetErrorString(e));
        g_scratch_addr[dev] = static_cast<double*>(p);
    } else if (!g_scratch_addr[dev]) {
        return bad(LB_ESTATE, "the first call on a device must come before any stream capture");
    }
    *ptr = g_scratch_addr[dev];
    return LB_OK;
}

}  // namespace

extern "C" lb_status lb_field_monitor_static(const void* u_now, const void* u_prev, int dtype, int n_channels,
                                             const long long* node_offsets, int nx, double* out, void* cuda_stream) {
    if (!u_now || !u_prev || !node_offsets || !out) return bad(LB_EINVAL, "null pointer argument");
    if (dtype != 0 && dtype != 1) return bad(LB_EINVAL, "dtype must be 0 (double) or 1 (float)");
    if (nx < 1 || n_channels < 1) return bad(LB_EINVAL, "need nx >= 1 and n_channels >= 1");
    if ((long long)n_channels * kBlocksPerChannel > kMaxRecords)
        return bad(LB_EINVAL, "too many channels for the fixed scratch (at most 1024 channels per call)");
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    double* scratch = nullptr;
    lb_status st = scratch_for_current_device(s, &scratch);
    if (st != LB_OK) return st;
    const dim3 grid(kBlocksPerChannel, n_channels);
    if (dtype == 0)
        k_field_partials<double><<<grid, kThreads, 0, s>>>(static_cast<const double*>(u_now),
                                                            static_cast<const double*>(u_prev), node_offsets, scratch);
    else
        k_field_partials<float><<<grid, kThreads, 0, s>>>(static_cast<const float*>(u_now),
                                                           static_cast<const float*>(u_prev), node_offsets, scratch);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return bad(LB_ECUDA, cudaGetErrorString(e));
    k_field_finish<<<(n_channels + 127) / 128, 128, 0, s>>>(scratch, n_channels, nx, out);
    e = cudaGetLastError();
    if (e != cudaSuccess) return bad(LB_ECUDA, cudaGetErrorString(e));
    return LB_OK;
}
