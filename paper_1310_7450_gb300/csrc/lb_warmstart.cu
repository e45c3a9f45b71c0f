// lb_warmstart.cu -- the learned warm start's profile arithmetic on the device (not in the paper):
// the closed-form steady channel profile of Sec. III B, the resampling between a channel's Ny rows
// and the network's 256-point grid, the encoding of steady LB profiles as training targets, and
// the decoding of network outputs into per-node start fields (u, rho = 1, delta rho).
//
// Grid: d = (y - y_c)/H at the centres of 256 equal cells, d_k = (k + 1/2)/256 * 2 - 1; rows:
// d_y = (y - (ny-1)/2)/(ny/2).  Resampling is linear interpolation with the end values held.
// Network target of field j on the grid: (profile - closed form) / scale_j, scale_j = max |closed
// form_j| (u_x, sigma_xy, N1).
#include <cuda_runtime.h>

#include "lb_device.cuh"

namespace lbk {

constexpr int kWsGrid = 256;   // network grid points per field
constexpr int kWsPts = 4001;   // points of the trapezoid integration of the closed form
constexpr int kWsThreads = 256;

struct WsChan {
    double g, G, tau0, theta, gamma_c;  // body force, G_inf, tau0, theta, gamma_c of the channel
};

// Linear interpolation of f (n points at x0 + i h) at x, end values held (np.interp on a uniform
// abscissa).
__device__ inline double interp_uniform(double x, double x0, double h, const double* f, int n, int stride = 1) {
    if (x <= x0) return f[0];
    const double xe = x0 + (n - 1) * h;
    if (x >= xe) return f[(n - 1) * stride];
    int i = (int)floor((x - x0) / h);
    if (i > n - 2) i = n - 2;
    if (i < 0) i = 0;
    const double xa = x0 + i * h;
    const double t = (x - xa) / h;
    return f[i * stride] + t * (f[(i + 1) * stride] - f[i * stride]);
}

__device__ inline double grid_d(int k) { return (k + 0.5) / kWsGrid * 2.0 - 1.0; }

// Block-wide inclusive scan of `v` (n values, in place) by one contiguous chunk per thread.
__device__ void block_scan(double* v, int n, double* part) {
    const int t = threadIdx.x;
    const int per = (n + kWsThreads - 1) / kWsThreads;
    const int a = t * per, b = min(n, a + per);
    double s = 0.0;
    for (int i = a; i < b; ++i) { s += v[i]; v[i] = s; }
    part[t] = s;
    __syncthreads();
    if (t == 0) {
        double acc = 0.0;
        for (int k = 0; k < kWsThreads; ++k) { const double q = part[k]; part[k] = acc; acc += q; }
    }
    __syncthreads();
    for (int i = a; i < b; ++i) v[i] += part[t];
    __syncthreads();
}

// One CTA per channel: the closed-form steady profile (the quadratic for dv/dd of Sec. III B,
// v(1) = 0, integrated by the trapezoid rule on kWsPts points, u = (H/tau0) v) on the rows
// (rows[row_off + y][3] = u_x, sigma_xy, N1) and on the grid (grid[c][3][256]), and the scales.
__global__ void __launch_bounds__(kWsThreads) k_ws_closed_form(const WsChan* __restrict__ prm, const int* __restrict__ nys,
                                                               const int* __restrict__ row_off, double* __restrict__ rows,
                                                               double* __restrict__ grid, double* __restrict__ scale) {
    extern __shared__ double sh[];
    double* v = sh;                 // [kWsPts] v(d)
    double* dv = v + kWsPts;        // [kWsPts] dv/dd
    double* part = dv + kWsPts;     // [kWsThreads]
    const int c = blockIdx.x, t = threadIdx.x, ny = nys[c];
    const WsChan p = prm[c];
    const double H = ny / 2.0, wpH = p.g * H / p.G;
    const double step = 1.0 / (kWsPts - 1);
    auto dpt = [&](int k) { return k == kWsPts - 1 ? 1.0 : k * step; };
    for (int k = t; k < kWsPts; k += kWsThreads) {
        const double d = dpt(k);
        if (p.theta == 0.0) {
            dv[k] = -wpH * d;
        } else {
            const double a = wpH * d / 2.0, b = p.gamma_c * (1.0 + p.theta) / (2.0 * p.theta);
            dv[k] = -a + b - sqrt((a - b) * (a - b) + wpH * d * p.gamma_c / p.theta);
        }
    }
    __syncthreads();
    for (int k = t; k < kWsPts; k += kWsThreads)
        v[k] = k == 0 ? 0.0 : 0.5 * (dv[k] + dv[k - 1]) * (dpt(k) - dpt(k - 1));
    __syncthreads();
    block_scan(v, kWsPts, part);
    const double vend = v[kWsPts - 1];
    __syncthreads();
    for (int k = t; k < kWsPts; k += kWsThreads) v[k] -= vend;
    __syncthreads();
    const double tau = p.theta * p.tau0;
    for (int y = t; y < ny; y += kWsThreads) {
        const double dy = (y - (ny - 1) / 2.0) / H;
        const double dd = fabs(dy);
        const double u = (H / p.tau0) * interp_uniform(dd, 0.0, step, v, kWsPts);
        const double sg = dy > 0.0 ? 1.0 : (dy < 0.0 ? -1.0 : 0.0);
        const double gd = interp_uniform(dd, 0.0, step, dv, kWsPts) / p.tau0 * sg;
        const double tm = tau > 0.0 ? tau / (1.0 + tau * fabs(gd) / p.gamma_c) : 0.0;
        const double sxy = p.G * tm * gd, n1 = 2.0 * p.G * gd * gd * tm * tm;
        double* r = rows + 3LL * (row_off[c] + y);
        r[0] = u;
        r[1] = sxy;
        r[2] = n1;
    }
    __syncthreads();  // (the block's global writes of the rows are visible to it after the barrier)
    const double r0 = -(ny - 1) / 2.0 / H, rh = 1.0 / H;
    const double* crow = rows + 3LL * row_off[c];
    double* gc = grid + 3LL * kWsGrid * c;
    double m[3] = {0.0, 0.0, 0.0};
    for (int k = t; k < kWsGrid; k += kWsThreads)
        for (int j = 0; j < 3; ++j) {
            const double g = interp_uniform(grid_d(k), r0, rh, crow + j, ny, 3);
            gc[j * kWsGrid + k] = g;
            m[j] = fmax(m[j], fabs(g));
        }
    for (int j = 0; j < 3; ++j) {
        part[t] = m[j];
        __syncthreads();
        for (int h = kWsThreads / 2; h > 0; h >>= 1) {
            if (t < h) part[t] = fmax(part[t], part[t + h]);
            __syncthreads();
        }
        if (t == 0) scale[3 * c + j] = fmax(part[0], 1e-300);
        __syncthreads();
    }
}

// One CTA per channel: the start fields of every node from a network output (pred [c][768],
// standardised outputs; de-standardised with t_mu, t_sd when given) or, with pred == nullptr,
// from the closed form on the rows: u = (u_x(y), 0), rho = 1, delta rho = -(3/2) N1(y) (the trace
// of a simple-shear stress is N1; Eq. rhoplus).  Outputs in node order: u [node][2], rho, drho.
__global__ void __launch_bounds__(kWsThreads) k_ws_decode(const float* __restrict__ pred, const float* __restrict__ t_mu,
                                                          const float* __restrict__ t_sd, const double* __restrict__ grid,
                                                          const double* __restrict__ scale, const double* __restrict__ rows,
                                                          const int* __restrict__ nys, const int* __restrict__ row_off,
                                                          const long long* __restrict__ node_off, int nx,
                                                          double* __restrict__ u, double* __restrict__ rho,
                                                          double* __restrict__ drho) {
    __shared__ double prof[2][kWsGrid];  // decoded u_x and N1 on the grid
    const int c = blockIdx.x, t = threadIdx.x, ny = nys[c];
    if (pred) {
        for (int k = t; k < kWsGrid; k += kWsThreads)
            for (int jj = 0; jj < 2; ++jj) {
                const int j = jj == 0 ? 0 : 2;  // fields u_x and N1
                const int o = j * kWsGrid + k;
                double y = (double)pred[(long long)c * 3 * kWsGrid + o];
                if (t_sd) y = y * (double)t_sd[o] + (double)t_mu[o];
                prof[jj][k] = grid[3LL * kWsGrid * c + o] + scale[3 * c + j] * y;
            }
    }
    __syncthreads();
    const double H = ny / 2.0;
    const double g0 = grid_d(0), gh = 2.0 / kWsGrid;
    const long long n = (long long)nx * ny;
    for (long long q = t; q < n; q += kWsThreads) {
        const int y = (int)(q / nx);
        double ux, n1;
        if (pred) {
            const double dy = (y - (ny - 1) / 2.0) / H;
            ux = interp_uniform(dy, g0, gh, prof[0], kWsGrid);
            n1 = interp_uniform(dy, g0, gh, prof[1], kWsGrid);
        } else {
            const double* r = rows + 3LL * (row_off[c] + y);
            ux = r[0];
            n1 = r[2];
        }
        const long long node = node_off[c] + q;
        u[2 * node] = ux;
        u[2 * node + 1] = 0.0;
        rho[node] = 1.0;
        drho[node] = -1.5 * n1;
    }
}

// One CTA per channel: training targets from the fields of a state (u [node][2], sigma [node][4]
// as xx, yy, zz, xy; column x = 0 of each row): (profile - closed form)/scale on the grid, float.
template <typename F>
__global__ void __launch_bounds__(kWsThreads) k_ws_targets(const F* __restrict__ fu, const F* __restrict__ fs,
                                                           const double* __restrict__ grid, const double* __restrict__ scale,
                                                           const int* __restrict__ nys, const long long* __restrict__ node_off,
                                                           int nx, float* __restrict__ targets) {
    const int c = blockIdx.x, t = threadIdx.x, ny = nys[c];
    const double H = ny / 2.0, r0 = -(ny - 1) / 2.0 / H, rh = 1.0 / H;
    for (int k = t; k < kWsGrid; k += kWsThreads) {
        const double x = grid_d(k);
        // the row interval that holds x (end values held), then the three fields there
        double vals[3];
        if (x <= r0 || ny == 1) {
            const long long nd = node_off[c];
            vals[0] = (double)fu[2 * nd];
            vals[1] = (double)fs[4 * nd + 3];
            vals[2] = (double)fs[4 * nd] - (double)fs[4 * nd + 1];
        } else if (x >= r0 + (ny - 1) * rh) {
            const long long nd = node_off[c] + (long long)(ny - 1) * nx;
            vals[0] = (double)fu[2 * nd];
            vals[1] = (double)fs[4 * nd + 3];
            vals[2] = (double)fs[4 * nd] - (double)fs[4 * nd + 1];
        } else {
            int i = (int)floor((x - r0) / rh);
            if (i > ny - 2) i = ny - 2;
            const double tt = (x - (r0 + i * rh)) / rh;
            const long long na = node_off[c] + (long long)i * nx, nb = na + nx;
            const double ua = (double)fu[2 * na], ub = (double)fu[2 * nb];
            const double sa = (double)fs[4 * na + 3], sb = (double)fs[4 * nb + 3];
            const double qa = (double)fs[4 * na] - (double)fs[4 * na + 1], qb = (double)fs[4 * nb] - (double)fs[4 * nb + 1];
            vals[0] = ua + tt * (ub - ua);
            vals[1] = sa + tt * (sb - sa);
            vals[2] = qa + tt * (qb - qa);
        }
        for (int j = 0; j < 3; ++j) {
            const int o = j * kWsGrid + k;
            targets[(long long)c * 3 * kWsGrid + o] =
                (float)((vals[j] - grid[3LL * kWsGrid * c + o]) / scale[3 * c + j]);
        }
    }
}

cudaError_t launch_ws_closed_form(int n_ch, const WsChan* prm, const int* nys, const int* row_off, double* rows,
                                  double* grid, double* scale, cudaStream_t s) {
    const size_t smem = sizeof(double) * (2 * kWsPts + kWsThreads);
    cudaError_t e = cudaFuncSetAttribute(k_ws_closed_form, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k_ws_closed_form<<<n_ch, kWsThreads, smem, s>>>(prm, nys, row_off, rows, grid, scale);
    return cudaGetLastError();
}

cudaError_t launch_ws_decode(int n_ch, const float* pred, const float* t_mu, const float* t_sd, const double* grid,
                             const double* scale, const double* rows, const int* nys, const int* row_off,
                             const long long* node_off, int nx, double* u, double* rho, double* drho, cudaStream_t s) {
    k_ws_decode<<<n_ch, kWsThreads, 0, s>>>(pred, t_mu, t_sd, grid, scale, rows, nys, row_off, node_off, nx, u, rho, drho);
    return cudaGetLastError();
}

template <typename F>
cudaError_t launch_ws_targets(int n_ch, const F* fu, const F* fs, const double* grid, const double* scale, const int* nys,
                              const long long* node_off, int nx, float* targets, cudaStream_t s) {
    k_ws_targets<F><<<n_ch, kWsThreads, 0, s>>>(fu, fs, grid, scale, nys, node_off, nx, targets);
    return cudaGetLastError();
}
template cudaError_t launch_ws_targets<double>(int, const double*, const double*, const double*, const double*, const int*,
                                               const long long*, int, float*, cudaStream_t);
template cudaError_t launch_ws_targets<float>(int, const float*, const float*, const double*, const double*, const int*,
                                              const long long*, int, float*, cudaStream_t);

}  // namespace lbk
