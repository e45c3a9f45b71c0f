// lb_sweep.cuh -- the batched sweep: many independent channels stepped to a steady state in ONE
// persistent launch.
//
// Each channel is owned by a thread-block cluster of CL CTAs (CTA r of the cluster owns rows
// [r*ny/CL, (r+1)*ny/CL) of that channel, full width nx).  The cluster runs the channel's time loop
// by itself: per step every CTA pulls its rows (and a two-row halo, whose moments it recomputes) from
// the channel's current population buffer in L2 (ld.global.cg: other CTAs wrote them), collides its
// own rows into the other buffer, and the cluster meets at a hardware cluster barrier (release /
// acquire) before the next step.  Every `check` = k steps the mean one-step change over the interval,
// ||u(t) - u(t-k)|| / (k ||u(t)||), is reduced across the cluster through distributed shared memory
// (over one step it would sit on the FP32 rounding floor of a steady state; over k steps that floor
// falls as 1/k while a smooth exponential approach gives the one-step value); when it is <= tol (or
// the channel became unstable, or max_steps is reached) the whole cluster leaves and its SMs take
// the next channel.  Channels are launched widest first.  Step counts stay multiples of `check`
// (even), so every channel ends on the buffer it started from.
#pragma once

#include <cooperative_groups.h>

#include "lb_device.cuh"

namespace lbk {

namespace cg = cooperative_groups;

template <typename T, typename C>
struct SweepArgs {
    T* popA;                       // buffer holding the current state at launch
    T* popB;
    C* drho;
    C* uprev;                      // 2 planes per channel
    const ChanParams<C>* chan;
    int* status;
    const int* order;              // channel of cluster k
    long long* steps_out;          // per channel: steps to reach tol, -1 not reached, -2 unstable
    double* res_out;               // per channel: last residual
    int nx;
    int check;                     // residual interval (even, >= 2)
    long long max_steps;           // multiple of check
    double tol;
    bool sr;                       // BF16 storage: stochastic rounding
    uint32_t sr_key;
};

template <typename T>
__device__ __forceinline__ T ld_cg(const T* p) { return __ldcg(p); }
template <>
__device__ __forceinline__ __nv_bfloat16 ld_cg<__nv_bfloat16>(const __nv_bfloat16* p) {
    const unsigned short v = __ldcg(reinterpret_cast<const unsigned short*>(p));
    return __ushort_as_bfloat16(v);
}

// Pull-stream with bounce-back, reading through L2 (the sources were written by other CTAs).
template <typename T, typename C>
__device__ __forceinline__ void pull9_l2(const T* __restrict__ pc, long long P, int nx, int ny, int x, int y, C (&d)[9]) {
#pragma unroll
    for (int i = 0; i < 9; ++i) {
        const int ys = y - cy(i);
        const T* src;
        if (ys < 0 || ys >= ny) {
            src = pc + (long long)opp(i) * P + (long long)y * nx + x;
        } else {
            int xs = x - cx(i);
            xs = xs < 0 ? xs + nx : (xs >= nx ? xs - nx : xs);
            src = pc + (long long)i * P + (long long)ys * nx + xs;
        }
        d[i] = (C)Store<T>::cvt(ld_cg<T>(src));
    }
}

// NT threads per CTA; each thread owns up to NPT nodes of the CTA's rows (host guarantees
// rows * nx <= NT * NPT).
// NX > 0: the handle's width as a compile-time constant (shifts and masks in the node index
// arithmetic for NX = 4); NX = 0: any width.  FP32 arithmetic is bounded to 128 registers.
template <typename T, typename C, int NT, int NPT, int NX = 0>
__global__ void __launch_bounds__(NT, sizeof(C) == 8 ? 1 : 512 / NT) k_sweep(const SweepArgs<T, C> a) {
    cg::cluster_group cluster = cg::this_cluster();
    const int CL = (int)cluster.num_blocks();
    const int rank = (int)cluster.block_rank();
    const int ch = a.order[blockIdx.x / CL];
    const ChanParams<C> P = a.chan[ch];
    const int nx = NX > 0 ? NX : a.nx, ny = P.ny, t = threadIdx.x;
    const int y0 = (int)((long long)ny * rank / CL), y1 = (int)((long long)ny * (rank + 1) / CL);
    const int ey0 = max(y0 - 2, 0), ey1 = min(y1 + 2, ny);  // rows whose gradient velocity we need
    const int n_own = (y1 - y0) * nx, n_ext = (ey1 - ey0) * nx;

    extern __shared__ __align__(16) unsigned char smem[];
    C* su = reinterpret_cast<C*>(smem);                               // [ext rows][nx][2]
    __shared__ double part[4];                                        // residual partials of this CTA
    __shared__ int done;                                              // decision of rank 0

    T* bufs[2] = {a.popA + 9 * P.base, a.popB + 9 * P.base};
    C* dr = a.drho + P.base;
    C* up = a.uprev + 2 * P.base;
    if (t == 0) done = 0;
    cluster.sync();

    long long s = 0;
    for (; s < a.max_steps; ++s) {
        const T* pin = bufs[s & 1];
        T* pout = bufs[(s & 1) ^ 1];
        // residual steps: every `check` steps; the first one only saves the velocity
        const bool save = ((s + 1) % a.check) == 0;
        const bool resid = save && (s + 1 >= 2 * (long long)a.check);

        // phase 1: own nodes (kept in registers) and halo rows -> gradient velocity in shared memory
        C d[NPT][9], dR[NPT], jx[NPT], jy[NPT];
#pragma unroll
        for (int k = 0; k < NPT; ++k) {
            const int e = t + k * NT;
            if (e < n_own) {
                const int y = y0 + e / nx, x = e % nx;
                C ux, uy;
                pull9_l2<T, C>(pin, P.P, nx, ny, x, y, d[k]);
                gradient_velocity<C>(d[k], P.gx, dR[k], jx[k], jy[k], ux, uy);
                const int r = (y - ey0) * nx + x;
                su[2 * r] = ux;
                su[2 * r + 1] = uy;
            }
        }
        const int n_halo = n_ext - n_own;
        for (int e = t; e < n_halo; e += NT) {
            const int below = (y0 - ey0) * nx;           // halo nodes under the own rows come first
            const int row = e < below ? ey0 + e / nx : y1 + (e - below) / nx;
            const int x = e % nx;
            C dh[9], hR, hx, hy, ux, uy;
            pull9_l2<T, C>(pin, P.P, nx, ny, x, row, dh);
            gradient_velocity<C>(dh, P.gx, hR, hx, hy, ux, uy);
            const int r = (row - ey0) * nx + x;
            su[2 * r] = ux;
            su[2 * r + 1] = uy;
        }
        __syncthreads();

        // phase 2: collide the own nodes
        double r0 = 0.0, r1 = 0.0, r2 = 0.0, r3 = 0.0;
#pragma unroll
        for (int k = 0; k < NPT; ++k) {
            const int e = t + k * NT;
            if (e < n_own) {
                const int y = y0 + e / nx, x = e % nx;
                const int xm = x == 0 ? nx - 1 : x - 1, xp = x == nx - 1 ? 0 : x + 1;
                const C* row = su + 2 * ((y - ey0) * nx);
                const C ka = C(0.5) * (row[2 * xp] - row[2 * xm]);
                const C kc = C(0.5) * (row[2 * xp + 1] - row[2 * xm + 1]);
                C kb, ke;
                if (y == 0) {
                    const C* r1p = row + 2 * nx;
                    const C* r2p = row + 4 * nx;
                    kb = C(0.5) * (C(-3) * row[2 * x] + C(4) * r1p[2 * x] - r2p[2 * x]);
                    ke = C(0.5) * (C(-3) * row[2 * x + 1] + C(4) * r1p[2 * x + 1] - r2p[2 * x + 1]);
                } else if (y == ny - 1) {
                    const C* r1m = row - 2 * nx;
                    const C* r2m = row - 4 * nx;
                    kb = C(0.5) * (C(3) * row[2 * x] - C(4) * r1m[2 * x] + r2m[2 * x]);
                    ke = C(0.5) * (C(3) * row[2 * x + 1] - C(4) * r1m[2 * x + 1] + r2m[2 * x + 1]);
                } else {
                    kb = C(0.5) * (row[2 * nx + 2 * x] - row[-2 * nx + 2 * x]);
                    ke = C(0.5) * (row[2 * nx + 2 * x + 1] - row[-2 * nx + 2 * x + 1]);
                }
                const long long pn = (long long)y * nx + x;
                const NodeState<C> st = constitutive<C, 0>(P, ka, kb, kc, ke, dR[k], jx[k], jy[k], dr[pn], C(0), C(0), C(0));
                const C rho_h = C(1) + st.dReq - st.drho;
                if (!velocity_ok<C>(jx[k], jy[k], rho_h, (C)0.3)) atomicOr(a.status + ch, 1);
                C D[9];
                collide_node<C>(P, st, d[k], D);
                store_node<T, C>(pout + pn, P.P, d[k], D, a.sr, mix32(a.sr_key ^ (uint32_t)(s * 0x9E3779B9ull) ^ (uint32_t)(ch * 0x85EBCA6Bu)), (uint32_t)pn);
                dr[pn] = st.drho;
                if (save) {
                    const C ih = Arith<C>::div(C(1), rho_h);
                    const C urx = jx[k] * ih, ury = jy[k] * ih;
                    if (resid) {
                        const double dx_ = (double)urx - (double)up[pn], dy_ = (double)ury - (double)up[P.P + pn];
                        r0 += dx_ * dx_ + dy_ * dy_;
                        r1 += (double)urx * urx + (double)ury * ury;
                    }
                    up[pn] = urx;
                    up[P.P + pn] = ury;
                }
            }
        }
        if (resid) {
            // CTA partials (warp shuffles, then shared atomics)
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                r0 += __shfl_xor_sync(0xffffffffu, r0, o);
                r1 += __shfl_xor_sync(0xffffffffu, r1, o);
            }
            if (t == 0) { part[0] = 0.0; part[1] = 0.0; }
            __syncthreads();
            if ((t & 31) == 0) {
                atomicAdd(&part[0], r0);
                atomicAdd(&part[1], r1);
            }
        }
        (void)r2; (void)r3;
        cluster.sync();  // every CTA of the channel has written step s+1
        if (resid) {
            if (rank == 0 && t == 0) {
                double du2 = 0.0, u2 = 0.0;
                for (int q = 0; q < CL; ++q) {
                    const double* pq = cluster.map_shared_rank(part, q);
                    du2 += pq[0];
                    u2 += pq[1];
                }
                const double r = u2 > 0.0 ? sqrt(du2 / u2) / a.check : 0.0;
                const bool unstable = *(volatile int*)(a.status + ch) != 0;
                int dec = 0;
                if (unstable) dec = 2;
                else if (r <= a.tol) dec = 1;
                done = dec;
                a.res_out[ch] = r;
            }
            cluster.sync();
            const int dec = *cluster.map_shared_rank(&done, 0);
            if (dec) {
                if (rank == 0 && t == 0) a.steps_out[ch] = dec == 2 ? -2 : s + 1;
                cluster.sync();  // no CTA leaves while another may still read its shared memory
                return;
            }
        }
    }
    if (rank == 0 && t == 0) a.steps_out[ch] = -1;
    cluster.sync();  // no CTA leaves while another may still read its shared memory
}

// How many clusters of `cl` CTAs with `smem` bytes the device can hold at once (0: the shape cannot
// be co-scheduled, so it is never launched).
template <typename T, typename C, int NT, int NPT, int NX = 0>
cudaError_t launch_sweep_capacity(int cl, size_t smem, int* n_clusters) {
    auto k = k_sweep<T, C, NT, NPT, NX>;
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(cl);
    cfg.blockDim = dim3(NT);
    cfg.dynamicSmemBytes = smem;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = cl;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaOccupancyMaxActiveClusters(n_clusters, k, &cfg);
}

template <typename T, typename C, int NT, int NPT, int NX = 0>
cudaError_t launch_sweep(const SweepArgs<T, C>& a, int n_clusters, int cl, size_t smem, cudaStream_t s) {
    auto k = k_sweep<T, C, NT, NPT, NX>;
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    if (e != cudaSuccess) return e;
    // set every time: an earlier capacity query may have left a smaller limit
    e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(n_clusters * cl);
    cfg.blockDim = dim3(NT);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = cl;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, k, a);
}

}  // namespace lbk
