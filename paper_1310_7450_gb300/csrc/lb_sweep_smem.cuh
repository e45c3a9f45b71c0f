// lb_sweep_smem.cuh -- the batched sweep with the channel state resident in shared memory.
//
// Same contract as k_sweep (lb_sweep.cuh): one thread-block cluster of CL CTAs per channel runs
// that channel's time loop to a steady residual.  Here CTA r keeps its rows [y0, y1) of the
// populations, plus three halo rows on each side, in its own shared memory (two buffers), and the
// flow-induced density and the saved velocity of its nodes in registers.  Per step:
//   1. pull-stream (Eq. lbupdate; bounce-back at the walls) from the current buffer, moments of the
//      own rows and of two halo rows on each side (same-time gradients) -> shared velocity rows;
//   2. barrier; collision of the own rows into the other buffer;
//   3. cluster barrier; the halo rows of the new state are read from the neighbouring CTAs'
//      shared memory (distributed shared memory) -- the state never travels through L2 or HBM
//      inside the time loop;
//   4. every `check` steps the residual ||u(t) - u(t-k)|| / (k ||u(t)||) is reduced across the
//      cluster; on convergence, instability or max_steps the CTAs write their rows of the state and
//      their densities back to the channel's first buffer in HBM and leave.
// The host requires ny / CL >= 3 for every channel (halo rows come from the two neighbours only).
#pragma once

#include <cooperative_groups.h>

#include "lb_sweep.cuh"

namespace lbk {

// NX > 0: the handle's width as a compile-time constant (the node index arithmetic of every step
// becomes shifts and masks for NX = 4); NX = 0: any width, read from the arguments.
template <typename T, typename C, int NT, int NPT, int NX = 0>
// FP32 arithmetic: at most 128 registers (4 x 128 or 2 x 256 threads per SM; the width-4 kernel
// would otherwise keep its loop-invariant node indices in 254); FP64: unbounded, as before.
__global__ void __launch_bounds__(NT, sizeof(C) == 8 ? 1 : 512 / NT) k_sweep_smem(const SweepArgs<T, C> a) {
    constexpr int HR = 3;  // halo rows of populations on each side
    cg::cluster_group cluster = cg::this_cluster();
    const int CL = (int)cluster.num_blocks();
    const int rank = (int)cluster.block_rank();
    const int ch = a.order[blockIdx.x / CL];
    const ChanParams<C> P = a.chan[ch];
    const int nx = NX > 0 ? NX : a.nx, ny = P.ny, t = threadIdx.x;
    const int y0 = (int)((long long)ny * rank / CL), y1 = (int)((long long)ny * (rank + 1) / CL);
    const int yb = y0 - HR;                                  // global row of local row 0
    const int R = (y1 - y0) + 2 * HR;                        // local rows per buffer
    const int PS = R * nx;                                   // plane stride in shared memory
    const int ey0 = max(y0 - 2, 0), ey1 = min(y1 + 2, ny);   // rows whose gradient velocity we need
    const int n_own = (y1 - y0) * nx;

    extern __shared__ __align__(16) unsigned char smem[];
    T* buf0 = reinterpret_cast<T*>(smem);
    T* buf1 = buf0 + 9 * PS;
    const size_t pop_bytes = ((size_t)2 * 9 * PS * sizeof(T) + 15) / 16 * 16;
    C* su = reinterpret_cast<C*>(smem + pop_bytes);          // [ey1 - ey0][nx][2]
    __shared__ double part[2];
    __shared__ int done;

    T* gpop = a.popA + 9 * P.base;                           // the state at launch, and at exit
    C* gdr = a.drho + P.base;
    if (t == 0) done = 0;

    // load the own rows and the halo rows that exist
    const int ly0 = max(y0 - HR, 0) - yb, ly1 = min(y1 + HR, ny) - yb;
    for (int e = t; e < 9 * (ly1 - ly0) * nx; e += NT) {
        const int i = e / ((ly1 - ly0) * nx), rem = e % ((ly1 - ly0) * nx);
        const int lr = ly0 + rem / nx, x = rem % nx;
        buf0[i * PS + lr * nx + x] = gpop[(long long)i * P.P + (long long)(lr + yb) * nx + x];
    }
    C drv[NPT], upx[NPT], upy[NPT];
#pragma unroll
    for (int k = 0; k < NPT; ++k) {
        const int e = t + k * NT;
        drv[k] = e < n_own ? gdr[(long long)y0 * nx + e] : C(0);
        upx[k] = upy[k] = C(0);
    }
    cluster.sync();

    auto pull = [&](const T* cur, int y, int x, C (&d)[9]) {
#pragma unroll
        for (int i = 0; i < 9; ++i) {
            const int ys = y - cy(i);
            if (ys < 0 || ys >= ny) {
                d[i] = (C)Store<T>::cvt(cur[opp(i) * PS + (y - yb) * nx + x]);
            } else {
                int xs = x - cx(i);
                xs = xs < 0 ? xs + nx : (xs >= nx ? xs - nx : xs);
                d[i] = (C)Store<T>::cvt(cur[i * PS + (ys - yb) * nx + xs]);
            }
        }
    };

    long long s = 0;
    int dec = 0;
    for (; s < a.max_steps; ++s) {
        const T* cur = (s & 1) ? buf1 : buf0;
        T* nxt = (s & 1) ? buf0 : buf1;
        const bool save = ((s + 1) % a.check) == 0;
        const bool resid = save && (s + 1 >= 2 * (long long)a.check);

        // 1. own nodes (kept in registers) and halo rows -> gradient velocity in shared memory
        C d[NPT][9], dR[NPT], jx[NPT], jy[NPT];
#pragma unroll
        for (int k = 0; k < NPT; ++k) {
            const int e = t + k * NT;
            if (e < n_own) {
                const int y = y0 + e / nx, x = e % nx;
                C ux, uy;
                pull(cur, y, x, d[k]);
                gradient_velocity<C>(d[k], P.gx, dR[k], jx[k], jy[k], ux, uy);
                const int r = (y - ey0) * nx + x;
                su[2 * r] = ux;
                su[2 * r + 1] = uy;
            }
        }
        const int below = (y0 - ey0) * nx;
        const int n_halo = (ey1 - ey0) * nx - n_own;
        for (int e = t; e < n_halo; e += NT) {
            const int row = e < below ? ey0 + e / nx : y1 + (e - below) / nx;
            const int x = e % nx;
            C dh[9], hR, hx, hy, ux, uy;
            pull(cur, row, x, dh);
            gradient_velocity<C>(dh, P.gx, hR, hx, hy, ux, uy);
            const int r = (row - ey0) * nx + x;
            su[2 * r] = ux;
            su[2 * r + 1] = uy;
        }
        __syncthreads();

        // 2. collide the own nodes into the other buffer
        C r0 = C(0), r1 = C(0);
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
                const NodeState<C> st = constitutive<C, 0>(P, ka, kb, kc, ke, dR[k], jx[k], jy[k], drv[k], C(0), C(0), C(0));
                const C rho_h = C(1) + st.dReq - st.drho;
                if (!velocity_ok<C>(jx[k], jy[k], rho_h, (C)0.3)) atomicOr(a.status + ch, 1);
                C D[9];
                collide_node<C>(P, st, d[k], D);
                const long long pn = (long long)y * nx + x;
                store_node<T, C>(nxt + (y - yb) * nx + x, PS, d[k], D, a.sr,
                                 mix32(a.sr_key ^ (uint32_t)(s * 0x9E3779B9ull) ^ (uint32_t)(ch * 0x85EBCA6Bu)), (uint32_t)pn);
                drv[k] = st.drho;
                if (save) {
                    const C ih = Arith<C>::div(C(1), rho_h);
                    const C urx = jx[k] * ih, ury = jy[k] * ih;
                    if (resid) {
                        const C dx_ = urx - upx[k], dy_ = ury - upy[k];
                        r0 += dx_ * dx_ + dy_ * dy_;
                        r1 += urx * urx + ury * ury;
                    }
                    upx[k] = urx;
                    upy[k] = ury;
                }
            }
        }
        if (resid) {
            double v0 = (double)r0, v1 = (double)r1;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                v0 += __shfl_xor_sync(0xffffffffu, v0, o);
                v1 += __shfl_xor_sync(0xffffffffu, v1, o);
            }
            if (t == 0) { part[0] = 0.0; part[1] = 0.0; }
            __syncthreads();
            if ((t & 31) == 0) {
                atomicAdd(&part[0], v0);
                atomicAdd(&part[1], v1);
            }
        }
        // 3. every CTA of the channel has written step s+1 into its own rows of `nxt`; read the
        //    halo rows of `nxt` from the neighbours (ny / CL >= 3: they own all three)
        cluster.sync();
        {
            const int nb_lo = y0 > 0 ? HR : 0;                 // halo rows below the own rows
            const int nb_hi = y1 < ny ? HR : 0;                // and above
            const int n_copy = 9 * (nb_lo + nb_hi) * nx;  // element e: column e % nx, then
                                                          // direction (e / nx) % 9, halo row (e / nx) / 9
            // a neighbour's buffers start at the same shared-memory offset as ours, but its plane
            // stride follows its own row count
            const bool second = (s & 1) == 0;                  // `nxt` is the second buffer
            const T* nxt_lo = nullptr;
            const T* nxt_hi = nullptr;
            int yb_lo = 0, yb_hi = 0, PS_lo = 0, PS_hi = 0;
            if (nb_lo) {
                const int y0_lo = (int)((long long)ny * (rank - 1) / CL);
                yb_lo = y0_lo - HR;
                PS_lo = ((y0 - y0_lo) + 2 * HR) * nx;
                const T* base = cluster.map_shared_rank(buf0, rank - 1);
                nxt_lo = second ? base + 9 * PS_lo : base;
            }
            if (nb_hi) {
                const int y1_hi = (int)((long long)ny * (rank + 2) / CL);
                yb_hi = y1 - HR;                               // the upper neighbour starts at y1
                PS_hi = ((y1_hi - y1) + 2 * HR) * nx;
                const T* base = cluster.map_shared_rank(buf0, rank + 1);
                nxt_hi = second ? base + 9 * PS_hi : base;
            }
            for (int e = t; e < n_copy; e += NT) {
                const int x = e % nx, q = e / nx;
                const int i = q % 9, hr = q / 9;
                if (hr < nb_lo) {
                    const int y = y0 - HR + hr;
                    nxt[i * PS + (y - yb) * nx + x] = nxt_lo[i * PS_lo + (y - yb_lo) * nx + x];
                } else {
                    const int y = y1 + (hr - nb_lo);
                    nxt[i * PS + (y - yb) * nx + x] = nxt_hi[i * PS_hi + (y - yb_hi) * nx + x];
                }
            }
        }
        // 4. residual decision (rank 0), broadcast through distributed shared memory
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
                done = unstable ? 2 : (r <= a.tol ? 1 : 0);
                a.res_out[ch] = r;
            }
            cluster.sync();
            dec = *cluster.map_shared_rank(&done, 0);
        }
        // the next step's pulls read the halo rows written above (and, after a decision, the
        // write-back reads `nxt`)
        __syncthreads();
        if (dec) {
            ++s;
            break;
        }
    }
    // write the state after step s back to the first buffer of the channel in HBM
    const T* fin = (s & 1) ? buf1 : buf0;
    for (int e = t; e < 9 * n_own; e += NT) {
        const int i = e / n_own, rem = e % n_own;
        gpop[(long long)i * P.P + (long long)y0 * nx + rem] = fin[i * PS + HR * nx + rem];
    }
#pragma unroll
    for (int k = 0; k < NPT; ++k) {
        const int e = t + k * NT;
        if (e < n_own) {
            gdr[(long long)y0 * nx + e] = drv[k];
            C* up = a.uprev + 2 * P.base;
            up[(long long)y0 * nx + e] = upx[k];
            up[P.P + (long long)y0 * nx + e] = upy[k];
        }
    }
    if (rank == 0 && t == 0) a.steps_out[ch] = dec == 2 ? -2 : (dec == 1 ? s : -1);
    cluster.sync();  // no CTA leaves while another may still read its shared memory
}

// Dynamic shared memory of k_sweep_smem for a CTA owning `rows` rows.
template <typename T, typename C>
constexpr size_t sweep_smem_bytes(int rows, int nx) {
    return ((size_t)2 * 9 * (rows + 6) * nx * sizeof(T) + 15) / 16 * 16 + (size_t)(rows + 4) * nx * 2 * sizeof(C);
}

// How many clusters of `cl` CTAs with `smem` bytes the device can hold at once (0: the shape cannot
// be co-scheduled, so it is never launched).
template <typename T, typename C, int NT, int NPT, int NX = 0>
cudaError_t launch_sweep_smem_capacity(int cl, size_t smem, int* n_clusters) {
    auto k = k_sweep_smem<T, C, NT, NPT, NX>;
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
cudaError_t launch_sweep_smem(const SweepArgs<T, C>& a, int n_clusters, int cl, size_t smem, cudaStream_t s) {
    auto k = k_sweep_smem<T, C, NT, NPT, NX>;
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    if (e != cudaSuccess) return e;
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
