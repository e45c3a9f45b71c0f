// lb_step_tile.cuh -- the fused lattice-Boltzmann step over a 2-D tile of one channel.
//
// One CTA owns a tile (x0..x0+nxt-1, y0..y0+nyt-1) of one channel; one thread owns one node.
//   phase 1  pull-stream the 9 populations of the own node (Eq. lbupdate, pull form; half-way
//            bounce-back where the source lies beyond a wall, Sec. II B) and keep them in
//            registers; moments (Eq. rhoj) -> gradient velocity j/R0 into shared memory;
//   phase 2  the same moments for the one-node halo ring around the tile (recomputed from a
//            second ring of pulled sources, so the velocity gradient uses same-time neighbours);
//   phase 3  kappa by three-point differences from shared memory (central; one-sided second
//            order on the first/last fluid row), the nlM stress, Sigma^nN, delta rho, n^eq, F_i
//            and the BGK collision; store n*, delta rho, optional stress / velocity / residual.
// The comparison schemes of Sec. II C run here too: the generalized-Newtonian tau_LB(gdot)
// (scheme 1) and the divergence of Sigma^nN as a force density (scheme 2, two launches per step:
// F_SNN writes Sigma^nN of every node, then the step with F_DIV differentiates it); scheme 3 is
// the paper's forcing with the relaxation-time extensions (tau(rho), fluidity memory).
// A full-width tile (nxt == nx) wraps x inside the tile and needs no x halo.
#pragma once

#include "lb_device.cuh"

namespace lbk {

// Boundary data of one channel: GPBC columns (col == nullptr: periodic x) and the moving wall.
template <typename C>
struct GpbcView {
    const C* col;  // gcol + row_off: rho - 1 at [c * gny + y], jx at [(2 + c) * gny + y], jy at [(4 + c) * gny + y]
    int gny;
    C dplus;       // rho_in - mean rho of the outlet column (populations entering at x = 0)
    C dminus;      // rho_out - mean rho of the inlet column (populations entering at x = nx-1)
    int moving;    // 1: Zou-He moving wall on the last row
    C u_wall;
};

template <typename T, typename C>
__device__ __forceinline__ void pull9(const T* __restrict__ pc, long long P, int nx, int ny, int x, int y,
                                      C (&d)[9], const GpbcView<C>& g) {
#pragma unroll
    for (int i = 0; i < 9; ++i) {
        const int ys = y - cy(i);
        if (ys < 0 || ys >= ny) {
            d[i] = Store<T>::ld(pc + (long long)opp(i) * P + (long long)y * nx + x);
        } else {
            const int xr = x - cx(i);
            const int xs = xr < 0 ? xr + nx : (xr >= nx ? xr - nx : xr);
            d[i] = Store<T>::ld(pc + (long long)i * P + (long long)ys * nx + xs);
            if (g.col && xs != xr) {
                // crossing the end of the channel: rebuilt from the node it leaves (column
                // c = 1 for x = nx-1 when entering the inlet, c = 0 when entering the outlet)
                const int c = xr < 0 ? 1 : 0;
                gpbc_add<C>(d[i], i, gpbc_shift_core<C>(i, g.col[c * g.gny + ys], g.col[(2 + c) * g.gny + ys],
                                                        g.col[(4 + c) * g.gny + ys], xr < 0 ? g.dplus : g.dminus));
            }
        }
    }
    if (g.moving && y == ny - 1) zou_he_top<C>(d, g.u_wall);
}

template <typename C>
__device__ __forceinline__ C warp_sum(C v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
template <typename C>
__device__ __forceinline__ C warp_max(C v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

// Block size: NT threads; tile nxt*nyt <= NT.  SCHEME: 0 the paper's forcing; 1, 2 the comparison
// schemes (compile-time, so that the paper's instantiation carries none of their code).
template <typename T, typename C, int SMODE, int NT, int SCHEME = 0>
__global__ void __launch_bounds__(NT) k_step_tile(const StepArgs<T, C> a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* su = reinterpret_cast<C*>(smem_raw);  // [EY*EX][2] gradient velocity

    const WorkItem it = a.items[blockIdx.x];
    if (a.status[it.ch] != 0) return;  // retired channel (uniform for the CTA)
    const ChanParams<C> P = a.chan[it.ch];
    const int nx = a.nx, ny = P.ny;
    const bool full = (it.nxt == nx);
    const int EX = full ? nx : it.nxt + 2;
    const int ex0 = full ? 0 : 1;
    const int EY = it.nyt + 2;
    const int t = threadIdx.x;
    const int ntile = it.nxt * it.nyt;
    const T* pc = a.pin + 9 * P.base;
    GpbcView<C> gv{nullptr, 0, C(0), C(0), P.moving, P.u_wall};
    if (a.gcol && P.gpbc) {
        const C* means = a.gcol + 6LL * a.gny + 2 * it.ch;
        gv.col = a.gcol + P.row_off;
        gv.gny = a.gny;
        gv.dplus = P.rho_in - means[1];
        gv.dminus = P.rho_out - means[0];
    }

    // phase 1: own node
    const bool own = t < ntile;
    const int tx = own ? t % it.nxt : 0;
    const int ty = own ? t / it.nxt : 0;
    const int x = it.x0 + tx, y = it.y0 + ty;
    C d[9];
    C dR = C(0), jx = C(0), jy = C(0);
    if (own) {
        pull9<T, C>(pc, P.P, nx, ny, x, y, d, gv);
        C ux, uy;
        gradient_velocity<C>(d, P.gx, dR, jx, jy, ux, uy);
        const int e = (ty + 1) * EX + (tx + ex0);
        su[2 * e] = ux;
        su[2 * e + 1] = uy;
    }
    // phase 2: halo ring (rows y0-1 and y0+nyt; columns x0-1 and x0+nxt for split tiles)
    const int R = 2 * EX + (full ? 0 : 2 * it.nyt);
    for (int r = t; r < R; r += NT) {
        int ex, ey;
        if (r < EX) { ex = r; ey = 0; }
        else if (r < 2 * EX) { ex = r - EX; ey = EY - 1; }
        else { const int k = r - 2 * EX; ey = 1 + (k >> 1); ex = (k & 1) ? EX - 1 : 0; }
        const int hy = it.y0 - 1 + ey;
        C ux = C(0), uy = C(0);
        if (hy >= 0 && hy < ny) {
            int hx = full ? ex : it.x0 - 1 + ex;
            hx = hx < 0 ? hx + nx : (hx >= nx ? hx - nx : hx);
            C dh[9], hR, hjx, hjy;
            pull9<T, C>(pc, P.P, nx, ny, hx, hy, dh, gv);
            gradient_velocity<C>(dh, P.gx, hR, hjx, hjy, ux, uy);
        }
        const int e = ey * EX + ex;
        su[2 * e] = ux;
        su[2 * e + 1] = uy;
    }
    __syncthreads();

    C res_du2 = C(0), res_u2 = C(0), res_ux = C(0), res_umax = C(0);
    if (own) {
        // phase 3: velocity gradient kappa_ab = d_b u_a (three-point differences)
        const int ecx = tx + ex0, ecy = ty + 1;
        int exm, exp_;
        if (full) { exm = ecx == 0 ? EX - 1 : ecx - 1; exp_ = ecx == EX - 1 ? 0 : ecx + 1; }
        else { exm = ecx - 1; exp_ = ecx + 1; }
        const C* rowc = su + 2 * (ecy * EX);
        const C ka = C(0.5) * (rowc[2 * exp_] - rowc[2 * exm]);          // d_x u_x
        const C kc = C(0.5) * (rowc[2 * exp_ + 1] - rowc[2 * exm + 1]);  // d_x u_y
        C kb, ke;
        if (y == 0) {
            const C* r1 = su + 2 * ((ecy + 1) * EX + ecx);
            const C* r2 = su + 2 * ((ecy + 2) * EX + ecx);
            const C* r0 = su + 2 * (ecy * EX + ecx);
            kb = C(0.5) * (C(-3) * r0[0] + C(4) * r1[0] - r2[0]);
            ke = C(0.5) * (C(-3) * r0[1] + C(4) * r1[1] - r2[1]);
        } else if (y == ny - 1) {
            const C* r1 = su + 2 * ((ecy - 1) * EX + ecx);
            const C* r2 = su + 2 * ((ecy - 2) * EX + ecx);
            const C* r0 = su + 2 * (ecy * EX + ecx);
            kb = C(0.5) * (C(3) * r0[0] - C(4) * r1[0] + r2[0]);
            ke = C(0.5) * (C(3) * r0[1] - C(4) * r1[1] + r2[1]);
        } else {
            const C* rp = su + 2 * ((ecy + 1) * EX + ecx);
            const C* rm = su + 2 * ((ecy - 1) * EX + ecx);
            kb = C(0.5) * (rp[0] - rm[0]);
            ke = C(0.5) * (rp[1] - rm[1]);
        }
        const long long pn = (long long)y * nx + x;  // node inside the channel planes
        C* dr = a.drho + P.base;
        const C drho_prev = dr[pn];
        C so_xx = C(0), so_xy = C(0), so_yy = C(0);
        if (SMODE == 1) {
            const C* s3 = a.sig3 + 3 * P.base;
            so_xx = s3[pn];
            so_xy = s3[P.P + pn];
            so_yy = s3[2 * P.P + pn];
        }
        // the comparison schemes of Sec. II C use their own relaxation rate / force (collide_impl)
        C om = P.omega, k2 = P.k2, fx = P.gx, fy = C(0);
        NodeState<C> s;
        if constexpr (SCHEME == 1) {
            s = constitutive_gn<C>(P, ka, kb, kc, ke, dR, jx, jy, &om);
            k2 = C(1) - C(0.5) * om;
        } else if constexpr (SCHEME == 3) {
            double phi_new;
            const C tau_M = relaxation_time_ext<C>(P, ka, kb, kc, ke, dR, drho_prev, a.phi[P.base + pn], &phi_new);
            s = constitutive<C, SMODE, true>(P, ka, kb, kc, ke, dR, jx, jy, drho_prev, so_xx, so_xy, so_yy, tau_M);
            if (!(a.flags & F_FIELDS) && P.tau_f > C(0)) a.phi[P.base + pn] = phi_new;  // own node only
        } else {
            s = constitutive<C, SMODE>(P, ka, kb, kc, ke, dR, jx, jy, drho_prev, so_xx, so_xy, so_yy);
        }
        if (SCHEME == 2 && (a.flags & F_SNN)) {
            // scheme 2, first pass: Sigma^nN = sigma + (eta_inf - eta^N) D of every node of this step
            C* q = a.snn + 3 * P.base;
            q[pn] = s.sxx + P.cD * (C(2) * ka);
            q[P.P + pn] = s.sxy + P.cD * (kb + kc);
            q[2 * P.P + pn] = s.syy + P.cD * (C(2) * ke);
        } else {
        if (SCHEME == 2 && (a.flags & F_DIV)) {
            // scheme 2, second pass: f^nN = div Sigma^nN by three-point differences (central along
            // the periodic x axis and inside the channel, one-sided on the first and last row),
            // added to the force density in j (Eq. rhoj) and in the force terms of Eq. (bodyforce)
            const C* q = a.snn + 3 * P.base;
            const int xp = x + 1 == nx ? 0 : x + 1, xm = x == 0 ? nx - 1 : x - 1;
            auto at = [&](int comp, int yy, int xx) -> C { return q[comp * P.P + (long long)yy * nx + xx]; };
            auto ddy = [&](int comp) -> C {
                if (y == 0) return C(0.5) * (C(-3) * at(comp, 0, x) + C(4) * at(comp, 1, x) - at(comp, 2, x));
                if (y == ny - 1)
                    return C(0.5) * (C(3) * at(comp, ny - 1, x) - C(4) * at(comp, ny - 2, x) + at(comp, ny - 3, x));
                return C(0.5) * (at(comp, y + 1, x) - at(comp, y - 1, x));
            };
            const C fnx = C(0.5) * (at(0, y, xp) - at(0, y, xm)) + ddy(1);
            const C fny = C(0.5) * (at(1, y, xp) - at(1, y, xm)) + ddy(2);
            fx += fnx;
            fy += fny;
            jx += C(0.5) * fnx;
            jy += C(0.5) * fny;
            const C inv = Arith<C>::div(C(1), C(1) + s.dReq);
            s.ux = jx * inv;
            s.uy = jy * inv;
        }

        // reported fields: hydrodynamic density rho_eq - delta rho (Eq. rhoj), u = j / rho
        const C rho_h = C(1) + s.dReq - s.drho;
        if (!velocity_ok<C>(jx, jy, rho_h, a.guard)) atomicOr(a.status + it.ch, 1);  // NaN or too fast
        C urx = C(0), ury = C(0);
        if (a.flags & (F_FIELDS | F_SAVE_U | F_RESID | F_MON)) {
            const C ih = Arith<C>::div(C(1), rho_h);
            urx = jx * ih;
            ury = jy * ih;
        }

        if (a.flags & F_FIELDS) {
            const long long node = P.node_off + pn;
            a.fu[2 * node] = urx;
            a.fu[2 * node + 1] = ury;
            a.fsig[4 * node + 0] = s.sxx;
            a.fsig[4 * node + 1] = s.syy;
            a.fsig[4 * node + 2] = C(0);
            a.fsig[4 * node + 3] = s.sxy;
            a.frho[node] = rho_h;
        } else {
            C D[9];
            if constexpr (SCHEME != 0) collide_impl<C, true>(P, s, d, D, om, k2, fx, fy);
            else collide_node<C>(P, s, d, D);
            T* po = a.pout + 9 * P.base + pn;
            store_node<T, C>(po, P.P, d, D, (a.flags & F_SR) != 0, a.sr_key ^ (uint32_t)(it.ch * 0x9E3779B9u), (uint32_t)pn);
            dr[pn] = s.drho;
            if (SMODE == 1) {
                C* s3 = a.sig3 + 3 * P.base;
                s3[pn] = s.sxx;
                s3[P.P + pn] = s.sxy;
                s3[2 * P.P + pn] = s.syy;
            }
            if (a.flags & F_STORE_SIGMA) {  // (the zz plane holds 0 from lb_create on)
                C* s4 = a.sig4 + 4 * P.base;
                s4[pn] = s.sxx;
                s4[P.P + pn] = s.syy;
                s4[3 * P.P + pn] = s.sxy;
            }
        }
        if (a.flags & (F_RESID | F_SAVE_U | F_MON)) {
            C* up = a.uprev + 2 * P.base;
            if (a.flags & (F_RESID | F_MON)) {
                if (a.flags & F_RESID) {
                    const C dx_ = urx - up[pn], dy_ = ury - up[P.P + pn];
                    res_du2 = dx_ * dx_ + dy_ * dy_;
                }
                res_u2 = urx * urx + ury * ury;
                res_ux = urx;
                res_umax = Arith<C>::sqrt(res_u2);
            }
            if (a.flags & F_SAVE_U) {
                up[pn] = urx;
                up[P.P + pn] = ury;
            }
        }
        }  // not the Sigma^nN pass
    }
    if (a.flags & (F_RESID | F_MON)) {
        // block reduction of (sum du^2, sum u^2, sum u_x, max |u|) in double
        __shared__ double red[NT / 32][4];
        double v0 = warp_sum<double>((double)res_du2), v1 = warp_sum<double>((double)res_u2);
        double v2 = warp_sum<double>((double)res_ux), v3 = warp_max<double>((double)res_umax);
        const int w = t >> 5, l = t & 31;
        if (l == 0) { red[w][0] = v0; red[w][1] = v1; red[w][2] = v2; red[w][3] = v3; }
        __syncthreads();
        if (t == 0) {
            double s0 = 0, s1 = 0, s2 = 0, s3 = 0;
            for (int k = 0; k < NT / 32; ++k) { s0 += red[k][0]; s1 += red[k][1]; s2 += red[k][2]; s3 = fmax(s3, red[k][3]); }
            double* o = a.partials + 4 * (long long)blockIdx.x;
            o[0] = s0; o[1] = s1; o[2] = s2; o[3] = s3;
        }
    }
}

// GPBC boundary columns of the stored state: per node of the columns x = 0 and x = nx-1 the
// density (as rho - 1) and momentum of its post-collision populations, and per column the mean
// of rho - 1.  One thread per row, RB blocks of NT rows per (channel, column); each block writes
// its fixed-order partial sum, and the last block of a column to finish (a counter per column,
// reset by that block) adds the partials in block order -- the same value every step kernel
// sees, independent of the order in which blocks finish.  Channels without GPBC are skipped.
template <typename T, typename C, int NT>
__global__ void __launch_bounds__(NT) k_gpbc_columns(const T* __restrict__ pin, const ChanParams<C>* __restrict__ chan,
                                                     C* __restrict__ gcol, int nx, int gny, int RB,
                                                     double* __restrict__ gpart, unsigned* __restrict__ gcount) {
    const int cc = blockIdx.x / RB, rb = blockIdx.x % RB;   // cc = 2 * channel + column
    const int ch = cc >> 1, c = cc & 1;
    const ChanParams<C> P = chan[ch];
    const int nrb = (P.ny + NT - 1) / NT;
    if (!P.gpbc || rb >= nrb) return;
    const int x = c ? nx - 1 : 0;
    const int y = rb * NT + (int)threadIdx.x;
    double v = 0.0;
    if (y < P.ny) {
        const T* pc = pin + 9 * P.base;
        C d[9];
#pragma unroll
        for (int i = 0; i < 9; ++i) d[i] = Store<T>::ld(pc + (long long)i * P.P + (long long)y * nx + x);
        C dR, jx, jy;
        moments<C>(d, dR, jx, jy);
        C* col = gcol + P.row_off;
        col[c * gny + y] = dR;
        col[(2 + c) * gny + y] = jx;
        col[(4 + c) * gny + y] = jy;
        v = (double)dR;
    }
    __shared__ double red[NT];
    __shared__ bool last;
    red[threadIdx.x] = v;
    __syncthreads();
    for (int h = NT / 2; h > 0; h >>= 1) {
        if ((int)threadIdx.x < h) red[threadIdx.x] += red[threadIdx.x + h];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        gpart[(long long)cc * RB + rb] = red[0];
        __threadfence();
        last = atomicAdd(gcount + cc, 1u) == (unsigned)(nrb - 1);
    }
    __syncthreads();
    if (last && threadIdx.x == 0) {
        __threadfence();
        double sum = 0.0;
        for (int k = 0; k < nrb; ++k) sum += *(volatile double*)(gpart + (long long)cc * RB + k);
        gcol[6LL * gny + cc] = (C)(sum / (double)P.ny);
        gcount[cc] = 0u;
    }
}

}  // namespace lbk

namespace lbk {
template <typename T, typename C>
cudaError_t launch_gpbc_columns(const T* pin, const ChanParams<C>* chan, C* gcol, int n_ch, int nx, int gny,
                                int max_ny, double* gpart, unsigned* gcount, cudaStream_t s) {
    constexpr int NT = 256;
    const int RB = (max_ny + NT - 1) / NT;
    k_gpbc_columns<T, C, NT><<<2 * n_ch * RB, NT, 0, s>>>(pin, chan, gcol, nx, gny, RB, gpart, gcount);
    return cudaGetLastError();
}

// Host-side launcher, explicitly instantiated per storage type in lb_kernels_*.cu.
template <typename T, typename C, int SMODE, int SCHEME = 0>
cudaError_t launch_step_tile(const StepArgs<T, C>& a, int n_items, size_t smem, cudaStream_t s) {
    constexpr int NT = 256;
    auto k = k_step_tile<T, C, SMODE, NT, SCHEME>;
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    if (n_items > 0) k<<<n_items, NT, smem, s>>>(a);
    return cudaGetLastError();
}
}  // namespace lbk
