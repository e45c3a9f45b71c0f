// lb_device.cuh -- device-side types and the per-node arithmetic of the nlM lattice-Boltzmann
// step (Papenkort & Voigtmann, arXiv:1310.7450, Sec. II and III A).
//
// Storage: populations are kept as deviations d_i = n_i - w_i from the rest equilibrium at unit
// density (FP64, FP32 or BF16); all arithmetic below works on deviations so that FP32 keeps the
// precision of the small quantities (sum_i w_i = 1 and sum_i c_i w_i = 0 make this exact).
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <type_traits>

namespace lbk {

// D2Q9 velocity set (Sec. II A).  Numbering: 0:(0,0) 1:(1,0) 2:(0,1) 3:(-1,0) 4:(0,-1)
// 5:(1,1) 6:(-1,1) 7:(-1,-1) 8:(1,-1).
__host__ __device__ constexpr int cx(int i) {
    return (i == 1 || i == 5 || i == 8) ? 1 : ((i == 3 || i == 6 || i == 7) ? -1 : 0);
}
__host__ __device__ constexpr int cy(int i) {
    return (i == 2 || i == 5 || i == 6) ? 1 : ((i == 4 || i == 7 || i == 8) ? -1 : 0);
}
__host__ __device__ constexpr int opp(int i) {
    return i == 0 ? 0 : (i == 1 ? 3 : (i == 2 ? 4 : (i == 3 ? 1 : (i == 4 ? 2 : (i == 5 ? 7 : (i == 6 ? 8 : (i == 7 ? 5 : 6)))))));
}
// lattice weights a^{c_i}: 4/9, 1/9, 1/36
template <typename C>
__host__ __device__ constexpr C wgt(int i) {
    return i == 0 ? C(4) / C(9) : (i < 5 ? C(1) / C(9) : C(1) / C(36));
}

// ---- storage precision ---------------------------------------------------------------------
// Two-component vector of an arithmetic type (8- or 16-byte accesses of (x, y) pairs).
template <typename C> struct Vec2;
template <> struct Vec2<float> { using type = float2; };
template <> struct Vec2<double> { using type = double2; };

template <typename T> struct Store;
template <> struct Store<double> {
    using C = double;
    static __device__ __forceinline__ double cvt(double v) { return v; }
    static __device__ __forceinline__ double ld(const double* p) { return __ldg(p); }
    static __device__ __forceinline__ void st(double* p, double v) { *p = v; }
};
template <> struct Store<float> {
    using C = float;
    static __device__ __forceinline__ float cvt(float v) { return v; }
    static __device__ __forceinline__ float ld(const float* p) { return __ldg(p); }
    static __device__ __forceinline__ void st(float* p, float v) { *p = v; }
};
template <> struct Store<__nv_bfloat16> {
    using C = float;
    static __device__ __forceinline__ float cvt(__nv_bfloat16 v) { return __bfloat162float(v); }
    static __device__ __forceinline__ float ld(const __nv_bfloat16* p) { return __bfloat162float(__ldg(p)); }
    static __device__ __forceinline__ void st(__nv_bfloat16* p, float v) { *p = __float2bfloat16_rn(v); }
};

// Stochastic rounding of an FP32 value to BF16: add 16 uniformly random bits below the BF16
// mantissa and truncate, which rounds the magnitude up with probability equal to the discarded
// fraction, so the expected stored value is v (unbiased; round-to-nearest would drop every increment
// smaller than half a BF16 step).  Inf/NaN go through the ordinary conversion.
__device__ __forceinline__ __nv_bfloat16 bf16_stochastic(float v, uint32_t r16) {
    uint32_t b = __float_as_uint(v);
    if ((b & 0x7f800000u) == 0x7f800000u) return __float2bfloat16_rn(v);
    b += (r16 & 0xffffu);
    return __ushort_as_bfloat16((unsigned short)(b >> 16));
}

// 32-bit integer mixer ("lowbias32" of C. Wellons' hash-prospector, public domain) used as a
// counter-based generator: mix32(key ^ counter).
__device__ __forceinline__ uint32_t mix32(uint32_t x) {
    x ^= x >> 16;
    x *= 0x7feb352du;
    x ^= x >> 15;
    x *= 0x846ca68bu;
    x ^= x >> 16;
    return x;
}

// Store the nine post-collision deviations d + D of one node (node = its index in the channel
// planes).  BF16 storage with stochastic rounding draws 16 random bits per value from
// mix32(key ^ (5 node + pair)); `key` changes every step.
template <typename T, typename C>
__device__ __forceinline__ void store_node(T* po, long long P, const C (&d)[9], const C (&D)[9], bool sr, uint32_t key,
                                           uint32_t node) {
    if constexpr (std::is_same<T, __nv_bfloat16>::value) {
        if (sr) {
            uint32_t h = 0;
#pragma unroll
            for (int i = 0; i < 9; ++i) {
                if ((i & 1) == 0) h = mix32(key ^ (node * 5u + (uint32_t)(i >> 1)));
                po[(long long)i * P] = bf16_stochastic((float)(d[i] + D[i]), (i & 1) ? (h >> 16) : (h & 0xffffu));
            }
            return;
        }
    }
#pragma unroll
    for (int i = 0; i < 9; ++i) Store<T>::st(po + (long long)i * P, d[i] + D[i]);
}

// ---- launch descriptors ----------------------------------------------------------------------
// Per-channel constants, precomputed on the host in the arithmetic type C.
template <typename C>
struct ChanParams {
    long long base;      // plane offset: channel planes start at k*base (k planes per field)
    long long P;         // plane stride (elements), >= nx*ny, padded
    long long node_off;  // compact node offset of the channel (field outputs)
    int ny;
    int gpbc;     // 1: generalized periodic boundaries along x (pressure-driven, Sec. II B)
    int row_off;  // first row of the channel in the stacked boundary-column arrays (GPBC)
    int moving;   // 1: the last row lies on a wall moving with (u_wall, 0) (Zou-He, Sec. IV C)
    int scheme;   // 0: the paper's forcing; 1: generalized Newtonian; 2: div Sigma^nN as a force
    C omega;    // 1/tau_LB (BGK)
    C k1;       // -1/(2 c_s^4 tau_LB) = -9/(2 tau_LB): traceless-stress line of Eq. (bodyforce)
    C k2;       // 1 - 1/(2 tau_LB)
    C gx;       // body force density f^ex_x
    C G;        // G_inf
    C tau;      // theta * tau0
    C inv_gc;   // 1/gamma_c (0 = no shear thinning)
    C cD;       // eta_inf - eta^N = G tau0 - rho0 (tau_LB - 1/2)/3: Sigma^nN = sigma + cD D
    C kdr;      // 1 with the flow-induced density of Eq. (rhoplus); 0 under GPBC (Sec. II B)
    C rho0_m1;  // rho0 - 1
    C rho_in;   // GPBC: c_s^-2 p_+ - 1 at the inlet ghost column x = -1 (densities near 1 are kept
    C rho_out;  //       as offsets from 1, like the populations); c_s^-2 p_- - 1 at x = nx
    C u_wall;   // tangential velocity of the moving wall (moving == 1)
    C gn_a;     // scheme 1: tau_LB(gdot) = gn_b + gn_a tau_M, gn_a = G_inf / (rho0 c_s^2)
    C gn_b;     //           gn_b = 1/2 + eta_inf / (rho0 c_s^2)  (Eq. taulb with eta_eff)
    C beta_rho; // scheme 3: tau(rho) = tau exp(beta_rho (rho - rho_ref) / rho_ref)
    C rho_ref;
    C tau_f;    // scheme 3: memory time of the fluidity 1/tau_M (0: Eq. nlmaxwell, instantaneous)
};

struct WorkItem {
    int ch;   // channel
    int x0;   // first column
    int nxt;  // columns (== nx: full-width tile, x wraps inside the tile)
    int y0;   // first row
    int nyt;  // rows (>= 2, or the whole channel)
    int pad_[3];
};

enum : int {
    F_FIELDS = 1,       // compute the fields of the state only (no population/state writes)
    F_STORE_SIGMA = 2,  // write the sigma xx, yy, xy planes this step (zz = 0 is written at create)
    F_SAVE_U = 4,       // write the reported velocity into the u_prev planes
    F_RESID = 8,        // accumulate the residual against u_prev (block partials)
    F_SR = 16,          // BF16 storage: stochastic rounding of the populations
    F_MON = 32,         // accumulate flux and max |u| only (block partials; no u_prev read)
    F_SNN = 64,         // scheme 2, first pass: write Sigma^nN (xx, xy, yy) only (no state writes)
    F_DIV = 128,        // scheme 2, second pass: add div Sigma^nN of the written planes as a force
};

template <typename T, typename C>
struct StepArgs {
    const T* __restrict__ pin;     // populations of the stored state (deviations)
    T* __restrict__ pout;          // populations after this step
    C* __restrict__ drho;          // delta rho of the last collision [plane]
    C* __restrict__ sig3;          // carried stress (xx, xy, yy) [3 planes], stress mode 1
    C* __restrict__ sig4;          // stress output (xx, yy, zz, xy) [4 planes]
    C* __restrict__ uprev;         // saved velocity [2 planes]
    C* __restrict__ fu;            // fields-only outputs, compact node order: u [node][2]
    C* __restrict__ fsig;          //   sigma [node][4]
    C* __restrict__ frho;          //   rho [node]
    double* __restrict__ partials; // residual partials [item][4]
    C* __restrict__ snn;           // scheme 2: Sigma^nN (xx, xy, yy) of this step [3 planes]
    double* __restrict__ phi;      // scheme 3: fluidity 1/tau_M of the last step [plane] (0: unset),
                                   // FP64 in every precision (see relaxation_time_ext)
    const WorkItem* __restrict__ items;
    const ChanParams<C>* __restrict__ chan;
    int* __restrict__ status;      // per channel: 0 stable, 1 unstable
    int nx;
    int flags;
    C guard;                       // |u| above which a channel is declared unstable
    uint32_t sr_key;               // per-step key of the stochastic rounding (F_SR)
    const C* __restrict__ gcol;    // GPBC boundary columns of pin (null: periodic x), layout
                                   // [comp rho - 1, jx, jy][col 0: x = 0, 1: x = nx-1][row], then
                                   // the column means of rho - 1 [channel][col]
    int gny;                       // rows of all channels (the row stride of gcol)
};

// ---- per-node arithmetic -------------------------------------------------------------------

// Division and square root: exact IEEE operations in FP64 (the parity mode); in FP32 the PTX
// approximations rcp.approx.ftz and rsqrt.approx.ftz (one hardware instruction each, about 1 ulp;
// the .ftz forms skip the subnormal handling) -- every denominator here is a density near 1 or a
// positive quantity in the normal range, and the FP32 path's parity bound is 1e-5.  The square
// root returns 0 below the smallest normal float: sqrt(x) < 1.1e-19 there, which no quantity it
// enters (1 + tau sqrt(II)/gamma_c) can resolve.
template <typename C> struct Arith;
template <> struct Arith<double> {
    static __device__ __forceinline__ double div(double a, double b) { return a / b; }
    static __device__ __forceinline__ double sqrt(double x) { return ::sqrt(x); }
    static __device__ __forceinline__ double exp(double x) { return ::exp(x); }
};
#ifdef LBK_FP32_IEEE
// Compile-time alternative: correctly rounded FP32 division and square root (IEEE round to
// nearest even), for measuring what the approximations cost in parity and in throughput.
template <> struct Arith<float> {
    static __device__ __forceinline__ float div(float a, float b) { return __fdiv_rn(a, b); }
    static __device__ __forceinline__ float sqrt(float x) { return __fsqrt_rn(x); }
    static __device__ __forceinline__ float exp(float x) { return expf(x); }
};
#else
template <> struct Arith<float> {
    static __device__ __forceinline__ float rcp(float x) {
        float r;
        asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
        return r;
    }
    static __device__ __forceinline__ float div(float a, float b) { return a * rcp(b); }
    static __device__ __forceinline__ float sqrt(float x) {
        float r;
        asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
        return x >= 1.17549435e-38f ? x * r : 0.f;
    }
    static __device__ __forceinline__ float exp(float x) { return expf(x); }
};
#endif

// Moments of Eq. (rhoj) from the post-streaming deviations: dR = sum_i n_i - 1, J0 = sum c_i n_i.
template <typename C>
__device__ __forceinline__ void moments(const C (&d)[9], C& dR, C& jx, C& jy) {
    dR = ((d[0] + d[1]) + (d[2] + d[3])) + ((d[4] + d[5]) + (d[6] + d[7])) + d[8];
    jx = (d[1] - d[3]) + (d[5] - d[6]) + (d[8] - d[7]);
    jy = (d[2] - d[4]) + (d[5] + d[6]) - (d[7] + d[8]);
}

// Velocity used for the gradients (reading: j / R0 with R0 = sum_i n_i after streaming, because
// the density of Eq. (rhoj) needs S, which needs sigma(kappa)); one routine for the own node and
// the halo nodes so that both give bit-identical values.
template <typename C>
__device__ __forceinline__ void gradient_velocity(const C (&d)[9], C gx, C& dR, C& jx, C& jy, C& ux, C& uy) {
    moments<C>(d, dR, jx, jy);
    jx = jx + C(0.5) * gx;  // j = sum c n + f dt/2 (Eq. rhoj)
    const C inv = Arith<C>::div(C(1), C(1) + dR);
    ux = jx * inv;
    uy = jy * inv;
}

// Generalized periodic boundaries (Sec. II B, after Kim and Pitsch): a population that crosses
// the end of the channel is rebuilt from the node it leaves as n^eq_i(rho_s + delta, j_s) +
// n^neq*_i, with n^neq*_i = n*_i - n^eq_i(rho_s, j_s) and delta = rho_target - (column mean).
// With n^eq_i(rho, j) = w_i [rho + 3 c.j + (4.5 (c.j)^2 - 1.5 j^2) / rho] the rebuilt value is
// n*_i + w_i [delta - (4.5 (c.j)^2 - 1.5 j^2) delta / (rho_s (rho_s + delta))].  rho_s and j_s
// are the moments of the node's post-collision populations (the shortened forcing keeps both).
// The bracket depends only on the node left behind (its row, column and the direction), so a
// kernel may evaluate it once per boundary node and direction; gpbc_add applies it with one
// explicit fused multiply-add, which every kernel shares (bit-identical results whichever kernel
// evaluated the bracket).
template <typename C>
__device__ __forceinline__ C gpbc_shift_core(int i, C rho_s_m1, C jx, C jy, C delta) {
    const C rho_s = C(1) + rho_s_m1;
    const C cj = C(cx(i)) * jx + C(cy(i)) * jy;
    const C q = C(4.5) * cj * cj - C(1.5) * (jx * jx + jy * jy);
    return delta - q * Arith<C>::div(delta, rho_s * (rho_s + delta));
}
template <typename C>
__device__ __forceinline__ void gpbc_add(C& n, int i, C core) {
    if constexpr (sizeof(C) == 8) n = __fma_rn(wgt<C>(i), core, n);
    else n = __fmaf_rn(wgt<C>(i), core, n);
}

// Moving wall on the last row (Zou and He): the populations arriving from beyond the wall
// (directions 4, 7, 8) follow from the wall velocity (u_wall, 0): density from the mass and
// wall-normal momentum of the six known populations, n_4 by bounce-back of the non-equilibrium
// part, n_7 and n_8 from the tangential momentum rho u_wall.  On deviations the known weights sum
// to 1 and w_4 = w_2, w_7 = w_5, w_8 = w_6.
template <typename C>
__device__ __forceinline__ void zou_he_top(C (&d)[9], C u_wall) {
    const C rho = C(1) + (d[0] + d[1] + d[3] + C(2) * (d[2] + d[5] + d[6]));
    const C ht = C(0.5) * (d[1] - d[3]);
    const C hm = C(0.5) * rho * u_wall;
    d[4] = d[2];
    d[7] = d[5] + ht - hm;
    d[8] = d[6] - ht + hm;
}

// Polymer stress sigma = (xx, xy, yy) solving  s - alpha (kappa s + s kappa^T) = b  in closed
// form (Cramer's rule on the 3x3 system).  kappa = [[a, b], [c, e]] with kappa_ab = d_b u_a.
// Mode 0 (Eq. sigtsum, summed): alpha = tau_M, rhs = G tau_M D.  Mode 1 (backward Euler of
// Eq. gkder): alpha = tau_M/(tau_M+1), rhs = tau_M/(tau_M+1) (sigma_old + G D).
// det = (1 - alpha tr kappa)((1-2 alpha a)(1-2 alpha e) - 4 alpha^2 b c) is the product of
// 1 - alpha (lambda_i + lambda_j) over the eigenvalue pairs of kappa.
template <typename C>
__device__ __forceinline__ void convected_solve(C ka, C kb, C kc, C ke, C alpha, C b1, C b2, C b3,
                                                C& sxx, C& sxy, C& syy) {
    const C A = C(1) - C(2) * alpha * ka;
    const C E = C(1) - C(2) * alpha * ke;
    const C Pp = C(1) - alpha * (ka + ke);
    const C q = alpha * alpha * kb * kc;
    const C inv_det = Arith<C>::div(C(1), Pp * (A * E - C(4) * q));
    sxy = (alpha * kc * E * b1 + A * E * b2 + alpha * kb * A * b3) * inv_det;
    sxx = ((Pp * E - C(2) * q) * b1 + C(2) * alpha * kb * E * b2 + C(2) * alpha * alpha * kb * kb * b3) * inv_det;
    syy = (C(2) * alpha * alpha * kc * kc * b1 + C(2) * alpha * kc * A * b2 + (A * Pp - C(2) * q) * b3) * inv_det;
}

// Everything between the moments and the collision for one node (Sec. II A and III A):
// kappa -> tau_M (Eq. nlmaxwell) -> sigma -> Sigma^nN -> delta rho, S (Eq. rhoplus) ->
// rho_eq, u (reading: sum n^eq = sum (n*+n)/2 = R0 + S/2, so that sum (Delta + F) = S).
template <typename C>
struct NodeState {
    C sxx, sxy, syy;   // polymer stress
    C Bxx, Bxy;        // traceless Sigma^nN (Byy = -Bxx)
    C drho, S;         // delta rho(t), S = delta rho(t) - delta rho(t-1)
    C dReq;            // rho_eq - 1
    C ux, uy;          // velocity handed to n^eq and F_i: j / rho_eq
};

// TAUM = true: the relaxation time comes in as tau_M_in (the relaxation-time extensions of
// scheme 3) instead of Eq. (nlmaxwell) with the channel's tau.
template <typename C, int SMODE, bool TAUM = false>
__device__ __forceinline__ NodeState<C> constitutive(const ChanParams<C>& P, C ka, C kb, C kc, C ke,
                                                     C dR, C jx, C jy, C drho_prev,
                                                     C s_old_xx, C s_old_xy, C s_old_yy, C tau_M_in = C(0)) {
    NodeState<C> r;
    const C Dxx = C(2) * ka, Dxy = kb + kc, Dyy = C(2) * ke;
    C tau_M;
    if constexpr (TAUM) {
        tau_M = tau_M_in;
    } else {
        const C II = C(0.5) * (Dxx * Dxx + C(2) * Dxy * Dxy + Dyy * Dyy);  // (1/2) tr D^2
        // tau = 0 (Newtonian) gives tau_M = 0, alpha = 0 and a zero right-hand side, so sigma = 0
        tau_M = Arith<C>::div(P.tau, C(1) + P.tau * Arith<C>::sqrt(II) * P.inv_gc);
    }
    {
        if (SMODE == 0) {
            const C gt = P.G * tau_M;
            convected_solve<C>(ka, kb, kc, ke, tau_M, gt * Dxx, gt * Dxy, gt * Dyy, r.sxx, r.sxy, r.syy);
        } else {
            const C pre = Arith<C>::div(tau_M, tau_M + C(1));
            convected_solve<C>(ka, kb, kc, ke, pre, pre * (s_old_xx + P.G * Dxx), pre * (s_old_xy + P.G * Dxy),
                               pre * (s_old_yy + P.G * Dyy), r.sxx, r.sxy, r.syy);
        }
    }
    const C Nxx = r.sxx + P.cD * Dxx;
    const C Nxy = r.sxy + P.cD * Dxy;
    const C Nyy = r.syy + P.cD * Dyy;
    const C T = Nxx + Nyy;
    r.drho = P.kdr * (C(-1.5) * T);   // -tr Sigma^nN / (c_s^2 d), d = 2 (none under GPBC)
    r.S = r.drho - P.kdr * drho_prev; // dt d_t delta rho (Eq. rhoplus)
    r.Bxx = C(0.5) * (Nxx - Nyy);
    r.Bxy = Nxy;
    r.dReq = dR + C(0.5) * r.S;
    const C inv = Arith<C>::div(C(1), C(1) + r.dReq);
    r.ux = jx * inv;
    r.uy = jy * inv;
    return r;
}

// Scheme 1 (generalized Newtonian, the first alternative of Sec. II C): a locally Newtonian fluid
// whose viscosity is the model's effective viscosity in steady shear, eta_eff = G tau_M + eta_inf,
// through Eq. (taulb): tau_LB = 1/2 + eta_eff/(rho0 c_s^2).  No stress line, no flow-induced
// density; the reported stress is G tau_M D.  Returns the node's 1/tau_LB in *omega.
template <typename C>
__device__ __forceinline__ NodeState<C> constitutive_gn(const ChanParams<C>& P, C ka, C kb, C kc, C ke, C dR, C jx,
                                                        C jy, C* omega) {
    NodeState<C> r;
    const C Dxx = C(2) * ka, Dxy = kb + kc, Dyy = C(2) * ke;
    const C II = C(0.5) * (Dxx * Dxx + C(2) * Dxy * Dxy + Dyy * Dyy);
    const C tau_M = Arith<C>::div(P.tau, C(1) + P.tau * Arith<C>::sqrt(II) * P.inv_gc);
    const C gt = P.G * tau_M;
    r.sxx = gt * Dxx;
    r.sxy = gt * Dxy;
    r.syy = gt * Dyy;
    r.Bxx = r.Bxy = C(0);
    r.drho = r.S = C(0);
    r.dReq = dR;
    const C inv = Arith<C>::div(C(1), C(1) + dR);
    r.ux = jx * inv;
    r.uy = jy * inv;
    *omega = Arith<C>::div(C(1), P.gn_b + P.gn_a * tau_M);
    return r;
}

// Scheme 3, the relaxation-time extensions of the paper's outlook: the Maxwell time at the node's
// hydrodynamic density, tau(rho) = tau exp(beta_rho (rho_hat - rho_ref)/rho_ref) with rho_hat =
// R0 - delta rho(t-1) (the density known before the stress), and a fluidity phi = 1/tau_M that
// relaxes towards Eq. (nlmaxwell), phi_ss = 1/tau + II_D^{1/2}/gamma_c, with memory time tau_f
// (backward Euler: phi = (tau_f phi_old + phi_ss)/(tau_f + 1); phi_old = 0 means unset: phi_ss).
// Returns tau_M; *phi receives the new fluidity (0 without memory).  The fluidity and its recursion
// are FP64 in every precision: each step moves phi by 1/(tau_f + 1) of its distance to phi_ss, and
// an FP32 phi would drop those increments once they fall below half a unit in its last place,
// stalling up to (tau_f + 1) ulp / 2 away from phi_ss (1e-4 relative at tau_f = 2000).
template <typename C>
__device__ __forceinline__ C relaxation_time_ext(const ChanParams<C>& P, C ka, C kb, C kc, C ke, C dR, C drho_prev,
                                                 double phi_old, double* phi) {
    C tau = P.tau;
    if (P.beta_rho != C(0) && tau > C(0)) {
        const C rho_hat = C(1) + dR - drho_prev;
        tau *= Arith<C>::exp(Arith<C>::div(P.beta_rho * (rho_hat - P.rho_ref), P.rho_ref));
    }
    const C Dxx = C(2) * ka, Dxy = kb + kc, Dyy = C(2) * ke;
    const C sII = Arith<C>::sqrt(C(0.5) * (Dxx * Dxx + C(2) * Dxy * Dxy + Dyy * Dyy));
    *phi = 0.0;
    if (P.tau_f > C(0) && tau > C(0)) {
        // 1/tau and the weight 1/(tau_f + 1) are formed in the arithmetic type (the FP32 reciprocal
        // in the FP32 modes: FP64 divisions on this part would bound the step), the recursion in FP64
        // as an increment, phi = phi_old + (phi_ss - phi_old) / (tau_f + 1) -- the same backward
        // Euler step, whose fixed point is phi_ss exactly whatever the rounding of the weight
        const double phi_ss = (double)Arith<C>::div(C(1), tau) + (double)sII * (double)P.inv_gc;
        const double w = (double)Arith<C>::div(C(1), P.tau_f + C(1));
        *phi = phi_old > 0.0 ? phi_old + (phi_ss - phi_old) * w : phi_ss;
        return Arith<C>::div(C(1), (C)*phi);
    }
    return Arith<C>::div(tau, C(1) + tau * sII * P.inv_gc);
}

// Collision increments D_i = Delta_i + F_i = F_i + (n^eq_i - n_i)/tau_LB, with n^eq of Eq. (neq)
// as an offset from w_i and F_i of Eq. (bodyforce).  Opposite directions share the parts that are
// even in c_i (E) and differ in the sign of the odd part (O):
//   E = w [ (dReq - 1.5 rq u^2)/tau + k2 S + 4.5 (rq (c.u)^2/tau + k2 Q:Y) + k1 Sbar:Q ],
//   O = w 3 (rq (c.u)/tau + k2 c.f),     D(+c) = E + O - d/tau,  D(-c) = E - O - d/tau,
// rq = rho_eq, Y = -S u u + u f + f u, k1 = -1/(2 c_s^4 tau_LB), k2 = 1 - 1/(2 tau_LB).
// In exact arithmetic the increments carry mass S and momentum f (the conditions below
// Eq. lbfab).  In FP32 the rounding of n^eq repeats identically every step of a near-steady flow
// and would act as a spurious force (~1e-11 per step against forces of ~1e-7), so three
// increments are closed from those conditions instead of being evaluated: direction 3 from the
// x momentum f_x, direction 4 from the y momentum 0, and the rest direction from the mass S.
// In exact arithmetic the closed values equal the evaluated ones.
// GEN = true (the comparison schemes): the node's own om = 1/tau_LB and k2 = 1 - om/2, and a force
// density (gx, fy) with a y component; GEN = false is the paper's scheme with the channel's
// constants and f = (g_x, 0).
template <typename C, bool GEN>
__device__ __forceinline__ void collide_impl(const ChanParams<C>& P, const NodeState<C>& s, const C (&d)[9], C (&D)[9],
                                             C om, C k2, C gx, C fy) {
    const C ux = s.ux, uy = s.uy;
    const C rq = C(1) + s.dReq;
    const C orq = om * rq;
    const C usq = ux * ux + uy * uy;
    C Yxx = -s.S * ux * ux + C(2) * ux * gx;
    C Yyy = -s.S * uy * uy;
    C Yxy = -s.S * ux * uy + uy * gx;
    if constexpr (GEN) {
        Yyy += C(2) * uy * fy;
        Yxy += ux * fy;
    }
    const C trY3 = (Yxx + Yyy) * (C(1) / C(3));
    const C base = om * (s.dReq - C(1.5) * rq * usq) + k2 * s.S;
    const C w1 = wgt<C>(1), w5 = wgt<C>(5);
    // (1, 3): c = +-(1, 0)
    {
        const C cu = ux;
        const C E = w1 * (base + C(4.5) * (orq * cu * cu + k2 * (Yxx - trY3)) + P.k1 * s.Bxx);
        const C O = w1 * C(3) * (orq * cu + k2 * gx);
        D[1] = E + O - om * d[1];
    }
    // (2, 4): c = +-(0, 1)
    {
        const C cu = uy;
        const C E = w1 * (base + C(4.5) * (orq * cu * cu + k2 * (Yyy - trY3)) - P.k1 * s.Bxx);
        C O = w1 * C(3) * (orq * cu);
        if constexpr (GEN) O = w1 * C(3) * (orq * cu + k2 * fy);
        D[2] = E + O - om * d[2];
    }
    // (5, 7): c = +-(1, 1)
    {
        const C cu = ux + uy;
        const C E = w5 * (base + C(4.5) * (orq * cu * cu + k2 * (Yxx + Yyy + C(2) * Yxy - trY3)) + C(2) * P.k1 * s.Bxy);
        C O = w5 * C(3) * (orq * cu + k2 * gx);
        if constexpr (GEN) O = w5 * C(3) * (orq * cu + k2 * (gx + fy));
        D[5] = E + O - om * d[5];
        D[7] = E - O - om * d[7];
    }
    // (8, 6): c = +-(1, -1)
    {
        const C cu = ux - uy;
        const C E = w5 * (base + C(4.5) * (orq * cu * cu + k2 * (Yxx + Yyy - C(2) * Yxy - trY3)) - C(2) * P.k1 * s.Bxy);
        C O = w5 * C(3) * (orq * cu + k2 * gx);
        if constexpr (GEN) O = w5 * C(3) * (orq * cu + k2 * (gx - fy));
        D[8] = E + O - om * d[8];
        D[6] = E - O - om * d[6];
    }
    // closures: sum c_x D = f_x, sum c_y D = f_y (0 in the paper's scheme), sum D = S
    const C d57 = D[5] - D[7];
    D[3] = D[1] + d57 + (D[8] - D[6]) - gx;
    if constexpr (GEN) D[4] = D[2] + d57 + (D[6] - D[8]) - fy;
    else D[4] = D[2] + d57 + (D[6] - D[8]);
    D[0] = s.S - (((D[1] + D[2]) + (D[3] + D[4])) + ((D[5] + D[6]) + (D[7] + D[8])));
}

template <typename C>
__device__ __forceinline__ void collide_node(const ChanParams<C>& P, const NodeState<C>& s, const C (&d)[9], C (&D)[9]) {
    collide_impl<C, false>(P, s, d, D, P.omega, P.k2, P.gx, C(0));
}

// |u| <= guard for the reported velocity j/rho_h without a division or square root (false for NaN).
template <typename C>
__device__ __forceinline__ bool velocity_ok(C jx, C jy, C rho_h, C guard) {
    return jx * jx + jy * jy <= guard * guard * rho_h * rho_h;
}


// Channel monitor from per-item partials (sum du^2, sum u^2, sum u_x, max |u|) of items [b, e):
// one warp, lane l adding items b+l, b+l+32, ... in order, then a fixed butterfly, so every kernel
// that forms it gives the same bits.  mon[0..3] = residual sqrt(sum du^2 / sum u^2) (-1 without
// it), mean flux per column, max |u|, state index; NaN diagnostics when the channel's status is
// set.  The partials are read through L2 (they may come from other CTAs of the same kernel).
__device__ __forceinline__ void monitor_reduce_warp(const double* partials, int b, int e, int status, double* mon,
                                                    int nx, long long state_index, int with_residual, int lane) {
    double s0 = 0.0, s1 = 0.0, s2 = 0.0, s3 = 0.0;
    constexpr int U = 8;  // items per lane loaded together (one round trip to L2 per batch)
    for (int k0 = b + lane; k0 < e; k0 += 32 * U) {
        double2 v[U][2];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int k = k0 + 32 * u;
            if (k < e) {
                v[u][0] = __ldcg(reinterpret_cast<const double2*>(partials + 4 * k));
                v[u][1] = __ldcg(reinterpret_cast<const double2*>(partials + 4 * k + 2));
            }
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            if (k0 + 32 * u < e) {
                s0 += v[u][0].x;
                s1 += v[u][0].y;
                s2 += v[u][1].x;
                s3 = fmax(s3, v[u][1].y);
            }
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        s0 += __shfl_xor_sync(0xffffffffu, s0, o);
        s1 += __shfl_xor_sync(0xffffffffu, s1, o);
        s2 += __shfl_xor_sync(0xffffffffu, s2, o);
        s3 = fmax(s3, __shfl_xor_sync(0xffffffffu, s3, o));
    }
    if (lane == 0) {
        const bool ok = status == 0;
        mon[0] = !ok ? NAN : (!with_residual ? -1.0 : (s1 > 0 ? sqrt(s0 / s1) : 0.0));
        mon[1] = ok ? s2 / nx : NAN;
        mon[2] = ok ? s3 : NAN;
        mon[3] = (double)state_index;
    }
}

}  // namespace lbk
