/*
 * lb_oracle.c -- plain, slow, FP64 CPU oracle of the non-Newtonian lattice-Boltzmann
 * scheme of Papenkort & Voigtmann, "Channel flow of a tensorial shear-thinning Maxwell
 * model: lattice Boltzmann simulations" (arXiv:1310.7450).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing on the product path may call this file: only the
 * tests, the smoke check and the CPU-baseline leg of the benchmark use it.  It shares no
 * code, header, table or constant with the CUDA library.
 *
 * What it computes, one node at a time, in the order of the paper (Sec. II):
 *   1. streaming half of Eq. (lbupdate), pull form:  n_i(r,t) = n*_i(r - c_i, t-1),
 *      with simple (half-way) bounce-back at the two channel walls (Sec. II B);
 *   2. moments of Eq. (rhoj):  R0 = sum_i n_i,  j = sum_i c_i n_i + f^ex/2;
 *   3. velocity-gradient tensor kappa by three-point finite differences (Sec. II C);
 *   4. relaxation time tau_M of Eq. (nlmaxwell);
 *   5. polymer stress sigma by summing the series Eq. (sigtsum) with the recursion of
 *      Eq. (smalld)  [stress mode 0, the inlM model of Sec. III A], or one backward-Euler
 *      step of Eq. (gkder) with the Maxwell memory term -sigma/tau_M [stress mode 1];
 *   6. Sigma^nN = sigma + eta_inf D - eta^N D (Sec. IV), delta rho = -tr Sigma^nN/(c_s^2 d)
 *      and its one-step change (Eq. rhoplus);
 *   7. equilibrium n^eq of Eq. (neq) with the D2Q9 velocities and weights;
 *   8. forcing term F_i of Eq. (bodyforce);
 *   9. BGK collision  n*_i = n_i - (n_i - n^eq_i)/tau_LB + F_i  (Sec. II A).
 *
 * Number representation: the populations are stored as their offsets from the lattice weights,
 * dn_i = n_i - w_i (the rest equilibrium at unit density), and every formula is evaluated on
 * those offsets (sum_i w_i = 1 and sum_i c_i w_i = 0 make the moments exact).  The formulas are
 * the paper's; only the FP64 rounding acts on the small part instead of on n_i ~ 0.1-0.4.
 *
 * Readings where the paper is silent or ambiguous (each repeated at its use):
 *   - the density handed to n^eq is rho_eq = R0 + S/2 with S = drho(t) - drho(t-1), which
 *     is the only choice that satisfies the zeroth-moment condition sum_i(Delta_i + F_i) = S
 *     stated below Eq. (lbfab); the hydrodynamic density of Eq. (rhoj) is rho_eq - drho(t);
 *   - kappa is taken from the same-time velocity j/R0 of the neighbours (explicit order:
 *     S needs sigma, which needs kappa);
 *   - II_D = (1/2) tr D^2 with the full D = kappa + kappa^T;
 *   - d = 2, sigma_zz = 0 (kappa has no z components, so every d^n_zz vanishes);
 *   - three-point differences: central in the interior and along the periodic x axis,
 *     one-sided second-order (-3u0+4u1-u2)/2 at the first and last fluid rows;
 *   - f^ex = (g_x, 0) is a constant force density (Sec. III B: pressure drop per length);
 *   - the coefficient of the n >= 2 terms of Sigma^nN is 1, as in Eq. (sigtsum).
 *
 * Pressure-driven channels (boundary = 1): the generalized periodic boundaries of Sec. II B
 * (Kim and Pitsch) replace the periodic wrap of the populations that cross x = -1/2 or
 * x = nx - 1/2; there is no body force and no flow-induced density (delta rho = 0, so
 * S = 0 and Eq. (bodyforce) keeps its first line only, as Sec. II B prescribes).  Readings:
 *   - the moments (rho_s, j_s) of the node a crossing population leaves are those of its
 *     post-collision populations (the shortened forcing has no zeroth or first moment, so the
 *     collision keeps sum n* = R0 and sum c n* = j);
 *   - the averaged lattice density of a boundary column is the plain mean over its rows of
 *     sum_i n*_i;
 *   - bounce-back takes precedence for populations whose source lies beyond a wall;
 *   - the velocity gradients use the periodic image of the velocity field along x.
 *
 * Planar Couette flow (top_wall = 1, Sec. II B and Sec. IV C): the last fluid row y = ny-1 lies
 * on a wall moving with (u_wall, 0); its three populations arriving from beyond the wall are
 * set by the construction of Zou and He instead of bounce-back: the density follows from the
 * mass and wall-normal momentum of the known populations, the normal population from the
 * bounce-back of its non-equilibrium part, the two diagonal ones from the wall's tangential
 * momentum.  The bottom wall stays the half-way bounce-back wall at y = -1/2, so the gap is
 * ny - 1/2.
 *
 * Comparison schemes (Sec. II C lists them as the usual alternatives to the paper's forcing;
 * scheme = 1, 2; periodic x, bounce-back walls and stress mode 0 only):
 *   scheme 1, generalized Newtonian: tau_LB follows Eq. (taulb) with the Newtonian viscosity
 *     replaced by the effective viscosity of the model in steady shear, eta_eff = G tau_M +
 *     eta_inf (tau_M of Eq. nlmaxwell at the node's shear rate), and F_i keeps only its body-force
 *     terms: no stress line, no flow-induced density.  The stress reported is G tau_M D (such a
 *     fluid has no normal-stress differences).
 *   scheme 2, divergence of the stress as a body force: the stress enters as the force density
 *     f^nN = div Sigma^nN (three-point differences as for kappa) instead of the stress line and
 *     the flow-induced density.  Explicit order as for the paper's scheme: kappa from j / R0 with
 *     j = J0 + f^ex/2, then sigma and Sigma^nN at every node, their divergence, then
 *     j = J0 + (f^ex + f^nN)/2 for n^eq and the force terms of Eq. (bodyforce) with f^ex + f^nN.
 *     (A divergence lagged by one step went unstable once Sigma^nN acted as a negative viscosity
 *     beyond -0.3 eta^N, and oscillated from step to step near tau_LB = 1/2.)
 *
 * Extensions of the relaxation time that the paper leaves for further study (Sec. III A: tau_M
 * influenced by earlier times, the fluidity models; conclusions: tau depending on the local
 * density).  The paper fixes neither form; the oracle takes these, both off by default:
 *   - tau(rho) = tau exp(beta_rho (rho_hat - rho_ref) / rho_ref), with rho_hat = R0 - drho(t-1)
 *     the hydrodynamic density known before the stress (explicit order; equal to rho_eq - drho(t)
 *     in a steady state);
 *   - fluidity memory: phi = 1/tau_M relaxes towards its instantaneous value of Eq. (nlmaxwell),
 *     phi_ss = 1/tau + II_D^{1/2}/gamma_c, with the memory time tau_f:  d phi/dt = (phi_ss - phi)/
 *     tau_f, stepped by backward Euler, phi(t) = (tau_f phi(t-1) + phi_ss(t)) / (tau_f + 1), i.e.
 *     phi(t) is an exponentially weighted history of phi_ss.  The state carries phi per node (0
 *     before the first step: start from phi_ss).  With stress mode 1 this is the integral
 *     generalized Maxwell model sigma(t) = int G(t,t') [-d_t' B(t,t')] dt' with
 *     d_t G(t,t') = -G/tau_M(t) and a non-instantaneous tau_M.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* D2Q9 velocity set and weights (Sec. II A, below Eq. neq).  The paper fixes the set; the
 * numbering 0:(0,0) 1:(1,0) 2:(0,1) 3:(-1,0) 4:(0,-1) 5:(1,1) 6:(-1,1) 7:(-1,-1) 8:(1,-1)
 * is ours. */
static const int ORC_CX[9] = {0, 1, 0, -1, 0, 1, -1, -1, 1};
static const int ORC_CY[9] = {0, 0, 1, 0, -1, 1, 1, -1, -1};
static const double ORC_W[9] = {4.0 / 9.0,  1.0 / 9.0,  1.0 / 9.0,  1.0 / 9.0, 1.0 / 9.0,
                                1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0};
static const double ORC_CS2 = 1.0 / 3.0; /* c_s^2 = c^2/3 with c = dx/dt = 1 */
static const double ORC_DIM = 2.0;       /* spatial dimension d */

typedef struct {
    double tau_lb;  /* BGK relaxation time tau_LB (Eq. taulb)                      */
    double g_x;     /* body-force density f^ex_x (lattice units)                    */
    double G_inf;   /* plateau modulus G_inf                                        */
    double tau0;    /* microscopic time tau_0;  eta_inf = G_inf tau_0 (Eq. Sigmamodel) */
    double theta;   /* tau / tau_0                                                  */
    double gamma_c; /* critical strain of Eq. (nlmaxwell); +inf switches thinning off */
    double rho0;    /* reference density in eta^N = rho0 c_s^2 (tau_LB - 1/2)       */
    int stress_mode;/* 0: instantaneous nlM (Eq. sigtsum); 1: backward Euler of Eq. (gkder) */
    int boundary;   /* 0: periodic x, body force g_x; 1: generalized periodic boundaries (GPBC) */
    double rho_in;  /* GPBC: c_s^-2 p_+ - 1, the lattice density imposed at the inlet (x = -1),
                       as an offset from 1 like the populations                              */
    double rho_out; /* GPBC: c_s^-2 p_- - 1 at the outlet (x = nx)                            */
    int top_wall;   /* 0: half-way bounce-back; 1: wall on row ny-1 moving with u_wall (Zou-He) */
    int scheme;     /* 0: the paper's forcing; 1: generalized Newtonian tau_LB; 2: div Sigma force */
    double u_wall;  /* tangential velocity of the moving wall                                   */
    double beta_rho;/* density dependence tau(rho) = tau exp(beta_rho (rho - rho_ref)/rho_ref)   */
    double rho_ref; /* reference density of tau(rho)                                             */
    double tau_f;   /* memory time of the fluidity 1/tau_M (0: instantaneous, Eq. nlmaxwell)      */
} orc_params;

/* the body-force density of Eq. (rhoj) / Eq. (bodyforce): none in a pressure-driven channel */
static double body_force(const orc_params *p) { return p->boundary == 1 ? 0.0 : p->g_x; }

/* ---------------------------------------------------------------------------------- */
/* Small 2x2 tensor helpers (plain, row-major t[a][b]).                                */
typedef struct { double t[2][2]; } mat2;

static mat2 mat2_zero(void) { mat2 m; memset(&m, 0, sizeof m); return m; }

/* kappa X + X kappa^T : the map that generates d^{n+1} from d^n (Eq. smalld). */
static mat2 upper_convect(const mat2 *kap, const mat2 *x) {
    mat2 r = mat2_zero();
    for (int a = 0; a < 2; ++a)
        for (int b = 0; b < 2; ++b) {
            double s = 0.0;
            for (int k = 0; k < 2; ++k) s += kap->t[a][k] * x->t[k][b] + x->t[a][k] * kap->t[b][k];
            r.t[a][b] = s;
        }
    return r;
}

static double mat2_maxabs(const mat2 *m) {
    double r = 0.0;
    for (int a = 0; a < 2; ++a)
        for (int b = 0; b < 2; ++b) r = fmax(r, fabs(m->t[a][b]));
    return r;
}

/* Largest |lambda_i + lambda_j| over the eigenvalues of kappa: the spectral radius of the
 * map X -> kappa X + X kappa^T, which decides whether the series of Eq. (sigtsum) converges. */
static double convect_spectral_radius(const mat2 *kap) {
    double tr = kap->t[0][0] + kap->t[1][1];
    double det = kap->t[0][0] * kap->t[1][1] - kap->t[0][1] * kap->t[1][0];
    double disc = tr * tr - 4.0 * det;
    if (disc >= 0.0) {
        double l1 = 0.5 * (tr + sqrt(disc)), l2 = 0.5 * (tr - sqrt(disc));
        return fmax(fmax(fabs(2.0 * l1), fabs(2.0 * l2)), fabs(l1 + l2));
    }
    /* complex pair tr/2 +- i w:  |2 lambda| = 2 sqrt(det),  |lambda1 + lambda2| = |tr| */
    return fmax(2.0 * sqrt(det), fabs(tr));
}

/* ---------------------------------------------------------------------------------- */
/* Eq. (neq): second-order equilibrium.  (The printed u_{i alpha} is read as u_alpha.)    */
void orc_equilibrium(double rho, double ux, double uy, double *neq) {
    for (int i = 0; i < 9; ++i) {
        double cu = ORC_CX[i] * ux + ORC_CY[i] * uy;
        double q_uu = (ORC_CX[i] * ORC_CX[i] - ORC_CS2) * ux * ux +
                      2.0 * ORC_CX[i] * ORC_CY[i] * ux * uy +
                      (ORC_CY[i] * ORC_CY[i] - ORC_CS2) * uy * uy;
        neq[i] = ORC_W[i] * rho * (1.0 + cu / ORC_CS2 + q_uu / (2.0 * ORC_CS2 * ORC_CS2));
    }
}

/* Eq. (neq) as an offset from the weights: n^eq_i - w_i = w_i [(rho - 1) + rho X_i] with
 * X_i = u.c_i/c_s^2 + Q_i:uu/(2 c_s^4); rho_m1 = rho - 1. */
void orc_equilibrium_offset(double rho_m1, double ux, double uy, double *dneq) {
    double rho = 1.0 + rho_m1;
    for (int i = 0; i < 9; ++i) {
        double cu = ORC_CX[i] * ux + ORC_CY[i] * uy;
        double q_uu = (ORC_CX[i] * ORC_CX[i] - ORC_CS2) * ux * ux +
                      2.0 * ORC_CX[i] * ORC_CY[i] * ux * uy +
                      (ORC_CY[i] * ORC_CY[i] - ORC_CS2) * uy * uy;
        double X = cu / ORC_CS2 + q_uu / (2.0 * ORC_CS2 * ORC_CS2);
        dneq[i] = ORC_W[i] * (rho_m1 + rho * X);
    }
}

/* Eq. (bodyforce) with dt = 1.  sbar = traceless Sigma^nN as (xx, xy, yy); ddrho = dt *
 * d_t(delta rho) = S; u = velocity; f = body-force density. */
void orc_forcing(double tau_lb, const double *sbar, double ddrho, const double *u,
                 const double *f, double *F) {
    double S[2][2] = {{sbar[0], sbar[1]}, {sbar[1], sbar[2]}};
    /* the tensor multiplying Q_i in the bracket: -S u u + (u f + f u) */
    double Y[2][2];
    for (int a = 0; a < 2; ++a)
        for (int b = 0; b < 2; ++b) Y[a][b] = -ddrho * u[a] * u[b] + (u[b] * f[a] + u[a] * f[b]);
    for (int i = 0; i < 9; ++i) {
        int c[2] = {ORC_CX[i], ORC_CY[i]};
        double s_q = 0.0, y_q = 0.0, fc = 0.0;
        for (int a = 0; a < 2; ++a) {
            fc += f[a] * c[a];
            for (int b = 0; b < 2; ++b) {
                double q = c[a] * c[b] - (a == b ? ORC_CS2 : 0.0);
                s_q += S[a][b] * q;
                y_q += Y[a][b] * q;
            }
        }
        double line1 = -1.0 / (2.0 * ORC_CS2 * ORC_CS2 * tau_lb) * s_q;
        double line2 = (1.0 - 1.0 / (2.0 * tau_lb)) *
                       (ddrho + fc / ORC_CS2 + y_q / (2.0 * ORC_CS2 * ORC_CS2));
        F[i] = ORC_W[i] * (line1 + line2);
    }
}

/* Eq. (nlmaxwell): 1/tau_M = 1/tau + II_D^{1/2}/gamma_c, written in the form that stays
 * finite at tau = 0 (theta = 0 gives tau_M = 0, i.e. no polymer stress). */
double orc_relaxation_time(double tau, double gamma_c, double II_D) {
    if (tau <= 0.0) return 0.0;
    double inv_gc = isinf(gamma_c) ? 0.0 : 1.0 / gamma_c;
    return tau / (1.0 + tau * sqrt(II_D) * inv_gc);
}

/* Eq. (sigtsum) with the recursion of Eq. (smalld):  sigma = sum_{n>=1} G tau_M^n d^n,
 * d^1 = D, d^{n+1} = kappa d^n + d^n kappa^T.  kappa = (xx, xy, yx, yy) with
 * kappa_ab = d_b u_a.  Returns the number of terms used, or -1 if the series does not
 * converge geometrically fast enough (tau_M * radius > 0.8). */
int orc_stress_series(const double *kappa, double tau_M, double G, double *out) {
    mat2 kap = {{{kappa[0], kappa[1]}, {kappa[2], kappa[3]}}};
    out[0] = out[1] = out[2] = 0.0;
    if (tau_M == 0.0) return 0;
    if (tau_M * convect_spectral_radius(&kap) > 0.8) return -1;
    mat2 dn; /* d^1 = D = kappa + kappa^T */
    for (int a = 0; a < 2; ++a)
        for (int b = 0; b < 2; ++b) dn.t[a][b] = kap.t[a][b] + kap.t[b][a];
    mat2 sum = mat2_zero();
    double taun = 1.0;
    int n;
    for (n = 1; n <= 200; ++n) {
        taun *= tau_M;
        mat2 term;
        for (int a = 0; a < 2; ++a)
            for (int b = 0; b < 2; ++b) {
                term.t[a][b] = G * taun * dn.t[a][b];
                sum.t[a][b] += term.t[a][b];
            }
        double tn = mat2_maxabs(&term), sn = mat2_maxabs(&sum);
        if (tn == 0.0 || tn <= 1e-17 * sn) break;
        dn = upper_convect(&kap, &dn);
    }
    out[0] = sum.t[0][0];
    out[1] = sum.t[0][1];
    out[2] = sum.t[1][1];
    return n;
}

/* Gaussian elimination (partial pivoting) of  s - alpha (kappa s + s kappa^T) = b  for a
 * symmetric 2x2 s = (xx, xy, yy).  The 3x3 matrix is assembled by applying the map to the
 * three basis tensors.  Used where the series is not convergent, and for stress mode 1. */
static int solve_convected(const mat2 *kap, double alpha, const double *b, double *s) {
    double M[3][4];
    mat2 basis[3] = {{{{1, 0}, {0, 0}}}, {{{0, 1}, {1, 0}}}, {{{0, 0}, {0, 1}}}};
    for (int k = 0; k < 3; ++k) {
        mat2 L = upper_convect(kap, &basis[k]);
        double col[3] = {basis[k].t[0][0] - alpha * L.t[0][0], basis[k].t[0][1] - alpha * L.t[0][1],
                         basis[k].t[1][1] - alpha * L.t[1][1]};
        for (int r = 0; r < 3; ++r) M[r][k] = col[r];
    }
    for (int r = 0; r < 3; ++r) M[r][3] = b[r];
    for (int p = 0; p < 3; ++p) {
        int piv = p;
        for (int r = p + 1; r < 3; ++r)
            if (fabs(M[r][p]) > fabs(M[piv][p])) piv = r;
        if (M[piv][p] == 0.0) return -1;
        if (piv != p)
            for (int k = 0; k < 4; ++k) { double t = M[p][k]; M[p][k] = M[piv][k]; M[piv][k] = t; }
        for (int r = p + 1; r < 3; ++r) {
            double m = M[r][p] / M[p][p];
            for (int k = p; k < 4; ++k) M[r][k] -= m * M[p][k];
        }
    }
    for (int r = 2; r >= 0; --r) {
        double acc = M[r][3];
        for (int k = r + 1; k < 3; ++k) acc -= M[r][k] * s[k];
        s[r] = acc / M[r][r];
    }
    return 0;
}

/* The steady-state equation behind Eq. (sigtsum): sigma/tau_M - kappa sigma - sigma
 * kappa^T = G D, solved directly (the series is its Neumann expansion). */
int orc_stress_gauss(const double *kappa, double tau_M, double G, double *out) {
    mat2 kap = {{{kappa[0], kappa[1]}, {kappa[2], kappa[3]}}};
    out[0] = out[1] = out[2] = 0.0;
    if (tau_M == 0.0) return 0;
    double b[3] = {G * tau_M * 2.0 * kappa[0], G * tau_M * (kappa[1] + kappa[2]),
                   G * tau_M * 2.0 * kappa[3]};
    return solve_convected(&kap, tau_M, b, out);
}

/* Stress mode 1: one backward-Euler step (dt = 1) of the upper-convected equation
 * Eq. (gkder) with the memory integral replaced by -sigma/tau_M (generalized Maxwell,
 * Sec. III A, time-dependent generalization):
 *   (1 + dt/tau_M) s' - dt (kappa s' + s' kappa^T) = s + dt G D.
 * Summed as the Neumann series s' = sum_n beta^n L^n(b') with beta = dt tau_M/(tau_M+dt),
 * b' = tau_M/(tau_M+dt) (s + dt G D); Gaussian elimination if that does not converge. */
int orc_stress_step(const double *kappa, double tau_M, double G, const double *s_old, double *out) {
    mat2 kap = {{{kappa[0], kappa[1]}, {kappa[2], kappa[3]}}};
    out[0] = out[1] = out[2] = 0.0;
    if (tau_M == 0.0) return 0; /* infinitely fast relaxation: no polymer stress */
    const double dt = 1.0;
    double beta = dt * tau_M / (tau_M + dt);
    double pre = tau_M / (tau_M + dt);
    double b[3] = {pre * (s_old[0] + dt * G * 2.0 * kappa[0]),
                   pre * (s_old[1] + dt * G * (kappa[1] + kappa[2])),
                   pre * (s_old[2] + dt * G * 2.0 * kappa[3])};
    if (beta * convect_spectral_radius(&kap) > 0.8) return solve_convected(&kap, beta, b, out) == 0 ? -1 : -2;
    /* (-1: the elimination fallback was used and out holds its result; -2: singular) */
    mat2 x = {{{b[0], b[1]}, {b[1], b[2]}}};
    mat2 sum = x;
    double bn = 1.0;
    for (int n = 1; n <= 200; ++n) {
        x = upper_convect(&kap, &x);
        bn *= beta;
        double tn = bn * mat2_maxabs(&x);
        for (int a = 0; a < 2; ++a)
            for (int c = 0; c < 2; ++c) sum.t[a][c] += bn * x.t[a][c];
        if (tn == 0.0 || tn <= 1e-17 * mat2_maxabs(&sum)) break;
    }
    out[0] = sum.t[0][0];
    out[1] = sum.t[0][1];
    out[2] = sum.t[1][1];
    return 0;
}

/* ---------------------------------------------------------------------------------- */
/* Whole-grid state: dn[i][y][x] = n*_i - w_i, offsets of the post-collision populations
 * from the weights; drho[y][x] = delta rho of the last collision; sig[3][y][x] the carried
 * polymer stress (xx, xy, yy) of stress mode 1 (unused in mode 0).                       */

static long orc_fallbacks = 0; /* series -> Gaussian elimination fallbacks (logged) */
long orc_fallback_count(void) { return orc_fallbacks; }
void orc_reset_fallback_count(void) { orc_fallbacks = 0; }

/* Initial state: every population at rest equilibrium n_i = w_i rho(r), i.e. offsets
 * w_i (rho - 1); no flow-induced density (drho = 0), no polymer stress. */
void orc_init(int nx, int ny, const double *rho, double *dn, double *drho, double *sig) {
    long N = (long)nx * ny;
    for (int i = 0; i < 9; ++i)
        for (long k = 0; k < N; ++k) dn[i * N + k] = ORC_W[i] * (rho[k] - 1.0);
    for (long k = 0; k < N; ++k) drho[k] = 0.0;
    if (sig)
        for (long k = 0; k < 3 * N; ++k) sig[k] = 0.0;
}

/* Per-node results of one update (everything the collision and the field output need). */
typedef struct {
    double R0m1, j[2];     /* zeroth moment after streaming minus 1, current j (Eq. rhoj) */
    double kap[4];         /* kappa (xx, xy, yx, yy)                                  */
    double tau_M;          /* Eq. (nlmaxwell)                                          */
    double sigma[3];       /* polymer stress (xx, xy, yy)                             */
    double sbar[3];        /* traceless part of Sigma^nN (xx, xy, yy)                 */
    double drho, S;        /* delta rho(t) and S = delta rho(t) - delta rho(t-1)       */
    double rho_eq_m1, u[2];/* density (minus 1) and velocity handed to n^eq           */
    double tau_lb;         /* relaxation time of this node's collision                */
    double snn[3];         /* Sigma^nN (xx, xy, yy)                                   */
    double phi;            /* fluidity 1/tau_M after this step's memory update (tau_f > 0) */
} node_result;

/* One backward-Euler step of the fluidity memory: d phi/dt = (phi_ss - phi)/tau_f (dt = 1). */
double orc_fluidity_step(double phi_old, double phi_ss, double tau_f) {
    if (tau_f <= 0.0 || !(phi_old > 0.0)) return phi_ss;
    return (tau_f * phi_old + phi_ss) / (tau_f + 1.0);
}

static inline long idx(int nx, int x, int y) { return (long)y * nx + x; }

/* Three-point finite difference of a field v along y at row y (reading of Sec. II C). */
static double ddy(const double *v, int nx, int ny, int x, int y, int comp) {
    if (y == 0)
        return 0.5 * (-3.0 * v[2 * idx(nx, x, 0) + comp] + 4.0 * v[2 * idx(nx, x, 1) + comp] -
                      v[2 * idx(nx, x, 2) + comp]);
    if (y == ny - 1)
        return 0.5 * (3.0 * v[2 * idx(nx, x, ny - 1) + comp] - 4.0 * v[2 * idx(nx, x, ny - 2) + comp] +
                      v[2 * idx(nx, x, ny - 3) + comp]);
    return 0.5 * (v[2 * idx(nx, x, y + 1) + comp] - v[2 * idx(nx, x, y - 1) + comp]);
}
/* ... and along the periodic x axis. */
static double ddx(const double *v, int nx, int x, int y, int comp) {
    int xp = (x + 1) % nx, xm = (x - 1 + nx) % nx;
    return 0.5 * (v[2 * idx(nx, xp, y) + comp] - v[2 * idx(nx, xm, y) + comp]);
}

/* The same three-point differences of a scalar field f[y][x] (scheme 2: the stress planes). */
static double plane_ddy(const double *f, int nx, int ny, int x, int y) {
    if (y == 0) return 0.5 * (-3.0 * f[idx(nx, x, 0)] + 4.0 * f[idx(nx, x, 1)] - f[idx(nx, x, 2)]);
    if (y == ny - 1) return 0.5 * (3.0 * f[idx(nx, x, ny - 1)] - 4.0 * f[idx(nx, x, ny - 2)] + f[idx(nx, x, ny - 3)]);
    return 0.5 * (f[idx(nx, x, y + 1)] - f[idx(nx, x, y - 1)]);
}
static double plane_ddx(const double *f, int nx, int x, int y) {
    int xp = (x + 1) % nx, xm = (x - 1 + nx) % nx;
    return 0.5 * (f[idx(nx, xp, y)] - f[idx(nx, xm, y)]);
}

/* Scheme 2: f^nN_a = d_b Sigma^nN_ab of the stored stress planes snn = (xx, xy, yy); out [2][N]. */
static void stress_divergence(int nx, int ny, const double *snn, double *out) {
    long N = (long)nx * ny;
    const double *sxx = snn, *sxy = snn + N, *syy = snn + 2 * N;
    for (int y = 0; y < ny; ++y)
        for (int x = 0; x < nx; ++x) {
            long k = idx(nx, x, y);
            out[k] = plane_ddx(sxx, nx, x, y) + plane_ddy(sxy, nx, ny, x, y);
            out[N + k] = plane_ddx(sxy, nx, x, y) + plane_ddy(syy, nx, ny, x, y);
        }
}

/* Steps 3-6 of the header, and the density / velocity of step 7, for node (x,y): needs the
 * moments R0 / j and gradient velocity ug of every node, drho_prev and the carried stress. */
static void node_update(const orc_params *p, int nx, int ny, int x, int y,
                        const double *R0m1, const double *j, const double *ug,
                        const double *drho_prev, const double *sig_prev, const double *phi_prev,
                        node_result *r) {
    long N = (long)nx * ny, k = idx(nx, x, y);
    r->R0m1 = R0m1[k];
    r->j[0] = j[2 * k];
    r->j[1] = j[2 * k + 1];
    /* kappa_ab = d_b u_a */
    r->kap[0] = ddx(ug, nx, x, y, 0);     /* d_x u_x */
    r->kap[1] = ddy(ug, nx, ny, x, y, 0); /* d_y u_x */
    r->kap[2] = ddx(ug, nx, x, y, 1);     /* d_x u_y */
    r->kap[3] = ddy(ug, nx, ny, x, y, 1); /* d_y u_y */
    double D[2][2] = {{2.0 * r->kap[0], r->kap[1] + r->kap[2]}, {r->kap[1] + r->kap[2], 2.0 * r->kap[3]}};
    double II_D = 0.0;
    for (int a = 0; a < 2; ++a)
        for (int b = 0; b < 2; ++b) II_D += 0.5 * D[a][b] * D[b][a];
    double tau = p->theta * p->tau0;
    if (p->beta_rho != 0.0 && tau > 0.0) { /* tau(rho) of the node's hydrodynamic density */
        double rho_hat = 1.0 + R0m1[k] - drho_prev[k];
        tau *= exp(p->beta_rho * (rho_hat - p->rho_ref) / p->rho_ref);
    }
    r->tau_M = orc_relaxation_time(tau, p->gamma_c, II_D);
    r->phi = 0.0;
    if (p->tau_f > 0.0 && tau > 0.0) { /* fluidity memory */
        double inv_gc = isinf(p->gamma_c) ? 0.0 : 1.0 / p->gamma_c;
        double phi_ss = 1.0 / tau + sqrt(II_D) * inv_gc;
        r->phi = orc_fluidity_step(phi_prev[k], phi_ss, p->tau_f);
        r->tau_M = 1.0 / r->phi;
    }
    r->tau_lb = p->tau_lb;
    if (p->scheme == 1) {
        /* generalized Newtonian: a locally Newtonian fluid with the effective viscosity of the
         * model in steady shear, eta_eff = G tau_M + eta_inf, through Eq. (taulb):
         * tau_LB = 1/2 + eta_eff / (rho0 c_s^2); the stress is G tau_M D, F_i has no stress line */
        r->sigma[0] = p->G_inf * r->tau_M * D[0][0];
        r->sigma[1] = p->G_inf * r->tau_M * D[0][1];
        r->sigma[2] = p->G_inf * r->tau_M * D[1][1];
        double eta_eff = p->G_inf * r->tau_M + p->G_inf * p->tau0;
        r->tau_lb = 0.5 + eta_eff / (p->rho0 * ORC_CS2);
        r->sbar[0] = r->sbar[1] = r->sbar[2] = 0.0;
        r->snn[0] = r->snn[1] = r->snn[2] = 0.0;
        r->drho = r->S = 0.0;
        r->rho_eq_m1 = r->R0m1;
        r->u[0] = r->j[0] / (1.0 + r->rho_eq_m1);
        r->u[1] = r->j[1] / (1.0 + r->rho_eq_m1);
        return;
    }
    if (p->stress_mode == 0) {
        if (orc_stress_series(r->kap, r->tau_M, p->G_inf, r->sigma) < 0) {
            orc_stress_gauss(r->kap, r->tau_M, p->G_inf, r->sigma);
#ifdef _OPENMP
#pragma omp atomic
#endif
            orc_fallbacks++;
        }
    } else {
        double s_old[3] = {sig_prev[k], sig_prev[N + k], sig_prev[2 * N + k]};
        if (orc_stress_step(r->kap, r->tau_M, p->G_inf, s_old, r->sigma) < 0) {
#ifdef _OPENMP
#pragma omp atomic
#endif
            orc_fallbacks++;
        }
    }
    /* Sigma = sigma + eta_inf D (Eq. Sigmamodel); the LB itself carries eta^N D, so
     * Sigma^nN = sigma + (eta_inf - eta^N) D  (= sigma - G tau D when tau_LB is matched to
     * the low-shear viscosity, Sec. IV). */
    double eta_inf = p->G_inf * p->tau0;
    double eta_N = p->rho0 * ORC_CS2 * (p->tau_lb - 0.5);
    double nn_xx = r->sigma[0] + (eta_inf - eta_N) * D[0][0];
    double nn_xy = r->sigma[1] + (eta_inf - eta_N) * D[0][1];
    double nn_yy = r->sigma[2] + (eta_inf - eta_N) * D[1][1];
    double trace = nn_xx + nn_yy;
    r->snn[0] = nn_xx;
    r->snn[1] = nn_xy;
    r->snn[2] = nn_yy;
    r->sbar[0] = nn_xx - trace / ORC_DIM;     /* overbar: traceless part (Sec. II A)     */
    r->sbar[1] = nn_xy;
    r->sbar[2] = nn_yy - trace / ORC_DIM;
    r->drho = -trace / (ORC_CS2 * ORC_DIM);   /* flow-induced density change (Sec. II A) */
    r->S = r->drho - drho_prev[k];            /* dt d_t delta rho, Eq. (rhoplus)         */
    if (p->boundary == 1) r->drho = r->S = 0.0; /* GPBC: no density correction (Sec. II B) */
    if (p->scheme == 2) {
        /* the stress acts through its divergence (a force density, in j and the force terms
         * of Eq. bodyforce) instead of the stress line and the flow-induced density */
        r->sbar[0] = r->sbar[1] = r->sbar[2] = 0.0;
        r->drho = r->S = 0.0;
    }
    /* reading: sum_i n^eq = sum_i (n* + n)/2 = R0 + S/2, so that sum_i (Delta_i + F_i) = S */
    r->rho_eq_m1 = r->R0m1 + 0.5 * r->S;
    r->u[0] = r->j[0] / (1.0 + r->rho_eq_m1);
    r->u[1] = r->j[1] / (1.0 + r->rho_eq_m1);
}

/* Generalized periodic boundaries (Sec. II B): per boundary column (0: x = 0, 1: x = nx-1) the
 * density and momentum of every node's post-collision populations and the column mean of the
 * density.  colrho/coljx/coljy: [2][ny]; colmean: [2].  Densities are kept as rho - 1 (sums of
 * the population offsets), so that their rounding acts on the small part. */
static void gpbc_columns(int nx, int ny, const double *dnstar, double *colrho, double *coljx,
                         double *coljy, double *colmean) {
    long N = (long)nx * ny;
    for (int c = 0; c < 2; ++c) {
        int x = c == 0 ? 0 : nx - 1;
        double sum = 0.0;
        for (int y = 0; y < ny; ++y) {
            double r = 0.0, jx = 0.0, jy = 0.0;
            for (int i = 0; i < 9; ++i) {
                double v = dnstar[i * N + idx(nx, x, y)];
                r += v;
                jx += ORC_CX[i] * v;
                jy += ORC_CY[i] * v;
            }
            colrho[c * ny + y] = r;
            coljx[c * ny + y] = jx;
            coljy[c * ny + y] = jy;
            sum += r;
        }
        colmean[c] = sum / ny;
    }
}

/* The population i that enters through the inlet (entering_inlet = 1: it would wrap from the
 * outlet column) or through the outlet (0: from the inlet column) at row ys of the source node:
 * n^eq_i(rho_target + rho_s - mean, j_s) + [n*_i(s) - n^eq_i(rho_s, j_s)], as an offset. */
static double gpbc_ghost(const orc_params *p, int i, int entering_inlet, int ny, int ys, double dnstar_s,
                         const double *colrho, const double *coljx, const double *coljy,
                         const double *colmean) {
    int c = entering_inlet ? 1 : 0; /* the column the population leaves */
    double rs_m1 = colrho[c * ny + ys], jx = coljx[c * ny + ys], jy = coljy[c * ny + ys];
    double rt_m1 = (entering_inlet ? p->rho_in : p->rho_out) + rs_m1 - colmean[c]; /* offsets */
    double eq_t[9], eq_s[9];
    orc_equilibrium_offset(rt_m1, jx / (1.0 + rt_m1), jy / (1.0 + rt_m1), eq_t);
    orc_equilibrium_offset(rs_m1, jx / (1.0 + rs_m1), jy / (1.0 + rs_m1), eq_s);
    return eq_t[i] + (dnstar_s - eq_s[i]);
}

/* Streaming (pull form of Eq. lbupdate) plus bounce-back, then the moments of Eq. (rhoj).
 * Works on offsets: R0 - 1 = sum_i dn_i and sum_i c_i n_i = sum_i c_i dn_i. */
static void stream_and_moments(const orc_params *p, int nx, int ny, const double *dnstar, double *dn,
                               double *R0m1, double *j, double *ug) {
    long N = (long)nx * ny;
    double *colrho = NULL, *coljx = NULL, *coljy = NULL, colmean[2] = {0.0, 0.0};
    if (p->boundary == 1) {
        colrho = (double *)malloc(sizeof(double) * 6 * ny);
        coljx = colrho + 2 * ny;
        coljy = colrho + 4 * ny;
        gpbc_columns(nx, ny, dnstar, colrho, coljx, coljy, colmean);
    }
    const double fx = body_force(p);
#ifdef _OPENMP
#pragma omp parallel for schedule(static)
#endif
    for (int y = 0; y < ny; ++y)
        for (int x = 0; x < nx; ++x) {
            long k = idx(nx, x, y);
            double r0 = 0.0, jx = 0.0, jy = 0.0;
            for (int i = 0; i < 9; ++i) {
                int xr = x - ORC_CX[i]; /* source column before any wrap */
                int xs = (xr % nx + nx) % nx;
                int ys = y - ORC_CY[i];
                double v;
                if (ys < 0 || ys >= ny) {
                    /* simple bounce-back at a wall half-way between rows: the population
                     * that left this node towards the wall returns reversed */
                    int opp = -1;
                    for (int o = 0; o < 9; ++o)
                        if (ORC_CX[o] == -ORC_CX[i] && ORC_CY[o] == -ORC_CY[i]) opp = o;
                    v = dnstar[opp * N + k];
                } else if (p->boundary == 1 && (xr < 0 || xr >= nx)) {
                    v = gpbc_ghost(p, i, xr < 0, ny, ys, dnstar[i * N + idx(nx, xs, ys)], colrho, coljx,
                                   coljy, colmean);
                } else {
                    v = dnstar[i * N + idx(nx, xs, ys)];
                }
                dn[i * N + k] = v;
                r0 += v;
                jx += ORC_CX[i] * v;
                jy += ORC_CY[i] * v;
            }
            if (p->top_wall == 1 && y == ny - 1) {
                /* Zou-He moving wall: replace the three populations that came from beyond the
                 * wall (c_y = -1: directions 4, 7, 8).  On offsets (w_4 = w_2, w_7 = w_5, w_8 = w_6,
                 * and the known weights w_0 + w_1 + w_3 + 2 (w_2 + w_5 + w_6) sum to 1). */
                double *d = dn + k;
                double known = d[0 * N] + d[1 * N] + d[3 * N] + 2.0 * (d[2 * N] + d[5 * N] + d[6 * N]);
                double rho = 1.0 + known;          /* u_y = 0 at the wall */
                double half_t = 0.5 * (d[1 * N] - d[3 * N]);
                d[4 * N] = d[2 * N];
                d[7 * N] = d[5 * N] + half_t - 0.5 * rho * p->u_wall;
                d[8 * N] = d[6 * N] - half_t + 0.5 * rho * p->u_wall;
                r0 = 0.0; jx = 0.0; jy = 0.0;
                for (int i = 0; i < 9; ++i) {
                    r0 += d[i * N];
                    jx += ORC_CX[i] * d[i * N];
                    jy += ORC_CY[i] * d[i * N];
                }
            }
            R0m1[k] = r0;
            j[2 * k] = jx + 0.5 * fx; /* j = sum c n + f dt/2 (Eq. rhoj, with the forcing) */
            j[2 * k + 1] = jy;
            ug[2 * k] = j[2 * k] / (1.0 + r0);    /* reading: gradients from j / R0 */
            ug[2 * k + 1] = j[2 * k + 1] / (1.0 + r0);
        }
    free(colrho);
}

typedef struct {
    double *n, *R0m1, *j, *ug, *fnn, *snn;
} orc_work;

static int work_alloc(orc_work *w, long N) {
    w->n = (double *)malloc(sizeof(double) * 9 * N);
    w->R0m1 = (double *)malloc(sizeof(double) * N);
    w->j = (double *)malloc(sizeof(double) * 2 * N);
    w->ug = (double *)malloc(sizeof(double) * 2 * N);
    w->fnn = (double *)malloc(sizeof(double) * 2 * N);
    w->snn = (double *)malloc(sizeof(double) * 3 * N);
    return (w->n && w->R0m1 && w->j && w->ug && w->fnn && w->snn) ? 0 : -1;
}
static void work_free(orc_work *w) {
    free(w->n); free(w->R0m1); free(w->j); free(w->ug); free(w->fnn); free(w->snn);
}

static int valid_grid(int nx, int ny) { return nx >= 1 && ny >= 3; }

/* The comparison schemes run with periodic x, bounce-back walls and stress mode 0, without the
 * relaxation-time extensions; the fluidity memory needs its state array. */
static int valid_scheme(const orc_params *p, const double *phi) {
    if (p->tau_f < 0.0 || !(p->rho_ref > 0.0) || (p->tau_f > 0.0 && !phi)) return 0;
    if (p->scheme == 0) return 1;
    if (p->scheme != 1 && p->scheme != 2) return 0;
    if (p->beta_rho != 0.0 || p->tau_f != 0.0) return 0;
    return p->stress_mode == 0 && p->boundary == 0 && p->top_wall == 0;
}

/* Moments of the streamed state.  Scheme 2 then needs the stress of every node before any node
 * can collide (explicit order, as for the paper's scheme: kappa from j / R0 with j = J0 + f^ex/2;
 * sigma and Sigma^nN; their divergence f^nN; then j = J0 + (f^ex + f^nN)/2 for n^eq and F_i):
 * w->fnn receives f^nN [2][N], and j and ug are not changed by it. */
static void moments_for_step(const orc_params *p, int nx, int ny, const double *dn_star, const double *drho,
                             const double *sig, orc_work *w) {
    stream_and_moments(p, nx, ny, dn_star, w->n, w->R0m1, w->j, w->ug);
    if (p->scheme != 2) return;
    long N = (long)nx * ny;
    for (int y = 0; y < ny; ++y)
        for (int x = 0; x < nx; ++x) {
            long k = idx(nx, x, y);
            node_result r;
            node_update(p, nx, ny, x, y, w->R0m1, w->j, w->ug, drho, sig, NULL, &r);
            w->snn[k] = r.snn[0];
            w->snn[N + k] = r.snn[1];
            w->snn[2 * N + k] = r.snn[2];
        }
    stress_divergence(nx, ny, w->snn, w->fnn);
}

/* Scheme 2: the node's force density f^ex + f^nN, and j, u of Eq. (rhoj) / Eq. (neq) with it. */
static void stress_force(const orc_params *p, const orc_work *w, long N, long k, node_result *r, double *f) {
    f[0] = body_force(p);
    f[1] = 0.0;
    if (p->scheme != 2) return;
    f[0] += w->fnn[k];
    f[1] += w->fnn[N + k];
    r->j[0] += 0.5 * w->fnn[k];
    r->j[1] += 0.5 * w->fnn[N + k];
    r->u[0] = r->j[0] / (1.0 + r->rho_eq_m1);
    r->u[1] = r->j[1] / (1.0 + r->rho_eq_m1);
}

/* Advance the state (dn_star, drho, sig) by nsteps steps in place.  Returns 0, or -1 on a bad
 * argument / allocation failure. */
int orc_run(const orc_params *p, int nx, int ny, double *dn_star, double *drho, double *sig, double *phi,
            long nsteps, int nthreads) {
    if (!valid_grid(nx, ny) || (p->stress_mode == 1 && !sig) || !valid_scheme(p, phi)) return -1;
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#else
    (void)nthreads;
#endif
    long N = (long)nx * ny;
    orc_work w;
    if (work_alloc(&w, N)) { work_free(&w); return -1; }
    for (long s = 0; s < nsteps; ++s) {
        moments_for_step(p, nx, ny, dn_star, drho, sig, &w);
#ifdef _OPENMP
#pragma omp parallel for schedule(static)
#endif
        for (int y = 0; y < ny; ++y)
            for (int x = 0; x < nx; ++x) {
                long k = idx(nx, x, y);
                node_result r;
                node_update(p, nx, ny, x, y, w.R0m1, w.j, w.ug, drho, sig, phi, &r);
                double dneq[9], F[9], f[2];
                stress_force(p, &w, N, k, &r, f);
                orc_equilibrium_offset(r.rho_eq_m1, r.u[0], r.u[1], dneq);
                orc_forcing(r.tau_lb, r.sbar, r.S, r.u, f, F);
                for (int i = 0; i < 9; ++i) {
                    /* BGK: n* = n - (n - n^eq)/tau_LB + F, on offsets from w_i */
                    double dni = w.n[i * N + k];
                    dn_star[i * N + k] = dni - (dni - dneq[i]) / r.tau_lb + F[i];
                }
                drho[k] = r.drho;
                if (p->tau_f > 0.0) phi[k] = r.phi; /* (only this node reads its own phi) */
                if (p->stress_mode == 1) {
                    sig[k] = r.sigma[0];
                    sig[N + k] = r.sigma[1];
                    sig[2 * N + k] = r.sigma[2];
                }

            }
    }
    work_free(&w);
    return 0;
}

/* Macroscopic fields of a stored state: what the next collision would use.
 *   u[y][x][2]   = j / rho   with rho the hydrodynamic density of Eq. (rhoj),
 *   sigma[y][x][4] = polymer stress (xx, yy, zz, xy), zz = 0 in 2-D flow,
 *   rho[y][x]    = hydrodynamic density rho_eq - delta rho(t)  (Eq. rhoj, reading C1).
 * The state is not modified. */
int orc_fields(const orc_params *p, int nx, int ny, const double *dn_star, const double *drho,
               const double *sig, const double *phi, double *u, double *sigma, double *rho) {
    if (!valid_grid(nx, ny) || (p->stress_mode == 1 && !sig) || !valid_scheme(p, phi)) return -1;
    long N = (long)nx * ny;
    orc_work w;
    if (work_alloc(&w, N)) { work_free(&w); return -1; }
    moments_for_step(p, nx, ny, dn_star, drho, sig, &w);
    for (int y = 0; y < ny; ++y)
        for (int x = 0; x < nx; ++x) {
            long k = idx(nx, x, y);
            node_result r;
            double f[2];
            node_update(p, nx, ny, x, y, w.R0m1, w.j, w.ug, drho, sig, phi, &r);
            stress_force(p, &w, N, k, &r, f);
            double rho_h = 1.0 + (r.rho_eq_m1 - r.drho);
            if (u) { u[2 * k] = r.j[0] / rho_h; u[2 * k + 1] = r.j[1] / rho_h; }
            if (sigma) {
                sigma[4 * k + 0] = r.sigma[0];
                sigma[4 * k + 1] = r.sigma[2];
                sigma[4 * k + 2] = 0.0;
                sigma[4 * k + 3] = r.sigma[1];
            }
            if (rho) rho[k] = rho_h;
        }
    work_free(&w);
    return 0;
}

/* Diagnostic access to the per-node intermediates of one update (kappa, tau_M, drho, S),
 * used by tests: out[y][x][9] = kxx, kxy, kyx, kyy, tau_M, drho, S, rho_eq, tau_LB of the node. */
int orc_node_intermediates(const orc_params *p, int nx, int ny, const double *dn_star,
                           const double *drho, const double *sig, const double *phi, double *out) {
    if (!valid_grid(nx, ny) || (p->stress_mode == 1 && !sig) || !valid_scheme(p, phi)) return -1;
    long N = (long)nx * ny;
    orc_work w;
    if (work_alloc(&w, N)) { work_free(&w); return -1; }
    moments_for_step(p, nx, ny, dn_star, drho, sig, &w);
    for (int y = 0; y < ny; ++y)
        for (int x = 0; x < nx; ++x) {
            long k = idx(nx, x, y);
            node_result r;
            double f[2];
            node_update(p, nx, ny, x, y, w.R0m1, w.j, w.ug, drho, sig, phi, &r);
            stress_force(p, &w, N, k, &r, f);
            double *o = out + 9 * k;
            o[0] = r.kap[0]; o[1] = r.kap[1]; o[2] = r.kap[2]; o[3] = r.kap[3];
            o[4] = r.tau_M; o[5] = r.drho; o[6] = r.S; o[7] = 1.0 + r.rho_eq_m1; o[8] = r.tau_lb;
        }
    work_free(&w);
    return 0;
}
