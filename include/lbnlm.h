/*
 * lbnlm.h -- C ABI of the GB300 lattice-Boltzmann library for the tensorial nonlinear
 * generalized Maxwell (nlM) fluid of Papenkort & Voigtmann, arXiv:1310.7450.
 *
 * One library call advances one or many independent 2-D channels with the paper's scheme:
 * D2Q9 pull-streaming with half-way bounce-back walls (Sec. II B), the BGK collision with
 * the non-Newtonian forcing term of Eq. (bodyforce), the flow-induced density of Eq. (rhoplus),
 * three-point velocity gradients (Sec. II C) and the nlM stress of Eqs. (sigtsum, smalld,
 * nlmaxwell).  All of a step runs in CUDA kernels of this library on the caller's stream.
 *
 * Conventions
 *   - Lattice units: dx = dt = 1, c_s^2 = 1/3.  D2Q9 numbering: 0:(0,0) 1:(1,0) 2:(0,1)
 *     3:(-1,0) 4:(0,-1) 5:(1,1) 6:(-1,1) 7:(-1,-1) 8:(1,-1).
 *   - Channel c has nx columns (x periodic) and ny[c] fluid rows; walls sit half-way below row
 *     0 and above row ny[c]-1, so the width is 2H = ny[c].
 *   - "Node order" of every field array: channel after channel, inside a channel row-major
 *     (y outer, x inner): node = node_offset(c) + y*nx + x, node_offset(c) = nx * sum_{c'<c} ny[c'].
 *   - "Plane order" of population arrays: channel after channel, inside a channel 9 planes
 *     (direction i) of ny[c]*nx values in row-major order.
 *   - Ownership: the handle owns all device state; every output buffer is the caller's
 *     (host memory unless on_device != 0, then device memory of the handle's device); the
 *     CUDA stream is borrowed and must outlive the handle.
 *   - Errors: every call returns an lb_status; nothing throws across the ABI.  lb_last_error()
 *     gives a human-readable detail of the most recent failure on the calling thread.
 *   - Asynchrony: lb_step only enqueues work on the stream.  Calls that return host data
 *     (lb_get_fields to host, lb_residual, lb_monitor, lb_channel_status, lb_get_*) synchronise
 *     the stream first.
 */
#ifndef LBNLM_H
#define LBNLM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct lb_handle lb_handle; /* opaque, library-owned */

typedef enum {
    LB_OK = 0,
    LB_EINVAL = 1,     /* bad argument: null pointer, size, tau_lb <= 1/2, ny < 3, NaN, ... */
    LB_ENOMEM = 2,     /* device or host allocation failed                                  */
    LB_ECUDA = 3,      /* a CUDA call or kernel launch failed (detail in lb_last_error)       */
    LB_EUNSTABLE = 4,  /* a channel produced NaN/Inf or |u| > 0.3; it is retired (not stepped) */
    LB_ETIMEOUT = 5,   /* a bounded device-side wait gave up (status word bit 2)              */
    LB_ESTATE = 6      /* the call needs state that does not exist yet (e.g. no residual)     */
} lb_status;

enum { LB_PREC_F64 = 0, LB_PREC_F32 = 1, LB_PREC_BF16 = 2, LB_PREC_F64S_F32M = 3, LB_PREC_F32S_F64M = 4 };
enum { LB_STRESS_INLM = 0, LB_STRESS_TIMESTEPPED = 1 };
/* lb_grid.flags: LB_GRID_STORE_SIGMA writes the 4-component stress every step; LB_GRID_TILE_ONLY
 * keeps every step on the general tile kernel (single wide FP32/BF16 channels otherwise use the
 * row-march kernel); LB_GRID_BF16_STOCHASTIC rounds BF16 populations stochastically (unbiased:
 * increments below half a BF16 step survive on average) instead of to nearest;
 * LB_GRID_NO_GRAPH launches every tile-kernel step separately (by default lb_step replays runs of
 * plain tile-kernel steps from a captured CUDA graph: the same kernels with the same arguments,
 * bitwise the same result, without the per-launch host overhead).
 * The comparison schemes of Sec. II C (the usual alternatives to the paper's forcing; at most one,
 * stress mode 0, periodic x and bounce-back walls, not in lb_run_until_steady; the
 * generalized-Newtonian scheme runs on the row-march kernel for wide single FP32/BF16 channels,
 * the divergence scheme on the tile kernel):
 * LB_GRID_GENERALIZED_NEWTONIAN relaxes each node with tau_LB(gdot) = 1/2 + eta_eff/(rho0 c_s^2)
 * (Eq. taulb with the model's steady-shear viscosity eta_eff = G_inf tau_M + G_inf tau0, tau_M of
 * Eq. nlmaxwell at the node's shear rate) and keeps only the body-force terms of Eq. (bodyforce);
 * the stress reported is G_inf tau_M D (no normal-stress differences).
 * LB_GRID_STRESS_DIVERGENCE feeds f^nN = div Sigma^nN (three-point differences of the same-time
 * stress of every node, Sigma^nN = sigma + (G_inf tau0 - eta^N) D) as a force density into
 * Eq. (rhoj) and the force terms of Eq. (bodyforce) instead of the stress line and the
 * flow-induced density (two launches per step).  Both have delta rho = 0.
 * LB_GRID_RELAXATION_MODEL keeps the paper's scheme and enables the relaxation-time extensions of
 * its outlook (lb_set_relaxation_model; off until set): FP64, FP32 or BF16, either stress mode,
 * any boundary, not in lb_run_until_steady; one more plane per node (the fluidity).  Wide single
 * FP32/BF16 channels with periodic x and bounce-back walls step on the row-march kernel's variant,
 * the others on the tile kernel. */
enum { LB_GRID_STORE_SIGMA = 1, LB_GRID_TILE_ONLY = 2, LB_GRID_BF16_STOCHASTIC = 4, LB_GRID_NO_GRAPH = 8,
       LB_GRID_GENERALIZED_NEWTONIAN = 16, LB_GRID_STRESS_DIVERGENCE = 32, LB_GRID_RELAXATION_MODEL = 64 };

typedef struct {
    int n_channels;   /* >= 1                                                              */
    int nx;           /* periodic length shared by all channels, >= 1                      */
    const int *ny;    /* [n_channels] fluid rows per channel, each >= 3 (copied)           */
    int precision;    /* LB_PREC_F64: FP64 storage and arithmetic;
                         LB_PREC_F32: populations stored as FP32 deviations n_i - w_i, FP32 math;
                         LB_PREC_BF16: BF16 deviations, FP32 math;
                         diagnostic mixes: LB_PREC_F64S_F32M (FP64 storage, FP32 math) and
                         LB_PREC_F32S_F64M (FP32 storage, FP64 math) separate the two errors */
    int stress_mode;  /* LB_STRESS_INLM: instantaneous nlM stress, Eq. (sigtsum) (the paper's
                         model, Sec. III A); LB_STRESS_TIMESTEPPED: one backward-Euler step of
                         the upper-convected Maxwell equation Eq. (gkder) per LB step           */
    int flags;        /* LB_GRID_* bits or 0                                               */
} lb_grid;

/* Per-channel physical parameters (lattice units).  The BGK collision carries the Newtonian
 * viscosity eta^N = rho0 (tau_lb - 1/2)/3 (Eq. taulb); the forcing adds
 * Sigma^nN = sigma + (G_inf tau0 - eta^N) D (Sec. IV; = sigma - G_inf tau D when eta^N is the
 * low-shear viscosity G_inf (tau + tau0)). */
typedef struct {
    double tau_lb;       /* BGK relaxation time, > 1/2                                      */
    double g_x;          /* body-force density along x (constant; Sec. III B)               */
    double G_inf;        /* plateau modulus, >= 0                                           */
    double tau0;         /* microscopic time; eta_inf = G_inf tau0 (Eq. Sigmamodel), >= 0    */
    double theta;        /* tau / tau0 (structural relaxation time tau = theta tau0), >= 0   */
    double gamma_c;      /* critical strain of Eq. (nlmaxwell), > 0; +inf = no thinning     */
    double rho0;         /* reference density of eta^N and of the initial state, > 0        */
    double rho_pert_amp; /* initial rho = rho0 (1 + amp U(-1,1)), U from SplitMix64         */
    uint64_t seed;       /* SplitMix64 seed; counter = y*nx + x + 1 within the channel       */
} lb_params;

/* lb_boundary.x_mode: how the channel ends are joined.
 *   LB_X_PERIODIC  periodic x; the flow is driven by the body force g_x (Eq. bodyforce with the
 *                  flow-induced density of Eq. rhoplus).
 *   LB_X_GPBC      generalized periodic boundaries (Sec. II B, after Kim and Pitsch): a population
 *                  that crosses an end is rebuilt from the node it leaves, n^eq(rho_+- + rho_s -
 *                  mean, j_s) + n^neq*, with rho_+- = c_s^-2 p_+- the inlet/outlet densities held at
 *                  the ghost columns x = -1 and x = nx.  g_x is then the imposed pressure gradient:
 *                  p_+ - p_- = g_x (nx + 1), rho_+- = rho0 +- (3/2) g_x (nx + 1); there is no body
 *                  force and no flow-induced density (delta rho = 0, Eq. bodyforce keeps its first
 *                  line), and lb_create starts from the linear density between rho_+ and rho_- .
 *                  lb_set_body_force changes the pressure gradient.  Wide single FP32/BF16 channels
 *                  step on the row-march kernel's boundary variant, the others on the tile kernel;
 *                  lb_run_until_steady / lb_sweep_tune return LB_EINVAL. */
enum { LB_X_PERIODIC = 1, LB_X_GPBC = 2 };
/* lb_boundary.walls:
 *   LB_WALLS_BOUNCE_BACK  half-way bounce-back walls at y = -1/2 and y = ny - 1/2 (Sec. II B).
 *   LB_WALLS_COUETTE      planar Couette flow (Sec. IV C): half-way bounce-back at y = -1/2; the
 *                         last row y = ny-1 lies on a wall moving with (u_wall, 0) whose incoming
 *                         populations follow Zou and He (gap ny - 1/2).  u_wall starts at 0 and is
 *                         set with lb_set_wall_velocity.  The prescribed velocity is that of the
 *                         wall row's populations, j / sum_i n_i.  Wide single FP32/BF16 channels
 *                         step on the row-march kernel's boundary variant, the others on the tile
 *                         kernel; lb_run_until_steady / lb_sweep_tune return LB_EINVAL. */
enum { LB_WALLS_BOUNCE_BACK = 1, LB_WALLS_COUETTE = 2 };

typedef struct {
    int walls;      /* LB_WALLS_BOUNCE_BACK or LB_WALLS_COUETTE                             */
    int x_mode;     /* LB_X_PERIODIC or LB_X_GPBC                                            */
} lb_boundary;

/* Create the channels on the current CUDA device, allocate their state and initialise it to
 * rest equilibrium n_i = w_i rho(r) with delta rho = 0 and zero polymer stress.
 * params: [n_channels].  cuda_stream: a cudaStream_t (0 = legacy default stream).
 * On failure *out is NULL and nothing is leaked. */
lb_status lb_create(const lb_grid *grid, const lb_params *params, const lb_boundary *boundary,
                    void *cuda_stream, lb_handle **out);

/* Advance every stable channel by n >= 0 steps (Eq. lbupdate: stream, then collide with
 * Eq. bodyforce).  The last two steps also save the velocity so that the last step can
 * evaluate the one-step residual (lb_residual).  Returns LB_EUNSTABLE once any channel has
 * been found unstable (the other channels keep being stepped). */
lb_status lb_step(lb_handle *h, long n);

/* Macroscopic fields of the current state: the velocity u = j/rho [node][2], the polymer
 * stress sigma [node][4] as (xx, yy, zz, xy) with zz = 0 in 2-D flow, and the hydrodynamic
 * density rho = sum_i (n* + n)/2 - delta rho [node] (Eq. rhoj) that the next collision uses.
 * Any of u, sigma, rho may be NULL.  out_dtype: 0 = double, 1 = float.  on_device: the
 * pointers are device memory (no synchronisation) or host memory (synchronises).  The state
 * is not changed. */
lb_status lb_get_fields(lb_handle *h, void *u, void *sigma, void *rho, int out_dtype, int on_device);

/* Per-channel one-step residual ||u(t) - u(t-1)||_2 / ||u(t)||_2 of the state before the last
 * step of the most recent lb_step call (warp/block reductions fused into that step).
 * r: host [n_channels].  LB_ESTATE if no residual has been evaluated yet, or if the last
 * evaluation was taken in LB_MONITOR_FLUX_MAX mode. */
lb_status lb_residual(lb_handle *h, double *r);

/* Per-channel diagnostics of the same evaluation, host [n_channels][4]:
 * (residual, flux = sum over nodes of u_x / nx, max |u|, step index of the evaluated state).
 * The residual slot holds -1 when the evaluation was taken in LB_MONITOR_FLUX_MAX mode, NaN for
 * a channel whose status word is set. */
lb_status lb_monitor(lb_handle *h, double *out);

/* What the last step of each lb_step call evaluates (not in the paper: run control).
 * LB_MONITOR_RESIDUAL (default): the last two steps save the velocity and the last one forms the
 * residual, flux and max |u| (16 B per node more HBM traffic on the saving steps, 16 B more
 * again on the residual step).  LB_MONITOR_FLUX_MAX: the last step forms flux and max |u| only,
 * from its own state, at the traffic of a plain step -- what a cessation run needs every step
 * (its stop is max |u| < 1e-10); lb_monitor then reports -1 as the residual and lb_residual
 * returns LB_ESTATE.  LB_EINVAL for another mode. */
enum { LB_MONITOR_RESIDUAL = 0, LB_MONITOR_FLUX_MAX = 1 };
lb_status lb_set_monitor_mode(lb_handle *h, int mode);

/* The same diagnostics without waiting: enqueues their transfer into out ([n_channels][4], pinned
 * host memory or device memory) on the handle's stream and returns at once.  Pinned host memory
 * mapped into the device's address space (cudaHostAlloc, or any pinned allocation under unified
 * addressing) is written by a one-block kernel, anything else by a stream-ordered copy.  The values
 * are there when the stream has passed this point (cudaStreamSynchronize, or an event recorded
 * after the call); a monitoring loop can read step k's diagnostics while step k+1 runs.
 * LB_ESTATE if no residual has been evaluated yet. */
lb_status lb_monitor_async(lb_handle *h, double *out);

/* Change the body force of one channel (channel = -1: all), e.g. 0 for cessation.  Stream-
 * ordered: the force is staged in mapped pinned memory, which a small kernel on the handle's stream
 * reads and applies to every step enqueued after this call; the call does not wait for the steps
 * enqueued before it (a ring of 8 staging slots: it waits only when the host is 8 changes ahead). */
lb_status lb_set_body_force(lb_handle *h, int channel, double g_x);

/* Set the velocity of the moving wall of one channel (channel = -1: all) of a LB_WALLS_COUETTE
 * handle: start-up (u_wall > 0) and cessation (0) of planar Couette flow.  Stream-ordered like
 * lb_set_body_force.  LB_EINVAL for handles without a moving wall. */
lb_status lb_set_wall_velocity(lb_handle *h, int channel, double u_wall);

/* Warm start: set every node to the equilibrium of the given hydrodynamic density and velocity
 * (host, node order: u [node][2], rho [node]), with the population current chosen so that
 * j = rho u including the half force of Eq. (rhoj).  drho (host [node], may be NULL = 0) sets
 * the stored flow-induced density change delta rho(t-1).  The carried stress (stress mode 1)
 * is reset to zero. */
lb_status lb_set_fields(lb_handle *h, const double *u, const double *rho, const double *drho);

/* Full FP64 populations n*_i in plane order, delta rho [node], and the carried stress of
 * stress mode 1 in plane order of 3 planes (xx, xy, yy) per channel (may be NULL otherwise).
 * Values are converted to / from the storage precision (deviations n_i - w_i). */
lb_status lb_set_populations(lb_handle *h, const double *n, const double *drho, const double *sig3);
lb_status lb_get_populations(lb_handle *h, double *n, double *drho, double *sig3);

/* Checkpoint: the raw device state (populations in storage precision, delta rho, carried
 * stress, step counter) as an opaque byte image of lb_state_bytes() bytes.  Restoring it into a
 * handle created with the same grid continues bit-for-bit.  lb_set_state rejects (LB_EINVAL) an
 * image of another library version, grid, precision, stress mode or per-channel ny list (the
 * header carries a hash of the list, so channels [24, 40] never load an image of [40, 24]), and
 * clears the per-channel status word and the sticky LB_EUNSTABLE / LB_ETIMEOUT state: rolling
 * back to an image taken before an instability steps every channel again. */
size_t lb_state_bytes(const lb_handle *h);
lb_status lb_get_state(lb_handle *h, void *buf, size_t bytes);
lb_status lb_set_state(lb_handle *h, const void *buf, size_t bytes);

/* Per-channel status words (host [n_channels]): 0 = stable; bit 1 = unstable (NaN/Inf or
 * |u| > 0.3; the channel is retired); bit 2 = a bounded device-side wait timed out. */
lb_status lb_channel_status(lb_handle *h, int *status);

/* Batched sweep: step every stable channel until its residual over the check interval k,
 * ||u(t) - u(t-k)|| / (k ||u(t)||), is <= tol, checked every k = check_every steps (even, >= 2), or
 * until max_steps (rounded up to a multiple of k).  Over one step that change sits on the FP32
 * rounding floor of a steady state; over k steps the floor falls as 1/k while a smooth exponential
 * approach to the steady state gives the one-step value.  Each channel is owned by a
 * thread-block cluster that runs its own time loop (hardware cluster barrier per step) and leaves
 * when the channel has converged; the channels run as width classes, one persistent launch per
 * class, the class launches captured as one CUDA graph (see lb_sweep_groups).  The run proceeds in
 * segments of 64, 256, 1024, ... check intervals: after each, converged channels drop out and a
 * class that lost half of its channels is tuned again (the slowest channels then run with the
 * shape of lowest per-step latency); a channel's first check interval in a segment only saves its
 * velocity.  The first call tunes each class by timing short sweeps from the current state (the
 * state is restored).  Outputs (host, [n_channels], may be NULL): steps taken (-1: max_steps
 * reached, -2: unstable) and the last residual.  Each channel advances by its own number of
 * steps; lb_step_count() is not changed.  Stress mode 0, periodic x, bounce-back walls only.
 * Synchronises the stream. */
lb_status lb_run_until_steady(lb_handle *h, double tol, long check_every, long max_steps, long long *steps_out,
                              double *residual_out);
/* Run the sweep autotuner now (otherwise the first lb_run_until_steady does); the state is kept. */
lb_status lb_sweep_tune(lb_handle *h);
/* The sweep configuration chosen by the autotuner (0 before the first sweep) and the time of its
 * tuning run (ms for 256 steps of every channel). */
lb_status lb_sweep_config(lb_handle *h, int *threads, int *cluster, double *tune_ms);

/* The sweep runs the stable channels in width classes (floor(log2 ny)), one persistent launch per
 * class on forked streams, each class with its own configuration: kernel variant 0 = the state
 * streamed through L2 every step (k_sweep), 1 = the state resident in the cluster's shared memory,
 * halo rows read from the neighbouring CTAs (k_sweep_smem; needs ny / cluster >= 3); threads per
 * CTA; CTAs per cluster.  lb_sweep_groups writes up to max_groups entries (any pointer may be NULL;
 * threads 0 = not tuned yet) and returns the number of classes (-1: null handle).
 * lb_sweep_config reports the widest class and the summed tuning time; lb_sweep_variant the
 * widest class's kernel (-1 before the first tuning / setting). */
int lb_sweep_groups(const lb_handle *h, int *variant, int *threads, int *cluster, int *channels, int max_groups);
int lb_sweep_variant(const lb_handle *h);

/* Fix one configuration for every class instead of tuning (variant 0/1, threads 128/256, cluster
 * size 1..16); LB_EINVAL if it does not fit every class of the handle. */
lb_status lb_sweep_set_config(lb_handle *h, int variant, int threads, int cluster);

/* Allocation-free diagnostics.  The paper has no counterpart: this is a service for callers that
 * must not allocate device memory when they ask for the convergence measures -- e.g. a monitoring
 * loop that cannot take cudaMalloc's implicit device synchronisation mid-run, or a process whose
 * device memory is fully reserved by another allocator.  From two velocity fields on the device
 * (u_now, u_prev: [node][2], dtype 0 = double, 1 = float, node order as lb_get_fields) and the
 * channel boundaries node_offsets (device, [n_channels + 1], long long), it writes per channel
 * (residual ||u_now - u_prev||_2/||u_now||_2, flux = sum of u_x / nx, max |u|) to out (device,
 * [n_channels][3], double), on cuda_stream.  It calls no allocating routine: its scratch is a fixed
 * 2 MiB array inside the library (65536 records; at most 1024 channels per call, larger requests
 * fail with LB_EINVAL) that every GPU using the library keeps until the process exits.  Each call
 * on a stream that is not capturing looks the array's address up (cudaGetSymbolAddress, with the
 * current device); the first call on a device must come before any stream capture (LB_ESTATE
 * otherwise).  cuda_stream (NULL = legacy default stream) must belong to the current device
 * (LB_EINVAL otherwise).  Calls share the array, so calls that overlap on the GPU (e.g. on two
 * streams) race; each call writes every scratch record it reads, so nothing needs clearing
 * between calls.  A NaN or Inf anywhere in a channel's u_now or u_prev makes all three of that
 * channel's outputs NaN; a channel at rest (u_now = 0) reports residual 0. */
lb_status lb_field_monitor_static(const void *u_now, const void *u_prev, int dtype, int n_channels,
                                  const long long *node_offsets, int nx, double *out, void *cuda_stream);

/* Warm starts on the device (not in the paper; the learned warm start below).  Grid: the network
 * sees each channel on 256 points d_k = (k + 1/2)/128 - 1 across the channel (d = (y - y_c)/H);
 * its 768 outputs per channel are, for u_x, sigma_xy and N1 in turn, (steady profile - closed form)
 * / scale on the grid, where the closed form is the steady channel solution of Sec. III B (the
 * quadratic for dv/dd integrated to v(1) = 0; u = (H/tau0) v) at the channel's current parameters
 * and scale = max |closed form| per field.  Rows <-> grid by linear interpolation, end values held.
 * lb_warmstart_apply: writes a start state into every channel from pred (device, [n_channels][768]
 * FP32 network outputs, de-standardised as pred * t_sd + t_mu when t_mu and t_sd, device [768],
 * are given; both or neither) or, with pred = NULL, from the closed form itself: u = (u_x(y), 0),
 * rho = 1, delta rho = -(3/2) N1(y), as lb_set_fields does.  lb_warmstart_targets: the network
 * targets of the handle's current state (column x = 0 of each row) into targets (device,
 * [n_channels][768], FP32).  Both need G_inf > 0, tau0 > 0 and g_x > 0 in every channel
 * (LB_EINVAL); both run on the handle's stream (apply synchronises it). */
lb_status lb_warmstart_apply(lb_handle *h, const float *pred, const float *t_mu, const float *t_sd);
lb_status lb_warmstart_targets(lb_handle *h, float *targets);

/* ---- Learned warm start (not in the paper): a three-layer perceptron n_in -> width -> width ->
 * n_out (tanh hidden layers) with BF16 working weights, FP32 master weights and FP32 accumulation,
 * trained with Adam on a mean-squared-error loss by this library's kernels.  Parameters are flat
 * FP32 in the order W1 [width][n_in], b1, W2 [width][width], b2, W3 [n_out][width], b3.  Arrays x
 * [batch][n_in], y / target [batch][n_out] and grads [n_params] are device memory; every call runs
 * on the stream given at creation (loss is returned on the host and synchronises). */
typedef struct lb_mlp lb_mlp;
lb_status lb_mlp_create(int n_in, int width, int n_out, int max_batch, uint64_t seed, void *cuda_stream,
                        lb_mlp **out);
void lb_mlp_destroy(lb_mlp *m);
long long lb_mlp_num_params(const lb_mlp *m);
lb_status lb_mlp_forward(lb_mlp *m, const float *x, int batch, float *y);
lb_status lb_mlp_gradients(lb_mlp *m, const float *x, const float *target, int batch, float *grads, double *loss);
lb_status lb_mlp_train_step(lb_mlp *m, const float *x, const float *target, int batch, float lr, double *loss);
lb_status lb_mlp_get_params(lb_mlp *m, float *host);        /* FP32 masters -> host [n_params]     */
lb_status lb_mlp_set_params(lb_mlp *m, const float *host);  /* host [n_params] -> masters and BF16 */

/* Relaxation-time extensions that the paper leaves for further study (its conclusions: the Maxwell
 * time should depend on the local density; Sec. III A: a flow dependence of tau_M influenced by
 * earlier times, as in the fluidity models).  The paper fixes neither form; this library takes
 *   tau(rho) = tau exp(beta_rho (rho - rho_ref) / rho_ref), rho = R0 - delta rho(t-1) at the node,
 *   d phi/dt = (phi_ss - phi) / tau_f for the fluidity phi = 1/tau_M, phi_ss = 1/tau(rho) +
 *   II_D^{1/2}/gamma_c (Eq. nlmaxwell), stepped by backward Euler (tau_f = 0: Eq. nlmaxwell).
 * For one channel (channel >= 0) or all (-1); rho_ref > 0, tau_f >= 0, all finite; LB_EINVAL
 * otherwise or if the handle was created without LB_GRID_RELAXATION_MODEL.  Synchronises the
 * stream.  The fluidity of every node is part of the checkpoint image and is cleared (unset:
 * the next step starts from phi_ss) by lb_set_populations. */
lb_status lb_set_relaxation_model(lb_handle *h, int channel, double beta_rho, double rho_ref, double tau_f);

/* Limit of every bounded device-side wait of the row-march step kernel (the mbarrier waits for its
 * row copies), in seconds: 0 <= seconds <= 60, default 2.  0 makes each wait a single non-blocking
 * probe.  A wait that gives up sets bit 2 of the channel's status word; the kernel then waits (at
 * most 1 s, independent of this limit) for its own copies in flight and returns, and the next
 * lb_step reports LB_ETIMEOUT.  Not in the paper: failure detection of this library's kernels. */
lb_status lb_set_wait_limit(lb_handle *h, double seconds);

long lb_step_count(const lb_handle *h);     /* steps taken since creation (or restored)      */
int lb_uses_row_march(const lb_handle *h);  /* 1 if plain steps run on the row-march kernel   */

/* Work items of the row-march kernel for a single nx x ny channel (host only, no GPU needed):
 * strips of 128 columns cut into row ranges, at most one per resident CTA (ctas_per_sm x n_sm),
 * with rows dealt so that every item is expected to take the same time (later CTAs on an SM run
 * slower under the warp schedulers' age priority; the two edge strips cost more per row).  Grids
 * of three or more strips give all interior strips the same row boundaries (their halo reads then
 * hit L2).
 * precision LB_PREC_F32 or LB_PREC_BF16, gpbc nonzero for pressure-driven ends (the model's edge
 * cost depends on both).  Writes (x0, y0, y1) per item into items[3 * max_items] (caller-owned
 * host memory; items may be NULL to query the count) and returns the number of items, or
 * -LB_EINVAL for nx not a positive multiple of 128, ny < 16, counts < 1, another precision, or
 * more items than max_items.  Not in the paper: a scheduling detail of this library's kernel. */
int lb_row_march_plan(int nx, int ny, int ctas_per_sm, int n_sm, int precision, int gpbc, int *items,
                      int max_items);
long lb_graph_replays(const lb_handle *h);  /* CUDA-graph launches made by lb_step so far      */
size_t lb_num_nodes(const lb_handle *h);     /* total fluid nodes over all channels           */
void lb_destroy(lb_handle *h);               /* synchronises the stream, frees everything     */
const char *lb_strerror(lb_status s);
const char *lb_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* LBNLM_H */
