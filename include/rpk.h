/*
 * rpk.h -- C interface of librpk, a single-GPU (sm_103a) implementation of the
 * lattice-Boltzmann time step of the reduced polyatomic ES-BGK model of
 * Kolluru, Atif & Ansumali, "Reduced kinetic model of polyatomic gases"
 * (arXiv 2201.05280).
 *
 * What one step computes (Sec. 4, eq. kinEqBGK; Sec. 5):
 *   - every point of the body-centred-cubic grid pulls its 41 RD3Q41
 *     populations (Sec. 5, Table 1) from its neighbours,
 *   - forms rho, rho u and the pressure tensor, recovers theta_T, theta_R and
 *     sigma of the physical distribution from the auxiliary population
 *     g = f - (dt/2) Omega (Sec. 5, g/f moment relations),
 *   - relaxes toward tau*(f^ES/tau + f^Eq/tau1) with the explicit trapezoid
 *     update g' = (1 - 2 beta*) g + 2 beta* tau*(f^ES/tau + f^Eq/tau1),
 *   - moves the matching energy into the rotational energy density E_R, and
 *   - advects (MacCormack) and diffuses (FTCS) E_R (Sec. 5, steps 2 and 3).
 *
 * Conventions for every call:
 *   - Units are lattice units: sublattice spacing 1, dt = 1, reference
 *     temperature theta0 = rpk_theta0() (Sec. 5, Table 1).
 *   - A scalar field is 2*nx*ny*nz doubles indexed
 *         p = ((s*nz + z)*ny + y)*nx + x,
 *     s = 0 for the corner sublattice, s = 1 for the body-centre sublattice at
 *     (x, y, z) + (1/2, 1/2, 1/2). A vector field (u) is three such planes, x
 *     component first.
 *   - Every call is made from the host. Kernels run on the CUDA stream given
 *     to rpk_create (NULL = the legacy default stream) on the device that was
 *     current at rpk_create; calls restore nothing else.
 *   - Ownership: the library allocates and owns all device state of a lattice
 *     and frees it in rpk_destroy. Caller arrays are only read or written
 *     during the call that receives them; device pointers passed with
 *     on_device = 1 must be device memory of the lattice's device.
 *   - Errors: every call returns an rpk_status; nothing throws across the
 *     interface. rpk_last_error() returns a message for the most recent failed
 *     call of the calling thread. A failed call leaves the lattice usable
 *     unless it reports RPK_ERR_CUDA (the CUDA context may then be broken).
 */
#ifndef RPK_H
#define RPK_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define RPK_ABI_VERSION 1

typedef enum {
  RPK_OK = 0,
  RPK_ERR_ARG = 1,     /* null pointer, bad size or bad enum */
  RPK_ERR_PARAM = 2,   /* physically invalid parameter (see rpk_set_relax) */
  RPK_ERR_CUDA = 3,    /* a CUDA call failed */
  RPK_ERR_NUMERIC = 4, /* the device flagged a non-finite or non-positive moment */
  RPK_ERR_STATE = 5,   /* call out of order (e.g. step before init) */
  RPK_ERR_OOM = 6,     /* device or host allocation failed */
  RPK_ERR_IO = 7       /* checkpoint file error */
} rpk_status;

/* Storage precision of the populations. Arithmetic is FP64 for RPK_F64 and
 * FP32 otherwise. RPK_F32/F16DEV/BF16DEV store h_i = g_i/w_i - 1. */
enum { RPK_F64 = 0, RPK_F32 = 1, RPK_F16DEV = 2, RPK_BF16DEV = 3 };

/* Boundary in x: periodic, or fixed equilibrium reservoirs beyond both ends
 * (rpk_set_reservoirs); a periodic x becomes walled with rpk_set_x_walls. y is
 * periodic unless rpk_set_walls puts diffuse walls there; z is always
 * periodic. */
enum { RPK_BC_PERIODIC = 0, RPK_BC_RESERVOIR = 1 };

typedef struct {
  int nx, ny, nz; /* cells per sublattice along each axis, each >= 1 */
  int precision;  /* RPK_F64 ... RPK_BF16DEV */
  int bc_x;       /* RPK_BC_PERIODIC or RPK_BC_RESERVOIR */
} rpk_grid;

/* Raw relaxation parameters, as in Sec. 4 eq. kinEqBGK and Sec. 5. */
typedef struct {
  double delta; /* rotational degrees of freedom, > 0 (Sec. 3, eq. thetadef) */
  double tau;   /* ES-BGK relaxation time, > 0 */
  double tau1;  /* relaxation time of the BGK term and of E_R, > 0 */
  double b;     /* ES-BGK parameter (Sec. 2, eq. lambdaij), B - b > 0 */
  double k_r;   /* kappa_R / kappa_T >= 0 (Sec. 4, conductivity paragraph) */
  double dt;    /* time step; must be 1 (lattice units) */
  int nsub;     /* FTCS sub-steps of the E_R diffusion per step; 0 = choose at
                   rpk_init_fields from the initial fields (rpk_auto_nsub) */
} rpk_relax;

typedef struct {
  double mass;      /* sum over points of rho */
  double mom[3];    /* sum of rho u */
  double energy;    /* sum of (sum_i g_i c_i^2 / 2 + auxiliary E_R), which
                       equals the physical E_T + E_R (Sec. 4, ConservedMomEq) */
  double H1;        /* sum of sum_i (f_i ln(f_i/w_i) - f_i) - (delta/2) rho ln theta_R
                       (Sec. 4, H-theorem paragraph, k = -delta/2); NaN if
                       some f_i <= 0 */
  double min_g;     /* smallest auxiliary population g_i */
  uint32_t status;  /* device flags since creation: 1 non-finite moment,
                       2 rho <= 0, 4 theta_T <= 0 or theta_R <= 0 */
  uint32_t pad;
  int64_t steps;    /* steps taken since the last rpk_init_fields/rpk_load */
} rpk_diag;

typedef struct rpk_lattice rpk_lattice;

/* Library facts. */
int rpk_abi_version(void);
double rpk_theta0(void); /* Sec. 5, Table 1 */
const char* rpk_last_error(void);

/* Parameter mapping of Sec. 4 (eq. viscosities and the conductivity
 * paragraph) at the reference state p0 = rho0 * theta0; host only, needs no
 * GPU. gamma -> delta = (5 - 3 gamma)/(gamma - 1); eta_b = c p0 tau1 with
 * c = 2 delta/(3(3 + delta)); eta = p0 tau/(B - b), B = 1 + tau/tau1;
 * kappa = 5 p0 tau (1 + k_r)/(2B). Writes out->{delta,tau,tau1,b,k_r},
 * out->dt = 1, out->nsub = 0. RPK_ERR_PARAM when no tau > 0, tau1 > 0,
 * k_r >= 0 realises the request (eta_B/eta < c needs b > 1). */
rpk_status rpk_map_gas(double gamma, double eta, double eta_B, double kappa, double b,
                       double rho0, rpk_relax* out);

/* FTCS sub-steps for the E_R diffusion, host only: the diffusivity of
 * theta_R = 2 E_R/(delta rho) is D = 5 k_r tau theta/(delta B); explicit
 * stability in ndim dimensions needs 2 ndim D dt/nsub <= 1, kept at 0.9 with
 * theta = 1.25 theta_max. Returns >= 1. */
int rpk_auto_nsub(const rpk_relax* r, double theta_max, int ndim);

/* The gas as the experiments specify it -- kinematic viscosity nu, bulk to
 * shear viscosity ratio lam = eta_B/eta and Prandtl number Pr -- in the
 * (eta, eta_B, kappa) that rpk_map_gas takes (Sec. 4, eq. viscosities and the
 * Prandtl-number paragraph); host only, needs no GPU. delta from gamma as in
 * rpk_map_gas, eta = rho0 nu, eta_B = lam eta and kappa = eta c_p/Pr with the
 * heat capacity per unit mass c_p = (5 + delta)/2 (theta units). Writes
 * out[0..2] = eta, eta_B, kappa (host array of 3). RPK_ERR_ARG for out = NULL,
 * RPK_ERR_PARAM for gamma outside (1, 5/3] or nu, lam, Pr, rho0 not finite
 * and positive. */
rpk_status rpk_gas_from_nondim(double gamma, double nu, double lam, double Pr, double rho0,
                               double out[3]);

/* Adiabatic sound speed c_s = sqrt(gamma theta0) of the lattice reference
 * state (Sec. 4, hydrodynamic limit; Sec. 6 measures it); NaN for gamma
 * outside (1, 5/3]. Host only. */
double rpk_sound_speed(double gamma);

/* rpk_auto_nsub at the hottest state of a set of fields: theta_max is the
 * largest theta = (3 theta_T + delta theta_R)/(3 + delta) (eq. thetadef) over
 * the n host values theta_T[p], theta_R[p] and, if res is not NULL, the two
 * reservoir states res[12] (layout of rpk_set_reservoirs). Host only; returns
 * 1 for NULL or non-positive input. */
int rpk_auto_nsub_fields(const rpk_relax* r, const double* theta_T, const double* theta_R,
                         int64_t n, const double* res, int ndim);

/* Create a lattice on the current device. cuda_stream is a cudaStream_t (or
 * NULL). Allocates 2 x 41 populations per point (ping-pong) plus ~12 scalar
 * planes. */
rpk_status rpk_create(const rpk_grid* grid, void* cuda_stream, rpk_lattice** out);
void rpk_destroy(rpk_lattice* lat); /* NULL is allowed */

/* Set the relaxation parameters (validated: delta > 0, tau > 0, tau1 > 0,
 * B - b > 0, k_r >= 0, dt == 1, 0 <= nsub <= 4096). Takes effect at the next
 * rpk_step; nsub = 0 is resolved at the next rpk_init_fields. */
rpk_status rpk_set_relax(rpk_lattice* lat, const rpk_relax* r);
/* rpk_map_gas with rho0 = 1, then rpk_set_relax. */
rpk_status rpk_set_gas(rpk_lattice* lat, double gamma, double eta, double eta_B, double kappa,
                       double b);

/* RPK_BC_RESERVOIR only: the equilibrium states beyond the low-x and the
 * high-x end, 12 doubles: rho, ux, uy, uz, theta_T, theta_R of the low end,
 * then of the high end. Must be called after rpk_set_relax and before
 * rpk_init_fields. */
rpk_status rpk_set_reservoirs(rpk_lattice* lat, const double* states12);
/* Rotational solver. mode 0 (default): the conservative form -- the state is
 * the auxiliary energy E~_R = E_R - (dt/2)(delta rho/2)(theta - theta_R)/tau1,
 * exchanged inside the collision and transported in flux form (total energy
 * conserved to round-off). mode 1: the paper's four steps on theta_R (Sec. 5):
 * backward-Euler half step theta_R <- (theta_R + X theta_T(f))/(1 + X),
 * X = 3 dt/(2 tau1 (3 + delta)), with theta_T(f) of time t; MacCormack on
 * u . grad theta_R (forward then backward differences, u of time t); nsub FTCS
 * sub-steps of (2/(rho delta)) kappa_R lap theta_R; the second half step. The
 * state is then theta_R, theta_T(f) follows from the printed theta_T(g)
 * relation, and total energy is conserved only to first order in dt/tau1.
 * Changing the mode discards the state (initialise again); checkpoints record
 * it. */
rpk_status rpk_set_rot_mode(rpk_lattice* lat, int mode);

/* Diffuse walls normal to y (the diffusive wall condition of Ansumali & Karlin
 * that Sec. 6 cites for its Couette and cavity flows; the paper does not write
 * it out, this is the library's reading). walls8 = ux, uy, uz, theta of the
 * low-y wall, then of the high-y wall (uy must be 0: the walls slide; theta >
 * 0); NULL makes y periodic again. The walls are the planes y = -1/4 and
 * y = ny - 1/4 in sublattice-spacing units, half way between layers of points
 * (which sit at y + s/2), so the channel height is ny.
 *   Kinetic part: a population whose pull source lies beyond a wall is emitted
 *   by the wall as rho_w f^eq(1, u_w, theta_w), the discrete Gaussian of the
 *   wall's velocity and temperature, with rho_w per (x, z) column and wall set
 *   so that the wall emits into the column exactly the mass that left the
 *   column through it in the same step: mass is conserved to round-off.
 *   Rotational energy: Dirichlet theta_R = theta_w; the diffusive flux through
 *   the wall face of a point at distance d (1/4 or 3/4) from the wall is
 *   kappa_R(p)(theta_w - theta_R(p))/d; no advective flux through a wall. In
 *   rotational mode 1 the same Dirichlet value enters the advection
 *   differences and the Laplacian as the straight line through theta_w.
 * Requires ny >= 2, bc_x = RPK_BC_PERIODIC and the relaxation parameters set
 * (RPK_ERR_STATE otherwise); a non-finite state, uy != 0 or theta <= 0 gives
 * RPK_ERR_PARAM and leaves the walls as they were.
 * Takes effect at the next step or moment read; the automatic nsub of
 * rpk_init_fields accounts for the stiffer near-wall diffusion (one face with
 * coefficient 4 kappa_R) and for the wall temperatures. Checkpoints record the
 * walls. Synchronises the lattice's stream. */
rpk_status rpk_set_walls(rpk_lattice* lat, const double* walls8);
/* Diffuse walls normal to x, for the square cavity of Sec. 6: the same
 * condition as rpk_set_walls with x and y exchanged, at x = -1/4 and
 * x = nx - 1/4. walls8 = ux, uy, uz, theta of the low-x wall, then of the
 * high-x wall (ux must be 0; theta > 0); NULL makes x periodic again. With
 * walls on both axes, a population whose pull source lies beyond a y wall and
 * an x wall (a corner) is emitted by the y wall, and each x wall balances the
 * mass of the entries the y walls leave to it. Requires nx >= 2 and
 * bc_x = RPK_BC_PERIODIC (the x walls take the reservoirs' place); otherwise
 * as rpk_set_walls. */
rpk_status rpk_set_x_walls(rpk_lattice* lat, const double* walls8);

/* Initial state from hydrodynamic fields (layout above): rho > 0, u (3
 * planes), theta_T > 0, theta_R > 0. f = f^Eq(rho, u, theta_T I), then
 * g = f - (dt/2) Omega(f) and the auxiliary E_R (Sec. 5). Host arrays when
 * on_device = 0 (pinned host memory is read in place by the device over the
 * host link; pageable memory is copied through a staging buffer), device arrays
 * of this device when 1. The same device pass checks the inputs:
 * RPK_ERR_PARAM if some rho, theta_T, theta_R is not finite and positive or
 * some u is not finite, and then the lattice is left uninitialised (its
 * previous state is lost). Resets the step count. Synchronises the stream. */
rpk_status rpk_init_fields(rpk_lattice* lat, const double* rho, const double* u,
                           const double* theta_T, const double* theta_R, int on_device);

/* Advance n >= 0 steps. Asynchronous: only enqueues kernels on the stream. */
rpk_status rpk_step(rpk_lattice* lat, int64_t n);

/* Hydrodynamic fields of the current state: rho, u (3 planes), theta_T and
 * theta_R of the physical distribution, and E_R = delta rho theta_R / 2. Any
 * output pointer may be NULL to skip it. Host arrays when on_device = 0
 * (pinned memory written in place by the device, pageable memory through the
 * staging buffer), device arrays when
 * 1. Synchronises the stream; returns RPK_ERR_NUMERIC if the device status
 * flags are set (the arrays are still written). */
rpk_status rpk_read_moments(rpk_lattice* lat, double* rho, double* u, double* theta_T,
                            double* theta_R, double* E_rot, int on_device);

/* FP64 global diagnostics of the current state (rpk_diag). Synchronises the
 * stream; returns RPK_ERR_NUMERIC if status != 0 (out is still filled). */
rpk_status rpk_diagnostics(rpk_lattice* lat, rpk_diag* out);

/* Checkpoint: raw state (populations, auxiliary E_R, the last two velocity
 * fields, step count, parameters) with a header. rpk_load requires a lattice
 * created with the same grid. Bitwise restart. Synchronise the stream. */
rpk_status rpk_save(rpk_lattice* lat, const char* path);
rpk_status rpk_load(rpk_lattice* lat, const char* path);

/* Facts about a lattice: out[0] nsub in use, out[1] steps, out[2] number of
 * points, out[3] bytes of device memory held. */
rpk_status rpk_get_info(rpk_lattice* lat, int64_t out[4]);

/* Kernel timing (a tracing aid; the paper has no counterpart). While enabled,
 * rpk_step brackets each kernel class with CUDA events recorded on the
 * lattice's stream: RPK_KC_COLLIDE (pull-stream + collide + exchange) and
 * RPK_KC_TRANSPORT (MacCormack advection and all FTCS sub-steps of E_R). rpk_timing(lat, 1) clears the counters and starts;
 * rpk_timing(lat, 0) stops. rpk_timing_read synchronises the stream and
 * returns the summed milliseconds and the number of kernel launches per class
 * since the last start (arrays of RPK_KC_COUNT entries). */
enum { RPK_KC_COLLIDE = 0, RPK_KC_TRANSPORT = 1, RPK_KC_COUNT = 2 };
rpk_status rpk_timing(rpk_lattice* lat, int enable);
rpk_status rpk_timing_read(rpk_lattice* lat, double* ms, int64_t* launches);

/* ---- Batched quasi-1-D tubes (many independent shock tubes in one launch) ----
 * Each tube is an nx x 1 x 1 lattice of the same model with its own relaxation
 * parameters, x-reservoirs (RPK_BC_RESERVOIR semantics) and step count; the
 * arithmetic per tube is the one of rpk_step on such a lattice. All tubes run
 * in one persistent kernel launch (captured once into a CUDA graph): every CTA
 * takes whole tubes from a work queue (longest work first) and runs their time
 * loops itself, with the tube's rotational-energy and transport fields in
 * shared memory and only the populations in device memory. The paper's
 * shock-tube validations are single runs; batching is this library's.
 * Field layout: tube b's 2*nx_b points (p = s*nx_b + x) follow tube b-1's in
 * the concatenated arrays; u is three such concatenated planes. */
typedef struct {
  int nx;          /* cells per sublattice along x, 2 <= nx <= rpk_batch_max_nx() */
  int nsteps;      /* steps that rpk_batch_run advances this tube, >= 0 */
  rpk_relax relax; /* per-tube parameters (validated as in rpk_set_relax); nsub =
                      0 is resolved at rpk_batch_init from the tube's fields */
  double res[12];  /* reservoir states, as in rpk_set_reservoirs */
} rpk_tube;

typedef struct rpk_batch rpk_batch;

/* Largest tube length the shared-memory layout supports for a precision. */
int rpk_batch_max_nx(int precision);

/* precision: RPK_F64 or RPK_F32. save_every >= 1: during rpk_batch_run, the
 * moments (rho, u_x, theta_T, E_R) of every tube at steps 0, save_every,
 * 2 save_every, ... (< nsteps) are stored as float snapshots. Copies the tube
 * descriptions. */
rpk_status rpk_batch_create(int precision, int ntubes, const rpk_tube* tubes, int save_every,
                            void* cuda_stream, rpk_batch** out);
void rpk_batch_destroy(rpk_batch* b);

/* Initial state of every tube from concatenated host fields (rho, u (3 planes),
 * theta_T, theta_R), as rpk_init_fields per tube. Synchronises. */
rpk_status rpk_batch_init(rpk_batch* b, const double* rho, const double* u, const double* theta_T,
                          const double* theta_R);

/* Launch configuration of the persistent kernel: threads per CTA (a multiple
 * of 32 in [64, 512]) and CTAs per SM (>= 1, limited by shared memory). */
rpk_status rpk_batch_set_config(rpk_batch* b, int threads, int ctas_per_sm);
/* Rotational diffusion of the batch: mode 0 (default) the nsub FTCS sub-steps
 * of the paper's scheme (Sec. 5, rotational step 3); mode 1 a variant that
 * takes the same flux-form equation in one backward-Euler step per time step,
 * (delta rho / 2) theta' - dt [K+ (theta'_+ - theta') - K- (theta' - theta'_-)]
 * = E_R, solved per sublattice line by cyclic reduction (unconditionally
 * stable: nsub is ignored). Takes effect at the next rpk_batch_run. */
rpk_status rpk_batch_set_diffusion(rpk_batch* b, int mode);

/* Time every supported launch configuration on a sample of the batch's own
 * tubes (a scratch copy; the batch state is untouched) and keep the fastest.
 * out[0] = threads, out[1] = CTAs per SM, out[2] = sample milliseconds x 1000.
 * Synchronises. */
rpk_status rpk_batch_autotune(rpk_batch* b, int64_t out[3]);

/* Advance every tube by its nsteps in one launch. Asynchronous. */
rpk_status rpk_batch_run(rpk_batch* b);

/* Moments of the current state of every tube (concatenated layout, host
 * arrays; any may be NULL). Synchronises; RPK_ERR_NUMERIC if any tube flagged
 * a non-finite or non-positive moment. */
rpk_status rpk_batch_read_moments(rpk_batch* b, double* rho, double* u, double* theta_T,
                                  double* theta_R, double* E_rot);

/* Snapshots of the last rpk_batch_run: for tube b, nsnap_b = ceil(nsteps_b /
 * save_every) records of 4 x 2 nx_b floats (rho, u_x, theta_T, E_R), tubes in
 * order. Returns the total float count in *count; copies to host `out` when it
 * is not NULL. Synchronises. */
rpk_status rpk_batch_snapshots(rpk_batch* b, float* out, int64_t* count);
/* Moment blocks: per tube, in tube order, [4][2 nx] floats holding rho, u_x,
 * theta_T and E_R = delta rho theta_R / 2 at the tube's 2 nx points (point
 * order as in the fields), i.e. tube b's block starts at float 8 sum_{b'<b}
 * nx_b' -- the layout of one snapshot. Device pointers. */
/* Initialise every tube from moment blocks (u_y = u_z = 0; theta_R from E_R).
 * Needs every tube's FTCS sub-step count: relax.nsub > 0, or an earlier
 * rpk_batch_init from host fields. Invalid values (non-positive or non-finite)
 * are reported by the next rpk_batch_read_moments. Synchronises. */
rpk_status rpk_batch_init_device(rpk_batch* b, const float* state);
/* Steps of the next rpk_batch_run per tube (host array), each in [0, the count
 * given at creation]; snapshots keep their creation-time offsets. Synchronises. */
rpk_status rpk_batch_set_steps(rpk_batch* b, const int* nsteps);
/* Current moments into device moment blocks. Asynchronous (the batch's stream). */
rpk_status rpk_batch_moments_device(rpk_batch* b, float* state);

/* ---- Learned surrogate network (a 1-D convolutional operator) --------------
 * Maps the moment fields of quasi-1-D tubes at step t to step t + 32 (the
 * paper has no learned component). Architecture on a sequence of L fine points
 * (L a multiple of 4), position-major tensors [sequence][point][channel]:
 * unshuffle by 4 -> conv k=1 (4 cin -> width) -> nblocks residual blocks
 * h + conv5(relu(conv5(relu(h)))) -> conv k=1 of relu(h) (width -> 4 cout) ->
 * shuffle. Every contraction runs on the tensor cores with BF16 operands and
 * FP32 accumulation; parameters are FP32 master copies with Adam state.
 * Parameter vector: per layer (lift, block convs, head) the weights W[o][t][i]
 * then the biases. All pointers to tensors are device pointers on the
 * network's device; calls on the network's stream. */
typedef struct rpk_net rpk_net;
rpk_status rpk_net_create(int cin, int cout, int width, int nblocks, uint64_t seed,
                          void* cuda_stream, rpk_net** out);
void rpk_net_destroy(rpk_net* net);
int64_t rpk_net_num_params(const rpk_net* net);
/* which = 0: parameters, 1: gradients of the last rpk_net_loss_grad (host
 * array of rpk_net_num_params floats). Synchronises. */
rpk_status rpk_net_get_params(rpk_net* net, float* host, int which);
rpk_status rpk_net_set_params(rpk_net* net, const float* host);
/* y[nseq][len][cout] = network(x[nseq][len][cin]). Asynchronous. */
rpk_status rpk_net_forward(rpk_net* net, const float* x, int nseq, int len, float* y);
/* The same network over nseq sequences of different lengths lens[s] (host
 * array, each a positive multiple of 4), concatenated position-major in x
 * [sum lens][cin] and y [sum lens][cout]; zero padding at every sequence's ends.
 * Synchronises the network's stream. */
rpk_status rpk_net_forward_ragged(rpk_net* net, const float* x, int nseq, const int* lens, float* y);
/* Masked mean-squared error sum(mask (y - target)^2)/(sum(mask) cout) of the
 * network output against target[nseq][len][cout], mask[nseq][len]; writes the
 * loss to *loss and the gradients to the network. Synchronises. */
rpk_status rpk_net_loss_grad(rpk_net* net, const float* x, const float* target,
                             const float* mask, int nseq, int len, double* loss);
/* One Adam step (bias-corrected) with the stored gradients. Asynchronous. */
rpk_status rpk_net_adam(rpk_net* net, float lr, float beta1, float beta2, float eps);

/* ---- Surrogate rollout of batched tubes with LBM fallback -----------------
 * (the paper has no learned component). The network maps the moments of a
 * tube at step t to the increments of its conserved densities over `jump`
 * steps: inputs per fine point (position 2x + s of point (s, x)) are 11
 * features -- v = (rho, u_x, theta_T, E_R) shifted and scaled, the change of v
 * since the previous window scaled (zero without one), two per-tube
 * conditioning values, and 1 inside the tube / 0 in the reservoir padding --
 * and outputs are 4 scaled increments of U = (rho, rho u_x,
 * E = rho u_x^2 / 2 + 3 rho theta_T / 2 + E_R, E_R). */
typedef struct {
  int jump;            /* LBM steps one network application stands for (e.g. 32) */
  int pad;             /* reservoir points each side of a tube in its sequence, >= 0 */
  int spot_every;      /* spot check at windows 0, spot_every, 2 spot_every, ...; 0: none */
  int project;         /* 1: rescale the mass and energy increments to zero net change */
  int anchor;          /* 1: spot-check windows keep the LBM's result and a handed-over
                          tube continues on the LBM from its last accepted state;
                          0: the network's windows are kept and a handed-over tube
                          runs on the LBM from its initial state */
  double drift_tol;    /* relative mass or energy drift that hands a tube to the LBM */
  double l1_tol;       /* estimated relative L1 density error that hands a tube to the LBM */
  float in_shift[4];   /* feature k = (v_k - in_shift[k]) / in_scale[k], v = (rho, u_x, theta_T, E_R) */
  float in_scale[4];
  float out_scale[4];  /* increment of U_k = out_scale[k] * network output k */
  float in_dscale[4];  /* feature 4 + k = (v_k - v_k(previous window)) / in_dscale[k] */
  int lbm_threads;     /* launch configuration of the LBM arm (rpk_batch_set_config) */
  int lbm_ctas_per_sm;
  int lbm_diffusion;   /* rotational diffusion of the LBM arm (rpk_batch_set_diffusion) */
} rpk_sur_config;

/* One sequence of network input: the padded tube, from padded position `crop`
 * on, `len` points (a multiple of 4) written at point `out` of x / target /
 * mask. Padded position c holds tube position c - pad when that lies in
 * [0, 2 nx), else the left (c < pad) or right reservoir state. */
typedef struct {
  int64_t src;         /* float offset of the source moment block [4][2 nx] */
  int64_t tgt;         /* float offset of the target moment block, or -1 (no target) */
  int64_t prev;        /* float offset of the previous window's block, or -1 (none) */
  int64_t out;         /* first point of the sequence in x, target and mask */
  int nx, len, crop, pad_;
  float res[2][4];     /* reservoir (rho, u_x, theta_T, E_R), left then right */
  float cond[2];       /* conditioning features */
} rpk_sur_seq;

/* Network inputs (and, where tgt >= 0, normalised target increments
 * (U_k(target) - U_k(source)) / out_scale[k] and a mask that is 1 at tube
 * points at least `margin` points from both ends of the sequence) for nseq
 * sequences; store and seqs are device pointers (prev offsets index `store`
 * too), maxlen bounds every len. x [..][11], target [..][4], mask [..]
 * (target and mask may be NULL when no sequence has a target). noise (host,
 * 4 values, may be NULL): the source state of tube points is perturbed by
 * noise[k] sqrt(3) (2 u - 1) per variable, u uniform in [0, 1) from output
 * ((s << 32 | l) * 4 + k) + 1 of SplitMix64 seeded with `seed` (sequence s of
 * the call, point l of the sequence); features and targets use the perturbed
 * state. Asynchronous on cuda_stream. */
rpk_status rpk_sur_pack(const rpk_sur_config* cfg, const float* store, const rpk_sur_seq* seqs,
                        int nseq, int maxlen, int margin, const float* noise, uint64_t seed,
                        float* x, float* target, float* mask, void* cuda_stream);

/* Moment blocks after one network application: for every tube of `seqs`
 * (device, nseq entries, src = the tube's block in `state`, out = its
 * sequence's first point in y), next[src..] = moments of U + increments,
 * with the projection of cfg->project; flags[i] = 1 where a result is
 * non-positive or non-finite; totals[2 i] = sum rho, totals[2 i + 1] = sum E
 * over the tube (FP64). Device pointers; asynchronous. */
rpk_status rpk_sur_apply(const rpk_sur_config* cfg, const float* state, const float* y,
                         const rpk_sur_seq* seqs, int nseq, float* next, int* flags,
                         double* totals, void* cuda_stream);

typedef struct rpk_rollout rpk_rollout;
/* The values (rho, u_x, theta_T, E_R) that a tube's low and high reservoir
 * states take in the moment blocks the surrogate reads, E_R = delta rho
 * theta_R / 2 (eq. thetadef's rotational energy): out (host, 8 floats) =
 * low side then high side. The paper has no counterpart (the surrogate is
 * this library's). RPK_ERR_ARG for a NULL argument. */
rpk_status rpk_sur_reservoirs(const rpk_tube* tube, float* out);

/* A rollout engine for ntubes tubes (every relax.nsub > 0): the network `net`
 * (not owned), per-tube conditioning cond[2 i], cond[2 i + 1] (host), and an
 * internal FP32 batch of the same tubes for spot checks and fallback. */
rpk_status rpk_rollout_create(rpk_net* net, const rpk_sur_config* cfg, int ntubes,
                              const rpk_tube* tubes, const float* cond, void* cuda_stream,
                              rpk_rollout** out);
void rpk_rollout_destroy(rpk_rollout* r);
/* Advance every tube by its nsteps from the moment blocks `state` (device,
 * updated in place): floor(nsteps / jump) windows by the network; at a spot
 * check the LBM also runs the window and the network's density is compared
 * with it (the error, times the windows until the next check, is added to the
 * tube's estimate); a tube whose mass or energy drift exceeds drift_tol, whose
 * result is invalid, or whose estimated accumulated L1 error exceeds l1_tol
 * is handed to the LBM (see anchor); remainders
 * (nsteps mod jump) run on the LBM; a tube whose final moments are invalid is
 * run again by the LBM from its initial state. stats (host, 5 per tube, may be
 * NULL): step at which the LBM took over (-1: never), network windows kept,
 * spot checks, LBM steps after the windows, 1 if run again from the start;
 * est (host, per tube, may be NULL): the estimated L1 error; ms (host, 4, may
 * be NULL): device time of the network windows, the spot checks, the final LBM
 * run and the repeated runs. Synchronises. */
rpk_status rpk_rollout_run(rpk_rollout* r, float* state, int64_t* stats, double* est, double* ms);
/* Spot-check errors of the last run: *windows = the largest window count; out
 * (host, ntubes x *windows, may be NULL) = relative L1 density error of the
 * network against the LBM per tube and checked window (NaN where unchecked,
 * +inf where the network's result was invalid). */
rpk_status rpk_rollout_errors(const rpk_rollout* r, double* out, int* windows);

/* Conserved totals of hydrodynamic fields held by the caller in device memory,
 * computed without allocating anything. The paper has no counterpart. It is
 * for callers that may not call cudaMalloc where they need the totals: an
 * application whose own memory manager owns all device memory (a pooling
 * allocator or a fixed budget) and forbids libraries to allocate, or a loop
 * that must not stall on cudaMalloc/cudaFree, which can synchronise the
 * device. Inputs: rho, u (3 planes), theta_T, theta_R, npts values each, in
 * the field layout above (e.g. written by rpk_read_moments with on_device = 1);
 * delta as in rpk_relax. Output: out[0..4] in device memory =
 *   sum rho, sum rho u_x, sum rho u_y, sum rho u_z,
 *   sum (rho |u|^2/2 + 3 rho theta_T/2 + delta rho theta_R/2)   (E_T + E_R),
 * which equal rpk_diagnostics' mass, mom and energy of the same state.
 * Asynchronous on cuda_stream (NULL = legacy default stream); the device is
 * the current one, and every pointer must be device memory of that device and
 * the stream one of its streams, else RPK_ERR_ARG (nothing is launched). The
 * per-block partial sums live in a static 320 KiB device array that every GPU
 * loading the library keeps until exit; npts is limited to 67,108,864 (8192
 * blocks of 8192 points), larger sizes return RPK_ERR_ARG. The first call on
 * each device looks up that array's address; make that first call before any
 * stream capture. All calls share the array, so calls whose kernels overlap
 * on the GPU race: order them on one stream. No part of the array needs to
 * start at zero: a call reads only the slots its own blocks wrote. */
rpk_status rpk_field_totals_noalloc(const double* rho, const double* u, const double* theta_T,
                                    const double* theta_R, int64_t npts, double delta,
                                    void* cuda_stream, double* out);

#ifdef __cplusplus
}
#endif

#endif /* RPK_H */
