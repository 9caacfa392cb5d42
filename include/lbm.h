/*
 * lbm.h - C interface of the GB300 (sm_103a) lattice Boltzmann solver for
 * non-ideal compressible flow (Hosseini, Feinberg & Karlin, "Lattice
 * Boltzmann model for non-ideal compressible fluid dynamics").
 *
 * One step of the method, at every node (Sec. 3.2 and Fig. FlowChart):
 * pull-stream the mass-momentum populations f_i and the bulk-energy
 * populations g_i, take the moments rho, rho u, rho E (Eqs. def_h, def_u,
 * def_E), evaluate the equation of state and the temperature (van der
 * Waals: Eqs. Pvdw, lbm_temp, explicit; Peng-Robinson: a closed-form root of
 * its caloric relation), build the Korteweg force, the Galilean correction
 * Phi and the heat-flux correction q^c from neighbour moments (Eqs. FK,
 * correction, qc_1), form the equilibria and shifted equilibria in product
 * form (Eqs. LBMeq, LBMstar, LBMeqG, LBMgstar) and collide (Eqs. fLBGK,
 * gLBGK).  Lattices: D2Q9 and D3Q27 (Eq. D3Q27c).  Lattice units:
 * delta x = delta t = 1.
 *
 * Conventions (all entry points):
 *  - Every call returns an int status (LBM_OK = 0 or a negative LBM_E*).
 *    No exception or abort crosses this interface.
 *  - Host arrays are caller-owned; the library copies in or out and keeps
 *    no pointer to them.  Device memory is owned by the handle.
 *  - Field arrays hold the Nx*Ny*Nz interior nodes in the order
 *    n = x + Nx*(y + Ny*z) (x fastest).  Vector fields are D consecutive
 *    planes of that size (u_x plane, then u_y, then u_z).
 *  - A handle is not thread-safe; distinct handles are independent.
 *  - All GPU work of a handle runs on its stream (lbm_set_stream).
 *  - Errors are reported, never trapped: a non-finite or non-positive
 *    density or temperature found during lbm_step sets a sticky device
 *    error word; lbm_step then returns LBM_EUNSTABLE, keeps the state for
 *    inspection, and refuses further steps with LBM_ESTATE until lbm_init.
 *
 * Boundaries: y and z are periodic.  The two x faces are either both
 * periodic, or each is one of:
 *  - an inflow face: post-collision populations of four ghost layers set to
 *    the equilibrium of a prescribed state, every step;
 *  - a zero-gradient outflow face: the ghost layers copy the nearest
 *    interior layer;
 *  - a moving isothermal wall: diffuse reflection at the wall velocity and
 *    temperature (LBM_BC_WALL, lbm_set_boundary).
 * The paper gives no boundary scheme; these are the library's.
 */
#ifndef LBM_H
#define LBM_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct lbm_s* lbm_t;

/* lattices (Eq. D3Q27c; D2Q9 is its two-dimensional product reduction) */
enum { LBM_D2Q9 = 9, LBM_D3Q27 = 27 };

/* status codes */
enum {
  LBM_OK = 0,
  LBM_EINVAL = -1,     /* bad argument (size, pointer, parameter range)       */
  LBM_ENOMEM = -2,     /* device or host allocation failed                    */
  LBM_ECUDA = -3,      /* a CUDA runtime call failed (message: lbm_last_error)*/
  LBM_EUNSTABLE = -4,  /* non-finite or non-positive rho / T produced         */
  LBM_ESTATE = -5      /* call not valid in the handle's state                */
};

/* storage / arithmetic precision of the populations */
enum {
  LBM_FP64 = 0,        /* FP64 storage, FP64 arithmetic                       */
  LBM_FP32 = 1,        /* FP32 storage, FP32 arithmetic                       */
  LBM_FP16DEV = 2      /* FP16 storage of p_i - p_i^ref, FP32 arithmetic      */
};

/* thermodynamic closure of the (rho, e) -> (T, P, c_s^2) step */
enum { LBM_CLOSURE_EXACT = 0, LBM_CLOSURE_MLP = 1 };

/* x-face boundary types */
enum { LBM_BC_PERIODIC = 0, LBM_BC_OUTFLOW = 1, LBM_BC_INFLOW = 2, LBM_BC_WALL = 3 };

/* faces for lbm_set_boundary */
enum { LBM_FACE_XLO = 0, LBM_FACE_XHI = 1 };

/* sticky status bits (lbm_get_flags) */
enum {
  LBM_FLAG_NONFINITE = 1u,   /* fatal: rho, u or T not finite                 */
  LBM_FLAG_NEGATIVE = 2u,    /* fatal: rho <= 0 or T <= 0                      */
  LBM_FLAG_THETA = 4u,       /* warning: theta = P/rho >= 1/3 (Sec. 5 bound)   */
  LBM_FLAG_PRESSURE = 8u     /* warning: P <= 0                                */
};

/* equations of state (lbm_eos.kind) */
enum { LBM_EOS_VDW = 0, LBM_EOS_PR = 1 };

/* Fluid and model parameters, lattice units.
 * kind LBM_EOS_VDW, the van der Waals fluid of the paper:
 *   P = rho R T / (1 - b rho) - a rho^2               (Eq. Pvdw)
 *   e = c_v T - a rho                                 (Eq. de_vdW)
 * kind LBM_EOS_PR, the Peng-Robinson fluid (the general equation of state of
 * Sec. 2, whose temperature needs a non-linear caloric inversion):
 *   P = rho R T / (1 - b rho) - a alpha(T) rho^2 / (1 + 2 b rho - b^2 rho^2),
 *   alpha = (1 + m (1 - sqrt(T / Tc)))^2,
 *   e = c_v T + (T a alpha' - a alpha) L(rho) / (2 sqrt2 b),
 *   L = ln((1 + (1 + sqrt2) b rho) / (1 + (1 - sqrt2) b rho))
 * (the identity e = c_v T + int_0^rho (P - T dP/dT)/rho'^2 drho', c_v the
 * ideal-gas part); T(rho, e) is the positive root of a quadratic in sqrt(T),
 * taken in a form without cancellation in the arithmetic precision.
 * Peng-Robinson handles step with the exact closure in FP32 or FP64 (fused
 * or multipass); FP16-deviation storage, the learned closure and batches are
 * van der Waals only.
 * kappa: Korteweg capillarity coefficient, F = kappa rho grad lap rho (Eq. FK).
 * eta_over_mu: bulk to shear viscosity ratio entering alpha (Eq. corr_bulk).
 * rho_ref, T_ref: reference state fixing the constant mu = tau P(rho_ref, T_ref)
 *   and k = mu c_p(rho_ref, T_ref) / Pr; for LBM_FP16DEV also the state whose
 *   equilibria are subtracted before storage.
 * Tc, m: Peng-Robinson only (Tc > 0, m >= 0). */
typedef struct {
  int kind;            /* LBM_EOS_VDW | LBM_EOS_PR */
  double a, b, R;
  double kappa;
  double eta_over_mu;
  double rho_ref, T_ref;
  int precision;       /* LBM_FP64 | LBM_FP32 | LBM_FP16DEV */
  int closure;         /* LBM_CLOSURE_EXACT | LBM_CLOSURE_MLP */
  double Tc, m;        /* Peng-Robinson critical temperature and alpha slope */
} lbm_eos;

/* Create a solver of Nx*Ny*Nz interior nodes (Nz = 1 for D2Q9).
 * tau: relaxation time at the reference state; the shear viscosity is the
 *   constant mu = tau P(rho_ref, T_ref) and the local relaxation time is
 *   mu / P (Sec. 3.1, tau = mu/P; beta of Eq. beta_main).
 * Pr: Prandtl number mu c_p / k at the reference state (enters q^c, Eq. qc).
 * cv: specific heat at constant volume.
 * Allocates the device state (two population buffers, scratch).  Both x faces
 * start periodic.  Errors: LBM_EINVAL (out is NULL, lattice not 9/27, a size
 * < 1, Nz != 1 with D2Q9, a non-positive tau, Pr, cv, b rho_ref >= 1,
 * unsupported kind/precision/closure, a Peng-Robinson fluid with Tc <= 0,
 * m < 0 or FP16-deviation storage), LBM_ENOMEM, LBM_ECUDA. */
int lbm_create(lbm_t* out, int lattice, int Nx, int Ny, int Nz, const lbm_eos* eos,
               double tau, double Pr, double cv);

/* Set the type of one x face before lbm_init.  state: for LBM_BC_INFLOW
 * D+2 doubles (rho, u_1..u_D, T) of the inflow state; for LBM_BC_WALL D+1
 * doubles (u_1..u_D, T) of the wall's velocity and temperature; otherwise it
 * may be NULL.  Setting one face to LBM_BC_PERIODIC sets both.  Changing
 * between periodic and non-periodic after lbm_create re-lays out the device
 * state (the state must then be re-initialised).
 *
 * LBM_BC_WALL: a moving isothermal wall (the thermal Couette flow of Sec.
 * 4.1; the paper gives no wall scheme, this is a diffuse-reflection
 * reading).  After each collision the ghost layers of the face take
 * s f^eq, s g^eq at (rho_e, u_wall, T_wall), rho_e the density of the first
 * fluid node and s the ratio of that node's post-collision f streaming into
 * the wall to the f^eq streaming out of it, so no mass crosses the wall.  The
 * Laplacian of the Korteweg force (Eq. FK) sees the wall as a symmetry plane:
 * a ghost column's density there is that of its mirror image in the fluid.
 * The normal wall velocity u_1 should be 0.
 * Errors: LBM_EINVAL (bad face/type, NULL state for inflow or wall,
 * non-positive rho or T, a wall with Nx < 4), LBM_ENOMEM, LBM_ECUDA. */
int lbm_set_boundary(lbm_t h, int face, int type, const double* state);

/* Use the given cudaStream_t (passed as void*) for all later work of this
 * handle; NULL selects the legacy default stream.  Errors: LBM_EINVAL. */
int lbm_set_stream(lbm_t h, void* stream);

/* Initialise every node (ghosts included, extended by the face rules) to the
 * equilibria f^eq(rho, u, theta), g^eq(rho, u, T, theta) with theta = P/rho
 * (Fig. FlowChart, "Initialize").  rho, T: Nx*Ny*Nz doubles; u: D planes.
 * All three are required host arrays.  Clears the sticky error word.
 * Errors: LBM_EINVAL (NULL pointer), LBM_ECUDA. */
int lbm_init(lbm_t h, const double* rho, const double* u, const double* T);

/* Same as lbm_init but the three arrays are device pointers (FP64, same
 * layout) already resident on the handle's device. */
int lbm_init_device(lbm_t h, const double* d_rho, const double* d_u, const double* d_T);

/* Advance n >= 0 time steps.  Returns after enqueuing the work and reading
 * the 4-byte sticky error word once (one stream synchronisation).
 * Errors: LBM_ESTATE (not initialised, or a previous step was unstable),
 * LBM_EINVAL (n < 0), LBM_EUNSTABLE (fatal flag raised; state kept),
 * LBM_ECUDA. */
int lbm_step(lbm_t h, int n);

/* Enqueue n steps without reading the error word (no synchronisation); the
 * fatal flags are reported by the next lbm_step, lbm_sync or lbm_moments.
 * Errors: LBM_ESTATE, LBM_EINVAL, LBM_ECUDA. */
int lbm_step_async(lbm_t h, int n);

/* Wait for the handle's stream and report the sticky error word as
 * lbm_step does. */
int lbm_sync(lbm_t h);

/* Macroscopic fields of the current state (Eqs. def_h, def_u, def_E,
 * lbm_temp): rho (Nx*Ny*Nz), u (D planes), T (Nx*Ny*Nz) as FP64 host arrays,
 * and totals[D+2] = (sum rho, sum rho u_1..u_D, sum rho E) over the interior
 * in FP64.  Any pointer may be NULL to skip that output.  Synchronises.
 * Errors: LBM_ESTATE (not initialised), LBM_ECUDA. */
int lbm_moments(lbm_t h, double* rho, double* u, double* T, double* totals);

/* Same outputs as lbm_moments into device pointers (FP64, same layout);
 * totals stays a host pointer.  Any pointer may be NULL. */
int lbm_moments_device(lbm_t h, double* d_rho, double* d_u, double* d_T, double* totals);

/* Sticky status bits (LBM_FLAG_*) raised since the last lbm_init. */
int lbm_get_flags(lbm_t h, unsigned* flags);

/* Copy the raw population buffer (the post-collision populations of the
 * last step, ghosts included, library layout) out to / in from a host buffer
 * of lbm_population_bytes() bytes; used for checkpoint and resume.  A resumed
 * run continues bit-identically.  Errors: LBM_EINVAL (size mismatch / NULL),
 * LBM_ESTATE (get before init), LBM_ECUDA. */
size_t lbm_population_bytes(lbm_t h);
int lbm_get_populations(lbm_t h, void* host, size_t bytes);
int lbm_set_populations(lbm_t h, const void* host, size_t bytes);

/* step implementations (lbm_set_step_kernel) */
enum { LBM_STEP_FUSED = 0, LBM_STEP_MULTIPASS = 1 };

/* Select how lbm_step runs one time step: LBM_STEP_FUSED (default) is one
 * single-pass kernel per step (plus the ghost fill when x is not periodic);
 * LBM_STEP_MULTIPASS runs moments, primitive fields and collision as three
 * kernels through FP-typed scratch fields.  Both compute the same update.
 * Errors: LBM_EINVAL (NULL handle or unknown kind). */
int lbm_set_step_kernel(lbm_t h, int kind);

/* Time each tile shape of the fused step kernel for `reps` steps from the
 * current state (writing only the spare buffer: the state does not advance)
 * and use the fastest from then on.  *chosen (may be NULL) receives the index
 * of the shape (0 is the default), *ms_per_step (may be NULL) its time.
 * The choice is remembered for the process: a later lbm_init of any handle
 * with the same lattice, precision, size and x boundary type uses it.
 * Synchronises.  Errors: LBM_EINVAL, LBM_ESTATE (before lbm_init), LBM_ECUDA. */
int lbm_autotune(lbm_t h, int reps, int* chosen, float* ms_per_step);

/* Shock capturing (Sec. 4.4, Eqs. shock_cap and shock_cap_k): numerical
 * transport coefficients added to the constant mu, eta, k of the handle,
 *   {mu, eta}^num = rho C_{mu,eta} F(|grad^4 S|),  k^num = rho c_s C_k F(|grad^4 |grad s||),
 * S the strain-rate magnitude |grad u + grad u^T|/2, grad s the entropy
 * gradient (c_v/T) grad T - R/(rho (1 - b rho)) grad rho of the van der
 * Waals fluid (Peng-Robinson: (c_v(rho, T)/T) grad T - (dP/dT)_rho / rho^2
 * grad rho, the same identity), |grad^4 f| the norm of the per-axis
 * five-point fourth differences (r = 5, delta x = 1), F the separable
 * binomial (1,4,6,4,1)/16 filter, c_s the fluid's sound speed at (rho, T).  The coefficients used by a
 * step are computed from the previous step's rho, u, T (none for the first
 * step after lbm_init).  All three C = 0 switches it off (the default).
 * The shear part is what stabilises planar shocks: with C_eta = 0 and
 * C_mu = C_k = 0.1 a D3Q27 Ma 1.2 shock 32 x 32 nodes wide stays stable,
 * Ma 1.25 needs 0.3 (without: blow-up within 100-200 steps).  C_eta > 0
 * enlarges the explicit bulk shift alpha (Eq. corr_bulk) and can
 * destabilise.  Costs D+2 planes written by the step and extra launches per
 * step: 2 in 2-D (strain with fourth differences over shared-memory tiles;
 * both filter passes with the coefficients), D+2 in 3-D (the last filter pass
 * fused with the coefficients).
 * Errors: LBM_EINVAL (NULL handle, negative or non-finite C), LBM_ENOMEM. */
int lbm_set_shock_capturing(lbm_t h, double C_mu, double C_eta, double C_k);

/* Graph replay (on = 1) or plain launches (on = 0, the default) for
 * lbm_step / lbm_step_async with n >= 2: two consecutive steps are captured
 * once per buffer parity into CUDA graphs and replayed n/2 times (an odd
 * last step is launched plainly).  The graphs are re-captured automatically
 * after any change of boundary, closure, tile, step kernel or stream.  With
 * the legacy default stream the library replays on a stream of its own
 * (ordered with the legacy stream).  Same results as plain launches.
 * Errors: LBM_EINVAL (NULL handle), LBM_ECUDA. */
int lbm_set_graphs(lbm_t h, int on);

/* Times of every tile candidate measured by the last lbm_autotune on `h`
 * (ms per step, in candidate order; the chosen one is the smallest).
 * Copies min(count, n) values to ms_per_step (host, may be NULL) and
 * returns the candidate count (0 before any autotune), or LBM_EINVAL for
 * a NULL handle. */
int lbm_autotune_times(lbm_t h, float* ms_per_step, int n);

/* Number of tile shapes of the fused step kernel for this handle's lattice,
 * precision and closure (the candidates lbm_autotune times, in its order).
 * Returns the count (>= 1), or LBM_EINVAL for a NULL handle. */
int lbm_tile_count(lbm_t h);

/* Mixed-precision form of the FP32 and FP16-deviation handles (FP32
 * collision, FP64 kept for the temperature inversion).  With `on` the
 * temperature of Eq. lbm_temp, T = (E - |u|^2/2 + a rho) / c_v, is evaluated
 * in FP64 from the FP32 moments E = (S + u.F/2)/rho and u, and rounded once to
 * FP32; for the Peng-Robinson fluid (Sec. 2: T from the non-linear caloric
 * relation) e = E - |u|^2/2 and the root's argument e - B0 are formed in FP64.
 * Off (the default): the whole step in FP32.  The FP64 form costs about 6% of
 * the 256^3 D3Q27 step.  Its effect on the error against the FP64 oracle
 * depends on the flow: on Ma 1.2 shock tubes it lowers it (T about threefold),
 * on a drifting Taylor-Green vortex it raises it (rho about twofold); the
 * trajectory error of FP32 runs is set by rounding throughout the step, not
 * by the inversion alone.  FP64 handles ignore the setting (their arithmetic
 * is FP64), and so do the learned closure (its network replaces the
 * inversion) and the batched step (FP32 inversion).  Applies to the fused
 * and multi-pass steps from the next step on; does not synchronise.
 * Errors: LBM_EINVAL (NULL handle). */
int lbm_set_temperature_fp64(lbm_t h, int on);
/* 1 while the FP64 temperature inversion is in use (FP32 / FP16-deviation
 * handles with it switched on), else 0 (also for a NULL handle). */
int lbm_get_temperature_fp64(lbm_t h);

/* Use tile shape `index` (0 <= index < lbm_tile_count(h); 0 is the default)
 * for the fused step from now on, instead of the autotuner's choice.  Every
 * shape computes the same step.  The setting lasts until the next lbm_init,
 * lbm_autotune or closure change (those re-select the remembered or default
 * shape).  Does not synchronise.
 * Errors: LBM_EINVAL (NULL handle, index out of range). */
int lbm_set_tile(lbm_t h, int index);

/* Kernel launches enqueued by this handle since creation (for accounting). */
long long lbm_launch_count(lbm_t h);

/* ---- batches ------------------------------------------------------------
 * Many independent instances of one lattice, fluid and precision, each with
 * its own size and x faces, advanced together: every step is one launch of a
 * persistent fused kernel over a work list of (instance, column, plane range)
 * items sorted longest first and taken from an atomic counter, followed by one
 * batched ghost fill; the two launches of a step are captured in a CUDA graph
 * (one per buffer parity).  Results are bit-identical to stepping each
 * instance alone.  Instances are numbered 0..n-1; all per-instance calls take
 * that index.  The batch uses its own non-blocking stream unless
 * lbm_batch_set_stream gives one (the default stream cannot be captured). */
typedef struct lbm_batch_s* lbm_batch_t;

/* n instances of sizes Nx[k] x Ny[k] (x Nz[k] for D3Q27; Nz may be NULL for
 * D2Q9); eos, tau, Pr, cv as for lbm_create, shared by all instances.
 * Errors: LBM_EINVAL, LBM_ENOMEM, LBM_ECUDA (message: lbm_batch_last_error). */
int lbm_batch_create(lbm_batch_t* out, int lattice, int n, const int* Nx, const int* Ny, const int* Nz,
                     const lbm_eos* eos, double tau, double Pr, double cv);
/* lbm_set_boundary for instance k. */
int lbm_batch_set_boundary(lbm_batch_t b, int k, int face, int type, const double* state);
/* lbm_set_shock_capturing for instance k, or for every instance with k = -1.
 * The batched step then runs the shock-capturing stencils (Sec. 4.4) of all
 * instances with it on in D + 2 further launches per step, one block per row
 * of those instances.  Errors: as lbm_set_shock_capturing, LBM_EINVAL (bad k). */
int lbm_batch_set_shock_capturing(lbm_batch_t b, int k, double C_mu, double C_eta, double C_k);
/* Use a caller stream (non-NULL) instead of the batch's own. */
int lbm_batch_set_stream(lbm_batch_t b, void* stream);
/* lbm_init for instance k (host arrays); may be called at any step. */
int lbm_batch_init(lbm_batch_t b, int k, const double* rho, const double* u, const double* T);
/* Advance every instance n steps (n graph launches), then read the status
 * words of all instances.  Errors: LBM_ESTATE (an instance not initialised,
 * or unstable since its last init), LBM_EUNSTABLE, LBM_EINVAL, LBM_ECUDA. */
int lbm_batch_step(lbm_batch_t b, int n);
/* Same without the status read (no synchronisation). */
int lbm_batch_step_async(lbm_batch_t b, int n);
/* Wait for the batch stream and report the status words as lbm_batch_step. */
int lbm_batch_sync(lbm_batch_t b);
/* lbm_moments for instance k. */
int lbm_batch_moments(lbm_batch_t b, int k, double* rho, double* u, double* T, double* totals);
/* Status bits (LBM_FLAG_*) of instance k since its last init. */
int lbm_batch_flags(lbm_batch_t b, int k, unsigned* flags);
/* Time each tile shape of the batched kernel for `reps` steps from the
 * current state (spare buffers only; the state does not advance) and keep the
 * fastest.  *chosen and *ms_per_step may be NULL. */
int lbm_batch_autotune(lbm_batch_t b, int reps, int* chosen, float* ms_per_step);
/* Interior nodes summed over the instances. */
long long lbm_batch_nodes(lbm_batch_t b);
/* Kernel launches enqueued by the batch's steps (2 per step, D + 4 with shock
 * capturing on in any instance). */
long long lbm_batch_launch_count(lbm_batch_t b);
/* Free the batch and all its instances.  lbm_batch_destroy(NULL) is a no-op. */
int lbm_batch_destroy(lbm_batch_t b);
/* Message of the last failed lbm_batch_* call on this thread. */
const char* lbm_batch_last_error(void);

/* Conservation totals of caller-provided FP64 device fields, with no memory
 * allocation of any kind (the paper has no counterpart: this is a service
 * for callers that cannot allocate).  For example, code that is capturing a
 * stream into a CUDA graph may not call cudaMalloc; a real-time loop may run
 * under a fixed device-memory budget; a host framework may route every
 * allocation through its own pool.  Such callers cannot use a handle (whose
 * creation allocates) but can still reduce fields they already own.
 *   lattice: LBM_D2Q9 or LBM_D3Q27 (D = 2 or 3).
 *   n: number of nodes, 1 <= n <= 67,108,864 (the fixed scratch holds 8192
 *      blocks of 8192 nodes); larger n is rejected with LBM_EINVAL.
 *   d_rho, d_T: n doubles; d_u: D planes of n doubles (layout of lbm_moments).
 *   a, cv: van der Waals a and c_v, for rho E = rho (c_v T - a rho + u^2/2).
 *   d_totals: device output of D+2 doubles (sum rho, sum rho u_1..u_D,
 *      sum rho E), the same quantities as the totals of lbm_moments.
 *   stream: cudaStream_t (as void*) on which the two kernels are enqueued;
 *      the call returns without waiting.
 * The block partials live in one file-scope device array of 320 KiB that
 * every GPU loading the library holds until exit.  The first call on a
 * device looks up that array's device address (cudaGetSymbolAddress) with
 * the device current; make that first call before any stream capture.  All
 * calls on a device share the array, which keeps the last call's contents;
 * every call overwrites all the partials it reads, so nothing needs
 * clearing, but calls that overlap on the GPU race and give wrong totals.
 * The looked-up address is kept for the life of the process: after
 * cudaDeviceReset (or any teardown of the device's primary context) it is
 * stale, and the entry point must not be called again in that process.
 * An error left pending by earlier, unrelated CUDA work is cleared before
 * the launches, so that a launch failure reported here is this call's own.
 * Errors: LBM_EINVAL (bad lattice, NULL pointer, n out of range), LBM_ECUDA;
 * the message is returned by lbm_totals_noalloc_error(). */
int lbm_totals_noalloc(int lattice, long long n, const double* d_rho, const double* d_u, const double* d_T,
                       double a, double cv, double* d_totals, void* stream);
const char* lbm_totals_noalloc_error(void);

/* Free all resources of the handle.  lbm_destroy(NULL) is a no-op. */
int lbm_destroy(lbm_t h);

/* Test hook for the out-of-memory paths: the k-th device allocation that the
 * library makes from now on (counted over all handles and batches of the
 * process) fails as cudaMalloc does when memory is exhausted, without
 * allocating, so that the calling entry point returns LBM_ENOMEM after
 * releasing what it had allocated; k = 0 disarms it.  Production code has no
 * reason to call it.  Errors: LBM_EINVAL (k < 0). */
int lbm_debug_fail_alloc(int k);

/* Population accesses of the step kernels (fused, multi-pass, ghost fill,
 * initialisation) that fell outside the handle's population buffers since the
 * library was loaded, in a library built with -DLBM_BOUNDS_CHECK (each such
 * access is skipped: a load gives 0, a store is dropped); -1 in other builds,
 * which compile the checks away.  A test hook, like lbm_debug_fail_alloc. */
long long lbm_debug_bounds_violations(void);

/* Human-readable description of the last error on this thread. */
const char* lbm_last_error(void);

/* Library version string. */
const char* lbm_version(void);

#ifdef __cplusplus
}
#endif

#endif /* LBM_H */
