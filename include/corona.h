/*
 * corona.h -- C ABI of the GB300 (sm_103a) library for the finite-volume
 * ideal-MHD + GLM residual of a global coronal model (arXiv 2209.04481).
 *
 * The operator: on a spherical shell r in [r_in, r_out] (1 -> 21.5 R_sun) with
 * N_r x N_theta x N_phi cells (geometric radial stretch, uniform theta and phi,
 * poles included), the residual R = dU/dt of the conservative state
 * U = (rho, rho V, B, E, psi):
 *   - ideal MHD in Alfven-speed units with gravity (Sect. 2.2 system; the
 *     printed 8 pi / 4 pi factors are absorbed by the Sect. 2.1 reference
 *     values), E = p/(gamma-1) + rho V^2/2 + B^2/2;
 *   - second-order finite volumes (Sect. 2.1) with limited linear
 *     reconstruction of the primitives (rho, V, B, p, psi);
 *   - Rusanov face fluxes with GLM hyperbolic divergence cleaning, cleaning
 *     speed c_h (Sect. 2.1; c_h = 1 in Sect. 3.3);
 *   - inner boundary of Sect. 3.2 ("low E"): B_r prescribed from a
 *     magnetogram, B_theta and B_phi Neumann, V_b parallel to B_b so that
 *     E_b = -V_b x B_b = 0, psi_b = 0 (Sect. 3.3);
 *   - outer boundary of Sect. 4.1 / Table 2 (rho, p ~ r^-a, B_r ~ r^-b,
 *     psi_b = 0), across-pole theta ghosts, periodic phi;
 *   - gravity source rho g, rho g.V (Sect. 2.2), g = -g0 rhat / r^2;
 *   - the residual monitor res(a) = log10 ||a^t - a^{t+1}||_2 of Sect. 2.1.
 *
 * Layout of every state-like array: structure of arrays, variable-major,
 * U[v][k][j][i] with v = 0..8 (rho, rho Vx, rho Vy, rho Vz, Bx, By, Bz, E, psi),
 * k = r index, j = theta index, i = phi index (contiguous).  Vector components
 * are Cartesian.  Element type: double for CRN_FP64 grids, float for
 * CRN_FP32_BULK grids (the bulk flux arithmetic in FP32; pressure recovery in
 * low-beta cells, norms and the pseudo-time update in FP64).
 *
 * Pointers named *_dev are device pointers on the grid's device; the library
 * never frees caller memory and allocates only in crn_grid_create.  All
 * compute calls are asynchronous on the given stream (a cudaStream_t passed as
 * void*, NULL = the legacy default stream) and never synchronise, except
 * crn_sync_status.  Functions return a crn_status; argument errors are
 * reported synchronously, errors detected by kernels are sticky in the grid's
 * device error word until crn_sync_status reads and clears them.
 */
#ifndef CORONA_H
#define CORONA_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  CRN_OK = 0,
  CRN_E_ARG = 1,          /* bad pointer, size, layout or descriptor field      */
  CRN_E_CUDA = 2,         /* CUDA runtime / launch error (text: crn_last_error)  */
  CRN_E_NONPHYSICAL = 3,  /* kernel saw rho <= 0, p <= 0 or a non-finite value   */
  CRN_E_TIMEOUT = 4,      /* a bounded device wait gave up                       */
  CRN_E_STATE = 5         /* call out of order (e.g. no inner boundary set)      */
} crn_status;

typedef enum { CRN_FP64 = 0, CRN_FP32_BULK = 1 } crn_precision;
typedef enum { CRN_LIM_NONE = 0, CRN_LIM_MINMOD = 1, CRN_LIM_VANALBADA = 2 } crn_limiter;
/* Residual kernel.  TILED (default) and TILED_REGS: the tiled kernel, raw
 * state prefetched in registers by plain per-thread loads (any shape, FP32 and
 * FP64).  STAGED (FP32_BULK only): each plane's own 8 x 32 block arrives by a
 * TMA tensor copy and the halo by cp.async; it needs n_theta a multiple of 8,
 * n_phi a multiple of 32 and a 16-byte aligned state, else the tiled kernel
 * runs.  It computes the same residual and is slower on GB300 (127 us against
 * 86 us on 128 x 64 x 128).  CELLWISE: a simple reference kernel, one thread
 * per cell.  crn_last_kernel reports the kernel that ran. */
typedef enum {
  CRN_KERNEL_TILED = 0,
  CRN_KERNEL_CELLWISE = 1,
  CRN_KERNEL_TILED_REGS = 2,
  CRN_KERNEL_STAGED = 3
} crn_kernel;
/* Inner-boundary formulation (Sect. 3.2): LOW_E: B_r prescribed, B_theta and
 * B_phi Neumann, V_b parallel to B_b (E_b = 0), |V_b| from the interior
 * velocity projected on B_b.  LARGE_E: the Wind-Predict form, B_r and B_theta
 * prescribed (from a potential field), B_phi Neumann, V_b = V_par (B_r rhat +
 * B_theta thetahat), V_par = V_r* B_r / B_pol^2.  LOW_E_WP: as LOW_E but with
 * the prescribed Wind-Predict outflow magnitude, V_b = V_r* B_r B_b / |B_b|^2
 * (E_b = 0; V_b does not depend on the interior velocity). */
typedef enum { CRN_INNER_LOW_E = 0, CRN_INNER_LARGE_E = 1, CRN_INNER_LOW_E_WP = 2 } crn_inner_bc;

/* Grid and physics description.  crn_grid_desc_default fills the solar-wind
 * defaults: r in [1, 21.5], gamma = 1.05, c_h = 1, g0 = 0.8271 (G M_sun /
 * (R_sun V_ref^2) with V_ref = B_ref / sqrt(mu0 rho_ref) of Sect. 2.1), van
 * Albada limiter with eps = 1e-12, outer laws of Table 2 case 3 (a = b = 2,
 * B_phi, V zero-gradient, psi_b = 0), rho_b = 1, p_b = 0.0827, low-E inner
 * boundary, V_r* = 1935.07 m/s / V_ref (Sect. 3.2) for the large-E form,
 * FP32_BULK, tiled kernel.  The outer laws cover all cases of Table 2 and the
 * rho ~ r^-2.5 law of Sect. 4.2 (outer_rho_exp = 2.5). */
typedef struct {
  int32_t n_r, n_theta, n_phi;  /* cells; n_phi even and a multiple of 8         */
  int32_t precision;            /* crn_precision                                 */
  int32_t limiter;              /* crn_limiter                                   */
  int32_t kernel;               /* crn_kernel                                    */
  double r_in, r_out;           /* shell radii, 0 < r_in < r_out                 */
  double gamma;                 /* ratio of specific heats, > 1                  */
  double c_h;                   /* GLM cleaning speed, >= 0                      */
  double g0;                    /* gravity: g = -g0 rhat / r^2                   */
  double lim_eps;               /* van Albada epsilon: > 0 with that limiter
                                   (its smooth form is 0/0 where both slopes
                                   vanish), else ignored but >= 0             */
  double outer_rho_exp;         /* outer ghost rho, p scaled by (r_I/r_G)^a      */
  double outer_br_exp;          /* outer ghost B_r scaled by (r_I/r_G)^b         */
  double rho_b, p_b;            /* inner boundary density and pressure, > 0      */
  int32_t inner_bc;             /* crn_inner_bc                                  */
  int32_t outer_vr_mass;        /* outer ghost V_r: 0 zero-gradient, 1 V_r r^2 rho = const */
  int32_t outer_psi_extrap;     /* outer ghost psi: 0 psi_b = 0, 1 zero-gradient */
  int32_t reserved_;            /* must be 0                                     */
  double vr_star;               /* large-E: prescribed radial outflow V_r*       */
  double outer_bphi_exp;        /* outer ghost B_phi scaled by (r_I/r_G)^c       */
  double outer_vphi_exp;        /* outer ghost V_phi scaled by (r_I/r_G)^e       */
  double r_last;                /* 0: geometric radial faces r_k = r_in (r_out/r_in)^(k/n_r);
                                   in (r_in, r_out): n_r - 1 geometric cells up to r_last
                                   and one thin last cell [r_last, r_out], the mesh with a
                                   small outer ghost of Sect. 4.3 (not for crn_residual_static) */
  double psi_damp;              /* GLM damping rate alpha >= 0: source -alpha psi in the psi
                                   equation (0, the default: the undamped cleaning of Sect. 2.1) */
} crn_grid_desc;

typedef struct crn_grid crn_grid;

/* Fill *d with the defaults above for an n_r x n_theta x n_phi shell.
 * Returns CRN_E_ARG if d is NULL. */
int crn_grid_desc_default(crn_grid_desc* d, int32_t n_r, int32_t n_theta, int32_t n_phi);

/* Radial planes per CTA that crn_grid_create gives the tiled residual: the
 * chunk whose CTAs, list-scheduled in launch order (all `ntiles` (theta, phi)
 * tiles of chunk 0, then chunk 1, ...) onto `slots` resident CTAs, each costing
 * its planes plus `overhead` planes (crn_grid_create uses 3), finish first;
 * ties go to the larger chunk; at least 4 planes (n_r if smaller).  Pure host
 * function; -1 on a non-positive argument. */
int32_t crn_tiled_radial_chunk(int32_t n_r, int64_t ntiles, int64_t slots, int32_t overhead);

/* Create a grid on the current CUDA device: validates *d (CRN_E_ARG with a
 * message on any bad field), computes the exact face-area vectors and volumes
 * of the shell on the host in FP64 as 1D radial factors times per-column
 * angular factors and unit normals, uploads them (cast once to FP32 for
 * FP32_BULK grids), and allocates the grid-owned scratch: reduction partials,
 * error word, B_r copy, and the residual / FP32 shadow buffers used by
 * crn_pseudo_time_step.  *out receives the handle (NULL on error).
 * Synchronous.  Thread-compatible: one grid must not be used from two host
 * threads at once. */
int crn_grid_create(const crn_grid_desc* d, crn_grid** out);

/* Free everything crn_grid_create allocated (synchronises the device first).
 * NULL is accepted. */
int crn_grid_destroy(crn_grid* g);

/* Prescribe the inner-boundary radial field B_r [Sect. 1 and 3.2: B_r from the
 * magnetogram at the inner boundary].  Br_dev: FP64 device array
 * [n_theta][n_phi], B_r at the inner face centres (theta_c, phi_c); for
 * CRN_INNER_LARGE_E grids [2][n_theta][n_phi]: B_r, then B_theta.  Copied
 * into grid-owned storage asynchronously on the stream (the caller may reuse
 * its buffer once the stream has passed this point).  Must precede the first
 * residual / pseudo-time call (CRN_E_STATE otherwise). */
int crn_set_inner_boundary(crn_grid* g, const double* Br_dev, void* stream);

/* One residual evaluation R = dU/dt (per unit volume).  U_dev, R_dev: caller
 * device buffers of 9 * n_r * n_theta * n_phi elements of the grid's precision
 * (double for FP64, float for FP32_BULK), SoA layout above; they must not
 * overlap.  norms9_dev (optional, may be NULL): 9 doubles, the L2 norm over the
 * cells of each residual variable.  dtmin_dev (optional): 1 double,
 * min over cells of V_c / sum_f lambda_f |S_f| (the explicit step bound at
 * CFL 1).  Asynchronous; no allocation; no host synchronisation. */
int crn_residual(crn_grid* g, const void* U_dev, void* R_dev, double* norms9_dev,
                 double* dtmin_dev, void* stream);

/* Vector-Jacobian product of the residual (the adjoint of every step of
 * crn_residual: recovery, ghosts, limited reconstruction, Rusanov + GLM flux,
 * accumulation, gravity): Ubar = (dR/dU)^T Rbar (same layout and precision as
 * U) and Brbar = (dR/dB_r)^T Rbar (FP64 [n_theta][n_phi]), both overwritten.
 * Rbar_dev has the layout of R.  Brbar_dev may be NULL; for CRN_INNER_LARGE_E
 * grids it is [2][n_theta][n_phi] (cotangents of B_r and B_theta).  Face states are
 * recomputed, not stored.  Non-smooth points: max passes the derivative to
 * its first argument on a tie, d|x|/dx = +1 at 0.
 * CRN_FP32_BULK grids run the tiled VJP: a radial pass over blocks of 16
 * columns x 13 planes and a lateral pass over 8 x 32 (theta, phi) tiles of
 * one plane, every intermediate in shared memory; no scratch, 2 launches.
 * CRN_FP64 grids (and grids created with CRN_KERNEL_CELLWISE) run the
 * face/cell pair: one thread per face, then one per cell, 3 launches (2 with
 * FP32), with a scratch of 36 values of the grid's type per face (about 108
 * per cell) allocated by the grid's first VJP call: make that call before
 * any stream capture.  The environment variable CRN_VJP_KERNEL ("tiled" or
 * "faces"), read at each call, overrides the choice.  Ubar_dev must not
 * overlap U_dev or Rbar_dev (CRN_E_ARG).  Asynchronous. */
int crn_residual_vjp(crn_grid* g, const void* U_dev, const void* Rbar_dev, void* Ubar_dev,
                     double* Brbar_dev, void* stream);

/* nsteps explicit pseudo-time steps U <- U + dt R(U), dt = cfl * dtmin(U),
 * on the FP64 master state U64_dev (9 * N doubles, updated in place) [the
 * paper's solver steps in pseudo-time to a steady state, Sect. 2.1].  FP32_BULK
 * grids evaluate R on an FP32 shadow of the master and update the master in
 * FP64.  res_log10_dev (optional): nsteps x 9 doubles, the res(a) monitor of
 * Sect. 2.1 for the nine primitives a = (rho, Vx, Vy, Vz, Bx, By, Bz, p, psi):
 * log10 of the L2 norm over the cells of a^t - a^{t+1}.  No host
 * synchronisation; the sequence of launches can be captured in a CUDA graph. */
int crn_pseudo_time_step(crn_grid* g, double* U64_dev, int32_t nsteps, double cfl,
                         double* res_log10_dev, void* stream);

/* One residual evaluation that allocates nothing: the same operator and
 * kernel as crn_residual, for callers that cannot call cudaMalloc (a host
 * framework that fixes the device memory budget, a plugin that may not
 * allocate during a solve, code that must not trigger an allocator's implicit
 * device synchronisation).  The paper has no counterpart: this is a
 * deployment variant of the library, not part of the method.
 * No grid object is needed: *d describes the shell as for crn_grid_create
 * (d->kernel is ignored; the tiled kernel is used).  Br_dev: FP64 device
 * array [n_theta][n_phi] read during the call; U_dev, R_dev, norms9_dev,
 * dtmin_dev as for crn_residual (norms9_dev, dtmin_dev may be NULL).
 * For CRN_INNER_LARGE_E descriptors Br_dev holds [2][n_theta][n_phi].
 * Scratch (geometry, reduction partials, arrival counter, error word) is one
 * fixed device array of about 3.6 MB inside the library, held by every GPU
 * that loads the library until process exit.  Limits: n_r <= 1024,
 * n_theta <= 1024, n_phi <= 2048 (a multiple of 8), n_theta * n_phi <= 32768;
 * larger sizes return CRN_E_ARG (nothing is launched).  The first call on a
 * device, with that device current, resolves the array's address
 * (cudaGetSymbolAddress) and sets kernel attributes: make it before any
 * stream capture.  A call whose geometry fields (sizes, precision, radii, g0)
 * differ from the previous call's rebuilds the geometry on the stream first;
 * a call made while `stream` is being captured records the geometry build
 * with its residual, and from then on every call on that device rebuilds the
 * geometry (a replay may have rebuilt another).  Every call clears the
 * counter and error word it uses
 * and shares the array: calls that overlap on the GPU race and must be
 * serialised by the caller.  Non-physical states (rho <= 0, p <= 0) are not
 * reported by this entry point: there is no status call for it, and such a
 * state need not make the residual or the norms non-finite, so a caller that
 * needs the check makes it on the state.  Van Albada needs lim_eps > 0
 * (CRN_E_ARG otherwise).  Calls no cudaMalloc, cudaFree or other allocating
 * routine.  Asynchronous on `stream`. */
int crn_residual_static(const crn_grid_desc* d, const double* Br_dev, const void* U_dev,
                        void* R_dev, double* norms9_dev, double* dtmin_dev, void* stream);

/* Residuals of `count` independent states in HOST memory: R_host[i] =
 * R(U_host[i]) (layout as crn_residual, the grid's precision), optional
 * norms9_host[i][9] and dtmin_host[i].  The copies run on two internal
 * streams around the residual launches on `stream`, through two device
 * staging slots owned by the grid (allocated by the first call), so that the
 * copy of state i + 1 in, the residual of state i and the copy of R_{i-1} out
 * overlap; page-locked (pinned) host buffers are needed for the copies to
 * overlap.  Synchronous: returns when every result is in host memory. */
int crn_residual_host_batch(crn_grid* g, const void* const* U_host, void* const* R_host, double* norms9_host,
                            double* dtmin_host, int32_t count, void* stream);

/* Boundary electric field diagnostic [Sect. 2.2: E = -V x B; Sect. 3.2
 * compares the inner-boundary E of the low-E and large-E formulations]:
 * E_dev[3][n_theta][n_phi] (FP64, Cartesian components) receives
 * E = -V_b x B_b of the face-mean state (ghost + interior) / 2 at every inner
 * face, computed in FP64 from U_dev (the grid's precision).  Asynchronous. */
int crn_boundary_efield(crn_grid* g, const void* U_dev, double* E_dev, void* stream);

/* Volume electric field [Sect. 2.2: E = -V x B; Sect. 3.1 traces spurious E to
 * the initial state and to the inner boundary]: E_dev[3][n_r][n_theta][n_phi]
 * (FP64, Cartesian components) receives E = -(m x B) / rho of every cell,
 * computed in FP64 from U_dev (the grid's precision).  Needs no inner
 * boundary values.  Asynchronous on `stream`; one launch. */
int crn_efield(crn_grid* g, const void* U_dev, double* E_dev, void* stream);

/* ---- implicit pseudo-time iteration: matrix-free Newton-Krylov ----------
 * The backward-Euler pseudo-time step of Sect. 2.1 with local time steps,
 * linearised once:  (diag(1 / dtau_c) - dR/dU) dU = R(U),  dtau_c = CFL dt_c,
 *   dt_c = V_c / sum_f max(|V_c.n_f| + c_f(W_c, n_f), c_h) |S_f|
 * (the cell's own state on its six faces; pole faces drop out), solved by
 * restarted GMRES on y -> y - J(dtau . y), dU = dtau . y.  J z is the
 * central difference (R(U + eps z) - R(U - eps z)) / (2 eps) of two
 * crn_residual evaluations (or the forward difference against R(U)), eps the
 * largest step that moves no state entry by more than fd_rel of |u| + 1e-3 x
 * (the mean |u| of its variable + the mean |u| over all nine variables) and no
 * cell's pressure by more than a quarter (to first and to second order in eps).  U is then advanced by alpha dU, alpha = min(1,
 * max_rel_change / max_c max(|d rho|/rho, |dp_lin|/p)) (dp_lin the linearised
 * pressure change), halved while any cell would keep less than a tenth of
 * its density or pressure.
 * All vectors are FP64 on the device (the Krylov basis FP32 if basis_fp32
 * selects it); reductions are deterministic. */
typedef struct {
  int32_t krylov_dim;      /* GMRES restart length m, 1..500 (default 30)          */
  int32_t max_restarts;    /* GMRES restarts per step, 0..1000 (default 0)          */
  double lin_rtol;         /* GMRES relative tolerance, (0, 1) (default 1e-3)       */
  double fd_rel;           /* relative FD step b; 0 selects 2^-17 (central) or 2^-26
                              (forward) on FP64 grids, 2^-8 or 2^-12 on FP32-bulk
                              grids (default 0)                                     */
  double max_rel_change;   /* step limiter omega; <= 0 disables it (default 0.3)    */
  int32_t fd_central;      /* 1: central difference (two residuals per product),
                              0: forward difference (default 1)                     */
  int32_t precond;         /* right preconditioner: 0 scales by dtau (a Jacobi step
                              of the local time steps, default), 1 solves the radial
                              line-implicit tridiagonal (Rusanov dissipation part of
                              D - J along each radial column)                        */
  int32_t basis_fp32;      /* Krylov basis of crn_newton_krylov_step / crn_steady_solve:
                              1 FP32 (orthogonalisation on the FP32 pipe, half the
                              bytes; the basis vectors are rounded to FP32, which
                              is far below a loose lin_rtol), 0 FP64, -1 FP32 when
                              lin_rtol >= 1e-4 else FP64 (default -1).  The adjoint
                              solve always uses FP64.                                */
  int32_t adjoint_outer;   /* crn_adjoint_solve with adjoint_cfl > 0: passes of the
                              pseudo-time adjoint iteration, 1..100000 (default 200) */
  double adjoint_cfl;      /* crn_adjoint_solve: 0 (default) runs GMRES on J^T
                              diag(dt_c); > 0 runs the pseudo-time adjoint iteration
                              lambda <- lambda + delta, (D - J^T) delta = J^T lambda
                              - gbar with D = diag(1 / (adjoint_cfl dt_c)), each pass
                              solved by GMRES(krylov_dim) to 1e-1 on the shifted
                              operator (precond as for the primal lines, transposed)  */
  int32_t outer_fp64;      /* FP32-bulk grids: 1 (default) evaluates each step's
                              R(U), the right-hand side and the convergence norm, with
                              the FP64 residual on the FP64 state, so that the solve
                              converges past the FP32 rounding of the residual; the
                              Jacobian-vector products stay FP32-bulk.  0: R(U) in
                              FP32 bulk too.  Likewise in crn_adjoint_solve with
                              adjoint_fgmres > 0: the outer products J^T z, the true
                              residual and the sensitivity from the FP64 VJP of the
                              FP64 state, the passes with the FP32 VJP.  Ignored on
                              FP64 grids.                                            */
  int32_t adjoint_fgmres;  /* crn_adjoint_solve with adjoint_cfl > 0: > 0 (default 30)
                              accelerates the passes by flexible GMRES on J^T lambda =
                              gbar with restart length min(adjoint_fgmres, krylov_dim),
                              each pass its right preconditioner (one more vector of
                              9N doubles per direction, allocated by the first such
                              call); 0 runs the plain pass iteration.  adjoint_outer
                              bounds the passes either way.                           */
} crn_nk_options;

typedef struct {
  double res_l2;           /* ||R(U)||_2 over all 9N entries before the step        */
  double lin_rel;          /* GMRES relative residual estimate at exit              */
  double alpha;            /* step length applied                                   */
  int32_t krylov_iters;    /* Arnoldi steps (one Jacobian-vector product each)      */
  int32_t residual_evals;  /* residual evaluations of the step                      */
} crn_nk_stats;

/* The CFL law of Sect. 4.1: cfl0 (2), doubled every cfl_double_every steps
 * up to cfl_max (128). */
typedef struct {
  double cfl0, cfl_max;
  int32_t cfl_double_every;  /* default 10                                          */
  int32_t max_steps;         /* default 500                                         */
  double tol_drop;           /* stop once ||R||_2 <= tol_drop ||R(U0)||_2 (1e-6)    */
  crn_nk_options nk;
} crn_steady_options;

typedef struct {
  double res0, res_final;    /* ||R||_2 of the initial and of the final state        */
  int32_t steps;             /* updates applied                                     */
  int32_t krylov_iters;      /* Jacobian-vector products over the solve             */
  int32_t residual_evals;    /* residual evaluations over the solve                 */
  int32_t converged;         /* 1 if the drop tol_drop was reached                  */
} crn_steady_stats;

int crn_nk_options_default(crn_nk_options* o);
int crn_steady_options_default(crn_steady_options* o);

/* dtau_dev[n_r][n_theta][n_phi] = cfl dt_c from the FP64 state U64_dev
 * (device).  Asynchronous on `stream`. */
int crn_local_dt(crn_grid* g, const double* U64_dev, double cfl, double* dtau_dev, void* stream);

/* One Newton-Krylov pseudo-time step at CFL `cfl` on the FP64 master state
 * U64_dev[9][N] (device, updated in place to U + alpha dU).  The residual runs
 * in the grid's precision (FP32-bulk grids evaluate it on an FP32 copy).
 * dU_dev (device, optional) receives dU before alpha; stats (host, optional)
 * the step's figures.  The first call allocates the workspace ((m + 5) 9N
 * doubles and 3 x 9N of the grid type).  Synchronises `stream` several times
 * per Krylov step (the host runs the GMRES recurrences).  Returns
 * CRN_E_NONPHYSICAL if R(U) flags a cell or no alpha keeps rho, p > 0. */
int crn_newton_krylov_step(crn_grid* g, double* U64_dev, double cfl, const crn_nk_options* opt,
                           double* dU_dev, crn_nk_stats* stats, void* stream);

/* Steady solve: Newton-Krylov steps under the CFL law until ||R(U)||_2 <=
 * tol_drop ||R(U0)||_2 or max_steps updates.  history (host, optional)
 * receives per pass (cfl, ||R||_2, alpha, krylov_iters), at most history_len
 * rows of 4 doubles; the last row is the final residual check. */
int crn_steady_solve(crn_grid* g, double* U64_dev, const crn_steady_options* opt, crn_steady_stats* stats,
                     double* history, int32_t history_len, void* stream);

/* ---- ensembles: many shells in one persistent launch ---------------------
 * An ensemble borrows n grids (one precision and limiter, any sizes; they
 * must outlive it and must not run their own calls while an ensemble call
 * on them is in flight).  One persistent launch of the tiled residual takes
 * work items (member, (theta, phi) tile, radial chunk) from a device counter
 * until all members are done; every member's R, norms and dtmin are those of
 * its own crn_residual (bitwise with the same radial chunk).  Arrays of
 * per-member device pointers are host arrays of n entries. */
typedef struct crn_ensemble crn_ensemble;

/* CRN_E_ARG if a member is NULL or the members differ in precision, limiter
 * or device. */
int crn_ensemble_create(crn_grid* const* grids, int32_t n, crn_ensemble** out);
int crn_ensemble_destroy(crn_ensemble* e);

/* Radial planes per work item for every member (their tile shapes are kept);
 * 0 (default) uses each member's own choice (the one its crn_residual uses).
 * crn_ensemble_kchunk returns the last value set for all members, or after
 * crn_ensemble_autotune the chunk of its largest size class. */
int crn_ensemble_set_kchunk(crn_ensemble* e, int32_t kchunk);
int32_t crn_ensemble_kchunk(const crn_ensemble* e);

/* R_dev[m] = R(U_dev[m]) for every member in one launch; norms9_dev
 * ([n][9]) and dtmin_dev ([n]) are optional device outputs.  Asynchronous. */
int crn_ensemble_residual(crn_ensemble* e, const void* const* U_dev, void* const* R_dev, double* norms9_dev,
                          double* dtmin_dev, void* stream);

/* nsteps explicit pseudo-time steps of every member's FP64 master state
 * U64_dev[m] (as crn_pseudo_time_step, each member with its own dt = cfl x its
 * dtmin): per step one ensemble residual launch and one batched update
 * launch.  res_log10_dev ([n][9], optional, device) receives the res(a)
 * monitor of the last step.  Asynchronous. */
int crn_ensemble_pseudo_time_step(crn_ensemble* e, double* const* U64_dev, int32_t nsteps, double cfl,
                                  double* res_log10_dev, void* stream);

/* Tile autotuner.  Members are grouped in size classes (equal n_theta and
 * n_phi).  For each class it times the persistent launch over that class's
 * members alone (one warm-up, three timed launches, CUDA events) for each tile
 * shape (8 x 32 and 16 x 16 (theta, phi) columns per CTA) and each radial chunk
 * (the members' own, 4, 6, 8, 12, 16, 24, 32, 48 planes per item), and keeps
 * the fastest pair for the class's members (crn_ensemble_member_config reads
 * it back).  *kchunk_out receives the chunk chosen for the class with the most
 * cells.  R is the same for every tile shape and chunk up to rounding (the
 * first r face of a chunk is evaluated on the CTA's preamble path).
 * Synchronises `stream`; R_dev is overwritten. */
int crn_ensemble_autotune(crn_ensemble* e, const void* const* U_dev, void* const* R_dev, void* stream,
                          int32_t* kchunk_out);

/* Tile shape (0: 8 x 32, 1: 16 x 16 (theta, phi) columns per CTA) and radial
 * chunk (planes per work item; 0 = the member's own single-launch chunk) of
 * member m in the persistent launch.  CRN_E_ARG for an index, shape or chunk
 * out of range; a chunk that gives a member more work items than its
 * reduction scratch holds is rejected by the next residual call. */
int crn_ensemble_set_member_config(crn_ensemble* e, int32_t m, int32_t tile, int32_t kchunk);

/* The tile shape and radial chunk (in planes, resolved) member m runs with. */
int crn_ensemble_member_config(const crn_ensemble* e, int32_t m, int32_t* tile, int32_t* kchunk);

/* Kernel launches issued by the last call of the ensemble. */
int32_t crn_ensemble_launch_count(const crn_ensemble* e);

/* Sensitivity of a functional g(U) of a steady state U* (R(U*, B_b) = 0) to
 * the prescribed inner field B_b (B_r, or (B_r, B_theta) for large-E):
 * solves J^T lambda = gbar (J = dR/dU at U64_dev, gbar = dg/dU, FP64 [9][N],
 * device) by GMRES on J^T diag(dt_c) with the hand-written VJP of
 * crn_residual_vjp, and writes sens_dev = dg/dB_b = -(dR/dB_b)^T lambda
 * (FP64, the shape crn_set_inner_boundary takes) and, if lambda_dev is not
 * NULL, lambda.  opt: krylov_dim, max_restarts, lin_rtol and precond are used
 * (precond 1: the transposed radial line preconditioner, the lines of
 * crn_nk_options.precond at infinite CFL, negated and transposed).  With
 * opt->adjoint_cfl > 0 the solve is the pseudo-time adjoint iteration
 * described at that field, stopped at |gbar - J^T lambda| <= lin_rtol |gbar|
 * or after adjoint_outer passes; stats->lin_rel then holds that true relative
 * residual and stats->alpha the number of passes.  The first call allocates
 * the Newton-Krylov and VJP workspaces.  Synchronises `stream` once or twice
 * per Krylov step. */
int crn_adjoint_solve(crn_grid* g, const double* U64_dev, const double* gbar_dev, double* lambda_dev,
                      double* sens_dev, const crn_nk_options* opt, crn_nk_stats* stats, void* stream);

/* Synchronise the stream, then read and clear the grid's device error word.
 * Returns CRN_E_NONPHYSICAL if a kernel saw a non-physical state since the
 * last call (crn_last_bad_cell gives the lowest flagged cell index,
 * k * n_theta * n_phi + j * n_phi + i), CRN_E_TIMEOUT if a kernel's bounded
 * wait for an asynchronous (TMA) copy gave up (its outputs are then invalid),
 * CRN_E_CUDA on a CUDA error. */
int crn_sync_status(crn_grid* g, void* stream);

/* Lowest flat cell index flagged by the last crn_sync_status, -1 if none. */
int64_t crn_last_bad_cell(const crn_grid* g);

/* Message of the last error returned on the calling host thread ("" if none). */
const char* crn_last_error(void);

/* Number of kernel launches the last compute call of this grid issued. */
int32_t crn_last_launch_count(const crn_grid* g);

/* The residual kernel (crn_kernel: CELLWISE, TILED_REGS or STAGED) that the
 * last residual evaluation of this grid launched; -1 before the first one or
 * for a NULL grid. */
int32_t crn_last_kernel(const crn_grid* g);

#ifdef __cplusplus
}
#endif

#endif /* CORONA_H */
