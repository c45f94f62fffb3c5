/*
 * sd.h -- C ABI of the GB300-native monolithic Stokes-Darcy solver.
 *
 * Method (arXiv 2108.13229): the time-dependent Stokes-Darcy problem of
 * Sec. 2 (Eqs. (1)-(7)), discretised by backward Euler in time, MAC
 * staggered finite volumes in the free flow and cell-centred TPFA in the
 * porous medium, gives one linear system per time step, Eq. (8)/(9):
 *
 *     [ V    B   B'_1 ] [ v^ff ]   [ g ]
 *     [ C    0   0    ] [ p^ff ] = [ 0 ]
 *     [ C'_1 0   D'   ] [ p^pm ]   [ 0 ]
 *
 * solved monolithically by a flexible GMRES(m) with a block preconditioner
 * of the kind built in Sec. 4 (the zero block replaced, V and D' handled by
 * their own preconditioners -- here geometric multigrid V-cycles).
 *
 * Geometry: free flow [0,1]x[1,2] over porous medium [0,1]x[0,1], n x n
 * cells each, interface y = 1.  Whole-system vectors use the layout
 *     u    (n+1) x n  vertical ff faces, index j*(n+1)+i
 *     v    n x (n+1)  horizontal ff faces, index j*n+i   (j = 0 on the interface)
 *     p_ff n x n      ff cell centres, index j*n+i
 *     p_pm n x n      pm cell centres, index j*n+i       (j = 0 at y = 0)
 * concatenated in this order, 4n^2 + 2n doubles (the DoF count of Table 1).
 *
 * Conventions for every function:
 *  - returns SD_OK (0) or a negative SD_E_* code; sd_strerror() names it;
 *    no C++ exception crosses this interface;
 *  - every array argument may be host memory or CUDA device memory of the
 *    current device (the library inspects the pointer); it is owned by the
 *    caller and is not retained after the call returns;
 *  - a handle owns all device memory it allocates until sd_destroy();
 *    calls on one handle are serialised by the handle; distinct handles may
 *    be used from distinct threads at the same time.
 */
#ifndef SD_H
#define SD_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define SD_OK 0
#define SD_PENDING 1       /* sd_poll: the request is queued or running */
#define SD_E_INVAL -1      /* invalid argument (grid, mu, K, alpha_BJ, dt, options) */
#define SD_E_NOMEM -2      /* device memory (or the server's HBM budget) exhausted */
#define SD_E_NOCONV -3     /* max_iters reached; the state holds the last iterate */
#define SD_E_NUMERIC -4    /* NaN/Inf in the Krylov recurrence */
#define SD_E_TIMEOUT -5    /* reserved: no call returns it (nothing in the library waits on the device) */
#define SD_E_CUDA -6       /* a CUDA runtime call failed */
#define SD_E_STATE -7      /* unknown ticket, or call not valid in this state */

/* precision of the multigrid V-cycles inside the preconditioner; the outer
   FGMRES (residual, Gram-Schmidt, Hessenberg least squares) and the
   coarsest-grid solves are always FP64 */
#define SD_FP64 0
#define SD_MIXED 1

/* block preconditioner (Sec. 4):
   SD_TRI_SCHUR  block upper-triangular on (v, p_ff) with the zero block
                 replaced by a Schur approximation S^, S^-1 = (mu/(gamma h^2)) I
                 + (1/dt) L_p^-1 (viscous plus mass-dominated parts of
                 B^T V^-1 B), then the Darcy block after the velocity (C'_1
                 coupling kept): z_pff, z_v, z_pm;
   SD_PV_BJ_I    pressure-velocity block Jacobi P^pv_BJ(P_V, P_D') with the
                 identity on the p_ff block (Sec. 4);
   SD_PV_BGS_I   pressure-velocity block Gauss-Seidel P^pv_BGS(P_V, P_D')
                 with the identity on the p_ff block (Sec. 4). */
#define SD_TRI_SCHUR 0
#define SD_PV_BJ_I 1
#define SD_PV_BGS_I 2

/* boundary conditions and data:
   SD_BC_MMS           manufactured solution: Dirichlet ff velocity on the top
                       and the sides x = 0, 1, Dirichlet pressure at the pm
                       bottom, no flow through the pm sides; the state starts
                       at the exact solution of t = 0;
   SD_BC_MMS_TRACTION  the same solution with traction ff sides: on x = 0, 1
                       the normal stress -p + 2 mu du/dx and the tangential
                       velocity are prescribed (from the solution), and the
                       side u faces are unknowns whose rows are the x-momentum
                       balance of the half control volume inside the domain
                       (corner shear at half distance from the side's
                       tangential velocity, the interface corner through the
                       eliminated BJS slip of Eq. (6));
   SD_BC_PAPER         the pressure-driven problem of Sec. 5 on the square
                       geometry of Table 1: traction sides with the inflow
                       pressure p_in(t) = bc_dp (1 - cos(pi min(t, T)/T)) / 2
                       on the left (a half-cosine rise over [0, T], T =
                       bc_tend or 25 time steps when 0) and 0 on the right,
                       no tangential velocity on the sides, no slip on the
                       top, p = 0 at the pm bottom, no flow through the pm
                       sides, no sources; the state starts at rest. */
#define SD_BC_MMS 0
#define SD_BC_MMS_TRACTION 1
#define SD_BC_PAPER 2

/* geometry of the free flow over the n x n porous medium [0,1] x [0,1]:
   SD_GEO_SQUARE   the free flow [0,1] x [1,2], n x n cells (Table 1);
   SD_GEO_CHANNEL  the channel of the model problem of Sec. 5: free flow
                   [-1,2] x [1,2], 3n x n cells, whose floor's middle third
                   (x in [0,1]) is the interface and the rest a no-slip wall.
                   The boundary conditions of bc apply at the channel's ends
                   x = -1, 2 (the manufactured solution continued in x; the
                   pressure-driven problem's inflow on the left end); the
                   floor faces beside the interface are Dirichlet rows, their
                   values eliminated from the other rows.  Unknowns: 10 n^2 +
                   4 n (sd_dof_count_geometry).  Dense state vectors use the
                   layout [u | v | p_ff | p_pm] with u (3n+1) x n, v 3n x
                   (n+1), p_ff 3n x n and p_pm n x n, x fastest.  The channel
                   runs the monolithic coupling only, smooths in shared-memory
                   tiles for tile 1 and 2 (register-column tiles, tile 2, for
                   its Darcy block only; no fused coarse cycle: fuse_coarse
                   does not apply), and coarsens to
                   at most 8 x 8 porous-medium cells (coarsest above 8 counts
                   as 8), so n = m 2^k needs m <= 8. */
#define SD_GEO_SQUARE 0
#define SD_GEO_CHANNEL 1

/* coupling of the two subdomains in a time step:
   SD_MONOLITHIC  one block-preconditioned FGMRES solve of Eq. (9) (Sec. 4);
   SD_PARTITIONED the partitioned iteration of Sec. 3: the porous-medium
                  solver takes the interface normal velocity as flux data
                  (Eq. (7)) and passes on the pressure of the cells below the
                  interface; the free-flow solver takes that pressure into the
                  normal-stress balance of the interface faces (Eq. (5)) and
                  passes on the new interface velocity (or the two run in the
                  order of Sec. 3, coupling_order); the fixed-point residual
                  R(v) = S_ff(S_pm(v)) - v (or S_pm(S_ff(v)) - v) is driven to zero by
                  IQN-ILS post-processing (relaxed first step, least-squares
                  inverse-Jacobian model from the differences of the time
                  step's earlier iterations), stopping when the exchanged
                  pressure and velocity both change by less than coupling_eps
                  relative (the test of Sec. 3).  Each subdomain solve is an
                  FGMRES on that subdomain's rows of Eq. (9) with the other
                  side's data fixed, preconditioned by the same V-cycles (V and
                  Schur blocks / D' block), to coupling_rtol.  The converged state is
                  the monolithic solution.  The order of the two solves:
                  coupling_order below. */
#define SD_MONOLITHIC 0
#define SD_PARTITIONED 1

/* order of the subdomain solves of SD_PARTITIONED:
   SD_ORDER_FF_FIRST  Sec. 3's order: the free flow takes the interface
                      velocity as Dirichlet data (identity v_Gamma rows) and
                      returns the interface pressure, the normal stress that
                      balances the v_Gamma half control volumes (Eq. (5));
                      the porous medium takes that pressure on its top
                      boundary over the half cell below the interface and
                      returns the Darcy velocity through it (Eq. (7)).  Needs
                      traction free-flow sides (SD_BC_MMS_TRACTION,
                      SD_BC_PAPER): with the velocity prescribed on the rest of
                      the free-flow boundary the free-flow problem is singular;
   SD_ORDER_PM_FIRST  the porous medium takes the interface velocity as flux
                      data and returns the pressure of the cells below the
                      interface; the free flow takes that pressure into the
                      normal-stress balance and returns the velocity;
   SD_ORDER_AUTO      PM_FIRST.  (FF_FIRST's map multiplies the error of the
                      free-flow solve by the half-cell Darcy transmissibility
                      over h, 2K/(mu h), about 900 on the log-normal workload
                      at n = 24: the subdomain tolerance then limits how far
                      the coupling converges; PM_FIRST has no such factor:
                      its linearised map contracts, norm below 0.1 on the
                      pressure-driven problem at 24^2 and 32^2, against 600-850
                      for FF_FIRST.) */
#define SD_ORDER_AUTO 0
#define SD_ORDER_PM_FIRST 1
#define SD_ORDER_FF_FIRST 2

typedef struct sd_handle sd_handle;
typedef struct sd_server sd_server;

typedef struct {
  int32_t nx, ny; /* cells per subdomain side; square subdomains: nx == ny == n,
                     n = m * 2^k with m <= 16 so that multigrid reaches a small grid */
} sd_grid;

typedef struct {
  int32_t restart;     /* FGMRES restart length m, 1..30 (default 30) */
  double rtol;         /* stop when ||b - A x||_2 <= rtol ||b||_2 (default 1e-10) */
  int32_t max_iters;   /* FGMRES iterations allowed per time step (default 600) */
  int32_t precision;   /* SD_FP64 | SD_MIXED (default SD_MIXED) */
  int32_t precond;     /* SD_TRI_SCHUR | SD_PV_BJ_I | SD_PV_BGS_I (default SD_TRI_SCHUR) */
  int32_t bc;          /* SD_BC_MMS (default) | SD_BC_MMS_TRACTION | SD_BC_PAPER */
  int32_t cheb_degree; /* Chebyshev smoothing steps before and after each coarse
                          correction, 1..8 (default 3; on the log-normal workload 4
                          steps measured within 2 % of 3 and 2 steps 7-12 % slower) */
  int32_t cheb_degree_coarse; /* the same below the finest level (0: cheb_degree) */
  int32_t schur_degree;       /* the same in the pressure-Laplacian block (0: as above;
                                 default 1, one damped-Jacobi step) */
  int32_t coarsest;    /* coarsen while the grid has more than this many cells per
                          side (default 16: the coarsest grid, at most 16 x 16 cells,
                          is solved with its dense FP64 inverse spread over all SMs,
                          which measured 6.6 % faster per step than coarsening to 4 at
                          1024^2, 11.7 % at 2048^2 and 19 % at 256^2) */
  double schur_gamma;  /* gamma of S^ (default 0.5) */
  double cheb_ratio;   /* Chebyshev interval [lmax/ratio, 1.1 lmax] (default 8) */
  int32_t schur_mass;  /* SD_TRI_SCHUR: add the mass-dominated part (1/dt) L_p^-1 of
                          the Schur complement, L_p = B^T B / h^2 (default 1) */
  int32_t fuse_coarse; /* with coarsest < 16: run all levels with <= 16 cells per side
                          in one single-CTA kernel (default 1) */
  int32_t orth;        /* 0: classical Gram-Schmidt twice (CGS2); 1 (default): the second
                          pass only when ||w'|| < reorth_eta ||w|| (DGKS test, decided
                          on the device) */
  double reorth_eta;   /* default 1e-3: a second pass only after severe cancellation.
                          (Measured: with FGMRES cycles of 5-7 iterations the final
                          true residuals and iteration counts equal CGS2's, and the
                          step is 7-9 % faster; the true residual recomputed at every
                          restart still decides convergence.  1/sqrt(2), the classical
                          choice, took the second pass in 5 of 6 iterations.) */
  int32_t extrapolate; /* initial guess of step n+1: 3 x^n - 3 x^{n-1} + x^{n-2} (2,
                          default; quadratic in time), 4 x^n - 6 x^{n-1} + 4 x^{n-2} -
                          x^{n-3} (3, cubic), 2 x^n - x^{n-1} (1) or x^n (0), over solved
                          time levels only (the initial condition need not lie on the
                          discrete trajectory): x^1 as the guess of step 2, linear at
                          step 3, quadratic from step 4.  The stopping test is
                          unchanged.  Measured on the log-normal workload, steps 20-40:
                          quadratic 2-3 FGMRES iterations against linear 5 at 1024^2
                          (1.45 against 3.35 ms/step), 2-3 against 5 at 2048^2 and 3
                          against 6 at 256^2; cubic 3-4 at 1024^2 and 2048^2 (its larger
                          coefficients amplify the solves' own error), 2-3 at 256^2.  On
                          the pressure-driven problem: linear 16-19, quadratic 14-17,
                          cubic 12-16 (9.7 against 11.1 ms/step at 1024^2). */
  int32_t graph;       /* 1 (default): replay each Arnoldi step from a captured CUDA
                          graph, the host checking convergence after each; 2: a whole
                          FGMRES solve as one graph whose restart loop (WHILE node) and
                          Arnoldi steps (IF nodes) are decided on the device, one host
                          wait per solve; same iterates bit for bit, measured within
                          +-2 % of 1 (1024^2: +0.5 %, 128^2: -2.5 %); 0: direct launches.
                          Ignored on the legacy default stream and while profiling. */
  int32_t pdl;         /* programmatic dependent launch between consecutive kernels
                          of sd_step / sd_solve (default 1) */
  int32_t tile;        /* FP32 V-cycles: 1, all Chebyshev steps of one smoothing in one
                          shared-memory-tiled kernel, prolongation folded in; 2 (default),
                          the same, with the Darcy and pressure-Laplacian blocks of levels
                          of at least 1024 cells per side in register-column tiles (each
                          lane holds a column of the tile, lateral neighbours by warp
                          shuffles; measured 18 % and 15 % faster per launch at 1024^2);
                          0, one launch per Chebyshev step.  All three give the same bits. */
  int32_t tile_rows;   /* output rows of one smoothing tile, 4, 8 or 16; 0 (default):
                          4 on levels up to 256 cells per side, 8 up to 1024, 16 above;
                          tiles are 32 faces or cells wide.  Register-column tiles: 8 rows
                          for 8 or 16, else 4 */
  int32_t darcy_coupled; /* SD_TRI_SCHUR: 1 (default) keeps C'_1, the Darcy block follows
                          the velocity; 0 drops it and overlaps the Darcy V-cycle with
                          the Stokes part on a second stream; 2 solves the Darcy block
                          first (B'_1 kept), concurrently with the pressure block */
  int32_t coupling;    /* SD_MONOLITHIC (default) | SD_PARTITIONED */
  int32_t coupling_max;     /* SD_PARTITIONED: coupling iterations per step (default 100) */
  int32_t coupling_columns; /* SD_PARTITIONED: IQN-ILS difference columns kept, 1..30
                               (default 30; the oldest is dropped) */
  double coupling_eps;      /* SD_PARTITIONED: relative change of the exchanged pressure and
                               velocity that ends the iteration (default 1e-9) */
  double coupling_omega;    /* SD_PARTITIONED: relaxation of the first iteration of a step
                               (default 0.1) */
  int32_t coupling_order;   /* SD_PARTITIONED: SD_ORDER_AUTO (default) | SD_ORDER_PM_FIRST |
                               SD_ORDER_FF_FIRST */
  double coupling_rtol;     /* SD_PARTITIONED: relative tolerance of each subdomain solve;
                               0 (default): min(rtol, max(1e-3 coupling_eps, 1e-12)),
                               1e-12 being near the FP64 floor of these solves.  The coupling
                               test can only see changes above the subdomain solves' own
                               error: with solves to rtol = 1e-10 and coupling_eps = 1e-9 on
                               1024^2 lognormal K, 26 of 60 steps ran into coupling_max
                               (interface updates below the solves' tolerance returned no
                               change), with 1e-12 every step took 5-6 iterations.  A
                               subdomain solve whose restart cycle does not halve its true
                               residual has reached its rounding floor and stops there,
                               converged if the residual meets rtol.  The iteration also
                               stops when no subdomain solve moved its state. */
  double bc_dp;        /* SD_BC_PAPER: amplitude of the inflow pressure (default 1) */
  double bc_tend;      /* SD_BC_PAPER: rise time T of the inflow pressure (default 0:
                          25 time steps) */
  void *stream;        /* cudaStream_t to run on; NULL: the handle creates one */
  int32_t geometry;    /* SD_GEO_SQUARE (default) | SD_GEO_CHANNEL */
  int32_t darcy_schur; /* SD_MONOLITHIC: 1 (default) smooths the preconditioner's Darcy
                          block D' with the local Schur correction of the interface
                          velocity: eliminating v_Gamma from the cells below Gamma
                          (their C'_1 = h couples to v_Gamma, whose row couples back
                          through B'_1 = -h) adds h^2 / d to their diagonal, d the
                          diagonal of the v_Gamma row (Eq. (5)); 0: D' as it stands.
                          The operator is unchanged.  Measured over the first 8 steps
                          of the pressure-driven problem at the paper's own parameters
                          (Sec. 5: K = 1e-6, dt = 2e5, quasi-steady), FGMRES iterations
                          per step: 1024^2 119-162 -> 25-33 (107 -> 24 ms/step), 256^2
                          69-88 -> 19-23, channel 256^2 113-140 -> 21-25; on the
                          log-normal workload and the pressure-driven problem at
                          dt = 0.05 the counts stay the same. */
} sd_options;

typedef struct {
  int32_t iters;    /* FGMRES iterations of this step */
  int32_t restarts; /* restart cycles of this step */
  int32_t status;   /* SD_OK | SD_E_NOCONV | SD_E_NUMERIC */
  double relres;    /* final true ||b - A x||_2 / ||b||_2 (FP64, recomputed) */
  double ms;        /* device time of the step (CUDA events) */
  int32_t reorths;  /* Arnoldi steps that took the second Gram-Schmidt pass */
  int32_t coupling_iters; /* SD_PARTITIONED: subdomain-solve pairs of this step (0 otherwise);
                             iters then counts the FGMRES iterations of all subdomain solves
                             and relres is the monolithic residual of the coupled state */
  double relres_v;   /* the same residual restricted to the velocity rows [u | v], */
  double relres_pff; /*   the continuity rows p_ff and the Darcy rows p_pm, each over ||b||_2 */
  double relres_pm;  /*   (-1 when a cycle ended on NaN/Inf) */
} sd_step_info;

/* Fill *opt with the defaults above. */
void sd_options_default(sd_options *opt);

/* 4 n^2 + 2 n: unknowns of one instance (Table 1). */
int64_t sd_dof_count(int32_t n);

/* Unknowns of one instance of the given geometry (SD_GEO_SQUARE: 4 n^2 + 2 n,
   SD_GEO_CHANNEL: 10 n^2 + 4 n); -1 for an unknown geometry. */
int64_t sd_dof_count_geometry(int32_t n, int32_t geometry);

/* Device bytes sd_create() will allocate for this grid and options. */
int64_t sd_memory_estimate(const sd_grid *grid, const sd_options *opt);

/* Create one instance of the coupled problem (Sec. 2) and its solver.
 *   mu        dynamic viscosity (> 0), rho = 1;
 *   K         n*n permeabilities of the pm cells (> 0, finite), index j*n+i,
 *             host or device, copied before return;
 *   alpha_bj  Beavers-Joseph coefficient of Eq. (6) (> 0);
 *   dt        implicit-Euler step (> 0);
 *   opt       NULL for defaults.
 * Builds the multigrid hierarchy, coarsest-grid inverses and Chebyshev
 * bounds, and sets the state to the manufactured solution at t = 0 (to rest
 * for SD_BC_PAPER).
 * Errors: SD_E_INVAL, SD_E_NOMEM, SD_E_CUDA. */
int sd_create(const sd_grid *grid, double mu, const double *K, double alpha_bj, double dt, const sd_options *opt,
              sd_handle **out);

/* Advance nsteps implicit-Euler steps (Sec. 2): right-hand side from the
 * previous velocities, then FGMRES to rtol, warm-started from the
 * extrapolation in time of the previous solutions (sd_options.extrapolate).
 * info: NULL or nsteps entries.  Returns the first non-OK step status; a
 * step ending in SD_E_NOCONV or SD_E_NUMERIC still advances the state and
 * the remaining steps run.  SD_E_CUDA or SD_E_NOMEM returns at once: the
 * step count of sd_get_state says how many steps (and info entries) were
 * completed. */
int sd_step(sd_handle *h, int32_t nsteps, sd_step_info *info);

/* Copy the current fields out (any of the four may be NULL). */
int sd_get_fields(sd_handle *h, double *u, double *v, double *p_ff, double *p_pm);

/* Read / replace the whole state (checkpoint / resume): time, step count,
 * whole-system vector x^n and the previous time level x^{n-1} used by the
 * extrapolated initial guess (any output may be NULL; a NULL xprev in
 * sd_set_state clears the history, so the next step starts from x^n).
 * sd_set_state takes x (and xprev) as solved time levels.  With extrapolate 1
 * (or 0), resuming from a saved (t, step, x, xprev) reproduces the
 * uninterrupted run bit for bit; with extrapolate 2 the level before,
 * x^{n-2}, is also needed (sd_get_history / sd_set_history), else the first
 * resumed step extrapolates linearly (same tolerance, other bits).
 * With extrapolate 3 the first resumed step is quadratic (x^{n-3} is not
 * carried), so that run is reproduced to the tolerance, not bitwise.
 * A step's first residual is formed from the operator applied to these
 * levels, which sd_set_state and sd_set_history recompute (one operator
 * application per level given); a step whose first residual already met
 * the tolerance keeps that residual's extrapolated operator value instead,
 * so a run resumed right after such a step agrees to rounding only. */
int sd_get_state(sd_handle *h, double *t, int64_t *step, double *x, double *xprev);
int sd_set_state(sd_handle *h, double t, int64_t step, const double *x, const double *xprev);

/* x^{n-2} of the quadratic extrapolation (extrapolate 2), dense layout as x.
 * sd_get_history returns SD_E_STATE when the handle does not hold it (fewer
 * than three solved time levels, extrapolate < 2, or after sd_set_state
 * without sd_set_history); sd_set_history, called after sd_set_state with an
 * xprev, installs it (SD_E_STATE without that xprev or with extrapolate < 2). */
int sd_get_history(sd_handle *h, double *xprev2);
int sd_set_history(sd_handle *h, const double *xprev2);

/* y = A x with A the matrix of Eq. (9) (whole-system layout). */
int sd_apply(sd_handle *h, const double *x, double *y);

/* Right-hand side b of the implicit-Euler step to time t from the previous
 * state xprev (Sec. 2). */
int sd_rhs(sd_handle *h, const double *xprev, double t, double *b);

/* Solve A x = b by preconditioned FGMRES; x holds the initial guess on entry
 * and the solution on return.  info may be NULL. */
int sd_solve(sd_handle *h, const double *b, double *x, sd_step_info *info);

/* Wait for all work of the handle. */
int sd_sync(sd_handle *h);

/* Release the handle and its device memory. */
void sd_destroy(sd_handle *h);

/* Advance count independent instances (many instances of uneven grid sizes,
 * permeability fields and alpha_BJ; the batched workload has no counterpart
 * in the paper, whose solver runs one instance).  nsteps[k] steps for hs[k];
 * infos[k] NULL or nsteps[k] entries (ms: the step time of hs[k]'s group).
 *
 * Handles with the same grid size, mu, dt and options (the stream aside) and
 * the same nsteps form lockstep groups of at most about 2M DoF (larger grids
 * run one per stream, where a single grid already fills the GPU): every kernel launch of a group
 * serves all its instances (one instance per blockIdx.z, each instance's
 * buffers addressed from its own allocation), the Arnoldi steps of the
 * group are captured as one CUDA graph per basis index, and an instance
 * that has converged sits idle while the others iterate.  Groups and
 * single instances run concurrently, each on its own stream, from up to
 * max_threads host threads (0 = one per group).  Each instance does exactly
 * the arithmetic of its single-instance sd_step, so its result is bitwise
 * identical to running it alone.  Returns the first non-OK status;
 * SD_E_INVAL, before any work, for a NULL handle, a negative nsteps or a
 * handle listed twice.
 * sd_solve_batch_ex with flags = 0 runs every instance on its own stream
 * and host thread instead (no lockstep groups).  With SD_BATCH_GRAPH (and
 * SD_BATCH_LOCKSTEP) the solves of a time step of ALL groups, whatever their
 * grid sizes, run as one CUDA graph launched once per step: each group is a
 * branch of the graph whose restart loop (WHILE node) and Arnoldi steps (IF
 * nodes) are decided on the device, per instance, with the decisions of the
 * host-driven groups on the same values, so no host round trip happens
 * inside a solve and every result stays bitwise that of the run alone; the
 * right-hand sides are launched per group before it.  Every handle then has
 * to be able to join a group (SD_MONOLITHIC coupling, no sd_profile); the
 * graph is built again whenever the set of groups that still step changes,
 * and the handles' graph option does not apply. */
#define SD_BATCH_LOCKSTEP 1
#define SD_BATCH_GRAPH 2
int sd_solve_batch(sd_handle *const *hs, int32_t count, const int32_t *nsteps, sd_step_info *const *infos,
                   int32_t max_threads);
int sd_solve_batch_ex(sd_handle *const *hs, int32_t count, const int32_t *nsteps, sd_step_info *const *infos,
                      int32_t max_threads, int32_t flags);

/* Continuous-batching server: requests are admitted in arrival order as
 * running slots (max_running) and HBM budget free up, and run concurrently,
 * each on a worker thread and stream of its own (sd_server_create); each run
 * keeps its state on the device for all its steps.  sd_server_create_ex with
 * SD_SERVER_LOCKSTEP serves the runs of grids below 1M DoF by size class
 * (same grid, mu, dt) instead: every tick, each running request of a class
 * advances one time step in lockstep groups that share every launch (as
 * sd_solve_batch); requests join the class at the next tick after admission
 * and leave when their steps are done.  (Measured on the Poisson serving
 * workload it is slower: a class's graphs are recaptured whenever its
 * membership changes, and every tick waits for the slowest member, newly
 * joined runs needing twice the iterations of warm ones.)  Either way a
 * result is bitwise the same as the run alone.
 * opt NULL: defaults, except the multigrid depth, chosen per request from its
 * step count: runs under 40 steps coarsen to 4 x 4 cells (coarsest = 4),
 * longer ones stop at 16 x 16 (the default).  Building the dense inverse of
 * the 16 x 16 grid costs about 10 ms and some 1,600 dependent launches per
 * request, which queue behind the other runs' work, and saves 0.2-0.3 ms
 * per step.  Lockstep size classes are then also split by depth.
 * Memory: each run reserves sd_memory_estimate() of its own options (its
 * depth included) plus 4 MiB for setup temporaries and stream resources;
 * sd_submit returns SD_E_NOMEM for a request whose reservation exceeds the
 * whole budget, so every accepted request fits an idle server. */
#define SD_SERVER_LOCKSTEP 1
typedef struct {
  sd_grid grid;
  double mu, alpha_bj, dt;
  const double *K;   /* host, n*n, copied by sd_submit */
  int32_t nsteps;
  int32_t keep_fields; /* 1: the result keeps the final whole-system vector */
} sd_request;

typedef struct {
  int32_t status;      /* SD_OK or the first failing step's status */
  int32_t steps_done;
  int32_t total_iters;
  double max_relres;
  double queue_ms;     /* submit -> start */
  double run_ms;       /* start -> finished */
  double latency_ms;   /* submit -> finished */
  int64_t dof;
} sd_result;

int sd_server_create(int64_t hbm_budget_bytes, int32_t max_running, const sd_options *opt, sd_server **out);
int sd_server_create_ex(int64_t hbm_budget_bytes, int32_t max_running, const sd_options *opt, int32_t flags,
                        sd_server **out);
int sd_submit(sd_server *s, const sd_request *req, uint64_t *ticket);
/* SD_PENDING while queued or running; SD_OK (or the run's error) when done.
 * x: NULL or 4n^2+2n doubles (host) receiving the final state if keep_fields. */
int sd_poll(sd_server *s, uint64_t ticket, sd_result *out, double *x);
/* Block until every submitted request has finished. */
int sd_server_drain(sd_server *s);
void sd_server_destroy(sd_server *s);

/* Kernel timing for roofline reports.  While enabled, every launch of the
 * selected kernel class is bracketed by CUDA events on the handle's stream;
 * sd_profile_read() returns the summed device time, the number of launches,
 * and the summed algorithmic bytes (compulsory traffic: every input and
 * output array counted once) and floating-point operations of those
 * launches. */
#define SD_PROF_APPLY 0   /* whole-system FP64 operator y = A x (Eq. (9)) */
#define SD_PROF_CHEB_V 1  /* fine-level velocity-block Chebyshev step */
#define SD_PROF_MUPDATE 2 /* Gram-Schmidt update fused with the next dots */
#define SD_PROF_MDOT 3    /* Gram-Schmidt multi-dot */
int sd_profile(sd_handle *h, int32_t kernel, int32_t enable);
int sd_profile_read(sd_handle *h, double *total_ms, int64_t *launches, double *bytes, double *flops);

/* y = A x (the operator of sd_apply on a handle with bc = SD_BC_MMS, i.e.
 * Dirichlet free-flow sides; a handle with traction sides applies other side
 * rows, so the two agree only for SD_BC_MMS) for callers that cannot allocate
 * device memory: code running inside a framework that owns a fixed memory
 * pool, real-time loops where a cudaMalloc would stall the device, or
 * library code that may not create a handle (sd_create allocates).  This
 * function calls no cudaMalloc, cudaFree or other allocating routine; all
 * its working storage is one device array of SD_NOALLOC_MAX_N-sized
 * capacity (6 MiB) that every GPU loading this library holds until exit.
 * The paper has no counterpart: it is a deployment convenience.
 *   grid, mu, alpha_bj, dt  as in sd_create; n <= SD_NOALLOC_MAX_N, larger
 *                           grids return SD_E_INVAL;
 *   K, x, y                 CUDA device memory of the current device (host
 *                           pointers and memory of another device return
 *                           SD_E_INVAL); K (n*n, > 0, not checked here) and x
 *                           (4n^2+2n) in the layouts of sd_create and
 *                           sd_apply; y (4n^2+2n) receives A x;
 *   stream                  cudaStream_t (NULL: the default stream); the
 *                           work is queued on it and y is ready when the
 *                           stream reaches that point.
 * The first call on a device looks up the array's device address (once,
 * with that device current); make that first call before any stream
 * capture.  All calls share the one array: calls whose work can overlap on
 * the GPU (different streams without ordering) race and corrupt each other.
 * Errors: SD_E_INVAL; SD_E_CUDA when a launch fails, and also, without
 * running anything (the pending error is left in place), when a CUDA error
 * from earlier work is already pending on entry. */
#define SD_NOALLOC_MAX_N 256
int sd_apply_noalloc(const sd_grid *grid, double mu, const double *K, double alpha_bj, double dt, const double *x,
                     double *y, void *stream);

/* Autotuner: pick tile_rows, coarsest (V-cycle depth) and cheb_degree for
 * this grid size on the current device by timing.  Each candidate of the
 * grid {by level, 16, 8} rows (FP32 tiled smoothing only) x coarsest {4, 8, 16} x
 * cheb_degree {3, 2, 4} builds a fresh instance from (grid, mu, K,
 * alpha_bj, dt) with *base (NULL: defaults) and those three fields, runs 4
 * untimed and then `nsteps` timed implicit-Euler steps, and is scored by its
 * mean device time per step; candidates whose steps do not all converge are
 * dropped.  The tuned choice does not change what is solved: every step
 * still reaches base->rtol.
 *   K          host or device permeability as in sd_create;
 *   cache_path text file (NULL or "": no cache).  A line matching this device,
 *              n, precision, precond, darcy_coupled, restart, bc, coupling and rtol is
 *              returned without timing (the last such line whose options
 *              sd_create accepts); otherwise the winner is appended;
 *   best       receives *base with the three tuned fields;
 *   best_ms    (may be NULL) mean device ms per step of the winner.
 * Costs up to 27 instance setups plus 27 (nsteps + 4) steps on a cache miss
 * (9 of each with FP64 V-cycles or without tiling, fewer on grids too small
 * to coarsen to the deeper candidates).
 * Errors: SD_E_INVAL, SD_E_NOCONV (no candidate converged). */
int sd_autotune(const sd_grid *grid, double mu, const double *K, double alpha_bj, double dt, const sd_options *base,
                int32_t nsteps, const char *cache_path, sd_options *best, double *best_ms);

/* Kernel launches made by this library in this process so far (kernels replayed
 * from captured CUDA graphs included). */
int64_t sd_launch_count(void);

/* sizeof of the public structs, for bindings that check their layout:
 * 0 sd_grid, 1 sd_options, 2 sd_step_info, 3 sd_request, 4 sd_result; -1 otherwise. */
int64_t sd_struct_size(int32_t which);

const char *sd_strerror(int code);

#ifdef __cplusplus
}
#endif
#endif /* SD_H */
