/*
 * lesjet.h -- C ABI of the GB300 (sm_103a) implementation of the LES hot path
 * of "Computational Performance of a LES Solver for Supersonic Jet Flow
 * Applications" (arXiv 2301.00817): the residual of the filtered compressible
 * Navier-Stokes equations (System I energy) on a structured curvilinear grid,
 * fused into the paper's five-stage Runge-Kutta update.
 *
 * Conventions for every entry point:
 *  - Return value: LES_OK (0) or a negative LES_ERR_* code; les_last_error()
 *    gives a message.  No C++ exception crosses this boundary.
 *  - Memory: the library allocates no device memory.  The caller owns every
 *    device buffer (PyTorch tensors in the Python binding) and passes raw
 *    device pointers; one caller-owned workspace of les_workspace_bytes()
 *    holds the metrics, viscosity, stage states and scratch.  Every device
 *    pointer must be 16-byte aligned (LES_ERR_ALIGN otherwise).
 *  - Layout: structure of arrays, k (azimuthal, zeta) fastest, then j (radial,
 *    eta), then i (axial, xi): node n = (i*nj + j)*nk + k.  A field with C
 *    components is C contiguous arrays of N = ni*nj*nk values ([C][N]).
 *    Q is [5][N] FP64 holding the UNSCALED conserved variables
 *    rho, rho u, rho v, rho w, e (the paper's Q-hat is J^-1 Q).
 *  - Streams: work is queued on the given stream (NULL = legacy default
 *    stream).  Calls are asynchronous unless documented as synchronising.
 *  - Variables are dimensionless as in Sec. "Dimensionless Formulation":
 *    lengths by D, velocities by a_j, pressure by rho_j a_j^2, rho by rho_j.
 */
#ifndef LESJET_H
#define LESJET_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st *les_stream_t; /* same type as cudaStream_t */

enum {
  LES_OK = 0,
  LES_ERR_INVALID_ARG = -1, /* null pointer, bad enum or bad value */
  LES_ERR_SHAPE = -2,       /* grid too small or too large */
  LES_ERR_ALIGN = -3,       /* a device pointer is not 16-byte aligned */
  LES_ERR_CUDA = -4,        /* a CUDA runtime call failed */
  LES_ERR_NONFINITE = -5,   /* non-finite or non-positive rho/p/dt seen */
  LES_ERR_UNSUPPORTED = -6, /* option not available in this build */
  LES_ERR_STATE = -7        /* call order violated (e.g. no grid set) */
};

enum { LES_SGS_NONE = 0, LES_SGS_SMAGORINSKY = 1, LES_SGS_VREMAN = 2, LES_SGS_DYNAMIC = 3 };
/* LES_PREC_MIXED_COMPACT is the mixed form without the FP64 copy of the
 * metrics (80 bytes per point less): metrics are computed in FP64 and stored
 * once rounded to FP32, which the boundary conditions and the totals then
 * read; les_metrics() returns NULL.  It is the form for the largest grids. */
enum { LES_PREC_FP64 = 0, LES_PREC_MIXED = 1, LES_PREC_MIXED_COMPACT = 2 };
enum { LES_BC_FROZEN = 0, LES_BC_JET = 1, LES_BC_JET_CHAR = 2 };
enum { LES_DT_CFL = 0, LES_DT_FIXED = 1, LES_DT_LOCAL = 2 };
enum { LES_METRIC_CROSS = 0, LES_METRIC_CONSERVATIVE = 1 };

/* Flow and scheme parameters (Sec. "Large Eddy Simulation Filtering" to
 * Sec. "Boundary Conditions").  Defaults used by the jet workloads:
 * gamma 1.4, Pr 0.72, Pr_sgs 0.9, Mj 1.4, T_ref 288.15 K, k2 0.25,
 * k4 0.016, Cs 0.148, cfl 0.5, r_jet 0.5, theta_m 0.05, force_width 0.05,
 * St = {0.25, 0.5, 0.75, 1.0}. */
typedef struct les_params {
  double gamma;       /* ratio of specific heats */
  double Pr;          /* laminar Prandtl number */
  double Pr_sgs;      /* subgrid-scale Prandtl number */
  double Mj;          /* jet Mach number U_j / a_j (also U_j in a_j units) */
  double Re;          /* Reynolds number rho_j U_j D / mu_j; <= 0: inviscid */
  double T_ref;       /* Sutherland reference temperature, K */
  double k2, k4;      /* Turkel-Vatsa constants k^(2), k^(4) */
  double Cs;          /* Smagorinsky constant (Vreman uses 2.5 Cs^2) */
  double cfl;         /* CFL number of the global time step */
  double dt_fixed;    /* time step when dt_mode == LES_DT_FIXED */
  double r_jet;       /* jet radius of the inflow profile */
  double theta_m;     /* momentum thickness of the inflow shear layer */
  double force_width; /* radial width of the inflow forcing */
  double St[4];       /* forcing Strouhal numbers */
  double amp[16];     /* forcing amplitudes a_{m f}, index m*4 + f */
  int sgs_model;      /* LES_SGS_NONE, LES_SGS_SMAGORINSKY, LES_SGS_VREMAN,
                         or LES_SGS_DYNAMIC (dynamic Smagorinsky with the
                         Yoshizawa isotropic part and a dynamic Pr_sgs;
                         chosen at les_create; in the mixed forms the
                         procedure runs in FP32 with FP64 sums) */
  int periodic[3];    /* per direction xi, eta, zeta: 1 = periodic */
  int bc;             /* LES_BC_FROZEN (non-periodic faces never change),
                         LES_BC_JET (Dirichlet jet state over the whole
                         entrance plane) or LES_BC_JET_CHAR (Sec. "Entrance
                         Boundary": above r = r_jet the far-field Riemann
                         rule with the xi normal; in the jet area the jet
                         state if Mj >= 1, else the 1-D characteristic
                         relations: target u, v and w from the next plane,
                         T from the jet's total temperature, isentropic p).
                         Both jet modes need periodic = {0,0,1}; the adjoint
                         calls support LES_BC_FROZEN and LES_BC_JET. */
  int dt_mode;        /* LES_DT_CFL, LES_DT_FIXED or LES_DT_LOCAL (Eq.
                         localdt taken literally: node n advances with its
                         own CFL step cfl/(lambda_xi + lambda_eta +
                         lambda_zeta)(n) of Q^n, for steady problems; the
                         clock and les_diag.dt use the smallest of them).
                         LES_DT_LOCAL must be chosen at les_create (its
                         per-node steps live in the workspace); the adjoint
                         calls reject it. */
  int freeze_visc;    /* 1: mu_eff, kappa_eff from Q^n held for 5 stages */
  int precision;      /* LES_PREC_FP64, LES_PREC_MIXED or
                         LES_PREC_MIXED_COMPACT */
  int metric_form;    /* LES_METRIC_CROSS: the cross-product formulas of
                         Sec. "Transformation of Coordinates";
                         LES_METRIC_CONSERVATIVE: the same cofactors in the
                         Thomas-Lombard form d_t((p_s) q) - d_s((p_t) q),
                         whose central differences telescope, so a uniform
                         flow stays uniform on any grid.  Read by
                         les_set_grid. */
  int axis;           /* 1: a true centerline grid (Sec. "Centerline Boundary
                         Condition", Reading A27): ring j = 0 lies on the
                         axis r = 0, where J^-1 = 0.  Its nodes store the
                         J^-1-scaled metrics (finite cofactors) beside
                         J^-1 = 0, take the spectral radii of (i, 1, k) and,
                         as SGS viscosity, the azimuthal mean of ring 1's at
                         their plane; every interface metric is the
                         J^-1-weighted mean of its two nodes; the exit takes
                         ring 1's normal on the axis; the centerline rule sets
                         the axis state.  Needs periodic = {0, 0, 1} and a
                         static SGS model (not LES_SGS_DYNAMIC); the adjoint
                         calls reject it.  0: every node has J^-1 > 0. */
  int slab_ghost[2];  /* axial domain decomposition (Sec. "Communication":
                         axial partitions with two ghost layers): the number
                         of ghost planes at the low and the high xi end of
                         this context's grid, 0 at a physical face (the
                         entrance, the exit) and 2 at a cut between slabs.
                         A ghost plane belongs to the neighbouring slab: the
                         stages neither update it nor count it in the CFL
                         minimum or the totals, and the entrance (exit)
                         conditions apply only with slab_ghost[0] ([1]) = 0.
                         Stepping with ghost planes goes through the phase
                         calls below (les_step_begin ...), which let a driver
                         exchange the ghost planes and take the global time
                         step between the phases.  Needs periodic[0] = 0;
                         not with LES_SGS_DYNAMIC (its means are global) or
                         the adjoint calls. {0, 0}: an undivided grid. */
} les_params;

/* Diagnostics returned by the synchronising run calls. */
typedef struct les_diag {
  double t;          /* simulation time after the last step */
  double dt;         /* time step of the last step */
  double totals[5];  /* sum_n J^-1_n Q_c(n), fixed-order reduction */
  int status;        /* LES_OK or LES_ERR_NONFINITE */
  int steps;         /* steps taken by the call */
} les_diag;

typedef struct les_ctx les_ctx;

/* Create a context for an ni x nj x nk grid (each >= 5; N < 2^40, N < 2^31 in the mixed forms).  Host
 * memory only; *out is owned by the caller and released by les_destroy. */
int les_create(const les_params *p, int ni, int nj, int nk, les_ctx **out);
int les_destroy(les_ctx *ctx);
/* Synthetic annular jet grid (the stand-in for the paper's meshes, Table
 * tab:mesh): Cartesian coordinates of node (i, j, k) into xyz (device [3][N]
 * FP64, the layout les_set_grid reads):
 *   x_i = length (q^i - 1)/(q^(ni-1) - 1), q = ratio, or length i/(ni-1) for
 *         q = 1; ratio <= 0 selects 1.01 up to 288 planes and 1.01^(288/ni)
 *         beyond (the same geometric mapping, refined);
 *   r_j = r0 + (r1 - r0) g(s_j)/g(1), s_j = j/(nj-1),
 *         g(s) = s - (A/beta)[tanh(beta (s - s_c)) + tanh(beta s_c)], s_c the
 *         point the map sends to r_c (found by bisection; spacing is smallest
 *         there, (1 - A) times the mean);
 *   theta_k = 2 pi k/nk;  y = r cos theta, z = r sin theta.
 * Needs no context.  ni, nj, nk >= 2, N < 2^40, length > 0, 0 <= r0 < r_c <
 * r1, 0 <= A < 1, beta > 0; LES_ERR_SHAPE / LES_ERR_INVALID_ARG otherwise.
 * r0 = 0 writes a true centerline grid (ring j = 0 on the axis, J^-1 = 0
 * there), which les_set_grid does not support yet (see there).
 * Asynchronous. */
typedef struct les_jet_grid {
  double length;  /* axial extent (20 D) */
  double ratio;   /* geometric axial stretching (<= 0: the refinement rule) */
  double r0, r1;  /* radial extent (0.02 D, 10 D) */
  double r_c;     /* clustering radius (0.5 D) */
  double A, beta; /* clustering strength (0.9) and sharpness (8) */
} les_jet_grid;
int les_grid_jet(int ni, int nj, int nk, const les_jet_grid *grid, double *xyz,
                 les_stream_t stream);

/* Last error message of this context (never NULL; "" when none). */
const char *les_last_error(const les_ctx *ctx);
/* Replace the parameters (same grid and precision), e.g. new forcing.
 * dt_mode LES_DT_LOCAL and sgs_model LES_SGS_DYNAMIC are accepted only by a
 * context created with them (their data live in the workspace). */
int les_set_params(les_ctx *ctx, const les_params *p);

/* Bytes of the caller-owned device workspace this context needs: about
 * 416 B per point in FP64, 208 B mixed, 128 B compact mixed; plus one value
 * per point with LES_DT_LOCAL and, with LES_SGS_DYNAMIC, 408 B per point
 * more (FP64) or 236 B per point more (mixed). */
size_t les_workspace_bytes(const les_ctx *ctx);

/* Bind the workspace and compute the Jacobian and the nine metric terms on
 * the device (Sec. "Transformation of Coordinates"; the eta row is the
 * cofactor form, the printed eta row being garbled).  xyz: device [3][N]
 * FP64 Cartesian coordinates.  shift: host [3][3] coordinate jump over one
 * period of each periodic direction (shift[3*d + c]; zeros for the jet grid).
 * Derivatives are second-order central, one-sided second order at
 * non-periodic faces.  Every node needs J^-1 > 0, except on a grid with an
 * axis (r = 0 on ring j = 0, the paper's centerline singularity; params.axis
 * = 1), where the axis nodes have J^-1 = 0 exactly and store the J^-1-scaled
 * metrics.  The workspace must stay allocated while the context is used.
 * Asynchronous. */
int les_set_grid(les_ctx *ctx, const double *xyz, const double shift[9],
                 void *workspace, les_stream_t stream);

/* Device pointer to the FP64 metrics [10][N] inside the workspace:
 * xi_x xi_y xi_z eta_x eta_y eta_z zeta_x zeta_y zeta_z J^-1.  NULL before
 * les_set_grid and for LES_PREC_MIXED_COMPACT contexts. */
const double *les_metrics(const les_ctx *ctx);

/* Jet initial condition into Q (device [5][N]): rho = 1, p = 1/gamma,
 * u = Mj/2 [1 + tanh((r_jet - r)/(2 theta_m))], plus noise*Mj*N(0,1) on
 * u, v, w from Philox4x32-10 (counter = node, block; key = seed) and
 * Box-Muller.  xyz as in les_set_grid.  Asynchronous. */
int les_init_jet(les_ctx *ctx, const double *xyz, uint64_t seed,
                 double noise, double *Q, les_stream_t stream);

/* Effective viscosity/conductivity of state Q into MK (device [2][N] FP64):
 * Sutherland laminar part times Mj/Re plus the SGS model (Sec. "Subgrid
 * Scale Modeling").  With LES_SGS_DYNAMIC, MK is [3][N]: the third field is
 * the Yoshizawa isotropic SGS stress sigma_ll (Eq. yoshizawa).
 * Asynchronous. */
int les_mu_eff(les_ctx *ctx, const double *Q, double *MK, les_stream_t stream);

/* The dynamic Smagorinsky procedure (Sec. "Dynamic Smagorinsky Model",
 * Eqs. av_ci, av_cd, av_Pr_sgs) on state Q (device [5][N] FP64), into
 * out[9] (host): the J^-1-weighted interior means of the numerator and
 * denominator of C_ds, of C_I and of Pr_sgs/C_ds, then C_ds, C_I and
 * Pr_sgs as the stepping calls use them (C_ds, C_I clipped at 0; Pr_sgs
 * the configured value when the dynamic one is not positive).  Test filter:
 * (1/4, 1/2, 1/4) along each direction, width 2 Delta, identity along a
 * non-periodic direction at its faces.  Needs sgs_model LES_SGS_DYNAMIC at
 * les_create (FP64 form only: the workspace then holds 50 scratch fields
 * and a third viscosity field).  SYNCHRONISES the stream. */
int les_dynamic_coefficients(les_ctx *ctx, const double *Q, double out[9],
                             les_stream_t stream);

/* Residual RHS of Eq. spatial_discret for state Q into R (device [5][N]
 * FP64): interior nodes get sum_d (F_{+1/2} - F_{-1/2}) with F = centred
 * inviscid flux minus J^-1 times the Turkel-Vatsa dissipation minus the
 * viscous+SGS flux; boundary nodes of non-periodic directions get 0.  The
 * viscosity is evaluated from the same Q.  Computed in the context's
 * precision.  Asynchronous. */
int les_rhs(les_ctx *ctx, const double *Q, double *R, les_stream_t stream);

/* Global time step dt = cfl * min_n 1/(lambda_xi + lambda_eta + lambda_zeta)
 * of state Q (or dt_fixed).  SYNCHRONISES the stream; returns
 * LES_ERR_NONFINITE if rho, p or dt is not finite and positive. */
int les_time_step(les_ctx *ctx, const double *Q, double *dt_out,
                  les_stream_t stream);

/* Jet boundary conditions on Q at time t (entrance, far field, inner ring,
 * then exit).  Requires bc == LES_BC_JET or LES_BC_JET_CHAR.  Asynchronous. */
int les_apply_bc(les_ctx *ctx, double *Q, double t, les_stream_t stream);

/* Set the device-resident simulation time used by the stepping calls. */
int les_set_time(les_ctx *ctx, double t, les_stream_t stream);

/* One time step of Eq. localdt on Q in place: viscosity from Q^n, dt, five
 * stages Q^(l) = Q^(0) - alpha_l dt J RHS(Q^(l-1)) with alpha = 1/4, 1/6,
 * 3/8, 1/2, 1 (boundary nodes keep Q^(0)), then the boundary conditions at
 * t + dt.  t and dt stay on the device.  Asynchronous. */
int les_rk_step(les_ctx *ctx, double *Q, les_stream_t stream);

/* n time steps on Q in place, then SYNCHRONISES and fills *diag (may be
 * NULL).  Returns LES_ERR_NONFINITE if any step saw a non-finite state.
 * In the mixed forms the context's first step runs as plain kernel launches
 * and is then captured as a CUDA graph (on a stream the context creates and
 * les_destroy releases); later steps replay the graph on `stream`, unless
 * the event profiler is on.  les_set_params, les_set_grid and les_profile
 * drop the graph.  The same holds for les_run_host. */
int les_run_n_steps(les_ctx *ctx, int n, double *Q, les_diag *diag,
                    les_stream_t stream);

/* Same as les_run_n_steps for a HOST state Q_host (pinned or pageable host
 * [5][N]); the result is written back into Q_host.  In the mixed forms,
 * when Q_host is pinned memory mapped into the device's address space (as
 * cudaHostAlloc/torch pin_memory gives), the split and join kernels read
 * and write it directly over the host link and Q_dev is not touched;
 * otherwise (and always in FP64) Q_host is copied into the device buffer
 * Q_dev and back.  SYNCHRONISES. */
int les_run_host(les_ctx *ctx, int n, double *Q_host, double *Q_dev,
                 les_diag *diag, les_stream_t stream);

/* sum_n J^-1_n Q_c(n) for c = 0..4 (fixed-order, deterministic).
 * SYNCHRONISES. */
int les_totals(les_ctx *ctx, const double *Q, double out[5],
               les_stream_t stream);

/* Number of kernel launches the library issued on this context so far. */
uint64_t les_launch_count(const les_ctx *ctx);

/* Measurement support (no counterpart in the paper, which reports whole-
 * iteration CPU time only).  les_profile(ctx, 1) clears and enables an event
 * profiler: every later launch group records a CUDA event pair on its own
 * stream.  les_profile_read SYNCHRONISES the stream and returns, per kernel
 * class k < 16, the summed device milliseconds ms[k] and launch groups
 * counts[k]; les_profile_name(k) names class k ("" past the last). */
int les_profile(les_ctx *ctx, int enable);

/* FMA throughput of the current device's CUDA cores, the roof of the
 * ALU-bound kernels (the paper has no counterpart): every thread advances
 * 16 independent FMA chains on a grid of 8 CTAs per SM, timed with CUDA
 * events on `stream`.  precision LES_PREC_FP64 measures FP64, the mixed
 * values FP32.  *tflops = 2 x FMAs / time / 1e12.  Needs no context.
 * SYNCHRONISES; LES_ERR_INVALID_ARG or LES_ERR_CUDA on failure. */
int les_measure_fma_peak(int precision, double *tflops, les_stream_t stream);
int les_profile_read(les_ctx *ctx, double ms[16], uint64_t counts[16],
                     les_stream_t stream);
const char *les_profile_name(int kind);

/* ------------------------------------------------------------------------
 * Discrete adjoint of the FP64 time step (the paper has no adjoint; this is
 * the gradient form of the same scheme).  Requirements: precision FP64,
 * dt_mode LES_DT_FIXED (the step does not depend on the CFL minimum),
 * sgs_model LES_SGS_NONE, freeze_visc 1; LES_ERR_UNSUPPORTED otherwise.
 * Scratch lives in a caller-owned adjoint workspace of
 * les_adjoint_workspace_bytes(ctx, nsteps, ckpt_every) bytes: about
 * (300 + 5 ceil(nsteps/ckpt_every) + 72 ckpt_every) N doubles for a window
 * (checkpoints, plus every stage state and stage-input node quantity of one
 * segment), 300 N for nsteps = 0 (residual and single-step calls only); 135
 * N of it hold each interface's cotangent record, which a per-node gather
 * sums in a fixed order, so every adjoint result is bitwise reproducible
 * (no atomics).  At non-smooth
 * points the derivative follows the forward branch: |x| has slope -1 for
 * x < 0 and +1 otherwise; a max passes to the operand it selected.
 * ------------------------------------------------------------------------ */
size_t les_adjoint_workspace_bytes(const les_ctx *ctx, int nsteps, int ckpt_every);

/* Tangent of the residual (Eq. spatial_discret): R = RHS(Q, MK) and
 * dR = dRHS/dQ dQ + dRHS/dMK dMK at MK = mu_eff/kappa_eff of Q.  dMK may be
 * NULL (zero); R may be NULL.  Device [5][N] / [2][N] FP64.  Asynchronous. */
int les_rhs_jvp(les_ctx *ctx, const double *Q, const double *dQ,
                const double *dMK, double *R, double *dR, void *adj_ws,
                les_stream_t stream);

/* Adjoint of the residual: lamQ = (dRHS/dQ)^T lamR and lamMK =
 * (dRHS/dMK)^T lamR at MK of Q.  Entries of lamR on boundary nodes (where
 * the residual is defined as 0) are ignored.  Asynchronous. */
int les_rhs_vjp(les_ctx *ctx, const double *Q, const double *lamR,
                double *lamQ, double *lamMK, void *adj_ws, les_stream_t stream);

/* Adjoint of one time step Q^{n+1} = BC(RK5(Q^n)) taken at time t_n:
 * lam_out = (dQ^{n+1}/dQ^n)^T lam_next (lam_out may alias lam_next) and
 * grad[16] += (dQ^{n+1}/da)^T lam_next for the 16 inflow forcing amplitudes
 * a_{mf}.  Recomputes the five stage states from Q^n.  SYNCHRONISES. */
int les_adjoint_step(les_ctx *ctx, const double *Qn, double t_n,
                     const double *lam_next, double *lam_out, double grad[16],
                     void *adj_ws, les_stream_t stream);

/* Forward window of nsteps steps from Q_start at t0 and its adjoint: returns
 * J = sum_{n=1..nsteps} dt sum_{i,k} (p(i, j_surface, k) - 1/gamma)^2 dA with
 * dA = J^-1 |grad eta| (the eta-face area) and grad[16] = dJ/da.  Stores a
 * checkpoint every ckpt_every steps; the reverse sweep recomputes one
 * segment at a time, keeping its stage states, then runs its adjoint steps.
 * Q_start is not modified.  SYNCHRONISES. */
int les_adjoint_window(les_ctx *ctx, const double *Q_start, double t0,
                       int nsteps, int ckpt_every, int j_surface,
                       void *adj_ws, double *J_out, double grad[16],
                       les_stream_t stream);

/* One term of the window functional of les_adjoint_window for state Q
 * (device [5][N] FP64): J_out = w sum_{i,k} (p(i, j_surface, k) - 1/gamma)^2
 * J^-1 |grad eta| at (i, j_surface, k).  Works in every precision (the FP64
 * metrics, or the FP32 copy of a mixed context), so the functional can be
 * accumulated along a mixed-precision forward run and compared with the FP64
 * window (the paper has no counterpart).  SYNCHRONISES. */
int les_surface_functional(les_ctx *ctx, const double *Q, int j_surface, double w,
                           double *J_out, les_stream_t stream);

/* One Runge-Kutta step in phases (Table tab:JAZzY), for a driver of axial
 * slabs (slab_ghost) that exchanges ghost planes between the phases; on an
 * undivided grid the phases in order do exactly what les_rk_step does.  Per
 * step:
 *   les_step_begin   viscosity and the CFL step of this slab's own planes
 *                    from the state Q^n; returns that step in dt_local
 *                    (SYNCHRONISES; LES_ERR_NONFINITE as les_time_step);
 *   les_step_set_dt  the step all slabs take (the minimum of their dt_local
 *                    across slabs); advances the clock to t^{n+1};
 *   les_step_stage   stage l = 1..5 (Eq. localdt): Q^(l) = Q^(0) -
 *                    alpha_l dt J RHS(Q^(l-1)); exchange the ghost planes of
 *                    the state after it before the next phase;
 *   les_step_end     the boundary conditions at t^{n+1}; exchange again.
 * Q: device [5][N] FP64, the caller's state.  The mixed forms keep the state
 * as a float pair in the workspace between phases: les_state_load splits Q
 * into it before the first step, les_state_store joins it back into Q (both
 * no-ops in FP64).  les_state_buffer names the arrays that hold the state
 * after stage l (l = 1..4: the stage buffer, FP64 or float, *a; l = 0 or 5,
 * the state after stage 5 or after the boundary conditions: *a = NULL for
 * FP64, meaning the caller's Q, else the float pair hi *a and lo *b); each
 * is [5][N] with field stride N, elem_bytes 8 or 4; ghost plane i of field
 * f is the nj*nk values from (f N + i nj nk).  Asynchronous except
 * les_step_begin. */
int les_step_begin(les_ctx *ctx, double *Q, double *dt_local, les_stream_t stream);
int les_step_set_dt(les_ctx *ctx, double dt, les_stream_t stream);
int les_step_stage(les_ctx *ctx, int l, double *Q, les_stream_t stream);
int les_step_end(les_ctx *ctx, double *Q, les_stream_t stream);
int les_state_load(les_ctx *ctx, const double *Q, les_stream_t stream);
int les_state_store(les_ctx *ctx, double *Q, les_stream_t stream);
int les_state_buffer(les_ctx *ctx, int l, void **a, void **b, int *elem_bytes);

/* Ghost-plane exchange between two slab contexts of one process (the same
 * or peer devices): copies src's two own planes next to the cut into dst's
 * ghost planes, for the state after stage l (as in les_state_buffer; Qdst,
 * Qsrc are the callers' states, used for l = 0 or 5 in FP64).  side 0: dst
 * is the slab above src along xi (src planes [ni_src-4, ni_src-2) into dst
 * planes [0, 2)); side 1: dst is the slab below (src planes [2, 4) into dst
 * planes [ni_dst-2, ni_dst)).  One cudaMemcpy2DAsync per array (5 fields of
 * 2 planes, field strides N_src, N_dst) on stream.  Both contexts need the
 * same nj, nk and precision and the matching ghost planes.  Asynchronous. */
int les_halo_copy(les_ctx *dst, double *Qdst, les_ctx *src, const double *Qsrc, int l, int side,
                  les_stream_t stream);

/* Global time step of state Q, like les_time_step, for callers that cannot
 * allocate device memory (the paper has no counterpart): for example a
 * monitoring or steering hook that runs between solver steps in an
 * application that has committed all device memory to its own fixed pool, or
 * a plain-C tool that is handed only raw device pointers.  It needs no
 * workspace and no les_set_grid: only a context from les_create (host memory)
 * and the caller's Q (device [5][N] FP64) and FP64 metrics M (device [10][N],
 * e.g. les_metrics() of another context).  It allocates nothing: its scratch
 * is one static device array inside the library, sized for ni <=
 * LES_STATIC_MAX_NI axial planes (256 KiB, held on every GPU that loads the
 * library until the process exits); larger grids are rejected with
 * LES_ERR_SHAPE.  The array's device address differs between CUDA contexts
 * (a second context on a device, or the primary context re-created after
 * cudaDeviceReset), so the first call in each context looks it up with that
 * context current; make that first call before any stream capture.  All
 * calls share the array, so calls that overlap on the GPU race.
 * Always FP64.  SYNCHRONISES the stream; LES_ERR_NONFINITE as les_time_step. */
#define LES_STATIC_MAX_NI 16384
int les_time_step_static(les_ctx *ctx, const double *Q, const double *M,
                         double *dt_out, les_stream_t stream);

#ifdef __cplusplus
}
#endif

#endif /* LESJET_H */
