/*
 * les_oracle.h -- plain, slow FP64 CPU oracle of the LES residual and RK5 step
 * of "Computational Performance of a LES Solver for Supersonic Jet Flow
 * Applications" (arXiv 2301.00817).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test-suite, the smoke check and the
 * benchmark's CPU-baseline leg may call this library.  It shares no code,
 * header, table or helper with the CUDA library; the two are independent
 * restatements of the paper.
 *
 * Storage: structure of arrays, k (azimuthal, zeta) fastest, then j (radial,
 * eta), then i (axial, xi): node n = (i*nj + j)*nk + k.  A field with C
 * components is stored as [C][N].
 *   Q  [5][N]  unscaled conserved variables rho, rho u, rho v, rho w, e
 *   M  [10][N] xi_x xi_y xi_z eta_x eta_y eta_z zeta_x zeta_y zeta_z J^-1
 *   MK [2][N]  mu_eff, kappa_eff (dimensionless, viscous factor included)
 */
#ifndef LES_ORACLE_H
#define LES_ORACLE_H

#include <stddef.h>
#include <stdint.h>

typedef struct {
  double gamma;      /* ratio of specific heats */
  double Pr;         /* laminar Prandtl number (0.72) */
  double Pr_sgs;     /* SGS Prandtl number (0.9) */
  double Mj;         /* jet Mach number = U_j / a_j (U_j in a_j units) */
  double Re;         /* Reynolds number; Re <= 0 means inviscid */
  double T_ref;      /* Sutherland reference temperature in K */
  double k2, k4;     /* Turkel-Vatsa dissipation constants */
  double Cs;         /* Smagorinsky constant */
  double cfl;        /* CFL number for the global time step */
  double dt_fixed;   /* time step when dt_mode == 1 */
  double r_jet;      /* jet radius of the inflow profile (0.5 D) */
  double theta_m;    /* shear-layer momentum thickness (0.05 D) */
  double force_width;/* radial width of the inflow forcing (0.05 D) */
  double St[4];      /* forcing Strouhal numbers */
  double amp[16];    /* forcing amplitudes a_{m f}, index m*4 + f */
  int sgs_model;     /* 0 none, 1 Smagorinsky, 2 Vreman, 3 dynamic
                        Smagorinsky (MK then holds a third field,
                        sigma_ll) */
  int periodic[3];   /* per direction xi, eta, zeta */
  int bc;            /* 0 non-periodic boundary nodes frozen, 1 jet BCs,
                        2 jet BCs with the characteristic entrance */
  int dt_mode;       /* 0 CFL-limited global step, 1 fixed, 2 local steps */
  int freeze_visc;   /* 1: mu_eff/kappa_eff from Q^n held over 5 stages */
  int axis;          /* 1: a true centerline grid (r from 0; Reading A27) */
} orc_params;

/* Grid metrics (Sec. "Transformation of Coordinates"); xyz is [3][N]. */
void orc_metrics(int ni, int nj, int nk, const int periodic[3],
                 const double shift[9], const double *xyz, double *M);
void orc_metrics_conservative(int ni, int nj, int nk, const int periodic[3],
                              const double shift[9], const double *xyz,
                              double *M);

/* Primitive (rho,u,v,w,p) [5][N] -> conserved Q [5][N] (System I energy). */
void orc_prim_to_cons(const orc_params *P, size_t N, const double *prim,
                      double *Q);

/* Philox4x32-10 block (Salmon et al., SC'11). */
void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2],
                       uint32_t out[4]);
/* Three standard normals of node n from Philox4x32-10 + Box-Muller. */
void orc_normals3(uint64_t seed, uint64_t n, double z[3]);

/* Jet initial condition: tanh profile + seeded normal velocity noise. */
void orc_init_jet(const orc_params *P, int ni, int nj, int nk,
                  const double *xyz, uint64_t seed, double noise, double *Q);

/* Effective viscosity and conductivity at every node. */
void orc_mu_eff(const orc_params *P, int ni, int nj, int nk, const double *Q,
                const double *M, double *MK);

/* RHS of Eq. spatial_discret at interior nodes, 0 at boundary nodes. */
void orc_rhs(const orc_params *P, int ni, int nj, int nk, const double *Q,
             const double *M, const double *MK, double *R);

/* Single interface flux (inviscid+dissipation-viscous) between node (i,j,k)
 * and its +1 neighbour along direction d.  Exposed for unit tests. */
void orc_interface_flux(const orc_params *P, int ni, int nj, int nk,
                        const double *Q, const double *M, const double *MK,
                        int d, int i, int j, int k, double F[5]);

/* Global CFL time step: cfl * min 1/(lam_xi + lam_eta + lam_zeta). */
double orc_dt(const orc_params *P, int ni, int nj, int nk, const double *Q,
              const double *M);
/* Test filter of the dynamic model applied to the node field f. */
void orc_test_filter(int ni, int nj, int nk, const int periodic[3],
                     const double *f, double *out);
/* Dynamic Smagorinsky procedure on state Q: out = {<num>, <den>} of C_ds,
 * C_I and Pr_sgs/C_ds, then C_ds, C_I, Pr_sgs. */
void orc_dynamic_coefficients(const orc_params *P, int ni, int nj, int nk,
                              const double *Q, const double *M, double out[9]);

/* Local time steps dtn[n] = cfl / (lam_xi + lam_eta + lam_zeta) at node n. */
void orc_dt_local(const orc_params *P, int ni, int nj, int nk, const double *Q,
                  const double *M, double *dtn);

/* Jet boundary conditions at time t (Sec. "Boundary Conditions"). */
void orc_bc_jet(const orc_params *P, int ni, int nj, int nk, double *Q,
                const double *M, const double *xyz, double t);

/* Generic 5-stage driver: Q^(l) = Q^(0) - alpha_l dt J RHS(Q^(l-1)).
 * rhs(user, Qs, R) fills R [ncomp][N]; nodes with update[n]==0 keep Q^(0);
 * Jinv may be NULL (J = 1); dtn, when not NULL, gives node n its own step
 * dtn[n] in place of dt. */
typedef void (*orc_rhs_fn)(void *user, const double *Q, double *R);
void orc_rk5(int ncomp, size_t N, double *Q, const unsigned char *update,
             const double *Jinv, double dt, const double *dtn, orc_rhs_fn rhs,
             void *user);

/* One full time step (mu_eff, dt, 5 stages, BCs).  Returns dt used. */
double orc_rk_step(const orc_params *P, int ni, int nj, int nk, double *Q,
                   const double *M, const double *xyz, double t);

/* w sum_{i,k} (p(i, js, k) - 1/gamma)^2 J^-1 |grad eta| (i, js, k): the
 * far-field functional of the adjoint window, one state's term. */
double orc_surface_functional(const orc_params *P, int ni, int nj, int nk,
                              const double *Q, const double *M, int js,
                              double w);

/* sum_n J^-1_n Q_c(n) for c = 0..4, summed in increasing n. */
void orc_totals(int ni, int nj, int nk, const double *Q, const double *M,
                double out[5]);

int orc_num_threads(void);
void orc_set_num_threads(int n);

#endif
