/*
 * les_oracle.c -- plain FP64 CPU oracle of the LES method of arXiv 2301.00817
 * ("Computational Performance of a LES Solver for Supersonic Jet Flow
 * Applications").  TEST INFRASTRUCTURE: only tests, the smoke check and the
 * benchmark's CPU-baseline leg use it.  It shares nothing with the CUDA code.
 *
 * The scheme is written out step by step in the paper's order and notation;
 * every loop evaluates one definition for one node or one interface.  Nothing
 * is fused or reordered.  Where the paper is silent or garbled the reading
 * taken is stated at the spot (labelled "Reading").
 *
 * Parity status: every function below is pinned by the CPU test-suite
 * (metric identity, free-stream preservation, discrete conservation,
 * manufactured-solution convergence, closed-form 1-D/linear cases, RK
 * amplification polynomial, Philox known-answer vectors, BC invariants).
 *
 * Build: gcc -O2 -ffp-contract=off -fopenmp (no fused multiply-add, so the
 * result is the same on x86-64 and aarch64).  OpenMP only splits independent
 * per-node loops; results do not depend on the thread count.
 */
#include "les_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

int orc_num_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

/* Threads of the OpenMP loops (n >= 1); results do not depend on it. */
void orc_set_num_threads(int n) {
#ifdef _OPENMP
  if (n >= 1) omp_set_num_threads(n);
#else
  (void)n;
#endif
}

/* ------------------------------------------------------------------ grid */

typedef struct {
  int n[3];
  int per[3];
  size_t N;
} grid_t;

static grid_t make_grid(int ni, int nj, int nk, const int per[3]) {
  grid_t g;
  g.n[0] = ni; g.n[1] = nj; g.n[2] = nk;
  g.per[0] = per[0]; g.per[1] = per[1]; g.per[2] = per[2];
  g.N = (size_t)ni * nj * nk;
  return g;
}

static size_t lin(const grid_t *g, const int c[3]) {
  return ((size_t)c[0] * g->n[1] + c[1]) * g->n[2] + c[2];
}

static void unlin(const grid_t *g, size_t n, int c[3]) {
  c[2] = (int)(n % g->n[2]);
  n /= g->n[2];
  c[1] = (int)(n % g->n[1]);
  c[0] = (int)(n / g->n[1]);
}

/* Linear index of the node 'off' steps from c along direction d; -1 if that
 * node lies outside a non-periodic direction.  Periodic directions wrap:
 * the grid holds n distinct points per period (index mod n). */
static long nbr(const grid_t *g, const int c[3], int d, int off) {
  int cc[3] = {c[0], c[1], c[2]};
  int v = c[d] + off;
  if (g->per[d]) {
    v %= g->n[d];
    if (v < 0) v += g->n[d];
  } else if (v < 0 || v >= g->n[d]) {
    return -1;
  }
  cc[d] = v;
  return (long)lin(g, cc);
}

/* A node is interior when it is not on a face of a non-periodic direction. */
static int is_interior(const grid_t *g, const int c[3]) {
  for (int d = 0; d < 3; ++d)
    if (!g->per[d] && (c[d] == 0 || c[d] == g->n[d] - 1)) return 0;
  return 1;
}

/* --------------------------------------------------------------- metrics */

/* Derivative of coordinate component comp (0=x,1=y,2=z) along direction d at
 * node c.  Second-order central difference; in a periodic direction the
 * coordinate of a wrapped neighbour is shifted by one period (shift[d][comp]);
 * at the faces of a non-periodic direction the one-sided second-order
 * formulas (-3f0+4f1-f2)/2 and (3fn-4fn-1+fn-2)/2 are used. */
static double coord_deriv(const grid_t *g, const double *xyz,
                          const double shift[9], const int c[3], int d,
                          int comp) {
  const double *f = xyz + (size_t)comp * g->N;
  int n = g->n[d];
  if (g->per[d]) {
    int cp[3] = {c[0], c[1], c[2]}, cm[3] = {c[0], c[1], c[2]};
    double sp = 0.0, sm = 0.0;
    cp[d] = c[d] + 1;
    if (cp[d] == n) { cp[d] = 0; sp = shift[3 * d + comp]; }
    cm[d] = c[d] - 1;
    if (cm[d] < 0) { cm[d] = n - 1; sm = -shift[3 * d + comp]; }
    return 0.5 * ((f[lin(g, cp)] + sp) - (f[lin(g, cm)] + sm));
  }
  int c0[3] = {c[0], c[1], c[2]}, c1[3] = {c[0], c[1], c[2]},
      c2[3] = {c[0], c[1], c[2]};
  if (c[d] == 0) {
    c1[d] = 1; c2[d] = 2;
    return 0.5 * (-3.0 * f[lin(g, c0)] + 4.0 * f[lin(g, c1)] - f[lin(g, c2)]);
  }
  if (c[d] == n - 1) {
    c1[d] = n - 2; c2[d] = n - 3;
    return 0.5 * (3.0 * f[lin(g, c0)] - 4.0 * f[lin(g, c1)] + f[lin(g, c2)]);
  }
  c1[d] = c[d] + 1; c2[d] = c[d] - 1;
  return 0.5 * (f[lin(g, c1)] - f[lin(g, c2)]);
}

/* Jacobian and the nine metric terms (Sec. "Transformation of Coordinates").
 * J^-1 is the determinant of d(x,y,z)/d(xi,eta,zeta) written with the six
 * products the paper lists.  The xi and zeta rows are the paper's formulas;
 * Reading A1: the paper's eta row differentiates in eta twice, which cannot
 * be a cofactor; the eta row used here is the matching cofactor
 * eta_x = J (y_zeta z_xi - y_xi z_zeta), eta_y = J (z_zeta x_xi - z_xi
 * x_zeta), eta_z = J (x_zeta y_xi - x_xi y_zeta). */
void orc_metrics(int ni, int nj, int nk, const int periodic[3],
                 const double shift[9], const double *xyz, double *M) {
  grid_t g = make_grid(ni, nj, nk, periodic);
  size_t N = g.N;
#pragma omp parallel for schedule(static)
  for (long nn = 0; nn < (long)N; ++nn) {
    int c[3];
    unlin(&g, (size_t)nn, c);
    double x_xi = coord_deriv(&g, xyz, shift, c, 0, 0);
    double x_eta = coord_deriv(&g, xyz, shift, c, 1, 0);
    double x_zeta = coord_deriv(&g, xyz, shift, c, 2, 0);
    double y_xi = coord_deriv(&g, xyz, shift, c, 0, 1);
    double y_eta = coord_deriv(&g, xyz, shift, c, 1, 1);
    double y_zeta = coord_deriv(&g, xyz, shift, c, 2, 1);
    double z_xi = coord_deriv(&g, xyz, shift, c, 0, 2);
    double z_eta = coord_deriv(&g, xyz, shift, c, 1, 2);
    double z_zeta = coord_deriv(&g, xyz, shift, c, 2, 2);
    double Jinv = x_xi * y_eta * z_zeta + x_eta * y_zeta * z_xi +
                  x_zeta * y_xi * z_eta - x_xi * y_zeta * z_eta -
                  x_eta * y_xi * z_zeta - x_zeta * y_eta * z_xi;
    /* Reading A27 (a true centerline grid, r from 0): on the axis the zeta
     * tangent vanishes, so J^-1 = 0 exactly and grad xi, grad eta, grad zeta
     * are unbounded; an axis node stores the J^-1-scaled metrics (the
     * cofactors themselves, finite) beside J^-1 = 0. */
    double J = (Jinv == 0.0) ? 1.0 : 1.0 / Jinv;
    M[0 * N + nn] = J * (y_eta * z_zeta - y_zeta * z_eta);
    M[1 * N + nn] = J * (z_eta * x_zeta - z_zeta * x_eta);
    M[2 * N + nn] = J * (x_eta * y_zeta - x_zeta * y_eta);
    M[3 * N + nn] = J * (y_zeta * z_xi - y_xi * z_zeta);
    M[4 * N + nn] = J * (z_zeta * x_xi - z_xi * x_zeta);
    M[5 * N + nn] = J * (x_zeta * y_xi - x_xi * y_zeta);
    M[6 * N + nn] = J * (y_xi * z_eta - y_eta * z_xi);
    M[7 * N + nn] = J * (z_xi * x_eta - z_eta * x_xi);
    M[8 * N + nn] = J * (x_xi * y_eta - x_eta * y_xi);
    M[9 * N + nn] = Jinv;
  }
}

/* Coordinate component comp at node c, where c may lie one period outside a
 * periodic direction: the stored value of the wrapped node plus one period's
 * shift per wrap. */
static double coord_at(const grid_t *g, const double *xyz,
                       const double shift[9], const int c[3], int comp) {
  int w[3] = {c[0], c[1], c[2]};
  double v = 0.0;
  for (int d = 0; d < 3; ++d) {
    if (w[d] < 0) { w[d] += g->n[d]; v -= shift[3 * d + comp]; }
    if (w[d] >= g->n[d]) { w[d] -= g->n[d]; v += shift[3 * d + comp]; }
  }
  return xyz[(size_t)comp * g->N + lin(g, w)] + v;
}

/* The product (dp/ds) q at node c (c as in coord_at): coordinate p
 * differentiated along s, times coordinate q. */
static double metric_product(const grid_t *g, const double *xyz,
                             const double shift[9], const int c[3], int p,
                             int s, int q) {
  int w[3] = {c[0], c[1], c[2]};
  for (int d = 0; d < 3; ++d) {
    if (w[d] < 0) w[d] += g->n[d];
    if (w[d] >= g->n[d]) w[d] -= g->n[d];
  }
  return coord_deriv(g, xyz, shift, w, s, p) * coord_at(g, xyz, shift, c, q);
}

/* Derivative along t of metric_product(p, s, q) at node c, with the same
 * second-order formulas as coord_deriv (central; one-sided at the faces of a
 * non-periodic direction). */
static double product_deriv(const grid_t *g, const double *xyz,
                            const double shift[9], const int c[3], int t,
                            int p, int s, int q) {
  int a[3] = {c[0], c[1], c[2]}, b[3] = {c[0], c[1], c[2]},
      e[3] = {c[0], c[1], c[2]};
  int n = g->n[t];
  if (g->per[t] || (c[t] > 0 && c[t] < n - 1)) {
    a[t] = c[t] + 1; b[t] = c[t] - 1;
    return 0.5 * (metric_product(g, xyz, shift, a, p, s, q) -
                  metric_product(g, xyz, shift, b, p, s, q));
  }
  if (c[t] == 0) {
    b[t] = 1; e[t] = 2;
    return 0.5 * (-3.0 * metric_product(g, xyz, shift, a, p, s, q) +
                  4.0 * metric_product(g, xyz, shift, b, p, s, q) -
                  metric_product(g, xyz, shift, e, p, s, q));
  }
  b[t] = n - 2; e[t] = n - 3;
  return 0.5 * (3.0 * metric_product(g, xyz, shift, a, p, s, q) -
                4.0 * metric_product(g, xyz, shift, b, p, s, q) +
                metric_product(g, xyz, shift, e, p, s, q));
}

/* Metric terms in the conservative (Thomas-Lombard) form, an alternative to
 * the cross-product formulas of Sec. "Transformation of Coordinates".  For
 * direction r with (r, s, t) a cyclic order of (xi, eta, zeta) and
 * component c with (c, p, q) a cyclic order of (x, y, z):
 *   J^-1 r_c = ((p_s) q)_t - ((p_t) q)_s,
 * which equals the cofactor p_s q_t - p_t q_s of the continuous mapping and,
 * written with central differences, makes sum_r delta_r (J^-1 r_c) vanish at
 * every interior node (the discrete geometric conservation law: free-stream
 * preservation on any grid).  J^-1 is the same determinant as in
 * orc_metrics; the stored metric is (J^-1 r_c) / J^-1. */
void orc_metrics_conservative(int ni, int nj, int nk, const int periodic[3],
                              const double shift[9], const double *xyz,
                              double *M) {
  grid_t g = make_grid(ni, nj, nk, periodic);
  size_t N = g.N;
#pragma omp parallel for schedule(static)
  for (long nn = 0; nn < (long)N; ++nn) {
    int c[3];
    unlin(&g, (size_t)nn, c);
    double d[3][3];
    for (int comp = 0; comp < 3; ++comp)
      for (int dir = 0; dir < 3; ++dir)
        d[comp][dir] = coord_deriv(&g, xyz, shift, c, dir, comp);
    double Jinv = d[0][0] * d[1][1] * d[2][2] + d[0][1] * d[1][2] * d[2][0] +
                  d[0][2] * d[1][0] * d[2][1] - d[0][0] * d[1][2] * d[2][1] -
                  d[0][1] * d[1][0] * d[2][2] - d[0][2] * d[1][1] * d[2][0];
    for (int r = 0; r < 3; ++r) {
      int s = (r + 1) % 3, t = (r + 2) % 3;
      for (int comp = 0; comp < 3; ++comp) {
        int p = (comp + 1) % 3, q = (comp + 2) % 3;
        double cof = product_deriv(&g, xyz, shift, c, t, p, s, q) -
                     product_deriv(&g, xyz, shift, c, s, p, t, q);
        /* an axis node (J^-1 = 0) keeps the scaled metric (Reading A27) */
        M[(size_t)(3 * r + comp) * N + nn] = (Jinv == 0.0) ? cof : cof / Jinv;
      }
    }
    M[9 * N + nn] = Jinv;
  }
}

/* ------------------------------------------------------ state conversion */

/* System I total energy e = p/(gamma-1) + rho u_i u_i / 2. */
void orc_prim_to_cons(const orc_params *P, size_t N, const double *prim,
                      double *Q) {
  double gm1 = P->gamma - 1.0;
  for (size_t n = 0; n < N; ++n) {
    double rho = prim[n], u = prim[N + n], v = prim[2 * N + n],
           w = prim[3 * N + n], p = prim[4 * N + n];
    Q[n] = rho;
    Q[N + n] = rho * u;
    Q[2 * N + n] = rho * v;
    Q[3 * N + n] = rho * w;
    Q[4 * N + n] = p / gm1 + 0.5 * rho * (u * u + v * v + w * w);
  }
}

/* ---------------------------------------------------------------- Philox */

/* Philox4x32 with 10 rounds, as published by Salmon, Moraes, Dror and Shaw
 * ("Parallel random numbers: as easy as 1, 2, 3", SC'11): each round
 * multiplies words 0 and 2 by the two round multipliers, swaps and xors the
 * high halves with the other words and the key; the key is bumped by the two
 * Weyl constants between rounds. */
void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2],
                       uint32_t out[4]) {
  const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
  const uint32_t W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
  uint32_t x0 = ctr[0], x1 = ctr[1], x2 = ctr[2], x3 = ctr[3];
  uint32_t k0 = key[0], k1 = key[1];
  for (int r = 0; r < 10; ++r) {
    uint64_t p0 = (uint64_t)M0 * x0;
    uint64_t p1 = (uint64_t)M1 * x2;
    uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
    uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
    uint32_t y0 = hi1 ^ x1 ^ k0;
    uint32_t y1 = lo1;
    uint32_t y2 = hi0 ^ x3 ^ k1;
    uint32_t y3 = lo0;
    x0 = y0; x1 = y1; x2 = y2; x3 = y3;
    k0 += W0;
    k1 += W1;
  }
  out[0] = x0; out[1] = x1; out[2] = x2; out[3] = x3;
}

/* Uniform in (0,1) from 53 bits of a 64-bit word (midpoint of the bin). */
static double u01_53(uint32_t lo, uint32_t hi) {
  uint64_t b = (((uint64_t)hi << 32) | lo) >> 11;
  return ((double)b + 0.5) * (1.0 / 9007199254740992.0);
}

/* Three standard normals of node n: counter (n_lo, n_hi, block, 0), key
 * (seed_lo, seed_hi); each Philox block gives two uniforms and Box-Muller
 * (Box & Muller 1958) turns them into two normals.  Block 0 gives z0, z1;
 * block 1 gives z2 (its second normal is unused). */
void orc_normals3(uint64_t seed, uint64_t n, double z[3]) {
  const double two_pi = 6.283185307179586476925286766559;
  uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
  for (uint32_t blk = 0; blk < 2; ++blk) {
    uint32_t ctr[4] = {(uint32_t)n, (uint32_t)(n >> 32), blk, 0u}, o[4];
    orc_philox4x32_10(ctr, key, o);
    double u1 = u01_53(o[0], o[1]);
    double u2 = u01_53(o[2], o[3]);
    double rad = sqrt(-2.0 * log(u1));
    if (blk == 0) {
      z[0] = rad * cos(two_pi * u2);
      z[1] = rad * sin(two_pi * u2);
    } else {
      z[2] = rad * cos(two_pi * u2);
    }
  }
}

/* Inflow/initial axial velocity profile (hyperbolic-tangent shear layer):
 * u(r) = U_j/2 [1 + tanh((r_jet - r) / (2 theta_m))], U_j = M_j a_j. */
static double jet_profile(const orc_params *P, double r) {
  return 0.5 * P->Mj * (1.0 + tanh((P->r_jet - r) / (2.0 * P->theta_m)));
}

/* Initial condition: rho = 1, p = 1/gamma (cold isothermal jet), axial
 * velocity profile plus noise * U_j * N(0,1) on the three Cartesian velocity
 * components.  r = sqrt(y^2 + z^2). */
void orc_init_jet(const orc_params *P, int ni, int nj, int nk,
                  const double *xyz, uint64_t seed, double noise, double *Q) {
  size_t N = (size_t)ni * nj * nk;
  double *prim = (double *)malloc(5 * N * sizeof(double));
  for (size_t n = 0; n < N; ++n) {
    double y = xyz[N + n], zc = xyz[2 * N + n];
    double r = sqrt(y * y + zc * zc);
    double z[3];
    orc_normals3(seed, (uint64_t)n, z);
    prim[n] = 1.0;
    prim[N + n] = jet_profile(P, r) + noise * P->Mj * z[0];
    prim[2 * N + n] = noise * P->Mj * z[1];
    prim[3 * N + n] = noise * P->Mj * z[2];
    prim[4 * N + n] = 1.0 / P->gamma;
  }
  orc_prim_to_cons(P, N, prim, Q);
  free(prim);
}

/* ------------------------------------------------------------ primitives */

typedef struct {
  const orc_params *P;
  grid_t g;
  const double *Q, *M, *MK;
  /* per-node work arrays */
  double *u, *v, *w, *p, *T, *a;
  double *lam[3];    /* spectral radii lambda_xi, lambda_eta, lambda_zeta */
  double *lbar[3];   /* anisotropic scaled radii (overbar lambda) */
  double *nu[3];     /* pressure sensor per direction */
} state_t;

/* Primitive recovery: u_i = (rho u_i)/rho, p from the System I energy,
 * T = gamma p / rho (dimensionless, T_j = 1), a = sqrt(gamma p / rho). */
static void node_primitives(state_t *S) {
  const grid_t *g = &S->g;
  size_t N = g->N;
  double gam = S->P->gamma;
#pragma omp parallel for schedule(static)
  for (long n = 0; n < (long)N; ++n) {
    double rho = S->Q[n];
    double u = S->Q[N + n] / rho, v = S->Q[2 * N + n] / rho,
           w = S->Q[3 * N + n] / rho;
    double p = (gam - 1.0) * (S->Q[4 * N + n] - 0.5 * rho * (u * u + v * v + w * w));
    S->u[n] = u; S->v[n] = v; S->w[n] = w; S->p[n] = p;
    S->T[n] = gam * p / rho;
    S->a[n] = sqrt(gam * p / rho);
  }
}

/* Spectral radii and their anisotropic scaling (Sec. "Spatial
 * Discretization").  Reading A10: the paper labels all three radii lambda_xi
 * and uses sqrt(xi_x^2+eta_y^2+zeta_z^2); the radius of direction d is
 * |contravariant velocity| + a |grad d| with that direction's own metrics.
 * lbar_xi = lam_xi [1 + (lam_eta/lam_xi)^0.5 + (lam_zeta/lam_xi)^0.5] and
 * cyclically for eta and zeta. */
static void node_radii(state_t *S) {
  size_t N = S->g.N;
#pragma omp parallel for schedule(static)
  for (long n = 0; n < (long)N; ++n) {
    double l[3];
    for (int d = 0; d < 3; ++d) {
      double mx = S->M[(3 * d) * N + n], my = S->M[(3 * d + 1) * N + n],
             mz = S->M[(3 * d + 2) * N + n];
      double Ucon = mx * S->u[n] + my * S->v[n] + mz * S->w[n];
      l[d] = fabs(Ucon) + S->a[n] * sqrt(mx * mx + my * my + mz * mz);
      S->lam[d][n] = l[d];
    }
    S->lbar[0][n] = l[0] * (1.0 + sqrt(l[1] / l[0]) + sqrt(l[2] / l[0]));
    S->lbar[1][n] = l[1] * (1.0 + sqrt(l[0] / l[1]) + sqrt(l[2] / l[1]));
    S->lbar[2][n] = l[2] * (1.0 + sqrt(l[0] / l[2]) + sqrt(l[1] / l[2]));
  }
  /* Reading A27: an axis node (J^-1 = 0, on the face j = 0) has no radius of
   * its own (its metrics are J^-1-scaled); like a face node's sensor
   * (Reading A12) it takes the radii of its inward neighbour (i, 1, k). */
  for (long n = 0; n < (long)N; ++n) {
    if (S->M[9 * N + n] != 0.0) continue;
    int c[3];
    unlin(&S->g, (size_t)n, c);
    int c1[3] = {c[0], 1, c[2]};
    long n1 = (long)lin(&S->g, c1);
    for (int d = 0; d < 3; ++d) {
      S->lam[d][n] = S->lam[d][n1];
      S->lbar[d][n] = S->lbar[d][n1];
    }
  }
}

/* Pressure sensor of Eq. p_grad_sensor.  Reading A7: the printed ratio
 * |d2p|/d2p is +-1; the Jameson/Turkel-Vatsa sensor normalises by the sum,
 * nu_i = |p_{i+1} - 2 p_i + p_{i-1}| / (p_{i+1} + 2 p_i + p_{i-1}).
 * Reading A12: at a face of a non-periodic direction nu is the value of the
 * inward neighbour. */
static double sensor_at(const state_t *S, const int c[3], int d) {
  const grid_t *g = &S->g;
  long m = nbr(g, c, d, -1), pl = nbr(g, c, d, +1);
  if (m < 0 || pl < 0) {
    int cc[3] = {c[0], c[1], c[2]};
    cc[d] += (m < 0) ? 1 : -1;
    m = nbr(g, cc, d, -1);
    pl = nbr(g, cc, d, +1);
    long n0 = (long)lin(g, cc);
    double pp = S->p[pl], p0 = S->p[n0], pm = S->p[m];
    return fabs(pp - 2.0 * p0 + pm) / (pp + 2.0 * p0 + pm);
  }
  long n0 = (long)lin(g, c);
  double pp = S->p[pl], p0 = S->p[n0], pm = S->p[m];
  return fabs(pp - 2.0 * p0 + pm) / (pp + 2.0 * p0 + pm);
}

static void node_sensors(state_t *S) {
  size_t N = S->g.N;
#pragma omp parallel for schedule(static)
  for (long n = 0; n < (long)N; ++n) {
    int c[3];
    unlin(&S->g, (size_t)n, c);
    for (int d = 0; d < 3; ++d) S->nu[d][n] = sensor_at(S, c, d);
  }
}

static void state_alloc(state_t *S) {
  size_t N = S->g.N;
  double **all[] = {&S->u, &S->v, &S->w, &S->p, &S->T, &S->a,
                    &S->lam[0], &S->lam[1], &S->lam[2],
                    &S->lbar[0], &S->lbar[1], &S->lbar[2],
                    &S->nu[0], &S->nu[1], &S->nu[2]};
  for (size_t q = 0; q < sizeof(all) / sizeof(all[0]); ++q)
    *all[q] = (double *)malloc(N * sizeof(double));
}

static void state_free(state_t *S) {
  double *all[] = {S->u, S->v, S->w, S->p, S->T, S->a,
                   S->lam[0], S->lam[1], S->lam[2],
                   S->lbar[0], S->lbar[1], S->lbar[2],
                   S->nu[0], S->nu[1], S->nu[2]};
  for (size_t q = 0; q < sizeof(all) / sizeof(all[0]); ++q) free(all[q]);
}

static void state_build(state_t *S, const orc_params *P, int ni, int nj,
                        int nk, const double *Q, const double *M,
                        const double *MK) {
  S->P = P;
  S->g = make_grid(ni, nj, nk, P->periodic);
  S->Q = Q; S->M = M; S->MK = MK;
  state_alloc(S);
  node_primitives(S);
  node_radii(S);
  node_sensors(S);
}

/* ------------------------------------------------------------- viscosity */

/* Node-centred computational derivative of field f along d: central
 * difference, one-sided second order at non-periodic faces. */
static double node_deriv(const grid_t *g, const double *f, const int c[3],
                         int d) {
  long m = nbr(g, c, d, -1), pl = nbr(g, c, d, +1);
  long n0 = (long)lin(g, c);
  if (m >= 0 && pl >= 0) return 0.5 * (f[pl] - f[m]);
  if (m < 0) {
    long p2 = nbr(g, c, d, +2);
    return 0.5 * (-3.0 * f[n0] + 4.0 * f[pl] - f[p2]);
  }
  long m2 = nbr(g, c, d, -2);
  return 0.5 * (3.0 * f[n0] - 4.0 * f[m] + f[m2]);
}

/* Sutherland law (Eq. sutherland) in dimensionless form.  Reading A5: with
 * T scaled by T_ref (= T_j = T_inf for the cold jet),
 * mu/mu_ref = T^(3/2) (1 + S) / (T + S), S = 110.4 K / T_ref.
 * Reading A4: the dimensionless viscous terms carry the factor M_j/Re
 * (Eq. vec-underline-split-RANS), so mu_lam = (M_j/Re) mu/mu_ref; with
 * Cp T_j / a_j^2 = 1/(gamma-1), kappa = mu/((gamma-1) Pr). */
static double mu_laminar(const orc_params *P, double T) {
  if (P->Re <= 0.0) return 0.0;
  double S = 110.4 / P->T_ref;
  return (P->Mj / P->Re) * pow(T, 1.5) * (1.0 + S) / (T + S);
}

/* ------------------------------------------------- dynamic Smagorinsky */

/* Weight of offset off (-1, 0, 1) along direction d of the test filter at
 * node c (Reading A26): the trapezoidal (1/4, 1/2, 1/4) filter of width two
 * cells, the identity along a non-periodic direction at its faces. */
static double filter_weight(const grid_t *g, const int c[3], int d, int off) {
  if (!g->per[d] && (c[d] == 0 || c[d] == g->n[d] - 1)) return off == 0 ? 1.0 : 0.0;
  return off == 0 ? 0.5 : 0.25;
}

/* Test filter of the field f at every node: the 27-point tensor product of
 * the one-dimensional weights. */
static void test_filter(const grid_t *g, const double *f, double *out) {
#pragma omp parallel for schedule(static)
  for (long n = 0; n < (long)g->N; ++n) {
    int c[3];
    unlin(g, (size_t)n, c);
    double s = 0.0;
    for (int a = -1; a <= 1; ++a)
      for (int b = -1; b <= 1; ++b)
        for (int e = -1; e <= 1; ++e) {
          double wgt = filter_weight(g, c, 0, a) * filter_weight(g, c, 1, b) *
                       filter_weight(g, c, 2, e);
          if (wgt == 0.0) continue;
          int cc[3] = {c[0] + a, c[1] + b, c[2] + e};
          for (int d = 0; d < 3; ++d) cc[d] = (cc[d] + g->n[d]) % g->n[d];
          s += wgt * f[lin(g, cc)];
        }
    out[n] = s;
  }
}

/* Cartesian gradient of the node field f at node c (node-centred
 * differences through the node's metrics, as for the static models). */
static void cart_grad(const grid_t *g, const double *M, const double *f,
                      const int c[3], double out[3]) {
  size_t N = g->N, n = lin(g, c);
  double dd[3];
  for (int d = 0; d < 3; ++d) dd[d] = node_deriv(g, f, c, d);
  for (int x = 0; x < 3; ++x)
    out[x] = M[x * N + n] * dd[0] + M[(3 + x) * N + n] * dd[1] +
             M[(6 + x) * N + n] * dd[2];
}

/* Strain rate S_ij = (d_j u_i + d_i u_j)/2 of the velocity fields (u, v, w)
 * at node c, and |S| = (2 S_ij S_ij)^(1/2). */
static double strain_at(const grid_t *g, const double *M, const double *u,
                        const double *v, const double *w, const int c[3],
                        double Sij[3][3]) {
  const double *vel[3] = {u, v, w};
  double gr[3][3];
  for (int q = 0; q < 3; ++q) cart_grad(g, M, vel[q], c, gr[q]);
  double ss = 0.0;
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      Sij[i][j] = 0.5 * (gr[i][j] + gr[j][i]);
      ss += Sij[i][j] * Sij[i][j];
    }
  return sqrt(2.0 * ss);
}

/* The dynamic procedure (Sec. "Dynamic Smagorinsky Model", Eqs. av_ci,
 * av_cd, av_Pr_sgs) on the state Q with node primitives (u, v, w, T).
 * Readings (A26): the test filter is test_filter, of width Delta^ = 2 Delta;
 * Favre-filtered fields are u^_i = (rho u_i)^/rho^, T^ = (rho T)^/rho^, and
 * S^ is the strain of u^; by the Germano identity the trace term
 * T_ll - sigma^_ll of Eq. av_cd is L_kk, L_ij = (rho u_i u_j)^ -
 * (rho u_i)^ (rho u_j)^/rho^; the second term of Eq. av_Pr_sgs contracts the
 * gradient of T^ with that of T; <.> is the J^-1-weighted mean over the
 * interior nodes.  out = {<num>, <den>} of C_ds, C_I and Pr_sgs/C_ds, then
 * C_ds, C_I, Pr_sgs: C_ds and C_I are clipped at 0 (and are 0 when their
 * denominator vanishes); Pr_sgs falls back to the configured value when it
 * is not positive and finite. */
static void dynamic_procedure(const orc_params *P, const grid_t *g,
                              const double *Q, const double *M,
                              const double *u, const double *v,
                              const double *w, const double *T,
                              double out[9]) {
  size_t N = g->N;
  enum { NF = 25 };
  double *f = (double *)malloc(NF * N * sizeof(double));
  double *fh = (double *)malloc(NF * N * sizeof(double));
  /* node products: rho, rho u_i, rho T, rho u_i u_j (xx yy zz xy xz yz),
   * rho|S| S_ij (same order), rho|S| S_mm, rho|S|^2, rho u_j T,
   * rho|S| dT/dx_j */
  static const int I6[6] = {0, 1, 2, 0, 0, 1}, J6[6] = {0, 1, 2, 1, 2, 2};
  for (size_t n = 0; n < N; ++n) {
    int c[3];
    unlin(g, n, c);
    double rho = Q[n], vel[3] = {u[n], v[n], w[n]}, Sij[3][3], dT[3];
    double Sm = strain_at(g, M, u, v, w, c, Sij);
    cart_grad(g, M, T, c, dT);
    f[0 * N + n] = rho;
    for (int i = 0; i < 3; ++i) f[(1 + i) * N + n] = rho * vel[i];
    f[4 * N + n] = rho * T[n];
    for (int k = 0; k < 6; ++k) {
      f[(5 + k) * N + n] = rho * vel[I6[k]] * vel[J6[k]];
      f[(11 + k) * N + n] = rho * Sm * Sij[I6[k]][J6[k]];
    }
    f[17 * N + n] = rho * Sm * (Sij[0][0] + Sij[1][1] + Sij[2][2]);
    f[18 * N + n] = rho * Sm * Sm;
    for (int j = 0; j < 3; ++j) {
      f[(19 + j) * N + n] = rho * vel[j] * T[n];
      f[(22 + j) * N + n] = rho * Sm * dT[j];
    }
  }
  for (int q = 0; q < NF; ++q) test_filter(g, f + (size_t)q * N, fh + (size_t)q * N);
  /* Favre-filtered velocity and temperature */
  double *uh = (double *)malloc(4 * N * sizeof(double));
  for (size_t n = 0; n < N; ++n) {
    for (int i = 0; i < 3; ++i) uh[i * N + n] = fh[(1 + i) * N + n] / fh[n];
    uh[3 * N + n] = fh[4 * N + n] / fh[n];
  }
  double sum[7] = {0, 0, 0, 0, 0, 0, 0}; /* 6 weighted sums, then sum of J^-1 */
  for (size_t n = 0; n < N; ++n) {
    int c[3];
    unlin(g, n, c);
    if (!is_interior(g, c)) continue;
    double wgt = M[9 * N + n];
    double Delta = cbrt(M[9 * N + n]), D2 = Delta * Delta, Dh2 = 4.0 * D2;
    double Sij[3][3], dT[3], Sh[3][3], dTh[3];
    double Sm = strain_at(g, M, u, v, w, c, Sij);
    cart_grad(g, M, T, c, dT);
    double Shm = strain_at(g, M, uh, uh + N, uh + 2 * N, c, Sh);
    cart_grad(g, M, uh + 3 * N, c, dTh);
    (void)Sm;
    double rh = fh[n], mh[3] = {fh[N + n], fh[2 * N + n], fh[3 * N + n]};
    double L[3][3], Fs[3][3];
    for (int k = 0; k < 6; ++k) {
      int i = I6[k], j = J6[k];
      L[i][j] = L[j][i] = fh[(5 + k) * N + n] - mh[i] * mh[j] / rh;
      Fs[i][j] = Fs[j][i] = fh[(11 + k) * N + n];
    }
    double trS = Sij[0][0] + Sij[1][1] + Sij[2][2];
    double trSh = Sh[0][0] + Sh[1][1] + Sh[2][2];
    double LS = 0.0, FS = 0.0, ShS = 0.0;
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j) {
        LS += L[i][j] * Sij[i][j];
        FS += Fs[i][j] * Sij[i][j];
        ShS += Sh[i][j] * Sij[i][j];
      }
    double Lkk = L[0][0] + L[1][1] + L[2][2];
    double numC = LS - Lkk * trS / 3.0;
    double denC = 2.0 * D2 * (FS - fh[17 * N + n] * trS / 3.0) -
                  2.0 * Dh2 * (rh * Shm * ShS - rh * Shm * trSh * trS / 3.0);
    double numI = Lkk;
    double denI = 2.0 * Dh2 * rh * Shm * Shm - 2.0 * D2 * fh[18 * N + n];
    double numP = 0.0, denP = 0.0;
    for (int j = 0; j < 3; ++j) {
      double K = fh[(19 + j) * N + n] - mh[j] * fh[4 * N + n] / rh;
      numP += D2 * fh[(22 + j) * N + n] * dT[j] - Dh2 * rh * Shm * dTh[j] * dT[j];
      denP += K * dT[j];
    }
    sum[0] += wgt * numC; sum[1] += wgt * denC;
    sum[2] += wgt * numI; sum[3] += wgt * denI;
    sum[4] += wgt * numP; sum[5] += wgt * denP;
    sum[6] += wgt;
  }
  for (int q = 0; q < 6; ++q) out[q] = sum[q] / sum[6];
  double Cd = out[1] != 0.0 ? out[0] / out[1] : 0.0;
  if (!(Cd > 0.0)) Cd = 0.0;
  double CI = out[3] != 0.0 ? out[2] / out[3] : 0.0;
  if (!(CI > 0.0)) CI = 0.0;
  double Pr = out[5] != 0.0 ? Cd * out[4] / out[5] : 0.0;
  if (!(Pr > 0.0) || !(Pr < 1e300)) Pr = P->Pr_sgs;
  out[6] = Cd; out[7] = CI; out[8] = Pr;
  free(uh);
  free(fh);
  free(f);
}

void orc_test_filter(int ni, int nj, int nk, const int periodic[3],
                     const double *f, double *out) {
  grid_t g = make_grid(ni, nj, nk, periodic);
  test_filter(&g, f, out);
}

void orc_dynamic_coefficients(const orc_params *P, int ni, int nj, int nk,
                              const double *Q, const double *M, double out[9]) {
  state_t S;
  memset(&S, 0, sizeof(S));
  S.P = P;
  S.g = make_grid(ni, nj, nk, P->periodic);
  S.Q = Q; S.M = M;
  state_alloc(&S);
  node_primitives(&S);
  dynamic_procedure(P, &S.g, Q, M, S.u, S.v, S.w, S.T, out);
  state_free(&S);
}

/* Effective viscosity/conductivity (Sec. "Large Eddy Simulation Filtering",
 * "Subgrid Scale Modeling").  Reading A6: Smagorinsky is
 * mu_sgs = rho (Cs Delta)^2 |S| (the printed (rho Cs Delta)^2 squares rho),
 * the filter width is Delta = Delta_m = (J^-1)^(1/3) (unit computational
 * spacing), and mu_sgs is already in rho_j a_j D units (no M_j/Re).
 * Vreman: mu_sgs = rho c sqrt(B_beta / alpha_ij alpha_ij), c = 2.5 Cs^2,
 * alpha_ij = d u_j / d x_i, beta_ij = Delta^2 alpha_mi alpha_mj, zero when
 * alpha_ij alpha_ij = 0; Reading: B_beta, a sum of principal 2x2 minors of a
 * positive semi-definite matrix, is clipped at 0 against rounding.
 * kappa_eff = mu_lam/((gamma-1)Pr) + mu_sgs/((gamma-1)Pr_sgs). */
void orc_mu_eff(const orc_params *P, int ni, int nj, int nk, const double *Q,
                const double *M, double *MK) {
  state_t S;
  memset(&S, 0, sizeof(S));
  S.P = P;
  S.g = make_grid(ni, nj, nk, P->periodic);
  S.Q = Q; S.M = M;
  state_alloc(&S);
  node_primitives(&S);
  size_t N = S.g.N;
  double gm1 = P->gamma - 1.0;
  double dyn[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
  if (P->sgs_model == 3)
    dynamic_procedure(P, &S.g, Q, M, S.u, S.v, S.w, S.T, dyn);
  double *mus = (double *)malloc(N * sizeof(double));  /* mu_sgs per node */
#pragma omp parallel for schedule(static)
  for (long n = 0; n < (long)N; ++n) {
    int c[3];
    unlin(&S.g, (size_t)n, c);
    double rho = Q[n];
    double mu_l = mu_laminar(P, S.T[n]);
    double mu_s = 0.0;
    if (P->sgs_model == 3) {
      /* dynamic model: mu_sgs = C_ds rho Delta^2 |S| (Reading A26: C_ds
       * takes the place of Cs^2, as the dimensions of Eq. av_cd show),
       * kappa_sgs with the dynamic Pr_sgs, and the Yoshizawa isotropic part
       * sigma_ll = 2 C_I rho Delta^2 |S|^2 (Eq. yoshizawa) */
      double Sij[3][3];
      double Smag = strain_at(&S.g, M, S.u, S.v, S.w, c, Sij);
      double D2 = cbrt(M[9 * N + n]) * cbrt(M[9 * N + n]);
      mu_s = dyn[6] * rho * D2 * Smag;
      mus[n] = mu_s;
      MK[n] = mu_l + mu_s;
      MK[N + n] = mu_l / (gm1 * P->Pr) + mu_s / (gm1 * dyn[8]);
      MK[2 * N + n] = 2.0 * dyn[7] * rho * D2 * Smag * Smag;
      continue;
    }
    if (P->sgs_model != 0) {
      const double *vel[3] = {S.u, S.v, S.w};
      double g[3][3]; /* g[i][c] = d u_i / d x_c */
      for (int q = 0; q < 3; ++q) {
        double dd[3];
        for (int d = 0; d < 3; ++d) dd[d] = node_deriv(&S.g, vel[q], c, d);
        for (int cc = 0; cc < 3; ++cc)
          g[q][cc] = M[(0 + cc) * N + n] * dd[0] + M[(3 + cc) * N + n] * dd[1] +
                     M[(6 + cc) * N + n] * dd[2];
      }
      double Delta = cbrt(M[9 * N + n]);
      if (P->sgs_model == 1) {
        double SS = 0.0;
        for (int i = 0; i < 3; ++i)
          for (int j = 0; j < 3; ++j) {
            double Sij = 0.5 * (g[i][j] + g[j][i]);
            SS += Sij * Sij;
          }
        double Smag = sqrt(2.0 * SS);
        mu_s = rho * (P->Cs * Delta) * (P->Cs * Delta) * Smag;
      } else {
        double al[3][3], aa = 0.0; /* alpha_ij = d u_j / d x_i */
        for (int i = 0; i < 3; ++i)
          for (int j = 0; j < 3; ++j) {
            al[i][j] = g[j][i];
            aa += al[i][j] * al[i][j];
          }
        double be[3][3];
        for (int i = 0; i < 3; ++i)
          for (int j = 0; j < 3; ++j) {
            double s = 0.0;
            for (int m = 0; m < 3; ++m) s += al[m][i] * al[m][j];
            be[i][j] = Delta * Delta * s;
          }
        double B = be[0][0] * be[1][1] - be[0][1] * be[0][1] +
                   be[0][0] * be[2][2] - be[0][2] * be[0][2] +
                   be[1][1] * be[2][2] - be[1][2] * be[1][2];
        if (B < 0.0) B = 0.0;
        double c_v = 2.5 * P->Cs * P->Cs;
        mu_s = (aa == 0.0) ? 0.0 : rho * c_v * sqrt(B / aa);
      }
    }
    mus[n] = mu_s;
    MK[n] = mu_l + mu_s;
    MK[N + n] = mu_l / (gm1 * P->Pr) + mu_s / (gm1 * P->Pr_sgs);
  }
  /* Reading A27: an axis node (J^-1 = 0) has no velocity gradient of its own
   * (its metrics are J^-1-scaled); like its state under the centerline rule,
   * its mu_sgs is the azimuthal mean over the ring j = 1 at its plane, summed
   * in increasing k; mu_lam is its own.  (The reading covers the static
   * models: the dynamic model's test filter would carry the axis nodes'
   * scaled data into ring 1, so it is not defined on a grid with an axis.) */
  int nk_ = S.g.n[2];
  for (long n = 0; n < (long)N; ++n) {
    if (M[9 * N + n] != 0.0) continue;
    int c[3];
    unlin(&S.g, (size_t)n, c);
    double sm = 0.0, ss = 0.0;
    for (int k = 0; k < nk_; ++k) {
      int c1[3] = {c[0], 1, k};
      size_t n1 = lin(&S.g, c1);
      sm += mus[n1];
      if (P->sgs_model == 3) ss += MK[2 * N + n1];
    }
    double mu_s = sm / (double)nk_;
    double mu_l = mu_laminar(P, S.T[n]);
    double prs = (P->sgs_model == 3) ? dyn[8] : P->Pr_sgs;
    MK[n] = mu_l + mu_s;
    MK[N + n] = mu_l / (gm1 * P->Pr) + mu_s / (gm1 * prs);
    if (P->sgs_model == 3) MK[2 * N + n] = ss / (double)nk_;
  }
  free(mus);
  state_free(&S);
}

/* ------------------------------------------------------ interface fluxes */

/* Inviscid flux vector of direction d at node n (Eq. hat-flux-G), static
 * grid (metric time derivatives 0): J^-1 [rho Th, rho u Th + p m_x,
 * rho v Th + p m_y, rho w Th + p m_z, (e + p) Th], Th = m . u. */
static void node_inviscid_flux(const state_t *S, long n, int d, double F[5]) {
  size_t N = S->g.N;
  double mx = S->M[(3 * d) * N + n], my = S->M[(3 * d + 1) * N + n],
         mz = S->M[(3 * d + 2) * N + n];
  double Jinv = S->M[9 * N + n];
  double Th = mx * S->u[n] + my * S->v[n] + mz * S->w[n];
  double p = S->p[n];
  F[0] = Jinv * (S->Q[n] * Th);
  F[1] = Jinv * (S->Q[N + n] * Th + p * mx);
  F[2] = Jinv * (S->Q[2 * N + n] * Th + p * my);
  F[3] = Jinv * (S->Q[3 * N + n] * Th + p * mz);
  F[4] = Jinv * ((S->Q[4 * N + n] + p) * Th);
}

/* Dissipated vector W (Eq. W_dissip).  Reading A9: W is built from the
 * unscaled Q (plus p in the energy slot) and the J^-1 of Eq. inv_flux_vec is
 * applied once, at the interface, so d vanishes for any uniform state. */
static double W_of(const state_t *S, long n, int comp) {
  double q = S->Q[(size_t)comp * S->g.N + n];
  return comp == 4 ? q + S->p[n] : q;
}

static void interface_flux(const state_t *S, int d, const int ca[3],
                           double F[5]) {
  const grid_t *g = &S->g;
  const orc_params *P = S->P;
  size_t N = g->N;
  long a = (long)lin(g, ca);
  long b = nbr(g, ca, d, +1);
  long am = nbr(g, ca, d, -1);
  long bp = nbr(g, ca, d, +2);
  int cb[3] = {ca[0], ca[1], ca[2]};
  cb[d] = (int)((ca[d] + 1) % g->n[d]);

  /* (1) centred inviscid flux, Eq. inv_flux_vec: (F_a + F_b)/2 */
  double Fa[5], Fb[5];
  node_inviscid_flux(S, a, d, Fa);
  node_inviscid_flux(S, b, d, Fb);

  /* (2) Turkel-Vatsa dissipation d (Eqs. dissip_term, eps_2_dissip,
   * eps_4_dissip).  Reading A8: the operator lost at the line break is a
   * minus, d = lam [eps2 (W_b - W_a) - eps4 (W_{b+1} - 3 W_b + 3 W_a
   * - W_{a-1})], written with the differences DW of the boundary section:
   * D3 = DW_{+3/2} - 2 DW_{+1/2} + DW_{-1/2}.  Reading A12: at a face of a
   * non-periodic direction the missing outside difference is minus the first
   * inside one, (DW)_{1/2} = -(DW)_{1+1/2} (Sec. "Centerline Boundary
   * Condition"), applied at every non-periodic face. */
  double nu_a = S->nu[d][a], nu_b = S->nu[d][b];
  double eps2 = P->k2 * (nu_b > nu_a ? nu_b : nu_a);
  double eps4 = P->k4 - eps2;
  if (eps4 < 0.0) eps4 = 0.0;
  double lam = 0.5 * (S->lbar[d][a] + S->lbar[d][b]);
  double Jh = 0.5 * (S->M[9 * N + a] + S->M[9 * N + b]);
  double Fe[5];
  for (int q = 0; q < 5; ++q) {
    double D1 = W_of(S, b, q) - W_of(S, a, q);
    double Dm = (am >= 0) ? W_of(S, a, q) - W_of(S, am, q) : -D1;
    double Dp = (bp >= 0) ? W_of(S, bp, q) - W_of(S, b, q) : -D1;
    double D3 = Dp - 2.0 * D1 + Dm;
    double dq = lam * (eps2 * D1 - eps4 * D3);
    Fe[q] = 0.5 * (Fa[q] + Fb[q]) - Jh * dq;
  }

  /* (3) viscous + SGS interface flux (Eqs. hat-flux-Ev/Fv/Gv, tau_mod,
   * q_mod).  Reading A11: "differences of the viscous flux vectors use two
   * neighboring points of the interface": the normal derivative is
   * phi_b - phi_a and a tangential derivative is the mean of the central
   * differences at a and b, 1/4[(phi_{a+t} - phi_{a-t}) + (phi_{b+t} -
   * phi_{b-t})]; Cartesian gradients use the interface metrics (means of
   * the two nodes).  Reading A2: Fourier's law q_j = -kappa dT/dx_j (the
   * printed sign is anti-diffusive), beta_j = tau_jk u_k - q_j. */
  const double *phi[4] = {S->u, S->v, S->w, S->T};
  double dphi[4][3];
  for (int t = 0; t < 3; ++t) {
    if (t == d) {
      for (int q = 0; q < 4; ++q) dphi[q][t] = phi[q][b] - phi[q][a];
    } else {
      long ap = nbr(g, ca, t, +1), amt = nbr(g, ca, t, -1);
      long bpt = nbr(g, cb, t, +1), bmt = nbr(g, cb, t, -1);
      /* Interfaces of interior nodes always have both tangential
       * neighbours; an interface lying in a non-periodic face (never used
       * by the residual) gets a zero tangential derivative. */
      if (ap < 0 || amt < 0 || bpt < 0 || bmt < 0) {
        for (int q = 0; q < 4; ++q) dphi[q][t] = 0.0;
        continue;
      }
      for (int q = 0; q < 4; ++q)
        dphi[q][t] = 0.25 * ((phi[q][ap] - phi[q][amt]) +
                             (phi[q][bpt] - phi[q][bmt]));
    }
  }
  double mh[3][3]; /* mh[t][c]: interface metric of direction t, comp c */
  double Ja = S->M[9 * N + a], Jb = S->M[9 * N + b];
  if (!P->axis && Ja != 0.0 && Jb != 0.0) {
    for (int t = 0; t < 3; ++t)
      for (int cc = 0; cc < 3; ++cc)
        mh[t][cc] = 0.5 * (S->M[(3 * t + cc) * N + a] + S->M[(3 * t + cc) * N + b]);
  } else {
    /* Reading A27: on a grid with an axis (and at any interface touching an
     * axis node, where the plain mean is unbounded) the interface metric is
     * the J^-1-weighted mean, the mean of the scaled metrics J^-1 grad(t)
     * over the mean J^-1.  Near the axis |grad zeta| ~ 1/r changes by O(1)
     * between neighbours and the plain mean of 1/r misses 1/r at the
     * interface by O(1) (0.75 against 0.67 of 1/dr between rings 1 and 2);
     * the weighted mean gives 1/r there exactly on uniform radial spacing. */
    for (int t = 0; t < 3; ++t)
      for (int cc = 0; cc < 3; ++cc) {
        double sa = S->M[(3 * t + cc) * N + a], sb = S->M[(3 * t + cc) * N + b];
        if (Ja != 0.0) sa *= Ja;
        if (Jb != 0.0) sb *= Jb;
        mh[t][cc] = (sa + sb) / (Ja + Jb);
      }
  }
  double gr[4][3]; /* gr[q][c] = d phi_q / d x_c */
  for (int q = 0; q < 4; ++q)
    for (int cc = 0; cc < 3; ++cc)
      gr[q][cc] = mh[0][cc] * dphi[q][0] + mh[1][cc] * dphi[q][1] +
                  mh[2][cc] * dphi[q][2];
  double mu = 0.5 * (S->MK[a] + S->MK[b]);
  double kap = 0.5 * (S->MK[N + a] + S->MK[N + b]);
  double div = gr[0][0] + gr[1][1] + gr[2][2];
  double txx = mu * (2.0 * gr[0][0] - (2.0 / 3.0) * div);
  double tyy = mu * (2.0 * gr[1][1] - (2.0 / 3.0) * div);
  double tzz = mu * (2.0 * gr[2][2] - (2.0 / 3.0) * div);
  if (S->P->sgs_model == 3) {
    /* the modelled isotropic SGS stress sigma_ll/3 delta_ij (Eq. yoshizawa)
     * is subtracted from the resolved stress, at the interface mean */
    double iso = 0.5 * (S->MK[2 * N + a] + S->MK[2 * N + b]) / 3.0;
    txx -= iso;
    tyy -= iso;
    tzz -= iso;
  }
  double txy = mu * (gr[0][1] + gr[1][0]);
  double txz = mu * (gr[0][2] + gr[2][0]);
  double tyz = mu * (gr[1][2] + gr[2][1]);
  double uf = 0.5 * (S->u[a] + S->u[b]);
  double vf = 0.5 * (S->v[a] + S->v[b]);
  double wf = 0.5 * (S->w[a] + S->w[b]);
  double qx = -kap * gr[3][0], qy = -kap * gr[3][1], qz = -kap * gr[3][2];
  double bx = txx * uf + txy * vf + txz * wf - qx;
  double by = txy * uf + tyy * vf + tyz * wf - qy;
  double bz = txz * uf + tyz * vf + tzz * wf - qz;
  double mx = mh[d][0], my = mh[d][1], mz = mh[d][2];
  double Fv[5];
  Fv[0] = 0.0;
  Fv[1] = Jh * (mx * txx + my * txy + mz * txz);
  Fv[2] = Jh * (mx * txy + my * tyy + mz * tyz);
  Fv[3] = Jh * (mx * txz + my * tyz + mz * tzz);
  Fv[4] = Jh * (mx * bx + my * by + mz * bz);

  for (int q = 0; q < 5; ++q) F[q] = Fe[q] - Fv[q];
}

void orc_interface_flux(const orc_params *P, int ni, int nj, int nk,
                        const double *Q, const double *M, const double *MK,
                        int d, int i, int j, int k, double F[5]) {
  state_t S;
  state_build(&S, P, ni, nj, nk, Q, M, MK);
  int c[3] = {i, j, k};
  interface_flux(&S, d, c, F);
  state_free(&S);
}

/* RHS_{i,j,k} = sum over directions of (F_{+1/2} - F_{-1/2}) with unit
 * computational spacing (Eq. spatial_discret and the RHS definition below
 * it); F = inviscid-with-dissipation minus viscous.  Each interface is a pure
 * function of the state, so the two nodes sharing it see the same value and
 * the sum telescopes.  Boundary nodes of non-periodic directions get 0. */
void orc_rhs(const orc_params *P, int ni, int nj, int nk, const double *Q,
             const double *M, const double *MK, double *R) {
  state_t S;
  state_build(&S, P, ni, nj, nk, Q, M, MK);
  size_t N = S.g.N;
#pragma omp parallel for schedule(static)
  for (long n = 0; n < (long)N; ++n) {
    int c[3];
    unlin(&S.g, (size_t)n, c);
    if (!is_interior(&S.g, c)) {
      for (int q = 0; q < 5; ++q) R[(size_t)q * N + n] = 0.0;
      continue;
    }
    double acc[5] = {0, 0, 0, 0, 0};
    for (int d = 0; d < 3; ++d) {
      double Fp[5], Fm[5];
      int cm[3] = {c[0], c[1], c[2]};
      cm[d] = (c[d] - 1 + S.g.n[d]) % S.g.n[d];
      interface_flux(&S, d, c, Fp);
      interface_flux(&S, d, cm, Fm);
      for (int q = 0; q < 5; ++q) acc[q] += Fp[q] - Fm[q];
    }
    for (int q = 0; q < 5; ++q) R[(size_t)q * N + n] = acc[q];
  }
  state_free(&S);
}

/* ------------------------------------------------------------- time step */

/* Reading A18: global time-accurate step dt = CFL * min over all nodes of
 * 1 / (lambda_xi + lambda_eta + lambda_zeta); dt_mode 1 uses dt_fixed. */
double orc_dt(const orc_params *P, int ni, int nj, int nk, const double *Q,
              const double *M) {
  if (P->dt_mode == 1) return P->dt_fixed;
  state_t S;
  memset(&S, 0, sizeof(S));
  S.P = P;
  S.g = make_grid(ni, nj, nk, P->periodic);
  S.Q = Q; S.M = M;
  state_alloc(&S);
  node_primitives(&S);
  node_radii(&S);
  double best = INFINITY;
  for (size_t n = 0; n < S.g.N; ++n) {
    double v = 1.0 / (S.lam[0][n] + S.lam[1][n] + S.lam[2][n]);
    if (v < best) best = v;
  }
  state_free(&S);
  return P->cfl * best;
}

/* Local time stepping, the literal form of Eq. localdt: each node n advances
 * with its own step, the CFL limit of that node alone,
 * dtn[n] = cfl / (lam_xi + lam_eta + lam_zeta)(n). */
void orc_dt_local(const orc_params *P, int ni, int nj, int nk, const double *Q,
                  const double *M, double *dtn) {
  state_t S;
  memset(&S, 0, sizeof(S));
  S.P = P;
  S.g = make_grid(ni, nj, nk, P->periodic);
  S.Q = Q; S.M = M;
  state_alloc(&S);
  node_primitives(&S);
  node_radii(&S);
  for (size_t n = 0; n < S.g.N; ++n)
    dtn[n] = P->cfl / (S.lam[0][n] + S.lam[1][n] + S.lam[2][n]);
  state_free(&S);
}

/* ---------------------------------------------------------- jet boundary */

static void cons_from(double gam, double rho, double u, double v, double w,
                      double p, double q[5]) {
  q[0] = rho; q[1] = rho * u; q[2] = rho * v; q[3] = rho * w;
  q[4] = p / (gam - 1.0) + 0.5 * rho * (u * u + v * v + w * w);
}

static void prim_of(double gam, const double *Q, size_t N, long n,
                    double *rho, double *u, double *v, double *w, double *p) {
  *rho = Q[n];
  *u = Q[N + n] / *rho; *v = Q[2 * N + n] / *rho; *w = Q[3 * N + n] / *rho;
  *p = (gam - 1.0) * (Q[4 * N + n] - 0.5 * *rho * (*u * *u + *v * *v + *w * *w));
}

/* Riemann-invariant far-field state (Sec. "Far Field Boundary", Reading
 * A13) of a boundary node whose adjacent interior node holds (rho, u, v, w,
 * p), for the unit outward normal (nx, ny, nz) and the free stream at rest
 * (rho = 1, p = 1/gamma, a = 1): R+ = q_n,e + 2 a_e/(gamma-1) from the
 * interior, R- = q_n,inf - 2 a_inf/(gamma-1) from the free stream, and the
 * four branches chosen by q_n,e/a_e (0 counts as exit).  Returns 1 for the
 * supersonic exit, where the caller copies the interior node's conserved
 * values (q is then left unset), else 0 with the state in q. */
static int riemann_far_field(double gam, double rho, double u, double v,
                             double w, double p, double nx, double ny,
                             double nz, double q[5]) {
  double gm1 = gam - 1.0;
  const double rho_inf = 1.0, p_inf = 1.0 / gam, a_inf = 1.0;
  double a_e = sqrt(gam * p / rho);
  double qne = u * nx + v * ny + w * nz;
  double qninf = 0.0;
  double Rp = qne + 2.0 * a_e / gm1;
  double Rm = qninf - 2.0 * a_inf / gm1;
  double qnf = 0.5 * (Rp + Rm);
  double af = 0.25 * gm1 * (Rp - Rm);
  double Mn = qne / a_e;
  if (Mn >= 1.0) {
    return 1;
  } else if (Mn >= 0.0) {
    double uf = u + (qnf - qne) * nx, vf = v + (qnf - qne) * ny,
           wf = w + (qnf - qne) * nz;
    double rf = pow(pow(rho, gam) * af * af / (gam * p), 1.0 / gm1);
    double pf = rf * af * af / gam;
    cons_from(gam, rf, uf, vf, wf, pf, q);
  } else if (Mn > -1.0) {
    double uf = 0.0 + (qnf - qninf) * nx, vf = 0.0 + (qnf - qninf) * ny,
           wf = 0.0 + (qnf - qninf) * nz;
    double rf = pow(pow(rho_inf, gam) * af * af / (gam * p_inf), 1.0 / gm1);
    double pf = rf * af * af / gam;
    cons_from(gam, rf, uf, vf, wf, pf, q);
  } else {
    cons_from(gam, rho_inf, 0.0, 0.0, 0.0, p_inf, q);
  }
  return 0;
}

/* Jet boundary conditions applied after the fifth stage.  The free stream is
 * at rest with rho = 1, p = 1/gamma, a = 1.  Phase 1 reads only the state
 * left by the stages:
 *  - entrance i = 0.  bc = 1 (Reading A14): Dirichlet jet profile plus
 *    forcing, u = u(r) + sum_{m,f} a_{mf} g(r) cos(m theta - 2 pi St_f U_j
 *    t), g(r) = exp(-((r - r_jet)/w)^2), v = w = 0, rho = 1, p = 1/gamma
 *    (the paper's supersonic-entrance rule applied over the whole plane).
 *    bc = 2 (Sec. "Entrance Boundary", Reading A25): the plane is split at
 *    r = r_jet.  Above the jet, the far-field rule with the unit outward
 *    normal -grad(xi)/|grad(xi)| and the adjacent node (1, j, k).  In the jet
 *    area, a supersonic jet (Mj >= 1) gets the Dirichlet jet state as for
 *    bc = 1; a subsonic one the 1-D characteristic relations: u = the target
 *    u(r) plus forcing, v, w copied from (1, j, k), T = T_t/(1 + (gamma-1)
 *    |u|^2/2) with T_t = 1 + (gamma-1) Mj^2/2, p = T^(gamma/(gamma-1))/gamma,
 *    rho = gamma p/T;
 *  - far field j = nj-1, 0 < i < ni-1 (Sec. "Far Field Boundary", Reading
 *    A13): R- = q_n,inf - 2 a_inf/(gamma-1), R+ = q_n,e + 2 a_e/(gamma-1)
 *    (the printed R+ sign cannot give the printed a_f), unit normal
 *    grad(eta)/|grad(eta)|, the four sub/supersonic entrance/exit branches
 *    chosen by q_n,e/a_e (0 counts as exit);
 *  - inner ring j = 0, 0 < i < ni-1 (Reading A15, centerline rule of Sec.
 *    "Centerline Boundary Condition"): Q(i,0,k) = mean over k of Q(i,1,k),
 *    summed in increasing k.
 * Phase 2, exit i = ni-1 (Sec. "Exit Boundary Condition"), from the column
 * i = ni-2 after phase 1: supersonic (q/a >= 1 along grad(xi)) copies it;
 * subsonic takes p = p_inf and zero-order extrapolates u and the internal
 * energy p/((gamma-1) rho). */
void orc_bc_jet(const orc_params *P, int ni, int nj, int nk, double *Q,
                const double *M, const double *xyz, double t) {
  size_t N = (size_t)ni * nj * nk;
  double gam = P->gamma, gm1 = gam - 1.0;
  const double p_inf = 1.0 / gam;
  const double two_pi = 6.283185307179586476925286766559;
  double *Qs = (double *)malloc(5 * N * sizeof(double));
  memcpy(Qs, Q, 5 * N * sizeof(double));
#define ID(i, j, k) (((size_t)(i) * nj + (j)) * nk + (k))
  /* entrance */
  for (int j = 0; j < nj; ++j)
    for (int k = 0; k < nk; ++k) {
      size_t n = ID(0, j, k);
      double y = xyz[N + n], z = xyz[2 * N + n];
      double r = sqrt(y * y + z * z), th = atan2(z, y);
      double u = jet_profile(P, r);
      double gr = exp(-((r - P->r_jet) / P->force_width) *
                      ((r - P->r_jet) / P->force_width));
      for (int m = 0; m < 4; ++m)
        for (int f = 0; f < 4; ++f)
          u += P->amp[m * 4 + f] * gr *
               cos(m * th - two_pi * P->St[f] * P->Mj * t);
      double q[5];
      if (P->bc == 2 && r > P->r_jet) {
        size_t ne = ID(1, j, k);
        double ex = M[0 * N + n], ey = M[1 * N + n], ez = M[2 * N + n];
        double inv = 1.0 / sqrt(ex * ex + ey * ey + ez * ez);
        double rho, ue, ve, we, p;
        prim_of(gam, Qs, N, (long)ne, &rho, &ue, &ve, &we, &p);
        if (riemann_far_field(gam, rho, ue, ve, we, p, -ex * inv, -ey * inv,
                              -ez * inv, q))
          for (int c = 0; c < 5; ++c) q[c] = Qs[c * N + ne];
      } else if (P->bc == 2 && P->Mj < 1.0) {
        double rho, ue, ve, we, p;
        prim_of(gam, Qs, N, (long)ID(1, j, k), &rho, &ue, &ve, &we, &p);
        double Tt = 1.0 + 0.5 * gm1 * P->Mj * P->Mj;
        double T = Tt / (1.0 + 0.5 * gm1 * (u * u + ve * ve + we * we));
        double pf = pow(T, gam / gm1) / gam;
        cons_from(gam, gam * pf / T, u, ve, we, pf, q);
      } else {
        cons_from(gam, 1.0, u, 0.0, 0.0, p_inf, q);
      }
      for (int c = 0; c < 5; ++c) Q[c * N + n] = q[c];
    }
  /* far field */
  for (int i = 1; i < ni - 1; ++i)
    for (int k = 0; k < nk; ++k) {
      size_t nf = ID(i, nj - 1, k), ne = ID(i, nj - 2, k);
      double ex = M[3 * N + nf], ey = M[4 * N + nf], ez = M[5 * N + nf];
      double inv = 1.0 / sqrt(ex * ex + ey * ey + ez * ez);
      double rho, u, v, w, p;
      prim_of(gam, Qs, N, (long)ne, &rho, &u, &v, &w, &p);
      double q[5];
      if (riemann_far_field(gam, rho, u, v, w, p, ex * inv, ey * inv, ez * inv, q))
        for (int c = 0; c < 5; ++c) q[c] = Qs[c * N + ne];
      for (int c = 0; c < 5; ++c) Q[c * N + nf] = q[c];
    }
  /* inner ring */
  for (int i = 1; i < ni - 1; ++i)
    for (int c = 0; c < 5; ++c) {
      double s = 0.0;
      for (int k = 0; k < nk; ++k) s += Qs[c * N + ID(i, 1, k)];
      double mean = s / (double)nk;
      for (int k = 0; k < nk; ++k) Q[c * N + ID(i, 0, k)] = mean;
    }
  /* exit (phase 2, reads the updated column ni-2) */
  for (int j = 0; j < nj; ++j)
    for (int k = 0; k < nk; ++k) {
      size_t nx_ = ID(ni - 1, j, k), ne = ID(ni - 2, j, k);
      /* an axis node (J^-1 = 0) has a zero xi row: it takes the outward
       * normal of its neighbour (ni-1, 1, k) (Reading A27) */
      size_t nm = (M[9 * N + nx_] == 0.0) ? ID(ni - 1, 1, k) : nx_;
      double ex = M[0 * N + nm], ey = M[1 * N + nm], ez = M[2 * N + nm];
      double inv = 1.0 / sqrt(ex * ex + ey * ey + ez * ez);
      double rho, u, v, w, p;
      prim_of(gam, Q, N, (long)ne, &rho, &u, &v, &w, &p);
      double a_e = sqrt(gam * p / rho);
      double qn = (u * ex + v * ey + w * ez) * inv;
      double q[5];
      if (qn / a_e >= 1.0) {
        for (int c = 0; c < 5; ++c) q[c] = Q[c * N + ne];
      } else {
        double e_int = p / (gm1 * rho);
        double rf = p_inf / (gm1 * e_int);
        q[0] = rf; q[1] = rf * u; q[2] = rf * v; q[3] = rf * w;
        q[4] = rf * (e_int + 0.5 * (u * u + v * v + w * w));
      }
      for (int c = 0; c < 5; ++c) Q[c * N + nx_] = q[c];
    }
#undef ID
  free(Qs);
}

/* ------------------------------------------------------------ time march */

/* Five-stage scheme of Eq. localdt with the recommended coefficients
 * alpha = 1/4, 1/6, 3/8, 1/2, 1: Q^(0) = Q^n, Q^(l) = Q^(0) - alpha_l dt
 * RHS^(l-1) (the paper's Q is J^-1-scaled; for the stored unscaled Q the
 * update carries J = 1/J^-1), Q^(n+1) = Q^(5). */
void orc_rk5(int ncomp, size_t N, double *Q, const unsigned char *update,
             const double *Jinv, double dt, const double *dtn, orc_rhs_fn rhs,
             void *user) {
  static const double alpha[5] = {1.0 / 4.0, 1.0 / 6.0, 3.0 / 8.0, 1.0 / 2.0,
                                  1.0};
  size_t tot = (size_t)ncomp * N;
  double *Q0 = (double *)malloc(tot * sizeof(double));
  double *R = (double *)malloc(tot * sizeof(double));
  memcpy(Q0, Q, tot * sizeof(double));
  for (int l = 0; l < 5; ++l) {
    rhs(user, Q, R); /* RHS of the previous stage's state */
    for (int c = 0; c < ncomp; ++c)
      for (size_t n = 0; n < N; ++n) {
        size_t idx = (size_t)c * N + n;
        if (update && !update[n]) {
          Q[idx] = Q0[idx];
        } else {
          double Jn = Jinv ? 1.0 / Jinv[n] : 1.0;
          double h = dtn ? dtn[n] : dt;
          Q[idx] = Q0[idx] - alpha[l] * h * (Jn * R[idx]);
        }
      }
  }
  free(Q0);
  free(R);
}

typedef struct {
  const orc_params *P;
  int ni, nj, nk;
  const double *M;
  double *MK;
} flow_user_t;

static void flow_rhs(void *user, const double *Qs, double *R) {
  flow_user_t *U = (flow_user_t *)user;
  /* Reading A17: viscosity held at its Q^n value through the stages unless
   * freeze_visc = 0, in which case it follows every stage state. */
  if (!U->P->freeze_visc)
    orc_mu_eff(U->P, U->ni, U->nj, U->nk, Qs, U->M, U->MK);
  orc_rhs(U->P, U->ni, U->nj, U->nk, Qs, U->M, U->MK, R);
}

/* One iteration of the solver loop (Table tab:JAZzY): viscosity from Q^n,
 * time step, five stages, then the boundary conditions at t + dt. */
double orc_rk_step(const orc_params *P, int ni, int nj, int nk, double *Q,
                   const double *M, const double *xyz, double t) {
  grid_t g = make_grid(ni, nj, nk, P->periodic);
  size_t N = g.N;
  double *MK = (double *)malloc(3 * N * sizeof(double));
  unsigned char *upd = (unsigned char *)malloc(N);
  for (size_t n = 0; n < N; ++n) {
    int c[3];
    unlin(&g, n, c);
    upd[n] = (unsigned char)is_interior(&g, c);
  }
  orc_mu_eff(P, ni, nj, nk, Q, M, MK);
  double dt = orc_dt(P, ni, nj, nk, Q, M);
  /* Reading: with local steps the clock (and so the inflow forcing phase)
   * advances by the smallest local step, the global CFL step */
  double *dtn = NULL;
  if (P->dt_mode == 2) {
    dtn = (double *)malloc(N * sizeof(double));
    orc_dt_local(P, ni, nj, nk, Q, M, dtn);
  }
  flow_user_t U = {P, ni, nj, nk, M, MK};
  orc_rk5(5, N, Q, upd, M + 9 * N, dt, dtn, flow_rhs, &U);
  if (P->bc == 1 || P->bc == 2) orc_bc_jet(P, ni, nj, nk, Q, M, xyz, t + dt);
  free(dtn);
  free(MK);
  free(upd);
  return dt;
}

/* Far-field functional of the adjoint window (scope-table row a11; the
 * paper has none): w times the sum over the ring j = js of
 * (p - p_inf)^2 dA, with p_inf = 1/gamma (the free stream at rest), p from
 * System I (Sec. "Large Eddy Simulation Filtering") and dA = J^-1 |grad eta|
 * the area of the node's eta face (Sec. "Transformation of Coordinates":
 * J^-1 grad eta is the cross product of the xi and zeta tangents).  Summed
 * in increasing (i, k). */
double orc_surface_functional(const orc_params *P, int ni, int nj, int nk,
                              const double *Q, const double *M, int js,
                              double w) {
  size_t N = (size_t)ni * nj * nk;
  double gam = P->gamma, s = 0.0;
  for (int i = 0; i < ni; ++i) {
    for (int k = 0; k < nk; ++k) {
      long n = (long)(((size_t)i * nj + js) * nk + k);
      double rho, u, v, wv, p;
      prim_of(gam, Q, N, n, &rho, &u, &v, &wv, &p);
      double ex = M[3 * N + n], ey = M[4 * N + n], ez = M[5 * N + n];
      double dA = M[9 * N + n] * sqrt(ex * ex + ey * ey + ez * ez);
      double dp = p - 1.0 / gam;
      s += dp * dp * dA;
    }
  }
  return w * s;
}

void orc_totals(int ni, int nj, int nk, const double *Q, const double *M,
                double out[5]) {
  size_t N = (size_t)ni * nj * nk;
  for (int c = 0; c < 5; ++c) {
    double s = 0.0;
    for (size_t n = 0; n < N; ++n) s += M[9 * N + n] * Q[(size_t)c * N + n];
    out[c] = s;
  }
}
