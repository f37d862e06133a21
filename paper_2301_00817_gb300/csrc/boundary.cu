// boundary.cu -- jet boundary conditions (Sec. "Boundary Conditions"),
// conserved totals and time bookkeeping.  All arithmetic FP64; the metrics
// are read as FP64, or from the FP32 copy in the compact mixed form.
#include "lesjet_dev.cuh"
#include "lesjet_host.h"

namespace lesjet {

// State accessors: plain FP64 state, or the mixed form's unevaluated float
// pair hi + lo (read and written in FP64 here, surface nodes only).
struct AccD {
  double* q;
  __device__ __forceinline__ double ld(long long i) const { return q[i]; }
  __device__ __forceinline__ void st(long long i, double v) const { q[i] = v; }
};
struct AccHL {
  float* hi;
  float* lo;
  __device__ __forceinline__ double ld(long long i) const { return (double)hi[i] + (double)lo[i]; }
  __device__ __forceinline__ void st(long long i, double v) const {
    const float h = (float)v;
    hi[i] = h;
    lo[i] = (float)(v - (double)h);
  }
};

struct JetBC {
  int mode;     // LES_BC_JET or LES_BC_JET_CHAR
  int forced;   // some forcing amplitude is non-zero
  double gamma, Mj, r_jet, theta_m, force_width;
  double St[4];
  double amp[16];
};

template <class Acc>
__device__ __forceinline__ void store_prim(const Acc& Q, long long N, long long n, double gamma,
                                           double rho, double u, double v, double w, double p) {
  Q.st(n, rho);
  Q.st(N + n, rho * u);
  Q.st(2 * N + n, rho * v);
  Q.st(3 * N + n, rho * w);
  Q.st(4 * N + n, p / (gamma - 1.0) + 0.5 * rho * (u * u + v * v + w * w));
}

template <class Acc>
__device__ __forceinline__ void load_prim(const Acc& Q, long long N, long long n, double gamma,
                                          double& rho, double& u, double& v, double& w,
                                          double& p) {
  rho = Q.ld(n);
  u = Q.ld(N + n) / rho;
  v = Q.ld(2 * N + n) / rho;
  w = Q.ld(3 * N + n) / rho;
  p = (gamma - 1.0) * (Q.ld(4 * N + n) - 0.5 * rho * (u * u + v * v + w * w));
}

// Riemann-invariant state of a far-field node from its interior neighbour's
// primitives and the unit outward normal, the free stream at rest (rho = 1,
// p = 1/gamma, a = 1): R+ = q_n,e + 2 a_e/(gamma-1), R- = -2/(gamma-1), four
// branches by q_n,e/a_e.  Returns true for the supersonic exit (the caller
// copies the neighbour's conserved values); otherwise the primitives of the
// boundary state are in f = (rho, u, v, w, p).
// x^(2/(gamma-1)).  When 2/(gamma-1) is an integer up to 8 (gamma = 1.4: 5;
// gamma = 5/3: 3) the power is taken by repeated multiplication: it differs
// from pow(x, 2/(gamma-1)) only by the rounding of the computed exponent
// (about 1e-16 relative for x near 1), at a small fraction of FP64 pow's
// cost on a GPU whose FP64 rate is 1/64 of its FP32 rate.
__device__ __forceinline__ double pow_entropy(double x, double e) {
  const double n = rint(e);
  if (fabs(e - n) < 1e-12 && n >= 1.0 && n <= 8.0) {
    double r = x;
    for (int i = 1; i < (int)n; ++i) r *= x;
    return r;
  }
  return pow(x, e);
}

__device__ __forceinline__ bool far_field_state(double gamma, double rho, double u, double v,
                                                double w, double p, double nx, double ny,
                                                double nz, double f[5]) {
  const double gm1 = gamma - 1.0;
  const double ae = sqrt(gamma * p / rho);
  const double qne = u * nx + v * ny + w * nz;
  const double Rp = qne + 2.0 * ae / gm1;
  const double Rm = 0.0 - 2.0 * 1.0 / gm1;
  const double qnf = 0.5 * (Rp + Rm);
  const double af = 0.25 * gm1 * (Rp - Rm);
  const double Mn = qne / ae;
  if (Mn >= 1.0) return true;
  if (Mn >= 0.0) {
    // entropy of the interior node: rho_f = (rho_e^gamma a_f^2/(gamma p_e))^(1/(gamma-1))
    // = rho_e (a_f/a_e)^(2/(gamma-1)), one power instead of two
    const double dq = qnf - qne;
    const double rf = rho * pow_entropy(af / ae, 2.0 / gm1);
    f[0] = rf;
    f[1] = u + dq * nx;
    f[2] = v + dq * ny;
    f[3] = w + dq * nz;
    f[4] = rf * af * af / gamma;
  } else if (Mn > -1.0) {
    // free-stream entropy (rho = 1, p = 1/gamma): rho_f = a_f^(2/(gamma-1))
    const double rf = pow_entropy(af, 2.0 / gm1);
    f[0] = rf;
    f[1] = qnf * nx;
    f[2] = qnf * ny;
    f[3] = qnf * nz;
    f[4] = rf * af * af / gamma;
  } else {
    f[0] = 1.0;
    f[1] = f[2] = f[3] = 0.0;
    f[4] = 1.0 / gamma;
  }
  return false;
}

// Entrance i = 0.  The target axial velocity is the jet profile plus the
// 16-mode forcing sum a_{mf} g(r) cos(m theta - 2 pi St_f Mj t).
// LES_BC_JET: rho = 1, p = 1/gamma, v = w = 0, u = target on the whole plane.
// LES_BC_JET_CHAR (Sec. "Entrance Boundary"): above r_jet the far-field rule
// with the outward normal -grad(xi)/|grad(xi)| and the node (1, j, k); in the
// jet area the same jet state when Mj >= 1, else the 1-D characteristic
// relations (u = target, v and w from (1, j, k), T = T_t/(1 + (gamma-1)
// |u|^2/2) with the jet's T_t = 1 + (gamma-1) Mj^2/2, p = T^(gamma/(gamma-1))
// /gamma).  The plane i = 1 is read before any other boundary kernel runs.
// (blk, nblk: this block's index among the nblk blocks given to the part)
template <class Acc, typename TM>
__device__ __forceinline__ void bc_inflow_part(const Grid& g, const JetBC& b,
                                               const double* __restrict__ rth,
                                               const TM* __restrict__ M,
                                               const DevScalars* __restrict__ sc, int use_host_t,
                                               double t_host, const Acc& Q, int blk, int nblk) {
  const long long plane = (long long)g.n[1] * g.n[2];
  const long long N = g.N;
  const double t = use_host_t ? t_host : sc->t;
  const double two_pi = 6.283185307179586476925286766559;
  for (long long n = blk * (long long)blockDim.x + threadIdx.x; n < plane;
       n += (long long)nblk * blockDim.x) {
    const double r = rth[n], th = rth[plane + n];
    double u = 0.5 * b.Mj * (1.0 + tanh((b.r_jet - r) / (2.0 * b.theta_m)));
    if (b.forced) {
      // cos(m theta - phi_f) = cos(m theta) cos(phi_f) + sin(m theta) sin(phi_f),
      // with cos/sin(m theta) by the angle-addition recurrence from theta
      const double x = (r - b.r_jet) / b.force_width;
      const double gr = exp(-(x * x));
      double s1, c1;
      sincos(th, &s1, &c1);
      double cm[4] = {1.0, c1, 0.0, 0.0}, sm[4] = {0.0, s1, 0.0, 0.0};
#pragma unroll
      for (int m = 2; m < 4; ++m) {
        cm[m] = cm[m - 1] * c1 - sm[m - 1] * s1;
        sm[m] = sm[m - 1] * c1 + cm[m - 1] * s1;
      }
      double sf[4], cf[4];
#pragma unroll
      for (int f = 0; f < 4; ++f) sincos(two_pi * b.St[f] * b.Mj * t, &sf[f], &cf[f]);
      double acc = 0.0;
#pragma unroll
      for (int m = 0; m < 4; ++m)
#pragma unroll
        for (int f = 0; f < 4; ++f) acc += b.amp[m * 4 + f] * (cm[m] * cf[f] + sm[m] * sf[f]);
      u += gr * acc;
    }
    const long long ne = n + plane;  // node (1, j, k)
    if (b.mode == LES_BC_JET_CHAR && r > b.r_jet) {
      const double ex = (double)M[n], ey = (double)M[N + n], ez = (double)M[2 * N + n];
      const double inv = 1.0 / sqrt(ex * ex + ey * ey + ez * ez);
      double rho, ue, ve, we, p, f[5];
      load_prim(Q, N, ne, b.gamma, rho, ue, ve, we, p);
      if (far_field_state(b.gamma, rho, ue, ve, we, p, -ex * inv, -ey * inv, -ez * inv, f)) {
#pragma unroll
        for (int q = 0; q < 5; ++q) Q.st(q * N + n, Q.ld(q * N + ne));
      } else {
        store_prim(Q, N, n, b.gamma, f[0], f[1], f[2], f[3], f[4]);
      }
    } else if (b.mode == LES_BC_JET_CHAR && b.Mj < 1.0) {
      const double gm1 = b.gamma - 1.0;
      double rho, ue, ve, we, p;
      load_prim(Q, N, ne, b.gamma, rho, ue, ve, we, p);
      const double Tt = 1.0 + 0.5 * gm1 * b.Mj * b.Mj;
      const double T = Tt / (1.0 + 0.5 * gm1 * (u * u + ve * ve + we * we));
      const double pf = pow(T, b.gamma / gm1) / b.gamma;
      store_prim(Q, N, n, b.gamma, b.gamma * pf / T, u, ve, we, pf);
    } else {
      store_prim(Q, N, n, b.gamma, 1.0, u, 0.0, 0.0, 1.0 / b.gamma);
    }
  }
}

template <class Acc, typename TM>
__global__ void k_bc_inflow(Grid g, JetBC b, const double* __restrict__ rth,
                            const TM* __restrict__ M, const DevScalars* __restrict__ sc,
                            int use_host_t, double t_host, Acc Q) {
  bc_inflow_part(g, b, rth, M, sc, use_host_t, t_host, Q, blockIdx.x, gridDim.x);
}

// Far field j = nj-1 (0 < i < ni-1): Riemann invariants along the unit
// eta-normal with R+ from the adjacent interior node and R- from the free
// stream at rest (rho = 1, p = 1/gamma, a = 1); four branches by q_n/a.
template <class Acc, typename TM>
__device__ __forceinline__ void bc_farfield_part(const Grid& g, double gamma,
                                                 const TM* __restrict__ M, const Acc& Q, int blk,
                                                 int nblk) {
  const int ni = g.n[0], nj = g.n[1], nk = g.n[2];
  const long long count = (long long)(ni - 2) * nk;
  const long long N = g.N;
  for (long long e = blk * (long long)blockDim.x + threadIdx.x; e < count;
       e += (long long)nblk * blockDim.x) {
    const int i = 1 + (int)(e / nk), k = (int)(e % nk);
    const long long nf = idx3(g, i, nj - 1, k), ne = idx3(g, i, nj - 2, k);
    const double ex = (double)M[3 * N + nf], ey = (double)M[4 * N + nf], ez = (double)M[5 * N + nf];
    const double inv = 1.0 / sqrt(ex * ex + ey * ey + ez * ez);
    double rho, u, v, w, p, f[5];
    load_prim(Q, N, ne, gamma, rho, u, v, w, p);
    if (far_field_state(gamma, rho, u, v, w, p, ex * inv, ey * inv, ez * inv, f)) {
#pragma unroll
      for (int q = 0; q < 5; ++q) Q.st(q * N + nf, Q.ld(q * N + ne));
    } else {
      store_prim(Q, N, nf, gamma, f[0], f[1], f[2], f[3], f[4]);
    }
  }
}

template <class Acc, typename TM>
__global__ void k_bc_farfield(Grid g, double gamma, const TM* __restrict__ M, Acc Q) {
  bc_farfield_part(g, gamma, M, Q, blockIdx.x, gridDim.x);
}

// Inner ring j = 0 (0 < i < ni-1): azimuthal mean of the first interior
// ring, one block per axial station, fixed-order tree (deterministic).
template <class Acc>
__device__ __forceinline__ void bc_ring_part(const Grid& g, const Acc& Q, int blk) {
  const int i = 1 + blk;
  const int nk = g.n[2];
  const long long N = g.N;
  __shared__ double red[5][32];
  double s[5] = {0, 0, 0, 0, 0};
  const long long base1 = idx3(g, i, 1, 0), base0 = idx3(g, i, 0, 0);
  for (int k = threadIdx.x; k < nk; k += blockDim.x)
#pragma unroll
    for (int q = 0; q < 5; ++q) s[q] += Q.ld(q * N + base1 + k);
#pragma unroll
  for (int q = 0; q < 5; ++q)
    for (int off = 16; off > 0; off >>= 1) s[q] += __shfl_xor_sync(0xffffffffu, s[q], off);
  if ((threadIdx.x & 31) == 0)
#pragma unroll
    for (int q = 0; q < 5; ++q) red[q][threadIdx.x >> 5] = s[q];
  __syncthreads();
  if (threadIdx.x < 32) {
#pragma unroll
    for (int q = 0; q < 5; ++q) {
      double v = threadIdx.x < (blockDim.x >> 5) ? red[q][threadIdx.x] : 0.0;
      for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
      if (threadIdx.x == 0) red[q][0] = v / (double)nk;
    }
  }
  __syncthreads();
  for (int k = threadIdx.x; k < nk; k += blockDim.x)
#pragma unroll
    for (int q = 0; q < 5; ++q) Q.st(q * N + base0 + k, red[q][0]);
}

template <class Acc>
__global__ void k_bc_ring(Grid g, Acc Q) {
  bc_ring_part(g, Q, blockIdx.x);
}

// The Dirichlet entrance, the far field and the inner ring in one launch
// (blocks [0, nb_ff) the far field, then nb_in for the entrance, then one per
// axial station for the ring).  They write disjoint surfaces (i = 0; j = nj-1
// and j = 0 for 0 < i < ni-1) and read nothing another writes: the far field
// reads j = nj-2 and the ring j = 1 (distinct for nj >= 3), and the
// Dirichlet entrance reads no state.
template <class Acc, typename TM>
__global__ void k_bc_sides(Grid g, JetBC b, const double* __restrict__ rth,
                           const TM* __restrict__ M, const DevScalars* __restrict__ sc,
                           int use_host_t, double t_host, Acc Q, int nb_ff, int nb_in) {
  const int blk = blockIdx.x;
  if (blk < nb_ff)
    bc_farfield_part(g, b.gamma, M, Q, blk, nb_ff);
  else if (blk < nb_ff + nb_in)
    bc_inflow_part(g, b, rth, M, sc, use_host_t, t_host, Q, blk - nb_ff, nb_in);
  else
    bc_ring_part(g, Q, blk - nb_ff - nb_in);
}

// Exit i = ni-1 from the updated column i = ni-2: supersonic (q/a >= 1 along
// the unit xi-normal) copies; subsonic takes p = 1/gamma and extrapolates the
// velocity and the internal energy p/((gamma-1) rho).
template <class Acc, typename TM>
__global__ void k_bc_exit(Grid g, double gamma, const TM* __restrict__ M, Acc Q) {
  const int ni = g.n[0];
  const long long plane = (long long)g.n[1] * g.n[2];
  const long long N = g.N;
  const double gm1 = gamma - 1.0;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < plane;
       e += (long long)gridDim.x * blockDim.x) {
    const long long nx_ = (long long)(ni - 1) * plane + e, ne = nx_ - plane;
    // an axis node (J^-1 = 0, ring j = 0) has a zero xi row: it takes the
    // outward normal of (ni-1, 1, k) (Reading A27)
    const long long nm = (e < g.n[2] && (double)M[9 * N + nx_] == 0.0) ? nx_ + g.n[2] : nx_;
    const double ex = (double)M[nm], ey = (double)M[N + nm], ez = (double)M[2 * N + nm];
    const double inv = 1.0 / sqrt(ex * ex + ey * ey + ez * ez);
    double rho, u, v, w, p;
    load_prim(Q, N, ne, gamma, rho, u, v, w, p);
    const double ae = sqrt(gamma * p / rho);
    const double qn = (u * ex + v * ey + w * ez) * inv;
    if (qn / ae >= 1.0) {
#pragma unroll
      for (int q = 0; q < 5; ++q) Q.st(q * N + nx_, Q.ld(q * N + ne));
    } else {
      const double eint = p / (gm1 * rho);
      const double rf = (1.0 / gamma) / (gm1 * eint);
      Q.st(nx_, rf);
      Q.st(N + nx_, rf * u);
      Q.st(2 * N + nx_, rf * v);
      Q.st(3 * N + nx_, rf * w);
      Q.st(4 * N + nx_, rf * (eint + 0.5 * (u * u + v * v + w * w)));
    }
  }
}

// Read-only state views for the totals: FP64, or the float pair hi + lo
// (the value the join writes, so both give the same totals).
struct ViewD {
  const double* q;
  __device__ __forceinline__ double ld(long long i) const { return q[i]; }
};
struct ViewHL {
  const float* hi;
  const float* lo;
  __device__ __forceinline__ double ld(long long i) const { return (double)hi[i] + (double)lo[i]; }
};

// Block partials of sum_n J^-1 Q_c (grid-stride order fixed by the launch).
// JOIN: every node's state as read (for the float pair, the FP64 value hi +
// lo) is also written to qout, so one pass both joins the state and sums it.
template <class View, typename TM, bool JOIN = false>
__global__ void k_totals_partial(Grid g, View Q, const TM* __restrict__ M,
                                 double* __restrict__ partials, double* __restrict__ qout = nullptr) {
  const long long N = g.N;
  double s[5] = {0, 0, 0, 0, 0};
  for (long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x; n < N;
       n += (long long)gridDim.x * blockDim.x) {
    double v[5];
#pragma unroll
    for (int q = 0; q < 5; ++q) v[q] = Q.ld(q * N + n);
    if (JOIN) {
#pragma unroll
      for (int q = 0; q < 5; ++q) qout[q * N + n] = v[q];
    }
    if ((g.glo | g.ghi) != 0 && !owned_plane(g, (int)(n / g.stride[0]))) continue;  // a slab sums its own planes
    const double jv = (double)M[9 * N + n];
#pragma unroll
    for (int q = 0; q < 5; ++q) s[q] += jv * v[q];
  }
  __shared__ double red[5][32];
#pragma unroll
  for (int q = 0; q < 5; ++q)
    for (int off = 16; off > 0; off >>= 1) s[q] += __shfl_xor_sync(0xffffffffu, s[q], off);
  if ((threadIdx.x & 31) == 0)
#pragma unroll
    for (int q = 0; q < 5; ++q) red[q][threadIdx.x >> 5] = s[q];
  __syncthreads();
  if (threadIdx.x < 32) {
#pragma unroll
    for (int q = 0; q < 5; ++q) {
      double v = threadIdx.x < (blockDim.x >> 5) ? red[q][threadIdx.x] : 0.0;
      for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
      if (threadIdx.x == 0) partials[q * kRedBlocks + blockIdx.x] = v;
    }
  }
}

__global__ void k_totals_final(const double* __restrict__ partials, DevScalars* sc) {
  const int q = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (q >= 5) return;
  double v = 0.0;
  for (int b = lane; b < kRedBlocks; b += 32) v += partials[q * kRedBlocks + b];
  for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
  if (lane == 0) sc->totals[q] = v;
}

__global__ void k_set_time(DevScalars* sc, double t) {
  sc->t = t;
  sc->dt = 0.0;
  sc->status = 0;
  sc->steps = 0;
  sc->ticket = 0;
}

static int nblocks(long long count) {
  long long b = (count + 255) / 256;
  const long long cap = 16LL * sm_count();
  if (b > cap) b = cap;
  return (int)(b < 1 ? 1 : b);
}

template <class Acc, typename TM>
static void bc_jet(const Grid& g, const les_params& p, Acc Q, const TM* M,
                   const double* rth, const DevScalars* sc, int use_host_t, double t_host,
                   const Launch& L) {
  JetBC b;
  b.mode = p.bc;
  b.gamma = p.gamma;
  b.Mj = p.Mj;
  b.r_jet = p.r_jet;
  b.theta_m = p.theta_m;
  b.force_width = p.force_width;
  for (int i = 0; i < 4; ++i) b.St[i] = p.St[i];
  b.forced = 0;
  for (int i = 0; i < 16; ++i) {
    b.amp[i] = p.amp[i];
    if (p.amp[i] != 0.0) b.forced = 1;
  }
  const long long plane = (long long)g.n[1] * g.n[2];
  // an axial slab has the entrance only if it starts at the physical face
  // and the exit only if it ends there (its far field and inner ring cover
  // its ghost planes too, which the next exchange overwrites)
  const int nb_ff = nblocks((long long)(g.n[0] - 2) * g.n[2]);
  if (p.bc != LES_BC_JET_CHAR && g.n[1] >= 3) {
    const int nb_in = g.glo == 0 ? nblocks(plane) : 0;
    k_bc_sides<Acc, TM><<<nb_ff + nb_in + (g.n[0] - 2), 256, 0, L.s>>>(
        g, b, rth, M, sc, use_host_t, t_host, Q, nb_ff, nb_in);
    ++*L.counter;
  } else {
    // the characteristic entrance reads the plane i = 1 before the far field
    // and the ring write its edges
    if (g.glo == 0) {
      k_bc_inflow<Acc, TM><<<nblocks(plane), 256, 0, L.s>>>(g, b, rth, M, sc, use_host_t, t_host,
                                                             Q);
      ++*L.counter;
    }
    k_bc_farfield<Acc, TM><<<nb_ff, 256, 0, L.s>>>(g, p.gamma, M, Q);
    k_bc_ring<Acc><<<g.n[0] - 2, 256, 0, L.s>>>(g, Q);
    *L.counter += 2;
  }
  if (g.ghi == 0) {
    k_bc_exit<Acc, TM><<<nblocks(plane), 256, 0, L.s>>>(g, p.gamma, M, Q);
    ++*L.counter;
  }
}

void launch_bc_jet(const Grid& g, const les_params& p, double* Q, const double* M64,
                   const double* rth, const DevScalars* sc, int use_host_t, double t_host,
                   const Launch& L) {
  bc_jet(g, p, AccD{Q}, M64, rth, sc, use_host_t, t_host, L);
}

void launch_bc_jet(const Grid& g, const les_params& p, double* Q, const float* M32,
                   const double* rth, const DevScalars* sc, int use_host_t, double t_host,
                   const Launch& L) {
  bc_jet(g, p, AccD{Q}, M32, rth, sc, use_host_t, t_host, L);
}

void launch_bc_jet_hl(const Grid& g, const les_params& p, float* hi, float* lo, const double* M64,
                      const double* rth, const DevScalars* sc, const Launch& L) {
  bc_jet(g, p, AccHL{hi, lo}, M64, rth, sc, 0, 0.0, L);
}

void launch_bc_jet_hl(const Grid& g, const les_params& p, float* hi, float* lo, const float* M32,
                      const double* rth, const DevScalars* sc, const Launch& L) {
  bc_jet(g, p, AccHL{hi, lo}, M32, rth, sc, 0, 0.0, L);
}

template <class View, typename TM>
static void totals_t(const Grid& g, View Q, const TM* M, double* partials, DevScalars* sc,
                     const Launch& L) {
  k_totals_partial<View, TM><<<kRedBlocks, kRedThreads, 0, L.s>>>(g, Q, M, partials);
  k_totals_final<<<1, 160, 0, L.s>>>(partials, sc);
  *L.counter += 2;
}

void launch_totals(const Grid& g, const double* Q, const double* M64, double* partials,
                   DevScalars* sc, const Launch& L) {
  totals_t(g, ViewD{Q}, M64, partials, sc, L);
}

void launch_totals(const Grid& g, const double* Q, const float* M32, double* partials,
                   DevScalars* sc, const Launch& L) {
  totals_t(g, ViewD{Q}, M32, partials, sc, L);
}

void launch_totals_hl(const Grid& g, const float* hi, const float* lo, const double* M64,
                      double* partials, DevScalars* sc, const Launch& L) {
  totals_t(g, ViewHL{hi, lo}, M64, partials, sc, L);
}

void launch_totals_hl(const Grid& g, const float* hi, const float* lo, const float* M32,
                      double* partials, DevScalars* sc, const Launch& L) {
  totals_t(g, ViewHL{hi, lo}, M32, partials, sc, L);
}

template <typename TM>
static void join_totals_t(const Grid& g, const float* hi, const float* lo, const TM* M, double* q,
                          double* partials, DevScalars* sc, const Launch& L) {
  k_totals_partial<ViewHL, TM, true><<<kRedBlocks, kRedThreads, 0, L.s>>>(g, ViewHL{hi, lo}, M,
                                                                        partials, q);
  k_totals_final<<<1, 160, 0, L.s>>>(partials, sc);
  *L.counter += 2;
}

void launch_join_totals_hl(const Grid& g, const float* hi, const float* lo, const double* M64,
                           double* q, double* partials, DevScalars* sc, const Launch& L) {
  join_totals_t(g, hi, lo, M64, q, partials, sc, L);
}

void launch_join_totals_hl(const Grid& g, const float* hi, const float* lo, const float* M32,
                           double* q, double* partials, DevScalars* sc, const Launch& L) {
  join_totals_t(g, hi, lo, M32, q, partials, sc, L);
}

void launch_set_time(DevScalars* sc, double t, const Launch& L) {
  k_set_time<<<1, 1, 0, L.s>>>(sc, t);
  ++*L.counter;
}

}  // namespace lesjet
