// setup.cu -- one-off kernels: grid metrics, jet initial condition, inflow
// geometry, FP32 metric copy.
#include "lesjet_dev.cuh"
#include "lesjet_host.h"

namespace lesjet {

// d(coordinate)/d(direction d) at node n: second-order central difference;
// a periodic wrap adds/subtracts the period's coordinate jump sh; faces of a
// non-periodic direction use the one-sided second-order formulas.
__device__ double coord_deriv(const Grid& g, const double* __restrict__ f, long long n,
                              const int c[3], int d, double sh) {
  const int nd = g.n[d];
  const long long s = g.stride[d];
  if (g.per[d]) {
    double fp = (c[d] == nd - 1) ? f[n - (long long)(nd - 1) * s] + sh : f[n + s];
    double fm = (c[d] == 0) ? f[n + (long long)(nd - 1) * s] - sh : f[n - s];
    return 0.5 * (fp - fm);
  }
  if (c[d] == 0) return 0.5 * (-3.0 * f[n] + 4.0 * f[n + s] - f[n + 2 * s]);
  if (c[d] == nd - 1) return 0.5 * (3.0 * f[n] - 4.0 * f[n - s] + f[n - 2 * s]);
  return 0.5 * (f[n + s] - f[n - s]);
}

struct Shift {
  double v[9];
};

// Jacobian determinant J^-1 of d(x,y,z)/d(xi,eta,zeta) and the metric terms
// as its cofactors times J (Sec. "Transformation of Coordinates"; the eta
// row uses the zeta/xi cofactors).  Computed in FP64; stored as TM (FP64, or
// rounded once to FP32 for the compact mixed form).
template <typename TM>
__global__ void k_metrics(Grid g, const double* __restrict__ xyz, Shift sh,
                          TM* __restrict__ M) {
  const long long N = g.N;
  for (long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x; n < N;
       n += (long long)gridDim.x * blockDim.x) {
    int c[3];
    decompose(g, n, c);
    double d[3][3];  // d[comp][dir]
#pragma unroll
    for (int comp = 0; comp < 3; ++comp)
#pragma unroll
      for (int dir = 0; dir < 3; ++dir)
        d[comp][dir] = coord_deriv(g, xyz + comp * N, n, c, dir, sh.v[3 * dir + comp]);
    const double xa = d[0][0], xb = d[0][1], xc = d[0][2];
    const double ya = d[1][0], yb = d[1][1], yc = d[1][2];
    const double za = d[2][0], zb = d[2][1], zc = d[2][2];
    const double c00 = yb * zc - yc * zb, c01 = zb * xc - zc * xb, c02 = xb * yc - xc * yb;
    const double c10 = yc * za - ya * zc, c11 = zc * xa - za * xc, c12 = xc * ya - xa * yc;
    const double c20 = ya * zb - yb * za, c21 = za * xb - zb * xa, c22 = xa * yb - xb * ya;
    const double Jinv = xa * yb * zc + xb * yc * za + xc * ya * zb - xa * yc * zb -
                        xb * ya * zc - xc * yb * za;
    // an axis node (J^-1 = 0 exactly, Reading A27) stores the cofactors
    // themselves, the J^-1-scaled metrics, which stay finite
    const double J = (Jinv == 0.0) ? 1.0 : 1.0 / Jinv;
    M[0 * N + n] = (TM)(J * c00);
    M[1 * N + n] = (TM)(J * c01);
    M[2 * N + n] = (TM)(J * c02);
    M[3 * N + n] = (TM)(J * c10);
    M[4 * N + n] = (TM)(J * c11);
    M[5 * N + n] = (TM)(J * c12);
    M[6 * N + n] = (TM)(J * c20);
    M[7 * N + n] = (TM)(J * c21);
    M[8 * N + n] = (TM)(J * c22);
    M[9 * N + n] = (TM)Jinv;
  }
}

// Metric terms in the conservative (Thomas-Lombard) form: with (r, s, t) and
// (c, p, q) cyclic orders of the directions and of the coordinates,
//   J^-1 r_c = d/dt (p_s q) - d/ds (p_t q),
// the cofactor of the continuous mapping written so that central
// differences of the nine J^-1 r_c telescope (discrete geometric
// conservation: a uniform flow has zero residual on any grid).  Each thread
// walks the outer-difference stencil of its node along every direction e;
// at each stencil node it forms the products (p_f q) for both inner
// directions f != e and adds them, with the difference weight and the sign
// of the pair (e, f), to the one row r that is neither e nor f.  J^-1 is the
// same determinant as in k_metrics; the stored metric is (J^-1 r_c)/J^-1.
template <typename TM>
__global__ void k_metrics_conservative(Grid g, const double* __restrict__ xyz, Shift sh,
                                       TM* __restrict__ M) {
  const long long N = g.N;
  for (long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x; n < N;
       n += (long long)gridDim.x * blockDim.x) {
    int c[3];
    decompose(g, n, c);
    double cof[3][3] = {{0.0, 0.0, 0.0}, {0.0, 0.0, 0.0}, {0.0, 0.0, 0.0}};  // [row][coordinate]
#pragma unroll 1
    for (int e = 0; e < 3; ++e) {
      const int ne = g.n[e];
      int cnt, off[3];
      double wt[3];
      if (g.per[e] || (c[e] > 0 && c[e] < ne - 1)) {
        cnt = 2; off[0] = 1; off[1] = -1; off[2] = 0;
        wt[0] = 0.5; wt[1] = -0.5; wt[2] = 0.0;
      } else if (c[e] == 0) {
        cnt = 3; off[0] = 0; off[1] = 1; off[2] = 2;
        wt[0] = -1.5; wt[1] = 2.0; wt[2] = -0.5;
      } else {
        cnt = 3; off[0] = 0; off[1] = -1; off[2] = -2;
        wt[0] = 1.5; wt[1] = -2.0; wt[2] = 0.5;
      }
#pragma unroll 1
      for (int a = 0; a < cnt; ++a) {
        int cm[3] = {c[0], c[1], c[2]};
        int v = c[e] + off[a], wrap = 0;
        if (v >= ne) { v -= ne; wrap = 1; }
        if (v < 0) { v += ne; wrap = -1; }
        cm[e] = v;
        const long long m = n + (long long)(v - c[e]) * g.stride[e];
        double xm[3];
#pragma unroll
        for (int k = 0; k < 3; ++k) xm[k] = xyz[k * N + m] + wrap * sh.v[3 * e + k];
#pragma unroll
        for (int df = 1; df < 3; ++df) {
          const int f = (e + df) % 3;
          const int r = 3 - e - f;
          const double sgn = (f == (r + 1) % 3) ? wt[a] : -wt[a];
#pragma unroll
          for (int comp = 0; comp < 3; ++comp) {
            const int pc = (comp + 1) % 3, qc = (comp + 2) % 3;
            const double dp = coord_deriv(g, xyz + pc * N, m, cm, f, sh.v[3 * f + pc]);
            cof[r][comp] += sgn * (dp * xm[qc]);
          }
        }
      }
    }
    double d[3][3];  // d[comp][dir] at the node itself, for J^-1
#pragma unroll
    for (int comp = 0; comp < 3; ++comp)
#pragma unroll
      for (int dir = 0; dir < 3; ++dir)
        d[comp][dir] = coord_deriv(g, xyz + comp * N, n, c, dir, sh.v[3 * dir + comp]);
    const double Jinv = d[0][0] * d[1][1] * d[2][2] + d[0][1] * d[1][2] * d[2][0] +
                        d[0][2] * d[1][0] * d[2][1] - d[0][0] * d[1][2] * d[2][1] -
                        d[0][1] * d[1][0] * d[2][2] - d[0][2] * d[1][1] * d[2][0];
#pragma unroll
    for (int r = 0; r < 3; ++r)
#pragma unroll
      for (int comp = 0; comp < 3; ++comp)
        M[(3 * r + comp) * N + n] = (TM)((Jinv == 0.0) ? cof[r][comp] : cof[r][comp] / Jinv);
    M[9 * N + n] = (TM)Jinv;
  }
}

__global__ void k_to_float(long long count, const double* __restrict__ a, float* __restrict__ b) {
  for (long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x; n < count;
       n += (long long)gridDim.x * blockDim.x)
    b[n] = (float)a[n];
}

// Grid constants the FP64 form takes once here instead of per residual:
// |grad d| = |(d_x, d_y, d_z)| of the three computational coordinates (the
// metric norms of the spectral radii lambda_d = |U_d| + a |grad d|), and
// J/2 = 0.5 / J^-1 of the stage update (0 where J^-1 = 0: an axis node,
// which the stages do not update).
__global__ void k_grad_norms(long long N, const double* __restrict__ M, double* __restrict__ gn) {
  for (long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x; n < N;
       n += (long long)gridDim.x * blockDim.x) {
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      const double mx = M[(3 * d) * N + n], my = M[(3 * d + 1) * N + n], mz = M[(3 * d + 2) * N + n];
      gn[d * N + n] = dev_sqrt(mx * mx + my * my + mz * mz);
    }
    const double Ji = M[9 * N + n];
    gn[3 * N + n] = Ji == 0.0 ? 0.0 : 0.5 / Ji;
  }
}

// Synthetic annular jet grid (Table tab:mesh stand-in): node (i, j, k) at
// x_i = L (q^i - 1)/(q^(ni-1) - 1) (L i/(ni-1) for q = 1), radius
// r_j = r0 + (r1 - r0) g(s_j)/g(1) with s_j = j/(nj-1) and the clustering map
// g(s) = s - (A/beta)[tanh(beta (s - s_c)) + tanh(beta s_c)], azimuth
// theta_k = 2 pi k/nk; y = r cos theta, z = r sin theta.
struct JetGridArgs {
  double length, q, r0, r1, A, beta, sc;
};

__device__ __forceinline__ double jet_map(double s, const JetGridArgs& a) {
  return s - (a.A / a.beta) * (tanh(a.beta * (s - a.sc)) + tanh(a.beta * a.sc));
}

__global__ void k_grid_jet(Grid g, JetGridArgs a, double* __restrict__ xyz) {
  const long long N = g.N;
  const int ni = g.n[0], nj = g.n[1], nk = g.n[2];
  const double two_pi = 6.283185307179586476925286766559;
  const double g1 = jet_map(1.0, a);
  const double qn = pow(a.q, (double)(ni - 1)) - 1.0;
  for (long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x; n < N;
       n += (long long)gridDim.x * blockDim.x) {
    int c[3];
    decompose(g, n, c);
    const double x = (a.q == 1.0) ? a.length * c[0] / (double)(ni - 1)
                                  : a.length * (pow(a.q, (double)c[0]) - 1.0) / qn;
    const double r = a.r0 + (a.r1 - a.r0) * jet_map(c[1] / (double)(nj - 1), a) / g1;
    double sn, cs;
    sincos(two_pi * c[2] / (double)nk, &sn, &cs);
    xyz[n] = x;
    xyz[N + n] = r * cs;
    xyz[2 * N + n] = r * sn;
  }
}

// Radius and azimuth of the entrance-plane nodes (i = 0), used by the inflow
// profile and forcing.
__global__ void k_inflow_geometry(Grid g, const double* __restrict__ xyz, double* __restrict__ rth) {
  const long long plane = (long long)g.n[1] * g.n[2];
  for (long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x; n < plane;
       n += (long long)gridDim.x * blockDim.x) {
    double y = xyz[g.N + n], z = xyz[2 * g.N + n];
    rth[n] = sqrt(y * y + z * z);
    rth[plane + n] = atan2(z, y);
  }
}

__device__ __forceinline__ double u01_53(uint32_t lo, uint32_t hi) {
  uint64_t b = ((((uint64_t)hi) << 32) | lo) >> 11;
  return ((double)b + 0.5) * (1.0 / 9007199254740992.0);
}

// Jet initial condition: rho = 1, p = 1/gamma, tanh axial profile, and
// noise*Mj*N(0,1) on u, v, w from Philox4x32-10 + Box-Muller (counter =
// (node lo, node hi, block, 0), key = seed; block 0 -> u', v'; block 1 -> w').
__global__ void k_init_jet(Grid g, const double* __restrict__ xyz, uint64_t seed, double noise,
                           double gamma, double Mj, double r_jet, double theta_m,
                           double* __restrict__ Q) {
  const long long N = g.N;
  const double two_pi = 6.283185307179586476925286766559;
  for (long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x; n < N;
       n += (long long)gridDim.x * blockDim.x) {
    double z[3];
#pragma unroll
    for (uint32_t blk = 0; blk < 2; ++blk) {
      uint32_t x[4] = {(uint32_t)n, (uint32_t)((unsigned long long)n >> 32), blk, 0u};
      philox4x32_10(x, (uint32_t)seed, (uint32_t)(seed >> 32));
      double u1 = u01_53(x[0], x[1]);
      double u2 = u01_53(x[2], x[3]);
      double rad = sqrt(-2.0 * log(u1));
      double s, co;
      sincos(two_pi * u2, &s, &co);
      if (blk == 0) {
        z[0] = rad * co;
        z[1] = rad * s;
      } else {
        z[2] = rad * co;
      }
    }
    double y = xyz[N + n], zc = xyz[2 * N + n];
    double r = sqrt(y * y + zc * zc);
    double u = 0.5 * Mj * (1.0 + tanh((r_jet - r) / (2.0 * theta_m))) + noise * Mj * z[0];
    double v = noise * Mj * z[1];
    double w = noise * Mj * z[2];
    double rho = 1.0, p = 1.0 / gamma;
    Q[n] = rho;
    Q[N + n] = rho * u;
    Q[2 * N + n] = rho * v;
    Q[3 * N + n] = rho * w;
    Q[4 * N + n] = p / (gamma - 1.0) + 0.5 * rho * (u * u + v * v + w * w);
  }
}

static int grid_blocks(long long count, int threads) {
  long long b = (count + threads - 1) / threads;
  const long long cap = 32LL * sm_count();
  if (b > cap) b = cap;
  if (b < 1) b = 1;
  return (int)b;
}

template <typename TM>
static void metrics_any(const Grid& g, const double* xyz, const double shift[9], int form, TM* M,
                        const Launch& L) {
  Shift sh;
  for (int i = 0; i < 9; ++i) sh.v[i] = shift ? shift[i] : 0.0;
  if (form == LES_METRIC_CONSERVATIVE)
    k_metrics_conservative<TM><<<grid_blocks(g.N, 256), 256, 0, L.s>>>(g, xyz, sh, M);
  else
    k_metrics<TM><<<grid_blocks(g.N, 256), 256, 0, L.s>>>(g, xyz, sh, M);
  ++*L.counter;
}

void launch_metrics(const Grid& g, const double* xyz, const double shift[9], int form, double* M,
                    const Launch& L) {
  metrics_any(g, xyz, shift, form, M, L);
}

void launch_metrics(const Grid& g, const double* xyz, const double shift[9], int form, float* M,
                    const Launch& L) {
  metrics_any(g, xyz, shift, form, M, L);
}

void launch_to_float(long long count, const double* a, float* b, const Launch& L) {
  k_to_float<<<grid_blocks(count, 256), 256, 0, L.s>>>(count, a, b);
  ++*L.counter;
}

void launch_grad_norms(const Grid& g, const double* M, double* gn, const Launch& L) {
  k_grad_norms<<<grid_blocks(g.N, 256), 256, 0, L.s>>>(g.N, M, gn);
  ++*L.counter;
}

void launch_inflow_geometry(const Grid& g, const double* xyz, double* rth, const Launch& L) {
  k_inflow_geometry<<<grid_blocks((long long)g.n[1] * g.n[2], 256), 256, 0, L.s>>>(g, xyz, rth);
  ++*L.counter;
}

void launch_init_jet(const Grid& g, const double* xyz, uint64_t seed, double noise,
                     const les_params& p, double* Q, const Launch& L) {
  k_init_jet<<<grid_blocks(g.N, 256), 256, 0, L.s>>>(g, xyz, seed, noise, p.gamma, p.Mj, p.r_jet,
                                                      p.theta_m, Q);
  ++*L.counter;
}

void launch_grid_jet(const Grid& g, double length, double q, double r0, double r1, double A,
                     double beta, double sc, double* xyz, const Launch& L) {
  JetGridArgs a{length, q, r0, r1, A, beta, sc};
  k_grid_jet<<<grid_blocks(g.N, 256), 256, 0, L.s>>>(g, a, xyz);
  ++*L.counter;
}

}  // namespace lesjet
