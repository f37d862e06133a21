// stage64_kernels.cuh -- kernel templates of the per-pass residual (node,
// viscosity, interface flux, update).  Instantiated for double by stage64.cu
// (the FP64 form) and for Dual by adjoint.cu (exact Jacobian-vector products
// used to check the hand-written adjoint).
#pragma once

#include "lesjet_dev.cuh"
#include "lesjet_host.h"

namespace lesjet {

template <typename R>
inline Consts<R> make_consts(const les_params& p) {
  Consts<R> K;
  K.gamma = (R)p.gamma;
  K.gm1 = (R)(p.gamma - 1.0);
  K.k2 = (R)p.k2;
  K.k4 = (R)p.k4;
  K.mu_scale = (R)(p.Re > 0.0 ? p.Mj / p.Re : 0.0);
  K.S_suth = (R)(110.4 / p.T_ref);
  K.axis = p.axis;
  K.cs2 = (R)(p.sgs_model == LES_SGS_VREMAN ? 2.5 * p.Cs * p.Cs : p.Cs * p.Cs);
  K.inv_gm1_pr = (R)(1.0 / ((p.gamma - 1.0) * p.Pr));
  K.inv_gm1_prs = (R)(1.0 / ((p.gamma - 1.0) * p.Pr_sgs));
  K.sgs = p.sgs_model;
  return K;
}

inline int blocks_for(long long count, int threads, long long cap = 0) {
  if (cap <= 0) cap = 64LL * sm_count();
  long long b = (count + threads - 1) / threads;
  if (b > cap) b = cap;
  if (b < 1) b = 1;
  return (int)b;
}

// ------------------------------------------------------------------ k_node
// Primitive recovery (System I energy), spectral radii lambda_d = |U_d| +
// a |grad d| and lbar_xi = lambda_xi + sqrt(lambda_xi lambda_eta) +
// sqrt(lambda_xi lambda_zeta) (= lambda_xi [1 + (lambda_eta/lambda_xi)^0.5 +
// (lambda_zeta/lambda_xi)^0.5]), cyclic for eta and zeta.  |grad d| is read
// from gn ([3][N], taken once at set-up) when given, else evaluated from M.
template <typename R, typename TQ, typename TM, bool WITH_DT>
__global__ void __launch_bounds__(256) k_node(Grid g, Consts<R> K, const TQ* __restrict__ Q,
                                              const TM* __restrict__ M,
                                              const double* __restrict__ gn, R* __restrict__ node,
                                              double* __restrict__ partials,
                                              DevScalars* __restrict__ sc,
                                              double* __restrict__ dtl = nullptr,
                                              double cfl = 0.0) {
  const long long N = g.N;
  double local_min = 1.0e300;
  int bad = 0;
  for (long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x; n < N;
       n += (long long)gridDim.x * blockDim.x) {
    const R rho = (R)Q[n];
    const R inv_rho = R(1) / rho;
    const R u = (R)Q[N + n] * inv_rho;
    const R v = (R)Q[2 * N + n] * inv_rho;
    const R w = (R)Q[3 * N + n] * inv_rho;
    const R p = K.gm1 * ((R)Q[4 * N + n] - R(0.5) * rho * (u * u + v * v + w * w));
    const R T = K.gamma * p * inv_rho;
    const R a = dev_sqrt(T);
    // the radii's node: itself, or for an axis node (J^-1 = 0 on ring j = 0,
    // Reading A27) its inward neighbour (i, 1, k), whose radii it takes
    long long nr = n;
    R ur = u, vr = v, wr = w, ar = a;
    if (K.axis && (R)M[9 * N + n] == R(0) && (n / g.n[2]) % g.n[1] == 0) {
      nr = n + g.stride[1];
      const R rho1 = (R)Q[nr];
      const R ir1 = R(1) / rho1;
      ur = (R)Q[N + nr] * ir1;
      vr = (R)Q[2 * N + nr] * ir1;
      wr = (R)Q[3 * N + nr] * ir1;
      const R p1 = K.gm1 * ((R)Q[4 * N + nr] - R(0.5) * rho1 * (ur * ur + vr * vr + wr * wr));
      ar = dev_sqrt(K.gamma * p1 * ir1);
    }
    R lam[3];
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      const R mx = (R)M[(3 * d) * N + nr], my = (R)M[(3 * d + 1) * N + nr],
              mz = (R)M[(3 * d + 2) * N + nr];
      const R gd = gn ? (R)gn[d * N + nr] : dev_sqrt(mx * mx + my * my + mz * mz);
      lam[d] = dev_abs(mx * ur + my * vr + mz * wr) + ar * gd;
    }
    const R s01 = dev_sqrt(lam[0] * lam[1]);
    const R s02 = dev_sqrt(lam[0] * lam[2]);
    const R s12 = dev_sqrt(lam[1] * lam[2]);
    node[n] = u;
    node[N + n] = v;
    node[2 * N + n] = w;
    node[3 * N + n] = p;
    node[4 * N + n] = T;
    node[5 * N + n] = lam[0] + s01 + s02;
    node[6 * N + n] = lam[1] + s01 + s12;
    node[7 * N + n] = lam[2] + s02 + s12;
    if (WITH_DT) {
      const double inv = 1.0 / ((double)lam[0] + (double)lam[1] + (double)lam[2]);
      if ((g.glo | g.ghi) == 0 || owned_plane(g, (int)(n / g.stride[0]))) {  // a slab's ghost planes are its neighbour's
        if (!(rho > R(0)) || !(p > R(0)) || !(inv > 0.0) || !(inv < 1.0e300)) bad = 1;
        local_min = inv < local_min ? inv : local_min;
      }
      if (dtl) dtl[n] = cfl * inv;  // local step of Eq. localdt
    }
  }
  if (WITH_DT) {
    __shared__ double smin[32];
    __shared__ int sbad;
    if (threadIdx.x == 0) sbad = 0;
    for (int off = 16; off > 0; off >>= 1)
      local_min = fmin(local_min, __shfl_xor_sync(0xffffffffu, local_min, off));
    __syncthreads();
    if ((threadIdx.x & 31) == 0) smin[threadIdx.x >> 5] = local_min;
    if (bad) atomicOr(&sbad, 1);
    __syncthreads();
    if (threadIdx.x < 32) {
      double m = threadIdx.x < (blockDim.x >> 5) ? smin[threadIdx.x] : 1.0e300;
      for (int off = 16; off > 0; off >>= 1) m = fmin(m, __shfl_xor_sync(0xffffffffu, m, off));
      if (threadIdx.x == 0) {
        partials[blockIdx.x] = m;
        if (sbad) atomicOr(&sc->status, 1);
      }
    }
  }
}

// -------------------------------------------------------------------- k_mu
// Node-centred computational derivative (central; one-sided second order at
// non-periodic faces).
template <typename R>
__device__ __forceinline__ R node_deriv(const Grid& g, const R* __restrict__ f, long long n,
                                        const int c[3], int d) {
  const long long s = g.stride[d];
  const int nd = g.n[d];
  if (g.per[d]) {
    const long long np = (c[d] == nd - 1) ? n - (long long)(nd - 1) * s : n + s;
    const long long nm = (c[d] == 0) ? n + (long long)(nd - 1) * s : n - s;
    return R(0.5) * (f[np] - f[nm]);
  }
  if (c[d] == 0) return R(0.5) * (R(-3) * f[n] + R(4) * f[n + s] - f[n + 2 * s]);
  if (c[d] == nd - 1) return R(0.5) * (R(3) * f[n] - R(4) * f[n - s] + f[n - 2 * s]);
  return R(0.5) * (f[n + s] - f[n - s]);
}

// mu_eff = (Mj/Re) T^1.5 (1+S)/(T+S) + mu_sgs; kappa_eff = mu_lam/((g-1)Pr)
// + mu_sgs/((g-1)Pr_sgs).  Smagorinsky: rho (Cs Delta)^2 |S|; Vreman:
// rho c sqrt(B_beta/alpha:alpha) (0 when alpha:alpha = 0, B_beta >= 0);
// dynamic: C_ds rho Delta^2 |S| with the dynamic Pr_sgs and the Yoshizawa
// sigma_ll = 2 C_I rho Delta^2 |S|^2 as a third field (coefficients dyn[6..8]
// from the dynamic procedure); Delta = (J^-1)^(1/3).
template <typename R, typename TQ, typename TM>
__global__ void __launch_bounds__(256) k_mu(Grid g, Consts<R> K, const TQ* __restrict__ Q,
                                            const TM* __restrict__ M,
                                            const R* __restrict__ node, R* __restrict__ mk,
                                            const double* __restrict__ dyn = nullptr) {
  const long long N = g.N;
  for (long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x; n < N;
       n += (long long)gridDim.x * blockDim.x) {
    const R T = node[4 * N + n];
    const R mu_l = K.mu_scale * T * dev_sqrt(T) * (R(1) + K.S_suth) / (T + K.S_suth);
    R mu_s = R(0);
    R kap_s = R(0);
    bool kap_set = false;
    if (K.sgs != LES_SGS_NONE) {
      int c[3];
      decompose(g, n, c);
      R gr[3][3];  // gr[i][x] = d u_i / d x_x
#pragma unroll
      for (int q = 0; q < 3; ++q) {
        R dd[3];
#pragma unroll
        for (int d = 0; d < 3; ++d) dd[d] = node_deriv(g, node + q * N, n, c, d);
#pragma unroll
        for (int x = 0; x < 3; ++x)
          gr[q][x] = (R)M[x * N + n] * dd[0] + (R)M[(3 + x) * N + n] * dd[1] +
                     (R)M[(6 + x) * N + n] * dd[2];
      }
      const R Jinv = (R)M[9 * N + n];
      const R delta = cbrt(Jinv);
      const R rho = (R)Q[n];
      if (K.sgs == LES_SGS_SMAGORINSKY) {
        R ss = R(0);
#pragma unroll
        for (int i = 0; i < 3; ++i)
#pragma unroll
          for (int j = 0; j < 3; ++j) {
            const R sij = R(0.5) * (gr[i][j] + gr[j][i]);
            ss += sij * sij;
          }
        mu_s = rho * (delta * delta) * K.cs2 * dev_sqrt(R(2) * ss);
      } else if (K.sgs == LES_SGS_DYNAMIC) {
        R ss = R(0);
#pragma unroll
        for (int i = 0; i < 3; ++i)
#pragma unroll
          for (int j = 0; j < 3; ++j) {
            const R sij = R(0.5) * (gr[i][j] + gr[j][i]);
            ss += sij * sij;
          }
        const R smag = dev_sqrt(R(2) * ss);
        const R d2 = delta * delta;
        mu_s = R(dyn[6]) * rho * d2 * smag;
        kap_s = mu_s / (K.gm1 * R(dyn[8]));
        kap_set = true;
        mk[2 * N + n] = R(2) * R(dyn[7]) * rho * d2 * smag * smag;
      } else {
        // alpha_ij = d u_j / d x_i = gr[j][i]; beta_ij = Delta^2 alpha_mi alpha_mj
        R aa = R(0);
#pragma unroll
        for (int i = 0; i < 3; ++i)
#pragma unroll
          for (int j = 0; j < 3; ++j) aa += gr[i][j] * gr[i][j];
        R be[3][3];
#pragma unroll
        for (int i = 0; i < 3; ++i)
#pragma unroll
          for (int j = 0; j < 3; ++j)
            be[i][j] = delta * delta *
                       (gr[i][0] * gr[j][0] + gr[i][1] * gr[j][1] + gr[i][2] * gr[j][2]);
        R B = be[0][0] * be[1][1] - be[0][1] * be[0][1] + be[0][0] * be[2][2] -
              be[0][2] * be[0][2] + be[1][1] * be[2][2] - be[1][2] * be[1][2];
        B = B > R(0) ? B : R(0);
        mu_s = (aa == R(0)) ? R(0) : rho * K.cs2 * dev_sqrt(B / aa);
      }
    }
    mk[n] = mu_l + mu_s;
    mk[N + n] = mu_l * K.inv_gm1_pr + (kap_set ? kap_s : mu_s * K.inv_gm1_prs);
  }
}

// ------------------------------------------------------------------ k_flux
// Pressure sensor |p+ - 2p + p-| / (p+ + 2p + p-) of node x along D; a face
// node of a non-periodic direction takes its inward neighbour's value.
template <int D, typename R>
__device__ __forceinline__ R sensor(const Grid& g, const R* __restrict__ P, long long x, int cx) {
  const long long s = g.stride[D];
  const int nd = g.n[D];
  long long xc = x;
  int cc = cx;
  if (!g.per[D]) {
    if (cx == 0) { xc = x + s; cc = 1; }
    else if (cx == nd - 1) { xc = x - s; cc = nd - 2; }
  }
  const long long xp = (cc == nd - 1) ? xc - (long long)(nd - 1) * s : xc + s;
  const long long xm = (cc == 0) ? xc + (long long)(nd - 1) * s : xc - s;
  const R pp = P[xp], p0 = P[xc], pm = P[xm];
  return dev_abs(pp - R(2) * p0 + pm) / (pp + R(2) * p0 + pm);
}

// The three sensors of every node, once per residual evaluation (each node's
// sensor along D is read by its two interfaces along D).
template <typename R>
__global__ void __launch_bounds__(256) k_sensor(Grid g, const R* __restrict__ P,
                                                R* __restrict__ NU) {
  const long long N = g.N;
  for (long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x; n < N;
       n += (long long)gridDim.x * blockDim.x) {
    int c[3];
    decompose(g, n, c);
    NU[n] = sensor<0>(g, P, n, c[0]);
    NU[N + n] = sensor<1>(g, P, n, c[1]);
    NU[2 * N + n] = sensor<2>(g, P, n, c[2]);
  }
}

template <int D, typename R, typename TQ, typename TM>
__global__ void __launch_bounds__(256) k_flux(Grid g, Consts<R> K, const TQ* __restrict__ Q,
                                              const TM* __restrict__ M,
                                              const R* __restrict__ node,
                                              const R* __restrict__ mk, R* __restrict__ F,
                                              const R* __restrict__ NU = nullptr) {
  constexpr int T1 = (D + 1) % 3, T2 = (D + 2) % 3;
  const long long N = g.N;
  const R* __restrict__ U = node;
  const R* __restrict__ V = node + N;
  const R* __restrict__ Wv = node + 2 * N;
  const R* __restrict__ P = node + 3 * N;
  const R* __restrict__ Tt = node + 4 * N;
  const R* __restrict__ LB = node + (5 + D) * N;
  // The interface means are left as sums of the two nodes' values and their
  // powers of two are folded into a few factors (exact in binary floating
  // point): F is written as exactly 2x the interface flux, and k_update
  // halves J once per node.
  const R k2h = R(0.5) * K.k2, k4h = R(0.5) * K.k4;
  for (long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x; n < N;
       n += (long long)gridDim.x * blockDim.x) {
    int c[3];
    decompose(g, n, c);
    if (!g.per[D] && c[D] == g.n[D] - 1) continue;
    if (!g.per[T1] && (c[T1] == 0 || c[T1] == g.n[T1] - 1)) continue;
    if (!g.per[T2] && (c[T2] == 0 || c[T2] == g.n[T2] - 1)) continue;
    const long long a = n;
    const long long b = step(g, n, c, D, 1);
    const long long am = step(g, n, c, D, -1);
    const long long bp = step(g, n, c, D, 2);
    int cb[3] = {c[0], c[1], c[2]};
    cb[D] = (c[D] + 1 == g.n[D]) ? 0 : c[D] + 1;

    // centred inviscid flux (Eq. hat-flux-G, xi_t = 0)
    const R Ja = (R)M[9 * N + a], Jb = (R)M[9 * N + b];
    const R ma0 = (R)M[(3 * D) * N + a], ma1 = (R)M[(3 * D + 1) * N + a],
            ma2 = (R)M[(3 * D + 2) * N + a];
    const R mb0 = (R)M[(3 * D) * N + b], mb1 = (R)M[(3 * D + 1) * N + b],
            mb2 = (R)M[(3 * D + 2) * N + b];
    const R pa = P[a], pb = P[b];
    const R tha = ma0 * U[a] + ma1 * V[a] + ma2 * Wv[a];
    const R thb = mb0 * U[b] + mb1 * V[b] + mb2 * Wv[b];
    R Qa[5], Qb[5];
#pragma unroll
    for (int q = 0; q < 5; ++q) {
      Qa[q] = (R)Q[q * N + a];
      Qb[q] = (R)Q[q * N + b];
    }
    R Fa[5], Fb[5];
    Fa[0] = Ja * (Qa[0] * tha);
    Fa[1] = Ja * (Qa[1] * tha + pa * ma0);
    Fa[2] = Ja * (Qa[2] * tha + pa * ma1);
    Fa[3] = Ja * (Qa[3] * tha + pa * ma2);
    Fa[4] = Ja * ((Qa[4] + pa) * tha);
    Fb[0] = Jb * (Qb[0] * thb);
    Fb[1] = Jb * (Qb[1] * thb + pb * mb0);
    Fb[2] = Jb * (Qb[2] * thb + pb * mb1);
    Fb[3] = Jb * (Qb[3] * thb + pb * mb2);
    Fb[4] = Jb * ((Qb[4] + pb) * thb);

    // Turkel-Vatsa dissipation (Eqs. dissip_term, eps_2/4_dissip, W_dissip)
    const R nua = NU ? NU[D * N + a] : sensor<D>(g, P, a, c[D]);
    const R nub = NU ? NU[D * N + b] : sensor<D>(g, P, b, cb[D]);
    const R eps2 = k2h * dev_max(nua, nub);    // half of eps^(2)
    const R eps4 = dev_max(R(0), k4h - eps2);  // half of eps^(4)
    const R sJ = Ja + Jb;                      // 2 J^-1 at the interface
    const R lJ = (LB[a] + LB[b]) * sJ;         // 4 lambda J^-1 at the interface
    R Fq[5];                                   // 2x
#pragma unroll
    for (int q = 0; q < 5; ++q) {
      const R wa = (q == 4) ? Qa[4] + pa : Qa[q];
      const R wb = (q == 4) ? Qb[4] + pb : Qb[q];
      const R D1 = wb - wa;
      R Dm, Dp;
      if (am >= 0) {
        const R wm = (q == 4) ? (R)Q[4 * N + am] + P[am] : (R)Q[q * N + am];
        Dm = wa - wm;
      } else {
        Dm = -D1;
      }
      if (bp >= 0) {
        const R wp = (q == 4) ? (R)Q[4 * N + bp] + P[bp] : (R)Q[q * N + bp];
        Dp = wp - wb;
      } else {
        Dp = -D1;
      }
      const R D3 = Dp - R(2) * D1 + Dm;
      Fq[q] = (Fa[q] + Fb[q]) - lJ * (eps2 * D1 - eps4 * D3);
    }

    // viscous + SGS flux with compact interface gradients (Eqs.
    // hat-flux-Ev/Fv/Gv, tau_mod, q_mod with Fourier's sign); the tangential
    // derivatives are kept as 4x their value (the 1/4 of the mean of the two
    // central differences is folded away)
    const R* phi[4] = {U, V, Wv, Tt};
    R dphi[4][3];
#pragma unroll
    for (int q = 0; q < 4; ++q) dphi[q][D] = phi[q][b] - phi[q][a];
    {
      const long long ap = step(g, a, c, T1, 1), amm = step(g, a, c, T1, -1);
      const long long bpp = step(g, b, cb, T1, 1), bm = step(g, b, cb, T1, -1);
#pragma unroll
      for (int q = 0; q < 4; ++q)
        dphi[q][T1] = (phi[q][ap] - phi[q][amm]) + (phi[q][bpp] - phi[q][bm]);
    }
    {
      const long long ap = step(g, a, c, T2, 1), amm = step(g, a, c, T2, -1);
      const long long bpp = step(g, b, cb, T2, 1), bm = step(g, b, cb, T2, -1);
#pragma unroll
      for (int q = 0; q < 4; ++q)
        dphi[q][T2] = (phi[q][ap] - phi[q][amm]) + (phi[q][bpp] - phi[q][bm]);
    }
    // interface metrics: 8x the mean along the normal, 2x along the
    // tangents, so that every product with dphi is 8x its value
    R mh[3][3];
    if (K.axis) {
      // a grid with an axis (Reading A27): the J^-1-weighted mean
      // (J^-1_a m_a + J^-1_b m_b)/(J^-1_a + J^-1_b), kept at 2x like the
      // plain sum; an axis node's stored metric is J^-1 m already
      const R wa = (Ja == R(0)) ? R(1) : Ja, wb = (Jb == R(0)) ? R(1) : Jb;
      const R s2 = R(2) / sJ;
#pragma unroll
      for (int t = 0; t < 3; ++t)
#pragma unroll
        for (int x = 0; x < 3; ++x)
          mh[t][x] = (wa * (R)M[(3 * t + x) * N + a] + wb * (R)M[(3 * t + x) * N + b]) * s2;
    } else {
#pragma unroll
      for (int t = 0; t < 3; ++t)
#pragma unroll
        for (int x = 0; x < 3; ++x)
          mh[t][x] = (R)M[(3 * t + x) * N + a] + (R)M[(3 * t + x) * N + b];
    }
#pragma unroll
    for (int x = 0; x < 3; ++x) mh[D][x] = R(4) * mh[D][x];
    // The flux needs only m.tau and m.q (m = the interface metric of
    // direction D), which follow from the contractions g_t = m . m_t and
    // c_t = sum_j m_j dphi_j,t and the divergence without forming the
    // gradient tensor:
    //   m.tau_i / mu = sum_t g_t dphi_i,t + sum_t m_t,i c_t - 2/3 m_i div,
    //   m.grad T     = sum_t g_t dphi_T,t.
    // With mh (8 m_D, 2 m_t) and dphi (1x along D, 4x along the tangents)
    // every term below is 64x its value.
    const R mx = mh[D][0], my = mh[D][1], mz = mh[D][2];  // 8 m
    R G[3], Cc[3];
#pragma unroll
    for (int t = 0; t < 3; ++t) {
      G[t] = mx * mh[t][0] + my * mh[t][1] + mz * mh[t][2];
      Cc[t] = mx * dphi[0][t] + my * dphi[1][t] + mz * dphi[2][t];
    }
    R div = R(0);  // 8 div
#pragma unroll
    for (int t = 0; t < 3; ++t)
      div += mh[t][0] * dphi[0][t] + mh[t][1] * dphi[1][t] + mh[t][2] * dphi[2][t];
    const R d23 = R(2.0 / 3.0) * div;
    const R mv[3] = {mx, my, mz};
    R sv[3];  // 64 m.tau_i / mu
#pragma unroll
    for (int i = 0; i < 3; ++i)
      sv[i] = (G[0] * dphi[i][0] + G[1] * dphi[i][1] + G[2] * dphi[i][2]) +
              (mh[0][i] * Cc[0] + mh[1][i] * Cc[1] + mh[2][i] * Cc[2]) - mv[i] * d23;
    const R aT = G[0] * dphi[3][0] + G[1] * dphi[3][1] + G[2] * dphi[3][2];  // 64 m.grad T
    const R mu = mk[a] + mk[b];                    // 2 mu
    const R kap = R(2) * (mk[N + a] + mk[N + b]);  // 4 kappa
    const R uf = U[a] + U[b];  // 2 u at the interface
    const R vf = V[a] + V[b];
    const R wf = Wv[a] + Wv[b];
    // 2 J^-1 m.tau_i = sJ mu sv_i / 128; 2 J^-1 m.(tau u_f + kappa grad T) =
    // sJ (mu (u_f . sv) + kap aT) / 256
    const R c1 = sJ * mu * R(1.0 / 128.0), c2 = sJ * R(1.0 / 256.0);
    R f1 = c1 * sv[0], f2 = c1 * sv[1], f3 = c1 * sv[2];
    R f4 = c2 * (mu * (uf * sv[0] + vf * sv[1] + wf * sv[2]) + kap * aT);
    if (K.sgs == LES_SGS_DYNAMIC) {
      // the modelled isotropic SGS stress sigma_ll/3 (Eq. yoshizawa) at the
      // interface mean, subtracted from the normal stresses: m.tau_i gains
      // -m_i sigma/3 and u_f.(m.tau) gains -(u_f . m) sigma/3
      const R ss = mk[2 * N + a] + mk[2 * N + b];  // 2 sigma_ll
      const R e1 = sJ * ss * R(1.0 / 48.0);
      f1 -= e1 * mx;
      f2 -= e1 * my;
      f3 -= e1 * mz;
      f4 -= e1 * R(0.5) * (uf * mx + vf * my + wf * mz);
    }
    F[n] = Fq[0];
    F[N + n] = Fq[1] - f1;
    F[2 * N + n] = Fq[2] - f2;
    F[3 * N + n] = Fq[3] - f3;
    F[4 * N + n] = Fq[4] - f4;
  }
}

// ---------------------------------------------------------------- k_update
template <typename R, typename TM, typename TO, int MODE>
__global__ void __launch_bounds__(256) k_update(Grid g, const R* __restrict__ F,
                                                const double* __restrict__ Q0,
                                                const TM* __restrict__ M,
                                                const DevScalars* __restrict__ sc, double alpha,
                                                TO* __restrict__ out,
                                                const double* __restrict__ dtl = nullptr,
                                                const double* __restrict__ jh = nullptr) {
  const long long N = g.N;
  const R* F0 = F;
  const R* F1 = F + 5 * N;
  const R* F2 = F + 10 * N;
  const double adt = (MODE == 0) ? 0.0 : alpha * sc->dt;
  for (long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x; n < N;
       n += (long long)gridDim.x * blockDim.x) {
    int c[3];
    decompose(g, n, c);
    if (!is_interior(g, c)) {
      if (MODE == 0) {
#pragma unroll
        for (int q = 0; q < 5; ++q) out[q * N + n] = (TO)0;
      } else if (MODE == 1) {
#pragma unroll
        for (int q = 0; q < 5; ++q) out[q * N + n] = (TO)Q0[q * N + n];
      }
      continue;
    }
    const long long m0 = step(g, n, c, 0, -1);
    const long long m1 = step(g, n, c, 1, -1);
    const long long m2 = step(g, n, c, 2, -1);
    // J once per node, halved: k_flux writes 2x the interface fluxes (jh
    // holds the same quotient, taken at set-up)
    const double Jn = (MODE == 0) ? 0.0 : (jh ? jh[n] : 0.5 / (double)M[9 * N + n]);
    const double a = (MODE == 0) ? 0.0 : (dtl ? alpha * dtl[n] : adt);
#pragma unroll
    for (int q = 0; q < 5; ++q) {
      R r = R(0);
      r += F0[q * N + n] - F0[q * N + m0];
      r += F1[q * N + n] - F1[q * N + m1];
      r += F2[q * N + n] - F2[q * N + m2];
      if (MODE == 0) {
        out[q * N + n] = (TO)(R(0.5) * r);
      } else {
        out[q * N + n] = (TO)(Q0[q * N + n] - a * (Jn * (double)r));
      }
    }
  }
}

}  // namespace lesjet
