// adjoint.cu -- discrete adjoint (vector-Jacobian products) of the FP64 time
// step, and the tangent (Jacobian-vector product) of the residual used to
// check it.
//
// Residual adjoint: for every interface I = (a, b) the flux F_I enters RHS_a
// with + and RHS_b with -, so its cotangent is lamR_a - lamR_b.  The kernel
// k_adj_iface<D> recomputes the forward intermediates of the interface flux
// (centred inviscid flux, Turkel-Vatsa dissipation, compact viscous flux) and
// runs them in reverse, accumulating cotangents of the node quantities it
// read (conserved state, p, u, v, w, T, sensors, lbar, mu, kappa) into a
// record of that interface (what it owes each node it read); k_adj_gather
// then sums, per node and in a fixed order, the records of the interfaces
// that read it, so the accumulation is bitwise reproducible (no atomics).
// k_adj_sensor_terms / k_adj_sensor_gather move sensor cotangents to the
// pressures they were computed from the same way, and k_adj_node reverses
// the node quantities (radii, primitive recovery) into cotangents of Q.
//
// Non-differentiable points follow the forward kernels' branch choices:
// |x| has derivative -1 for x < 0 and +1 otherwise, max(a, b) passes the
// cotangent to the operand the comparison selected.
//
// Step adjoint (Eq. localdt with a fixed time step): with stage states S_l,
// Q^(l) = Q^(0) - alpha_l dt J RHS(Q^(l-1)) on interior nodes and Q^(l) =
// Q^(0) on boundary nodes, the reverse sweep accumulates lamQ0 += lamS_l and
// lamS_{l-1} = RHS^T(-alpha_l dt J lamS_l); the frozen viscosity mu(T(Q^n))
// collects its cotangent over the five stages and is reversed once.  The
// boundary conditions are reversed surface-only: the inner ring is linear,
// far-field and exit formulas use local 5x5 Jacobians from dual numbers, and
// the entrance plane turns its cotangent into the forcing-amplitude gradient.
#include <cuda_runtime.h>

#include "dual.cuh"
#include "lesjet_dev.cuh"
#include "lesjet_host.h"
#include "stage64_kernels.cuh"

namespace lesjet {

// accumulator slots (each [N] doubles)
enum {
  AQ0 = 0,   // AQ0..AQ0+4: direct cotangents of Q
  AP = 5,    // p
  AU = 6,    // u, v, w, T at AU..AU+3
  ANU = 10,  // sensor of direction d at ANU + d
  ALB = 13,  // lbar of direction d at ALB + d
  AMU = 16,  // mu_eff, kappa_eff at AMU, AMU+1
  NACC = 18
};

// Per-interface record (each [N] doubles, indexed by the interface's node a,
// one record array per direction): the cotangents it owes each node it read.
enum {
  RQA = 0,    // conserved state at a (5), then at b, a-1, b+1 (5 each)
  RQB = 5,
  RQM = 10,
  RQP = 15,
  RPA = 20,   // pressure at a, b, a-1, b+1
  RUA = 24,   // u, v, w, T at a (4), then at b
  RUB = 28,
  RG1 = 32,   // tangential derivative cotangents g1 (T1) and g2 (T2): +g at
  RG2 = 36,   //   a+t and b+t, -g at a-t and b-t, per component (4 each)
  RNUA = 40,  // sensor of direction D at a, at b
  RNUB = 41,
  RLB = 42,   // half the lbar cotangent (a and b each)
  RMU = 43,   // half the mu_eff and kappa_eff cotangents (a and b each)
  RKA = 44,
  NREC = 45
};

// face-shifted centre triple of the pressure sensor of node x along D
template <int D>
__device__ __forceinline__ void sensor_triple(const Grid& g, long long x, int cx, long long& xm,
                                              long long& xc, long long& xp) {
  const long long s = g.stride[D];
  const int nd = g.n[D];
  xc = x;
  int cc = cx;
  if (!g.per[D]) {
    if (cx == 0) {
      xc = x + s;
      cc = 1;
    } else if (cx == nd - 1) {
      xc = x - s;
      cc = nd - 2;
    }
  }
  xp = (cc == nd - 1) ? xc - (long long)(nd - 1) * s : xc + s;
  xm = (cc == 0) ? xc + (long long)(nd - 1) * s : xc - s;
}

__device__ __forceinline__ double sgn_abs(double x) { return x < 0.0 ? -1.0 : 1.0; }

// ------------------------------------------------------------- interface
template <int D>
__global__ void __launch_bounds__(256, 2) k_adj_iface(Grid g, Consts<double> K,
                                                   const double* __restrict__ Q,
                                                   const double* __restrict__ M,
                                                   const double* __restrict__ node,
                                                   const double* __restrict__ mk,
                                                   const double* __restrict__ lamR,
                                                   double* __restrict__ Rec,
                                                   const double* __restrict__ NU) {
  constexpr int T1 = (D + 1) % 3, T2 = (D + 2) % 3;
  const long long N = g.N;
  const double* U = node;
  const double* V = node + N;
  const double* Wv = node + 2 * N;
  const double* P = node + 3 * N;
  const double* Tt = node + 4 * N;
  const double* LB = node + (5 + D) * N;
  for (long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x; n < N;
       n += (long long)gridDim.x * blockDim.x) {
    int c[3];
    decompose(g, n, c);
    // no interface here, or no cotangent on it: an empty record
    auto empty = [&]() {
#pragma unroll 1
      for (int r = 0; r < NREC; ++r) Rec[(long long)r * N + n] = 0.0;
    };
    if ((!g.per[D] && c[D] == g.n[D] - 1) ||
        (!g.per[T1] && (c[T1] == 0 || c[T1] == g.n[T1] - 1)) ||
        (!g.per[T2] && (c[T2] == 0 || c[T2] == g.n[T2] - 1))) {
      empty();
      continue;
    }
    const long long a = n;
    const long long b = step(g, n, c, D, 1);
    int cb[3] = {c[0], c[1], c[2]};
    cb[D] = (c[D] + 1 == g.n[D]) ? 0 : c[D] + 1;
    // the residual is defined (and differentiated) on interior nodes only
    const bool a_in = g.per[D] || (c[D] > 0 && c[D] < g.n[D] - 1);
    const bool b_in = g.per[D] || (cb[D] > 0 && cb[D] < g.n[D] - 1);
    double lF[5];
    bool any = false;
#pragma unroll
    for (int q = 0; q < 5; ++q) {
      lF[q] = (a_in ? lamR[q * N + a] : 0.0) - (b_in ? lamR[q * N + b] : 0.0);
      any = any || lF[q] != 0.0;
    }
    if (!any) {
      empty();
      continue;
    }
    const long long am = step(g, n, c, D, -1);
    const long long bp = step(g, n, c, D, 2);

    // ---- forward recompute
    const double Ja = M[9 * N + a], Jb = M[9 * N + b];
    const double ma0 = M[(3 * D) * N + a], ma1 = M[(3 * D + 1) * N + a], ma2 = M[(3 * D + 2) * N + a];
    const double mb0 = M[(3 * D) * N + b], mb1 = M[(3 * D + 1) * N + b], mb2 = M[(3 * D + 2) * N + b];
    const double pa = P[a], pb = P[b];
    const double tha = ma0 * U[a] + ma1 * V[a] + ma2 * Wv[a];
    const double thb = mb0 * U[b] + mb1 * V[b] + mb2 * Wv[b];
    double Qa[5], Qb[5];
#pragma unroll
    for (int q = 0; q < 5; ++q) {
      Qa[q] = Q[q * N + a];
      Qb[q] = Q[q * N + b];
    }
    // the two nodes' sensors, as the forward read them (k_sensor of this
    // stage input)
    const double nua = NU[D * N + a], nub = NU[D * N + b];
    // forward: dev_max(nua, nub) = nua > nub ? nua : nub; max(0, x) keeps x for x >= 0
    const bool pick_b = !(nua > nub);
    const double eps2 = K.k2 * (pick_b ? nub : nua);
    const bool e4on = !(0.0 > K.k4 - eps2);
    const double eps4 = e4on ? K.k4 - eps2 : 0.0;
    const double lam = 0.5 * (LB[a] + LB[b]);
    const double Jh = 0.5 * (Ja + Jb);
    double Wa[5], Wb[5], Wm[5], Wp[5], D1[5], D3[5];
#pragma unroll
    for (int q = 0; q < 5; ++q) {
      Wa[q] = (q == 4) ? Qa[4] + pa : Qa[q];
      Wb[q] = (q == 4) ? Qb[4] + pb : Qb[q];
      Wm[q] = (am >= 0) ? ((q == 4) ? Q[4 * N + am] + P[am] : Q[q * N + am]) : 0.0;
      Wp[q] = (bp >= 0) ? ((q == 4) ? Q[4 * N + bp] + P[bp] : Q[q * N + bp]) : 0.0;
      D1[q] = Wb[q] - Wa[q];
      const double Dm = (am >= 0) ? Wa[q] - Wm[q] : -D1[q];
      const double Dp = (bp >= 0) ? Wp[q] - Wb[q] : -D1[q];
      D3[q] = Dp - 2.0 * D1[q] + Dm;
    }
    const double* phi[4] = {U, V, Wv, Tt};
    long long tn[2][4];  // tangential nodes: a+t, a-t, b+t, b-t for t = T1, T2
    tn[0][0] = step(g, a, c, T1, 1);
    tn[0][1] = step(g, a, c, T1, -1);
    tn[0][2] = step(g, b, cb, T1, 1);
    tn[0][3] = step(g, b, cb, T1, -1);
    tn[1][0] = step(g, a, c, T2, 1);
    tn[1][1] = step(g, a, c, T2, -1);
    tn[1][2] = step(g, b, cb, T2, 1);
    tn[1][3] = step(g, b, cb, T2, -1);
    double dphi[4][3];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      dphi[q][D] = phi[q][b] - phi[q][a];
      dphi[q][T1] = 0.25 * ((phi[q][tn[0][0]] - phi[q][tn[0][1]]) + (phi[q][tn[0][2]] - phi[q][tn[0][3]]));
      dphi[q][T2] = 0.25 * ((phi[q][tn[1][0]] - phi[q][tn[1][1]]) + (phi[q][tn[1][2]] - phi[q][tn[1][3]]));
    }
    double mh[3][3];
#pragma unroll
    for (int t = 0; t < 3; ++t)
#pragma unroll
      for (int x = 0; x < 3; ++x) mh[t][x] = 0.5 * (M[(3 * t + x) * N + a] + M[(3 * t + x) * N + b]);
    double gr[4][3];
#pragma unroll
    for (int q = 0; q < 4; ++q)
#pragma unroll
      for (int x = 0; x < 3; ++x)
        gr[q][x] = mh[0][x] * dphi[q][0] + mh[1][x] * dphi[q][1] + mh[2][x] * dphi[q][2];
    const double mu = 0.5 * (mk[a] + mk[b]);
    const double kap = 0.5 * (mk[N + a] + mk[N + b]);
    const double div = gr[0][0] + gr[1][1] + gr[2][2];
    const double two3 = 2.0 / 3.0;
    const double txx = mu * (2.0 * gr[0][0] - two3 * div);
    const double tyy = mu * (2.0 * gr[1][1] - two3 * div);
    const double tzz = mu * (2.0 * gr[2][2] - two3 * div);
    const double txy = mu * (gr[0][1] + gr[1][0]);
    const double txz = mu * (gr[0][2] + gr[2][0]);
    const double tyz = mu * (gr[1][2] + gr[2][1]);
    const double uf = 0.5 * (U[a] + U[b]), vf = 0.5 * (V[a] + V[b]), wf = 0.5 * (Wv[a] + Wv[b]);
    const double mx = mh[D][0], my = mh[D][1], mz = mh[D][2];

    // ---- reverse: F = Fq - Fv
    // Fv_1..3 = Jh (m . tau_row), Fv_4 = Jh (m . beta)
    const double lv1 = -lF[1], lv2 = -lF[2], lv3 = -lF[3], lv4 = -lF[4];
    double ltxx = Jh * mx * lv1, ltyy = Jh * my * lv2, ltzz = Jh * mz * lv3;
    double ltxy = Jh * (my * lv1 + mx * lv2), ltxz = Jh * (mz * lv1 + mx * lv3),
           ltyz = Jh * (mz * lv2 + my * lv3);
    const double lbx = Jh * mx * lv4, lby = Jh * my * lv4, lbz = Jh * mz * lv4;
    // beta_x = txx uf + txy vf + txz wf + kap grT_x, ...
    ltxx += lbx * uf;
    ltxy += lbx * vf + lby * uf;
    ltxz += lbx * wf + lbz * uf;
    ltyy += lby * vf;
    ltyz += lby * wf + lbz * vf;
    ltzz += lbz * wf;
    const double luf = lbx * txx + lby * txy + lbz * txz;
    const double lvf = lbx * txy + lby * tyy + lbz * tyz;
    const double lwf = lbx * txz + lby * tyz + lbz * tzz;
    const double lkap = lbx * gr[3][0] + lby * gr[3][1] + lbz * gr[3][2];
    double lgr[4][3];
    lgr[3][0] = kap * lbx;
    lgr[3][1] = kap * lby;
    lgr[3][2] = kap * lbz;
    // tau
    double lmu = ltxx * (2.0 * gr[0][0] - two3 * div) + ltyy * (2.0 * gr[1][1] - two3 * div) +
                 ltzz * (2.0 * gr[2][2] - two3 * div) + ltxy * (gr[0][1] + gr[1][0]) +
                 ltxz * (gr[0][2] + gr[2][0]) + ltyz * (gr[1][2] + gr[2][1]);
    const double ldiv = -two3 * mu * (ltxx + ltyy + ltzz);
    lgr[0][0] = 2.0 * mu * ltxx + ldiv;
    lgr[1][1] = 2.0 * mu * ltyy + ldiv;
    lgr[2][2] = 2.0 * mu * ltzz + ldiv;
    lgr[0][1] = mu * ltxy;
    lgr[1][0] = mu * ltxy;
    lgr[0][2] = mu * ltxz;
    lgr[2][0] = mu * ltxz;
    lgr[1][2] = mu * ltyz;
    lgr[2][1] = mu * ltyz;
    // gr[q][x] = sum_t mh[t][x] dphi[q][t]
    double ldphi[4][3];
#pragma unroll
    for (int q = 0; q < 4; ++q)
#pragma unroll
      for (int t = 0; t < 3; ++t)
        ldphi[q][t] = mh[t][0] * lgr[q][0] + mh[t][1] * lgr[q][1] + mh[t][2] * lgr[q][2];

    // Fq = (Fa + Fb)/2 - Jh lam (eps2 D1 - eps4 D3)
    double lWa[5] = {0, 0, 0, 0, 0}, lWb[5] = {0, 0, 0, 0, 0}, lWm[5] = {0, 0, 0, 0, 0},
           lWp[5] = {0, 0, 0, 0, 0};
    double llam = 0.0, leps2 = 0.0, leps4 = 0.0;
#pragma unroll
    for (int q = 0; q < 5; ++q) {
      const double ld = -Jh * lF[q];
      llam += ld * (eps2 * D1[q] - eps4 * D3[q]);
      leps2 += ld * lam * D1[q];
      leps4 -= ld * lam * D3[q];
      double lD1 = ld * lam * eps2;
      const double lD3 = -ld * lam * eps4;
      lD1 += -2.0 * lD3;
      if (am >= 0) {
        lWa[q] += lD3;
        lWm[q] -= lD3;
      } else {
        lD1 -= lD3;
      }
      if (bp >= 0) {
        lWp[q] += lD3;
        lWb[q] -= lD3;
      } else {
        lD1 -= lD3;
      }
      lWb[q] += lD1;
      lWa[q] -= lD1;
    }
    if (e4on) leps2 -= leps4;
    const double lnu = K.k2 * leps2;
    // centred flux: Fa_q = Ja (Qa_q tha + pa ma_q') ; Fa_4 = Ja (Qa4 + pa) tha
    double lQa[5], lQb[5];
    const double hFa[5] = {0.5 * lF[0], 0.5 * lF[1], 0.5 * lF[2], 0.5 * lF[3], 0.5 * lF[4]};
#pragma unroll
    for (int q = 0; q < 5; ++q) {
      lQa[q] = Ja * tha * hFa[q];
      lQb[q] = Jb * thb * hFa[q];
    }
    const double lpa_f = Ja * (ma0 * hFa[1] + ma1 * hFa[2] + ma2 * hFa[3] + tha * hFa[4]);
    const double lpb_f = Jb * (mb0 * hFa[1] + mb1 * hFa[2] + mb2 * hFa[3] + thb * hFa[4]);
    const double ltha = Ja * (Qa[0] * hFa[0] + Qa[1] * hFa[1] + Qa[2] * hFa[2] + Qa[3] * hFa[3] +
                              (Qa[4] + pa) * hFa[4]);
    const double lthb = Jb * (Qb[0] * hFa[0] + Qb[1] * hFa[1] + Qb[2] * hFa[2] + Qb[3] * hFa[3] +
                              (Qb[4] + pb) * hFa[4]);

    // ---- the record: conserved state and pressure (W4 = Q4 + p)
    auto put = [&](int r, double v) { Rec[(long long)r * N + n] = v; };
#pragma unroll
    for (int q = 0; q < 5; ++q) {
      put(RQA + q, lQa[q] + lWa[q]);
      put(RQB + q, lQb[q] + lWb[q]);
      put(RQM + q, am >= 0 ? lWm[q] : 0.0);
      put(RQP + q, bp >= 0 ? lWp[q] : 0.0);
    }
    put(RPA, lpa_f + lWa[4]);
    put(RPA + 1, lpb_f + lWb[4]);
    put(RPA + 2, am >= 0 ? lWm[4] : 0.0);
    put(RPA + 3, bp >= 0 ? lWp[4] : 0.0);
    // velocities: contravariant velocity and interface mean
    put(RUA + 0, ma0 * ltha + 0.5 * luf - ldphi[0][D]);
    put(RUA + 1, ma1 * ltha + 0.5 * lvf - ldphi[1][D]);
    put(RUA + 2, ma2 * ltha + 0.5 * lwf - ldphi[2][D]);
    put(RUA + 3, -ldphi[3][D]);
    put(RUB + 0, mb0 * lthb + 0.5 * luf + ldphi[0][D]);
    put(RUB + 1, mb1 * lthb + 0.5 * lvf + ldphi[1][D]);
    put(RUB + 2, mb2 * lthb + 0.5 * lwf + ldphi[2][D]);
    put(RUB + 3, ldphi[3][D]);
    // tangential derivatives: 1/4 (phi(a+t) - phi(a-t) + phi(b+t) - phi(b-t))
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      put(RG1 + q, 0.25 * ldphi[q][T1]);
      put(RG2 + q, 0.25 * ldphi[q][T2]);
    }
    // sensor, spectral radius, viscosity
    put(RNUA, pick_b ? 0.0 : lnu);
    put(RNUB, pick_b ? lnu : 0.0);
    put(RLB, 0.5 * llam);
    put(RMU, 0.5 * lmu);
    put(RKA, 0.5 * lkap);
  }
}

// Per node, in a fixed order (direction 0, 1, 2; then the roles), the sum of
// what the interface records owe it: as node a of the interface at n, as b
// of the one at n - e_D, as a - 1 of the one at n + e_D, as b + 1 of the one
// at n - 2 e_D, and as a tangential neighbour (a + t, a - t, b + t, b - t)
// of the interfaces at n - e_t, n + e_t, n - e_t - e_D, n + e_t - e_D.
// Writes every accumulator slot of every node (the sensor pass adds to the
// pressure slot afterwards).  One output slot at a time (its own fixed
// order of terms), so few accumulators are live and the kernel keeps
// enough warps resident to cover its memory latency.
__global__ void __launch_bounds__(256) k_adj_gather(Grid g, const double* __restrict__ R0,
                                                   const double* __restrict__ R1,
                                                   const double* __restrict__ R2,
                                                   double* __restrict__ A) {
  const long long N = g.N;
  const double* Rd[3] = {R0, R1, R2};
  for (long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x; n < N;
       n += (long long)gridDim.x * blockDim.x) {
    int c[3];
    decompose(g, n, c);
    long long mB[3], mM[3], mP[3];  // interfaces whose b, a - 1, b + 1 is n
#pragma unroll
    for (int D = 0; D < 3; ++D) {
      mB[D] = step(g, n, c, D, -1);
      mM[D] = step(g, n, c, D, 1);
      mP[D] = step(g, n, c, D, -2);
    }
    auto rec = [&](int D, int r, long long m) { return m >= 0 ? Rd[D][(long long)r * N + m] : 0.0; };
    // conserved state (k < 5) and pressure (k = 5): four roles per direction
#pragma unroll 1
    for (int k = 0; k < 6; ++k) {
      const int ra = k < 5 ? RQA + k : RPA, rb = k < 5 ? RQB + k : RPA + 1;
      const int rm = k < 5 ? RQM + k : RPA + 2, rp = k < 5 ? RQP + k : RPA + 3;
      double acc = 0.0;
#pragma unroll
      for (int D = 0; D < 3; ++D)
        acc += ((rec(D, ra, n) + rec(D, rb, mB[D])) + rec(D, rm, mM[D])) + rec(D, rp, mP[D]);
      A[(k < 5 ? AQ0 + k : AP) * N + n] = acc;
    }
    // u, v, w, T: as a and b, then as a tangential neighbour along T1, T2
#pragma unroll 1
    for (int k = 0; k < 4; ++k) {
      double acc = 0.0;
#pragma unroll
      for (int D = 0; D < 3; ++D) {
        acc += rec(D, RUA + k, n) + rec(D, RUB + k, mB[D]);
#pragma unroll
        for (int s = 1; s <= 2; ++s) {
          const int t = (D + s) % 3;
          const int G = (s == 1) ? RG1 : RG2;
          const long long tm = step(g, n, c, t, -1), tp = step(g, n, c, t, 1);
          long long tmb = -1, tpb = -1;  // n - e_t - e_D, n + e_t - e_D
          if (tm >= 0) {
            int ct[3] = {c[0], c[1], c[2]};
            ct[t] = coord_step(g, c, t, -1);
            tmb = step(g, tm, ct, D, -1);
          }
          if (tp >= 0) {
            int ct[3] = {c[0], c[1], c[2]};
            ct[t] = coord_step(g, c, t, 1);
            tpb = step(g, tp, ct, D, -1);
          }
          acc += ((rec(D, G + k, tm) - rec(D, G + k, tp)) + rec(D, G + k, tmb)) - rec(D, G + k, tpb);
        }
      }
      A[(AU + k) * N + n] = acc;
    }
    // sensor and lbar of each direction; mu_eff and kappa_eff over the three
#pragma unroll
    for (int D = 0; D < 3; ++D) {
      A[(ANU + D) * N + n] = rec(D, RNUA, n) + rec(D, RNUB, mB[D]);
      A[(ALB + D) * N + n] = rec(D, RLB, n) + rec(D, RLB, mB[D]);
    }
    double mu = 0.0, ka = 0.0;
#pragma unroll
    for (int D = 0; D < 3; ++D) {
      mu += rec(D, RMU, n) + rec(D, RMU, mB[D]);
      ka += rec(D, RKA, n) + rec(D, RKA, mB[D]);
    }
    A[AMU * N + n] = mu;
    A[(AMU + 1) * N + n] = ka;
  }
}

// Sensor cotangents to the pressures of the (face-shifted) centre triple:
// per node x and direction d the two terms it owes (ls + lden to its outer
// pair, -2 ls + 2 lden to its centre) into ST[2 d], ST[2 d + 1]; then each
// node gathers, in a fixed order, the terms of the nodes whose triple holds
// it (x within two nodes along d).
__global__ void k_adj_sensor_terms(Grid g, const double* __restrict__ node,
                                   const double* __restrict__ A, double* __restrict__ ST) {
  const long long N = g.N;
  const double* P = node + 3 * N;
  for (long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x; n < N;
       n += (long long)gridDim.x * blockDim.x) {
    int c[3];
    decompose(g, n, c);
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      const double ln = A[(ANU + d) * N + n];
      double outer = 0.0, centre = 0.0;
      if (ln != 0.0) {
        long long xm, xc, xp;
        if (d == 0) sensor_triple<0>(g, n, c[0], xm, xc, xp);
        else if (d == 1) sensor_triple<1>(g, n, c[1], xm, xc, xp);
        else sensor_triple<2>(g, n, c[2], xm, xc, xp);
        const double s = P[xp] - 2.0 * P[xc] + P[xm];
        const double den = P[xp] + 2.0 * P[xc] + P[xm];
        // nu = |s| / den
        const double iden = 1.0 / den;
        const double ls = ln * sgn_abs(s) * iden;
        const double lden = -ln * fabs(s) * iden * iden;
        outer = ls + lden;
        centre = -2.0 * ls + 2.0 * lden;
      }
      ST[(2 * d) * N + n] = outer;
      ST[(2 * d + 1) * N + n] = centre;
    }
  }
}

__global__ void k_adj_sensor_gather(Grid g, const double* __restrict__ ST, double* __restrict__ A) {
  const long long N = g.N;
  for (long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x; n < N;
       n += (long long)gridDim.x * blockDim.x) {
    int c[3];
    decompose(g, n, c);
    double add = 0.0;
#pragma unroll
    for (int d = 0; d < 3; ++d) {
#pragma unroll
      for (int off = -2; off <= 2; ++off) {
        const long long x = step(g, n, c, d, off);
        if (x < 0) continue;
        int cx[3] = {c[0], c[1], c[2]};
        cx[d] = coord_step(g, c, d, off);
        long long xm, xc, xp;
        if (d == 0) sensor_triple<0>(g, x, cx[0], xm, xc, xp);
        else if (d == 1) sensor_triple<1>(g, x, cx[1], xm, xc, xp);
        else sensor_triple<2>(g, x, cx[2], xm, xc, xp);
        if (xp == n) add += ST[(2 * d) * N + x];
        if (xc == n) add += ST[(2 * d + 1) * N + x];
        if (xm == n) add += ST[(2 * d) * N + x];
      }
    }
    A[AP * N + n] += add;
  }
}

// Node quantities back to Q: radii lbar(lambda_d), lambda_d = |m_d.u| +
// sqrt(T)|grad d|, then u = Q1/rho, p = (g-1)(Q4 - rho|u|^2/2), T = g p/rho.
// lamQ = direct + chained; mu/kappa cotangents are added to lamMK.  |grad d|
// comes from gn ([3][N], set-up) when given, else from M.
__global__ void __launch_bounds__(256, 2) k_adj_node(Grid g, Consts<double> K, const double* __restrict__ Q,
                           const double* __restrict__ M, const double* __restrict__ gn,
                           const double* __restrict__ node,
                           const double* __restrict__ A, double* __restrict__ lamQ,
                           double* __restrict__ lamMK) {
  const long long N = g.N;
  for (long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x; n < N;
       n += (long long)gridDim.x * blockDim.x) {
    const double rho = Q[n];
    const double ir = 1.0 / rho;
    const double u = node[n], v = node[N + n], w = node[2 * N + n], p = node[3 * N + n],
                 T = node[4 * N + n];
    double lu = A[(AU + 0) * N + n], lv = A[(AU + 1) * N + n], lw = A[(AU + 2) * N + n];
    double lT = A[(AU + 3) * N + n], lp = A[AP * N + n];
    // lbar -> lambda
    const double llb0 = A[(ALB + 0) * N + n], llb1 = A[(ALB + 1) * N + n], llb2 = A[(ALB + 2) * N + n];
    if (llb0 != 0.0 || llb1 != 0.0 || llb2 != 0.0) {
      const double a = sqrt(T);
      double l[3], th[3], gm[3];
#pragma unroll
      for (int d = 0; d < 3; ++d) {
        const double mx = M[(3 * d) * N + n], my = M[(3 * d + 1) * N + n], mz = M[(3 * d + 2) * N + n];
        th[d] = mx * u + my * v + mz * w;
        gm[d] = gn ? gn[d * N + n] : sqrt(mx * mx + my * my + mz * mz);
        l[d] = fabs(th[d]) + a * gm[d];
      }
      const double s01 = sqrt(l[0] * l[1]), s02 = sqrt(l[0] * l[2]), s12 = sqrt(l[1] * l[2]);
      const double c01 = llb0 + llb1, c02 = llb0 + llb2, c12 = llb1 + llb2;
      // d sqrt(l_a l_b)/d l_a = l_b/(2 sqrt(l_a l_b)): one reciprocal per pair
      const double h01 = c01 / (2.0 * s01), h02 = c02 / (2.0 * s02), h12 = c12 / (2.0 * s12);
      double ll[3];
      ll[0] = llb0 + h01 * l[1] + h02 * l[2];
      ll[1] = llb1 + h01 * l[0] + h12 * l[2];
      ll[2] = llb2 + h02 * l[0] + h12 * l[1];
      double la = 0.0;
#pragma unroll
      for (int d = 0; d < 3; ++d) {
        const double lth = ll[d] * sgn_abs(th[d]);
        lu += M[(3 * d) * N + n] * lth;
        lv += M[(3 * d + 1) * N + n] * lth;
        lw += M[(3 * d + 2) * N + n] * lth;
        la += ll[d] * gm[d];
      }
      lT += la / (2.0 * a);
    }
    // T = gamma p / rho
    lp += K.gamma * ir * lT;
    double lrho = -K.gamma * p * ir * ir * lT;
    // p = (gamma-1)(Q4 - rho |u|^2 / 2)
    double lQ4 = K.gm1 * lp;
    lrho += -0.5 * K.gm1 * (u * u + v * v + w * w) * lp;
    lu += -K.gm1 * rho * u * lp;
    lv += -K.gm1 * rho * v * lp;
    lw += -K.gm1 * rho * w * lp;
    // u = Q1 / rho
    const double lQ1 = ir * lu, lQ2 = ir * lv, lQ3 = ir * lw;
    lrho += -ir * (u * lu + v * lv + w * lw);
    lamQ[n] = A[AQ0 * N + n] + lrho;
    lamQ[N + n] = A[(AQ0 + 1) * N + n] + lQ1;
    lamQ[2 * N + n] = A[(AQ0 + 2) * N + n] + lQ2;
    lamQ[3 * N + n] = A[(AQ0 + 3) * N + n] + lQ3;
    lamQ[4 * N + n] = A[(AQ0 + 4) * N + n] + lQ4;
    if (lamMK) {
      lamMK[n] += A[AMU * N + n];
      lamMK[N + n] += A[(AMU + 1) * N + n];
    }
  }
}

// Sutherland viscosity (no SGS model): mu = s T^1.5 (1+S)/(T+S), kappa =
// mu/((g-1)Pr), T = g p/rho of Q^n; adds the Q cotangent to lamQ.
__global__ void k_adj_mu(Grid g, Consts<double> K, const double* __restrict__ Q,
                         const double* __restrict__ lamMK, double* __restrict__ lamQ) {
  const long long N = g.N;
  for (long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x; n < N;
       n += (long long)gridDim.x * blockDim.x) {
    const double lmu = lamMK[n] + lamMK[N + n] * K.inv_gm1_pr;
    if (lmu == 0.0) continue;
    const double rho = Q[n], ir = 1.0 / rho;
    const double u = Q[N + n] * ir, v = Q[2 * N + n] * ir, w = Q[3 * N + n] * ir;
    const double p = K.gm1 * (Q[4 * N + n] - 0.5 * rho * (u * u + v * v + w * w));
    const double T = K.gamma * p * ir;
    const double S = K.S_suth;
    const double sq = sqrt(T);
    // d/dT [T^1.5 / (T+S)] = (1.5 sqrt(T)(T+S) - T^1.5)/(T+S)^2
    const double dmu = K.mu_scale * (1.0 + S) * (1.5 * sq * (T + S) - T * sq) / ((T + S) * (T + S));
    const double lT = dmu * lmu;
    const double lp = K.gamma * ir * lT;
    double lrho = -K.gamma * p * ir * ir * lT;
    lrho += -0.5 * K.gm1 * (u * u + v * v + w * w) * lp;
    const double lu = -K.gm1 * rho * u * lp, lv = -K.gm1 * rho * v * lp, lw = -K.gm1 * rho * w * lp;
    lrho += -ir * (u * lu + v * lv + w * lw);
    lamQ[n] += lrho;
    lamQ[N + n] += ir * lu;
    lamQ[2 * N + n] += ir * lv;
    lamQ[3 * N + n] += ir * lw;
    lamQ[4 * N + n] += K.gm1 * lp;
  }
}

// ------------------------------------------------------------ RK helpers
// lamR = -alpha dt J lamS on interior nodes, 0 on boundary nodes; lamQ0 += lamS
__global__ void k_adj_stage_prep(Grid g, const double* __restrict__ M, double coef,
                                 const double* __restrict__ lamS, double* __restrict__ lamR,
                                 double* __restrict__ lamQ0) {
  const long long N = g.N;
  for (long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x; n < N;
       n += (long long)gridDim.x * blockDim.x) {
    int c[3];
    decompose(g, n, c);
    const bool in = is_interior(g, c);
    const double Jn = 1.0 / M[9 * N + n];
#pragma unroll
    for (int q = 0; q < 5; ++q) {
      const double ls = lamS[q * N + n];
      lamQ0[q * N + n] += ls;
      lamR[q * N + n] = in ? -coef * Jn * ls : 0.0;
    }
  }
}

__global__ void k_axpy(long long count, double a, const double* __restrict__ x, double* __restrict__ y) {
  for (long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x; n < count;
       n += (long long)gridDim.x * blockDim.x)
    y[n] += a * x[n];
}

// ------------------------------------------------------- boundary reverse
template <typename T>
__device__ void farfield_formula(const T qe[5], double nx, double ny, double nz, double gamma,
                                 T qf[5]) {
  const double gm1 = gamma - 1.0;
  const T rho = qe[0];
  const T u = qe[1] / rho, v = qe[2] / rho, w = qe[3] / rho;
  const T p = gm1 * (qe[4] - 0.5 * rho * (u * u + v * v + w * w));
  const T ae = sqrt(gamma * p / rho);
  const T qne = u * nx + v * ny + w * nz;
  const T Rp = qne + 2.0 * ae / gm1;
  const double Rm = 0.0 - 2.0 * 1.0 / gm1;
  const T qnf = 0.5 * (Rp + Rm);
  const T af = 0.25 * gm1 * (Rp - Rm);
  const T Mn = qne / ae;
  T rf, uf, vf, wf, pf;
  if (Mn >= 1.0) {
    for (int q = 0; q < 5; ++q) qf[q] = qe[q];
    return;
  } else if (Mn >= 0.0) {
    const T dq = qnf - qne;
    rf = pow(pow(rho, gamma) * af * af / (gamma * p), 1.0 / gm1);
    uf = u + dq * nx;
    vf = v + dq * ny;
    wf = w + dq * nz;
    pf = rf * af * af / gamma;
  } else if (Mn > -1.0) {
    rf = pow(af * af / (gamma * (1.0 / gamma)), 1.0 / gm1);
    uf = qnf * nx;
    vf = qnf * ny;
    wf = qnf * nz;
    pf = rf * af * af / gamma;
  } else {
    rf = T(1.0);
    uf = T(0.0);
    vf = T(0.0);
    wf = T(0.0);
    pf = T(1.0 / gamma);
  }
  qf[0] = rf;
  qf[1] = rf * uf;
  qf[2] = rf * vf;
  qf[3] = rf * wf;
  qf[4] = pf / gm1 + 0.5 * rf * (uf * uf + vf * vf + wf * wf);
}

template <typename T>
__device__ void exit_formula(const T qe[5], double ex, double ey, double ez, double gamma, T qo[5]) {
  const double gm1 = gamma - 1.0;
  const double inv = 1.0 / ::sqrt(ex * ex + ey * ey + ez * ez);
  const T rho = qe[0];
  const T u = qe[1] / rho, v = qe[2] / rho, w = qe[3] / rho;
  const T p = gm1 * (qe[4] - 0.5 * rho * (u * u + v * v + w * w));
  const T ae = sqrt(gamma * p / rho);
  const T qn = (u * ex + v * ey + w * ez) * inv;
  if (qn / ae >= 1.0) {
    for (int q = 0; q < 5; ++q) qo[q] = qe[q];
    return;
  }
  const T eint = p / (gm1 * rho);
  const T rf = (1.0 / gamma) / (gm1 * eint);
  qo[0] = rf;
  qo[1] = rf * u;
  qo[2] = rf * v;
  qo[3] = rf * w;
  qo[4] = rf * (eint + 0.5 * (u * u + v * v + w * w));
}

// out += J^T lam for a 5 -> 5 map evaluated by forward-mode dual numbers
template <int KIND>
__device__ void local_vjp(const double qe[5], double a0, double a1, double a2, double gamma,
                          const double lam[5], double out[5]) {
#pragma unroll 1
  for (int i = 0; i < 5; ++i) {
    Dual x[5], y[5];
    for (int q = 0; q < 5; ++q) x[q] = Dual(qe[q], q == i ? 1.0 : 0.0);
    if (KIND == 0)
      farfield_formula<Dual>(x, a0, a1, a2, gamma, y);
    else
      exit_formula<Dual>(x, a0, a1, a2, gamma, y);
    double s = 0.0;
    for (int q = 0; q < 5; ++q) s += y[q].d * lam[q];
    out[i] += s;
  }
}

// lamS = lamNext on interior nodes, 0 on boundary nodes (their stage values
// are overwritten by the boundary conditions)
__global__ void k_adjbc_init(Grid g, const double* __restrict__ lamNext, double* __restrict__ lamS) {
  const long long N = g.N;
  for (long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x; n < N;
       n += (long long)gridDim.x * blockDim.x) {
    int c[3];
    decompose(g, n, c);
    const bool in = is_interior(g, c);
#pragma unroll
    for (int q = 0; q < 5; ++q) lamS[q * N + n] = in ? lamNext[q * N + n] : 0.0;
  }
}

// exit: the plane i = ni-1 copies / extrapolates the post-phase-1 column
// i = ni-2 (taken from Qnext).  Interior rows go straight into lamS; the two
// face rows (j = 0, nj-1) go to E for the ring / far-field reverse.
__global__ void k_adjbc_exit(Grid g, double gamma, const double* __restrict__ M,
                             const double* __restrict__ Qnext, const double* __restrict__ lamNext,
                             double* __restrict__ lamS, double* __restrict__ E) {
  const int ni = g.n[0], nj = g.n[1], nk = g.n[2];
  const long long plane = (long long)nj * nk, N = g.N;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < plane;
       e += (long long)gridDim.x * blockDim.x) {
    const int j = (int)(e / nk);
    const long long nx_ = (long long)(ni - 1) * plane + e, ne = nx_ - plane;
    double qe[5], lam[5], out[5] = {0, 0, 0, 0, 0};
    for (int q = 0; q < 5; ++q) {
      qe[q] = Qnext[q * N + ne];
      lam[q] = lamNext[q * N + nx_];
    }
    local_vjp<1>(qe, M[nx_], M[N + nx_], M[2 * N + nx_], gamma, lam, out);
    if (j == 0 || j == nj - 1) {
      for (int q = 0; q < 5; ++q) E[q * plane + e] = out[q];
    } else {
      for (int q = 0; q < 5; ++q) lamS[q * N + ne] += out[q];
    }
  }
}

// far field: node (i, nj-1, k) from (i, nj-2, k) of the stage-5 state
__global__ void k_adjbc_farfield(Grid g, double gamma, const double* __restrict__ M,
                                 const double* __restrict__ S5, const double* __restrict__ lamNext,
                                 const double* __restrict__ E, double* __restrict__ lamS) {
  const int ni = g.n[0], nj = g.n[1], nk = g.n[2];
  const long long count = (long long)(ni - 2) * nk, N = g.N, plane = (long long)nj * nk;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < count;
       e += (long long)gridDim.x * blockDim.x) {
    const int i = 1 + (int)(e / nk), k = (int)(e % nk);
    const long long nf = idx3(g, i, nj - 1, k), ne = idx3(g, i, nj - 2, k);
    const double ex = M[3 * N + nf], ey = M[4 * N + nf], ez = M[5 * N + nf];
    const double inv = 1.0 / sqrt(ex * ex + ey * ey + ez * ez);
    double qe[5], lam[5], out[5] = {0, 0, 0, 0, 0};
    for (int q = 0; q < 5; ++q) {
      qe[q] = S5[q * N + ne];
      lam[q] = lamNext[q * N + nf] + (i == ni - 2 ? E[q * plane + (long long)(nj - 1) * nk + k] : 0.0);
    }
    local_vjp<0>(qe, ex * inv, ey * inv, ez * inv, gamma, lam, out);
    for (int q = 0; q < 5; ++q) lamS[q * N + ne] += out[q];
  }
}

// inner ring: Q(i,0,k) = mean_k S5(i,1,k), one block per axial station
__global__ void k_adjbc_ring(Grid g, const double* __restrict__ lamNext, const double* __restrict__ E,
                             double* __restrict__ lamS) {
  const int i = 1 + blockIdx.x;
  const int ni = g.n[0], nk = g.n[2];
  const long long N = g.N;
  __shared__ double red[5][32];
  double s[5] = {0, 0, 0, 0, 0};
  const long long base0 = idx3(g, i, 0, 0), base1 = idx3(g, i, 1, 0);
  for (int k = threadIdx.x; k < nk; k += blockDim.x)
    for (int q = 0; q < 5; ++q)
      s[q] += lamNext[q * N + base0 + k] + (i == ni - 2 ? E[q * (long long)g.n[1] * nk + k] : 0.0);
  for (int q = 0; q < 5; ++q)
    for (int off = 16; off > 0; off >>= 1) s[q] += __shfl_xor_sync(0xffffffffu, s[q], off);
  if ((threadIdx.x & 31) == 0)
    for (int q = 0; q < 5; ++q) red[q][threadIdx.x >> 5] = s[q];
  __syncthreads();
  if (threadIdx.x < 32) {
    for (int q = 0; q < 5; ++q) {
      double v = threadIdx.x < (blockDim.x >> 5) ? red[q][threadIdx.x] : 0.0;
      for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
      if (threadIdx.x == 0) red[q][0] = v / (double)nk;
    }
  }
  __syncthreads();
  for (int k = threadIdx.x; k < nk; k += blockDim.x)
    for (int q = 0; q < 5; ++q) lamS[q * N + base1 + k] += red[q][0];
}

// entrance: Q = (1, u, 0, 0, p/(g-1) + u^2/2), u = profile + sum a_mf g(r)
// cos(m theta - 2 pi St_f Mj t): grad_mf += sum over the plane of
// (lam1 + u lam4) g(r) cos(...); one partial per block and mode.
__global__ void k_adjbc_inflow(Grid g, double Mj, double r_jet, double theta_m, double width,
                               const double* __restrict__ St, const double* __restrict__ amp,
                               const double* __restrict__ rth, double t,
                               const double* __restrict__ lamNext, double* __restrict__ partials) {
  const long long plane = (long long)g.n[1] * g.n[2], N = g.N;
  const double two_pi = 6.283185307179586476925286766559;
  double acc[16];
  for (int m = 0; m < 16; ++m) acc[m] = 0.0;
  for (long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x; n < plane;
       n += (long long)gridDim.x * blockDim.x) {
    const double r = rth[n], th = rth[plane + n];
    double u = 0.5 * Mj * (1.0 + tanh((r_jet - r) / (2.0 * theta_m)));
    const double x = (r - r_jet) / width;
    const double gr = exp(-(x * x));
    double cs[16];
    for (int m = 0; m < 4; ++m)
      for (int f = 0; f < 4; ++f) {
        cs[m * 4 + f] = cos(m * th - two_pi * St[f] * Mj * t);
        u += amp[m * 4 + f] * gr * cs[m * 4 + f];
      }
    const double lu = lamNext[N + n] + u * lamNext[4 * N + n];
    for (int m = 0; m < 16; ++m) acc[m] += lu * gr * cs[m];
  }
  __shared__ double red[16][32];
  for (int m = 0; m < 16; ++m) {
    double v = acc[m];
    for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
    if ((threadIdx.x & 31) == 0) red[m][threadIdx.x >> 5] = v;
  }
  __syncthreads();
  if (threadIdx.x < 16) {
    double v = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) v += red[threadIdx.x][w];
    partials[blockIdx.x * 16 + threadIdx.x] = v;
  }
}

// grad[m] += sum of the block partials (fixed order)
__global__ void k_sum_partials16(const double* __restrict__ partials, int nb, double* __restrict__ grad) {
  const int m = threadIdx.x;
  if (m >= 16) return;
  double s = 0.0;
  for (int b = 0; b < nb; ++b) s += partials[b * 16 + m];
  grad[m] += s;
}

// ------------------------------------------------------------ functional
// J_f contribution of one state: dt sum_{i,k} (p(i, j5, k) - 1/gamma)^2 dA,
// dA = J^-1 |grad eta| (eta-face area); and its Q cotangent.
template <typename TM>
__global__ void k_functional(Grid g, double gamma, int j5, double dt, const TM* __restrict__ M,
                             const double* __restrict__ Q, double* __restrict__ lam,
                             double* __restrict__ partials) {
  const int ni = g.n[0], nk = g.n[2];
  const long long count = (long long)ni * nk, N = g.N;
  const double gm1 = gamma - 1.0;
  double acc = 0.0;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < count;
       e += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(e / nk), k = (int)(e % nk);
    const long long n = idx3(g, i, j5, k);
    const double ex = (double)M[3 * N + n], ey = (double)M[4 * N + n], ez = (double)M[5 * N + n];
    const double dA = (double)M[9 * N + n] * sqrt(ex * ex + ey * ey + ez * ez);
    const double rho = Q[n], u = Q[N + n] / rho, v = Q[2 * N + n] / rho, w = Q[3 * N + n] / rho;
    const double p = gm1 * (Q[4 * N + n] - 0.5 * rho * (u * u + v * v + w * w));
    const double dp = p - 1.0 / gamma;
    acc += dt * dp * dp * dA;
    if (lam) {
      const double lp = 2.0 * dt * dp * dA;
      lam[n] += lp * gm1 * 0.5 * (u * u + v * v + w * w);
      lam[N + n] += -lp * gm1 * u;
      lam[2 * N + n] += -lp * gm1 * v;
      lam[3 * N + n] += -lp * gm1 * w;
      lam[4 * N + n] += lp * gm1;
    }
  }
  for (int off = 16; off > 0; off >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off);
  __shared__ double red[32];
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += red[w];
    partials[blockIdx.x] = s;
  }
}

__global__ void k_sum_partials1(const double* __restrict__ partials, int nb, double* __restrict__ out) {
  if (threadIdx.x != 0) return;
  double s = 0.0;
  for (int b = 0; b < nb; ++b) s += partials[b];
  out[0] += s;
}

__global__ void k_pack_dual(long long count, const double* __restrict__ v,
                            const double* __restrict__ d, Dual* __restrict__ out) {
  for (long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x; n < count;
       n += (long long)gridDim.x * blockDim.x)
    out[n] = Dual(v[n], d ? d[n] : 0.0);
}

__global__ void k_unpack_dual(long long count, const Dual* __restrict__ in, double* __restrict__ v,
                              double* __restrict__ d) {
  for (long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x; n < count;
       n += (long long)gridDim.x * blockDim.x) {
    if (v) v[n] = in[n].v;
    d[n] = in[n].d;
  }
}

// ------------------------------------------------------------- launchers
constexpr int kAdjBlocks = kRedBlocks;  // fixed reduction grid (deterministic sums)

static int nb_for(long long count) {
  long long b = (count + 255) / 256;
  const long long cap = 32LL * sm_count();
  if (b > cap) b = cap;
  return (int)(b < 1 ? 1 : b);
}

void launch_rhs_vjp(const Grid& g, const les_params& p, const double* Q, const double* M,
                    const double* gn, const double* node, const double* mk, const double* lamR, double* acc,
                    double* lamQ, double* lamMK, const Launch& L, const double* nu) {
  // nu: the three sensors of the stage input (launch_sensor64 on node)
  const Consts<double> K = make_consts<double>(p);
  const int nb = nb_for(g.N);
  // acc holds the NACC accumulator slots, then the three directions' records
  double* rec = acc + (size_t)NACC * g.N;
  const size_t rs = (size_t)NREC * g.N;
  k_adj_iface<0><<<nb, 256, 0, L.s>>>(g, K, Q, M, node, mk, lamR, rec, nu);
  k_adj_iface<1><<<nb, 256, 0, L.s>>>(g, K, Q, M, node, mk, lamR, rec + rs, nu);
  k_adj_iface<2><<<nb, 256, 0, L.s>>>(g, K, Q, M, node, mk, lamR, rec + 2 * rs, nu);
  k_adj_gather<<<nb, 256, 0, L.s>>>(g, rec, rec + rs, rec + 2 * rs, acc);
  // the records are consumed: their space holds the sensor terms
  k_adj_sensor_terms<<<nb, 256, 0, L.s>>>(g, node, acc, rec);
  k_adj_sensor_gather<<<nb, 256, 0, L.s>>>(g, rec, acc);
  k_adj_node<<<nb, 256, 0, L.s>>>(g, K, Q, M, gn, node, acc, lamQ, lamMK);
  *L.counter += 7;
}

void launch_rhs_jvp(const Grid& g, const les_params& p, const Dual* Q, const double* M,
                    const Dual* mk, Dual* node, Dual* flux, Dual* R, const Launch& L) {
  const Consts<Dual> K = make_consts<Dual>(p);
  const int nb = nb_for(g.N);
  k_node<Dual, Dual, double, false><<<nb, 256, 0, L.s>>>(g, K, Q, M, nullptr, node, nullptr, nullptr);
  k_flux<0, Dual, Dual, double><<<nb, 256, 0, L.s>>>(g, K, Q, M, node, mk, flux);
  k_flux<1, Dual, Dual, double><<<nb, 256, 0, L.s>>>(g, K, Q, M, node, mk, flux + 5 * g.N);
  k_flux<2, Dual, Dual, double><<<nb, 256, 0, L.s>>>(g, K, Q, M, node, mk, flux + 10 * g.N);
  k_update<Dual, double, Dual, 0><<<nb, 256, 0, L.s>>>(g, flux, nullptr, M, nullptr, 0.0, R);
  *L.counter += 5;
}

void launch_pack_dual(long long count, const double* v, const double* d, Dual* out, const Launch& L) {
  k_pack_dual<<<nb_for(count), 256, 0, L.s>>>(count, v, d, out);
  ++*L.counter;
}

void launch_unpack_dual(long long count, const Dual* in, double* v, double* d, const Launch& L) {
  k_unpack_dual<<<nb_for(count), 256, 0, L.s>>>(count, in, v, d);
  ++*L.counter;
}

void launch_mu_vjp(const Grid& g, const les_params& p, const double* Q, const double* lamMK,
                   double* lamQ, const Launch& L) {
  k_adj_mu<<<nb_for(g.N), 256, 0, L.s>>>(g, make_consts<double>(p), Q, lamMK, lamQ);
  ++*L.counter;
}

void launch_stage_prep(const Grid& g, const double* M, double coef, const double* lamS,
                       double* lamR, double* lamQ0, const Launch& L) {
  k_adj_stage_prep<<<nb_for(g.N), 256, 0, L.s>>>(g, M, coef, lamS, lamR, lamQ0);
  ++*L.counter;
}

void launch_axpy(long long count, double a, const double* x, double* y, const Launch& L) {
  k_axpy<<<nb_for(count), 256, 0, L.s>>>(count, a, x, y);
  ++*L.counter;
}

void launch_bc_vjp(const Grid& g, const les_params& p, const double* M, const double* rth,
                   const double* S5, const double* Qnext, const double* lamNext, double t_next,
                   double* lamS, double* E, double* partials, double* grad, const Launch& L) {
  const long long plane = (long long)g.n[1] * g.n[2];
  k_adjbc_init<<<nb_for(g.N), 256, 0, L.s>>>(g, lamNext, lamS);
  k_adjbc_exit<<<nb_for(plane), 256, 0, L.s>>>(g, p.gamma, M, Qnext, lamNext, lamS, E);
  k_adjbc_farfield<<<nb_for((long long)(g.n[0] - 2) * g.n[2]), 256, 0, L.s>>>(g, p.gamma, M, S5,
                                                                               lamNext, E, lamS);
  k_adjbc_ring<<<g.n[0] - 2, 256, 0, L.s>>>(g, lamNext, E, lamS);
  // forcing parameters in a small device block after the partials
  double* par = partials + kAdjBlocks * 16;
  double hostpar[20];
  for (int i = 0; i < 4; ++i) hostpar[i] = p.St[i];
  for (int i = 0; i < 16; ++i) hostpar[4 + i] = p.amp[i];
  cudaMemcpyAsync(par, hostpar, sizeof(hostpar), cudaMemcpyHostToDevice, L.s);
  const int nbi = nb_for(plane) < kAdjBlocks ? nb_for(plane) : kAdjBlocks;
  k_adjbc_inflow<<<nbi, 256, 0, L.s>>>(g, p.Mj, p.r_jet, p.theta_m, p.force_width, par, par + 4,
                                       rth, t_next, lamNext, partials);
  k_sum_partials16<<<1, 32, 0, L.s>>>(partials, nbi, grad);
  *L.counter += 6;
}

void launch_functional(const Grid& g, const les_params& p, int j5, double dt, const double* M,
                       const double* Q, double* lam, double* partials, double* Jout,
                       const Launch& L) {
  const long long count = (long long)g.n[0] * g.n[2];
  const int nb = nb_for(count) < kAdjBlocks ? nb_for(count) : kAdjBlocks;
  k_functional<double><<<nb, 256, 0, L.s>>>(g, p.gamma, j5, dt, M, Q, lam, partials);
  k_sum_partials1<<<1, 32, 0, L.s>>>(partials, nb, Jout);
  *L.counter += 2;
}

void launch_functional(const Grid& g, const les_params& p, int j5, double dt, const float* M,
                       const double* Q, double* partials, double* Jout, const Launch& L) {
  const long long count = (long long)g.n[0] * g.n[2];
  const int nb = nb_for(count) < kAdjBlocks ? nb_for(count) : kAdjBlocks;
  k_functional<float><<<nb, 256, 0, L.s>>>(g, p.gamma, j5, dt, M, Q, nullptr, partials);
  k_sum_partials1<<<1, 32, 0, L.s>>>(partials, nb, Jout);
  *L.counter += 2;
}

}  // namespace lesjet
