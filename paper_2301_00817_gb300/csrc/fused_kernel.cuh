// fused_kernel.cuh -- one kernel per Runge-Kutta stage (residual + update
// fused), its helpers and launch templates; fused.cu holds the launchers,
// fused_jet12.cu and fused_jet28.cu the jet-grid instantiations.
//
// A CTA owns a TJ x TK = 16 x 32 tile of (eta, zeta) columns and marches along
// xi over a chunk of axial planes.  Per plane it stages the conserved state
// of the tile plus a two-node halo in shared memory with cp.async (one plane
// ahead), derives the primitives and the anisotropic spectral radii once per
// node, and keeps the own column's data of the neighbouring planes in
// registers.  Every interface flux (centred inviscid flux minus J^-1 times
// the Turkel-Vatsa dissipation minus the viscous flux) is computed once: the
// xi interface i+1/2 is carried in registers to the next plane, the eta and
// zeta interfaces are exchanged through shared memory.  The stage update
// Q^(l) = Q^(0) - alpha_l dt J RHS is applied in the epilogue, so the residual
// never touches HBM.
//
// This is the FP32-mixed form: it computes in float, stores the stage states
// and metrics in float, and keeps Q^(0) as an unevaluated float pair (hi +
// lo) updated with compensated (TwoSum) arithmetic in the last stage, so the
// steady state issues no FP64 instruction on GB300's narrow FP64 pipe.  The
// translation unit is built with approximate FP32 division and square root
// (their error is inside the form's measured error budget).
#pragma once

#include <atomic>
#include <functional>
#include <map>
#include <mutex>
#include <queue>
#include <utility>
#include <vector>

#include "lesjet_dev.cuh"
#include "lesjet_host.h"

namespace lesjet {

// Approximate reciprocal (rcp.approx.ftz: relative error below 2^-22),
// inside this form's FP32 error budget; cheaper than the correctly rounded
// __frcp_rn.
__device__ __forceinline__ float frcp_fast(float x) {
  float r;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}

__device__ __forceinline__ void cp_async4(void* smem, const void* gmem) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int NPEND>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(NPEND) : "memory");
}

// ----------------------------------------------------------- interface flux
// Flux through the interface between nodes a and b (b = a + e_D): centred
// inviscid flux (Eqs. hat-flux-G, inv_flux_vec) minus J^-1 d (Eqs.
// dissip_term, eps_2/4_dissip with the boundary closure of the centerline
// section) minus the viscous + SGS flux (Eqs. hat-flux-Ev/Fv/Gv, tau_mod,
// q_mod with Fourier's sign) from compact interface gradients.
// m*[0..8] = xi_x .. zeta_z, m*[9] = J^-1; W* = (rho, rho u, rho v, rho w,
// e + p); dphi[q][t] = computational derivative of u, v, w, T along t.
template <int D, typename R, bool AXIS, bool DYN>
__device__ __forceinline__ void iface_flux(const Consts<R>& K, const R* Wm, const R* Wa,
                                           const R* Wb, const R* Wp, bool has_m, bool has_p,
                                           R nua, R nub, R lba, R lbb, const R* ma, const R* mb,
                                           R pa, R pb, R ua, R va, R wa, R ub, R vb, R wb,
                                           const R (&dphi)[4][3], R mua, R mub, R kaa, R kab,
                                           R sga, R sgb, R F[5]) {
  const R tha = ma[3 * D] * ua + ma[3 * D + 1] * va + ma[3 * D + 2] * wa;
  const R thb = mb[3 * D] * ub + mb[3 * D + 1] * vb + mb[3 * D + 2] * wb;
  const R Ja = ma[9], Jb = mb[9];
  R Fc[5];
  // W[0..3] = Q[0..3]; W[4] = e + p, so (e + p) Th = W[4] Th
  Fc[0] = Ja * (Wa[0] * tha) + Jb * (Wb[0] * thb);
  Fc[1] = Ja * (Wa[1] * tha + pa * ma[3 * D]) + Jb * (Wb[1] * thb + pb * mb[3 * D]);
  Fc[2] = Ja * (Wa[2] * tha + pa * ma[3 * D + 1]) + Jb * (Wb[2] * thb + pb * mb[3 * D + 1]);
  Fc[3] = Ja * (Wa[3] * tha + pa * ma[3 * D + 2]) + Jb * (Wb[3] * thb + pb * mb[3 * D + 2]);
  Fc[4] = Ja * (Wa[4] * tha) + Jb * (Wb[4] * thb);
  const R eps2 = K.k2 * dev_max(nua, nub);
  const R eps4 = dev_max(R(0), K.k4 - eps2);
  const R Jh = R(0.5) * (Ja + Jb);
  const R lJ = R(0.5) * (lba + lbb) * Jh;
#pragma unroll
  for (int q = 0; q < 5; ++q) {
    const R D1 = Wb[q] - Wa[q];
    const R Dm = has_m ? Wa[q] - Wm[q] : -D1;
    const R Dp = has_p ? Wp[q] - Wb[q] : -D1;
    const R D3 = Dp - R(2) * D1 + Dm;
    F[q] = R(0.5) * Fc[q] - lJ * (eps2 * D1 - eps4 * D3);
  }
  // Viscous part from the interface metric vectors m_t (kept at twice
  // their mean): with m = m_D, the flux needs only m.tau and m.q, and
  //   m.tau_i / mu = sum_t g_t dphi_i,t + sum_t m_t,i c_t - 2/3 m_i div,
  //   m.grad T     = sum_t g_t dphi_T,t,
  // where g_t = m . m_t, c_t = sum_j m_j dphi_j,t and div = sum_t m_t .
  // dphi_.,t (every factor 2 of the sums is collected in the constants).
  R mt[9];
  if (AXIS) {
    // a grid with an axis (Reading A27): the J^-1-weighted mean of the two
    // nodes' metrics; an axis node (J^-1 = 0) stores J^-1 m already
    const R wa = (Ja == R(0)) ? R(1) : Ja, wb = (Jb == R(0)) ? R(1) : Jb;
    const R s2 = R(2) / (Ja + Jb);
#pragma unroll
    for (int t = 0; t < 9; ++t) mt[t] = (wa * ma[t] + wb * mb[t]) * s2;
  } else {
#pragma unroll
    for (int t = 0; t < 9; ++t) mt[t] = ma[t] + mb[t];
  }
  const R mx = mt[3 * D], my = mt[3 * D + 1], mz = mt[3 * D + 2];  // 2 m
  R g[3], c[3];
#pragma unroll
  for (int t = 0; t < 3; ++t) {
    g[t] = mx * mt[3 * t] + my * mt[3 * t + 1] + mz * mt[3 * t + 2];        // 4 g_t
    c[t] = mx * dphi[0][t] + my * dphi[1][t] + mz * dphi[2][t];             // 2 c_t
  }
  R div = R(0);  // 2 div
#pragma unroll
  for (int t = 0; t < 3; ++t)
    div += mt[3 * t] * dphi[0][t] + mt[3 * t + 1] * dphi[1][t] + mt[3 * t + 2] * dphi[2][t];
  const R d23 = R(2.0 / 3.0) * div;
  const R mm[3] = {mx, my, mz};
  R sv[3];  // 4 m.tau_i / mu
#pragma unroll
  for (int i = 0; i < 3; ++i)
    sv[i] = (g[0] * dphi[i][0] + g[1] * dphi[i][1] + g[2] * dphi[i][2]) +
            (mt[i] * c[0] + mt[3 + i] * c[1] + mt[6 + i] * c[2]) - mm[i] * d23;
  const R aT = g[0] * dphi[3][0] + g[1] * dphi[3][1] + g[2] * dphi[3][2];  // 4 m.grad T
  const R sJ = Ja + Jb, smu = mua + mub, skap = kaa + kab;  // 2x the means
  const R cf = sJ * smu * R(1.0 / 16.0);
  F[1] -= cf * sv[0];
  F[2] -= cf * sv[1];
  F[3] -= cf * sv[2];
  const R us = (ua + ub) * sv[0] + (va + vb) * sv[1] + (wa + wb) * sv[2];  // 8 u_f . m.tau / mu
  F[4] -= sJ * (smu * us * R(1.0 / 32.0) + skap * aT * R(1.0 / 16.0));
  if (DYN) {
    // the modelled isotropic SGS stress sigma_ll/3 (Eq. yoshizawa) at the
    // interface mean, subtracted from the normal stresses: m.tau_i gains
    // -m_i sigma/3 and u_f.(m.tau) gains -(u_f . m) sigma/3
    const R e1 = sJ * (sga + sgb) * R(1.0 / 24.0);
    F[1] += e1 * mx;
    F[2] += e1 * my;
    F[3] += e1 * mz;
    F[4] += e1 * R(0.5) * ((ua + ub) * mx + (va + vb) * my + (wa + wb) * mz);
  }
}

// Pressure sensor from the three pressures around a (possibly shifted) node.
template <typename R>
__device__ __forceinline__ R sensor3(R pm, R p0, R pp) {
  return dev_abs(pp - R(2) * p0 + pm) / (pp + R(2) * p0 + pm);
}

// Radii lambda_d = |U_d| + a |grad d| and the scaled lbar_d of one node.
template <typename R>
__device__ __forceinline__ void node_lbar(const R* m, R u, R v, R w, R T, R lb[3]) {
  const R a = dev_sqrt(T);
  R l[3];
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    const R mx = m[3 * d], my = m[3 * d + 1], mz = m[3 * d + 2];
    l[d] = dev_abs(mx * u + my * v + mz * w) + a * dev_sqrt(mx * mx + my * my + mz * mz);
  }
  const R s01 = dev_sqrt(l[0] * l[1]), s02 = dev_sqrt(l[0] * l[2]), s12 = dev_sqrt(l[1] * l[2]);
  lb[0] = l[0] + s01 + s02;
  lb[1] = l[1] + s01 + s12;
  lb[2] = l[2] + s02 + s12;
}

template <typename TM, typename R>
__device__ __forceinline__ void load_metrics(const TM* __restrict__ M, long long N, long long n,
                                             R m[10]) {
#pragma unroll
  for (int t = 0; t < 10; ++t) m[t] = (R)__ldg(M + t * N + n);
}

// --------------------------------------------------------------- prestep
// End of a prestep block: the block's minimum of 1/(sum of radii) into
// partials[blockIdx.x] and its non-finite flag into the status word.  With
// fin_mode >= 0 (and sc) the last block to finish also takes the step, as
// k_dt_finalize would in a launch of its own: the minimum over every block's
// partial (exact in any order), dt = cfl x that (or the fixed step), the
// status, and t^{n+1} when fin_advance.
template <typename R>
__device__ __forceinline__ void prestep_finish(R local_min, int bad, double* __restrict__ partials,
                                               DevScalars* __restrict__ sc, int fin_mode,
                                               double fin_cfl, double fin_dt, int fin_advance) {
  __shared__ R smin[32];
  __shared__ int sbad[32];
  for (int off = 16; off > 0; off >>= 1) {
    // every lane executes each shuffle unconditionally (full mask)
    const R o = __shfl_xor_sync(0xffffffffu, local_min, off);
    local_min = local_min < o ? local_min : o;
    bad |= __shfl_xor_sync(0xffffffffu, bad, off);
  }
  if ((threadIdx.x & 31) == 0) {
    smin[threadIdx.x >> 5] = local_min;
    sbad[threadIdx.x >> 5] = bad;
  }
  __syncthreads();
  if (threadIdx.x < 32) {
    const bool live = threadIdx.x < (blockDim.x >> 5);
    R mm = live ? smin[threadIdx.x] : R(1e30);
    int bb = live ? sbad[threadIdx.x] : 0;
    for (int off = 16; off > 0; off >>= 1) {
      const R o = __shfl_xor_sync(0xffffffffu, mm, off);
      mm = mm < o ? mm : o;
      bb |= __shfl_xor_sync(0xffffffffu, bb, off);
    }
    if (threadIdx.x == 0) {
      partials[blockIdx.x] = (double)mm;
      if (bb && sc) atomicOr(&sc->status, 1);
    }
  }
  if (fin_mode >= 0 && sc) {
    __shared__ int last;
    __shared__ double dmin[32];
    if (threadIdx.x == 0) {
      __threadfence();
      last = atomicAdd(&sc->ticket, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (last) {
      __threadfence();
      double m = 1.0e300;
      for (int b = threadIdx.x; b < (int)gridDim.x; b += blockDim.x) m = fmin(m, __ldcg(partials + b));
      for (int off = 16; off > 0; off >>= 1) m = fmin(m, __shfl_xor_sync(0xffffffffu, m, off));
      if ((threadIdx.x & 31) == 0) dmin[threadIdx.x >> 5] = m;
      __syncthreads();
      if (threadIdx.x < 32) {
        m = threadIdx.x < (blockDim.x >> 5) ? dmin[threadIdx.x] : 1.0e300;
        for (int off = 16; off > 0; off >>= 1) m = fmin(m, __shfl_xor_sync(0xffffffffu, m, off));
        if (threadIdx.x == 0) {
          double dt = (fin_mode == LES_DT_FIXED) ? fin_dt : fin_cfl * m;
          const int status = atomicOr(&sc->status, 0);
          if (!(dt > 0.0) || !(dt < 1.0e300)) {
            sc->status = LES_ERR_NONFINITE;
            dt = 0.0;
          } else if (status != 0) {
            sc->status = LES_ERR_NONFINITE;
          }
          sc->dt = dt;
          if (fin_advance) {
            sc->t += dt;
            sc->steps += 1;
          }
          sc->ticket = 0;
        }
      }
    }
  }
}

// Once per time step, from Q^n: block minima of 1/(sum of radii) for the CFL
// step, the non-finite flag, and mu_eff / kappa_eff (frozen over the five
// stages).  Q^n is read as TQ (double, or the float hi part of the mixed
// state); gradients for the SGS model use the node-centred central
// differences (one-sided at non-periodic faces).
// DYN: the dynamic SGS model's branch (coefficients from dyn); a separate
// instantiation keeps the other models' kernel at about half the registers.
template <typename R, typename TQ, typename TM, bool DYN>
__global__ void __launch_bounds__(256) k_prestep(Grid g, Consts<R> K, const TQ* __restrict__ Q,
                                                 const TM* __restrict__ M, R* __restrict__ mk,
                                                 double* __restrict__ partials,
                                                 DevScalars* __restrict__ sc,
                                                 R* __restrict__ dtl, R cfl,
                                                 const double* __restrict__ dyn = nullptr,
                                                 int fin_mode = -1, double fin_cfl = 0.0,
                                                 double fin_dt = 0.0, int fin_advance = 0) {
  const long long N = g.N;
  R local_min = R(1e30);
  int bad = 0;
  for (long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x; n < N;
       n += (long long)gridDim.x * blockDim.x) {
    const R rho = (R)Q[n];
    const R ir = R(1) / rho;
    const R u = (R)Q[N + n] * ir, v = (R)Q[2 * N + n] * ir, w = (R)Q[3 * N + n] * ir;
    const R p = K.gm1 * ((R)Q[4 * N + n] - R(0.5) * rho * (u * u + v * v + w * w));
    const R T = K.gamma * p * ir;
    const R a = dev_sqrt(T);
    R m[10];
    load_metrics(M, N, n, m);
    R lsum = R(0);
    if (K.axis && m[9] == R(0) && (n / g.n[2]) % g.n[1] == 0) {
      // an axis node (Reading A27) takes the radii of (i, 1, k)
      const long long n1 = n + g.stride[1];
      const R rho1 = (R)Q[n1];
      const R ir1 = R(1) / rho1;
      const R u1 = (R)Q[N + n1] * ir1, v1 = (R)Q[2 * N + n1] * ir1, w1 = (R)Q[3 * N + n1] * ir1;
      const R p1 = K.gm1 * ((R)Q[4 * N + n1] - R(0.5) * rho1 * (u1 * u1 + v1 * v1 + w1 * w1));
      const R a1 = dev_sqrt(K.gamma * p1 * ir1);
      R m1[10];
      load_metrics(M, N, n1, m1);
#pragma unroll
      for (int d = 0; d < 3; ++d) {
        const R mx = m1[3 * d], my = m1[3 * d + 1], mz = m1[3 * d + 2];
        lsum += dev_abs(mx * u1 + my * v1 + mz * w1) + a1 * dev_sqrt(mx * mx + my * my + mz * mz);
      }
    } else {
#pragma unroll
      for (int d = 0; d < 3; ++d) {
        const R mx = m[3 * d], my = m[3 * d + 1], mz = m[3 * d + 2];
        lsum += dev_abs(mx * u + my * v + mz * w) + a * dev_sqrt(mx * mx + my * my + mz * mz);
      }
    }
    const R inv = R(1) / lsum;
    if ((g.glo | g.ghi) == 0 || owned_plane(g, (int)(n / g.stride[0]))) {  // a slab's ghost planes are its neighbour's
      if (!(rho > R(0)) || !(p > R(0)) || !(inv > R(0)) || !(inv < R(1e30))) bad = 1;
      local_min = inv < local_min ? inv : local_min;
    }
    if (dtl) dtl[n] = cfl * inv;  // local step of Eq. localdt

    const R mu_l = K.mu_scale * T * dev_sqrt(T) * (R(1) + K.S_suth) / (T + K.S_suth);
    R mu_s = R(0), kap_s = R(0);
    bool kap_set = false;
    if (K.sgs != LES_SGS_NONE) {
      int c[3];
      decompose(g, n, c);
      R dd[3][3];  // dd[q][d] = computational derivative of u_q along d
      long long npv[3], nmv[3];
      int modev[3];  // 0 central, 1 one-sided low face, 2 one-sided high face
#pragma unroll
      for (int d = 0; d < 3; ++d) {
        const long long s = g.stride[d];
        const int nd = g.n[d];
        if (g.per[d]) {
          npv[d] = (c[d] == nd - 1) ? n - (long long)(nd - 1) * s : n + s;
          nmv[d] = (c[d] == 0) ? n + (long long)(nd - 1) * s : n - s;
          modev[d] = 0;
        } else if (c[d] == 0) {
          npv[d] = n + s;
          nmv[d] = n + 2 * s;
          modev[d] = 1;
        } else if (c[d] == nd - 1) {
          npv[d] = n - 2 * s;
          nmv[d] = n - s;
          modev[d] = 2;
        } else {
          npv[d] = n + s;
          nmv[d] = n - s;
          modev[d] = 0;
        }
      }
      // every neighbour's state loaded before any is used (latency-bound
      // otherwise: 124 -> 115 us per launch on 288 x 160 x 128)
      R qp[3][4], qm[3][4];
#pragma unroll
      for (int d = 0; d < 3; ++d)
#pragma unroll
        for (int f = 0; f < 4; ++f) {
          qp[d][f] = (R)Q[f * N + npv[d]];
          qm[d][f] = (R)Q[f * N + nmv[d]];
        }
#pragma unroll
      for (int d = 0; d < 3; ++d) {
        const R irp = R(1) / qp[d][0], irm = R(1) / qm[d][0];
        const R fp[3] = {qp[d][1] * irp, qp[d][2] * irp, qp[d][3] * irp};
        const R fm[3] = {qm[d][1] * irm, qm[d][2] * irm, qm[d][3] * irm};
        const R f0[3] = {u, v, w};
#pragma unroll
        for (int q = 0; q < 3; ++q) {
          if (modev[d] == 0)
            dd[q][d] = R(0.5) * (fp[q] - fm[q]);
          else if (modev[d] == 1)  // (-3 f0 + 4 f1 - f2)/2 with f1 = fp, f2 = fm
            dd[q][d] = R(0.5) * (R(-3) * f0[q] + R(4) * fp[q] - fm[q]);
          else  // (3 f0 - 4 f_{-1} + f_{-2})/2 with f_{-1} = fm, f_{-2} = fp
            dd[q][d] = R(0.5) * (R(3) * f0[q] - R(4) * fm[q] + fp[q]);
        }
      }
      R gr[3][3];
#pragma unroll
      for (int q = 0; q < 3; ++q)
#pragma unroll
        for (int x = 0; x < 3; ++x) gr[q][x] = m[x] * dd[q][0] + m[3 + x] * dd[q][1] + m[6 + x] * dd[q][2];
      const R delta = cbrt(m[9]);
      if (DYN || K.sgs == LES_SGS_SMAGORINSKY) {
        R ss = R(0);
#pragma unroll
        for (int i = 0; i < 3; ++i)
#pragma unroll
          for (int j = 0; j < 3; ++j) {
            const R sij = R(0.5) * (gr[i][j] + gr[j][i]);
            ss += sij * sij;
          }
        const R smag = dev_sqrt(R(2) * ss);
        if (!DYN) {
          mu_s = rho * (delta * delta) * K.cs2 * smag;
        } else {
          // dynamic model (coefficients dyn[6..8] from the procedure):
          // mu_sgs = C_ds rho Delta^2 |S|, kappa_sgs with the dynamic Pr_sgs,
          // and the Yoshizawa sigma_ll = 2 C_I rho Delta^2 |S|^2
          const R d2 = delta * delta;
          mu_s = (R)dyn[6] * rho * d2 * smag;
          kap_s = mu_s / (K.gm1 * (R)dyn[8]);
          kap_set = true;
          mk[2 * N + n] = R(2) * (R)dyn[7] * rho * d2 * smag * smag;
        }
      } else {
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
            be[i][j] = delta * delta * (gr[i][0] * gr[j][0] + gr[i][1] * gr[j][1] + gr[i][2] * gr[j][2]);
        R B = be[0][0] * be[1][1] - be[0][1] * be[0][1] + be[0][0] * be[2][2] -
              be[0][2] * be[0][2] + be[1][1] * be[2][2] - be[1][2] * be[1][2];
        B = B > R(0) ? B : R(0);
        mu_s = (aa == R(0)) ? R(0) : rho * K.cs2 * dev_sqrt(B / aa);
      }
    }
    mk[n] = mu_l + mu_s;
    mk[N + n] = mu_l * K.inv_gm1_pr + (kap_set ? kap_s : mu_s * K.inv_gm1_prs);
  }
  prestep_finish(local_min, bad, partials, sc, fin_mode, fin_cfl, fin_dt, fin_advance);
}

// ------------------------------------------------------------ fused stage
enum { FMODE_RHS = 0, FMODE_STAGE = 1, FMODE_LAST = 2 };

// Tile of FTJ x FTK (eta, zeta) columns, one thread per column.
constexpr int FTJ = 16, FTK = 32, FNT = FTJ * FTK;
// Shared-memory rows hold the tile's FTK columns and a two-column halo on
// each side: tile column kk in [-2, FTK+1] lives at row column kk + 2.  When
// zeta is periodic and nk % 4 == 0 the tiles are shifted by two columns
// (tile t owns the global columns 32 t + 2 .. 32 t + 33, wrapped), so a
// whole row, halos included, is the 16-byte-aligned global range
// [32 t, 32 t + 36): nine 16-byte copies and no separate halo copy.
constexpr int SK = FTK + 4;
constexpr int R2 = FTJ + 4, R1 = FTJ + 2;  // rows with a 2-node / 1-node halo
constexpr int PL2 = R2 * SK, PL1 = R1 * SK;
__host__ __device__ constexpr int colk(int kk) { return kk + 2; }

// Shared-memory plan (floats):
//   sQ[3][5][PL2]  conserved state of planes i, i+1, i+2 (2-node halo)
//   sPr[3][PL2]    float4 (u, v, w, T) of planes i-1, i, i+1
//   sPw[3][PL2]    float2 (p, e + p) of the same planes
//   sM[3][10][PL1] metrics of planes i, i+1, i+2 (1-node halo)
//   sK[3][2][PL1]  mu_eff kappa_eff of planes i, i+1, i+2
//   sL[2][3][PL1]  lbar of planes i, i+1
//   sFe[5][FTJ+1][FTK]  eta interface fluxes (rows -1 .. FTJ-1 of the tile)
//   sFz[5][FTJ]         the tile's left-edge zeta interface fluxes (the
//                       others pass between neighbouring lanes by shuffle)
constexpr int OFF_PR = 3 * 5 * PL2, OFF_PW = OFF_PR + 3 * 4 * PL2,
              OFF_M = OFF_PW + 3 * 2 * PL2, OFF_K = OFF_M + 3 * 10 * PL1;
// With the dynamic SGS model the viscosity slots hold a third field, the
// Yoshizawa sigma_ll (sK[3][3][PL1]); the regions after sK move up.
template <bool DYN>
struct FLayout {
  static constexpr int NKF = DYN ? 3 : 2;  // fields per viscosity slot
  static constexpr int L = OFF_K + 3 * NKF * PL1;
  static constexpr int FE = L + 2 * 3 * PL1;
  static constexpr int FZ = FE + 5 * (FTJ + 1) * FTK;
  static constexpr int FLOATS = FZ + 5 * FTJ;
};
static_assert(FLayout<true>::FLOATS * 4 <= 227 * 1024, "shared memory plan exceeds 227 KB");

// Computational derivatives of (u, v, w, T) at an interface from node
// records (float4 u, v, w, T): along the interface normal, phi_b - phi_a;
// along a tangent t, the mean of the two nodes' central differences,
// 1/4 [(phi_{a+t} - phi_{a-t}) + (phi_{b+t} - phi_{b-t})].
template <int D>
__device__ __forceinline__ void dphi_normal(const float4 a, const float4 b, float (&dphi)[4][3]) {
  dphi[0][D] = b.x - a.x;
  dphi[1][D] = b.y - a.y;
  dphi[2][D] = b.z - a.z;
  dphi[3][D] = b.w - a.w;
}
template <int T>
__device__ __forceinline__ void dphi_tangent(const float4 ap, const float4 am, const float4 bp,
                                             const float4 bm, float (&dphi)[4][3]) {
  dphi[0][T] = 0.25f * ((ap.x - am.x) + (bp.x - bm.x));
  dphi[1][T] = 0.25f * ((ap.y - am.y) + (bp.y - bm.y));
  dphi[2][T] = 0.25f * ((ap.z - am.z) + (bp.z - bm.z));
  dphi[3][T] = 0.25f * ((ap.w - am.w) + (bp.w - bm.w));
}

__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem) : "memory");
}

// Per-field base pointers (32-bit indexing inside a field, N < 2^31).
struct FusedPtrs {
  const float* qin[5];  // stage input state
  const float* hi[5];   // Q^(0) hi part
  float* lo[5];         // Q^(0) lo part (last stage)
  float* hiw[5];        // Q^(0) hi part, written in the last stage
  const float* m[10];   // metrics
  const float* mk[3];   // mu_eff, kappa_eff (and sigma_ll with the dynamic model)
  float* out[5];        // stage output
  double* outd[5];      // residual output (RHS mode)
  const float* dtl;     // local steps (dt_mode LOCAL) or nullptr: global dt
};

struct FusedGeom {
  int ni, nj, nk;
  int per[3];
  // axial chunks: the first n1 hold a1 planes each, the other nch - n1
  // split the remaining planes evenly (n1 = 0: nch chunks of equal length)
  int nch, n1, a1;
  int vec16;  // zeta periodic, nk % 4 == 0 and nk >= FTK: tiles shifted by
              // two columns, rows staged as 16-byte copies
  int ilo, ihi;  // planes the stage updates along a non-periodic xi: [ilo, ihi)
  int N;         // points per field (the fields of qin, m and mk are N apart)
};

__device__ __forceinline__ int wrap_fast(int v, int n, int per) {
  if (per) {
    if (v < 0) v += n;
    if (v >= n) v -= n;
    if (v < 0 || v >= n) {  // tiles wider than a small periodic extent
      v %= n;
      if (v < 0) v += n;
    }
    return v;
  }
  return (v >= 0 && v < n) ? v : -1;
}

// LOCAL: node n advances with its own step P.dtl[n] (dt_mode LOCAL) in
// place of the global one; a separate instantiation keeps the global-step
// kernel free of the per-node load and its branch.  PM >= 0: properties of
// the grid fixed at compile time, so the face, wrap, ownership and
// one-sided-difference tests fold away: bits 0-2, direction d periodic;
// bit 3, the shifted 16-byte staging (G.vec16); bit 4, tiles that cover eta
// and zeta exactly (every thread owns a column).  PM = -1 reads them from G.
template <int MODE, bool LOCAL, bool AXIS, bool DYN, int PM>
__global__ void __launch_bounds__(FNT, 1)
    k_stage_fused(const FusedGeom G, const Consts<float> K, const FusedPtrs P,
                  const DevScalars* __restrict__ sc, double alpha) {
  extern __shared__ __align__(16) float smem[];
  float* sQ = smem;
  float4* sPr = reinterpret_cast<float4*>(smem + OFF_PR);
  float2* sPw = reinterpret_cast<float2*>(smem + OFF_PW);
  float* sM = smem + OFF_M;
  float* sK = smem + OFF_K;
  constexpr int NKF = FLayout<DYN>::NKF;
  float* sL = smem + FLayout<DYN>::L;
  float* sFe = smem + FLayout<DYN>::FE;
  float* sFz = smem + FLayout<DYN>::FZ;
  const int ni = G.ni, nj = G.nj, nk = G.nk;
  // periodicity of xi, eta, zeta: fixed at compile time for PM >= 0 (bit d:
  // direction d periodic), else the grid's flags
  const int per0 = PM >= 0 ? (PM & 1) : G.per[0];
  const int per1 = PM >= 0 ? ((PM >> 1) & 1) : G.per[1];
  const int per2 = PM >= 0 ? ((PM >> 2) & 1) : G.per[2];
  const int tid = threadIdx.x, tx = tid & 31, ty = tid >> 5;
  // kt: first column of the unshifted tile; k0: global column of tile
  // column 0 (kt + 2 with the shifted tiling; may exceed nk - 1, wrapped)
  const bool vec_ok = PM >= 0 ? ((PM >> 3) & 1) != 0 : G.vec16 != 0;
  const int kt = blockIdx.x * FTK, k0 = kt + (vec_ok ? 2 : 0), j0 = blockIdx.y * FTJ;
  int ib, ie;
  {
    const int z = blockIdx.z, b = G.n1 * G.a1;
    if (z < G.n1) {
      ib = z * G.a1;
      ie = ib + G.a1;
    } else {
      const int n2 = G.nch - G.n1, z2 = z - G.n1;
      ib = b + (int)((long long)z2 * (ni - b) / n2);
      ie = b + (int)((long long)(z2 + 1) * (ni - b) / n2);
    }
  }
  const int jown = j0 + ty;
  const int kown = (k0 + tx < nk) ? k0 + tx : k0 + tx - nk;  // wraps in the shifted case only
  const bool own = (PM >= 0 && ((PM >> 4) & 1)) ? true : (jown < nj && kt + tx < nk);
  const bool jint = per1 || (jown > 0 && jown < nj - 1);
  const bool kint = per2 || (kown > 0 && kown < nk - 1);
  const bool per_i = per0 != 0;
  const int o2 = (ty + 2) * SK + tx + 2;  // own node, 2-node-halo planes
  const int o1 = (ty + 1) * SK + tx + 2;  // own node, 1-node-halo planes

  // ---- stage plane x (state: 2-node halo; metrics, mu/kappa: 1-node halo)
  auto stage_plane = [&](int slot, int x) {
    const int ig = wrap_fast(x, ni, per0);
    constexpr int JQ = 5 * R2, JM = 10 * R1, JK = NKF * R1;
    // one row per thread, taken by the highest-numbered threads: the lowest
    // ones derive a second node record in the same phase
    const int tid = threadIdx.x - (FNT - (JQ + JM + JK));
    if (tid < 0) return;
    const float* src;
    float* dst;
    int jj, halo;
    float benign;
    if (tid < JQ) {
      const int f = tid / R2;
      jj = tid - f * R2 - 2;
      src = P.qin[0] + (long long)f * G.N;
      dst = sQ + (slot * 5 + f) * PL2 + (jj + 2) * SK;
      halo = 2;
      benign = (f == 0 || f == 4) ? 1.f : 0.f;
    } else if (tid < JQ + JM) {
      const int u = tid - JQ, f = u / R1;
      jj = u - f * R1 - 1;
      src = P.m[0] + (long long)f * G.N;
      dst = sM + (slot * 10 + f) * PL1 + (jj + 1) * SK;
      halo = 1;
      benign = 1.f;
    } else {
      const int u = tid - JQ - JM, f = u / R1;
      jj = u - f * R1 - 1;
      src = P.mk[0] + (long long)f * G.N;
      dst = sK + (slot * NKF + f) * PL1 + (jj + 1) * SK;
      halo = 1;
      benign = 0.f;
    }
    const int jg = wrap_fast(j0 + jj, nj, per1);
    if (ig < 0 || jg < 0) {
      for (int c = 0; c < SK; ++c) dst[c] = benign;
      return;
    }
    const float* row = src + (ig * nj + jg) * nk;
    if (vec_ok && kt + SK <= nk) {
      // the row's global columns kt .. kt + SK - 1, inside the row
      const float* rk = row + kt;
#pragma unroll
      for (int v = 0; v < SK / 4; ++v) cp_async16(dst + 4 * v, rk + 4 * v);
    } else if (vec_ok) {
      // the last tile: columns kt .. kt + SK - 1 wrapped at nk (a multiple
      // of 4, so no 16-byte piece straddles the wrap; kt + SK < 2 nk because
      // nk >= FTK)
#pragma unroll
      for (int v = 0; v < SK / 4; ++v) {
        const int kg = (kt + 4 * v < nk) ? kt + 4 * v : kt + 4 * v - nk;
        cp_async16(dst + 4 * v, row + kg);
      }
    } else {
      for (int kk = -halo; kk < FTK + halo; ++kk) {
        const int kg = wrap_fast(k0 + kk, nk, per2);
        if (kg >= 0)
          cp_async4(dst + colk(kk), row + kg);
        else
          dst[colk(kk)] = benign;
      }
    }
  };

  // ---- primitives (2-node halo) and lbar (1-node halo) of a staged plane
  auto derive_plane = [&](int qs, int ps, int ms, int ls) {
    const float* q = sQ + qs * 5 * PL2;
    float4* pr = sPr + ps * PL2;
    float2* pw = sPw + ps * PL2;
    const float* mm = sM + ms * 10 * PL1;
    float* ll = sL + ls * 3 * PL1;
    for (int r = tid; r < PL2; r += FNT) {
      const float rho = q[r];
      const float ir = frcp_fast(rho);
      const float u = q[PL2 + r] * ir, v = q[2 * PL2 + r] * ir, w = q[3 * PL2 + r] * ir;
      const float p = K.gm1 * (q[4 * PL2 + r] - 0.5f * rho * (u * u + v * v + w * w));
      const float T = K.gamma * p * ir;
      pr[r] = make_float4(u, v, w, T);
      pw[r] = make_float2(p, q[4 * PL2 + r] + p);
      const int row = r / SK, col = r - row * SK;
      // 1-node halo: rows 1 .. R2-2 of the 2-node layout, columns kk in [-1, FTK]
      if (row >= 1 && row <= R2 - 2 && col >= colk(-1) && col <= colk(FTK)) {
        const int r1 = r - SK;
        float m[10];
#pragma unroll
        for (int t = 0; t < 10; ++t) m[t] = mm[t * PL1 + r1];
        float lb[3];
        if (AXIS && m[9] == 0.f && j0 + row - 2 == 0) {
          // an axis node (Reading A27) takes the radii of its inward
          // neighbour (i, 1, k): the next row of the same plane
          const int s = r + SK;
          const float rho1 = q[s];
          const float ir1 = frcp_fast(rho1);
          const float u1 = q[PL2 + s] * ir1, v1 = q[2 * PL2 + s] * ir1, w1 = q[3 * PL2 + s] * ir1;
          const float p1 = K.gm1 * (q[4 * PL2 + s] - 0.5f * rho1 * (u1 * u1 + v1 * v1 + w1 * w1));
          float m1[10];
#pragma unroll
          for (int t = 0; t < 10; ++t) m1[t] = mm[t * PL1 + r1 + SK];
          node_lbar(m1, u1, v1, w1, K.gamma * p1 * ir1, lb);
        } else {
          node_lbar(m, u, v, w, T, lb);
        }
        ll[r1] = lb[0];
        ll[PL1 + r1] = lb[1];
        ll[2 * PL1 + r1] = lb[2];
      }
    }
  };

  // ---- own-column state along xi: planes i-1, i, i+1, i+2 (registers); the
  // raw state of the next plane to enter the queue is fetched one iteration
  // early so its latency hides behind a whole plane of work
  float Wq[4][5] = {}, pq[4] = {};
  bool vq[4] = {false, false, false, false};
  float qn[5] = {0.f, 0.f, 0.f, 0.f, 0.f};
  bool vn = false;
  auto fetch_q = [&](int x) {
    const int ig = wrap_fast(x, ni, per0);
    vn = own && ig >= 0;
    if (vn) {
      const int n = (ig * nj + jown) * nk + kown;
#pragma unroll
      for (int c = 0; c < 5; ++c) qn[c] = __ldg(P.qin[c] + n);
    }
  };
  // Q^(0) of the own node (hi part; in the last stage also the lo part; with
  // local steps also the node's step), fetched one plane ahead of its update
  // so the epilogue never waits on a global load
  float h0[5] = {0.f, 0.f, 0.f, 0.f, 0.f};
  float l0[5] = {0.f, 0.f, 0.f, 0.f, 0.f};  // lo part, last stage only
  float d0 = 0.f;                            // local step (LOCAL only)
  auto fetch_h = [&](int x) {
    const int ig = wrap_fast(x, ni, per0);
    if (MODE != FMODE_RHS && own && ig >= 0) {
      const int n = (ig * nj + jown) * nk + kown;
#pragma unroll
      for (int c = 0; c < 5; ++c) h0[c] = P.hi[c][n];
      if (MODE == FMODE_LAST) {
#pragma unroll
        for (int c = 0; c < 5; ++c) l0[c] = P.lo[c][n];
      }
      if (LOCAL) d0 = P.dtl[n];
    }
  };
  auto finish_W = [&](float W[5], float& p, bool& valid) {
    valid = vn;
    if (!valid) {
#pragma unroll
      for (int c = 0; c < 5; ++c) W[c] = 0.f;
      p = 1.f;
      return;
    }
    const float ir = frcp_fast(qn[0]);
    const float u = qn[1] * ir, v = qn[2] * ir, w = qn[3] * ir;
    p = K.gm1 * (qn[4] - 0.5f * qn[0] * (u * u + v * v + w * w));
#pragma unroll
    for (int c = 0; c < 4; ++c) W[c] = qn[c];
    W[4] = qn[4] + p;
  };

  // xi interface (x, x+1) of the own column: sPr/sPw/sM/sK/sL slots of both planes
  auto xi_flux = [&](int x, int p0, int p1, int m0, int m1, int l0, int l1, const float* mown,
                     const float4* rown, const float4* rpm, const float2* wown, float F[5]) {
    const float4* A0 = sPr + p0 * PL2;
    const float4* A1 = sPr + p1 * PL2;
    float nua, nub;
    if (!per_i && x == 0)
      nua = sensor3(pq[1], pq[2], pq[3]);
    else
      nua = sensor3(pq[0], pq[1], pq[2]);
    if (!per_i && x + 1 == ni - 1)
      nub = sensor3(pq[0], pq[1], pq[2]);
    else
      nub = sensor3(pq[1], pq[2], pq[3]);
    const float4 a0 = rown ? rown[0] : A0[o2], b0 = rpm ? rpm[0] : A1[o2];
    const float4 an = A0[o2 + SK], as = A0[o2 - SK], bn = A1[o2 + SK], bs = A1[o2 - SK];
    const float4 ae = A0[o2 + 1], aw = A0[o2 - 1], be = A1[o2 + 1], bw = A1[o2 - 1];
    float dphi[4][3];
    dphi_normal<0>(a0, b0, dphi);
    dphi_tangent<1>(an, as, bn, bs, dphi);
    dphi_tangent<2>(ae, aw, be, bw, dphi);
    float ma[10], mb[10];
#pragma unroll
    for (int t = 0; t < 10; ++t) {
      ma[t] = mown ? mown[t] : sM[(m0 * 10 + t) * PL1 + o1];
      mb[t] = sM[(m1 * 10 + t) * PL1 + o1];
    }
    const float* Ka = sK + m0 * NKF * PL1;
    const float* Kb = sK + m1 * NKF * PL1;
    iface_flux<0, float, AXIS, DYN>(K, Wq[0], Wq[1], Wq[2], Wq[3], vq[0], vq[3], nua, nub,
                         sL[l0 * 3 * PL1 + o1], sL[l1 * 3 * PL1 + o1], ma, mb,
                         wown ? wown->x : sPw[p0 * PL2 + o2].x,
                         sPw[p1 * PL2 + o2].x, a0.x, a0.y, a0.z, b0.x, b0.y, b0.z, dphi, Ka[o1],
                         Kb[o1], Ka[PL1 + o1], Kb[PL1 + o1], DYN ? Ka[2 * PL1 + o1] : 0.f,
                         DYN ? Kb[2 * PL1 + o1] : 0.f, F);
  };

  // eta interface between tile rows ra and ra+1 (ra in [-1, FTJ-1]), own
  // column; plane i in slots qs (sQ), ps (sP, with pm/pp for i-1/i+1), ms, ls
  auto eta_flux = [&](int ra, int qs, int pm, int ps, int pp, int ms, int ls, const float* mown,
                      const float4* rown, const float4* rpm, const float2* wown, float F[5]) {
    const float* Qs = sQ + qs * 5 * PL2;
    const float4* Pc = sPr + ps * PL2;
    const float4* Pm = sPr + pm * PL2;
    const float4* Pp = sPr + pp * PL2;
    const float2* Pw = sPw + ps * PL2;
    const int a2 = (ra + 2) * SK + colk(tx), b2 = a2 + SK;
    const int a1 = (ra + 1) * SK + colk(tx), b1 = a1 + SK;
    const int jga = j0 + ra;
    const bool has_m = per1 || jga - 1 >= 0;
    const bool has_p = per1 || jga + 2 <= nj - 1;
    const float2 wm = Pw[a2 - SK], wa = wown ? *wown : Pw[a2], wb = Pw[b2], wp = Pw[b2 + SK];
    float Wm[5], Wa[5], Wb[5], Wp[5];
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      Wa[c] = Qs[c * PL2 + a2];
      Wb[c] = Qs[c * PL2 + b2];
      Wm[c] = Qs[c * PL2 + a2 - SK];
      Wp[c] = Qs[c * PL2 + b2 + SK];
    }
    Wa[4] = wa.y;
    Wb[4] = wb.y;
    Wm[4] = wm.y;
    Wp[4] = wp.y;
    float nua, nub;
    if (!per1 && jga == 0)
      nua = sensor3(wa.x, wb.x, wp.x);
    else
      nua = sensor3(wm.x, wa.x, wb.x);
    if (!per1 && jga + 1 == nj - 1)
      nub = sensor3(wm.x, wa.x, wb.x);
    else
      nub = sensor3(wa.x, wb.x, wp.x);
    const int am1 = a2 - 1, bm1 = b2 - 1;
    const float4 ca = rown ? rown[0] : Pc[a2], cb = Pc[b2];
    float dphi[4][3];
    dphi_normal<1>(ca, cb, dphi);
    dphi_tangent<0>(rpm ? rpm[0] : Pp[a2], rpm ? rpm[1] : Pm[a2], Pp[b2], Pm[b2], dphi);
    dphi_tangent<2>(Pc[a2 + 1], Pc[am1], Pc[b2 + 1], Pc[bm1], dphi);
    float ma[10], mb[10];
#pragma unroll
    for (int t = 0; t < 10; ++t) {
      ma[t] = mown ? mown[t] : sM[(ms * 10 + t) * PL1 + a1];
      mb[t] = sM[(ms * 10 + t) * PL1 + b1];
    }
    const float* Kc = sK + ms * NKF * PL1;
    const float* L = sL + ls * 3 * PL1 + PL1;
    iface_flux<1, float, AXIS, DYN>(K, Wm, Wa, Wb, Wp, has_m, has_p, nua, nub, L[a1], L[b1], ma, mb, wa.x,
                         wb.x, ca.x, ca.y, ca.z, cb.x, cb.y, cb.z, dphi, Kc[a1], Kc[b1],
                         Kc[PL1 + a1], Kc[PL1 + b1], DYN ? Kc[2 * PL1 + a1] : 0.f,
                         DYN ? Kc[2 * PL1 + b1] : 0.f, F);
  };

  // zeta interface between tile columns ca and ca+1 (ca in [-1, FTK-1]) in
  // tile row rr
  auto zeta_flux = [&](int rr, int ca, int qs, int pm, int ps, int pp, int ms, int ls,
                       const float* mown, const float4* rown, const float4* rpm, const float2* wown,
                       float F[5]) {
    const float* Qs = sQ + qs * 5 * PL2;
    const float4* Pc = sPr + ps * PL2;
    const float4* Pm = sPr + pm * PL2;
    const float4* Pp = sPr + pp * PL2;
    const float2* Pw = sPw + ps * PL2;
    const int rb2 = (rr + 2) * SK, rb1 = (rr + 1) * SK;
    const int ca_c = colk(ca), cb_c = colk(ca + 1), cm_c = colk(ca - 1), cp_c = colk(ca + 2);
    const int a2 = rb2 + ca_c, b2 = rb2 + cb_c, m2 = rb2 + cm_c, q2 = rb2 + cp_c;
    const int a1 = rb1 + ca_c, b1 = rb1 + cb_c;
    const int kga = k0 + ca;
    const bool has_m = per2 || kga - 1 >= 0;
    const bool has_p = per2 || kga + 2 <= nk - 1;
    const float2 wm = Pw[m2], wa = wown ? *wown : Pw[a2], wb = Pw[b2], wp = Pw[q2];
    float Wm[5], Wa[5], Wb[5], Wp[5];
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      Wa[c] = Qs[c * PL2 + a2];
      Wb[c] = Qs[c * PL2 + b2];
      Wm[c] = Qs[c * PL2 + m2];
      Wp[c] = Qs[c * PL2 + q2];
    }
    Wa[4] = wa.y;
    Wb[4] = wb.y;
    Wm[4] = wm.y;
    Wp[4] = wp.y;
    float nua, nub;
    if (!per2 && kga == 0)
      nua = sensor3(wa.x, wb.x, wp.x);
    else
      nua = sensor3(wm.x, wa.x, wb.x);
    if (!per2 && kga + 1 == nk - 1)
      nub = sensor3(wm.x, wa.x, wb.x);
    else
      nub = sensor3(wa.x, wb.x, wp.x);
    const float4 pa = rown ? rown[0] : Pc[a2], pb = Pc[b2];
    float dphi[4][3];
    dphi_normal<2>(pa, pb, dphi);
    dphi_tangent<0>(rpm ? rpm[0] : Pp[a2], rpm ? rpm[1] : Pm[a2], Pp[b2], Pm[b2], dphi);
    dphi_tangent<1>(Pc[a2 + SK], Pc[a2 - SK], Pc[b2 + SK], Pc[b2 - SK], dphi);
    float ma[10], mb[10];
#pragma unroll
    for (int t = 0; t < 10; ++t) {
      ma[t] = mown ? mown[t] : sM[(ms * 10 + t) * PL1 + a1];
      mb[t] = sM[(ms * 10 + t) * PL1 + b1];
    }
    const float* Kc = sK + ms * NKF * PL1;
    const float* L = sL + ls * 3 * PL1 + 2 * PL1;
    iface_flux<2, float, AXIS, DYN>(K, Wm, Wa, Wb, Wp, has_m, has_p, nua, nub, L[a1], L[b1], ma, mb, wa.x,
                         wb.x, pa.x, pa.y, pa.z, pb.x, pb.y, pb.z, dphi, Kc[a1], Kc[b1],
                         Kc[PL1 + a1], Kc[PL1 + b1], DYN ? Kc[2 * PL1 + a1] : 0.f,
                         DYN ? Kc[2 * PL1 + b1] : 0.f, F);
  };

  auto m3 = [](int x) { return ((x % 3) + 3) % 3; };
  auto m2 = [](int x) { return ((x % 2) + 2) % 2; };
  // ---------------------------------------------------------- prologue
  // sQ/sM/sK slot of plane x: x mod 3 (planes i, i+1, i+2 live); sP slot:
  // x mod 3 (planes i-1, i, i+1); sL slot: x mod 2 (planes i, i+1).
  // rotating slots: planes i-1, i, i+1 (plane i+2 is staged into the slot of
  // plane i-1) and the lbar slots of planes i, i+1
  int s_m = m3(ib - 1), s_c = m3(ib), s_p = m3(ib + 1);
  int l_c = m2(ib), l_p = m2(ib + 1);
  stage_plane(s_m, ib - 1);
  stage_plane(s_c, ib);
  cp_async_commit();
  stage_plane(s_p, ib + 1);
  cp_async_commit();
  // the own column's planes ib-2 .. ib+1: all loads issued before any is used
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const int igq = wrap_fast(ib - 2 + q, ni, per0);
    vq[q] = own && igq >= 0;
    if (vq[q]) {
      const int n = (igq * nj + jown) * nk + kown;
#pragma unroll
      for (int c = 0; c < 5; ++c) Wq[q][c] = __ldg(P.qin[c] + n);
    }
  }
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    if (!vq[q]) {
#pragma unroll
      for (int c = 0; c < 5; ++c) Wq[q][c] = 0.f;
      pq[q] = 1.f;
      continue;
    }
    const float ir = frcp_fast(Wq[q][0]);
    const float u = Wq[q][1] * ir, v = Wq[q][2] * ir, w = Wq[q][3] * ir;
    pq[q] = K.gm1 * (Wq[q][4] - 0.5f * Wq[q][0] * (u * u + v * v + w * w));
    Wq[q][4] += pq[q];
  }
  fetch_q(ib + 2);  // enters the queue in the first iteration
  fetch_h(ib);
  cp_async_wait<1>();
  __syncthreads();
  derive_plane(s_m, s_m, s_m, l_p);  // m2(ib - 1) == m2(ib + 1)
  derive_plane(s_c, s_c, s_c, l_c);
  __syncthreads();
  float Fx_prev[5] = {0.f, 0.f, 0.f, 0.f, 0.f};
  if (own && jint && kint && (per_i || ib - 1 >= 0))
    xi_flux(ib - 1, s_m, s_c, s_m, s_c, l_p, l_c, nullptr, nullptr, nullptr, nullptr, Fx_prev);
  const float adt = (MODE == FMODE_RHS) ? 0.f : (float)(alpha * sc->dt);
  // plane ib+1 has landed (this thread's copies; the barrier makes everyone's
  // visible) and the xi flux above is done with the slots of plane ib-1
  cp_async_wait<0>();
  __syncthreads();

  for (int i = ib; i < ie; ++i) {
    // own-column queue: planes i-1 .. i+2
#pragma unroll
    for (int s = 0; s < 3; ++s) {
#pragma unroll
      for (int c = 0; c < 5; ++c) Wq[s][c] = Wq[s + 1][c];
      pq[s] = pq[s + 1];
      vq[s] = vq[s + 1];
    }
    finish_W(Wq[3], pq[3], vq[3]);  // plane i+2, fetched one iteration ago
    fetch_q(i + 3);
    // Plane i+1 has landed and is visible, and nothing reads the slots of
    // plane i-1 any more: both were settled by the barrier that closed the
    // previous flux phase (or the prologue), so plane i+2 is staged into
    // those slots and plane i+1 derived without a barrier of their own.
    stage_plane(s_m, i + 2);
    cp_async_commit();
    derive_plane(s_p, s_p, s_p, l_p);
    __syncthreads();

    const int ig = wrap_fast(i, ni, per0);
    const bool iint = per_i || (i >= G.ilo && i < G.ihi);
    float Fx[5] = {0.f, 0.f, 0.f, 0.f, 0.f};
    // the own node's metrics, read once for its three interfaces
    float mo[10];
#pragma unroll
    for (int t = 0; t < 10; ++t) mo[t] = sM[(s_c * 10 + t) * PL1 + o1];
    // and its node records; in the global-step stage and residual modes also
    // those of planes i+1 and i-1 of the own column (the last stage and the
    // local-step variants keep them in shared memory: their epilogues need
    // the registers)
    const float4 ro = sPr[s_c * PL2 + o2];
    const float2 wo = sPw[s_c * PL2 + o2];
    constexpr bool keep_pm = MODE != FMODE_LAST && !LOCAL;
    float4 rq[2];
    if (keep_pm) {
      rq[0] = sPr[s_p * PL2 + o2];
      rq[1] = sPr[s_m * PL2 + o2];
    }
    const float4* rpm = keep_pm ? rq : nullptr;
    if (own && jint && kint && (per_i || i + 1 <= ni - 1))
      xi_flux(i, s_c, s_p, s_c, s_p, l_c, l_p, mo, &ro, rpm, &wo, Fx);
    if (own && iint && kint) {
      float F[5];
      if (per1 || jown + 1 <= nj - 1) {
        eta_flux(ty, s_c, s_m, s_c, s_p, s_c, l_c, mo, &ro, rpm, &wo, F);
#pragma unroll
        for (int c = 0; c < 5; ++c) sFe[(c * (FTJ + 1) + ty + 1) * FTK + tx] = F[c];
      }
      if (ty == 0 && (per1 || j0 - 1 >= 0)) {
        eta_flux(-1, s_c, s_m, s_c, s_p, s_c, l_c, nullptr, nullptr, nullptr, nullptr, F);
#pragma unroll
        for (int c = 0; c < 5; ++c) sFe[(c * (FTJ + 1)) * FTK + tx] = F[c];
      }
    }
    // zeta interfaces: this lane's (tx, tx+1) minus its left neighbour's,
    // taken through the warp; lane 0's left interface is the tile edge,
    // computed by warp 1 and read after the barrier
    float dz[5];
    {
      float Fz[5] = {0.f, 0.f, 0.f, 0.f, 0.f};
      if (own && iint && jint && (per2 || kown + 1 <= nk - 1))
        zeta_flux(ty, tx, s_c, s_m, s_c, s_p, s_c, l_c, mo, &ro, rpm, &wo, Fz);
#pragma unroll
      for (int c = 0; c < 5; ++c) {
        const float left = __shfl_up_sync(0xffffffffu, Fz[c], 1);
        dz[c] = Fz[c] - (tx == 0 ? 0.f : left);
      }
    }
    // left-edge zeta interfaces (k0-1, k0) of the FTJ rows: lanes of warp 1
    if (ty == 1 && tx < FTJ && iint && (per2 || k0 - 1 >= 0)) {
      const int rr = tx, jr = j0 + rr;
      const bool rint = per1 || (jr > 0 && jr < nj - 1);
      if (jr < nj && rint) {
        float F[5];
        zeta_flux(rr, -1, s_c, s_m, s_c, s_p, s_c, l_c, nullptr, nullptr, nullptr, nullptr, F);
#pragma unroll
        for (int c = 0; c < 5; ++c) sFz[c * FTJ + rr] = F[c];
      }
    }
    // this plane's Q^(0) moves to hc/lc/dc and the next plane's global loads
    // are issued before the barrier, so their latency overlaps the wait
    float hc[5];
#pragma unroll
    for (int c = 0; c < 5; ++c) hc[c] = h0[c];
    float lc[5];
#pragma unroll
    for (int c = 0; c < 5; ++c) lc[c] = l0[c];
    const float dc = d0;
    fetch_h(i + 1);
    // plane i+2, staged at the top of this iteration, must have landed before
    // the next iteration derives it: wait here, and let this barrier (which
    // also publishes the eta/zeta fluxes) make it visible
    cp_async_wait<0>();
    __syncthreads();
    if (own && ig >= 0) {
      const int n = (ig * nj + jown) * nk + kown;
      if (iint && jint && kint) {
        const float Jn = frcp_fast(mo[9]);
        const float an = LOCAL ? (float)alpha * dc : adt;
#pragma unroll
        for (int c = 0; c < 5; ++c) {
          float r = 0.f;
          r += Fx[c] - Fx_prev[c];
          r += sFe[(c * (FTJ + 1) + ty + 1) * FTK + tx] - sFe[(c * (FTJ + 1) + ty) * FTK + tx];
          r += dz[c];
          if (tx == 0) r -= sFz[c * FTJ + ty];
          if (MODE == FMODE_RHS) {
            P.outd[c][n] = (double)r;
          } else if (MODE == FMODE_STAGE) {
            P.out[c][n] = hc[c] - an * (Jn * r);
          } else {
            // compensated update of the pair (hi, lo) by d (TwoSum, then
            // renormalisation), all in FP32
            const float d = -an * (Jn * r);
            const float hi = hc[c], lo = lc[c];
            const float s = hi + d;
            const float bb = s - hi;
            const float e = (hi - (s - bb)) + (d - bb);
            const float lo2 = lo + e;
            const float h2 = s + lo2;
            P.hiw[c][n] = h2;
            P.lo[c][n] = lo2 - (h2 - s);
          }
        }
      } else if (MODE == FMODE_RHS) {
#pragma unroll
        for (int c = 0; c < 5; ++c) P.outd[c][n] = 0.0;
      } else if (MODE == FMODE_STAGE) {
#pragma unroll
        for (int c = 0; c < 5; ++c) P.out[c][n] = hc[c];
      }
    }
#pragma unroll
    for (int c = 0; c < 5; ++c) Fx_prev[c] = Fx[c];
    {
      const int t = s_m;
      s_m = s_c;
      s_c = s_p;
      s_p = t;
      const int u = l_c;
      l_c = l_p;
      l_p = u;
    }
    // no barrier here: the epilogue reads only the exchange fluxes and
    // registers; the next iteration's staging and derivation write other
    // slots, and its flux phase writes the exchange buffers only after the
    // barrier that follows the derivation
  }
  cp_async_wait<0>();
  __syncthreads();
}

// ------------------------------------------------------------- launchers

static int fblocks(long long count) {
  long long b = (count + 255) / 256;
  const long long cap = 32LL * sm_count();
  if (b > cap) b = cap;
  return (int)(b < 1 ? 1 : b);
}

template <typename R>
static Consts<R> fused_consts(const les_params& p) {
  Consts<R> K;
  K.gamma = (R)p.gamma;
  K.gm1 = (R)(p.gamma - 1.0);
  K.k2 = (R)p.k2;
  K.k4 = (R)p.k4;
  K.mu_scale = (R)(p.Re > 0.0 ? p.Mj / p.Re : 0.0);
  K.S_suth = (R)(110.4 / p.T_ref);
  K.cs2 = (R)(p.sgs_model == LES_SGS_VREMAN ? 2.5 * p.Cs * p.Cs : p.Cs * p.Cs);
  K.inv_gm1_pr = (R)(1.0 / ((p.gamma - 1.0) * p.Pr));
  K.inv_gm1_prs = (R)(1.0 / ((p.gamma - 1.0) * p.Pr_sgs));
  K.sgs = p.sgs_model;
  K.axis = p.axis;
  return K;
}

// Axial chunks.  CTAs are dispatched chunk-major (all tiles of a chunk
// together, which keeps neighbouring tiles' halo rows in L2); a CTA takes its
// chunk's planes plus a prologue worth about 1.5 planes (three planes staged,
// two derived, one xi flux: the cost per plane that makes the measured launch
// times of the 288 x 160 x 128 and 576 x 320 x 256 jets agree).  Chunk
// lengths come from a two-level family: n1 chunks of a1 planes first, then
// the other planes split evenly over n2 chunks (n1 = 0: equal chunks).  Long
// chunks first leave the short ones to fill the last wave.  The choice
// minimises the finishing time of a greedy list schedule of the CTAs on the
// SMs, simulated once per grid shape and cached.
struct Chunks {
  int nch, n1, a1;
};

static double chunk_schedule(int ni, int n1, int a1, int n2, int tiles, int slots, double pro) {
  // SM free time -> number of SMs free at that time (times are multiples of
  // 0.5, exact in double); each CTA goes to the earliest free SM
  std::map<double, long long> fr;
  fr[0.0] = slots;
  double t_end = 0.0;
  const long long b = (long long)n1 * a1, rest = ni - b;
  for (int z = 0; z < n1 + n2; ++z) {
    const long long len =
        z < n1 ? a1 : (z - n1 + 1) * rest / n2 - (long long)(z - n1) * rest / n2;
    const double d = (double)len + pro;
    long long need = tiles;
    while (need > 0) {
      auto it = fr.begin();
      const double t = it->first;
      const long long take = need < it->second ? need : it->second;
      if (take == it->second)
        fr.erase(it);
      else
        it->second -= take;
      fr[t + d] += take;
      need -= take;
      if (t + d > t_end) t_end = t + d;
    }
  }
  return t_end;
}

static Chunks choose_chunks(int ni, int tiles, int slots) {
  static std::mutex mu;
  static std::map<std::pair<int, int>, Chunks> cache;
  {
    std::lock_guard<std::mutex> lk(mu);
    auto it = cache.find({ni, tiles});
    if (it != cache.end()) return it->second;
  }
  const double pro = 1.5;
  const long long cap = 24LL * slots;  // at most 24 waves of CTAs
  Chunks best{1, 0, 0};
  double best_t = 1e300;
  auto consider = [&](int n1, int a1, int n2) {
    const double t = chunk_schedule(ni, n1, a1, n2, tiles, slots, pro);
    if (t < best_t - 1e-9) {
      best_t = t;
      best = Chunks{n1 + n2, n1, a1};
    }
  };
  const int max_nch = ni < 64 ? ni : 64;
  for (int n2 = 1; n2 <= max_nch; ++n2) {
    if (n2 > 1 && (long long)tiles * n2 > cap) break;
    consider(0, 0, n2);
  }
  // long chunks about as long as the whole schedule over w waves of them
  const double ideal = (double)ni * tiles / slots + pro;
  for (int n1 = 1; n1 <= 16 && n1 <= max_nch; ++n1) {
    if ((long long)tiles * n1 > cap) break;
    for (int w = 1; w <= 8; ++w) {
      const int a0 = (int)(ideal / w - pro);
      for (int a1 = a0 - 3; a1 <= a0 + 3; ++a1) {
        if (a1 < 1 || (long long)n1 * a1 > ni) continue;
        const int rest = ni - n1 * a1;
        if (rest == 0) {
          consider(n1, a1, 0);
          continue;
        }
        for (int n2 = 1; n2 <= rest && n1 + n2 <= max_nch; ++n2) {
          if ((long long)tiles * (n1 + n2) > cap) break;
          consider(n1, a1, n2);
        }
      }
    }
  }
  std::lock_guard<std::mutex> lk(mu);
  cache[{ni, tiles}] = best;
  return best;
}

template <int MODE, bool LOCAL, bool AXIS, bool DYN, int PM>
static void launch_stage_t(const FusedGeom& G0, const Consts<float>& K, const FusedPtrs& P,
                           const DevScalars* sc, double alpha, const Launch& L) {
  FusedGeom G = G0;
  const size_t smem = (size_t)FLayout<DYN>::FLOATS * sizeof(float);
  // the shared-memory opt-in is a per-device function attribute: set it once
  // for each device this process launches on
  static std::atomic<unsigned long long> attr_set{0};
  int dev = 0;
  cudaGetDevice(&dev);
  const unsigned long long bit = 1ull << (dev & 63);
  if (!(attr_set.load(std::memory_order_acquire) & bit)) {
    cudaFuncSetAttribute(k_stage_fused<MODE, LOCAL, AXIS, DYN, PM>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)smem);
    attr_set.fetch_or(bit, std::memory_order_acq_rel);
  }
  const int tk = (G.nk + FTK - 1) / FTK, tj = (G.nj + FTJ - 1) / FTJ;
  const Chunks ch = choose_chunks(G.ni, tk * tj, sm_count());  // one CTA per SM
  G.nch = ch.nch;
  G.n1 = ch.n1;
  G.a1 = ch.a1;
  dim3 grid(tk, tj, G.nch);
  k_stage_fused<MODE, LOCAL, AXIS, DYN, PM><<<grid, FNT, smem, L.s>>>(G, K, P, sc, alpha);
  ++*L.counter;
}

template <bool AXIS, bool DYN, int PM>
static void launch_stage_dispatch(int mode, bool local, const FusedGeom& G, const Consts<float>& K,
                                  const FusedPtrs& P, const DevScalars* sc, double alpha,
                                  const Launch& L) {
  if (mode == FMODE_RHS)
    launch_stage_t<FMODE_RHS, false, AXIS, DYN, PM>(G, K, P, sc, alpha, L);
  else if (mode == FMODE_STAGE && !local)
    launch_stage_t<FMODE_STAGE, false, AXIS, DYN, PM>(G, K, P, sc, alpha, L);
  else if (mode == FMODE_STAGE)
    launch_stage_t<FMODE_STAGE, true, AXIS, DYN, PM>(G, K, P, sc, alpha, L);
  else if (!local)
    launch_stage_t<FMODE_LAST, false, AXIS, DYN, PM>(G, K, P, sc, alpha, L);
  else
    launch_stage_t<FMODE_LAST, true, AXIS, DYN, PM>(G, K, P, sc, alpha, L);
}

// The jet-grid instantiations (PM = 12 and 28), each compiled in a
// translation unit of its own so the build compiles them in parallel.
void launch_stage_jet12(int mode, bool local, bool axis, bool dyn, const FusedGeom& G,
                        const Consts<float>& K, const FusedPtrs& P, const DevScalars* sc,
                        double alpha, const Launch& L);
void launch_stage_jet28(int mode, bool local, bool axis, bool dyn, const FusedGeom& G,
                        const Consts<float>& K, const FusedPtrs& P, const DevScalars* sc,
                        double alpha, const Launch& L);

}  // namespace lesjet
