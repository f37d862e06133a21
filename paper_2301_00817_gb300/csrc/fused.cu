// fused.cu -- launchers of the FP32-mixed form: the fused stage kernel
// (fused_kernel.cuh; the jet-grid instantiations in fused_jet12.cu and
// fused_jet28.cu), the once-per-step viscosity/CFL pass (k_prestep, and
// its four-node form k_prestep4 here) and the split and join of the
// float-pair state.  Built with approximate FP32 division and
// square root.
#include "fused_kernel.cuh"

namespace lesjet {

// ------------------------------------------------------- mixed-state helpers
// Q (double) -> (hi, lo) floats with hi + lo == Q to ~2^-48 relative.
__global__ void k_split(long long count, const double* __restrict__ q, float* __restrict__ hi,
                        float* __restrict__ lo) {
  for (long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x; n < count;
       n += (long long)gridDim.x * blockDim.x) {
    const double v = q[n];
    const float h = (float)v;
    hi[n] = h;
    lo[n] = (float)(v - (double)h);
  }
}

__global__ void k_join(long long count, const float* __restrict__ hi, const float* __restrict__ lo,
                       double* __restrict__ q) {
  for (long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x; n < count;
       n += (long long)gridDim.x * blockDim.x)
    q[n] = (double)hi[n] + (double)lo[n];
}

// Component j (0..3, a compile-time constant after unrolling) of a float4.
__device__ __forceinline__ float f4c(const float4& a, int j) {
  return j == 0 ? a.x : (j == 1 ? a.y : (j == 2 ? a.z : a.w));
}

// k_prestep for the static SGS models on grids with nk % 4 == 0 and no axis:
// one thread per four consecutive zeta nodes, so the state, metric and
// output rows and the xi and eta neighbour rows move as float4 and the zeta
// neighbours inside the group come from registers (about a third of the
// one-node form's load instructions).  The arithmetic per node is the one
// of k_prestep; the metrics are re-read per direction (from cache) rather
// than held, which keeps the kernel at two 256-thread blocks per SM.
__global__ void __launch_bounds__(256, 2) k_prestep4(Grid g, Consts<float> K,
                                                     const float* __restrict__ Q,
                                                     const float* __restrict__ M,
                                                     float* __restrict__ mk,
                                                     double* __restrict__ partials,
                                                     DevScalars* __restrict__ sc,
                                                     float* __restrict__ dtl, float cfl,
                                                     int fin_mode, double fin_cfl, double fin_dt,
                                                     int fin_advance) {
  const long long N = g.N, NQ = N >> 2;  // float4 rows per field
  const float4* Q4 = reinterpret_cast<const float4*>(Q);
  const float4* M4 = reinterpret_cast<const float4*>(M);
  float local_min = 1e30f;
  int bad = 0;
  for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < NQ;
       q += (long long)gridDim.x * blockDim.x) {
    const long long n = q << 2;
    int c[3];
    decompose(g, n, c);  // c[2] is a multiple of 4
    float rho[4], u[4], v[4], w[4], mul[4], ro[4];
    {
      const float4 f0 = Q4[q], f1 = Q4[NQ + q], f2 = Q4[2 * NQ + q], f3 = Q4[3 * NQ + q],
                   f4 = Q4[4 * NQ + q];
      float T[4], p[4];
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        rho[j] = f4c(f0, j);
        const float ir = 1.f / rho[j];
        u[j] = f4c(f1, j) * ir;
        v[j] = f4c(f2, j) * ir;
        w[j] = f4c(f3, j) * ir;
        p[j] = K.gm1 * (f4c(f4, j) - 0.5f * rho[j] * (u[j] * u[j] + v[j] * v[j] + w[j] * w[j]));
        T[j] = K.gamma * p[j] * ir;
      }
      float lsum[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
      for (int d = 0; d < 3; ++d) {
        const float4 mx = M4[(3 * d) * NQ + q], my = M4[(3 * d + 1) * NQ + q],
                     mz = M4[(3 * d + 2) * NQ + q];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          const float ax = f4c(mx, j), ay = f4c(my, j), az = f4c(mz, j);
          lsum[j] += dev_abs(ax * u[j] + ay * v[j] + az * w[j]) +
                     dev_sqrt(T[j]) * dev_sqrt(ax * ax + ay * ay + az * az);
        }
      }
      const bool owned = (g.glo | g.ghi) == 0 || owned_plane(g, c[0]);
      float inv[4];
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        inv[j] = 1.f / lsum[j];
        if (owned) {
          if (!(rho[j] > 0.f) || !(p[j] > 0.f) || !(inv[j] > 0.f) || !(inv[j] < 1e30f)) bad = 1;
          local_min = inv[j] < local_min ? inv[j] : local_min;
        }
        mul[j] = K.mu_scale * T[j] * dev_sqrt(T[j]) * (1.f + K.S_suth) / (T[j] + K.S_suth);
      }
      if (dtl)
        reinterpret_cast<float4*>(dtl)[q] =
            make_float4(cfl * inv[0], cfl * inv[1], cfl * inv[2], cfl * inv[3]);
    }
    float mus[4] = {0.f, 0.f, 0.f, 0.f};
    if (K.sgs != LES_SGS_NONE) {
      // gr[qq][x][j] = sum_d m[3d + x] dd[qq][d], accumulated direction by
      // direction in the order d = 0, 1, 2
      float gr[3][3][4];
#pragma unroll
      for (int d = 0; d < 3; ++d) {
        float dd[3][4];  // dd[qq][j] = computational derivative of u_qq along d
        if (d < 2) {
          // xi and eta: the neighbour rows are whole float4 rows
          const long long s = g.stride[d] >> 2;
          const int nd = g.n[d];
          long long qp, qm;
          int mode;
          if (g.per[d]) {
            qp = (c[d] == nd - 1) ? q - (long long)(nd - 1) * s : q + s;
            qm = (c[d] == 0) ? q + (long long)(nd - 1) * s : q - s;
            mode = 0;
          } else if (c[d] == 0) {
            qp = q + s;
            qm = q + 2 * s;
            mode = 1;
          } else if (c[d] == nd - 1) {
            qp = q - 2 * s;
            qm = q - s;
            mode = 2;
          } else {
            qp = q + s;
            qm = q - s;
            mode = 0;
          }
          const float4 p0 = Q4[qp], p1 = Q4[NQ + qp], p2 = Q4[2 * NQ + qp], p3 = Q4[3 * NQ + qp];
          const float4 m0 = Q4[qm], m1 = Q4[NQ + qm], m2 = Q4[2 * NQ + qm], m3 = Q4[3 * NQ + qm];
#pragma unroll
          for (int j = 0; j < 4; ++j) {
            const float irp = 1.f / f4c(p0, j), irm = 1.f / f4c(m0, j);
            const float fp[3] = {f4c(p1, j) * irp, f4c(p2, j) * irp, f4c(p3, j) * irp};
            const float fm[3] = {f4c(m1, j) * irm, f4c(m2, j) * irm, f4c(m3, j) * irm};
            const float f0[3] = {u[j], v[j], w[j]};
#pragma unroll
            for (int qq = 0; qq < 3; ++qq) {
              if (mode == 0)
                dd[qq][j] = 0.5f * (fp[qq] - fm[qq]);
              else if (mode == 1)  // (-3 f0 + 4 f1 - f2)/2 with f1 = fp, f2 = fm
                dd[qq][j] = 0.5f * (-3.f * f0[qq] + 4.f * fp[qq] - fm[qq]);
              else  // (3 f0 - 4 f_{-1} + f_{-2})/2 with f_{-1} = fm, f_{-2} = fp
                dd[qq][j] = 0.5f * (3.f * f0[qq] - 4.f * fm[qq] + fp[qq]);
            }
          }
        } else {
          // zeta: positions -1 .. 4 of the group, the outer two loaded
          const int nk = g.n[2], k0 = c[2];
          const bool per = g.per[2] != 0;
          float vl[3] = {0.f, 0.f, 0.f}, vr[3] = {0.f, 0.f, 0.f};
          if (per || k0 > 0) {
            const long long nl = (k0 == 0) ? n + nk - 1 : n - 1;
            const float ir = 1.f / Q[nl];
            vl[0] = Q[N + nl] * ir;
            vl[1] = Q[2 * N + nl] * ir;
            vl[2] = Q[3 * N + nl] * ir;
          }
          if (per || k0 + 4 < nk) {
            const long long nr = (k0 + 4 >= nk) ? n + 4 - nk : n + 4;
            const float ir = 1.f / Q[nr];
            vr[0] = Q[N + nr] * ir;
            vr[1] = Q[2 * N + nr] * ir;
            vr[2] = Q[3 * N + nr] * ir;
          }
#pragma unroll
          for (int qq = 0; qq < 3; ++qq) {
            const float* own = qq == 0 ? u : (qq == 1 ? v : w);
            float f[6];
            f[0] = vl[qq];
#pragma unroll
            for (int j = 0; j < 4; ++j) f[j + 1] = own[j];
            f[5] = vr[qq];
#pragma unroll
            for (int j = 0; j < 4; ++j) {
              const int k = k0 + j;
              // k0 is a multiple of 4, so only node 0 can lie on the face
              // k = 0 and only node 3 on the face k = nk - 1
              if (per || (k > 0 && k < nk - 1))
                dd[qq][j] = 0.5f * (f[j + 2] - f[j]);
              else if (j == 0)  // k == 0: (-3 f0 + 4 f1 - f2)/2
                dd[qq][0] = 0.5f * (-3.f * f[1] + 4.f * f[2] - f[3]);
              else  // k == nk - 1: (3 f0 - 4 f_{-1} + f_{-2})/2
                dd[qq][j] = 0.5f * (3.f * f[j + 1] - 4.f * f[j] + f[j - 1]);
            }
          }
        }
        const float4 mx = M4[(3 * d) * NQ + q], my = M4[(3 * d + 1) * NQ + q],
                     mz = M4[(3 * d + 2) * NQ + q];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          const float mr[3] = {f4c(mx, j), f4c(my, j), f4c(mz, j)};
#pragma unroll
          for (int qq = 0; qq < 3; ++qq)
#pragma unroll
            for (int x = 0; x < 3; ++x) {
              if (d == 0)
                gr[qq][x][j] = mr[x] * dd[qq][j];
              else
                gr[qq][x][j] += mr[x] * dd[qq][j];
            }
        }
      }
      const float4 Jv = M4[9 * NQ + q];
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const float delta = cbrtf(f4c(Jv, j));
        if (K.sgs == LES_SGS_SMAGORINSKY) {
          float ss = 0.f;
#pragma unroll
          for (int a = 0; a < 3; ++a)
#pragma unroll
            for (int b = 0; b < 3; ++b) {
              const float sab = 0.5f * (gr[a][b][j] + gr[b][a][j]);
              ss += sab * sab;
            }
          mus[j] = rho[j] * (delta * delta) * K.cs2 * dev_sqrt(2.f * ss);
        } else {
          float aa = 0.f;
#pragma unroll
          for (int a = 0; a < 3; ++a)
#pragma unroll
            for (int b = 0; b < 3; ++b) aa += gr[a][b][j] * gr[a][b][j];
          float be[3][3];
#pragma unroll
          for (int a = 0; a < 3; ++a)
#pragma unroll
            for (int b = 0; b < 3; ++b)
              be[a][b] = delta * delta *
                         (gr[a][0][j] * gr[b][0][j] + gr[a][1][j] * gr[b][1][j] +
                          gr[a][2][j] * gr[b][2][j]);
          float B = be[0][0] * be[1][1] - be[0][1] * be[0][1] + be[0][0] * be[2][2] -
                    be[0][2] * be[0][2] + be[1][1] * be[2][2] - be[1][2] * be[1][2];
          B = B > 0.f ? B : 0.f;
          mus[j] = (aa == 0.f) ? 0.f : rho[j] * K.cs2 * dev_sqrt(B / aa);
        }
      }
    }
#pragma unroll
    for (int j = 0; j < 4; ++j) ro[j] = mul[j] + mus[j];
    reinterpret_cast<float4*>(mk)[q] = make_float4(ro[0], ro[1], ro[2], ro[3]);
#pragma unroll
    for (int j = 0; j < 4; ++j) ro[j] = mul[j] * K.inv_gm1_pr + mus[j] * K.inv_gm1_prs;
    reinterpret_cast<float4*>(mk)[NQ + q] = make_float4(ro[0], ro[1], ro[2], ro[3]);
  }
  prestep_finish(local_min, bad, partials, sc, fin_mode, fin_cfl, fin_dt, fin_advance);
}

void launch_prestep(const Grid& g, const les_params& p, const float* Q0, const float* M,
                    float* mk, double* partials, DevScalars* sc, float* dtl, const double* dyn,
                    const Launch& L, int finalize) {
  // finalize >= 0: the kernel's last block also takes the step (advance = finalize)
  const int fm = finalize >= 0 ? p.dt_mode : -1;
  const Consts<float> K = fused_consts<float>(p);
  // four zeta nodes per thread where the rows are float4 rows (nk % 4 == 0,
  // 16-byte aligned fields), the static models and no axis
  const bool al16 = ((reinterpret_cast<uintptr_t>(Q0) | reinterpret_cast<uintptr_t>(M) |
                      reinterpret_cast<uintptr_t>(mk) | reinterpret_cast<uintptr_t>(dtl)) &
                     15) == 0;
  if (p.sgs_model != LES_SGS_DYNAMIC && !p.axis && g.n[2] % 4 == 0 && al16)
    k_prestep4<<<kRedBlocks, kRedThreads, 0, L.s>>>(g, K, Q0, M, mk, partials, sc, dtl,
                                                     (float)p.cfl, fm, p.cfl, p.dt_fixed, finalize);
  else if (p.sgs_model == LES_SGS_DYNAMIC)
    k_prestep<float, float, float, true><<<kRedBlocks, kRedThreads, 0, L.s>>>(
        g, K, Q0, M, mk, partials, sc, dtl, (float)p.cfl, dyn, fm, p.cfl, p.dt_fixed, finalize);
  else
    k_prestep<float, float, float, false><<<kRedBlocks, kRedThreads, 0, L.s>>>(
        g, K, Q0, M, mk, partials, sc, dtl, (float)p.cfl, dyn, fm, p.cfl, p.dt_fixed, finalize);
  ++*L.counter;
  if (p.axis) {
    k_mu_axis<float, TempFromState<float, float>><<<g.n[0], 128, g.n[2] * sizeof(float), L.s>>>(
        g, K, TempFromState<float, float>{Q0, g.N, K.gamma, K.gm1}, mk);
    ++*L.counter;
  }
}

void launch_stage_fused(int mode, const Grid& g, const les_params& p, const FusedIO& io,
                        double alpha, const Launch& L) {
  FusedGeom G;
  G.ni = g.n[0];
  G.nj = g.n[1];
  G.nk = g.n[2];
  for (int d = 0; d < 3; ++d) G.per[d] = g.per[d];
  G.nch = 1;
  G.n1 = 0;
  G.a1 = 0;
  G.vec16 = (g.per[2] && g.n[2] % 4 == 0 && g.n[2] >= FTK) ? 1 : 0;
  // inside the physical faces and, for an axial slab, its own planes
  G.ilo = g.glo > 0 ? g.glo : 1;
  G.ihi = g.n[0] - (g.ghi > 0 ? g.ghi : 1);
  const long long N = g.N;
  G.N = (int)N;  // the mixed forms hold N < 2^31 (checked at creation)
  FusedPtrs P;
  for (int c = 0; c < 5; ++c) {
    P.qin[c] = (const float*)io.Qin + c * N;
    P.hi[c] = (const float*)io.Q0 + c * N;
    P.hiw[c] = (float*)io.Q0 + c * N;
    P.lo[c] = io.Q0lo ? (float*)io.Q0lo + c * N : nullptr;
    P.out[c] = (mode == FMODE_STAGE) ? (float*)io.out + c * N : nullptr;
    P.outd[c] = (mode == FMODE_RHS) ? (double*)io.out + c * N : nullptr;
  }
  for (int t = 0; t < 10; ++t) P.m[t] = (const float*)io.M + t * N;
  const bool dyn = p.sgs_model == LES_SGS_DYNAMIC;
  for (int t = 0; t < 3; ++t) P.mk[t] = (t < 2 || dyn) ? (const float*)io.mk + t * N : nullptr;
  P.dtl = io.dtl;
  const Consts<float> K = fused_consts<float>(p);
  const bool local = P.dtl != nullptr;
  // The jet grids (xi and eta bounded, zeta periodic, shifted 16-byte
  // staging) get instantiations with these fixed at compile time, which fold
  // the face, wrap and one-sided-difference tests: PM = 12, and PM = 28 when
  // the tiles also cover eta and zeta exactly (every thread owns a column).
  // Other grids read them at run time (PM = -1).
  const bool jet = !g.per[0] && !g.per[1] && g.per[2] && G.vec16;
  const bool full = g.n[1] % FTJ == 0 && g.n[2] % FTK == 0;
  const int pm = jet ? (full ? 28 : 12) : -1;
  if (pm == 28)
    launch_stage_jet28(mode, local, p.axis != 0, dyn, G, K, P, io.sc, alpha, L);
  else if (pm == 12)
    launch_stage_jet12(mode, local, p.axis != 0, dyn, G, K, P, io.sc, alpha, L);
  else if (dyn)  // (not with an axis: rejected at creation)
    launch_stage_dispatch<false, true, -1>(mode, local, G, K, P, io.sc, alpha, L);
  else if (p.axis)
    launch_stage_dispatch<true, false, -1>(mode, local, G, K, P, io.sc, alpha, L);
  else
    launch_stage_dispatch<false, false, -1>(mode, local, G, K, P, io.sc, alpha, L);
}

void launch_split(long long count, const double* q, float* hi, float* lo, const Launch& L) {
  k_split<<<fblocks(count), 256, 0, L.s>>>(count, q, hi, lo);
  ++*L.counter;
}

void launch_join(long long count, const float* hi, const float* lo, double* q, const Launch& L) {
  k_join<<<fblocks(count), 256, 0, L.s>>>(count, hi, lo, q);
  ++*L.counter;
}

}  // namespace lesjet
