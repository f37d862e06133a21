// fused.cu -- launchers of the FP32-mixed form: the fused stage kernel
// (fused_kernel.cuh; the jet-grid instantiations in fused_jet12.cu and
// fused_jet28.cu), the once-per-step viscosity/CFL pass and the split and
// join of the float-pair state.  Built with approximate FP32 division and
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

void launch_prestep(const Grid& g, const les_params& p, const float* Q0, const float* M,
                    float* mk, double* partials, DevScalars* sc, float* dtl, const double* dyn,
                    const Launch& L, int finalize) {
  // finalize >= 0: the kernel's last block also takes the step (advance = finalize)
  const int fm = finalize >= 0 ? p.dt_mode : -1;
  const Consts<float> K = fused_consts<float>(p);
  if (p.sgs_model == LES_SGS_DYNAMIC)
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
