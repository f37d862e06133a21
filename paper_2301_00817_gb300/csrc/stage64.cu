// stage64.cu -- residual and Runge-Kutta stage kernels of the FP64 form.
//
// GB300 keeps little FP64 throughput, so the FP64 form is bound by its
// arithmetic, not by HBM: it computes every node quantity and every interface
// flux exactly once, in four passes per residual evaluation:
//   k_node    per node: primitives u v w p T and the anisotropic spectral
//             radii lbar (optionally the block minima of the CFL step);
//   k_mu      per node: mu_eff, kappa_eff (Sutherland + SGS);
//   k_flux<D> per interface (n, n + e_D): centred inviscid flux minus J^-1
//             times the Turkel-Vatsa dissipation minus the viscous flux,
//             stored as exactly twice its value (the interface means'
//             factors 1/2 are folded away);
//   k_update  per node: RHS = sum_D (F_{+1/2} - F_{-1/2}) and the stage
//             update Q^(l) = Q^(0) - alpha_l dt J RHS (or RHS itself), with
//             the factor 2 taken out once per node.
// Each interface is computed once and read by its two nodes, so the scheme
// telescopes exactly.  The kernels are written for a compute type R: double
// here, and dual numbers in adjoint.cu (the exact tangent of the residual);
// the mixed form uses fused.cu.
#include <cstddef>

#include "stage64_kernels.cuh"

namespace lesjet {

// ------------------------------------------------------------- launchers

void launch_node64(const Grid& g, const les_params& p, const StageIO64& io, bool with_dt,
                   const Launch& L) {
  const int th = 256;
  const int nb = with_dt ? kRedBlocks : blocks_for(g.N, th);
  auto K = make_consts<double>(p);
  if (with_dt)
    k_node<double, double, double, true><<<nb, th, 0, L.s>>>(g, K, io.Qin, io.M, io.gn, io.node,
                                                             io.partials, io.sc, io.dtl, p.cfl);
  else
    k_node<double, double, double, false><<<nb, th, 0, L.s>>>(g, K, io.Qin, io.M, io.gn, io.node,
                                                              io.partials, io.sc);
  ++*L.counter;
}

void launch_mu64(const Grid& g, const les_params& p, const StageIO64& io, const Launch& L) {
  const int th = 256, nb = blocks_for(g.N, th);
  const double* dyn = nullptr;
  if (p.sgs_model == LES_SGS_DYNAMIC) {
    launch_dynamic64(g, p, io, io.dyn, L);
    dyn = reinterpret_cast<const double*>(reinterpret_cast<const char*>(io.sc) +
                                          offsetof(DevScalars, dyn));
  }
  k_mu<double, double, double><<<nb, th, 0, L.s>>>(g, make_consts<double>(p), io.Qin, io.M,
                                                    io.node, io.mk, dyn);
  ++*L.counter;
  if (p.axis) {
    k_mu_axis<double, TempFromNode<double>><<<g.n[0], 128, g.n[2] * sizeof(double), L.s>>>(
        g, make_consts<double>(p), TempFromNode<double>{io.node, g.N}, io.mk);
    ++*L.counter;
  }
}

void launch_flux64(const Grid& g, const les_params& p, const StageIO64& io, int dir,
                   const Launch& L) {
  const int th = 256, nb = blocks_for(g.N, th);
  auto K = make_consts<double>(p);
  double* F = io.flux + 5 * g.N * dir;
  if (dir == 0)
    k_flux<0, double, double, double><<<nb, th, 0, L.s>>>(g, K, io.Qin, io.M, io.node, io.mk, F,
                                                          io.nu);
  else if (dir == 1)
    k_flux<1, double, double, double><<<nb, th, 0, L.s>>>(g, K, io.Qin, io.M, io.node, io.mk, F,
                                                          io.nu);
  else
    k_flux<2, double, double, double><<<nb, th, 0, L.s>>>(g, K, io.Qin, io.M, io.node, io.mk, F,
                                                          io.nu);
  ++*L.counter;
}

void launch_sensor64(const Grid& g, const StageIO64& io, const Launch& L) {
  if (!io.nu) return;
  const int th = 256, nb = blocks_for(g.N, th);
  k_sensor<double><<<nb, th, 0, L.s>>>(g, io.node + 3 * g.N, io.nu);
  ++*L.counter;
}

void launch_update64(const Grid& g, const StageIO64& io, const double* Q0, double alpha, int mode,
                     double* out, const Launch& L) {
  const int th = 256, nb = blocks_for(g.N, th);
  if (mode == 0)
    k_update<double, double, double, 0><<<nb, th, 0, L.s>>>(g, io.flux, Q0, io.M, io.sc, alpha, out, io.dtl);
  else if (mode == 1)
    k_update<double, double, double, 1><<<nb, th, 0, L.s>>>(g, io.flux, Q0, io.M, io.sc, alpha, out, io.dtl,
                                                            io.gn ? io.gn + 3 * g.N : nullptr);
  else
    k_update<double, double, double, 2><<<nb, th, 0, L.s>>>(g, io.flux, Q0, io.M, io.sc, alpha, out, io.dtl,
                                                            io.gn ? io.gn + 3 * g.N : nullptr);
  ++*L.counter;
}

}  // namespace lesjet
