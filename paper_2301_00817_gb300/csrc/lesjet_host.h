// lesjet_host.h -- host-side declarations shared by the .cu files of
// liblesjet: kernel launchers and the precision-dispatch helpers.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/lesjet.h"
#include "lesjet_dev.cuh"

namespace lesjet {

// setup.cu
void launch_metrics(const Grid& g, const double* xyz, const double shift[9], int form, double* M,
                    const Launch& L);
void launch_metrics(const Grid& g, const double* xyz, const double shift[9], int form, float* M,
                    const Launch& L);
void launch_to_float(long long count, const double* a, float* b, const Launch& L);
// the metric norms |grad xi_d| and J/2 of M ([10][N]) into gn ([4][N])
void launch_grad_norms(const Grid& g, const double* M, double* gn, const Launch& L);
void launch_inflow_geometry(const Grid& g, const double* xyz, double* rth, const Launch& L);
// synthetic jet grid coordinates [3][N] (s_c: the clustering centre in s)
void launch_grid_jet(const Grid& g, double length, double q, double r0, double r1, double A,
                     double beta, double sc, double* xyz, const Launch& L);
void launch_init_jet(const Grid& g, const double* xyz, uint64_t seed, double noise,
                     const les_params& p, double* Q, const Launch& L);

// stage.cu
// the step every slab takes (the minimum of their own): dt and t^{n+1}
void launch_set_dt(DevScalars* sc, double dt, const Launch& L);
void launch_dt_finalize(const les_params& p, double* partials, DevScalars* sc, int advance,
                        const Launch& L);
void launch_mk_to_double(int precision, const Grid& g, const void* mk, int fields, double* out,
                         const Launch& L);

// stage64.cu (FP64 form): node, viscosity, per-direction flux and update
// passes; each node quantity and interface flux is computed once.
struct StageIO64 {
  const double* Qin;   // [5][N] stage input state
  const double* M;     // [10][N] metrics
  const double* gn = nullptr;  // [4][N] metric norms |grad xi_d| and J/2
                               // (set-up), or nullptr: the kernels evaluate them
  double* node;        // [8][N] u v w p T lbar_xi lbar_eta lbar_zeta
  double* mk;          // [2][N] mu_eff kappa_eff
  double* flux;        // [3][5][N] interface fluxes
  double* partials;    // [kRedBlocks] block minima (dt)
  DevScalars* sc;
  double* dtl = nullptr;  // [N] local steps (dt_mode LOCAL), else nullptr
  double* nu = nullptr;   // [3][N] pressure sensors along xi, eta, zeta
                          // (k_sensor), or nullptr: k_flux evaluates them
  double* dyn = nullptr;  // [50][N] scratch of the dynamic SGS procedure
};
void launch_node64(const Grid& g, const les_params& p, const StageIO64& io, bool with_dt,
                   const Launch& L);
void launch_mu64(const Grid& g, const les_params& p, const StageIO64& io, const Launch& L);
// the dynamic procedure on io.Qin (node quantities in io.node): coefficients
// into io.sc->dyn; io.partials holds 7 x kRedBlocks block sums
void launch_dynamic64(const Grid& g, const les_params& p, const StageIO64& io, double* scratch,
                      const Launch& L);
// the mixed forms' procedure on the float state: FP32 node fields into node
// [8][N], the procedure's fields in FP32 (scratch [50][N]), its sums in
// FP64; coefficients into sc->dyn
void launch_dynamic32(const Grid& g, const les_params& p, const float* Q, const float* M,
                      float* node, float* scratch, double* partials, DevScalars* sc,
                      const Launch& L);
void launch_flux64(const Grid& g, const les_params& p, const StageIO64& io, int dir,
                   const Launch& L);
// the three pressure sensors of every node into io.nu (after launch_node64)
void launch_sensor64(const Grid& g, const StageIO64& io, const Launch& L);
// mode 0: RHS into out; 1: stage update into out; 2: last stage in place
void launch_update64(const Grid& g, const StageIO64& io, const double* Q0, double alpha, int mode,
                     double* out, const Launch& L);

// fused.cu
struct FusedIO {
  const void* Qin;      // stage input state [5][N] (stage type)
  const void* Q0;       // Q^(0): double (FP64) or float hi part (mixed) [5][N]
  void* Q0lo;           // mixed: float lo part of Q^(0) [5][N]
  const void* M;        // metrics [10][N] (double or float)
  const void* mk;       // mu_eff, kappa_eff [2][N] (compute type)
  const DevScalars* sc; // device scalars (dt)
  const float* dtl = nullptr;  // [N] local steps (dt_mode LOCAL), else nullptr
  void* out;            // RHS mode: double [5][N]; stage mode: stage type [5][N]
};
// mixed form: mu_eff/kappa_eff and CFL block minima of the float state
// dyn: the dynamic procedure's coefficients (device) with LES_SGS_DYNAMIC,
// else nullptr
// finalize >= 0 (with sc): the kernel's last block also sets dt from the
// block minima, as launch_dt_finalize(p, partials, sc, finalize) would
void launch_prestep(const Grid& g, const les_params& p, const float* Q0, const float* M,
                    float* mk, double* partials, DevScalars* sc, float* dtl, const double* dyn,
                    const Launch& L, int finalize = -1);
// mode 0: residual into io.out (double); 1: stage update into io.out;
// 2: last stage, Q^(0) (hi, lo) updated in place with compensated sums
void launch_stage_fused(int mode, const Grid& g, const les_params& p, const FusedIO& io,
                        double alpha, const Launch& L);
void launch_split(long long count, const double* q, float* hi, float* lo, const Launch& L);
void launch_join(long long count, const float* hi, const float* lo, double* q, const Launch& L);

// adjoint.cu (FP64): residual tangent / adjoint, viscosity adjoint, stage
// bookkeeping, boundary-condition adjoint and the surface functional
struct Dual;
void launch_rhs_vjp(const Grid& g, const les_params& p, const double* Q, const double* M,
                    const double* gn, const double* node, const double* mk, const double* lamR, double* acc,
                    double* lamQ, double* lamMK, const Launch& L, const double* nu);
void launch_rhs_jvp(const Grid& g, const les_params& p, const Dual* Q, const double* M,
                    const Dual* mk, Dual* node, Dual* flux, Dual* R, const Launch& L);
void launch_mu_vjp(const Grid& g, const les_params& p, const double* Q, const double* lamMK,
                   double* lamQ, const Launch& L);
void launch_stage_prep(const Grid& g, const double* M, double coef, const double* lamS,
                       double* lamR, double* lamQ0, const Launch& L);
void launch_axpy(long long count, double a, const double* x, double* y, const Launch& L);
void launch_bc_vjp(const Grid& g, const les_params& p, const double* M, const double* rth,
                   const double* S5, const double* Qnext, const double* lamNext, double t_next,
                   double* lamS, double* E, double* partials, double* grad, const Launch& L);
void launch_functional(const Grid& g, const les_params& p, int j5, double dt, const double* M,
                       const double* Q, double* lam, double* partials, double* Jout,
                       const Launch& L);
// the same term from FP32 metrics (mixed forms), value only
void launch_functional(const Grid& g, const les_params& p, int j5, double dt, const float* M,
                       const double* Q, double* partials, double* Jout, const Launch& L);
void launch_pack_dual(long long count, const double* v, const double* d, Dual* out, const Launch& L);
void launch_unpack_dual(long long count, const Dual* in, double* v, double* d, const Launch& L);

// boundary.cu
void launch_bc_jet(const Grid& g, const les_params& p, double* Q, const double* M64,
                   const double* rth, const DevScalars* sc, int use_host_t, double t_host,
                   const Launch& L);
void launch_bc_jet(const Grid& g, const les_params& p, double* Q, const float* M32,
                   const double* rth, const DevScalars* sc, int use_host_t, double t_host,
                   const Launch& L);
void launch_bc_jet_hl(const Grid& g, const les_params& p, float* hi, float* lo, const double* M64,
                      const double* rth, const DevScalars* sc, const Launch& L);
void launch_bc_jet_hl(const Grid& g, const les_params& p, float* hi, float* lo, const float* M32,
                      const double* rth, const DevScalars* sc, const Launch& L);
void launch_totals(const Grid& g, const double* Q, const double* M64, double* partials,
                   DevScalars* sc, const Launch& L);
void launch_totals(const Grid& g, const double* Q, const float* M32, double* partials,
                   DevScalars* sc, const Launch& L);
// totals of the mixed form's float pair state (hi + lo)
void launch_totals_hl(const Grid& g, const float* hi, const float* lo, const double* M64,
                      double* partials, DevScalars* sc, const Launch& L);
// the float pair joined into q ([5][N] FP64, e.g. mapped host memory) and
// summed in the same pass (totals_hl's sums, bit for bit)
void launch_join_totals_hl(const Grid& g, const float* hi, const float* lo, const double* M64,
                           double* q, double* partials, DevScalars* sc, const Launch& L);
void launch_join_totals_hl(const Grid& g, const float* hi, const float* lo, const float* M32,
                           double* q, double* partials, DevScalars* sc, const Launch& L);
void launch_totals_hl(const Grid& g, const float* hi, const float* lo, const float* M32,
                      double* partials, DevScalars* sc, const Launch& L);
void launch_set_time(DevScalars* sc, double t, const Launch& L);

}  // namespace lesjet
