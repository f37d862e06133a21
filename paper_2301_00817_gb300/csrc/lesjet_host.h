// lesjet_host.h -- host-side declarations shared by the .cu files of
// liblesjet: kernel launchers and the precision-dispatch helpers.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/lesjet.h"
#include "lesjet_dev.cuh"

namespace lesjet {

// setup.cu
void launch_metrics(const Grid& g, const double* xyz, const double shift[9], double* M,
                    const Launch& L);
void launch_to_float(long long count, const double* a, float* b, const Launch& L);
void launch_inflow_geometry(const Grid& g, const double* xyz, double* rth, const Launch& L);
void launch_init_jet(const Grid& g, const double* xyz, uint64_t seed, double noise,
                     const les_params& p, double* Q, const Launch& L);

// Pointers of one residual evaluation (v1 multi-kernel path).  R is the
// compute precision; Q_in is double (first stage) or the stage type.
struct StageIO {
  const void* Qin;      // [5][N] stage input state
  int qin_is_double;    // 1: double, 0: float
  const void* M;        // [10][N] metrics (double for FP64, float for mixed)
  void* node;           // [8][N] R: u v w p T lbar_xi lbar_eta lbar_zeta
  void* mk;             // [2][N] R: mu_eff kappa_eff
  void* flux;           // [3][5][N] R: interface fluxes per direction
  double* partials;     // [kRedBlocks] block minima (dt)
  DevScalars* sc;       // device scalars
};

// stage.cu
// precision: LES_PREC_FP64 or LES_PREC_MIXED
void launch_node(int precision, const Grid& g, const les_params& p, const StageIO& io,
                 bool with_dt, const Launch& L);
void launch_dt_finalize(const les_params& p, const StageIO& io, int advance, const Launch& L);
void launch_mu(int precision, const Grid& g, const les_params& p, const StageIO& io,
               const Launch& L);
void launch_flux(int precision, const Grid& g, const les_params& p, const StageIO& io, int dir,
                 const Launch& L);
// mode 0: write RHS to out (double [5][N]); 1: stage update into out
// (stage type: double for FP64, float for mixed); 2: final stage in place
// into out == Q0 (double).
void launch_update(int precision, const Grid& g, const StageIO& io, const double* Q0,
                   double alpha, int mode, void* out, const Launch& L);
void launch_mk_to_double(int precision, const Grid& g, const void* mk, double* out,
                         const Launch& L);

// boundary.cu
void launch_bc_jet(const Grid& g, const les_params& p, double* Q, const double* M64,
                   const double* rth, const DevScalars* sc, int use_host_t, double t_host,
                   const Launch& L);
void launch_totals(const Grid& g, const double* Q, const double* M64, double* partials,
                   DevScalars* sc, const Launch& L);
void launch_set_time(DevScalars* sc, double t, const Launch& L);

}  // namespace lesjet
