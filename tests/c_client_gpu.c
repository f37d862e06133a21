/* A plain-C client of the boundary that runs the method on the device: it
 * includes only lesjet.h and the CUDA runtime header (for the buffers it
 * owns: the library allocates no device memory) and links liblesjet.so and
 * libcudart.  Sequence: les_create, les_workspace_bytes, cudaMalloc,
 * les_grid_jet, les_set_grid, les_init_jet, les_run_n_steps, les_rhs, for
 * the FP64 and the FP32-mixed form on the 48 x 24 x 32 jet.  Writes the
 * initial state, the FP64 and mixed states after NSTEPS steps and the FP64
 * residual of the final state (all [5][N] doubles) to the file named by
 * argv[1], prints "ok <t> <dt>" and exits 0; names the first failing call
 * and exits 1 otherwise. */
#include <cuda_runtime.h>
#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include "lesjet.h"

#define NSTEPS 20

#define CHECK(cond)                                        \
  do {                                                     \
    if (!(cond)) {                                         \
      printf("failed: %s (line %d)\n", #cond, __LINE__);  \
      return 1;                                            \
    }                                                      \
  } while (0)

static les_params jet_params(int precision) {
  les_params p;
  memset(&p, 0, sizeof p);
  p.gamma = 1.4;
  p.Pr = 0.72;
  p.Pr_sgs = 0.9;
  p.Mj = 1.4;
  p.Re = 1.0e5;
  p.T_ref = 288.15;
  p.k2 = 0.25;
  p.k4 = 0.016;
  p.Cs = 0.148;
  p.cfl = 0.5;
  p.r_jet = 0.5;
  p.theta_m = 0.05;
  p.force_width = 0.05;
  p.St[0] = 0.25;
  p.St[1] = 0.5;
  p.St[2] = 0.75;
  p.St[3] = 1.0;
  p.sgs_model = LES_SGS_SMAGORINSKY;
  p.periodic[2] = 1;
  p.bc = LES_BC_JET;
  p.dt_mode = LES_DT_CFL;
  p.freeze_visc = 1;
  p.precision = precision;
  p.metric_form = LES_METRIC_CROSS;
  p.axis = 0;
  p.slab_ghost[0] = p.slab_ghost[1] = 0;
  return p;
}

/* Steps the form `precision` from the initial state Q0_dev; the state after
 * NSTEPS steps goes to host_out. */
static int run_form(int precision, const double *xyz, const double *Q0_dev, size_t N, int ni,
                    int nj, int nk, double *host_out, double *R_out, les_diag *diag) {
  les_params p = jet_params(precision);
  les_ctx *ctx = NULL;
  CHECK(les_create(&p, ni, nj, nk, &ctx) == LES_OK);
  void *ws = NULL, *Q = NULL, *R = NULL;
  CHECK(cudaMalloc(&ws, les_workspace_bytes(ctx)) == cudaSuccess);
  CHECK(cudaMalloc(&Q, 5 * N * sizeof(double)) == cudaSuccess);
  CHECK(cudaMalloc(&R, 5 * N * sizeof(double)) == cudaSuccess);
  CHECK(les_set_grid(ctx, xyz, NULL, ws, NULL) == LES_OK);
  CHECK(cudaMemcpy(Q, Q0_dev, 5 * N * sizeof(double), cudaMemcpyDeviceToDevice) == cudaSuccess);
  CHECK(les_run_n_steps(ctx, NSTEPS, (double *)Q, diag, NULL) == LES_OK);
  CHECK(diag->steps == NSTEPS && diag->status == LES_OK && diag->dt > 0.0 && diag->t > 0.0);
  CHECK(cudaMemcpy(host_out, Q, 5 * N * sizeof(double), cudaMemcpyDeviceToHost) == cudaSuccess);
  if (R_out) {
    CHECK(les_rhs(ctx, (const double *)Q, (double *)R, NULL) == LES_OK);
    CHECK(cudaMemcpy(R_out, R, 5 * N * sizeof(double), cudaMemcpyDeviceToHost) == cudaSuccess);
  }
  CHECK(les_destroy(ctx) == LES_OK);
  cudaFree(R);
  cudaFree(Q);
  cudaFree(ws);
  return 0;
}

int main(int argc, char **argv) {
  CHECK(argc == 2);
  const int ni = 48, nj = 24, nk = 32;
  const size_t N = (size_t)ni * nj * nk;
  double *xyz = NULL, *Q0 = NULL;
  CHECK(cudaMalloc((void **)&xyz, 3 * N * sizeof(double)) == cudaSuccess);
  CHECK(cudaMalloc((void **)&Q0, 5 * N * sizeof(double)) == cudaSuccess);
  const les_jet_grid g = {20.0, 0.0, 0.02, 10.0, 0.5, 0.9, 8.0};
  CHECK(les_grid_jet(ni, nj, nk, &g, xyz, NULL) == LES_OK);

  /* the initial state, from an FP64 context's les_init_jet */
  les_params p = jet_params(LES_PREC_FP64);
  les_ctx *ctx = NULL;
  void *ws = NULL;
  CHECK(les_create(&p, ni, nj, nk, &ctx) == LES_OK);
  CHECK(cudaMalloc(&ws, les_workspace_bytes(ctx)) == cudaSuccess);
  CHECK(les_set_grid(ctx, xyz, NULL, ws, NULL) == LES_OK);
  CHECK(les_init_jet(ctx, xyz, 0, 1.0e-3, Q0, NULL) == LES_OK);
  CHECK(cudaDeviceSynchronize() == cudaSuccess);
  CHECK(les_destroy(ctx) == LES_OK);
  cudaFree(ws);

  double *out = (double *)malloc(4 * 5 * N * sizeof(double));
  CHECK(out != NULL);
  CHECK(cudaMemcpy(out, Q0, 5 * N * sizeof(double), cudaMemcpyDeviceToHost) == cudaSuccess);
  les_diag d64, dm;
  CHECK(run_form(LES_PREC_FP64, xyz, Q0, N, ni, nj, nk, out + 5 * N, out + 15 * N, &d64) == 0);
  CHECK(run_form(LES_PREC_MIXED, xyz, Q0, N, ni, nj, nk, out + 10 * N, NULL, &dm) == 0);
  for (size_t n = 0; n < 20 * N; ++n) CHECK(isfinite(out[n]));
  /* the mixed form within 1e-5 (relative L2 of rho) of FP64, clocks alike */
  double num = 0.0, den = 0.0;
  for (size_t n = 0; n < N; ++n) {
    const double a = out[10 * N + n], b = out[5 * N + n];
    num += (a - b) * (a - b);
    den += b * b;
  }
  CHECK(sqrt(num / den) <= 1.0e-5);
  CHECK(fabs(dm.t - d64.t) <= 1.0e-5 * d64.t);
  FILE *f = fopen(argv[1], "wb");
  CHECK(f != NULL);
  CHECK(fwrite(out, sizeof(double), 20 * N, f) == 20 * N);
  fclose(f);
  free(out);
  cudaFree(Q0);
  cudaFree(xyz);
  printf("ok %.17g %.17g\n", d64.t, d64.dt);
  return 0;
}
