/* A plain-C client of the boundary: it includes only lesjet.h and links only
 * liblesjet.so (no Python, no torch).  It makes the host-only calls, which
 * touch no device: context creation and validation, workspace sizing, the
 * grid generator's argument checks, the state machine (stepping before a
 * grid is bound), and the error messages.  Prints "ok" and exits 0 when
 * every check holds, else names the first failing check and exits 1. */
#include <stdio.h>
#include <string.h>

#include "lesjet.h"

#define CHECK(cond)                                        \
  do {                                                     \
    if (!(cond)) {                                         \
      printf("failed: %s (line %d)\n", #cond, __LINE__);  \
      return 1;                                            \
    }                                                      \
  } while (0)

/* The jet workload's parameters, as the header documents them. */
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

int main(void) {
  const int ni = 48, nj = 24, nk = 32;
  const size_t N = (size_t)ni * nj * nk;
  les_ctx *ctx = NULL;

  les_params p64 = jet_params(LES_PREC_FP64);
  CHECK(les_create(&p64, ni, nj, nk, &ctx) == LES_OK && ctx != NULL);
  const size_t ws64 = les_workspace_bytes(ctx);
  CHECK(ws64 >= N * 8 * (10 + 2 + 10));  /* metrics, mu/kappa, two stage states */
  /* stepping before les_set_grid is refused without touching the device */
  CHECK(les_rk_step(ctx, (double *)16, NULL) == LES_ERR_STATE);
  CHECK(strlen(les_last_error(ctx)) > 0);
  CHECK(les_destroy(ctx) == LES_OK);

  les_params pm = jet_params(LES_PREC_MIXED);
  CHECK(les_create(&pm, ni, nj, nk, &ctx) == LES_OK);
  const size_t wsm = les_workspace_bytes(ctx);
  CHECK(wsm > 0 && wsm < ws64);
  CHECK(les_destroy(ctx) == LES_OK);

  /* shape and parameter validation */
  CHECK(les_create(&p64, 4, nj, nk, &ctx) == LES_ERR_SHAPE);
  les_params bad = jet_params(LES_PREC_FP64);
  bad.sgs_model = 7;
  CHECK(les_create(&bad, ni, nj, nk, &ctx) == LES_ERR_INVALID_ARG);
  bad = jet_params(LES_PREC_FP64);
  bad.periodic[0] = 1; /* the jet boundary conditions need periodic = {0, 0, 1} */
  CHECK(les_create(&bad, ni, nj, nk, &ctx) == LES_ERR_INVALID_ARG);

  /* the grid generator checks its arguments before any device work */
  les_jet_grid g = {20.0, 0.0, 0.02, 10.0, 0.5, 0.9, 8.0};
  CHECK(les_grid_jet(1, nj, nk, &g, (double *)16, NULL) == LES_ERR_SHAPE);
  CHECK(les_grid_jet(ni, nj, nk, NULL, (double *)16, NULL) == LES_ERR_INVALID_ARG);
  CHECK(les_grid_jet(ni, nj, nk, &g, (double *)24, NULL) == LES_ERR_ALIGN);
  g.r_c = 20.0; /* outside (r0, r1) */
  CHECK(les_grid_jet(ni, nj, nk, &g, (double *)16, NULL) == LES_ERR_INVALID_ARG);

  printf("ok\n");
  return 0;
}
