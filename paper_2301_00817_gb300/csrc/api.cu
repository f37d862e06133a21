// api.cu -- the extern "C" boundary of liblesjet: argument validation,
// workspace layout and the order of kernel launches of one time step
// (Table tab:JAZzY: viscosity, time step, five Runge-Kutta stages, boundary
// conditions).  The library allocates no device memory.
#include <cuda.h>  // driver types only (entry points come through the runtime)
#include <cuda_runtime.h>

#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include "../../include/lesjet.h"
#include "dual.cuh"
#include "lesjet_dev.cuh"
#include "lesjet_host.h"

using lesjet::DevScalars;
using lesjet::Grid;

// Kernel classes timed by the optional event profiler.
enum ProfKind {
  PK_PRESTEP = 0, PK_DT, PK_STAGE, PK_NODE, PK_MU, PK_FLUX, PK_UPDATE, PK_BC, PK_TOTALS,
  PK_CONVERT, PK_COUNT
};
static const char* kProfNames[PK_COUNT] = {"prestep", "dt_finalize", "stage_fused", "node",
                                           "mu_eff",  "flux",        "update",      "bc_jet",
                                           "totals",  "convert"};

struct ProfRec {
  int kind;
  cudaEvent_t a, b;
};

struct les_ctx {
  les_params p;
  Grid g;
  // workspace layout (byte offsets, 256-byte aligned)
  size_t off_m64, off_m32, off_mk, off_sa, off_sb, off_hi, off_lo, off_node, off_flux, off_nu, off_gn, off_rth,
      off_sc, off_part, off_dtl, off_dyn;
  size_t total;
  bool local_dt;  // the workspace holds per-node steps (dt_mode LOCAL at creation)
  bool dyn_ws;    // the workspace holds the dynamic SGS scratch (sgs DYNAMIC at creation)
  char* ws;
  bool grid_set;
  std::string err;
  unsigned long long launches;
  // event profiler (off unless les_profile(ctx, 1))
  bool prof_on;
  std::vector<ProfRec> prof_pending;
  std::vector<cudaEvent_t> prof_pool;
  double prof_ms[PK_COUNT];
  unsigned long long prof_n[PK_COUNT];
  // the FP32-mixed step as a CUDA graph (mixed_steps): its executable, the
  // stream it is captured on, and the kernel launches one replay stands for
  cudaGraphExec_t step_exec = nullptr;
  cudaStream_t cap_stream = nullptr;
  unsigned long long step_launches = 0;
  bool graph_failed = false;
};

namespace {

constexpr double kAlpha[5] = {1.0 / 4.0, 1.0 / 6.0, 3.0 / 8.0, 1.0 / 2.0, 1.0};

size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

int fail(les_ctx* c, int code, const char* msg) {
  if (c) c->err = msg;
  return code;
}

void drop_step_graph(les_ctx* c) {
  if (c->step_exec) cudaGraphExecDestroy(c->step_exec);
  c->step_exec = nullptr;
  c->graph_failed = false;
}

int cuda_check(les_ctx* c, const char* where) {
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    if (c) c->err = std::string(where) + ": " + cudaGetErrorString(e);
    return LES_ERR_CUDA;
  }
  return LES_OK;
}

cudaEvent_t prof_event(les_ctx* c) {
  if (!c->prof_pool.empty()) {
    cudaEvent_t e = c->prof_pool.back();
    c->prof_pool.pop_back();
    return e;
  }
  cudaEvent_t e;
  cudaEventCreate(&e);
  return e;
}

// Records an event pair around one launch group on its own stream.
struct ProfScope {
  les_ctx* c;
  int kind;
  cudaStream_t s;
  cudaEvent_t a;
  ProfScope(les_ctx* c_, int kind_, cudaStream_t s_) : c(c_), kind(kind_), s(s_), a(nullptr) {
    if (c->prof_on) {
      a = prof_event(c);
      cudaEventRecord(a, s);
    }
  }
  ~ProfScope() {
    if (c->prof_on && a) {
      cudaEvent_t b = prof_event(c);
      cudaEventRecord(b, s);
      c->prof_pending.push_back(ProfRec{kind, a, b});
    }
  }
};

bool aligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

int validate_params(const les_params* p, std::string& why) {
  if (!(p->gamma > 1.0) || !(p->Pr > 0.0) || !(p->Pr_sgs > 0.0) || !(p->Mj > 0.0) ||
      !(p->T_ref > 0.0) || !(p->k2 >= 0.0) || !(p->k4 >= 0.0) || !(p->Cs >= 0.0)) {
    why = "gamma > 1, Pr, Pr_sgs, Mj, T_ref > 0 and k2, k4, Cs >= 0 are required";
    return LES_ERR_INVALID_ARG;
  }
  if (p->sgs_model < 0 || p->sgs_model > 3) {
    why = "sgs_model must be LES_SGS_NONE, LES_SGS_SMAGORINSKY, LES_SGS_VREMAN or LES_SGS_DYNAMIC";
    return LES_ERR_INVALID_ARG;
  }
  if (p->precision != LES_PREC_FP64 && p->precision != LES_PREC_MIXED &&
      p->precision != LES_PREC_MIXED_COMPACT) {
    why = "precision must be LES_PREC_FP64, LES_PREC_MIXED or LES_PREC_MIXED_COMPACT";
    return LES_ERR_INVALID_ARG;
  }
  if (p->dt_mode == LES_DT_CFL || p->dt_mode == LES_DT_LOCAL
          ? !(p->cfl > 0.0)
          : (p->dt_mode != LES_DT_FIXED || !(p->dt_fixed > 0.0))) {
    why = "dt_mode CFL or LOCAL needs cfl > 0; dt_mode FIXED needs dt_fixed > 0";
    return LES_ERR_INVALID_ARG;
  }
  if (p->metric_form != LES_METRIC_CROSS && p->metric_form != LES_METRIC_CONSERVATIVE) {
    why = "metric_form must be LES_METRIC_CROSS or LES_METRIC_CONSERVATIVE";
    return LES_ERR_INVALID_ARG;
  }
  if (p->bc != LES_BC_FROZEN && p->bc != LES_BC_JET && p->bc != LES_BC_JET_CHAR) {
    why = "bc must be LES_BC_FROZEN, LES_BC_JET or LES_BC_JET_CHAR";
    return LES_ERR_INVALID_ARG;
  }
  const bool jet = p->bc == LES_BC_JET || p->bc == LES_BC_JET_CHAR;
  if (jet && !(p->periodic[0] == 0 && p->periodic[1] == 0 && p->periodic[2] == 1)) {
    why = "jet boundary conditions need periodic = {0, 0, 1}";
    return LES_ERR_INVALID_ARG;
  }
  if (jet && !(p->theta_m > 0.0 && p->force_width > 0.0)) {
    why = "jet boundary conditions need theta_m > 0 and force_width > 0";
    return LES_ERR_INVALID_ARG;
  }
  if (p->axis != 0 && p->axis != 1) {
    why = "axis must be 0 or 1";
    return LES_ERR_INVALID_ARG;
  }
  if (p->axis && !(p->periodic[0] == 0 && p->periodic[1] == 0 && p->periodic[2] == 1)) {
    why = "a grid with an axis needs periodic = {0, 0, 1} (ring j = 0 on the axis)";
    return LES_ERR_INVALID_ARG;
  }
  for (int e = 0; e < 2; ++e)
    if (p->slab_ghost[e] != 0 && p->slab_ghost[e] != 2) {
      why = "slab_ghost entries must be 0 (a physical face) or 2 (a cut between slabs)";
      return LES_ERR_INVALID_ARG;
    }
  const bool slab = p->slab_ghost[0] || p->slab_ghost[1];
  if (slab && p->periodic[0]) {
    why = "axial slabs need a non-periodic xi (periodic[0] = 0)";
    return LES_ERR_INVALID_ARG;
  }
  if (slab && p->sgs_model == LES_SGS_DYNAMIC) {
    why = "the dynamic SGS model's volume means are global: not with axial slabs";
    return LES_ERR_UNSUPPORTED;
  }
  if (p->axis && p->sgs_model == LES_SGS_DYNAMIC) {
    why = "the dynamic SGS model is not defined on a grid with an axis (its test filter would "
          "carry the axis nodes' scaled data into ring 1)";
    return LES_ERR_UNSUPPORTED;
  }
  return LES_OK;
}

void layout(les_ctx* c) {
  const size_t N = (size_t)c->g.N;
  const bool mixed = c->p.precision != LES_PREC_FP64;
  const bool m64 = c->p.precision != LES_PREC_MIXED_COMPACT;  // FP64 metrics kept
  const size_t rs = mixed ? sizeof(float) : sizeof(double);
  size_t o = 0;
  c->off_m64 = o; o = align256(o + (m64 ? 10 * N * sizeof(double) : 0));
  c->off_m32 = o; o = align256(o + (mixed ? 10 * N * sizeof(float) : 0));
  c->dyn_ws = c->p.sgs_model == LES_SGS_DYNAMIC;
  c->off_mk = o; o = align256(o + (c->dyn_ws ? 3 : 2) * N * rs);
  c->off_sa = o; o = align256(o + 5 * N * rs);
  c->off_sb = o; o = align256(o + 5 * N * rs);
  c->off_hi = o; o = align256(o + (mixed ? 5 * N * sizeof(float) : 0));
  c->off_lo = o; o = align256(o + (mixed ? 5 * N * sizeof(float) : 0));
  // node fields: FP64 form; FP32 for the mixed forms' dynamic procedure
  c->off_node = o; o = align256(o + (mixed ? (c->dyn_ws ? 8 * N * sizeof(float) : 0) : 8 * N * sizeof(double)));
  c->off_flux = o; o = align256(o + (mixed ? 0 : 15 * N * sizeof(double)));
  c->off_nu = o; o = align256(o + (mixed ? 0 : 3 * N * sizeof(double)));
  c->off_gn = o; o = align256(o + (mixed ? 0 : 4 * N * sizeof(double)));
  c->off_rth = o; o = align256(o + 2 * (size_t)c->g.n[1] * c->g.n[2] * sizeof(double));
  c->off_sc = o; o = align256(o + sizeof(DevScalars));
  c->off_part = o; o = align256(o + 8 * (size_t)lesjet::kMaxPartials * sizeof(double));
  c->off_dyn = o; o = align256(o + (c->dyn_ws ? 50 * N * rs : 0));
  c->off_dtl = o; o = align256(o + (c->p.dt_mode == LES_DT_LOCAL ? N * rs : 0));
  c->local_dt = c->p.dt_mode == LES_DT_LOCAL;
  c->total = o;
}

template <typename T>
T* at(les_ctx* c, size_t off) {
  return reinterpret_cast<T*>(c->ws + off);
}

int ready(les_ctx* c) {
  if (!c) return LES_ERR_INVALID_ARG;
  if (!c->grid_set || !c->ws) return fail(c, LES_ERR_STATE, "les_set_grid has not been called");
  return LES_OK;
}

bool is_mixed(const les_ctx* c) { return c->p.precision != LES_PREC_FP64; }
bool jet_bc(const les_ctx* c) { return c->p.bc == LES_BC_JET || c->p.bc == LES_BC_JET_CHAR; }
// The compact mixed form keeps no FP64 copy of the metrics: its boundary
// conditions and totals read the FP32 metrics.
bool has_m64(const les_ctx* c) { return c->p.precision != LES_PREC_MIXED_COMPACT; }

// ---- FP64 form: node, viscosity, per-direction flux and update passes
lesjet::StageIO64 io64(les_ctx* c, const double* Qin) {
  lesjet::StageIO64 io;
  io.Qin = Qin;
  io.M = at<double>(c, c->off_m64);
  io.gn = is_mixed(c) ? nullptr : at<double>(c, c->off_gn);
  io.node = at<double>(c, c->off_node);
  io.mk = at<double>(c, c->off_mk);
  io.flux = at<double>(c, c->off_flux);
  io.partials = at<double>(c, c->off_part);
  io.sc = at<DevScalars>(c, c->off_sc);
  io.dtl = c->p.dt_mode == LES_DT_LOCAL ? at<double>(c, c->off_dtl) : nullptr;
  io.dyn = c->dyn_ws ? at<double>(c, c->off_dyn) : nullptr;
  io.nu = at<double>(c, c->off_nu);
  return io;
}

void residual64(les_ctx* c, const lesjet::StageIO64& io, bool with_mu, bool with_dt,
                int advance, const lesjet::Launch& L) {
  {
    ProfScope ps(c, PK_NODE, L.s);
    lesjet::launch_node64(c->g, c->p, io, with_dt, L);
  }
  if (with_dt) {
    ProfScope ps(c, PK_DT, L.s);
    lesjet::launch_dt_finalize(c->p, io.partials, io.sc, advance, L);
  }
  if (with_mu) {
    ProfScope ps(c, PK_MU, L.s);
    lesjet::launch_mu64(c->g, c->p, io, L);
  }
  ProfScope ps(c, PK_FLUX, L.s);
  lesjet::launch_sensor64(c->g, io, L);
  for (int d = 0; d < 3; ++d) lesjet::launch_flux64(c->g, c->p, io, d, L);
}

// ---- mixed form: float pair (hi, lo) state in the workspace
void split_state(les_ctx* c, const double* Q, const lesjet::Launch& L) {
  ProfScope ps(c, PK_CONVERT, L.s);
  lesjet::launch_split(5 * c->g.N, Q, at<float>(c, c->off_hi), at<float>(c, c->off_lo), L);
}
void join_state(les_ctx* c, double* Q, const lesjet::Launch& L) {
  ProfScope ps(c, PK_CONVERT, L.s);
  lesjet::launch_join(5 * c->g.N, at<float>(c, c->off_hi), at<float>(c, c->off_lo), Q, L);
}

// mu_eff/kappa_eff of the float state (frozen for the step) and the block
// minima of the CFL step; sc == nullptr leaves the status word alone.
// finalize >= 0: the prestep kernel also sets dt (advance = finalize).
void prestep32(les_ctx* c, const float* Qs, DevScalars* sc, const lesjet::Launch& L,
               int finalize = -1) {
  const double* dyn = nullptr;
  if (c->dyn_ws) {
    // the dynamic procedure on the float state: coefficients into dyn[6..8]
    ProfScope ps(c, PK_MU, L.s);
    DevScalars* scd = at<DevScalars>(c, c->off_sc);
    lesjet::launch_dynamic32(c->g, c->p, Qs, at<float>(c, c->off_m32), at<float>(c, c->off_node),
                             at<float>(c, c->off_dyn), at<double>(c, c->off_part), scd, L);
    dyn = reinterpret_cast<const double*>(reinterpret_cast<const char*>(scd) +
                                          offsetof(DevScalars, dyn));
  }
  ProfScope ps(c, PK_PRESTEP, L.s);
  // the per-node steps are those of Q^n: written only by the step's first
  // prestep (the one that also takes the CFL minima, sc != nullptr)
  float* dtl = (sc && c->p.dt_mode == LES_DT_LOCAL) ? at<float>(c, c->off_dtl) : nullptr;
  lesjet::launch_prestep(c->g, c->p, Qs, at<float>(c, c->off_m32), at<float>(c, c->off_mk),
                         at<double>(c, c->off_part), sc, dtl, dyn, L, finalize);
}

lesjet::FusedIO fused_io(les_ctx* c, const void* Qin, void* out) {
  lesjet::FusedIO io;
  io.Qin = Qin;
  io.Q0 = at<float>(c, c->off_hi);
  io.Q0lo = at<float>(c, c->off_lo);
  io.M = at<float>(c, c->off_m32);
  io.mk = at<float>(c, c->off_mk);
  io.sc = at<DevScalars>(c, c->off_sc);
  io.dtl = c->p.dt_mode == LES_DT_LOCAL ? at<float>(c, c->off_dtl) : nullptr;
  io.out = out;
  return io;
}

// One time step (Table tab:JAZzY): viscosity + CFL step from Q^n, five
// stages Q^(l) = Q^(0) - alpha_l dt J RHS(Q^(l-1)), boundary conditions at
// t^{n+1}.  In the mixed form the state must already be split into (hi, lo).
void rk_step(les_ctx* c, double* Q, cudaStream_t s) {
  lesjet::Launch L{s, &c->launches};
  DevScalars* sc = at<DevScalars>(c, c->off_sc);
  if (!is_mixed(c)) {
    double* SA = at<double>(c, c->off_sa);
    double* SB = at<double>(c, c->off_sb);
    for (int l = 1; l <= 5; ++l) {
      const double* in = (l == 1) ? Q : ((l % 2 == 0) ? SA : SB);
      double* out = (l == 5) ? Q : ((l % 2 == 1) ? SA : SB);
      lesjet::StageIO64 io = io64(c, in);
      residual64(c, io, l == 1 || !c->p.freeze_visc, l == 1, 1, L);
      ProfScope ps(c, PK_UPDATE, s);
      lesjet::launch_update64(c->g, io, Q, kAlpha[l - 1], l == 5 ? 2 : 1, out, L);
    }
    if (jet_bc(c)) {
      ProfScope ps(c, PK_BC, s);
      lesjet::launch_bc_jet(c->g, c->p, Q, at<double>(c, c->off_m64), at<double>(c, c->off_rth),
                            sc, 0, 0.0, L);
    }
    return;
  }
  float* hi = at<float>(c, c->off_hi);
  float* SA = at<float>(c, c->off_sa);
  float* SB = at<float>(c, c->off_sb);
  prestep32(c, hi, sc, L, 1);  // its last block takes the step and advances t
  for (int l = 1; l <= 5; ++l) {
    const float* in = (l == 1) ? hi : ((l % 2 == 0) ? SA : SB);
    float* out = (l == 5) ? nullptr : ((l % 2 == 1) ? SA : SB);
    if (l > 1 && !c->p.freeze_visc) prestep32(c, in, nullptr, L);  // Reading A17, unfrozen
    ProfScope ps(c, PK_STAGE, s);
    lesjet::launch_stage_fused(l == 5 ? 2 : 1, c->g, c->p, fused_io(c, in, out), kAlpha[l - 1], L);
  }
  if (jet_bc(c)) {
    ProfScope ps(c, PK_BC, s);
    if (has_m64(c))
      lesjet::launch_bc_jet_hl(c->g, c->p, hi, at<float>(c, c->off_lo), at<double>(c, c->off_m64),
                               at<double>(c, c->off_rth), sc, L);
    else
      lesjet::launch_bc_jet_hl(c->g, c->p, hi, at<float>(c, c->off_lo), at<float>(c, c->off_m32),
                               at<double>(c, c->off_rth), sc, L);
  }
}

void totals(les_ctx* c, const double* Q, const lesjet::Launch& L) {
  if (has_m64(c))
    lesjet::launch_totals(c->g, Q, at<double>(c, c->off_m64), at<double>(c, c->off_part),
                          at<DevScalars>(c, c->off_sc), L);
  else
    lesjet::launch_totals(c->g, Q, at<float>(c, c->off_m32), at<double>(c, c->off_part),
                          at<DevScalars>(c, c->off_sc), L);
}

int read_scalars(les_ctx* c, DevScalars* h, cudaStream_t s) {
  cudaMemcpyAsync(h, c->ws + c->off_sc, sizeof(DevScalars), cudaMemcpyDeviceToHost, s);
  if (cudaStreamSynchronize(s) != cudaSuccess) return cuda_check(c, "stream synchronize");
  return cuda_check(c, "read scalars");
}

}  // namespace

extern "C" {

int les_create(const les_params* p, int ni, int nj, int nk, les_ctx** out) {
  if (!p || !out) return LES_ERR_INVALID_ARG;
  *out = nullptr;
  std::string why;
  int rc = validate_params(p, why);
  if (rc != LES_OK) return rc;
  if (ni < 5 || nj < 5 || nk < 5) return LES_ERR_SHAPE;
  // a slab owns at least one plane besides its ghost planes
  if (ni <= p->slab_ghost[0] + p->slab_ghost[1]) return LES_ERR_SHAPE;
  // the axis viscosity rule averages a ring in shared memory
  if (p->axis && nk > 4096) return LES_ERR_SHAPE;
  const long long N = (long long)ni * nj * nk;
  if (N >= (1LL << 40)) return LES_ERR_SHAPE;
  // the mixed form indexes each field with 32 bits
  if (p->precision != LES_PREC_FP64 && N >= (1LL << 31)) return LES_ERR_SHAPE;
  les_ctx* c = new (std::nothrow) les_ctx();
  if (!c) return LES_ERR_INVALID_ARG;
  c->p = *p;
  c->g.n[0] = ni;
  c->g.n[1] = nj;
  c->g.n[2] = nk;
  for (int d = 0; d < 3; ++d) c->g.per[d] = p->periodic[d] ? 1 : 0;
  c->g.N = N;
  c->g.stride[0] = (long long)nj * nk;
  c->g.stride[1] = nk;
  c->g.stride[2] = 1;
  c->g.glo = p->slab_ghost[0];
  c->g.ghi = p->slab_ghost[1];
  c->ws = nullptr;
  c->grid_set = false;
  c->launches = 0;
  c->prof_on = false;
  for (int k = 0; k < PK_COUNT; ++k) {
    c->prof_ms[k] = 0.0;
    c->prof_n[k] = 0;
  }
  layout(c);
  *out = c;
  return LES_OK;
}

int les_destroy(les_ctx* c) {
  if (!c) return LES_OK;
  for (auto& r : c->prof_pending) {
    cudaEventDestroy(r.a);
    cudaEventDestroy(r.b);
  }
  for (auto e : c->prof_pool) cudaEventDestroy(e);
  drop_step_graph(c);
  if (c->cap_stream) cudaStreamDestroy(c->cap_stream);
  delete c;
  return LES_OK;
}

const char* les_last_error(const les_ctx* c) { return c ? c->err.c_str() : "null context"; }

int les_set_params(les_ctx* c, const les_params* p) {
  if (!c || !p) return LES_ERR_INVALID_ARG;
  std::string why;
  int rc = validate_params(p, why);
  if (rc != LES_OK) return fail(c, rc, why.c_str());
  if (p->precision != c->p.precision) return fail(c, LES_ERR_INVALID_ARG, "precision is fixed at creation");
  if (p->dt_mode == LES_DT_LOCAL && !c->local_dt)
    return fail(c, LES_ERR_INVALID_ARG, "local time stepping must be chosen at creation");
  if (p->sgs_model == LES_SGS_DYNAMIC && !c->dyn_ws)
    return fail(c, LES_ERR_INVALID_ARG, "the dynamic SGS model must be chosen at creation");
  for (int d = 0; d < 3; ++d)
    if ((p->periodic[d] ? 1 : 0) != c->g.per[d])
      return fail(c, LES_ERR_INVALID_ARG, "periodicity is fixed at creation");
  if (p->slab_ghost[0] != c->g.glo || p->slab_ghost[1] != c->g.ghi)
    return fail(c, LES_ERR_INVALID_ARG, "the slab's ghost planes are fixed at creation");
  c->p = *p;
  drop_step_graph(c);
  return LES_OK;
}

size_t les_workspace_bytes(const les_ctx* c) { return c ? c->total : 0; }

int les_set_grid(les_ctx* c, const double* xyz, const double shift[9], void* workspace,
                 les_stream_t stream) {
  if (!c || !xyz || !workspace) return fail(c, LES_ERR_INVALID_ARG, "null pointer");
  if (!aligned16(xyz) || !aligned16(workspace))
    return fail(c, LES_ERR_ALIGN, "device pointers must be 16-byte aligned");
  cudaStream_t s = (cudaStream_t)stream;
  lesjet::Launch L{s, &c->launches};
  drop_step_graph(c);
  c->ws = (char*)workspace;
  if (has_m64(c)) {
    double* M64 = at<double>(c, c->off_m64);
    lesjet::launch_metrics(c->g, xyz, shift, c->p.metric_form, M64, L);
    if (is_mixed(c)) lesjet::launch_to_float(10 * c->g.N, M64, at<float>(c, c->off_m32), L);
    else lesjet::launch_grad_norms(c->g, M64, at<double>(c, c->off_gn), L);
  } else {
    lesjet::launch_metrics(c->g, xyz, shift, c->p.metric_form, at<float>(c, c->off_m32), L);
  }
  lesjet::launch_inflow_geometry(c->g, xyz, at<double>(c, c->off_rth), L);
  lesjet::launch_set_time(at<DevScalars>(c, c->off_sc), 0.0, L);
  int rc = cuda_check(c, "les_set_grid");
  if (rc == LES_OK) c->grid_set = true;
  return rc;
}

const double* les_metrics(const les_ctx* c) {
  if (!c || !c->ws || !has_m64(c)) return nullptr;
  return reinterpret_cast<const double*>(c->ws + c->off_m64);
}

int les_init_jet(les_ctx* c, const double* xyz, uint64_t seed, double noise, double* Q,
                 les_stream_t stream) {
  if (!c || !xyz || !Q) return fail(c, LES_ERR_INVALID_ARG, "null pointer");
  if (!aligned16(xyz) || !aligned16(Q)) return fail(c, LES_ERR_ALIGN, "unaligned device pointer");
  lesjet::Launch L{(cudaStream_t)stream, &c->launches};
  lesjet::launch_init_jet(c->g, xyz, seed, noise, c->p, Q, L);
  return cuda_check(c, "les_init_jet");
}

int les_mu_eff(les_ctx* c, const double* Q, double* MK, les_stream_t stream) {
  int rc = ready(c);
  if (rc != LES_OK) return rc;
  if (!Q || !MK) return fail(c, LES_ERR_INVALID_ARG, "null pointer");
  if (!aligned16(Q) || !aligned16(MK)) return fail(c, LES_ERR_ALIGN, "unaligned device pointer");
  lesjet::Launch L{(cudaStream_t)stream, &c->launches};
  if (is_mixed(c)) {
    split_state(c, Q, L);
    prestep32(c, at<float>(c, c->off_hi), nullptr, L);
  } else {
    lesjet::StageIO64 io = io64(c, Q);
    lesjet::launch_node64(c->g, c->p, io, false, L);
    lesjet::launch_mu64(c->g, c->p, io, L);
  }
  lesjet::launch_mk_to_double(c->p.precision, c->g, c->ws + c->off_mk,
                              c->p.sgs_model == LES_SGS_DYNAMIC ? 3 : 2, MK, L);
  return cuda_check(c, "les_mu_eff");
}

int les_dynamic_coefficients(les_ctx* c, const double* Q, double out[9], les_stream_t stream) {
  int rc = ready(c);
  if (rc != LES_OK) return rc;
  if (!Q || !out) return fail(c, LES_ERR_INVALID_ARG, "null pointer");
  if (!aligned16(Q)) return fail(c, LES_ERR_ALIGN, "unaligned device pointer");
  if (!c->dyn_ws)
    return fail(c, LES_ERR_UNSUPPORTED, "the context was not created with LES_SGS_DYNAMIC");
  cudaStream_t s = (cudaStream_t)stream;
  lesjet::Launch L{s, &c->launches};
  DevScalars* sc = at<DevScalars>(c, c->off_sc);
  if (is_mixed(c)) {
    split_state(c, Q, L);
    lesjet::launch_dynamic32(c->g, c->p, at<float>(c, c->off_hi), at<float>(c, c->off_m32),
                             at<float>(c, c->off_node), at<float>(c, c->off_dyn),
                             at<double>(c, c->off_part), sc, L);
  } else {
    lesjet::StageIO64 io = io64(c, Q);
    lesjet::launch_node64(c->g, c->p, io, false, L);
    lesjet::launch_dynamic64(c->g, c->p, io, io.dyn, L);
  }
  cudaMemcpyAsync(out, sc->dyn, 9 * sizeof(double), cudaMemcpyDeviceToHost, s);
  if (cudaStreamSynchronize(s) != cudaSuccess) return cuda_check(c, "les_dynamic_coefficients");
  return cuda_check(c, "les_dynamic_coefficients");
}

int les_rhs(les_ctx* c, const double* Q, double* R, les_stream_t stream) {
  int rc = ready(c);
  if (rc != LES_OK) return rc;
  if (!Q || !R) return fail(c, LES_ERR_INVALID_ARG, "null pointer");
  if (!aligned16(Q) || !aligned16(R)) return fail(c, LES_ERR_ALIGN, "unaligned device pointer");
  if (Q == R) return fail(c, LES_ERR_INVALID_ARG, "Q and R must not alias");
  lesjet::Launch L{(cudaStream_t)stream, &c->launches};
  if (is_mixed(c)) {
    split_state(c, Q, L);
    float* hi = at<float>(c, c->off_hi);
    prestep32(c, hi, nullptr, L);
    lesjet::launch_stage_fused(0, c->g, c->p, fused_io(c, hi, R), 0.0, L);
  } else {
    lesjet::StageIO64 io = io64(c, Q);
    residual64(c, io, true, false, 0, L);
    lesjet::launch_update64(c->g, io, Q, 0.0, 0, R, L);
  }
  return cuda_check(c, "les_rhs");
}

int les_time_step(les_ctx* c, const double* Q, double* dt_out, les_stream_t stream) {
  int rc = ready(c);
  if (rc != LES_OK) return rc;
  if (!Q || !dt_out) return fail(c, LES_ERR_INVALID_ARG, "null pointer");
  if (!aligned16(Q)) return fail(c, LES_ERR_ALIGN, "unaligned device pointer");
  cudaStream_t s = (cudaStream_t)stream;
  lesjet::Launch L{s, &c->launches};
  DevScalars* sc = at<DevScalars>(c, c->off_sc);
  if (is_mixed(c)) {
    split_state(c, Q, L);
    prestep32(c, at<float>(c, c->off_hi), sc, L);
  } else {
    lesjet::launch_node64(c->g, c->p, io64(c, Q), true, L);
  }
  lesjet::launch_dt_finalize(c->p, at<double>(c, c->off_part), sc, 0, L);
  if ((rc = cuda_check(c, "les_time_step")) != LES_OK) return rc;
  DevScalars h;
  if ((rc = read_scalars(c, &h, s)) != LES_OK) return rc;
  *dt_out = h.dt;
  if (h.status != 0) return fail(c, LES_ERR_NONFINITE, "non-finite or non-positive state");
  return LES_OK;
}

int les_apply_bc(les_ctx* c, double* Q, double t, les_stream_t stream) {
  int rc = ready(c);
  if (rc != LES_OK) return rc;
  if (!Q) return fail(c, LES_ERR_INVALID_ARG, "null pointer");
  if (!aligned16(Q)) return fail(c, LES_ERR_ALIGN, "unaligned device pointer");
  if (!jet_bc(c)) return fail(c, LES_ERR_STATE, "bc is not LES_BC_JET or LES_BC_JET_CHAR");
  lesjet::Launch L{(cudaStream_t)stream, &c->launches};
  if (has_m64(c))
    lesjet::launch_bc_jet(c->g, c->p, Q, at<double>(c, c->off_m64), at<double>(c, c->off_rth),
                          at<DevScalars>(c, c->off_sc), 1, t, L);
  else
    lesjet::launch_bc_jet(c->g, c->p, Q, at<float>(c, c->off_m32), at<double>(c, c->off_rth),
                          at<DevScalars>(c, c->off_sc), 1, t, L);
  return cuda_check(c, "les_apply_bc");
}

int les_set_time(les_ctx* c, double t, les_stream_t stream) {
  int rc = ready(c);
  if (rc != LES_OK) return rc;
  lesjet::Launch L{(cudaStream_t)stream, &c->launches};
  lesjet::launch_set_time(at<DevScalars>(c, c->off_sc), t, L);
  return cuda_check(c, "les_set_time");
}

// ------------------------------------------------ the mixed step as a graph
// One FP32-mixed RK step reads and writes only the workspace (the caller's
// state enters through the split and leaves through the join) and takes dt
// and t from the device scalars, so its launches are the same every step.
// The step is captured once on the context's own stream, and the graph is
// replayed for every later step: one graph launch in place of eight or more
// kernel launches, with shorter gaps between the kernels.  A new parameter
// set, grid (workspace) or profiler state drops the graph; a capture that
// fails leaves the context on plain launches.
static void capture_step_graph(les_ctx* c) {
  if (!c->cap_stream &&
      cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking) != cudaSuccess) {
    cudaGetLastError();
    c->graph_failed = true;
    return;
  }
  const unsigned long long before = c->launches;
  cudaGraph_t graph = nullptr;
  bool ok = cudaStreamBeginCapture(c->cap_stream, cudaStreamCaptureModeThreadLocal) == cudaSuccess;
  if (ok) {
    rk_step(c, nullptr, c->cap_stream);  // the mixed step does not touch Q
    ok = cudaStreamEndCapture(c->cap_stream, &graph) == cudaSuccess && graph != nullptr;
  }
  c->step_launches = c->launches - before;
  c->launches = before;  // captured, not run
  if (ok) ok = cudaGraphInstantiate(&c->step_exec, graph, 0) == cudaSuccess;
  if (graph) cudaGraphDestroy(graph);
  if (!ok) {
    c->step_exec = nullptr;
    c->graph_failed = true;
    cudaGetLastError();
  }
}

// n FP32-mixed steps on stream s.  A context's first step runs as plain
// launches (its first launches set the fused kernel's shared-memory
// attribute and choose the axial chunks), then the step is captured and
// every later step replays the graph; with the event profiler on, every
// step runs as plain launches (the profiler records events around them).
static void mixed_steps(les_ctx* c, int n, cudaStream_t s) {
  int i = 0;
  if (!c->prof_on && !c->step_exec && !c->graph_failed && n > 0) {
    rk_step(c, nullptr, s);
    ++i;
    capture_step_graph(c);
  }
  if (!c->prof_on && c->step_exec) {
    for (; i < n; ++i) {
      if (cudaGraphLaunch(c->step_exec, s) != cudaSuccess) break;
      c->launches += c->step_launches;
    }
  }
  for (; i < n; ++i) rk_step(c, nullptr, s);
}

int les_rk_step(les_ctx* c, double* Q, les_stream_t stream) {
  int rc = ready(c);
  if (rc != LES_OK) return rc;
  if (!Q) return fail(c, LES_ERR_INVALID_ARG, "null pointer");
  if (!aligned16(Q)) return fail(c, LES_ERR_ALIGN, "unaligned device pointer");
  cudaStream_t s = (cudaStream_t)stream;
  lesjet::Launch L{s, &c->launches};
  if (is_mixed(c)) split_state(c, Q, L);
  rk_step(c, Q, s);
  if (is_mixed(c)) join_state(c, Q, L);
  return cuda_check(c, "les_rk_step");
}

// Totals and diagnostics after a run; reads the device scalars (synchronises).
int finish_run(les_ctx* c, int n, les_diag* diag, cudaStream_t s) {
  int rc;
  if ((rc = cuda_check(c, "les_run_n_steps")) != LES_OK) return rc;
  DevScalars h;
  if ((rc = read_scalars(c, &h, s)) != LES_OK) return rc;
  if (diag) {
    diag->t = h.t;
    diag->dt = h.dt;
    for (int q = 0; q < 5; ++q) diag->totals[q] = h.totals[q];
    diag->status = h.status ? LES_ERR_NONFINITE : LES_OK;
    diag->steps = n;
  }
  if (h.status != 0) return fail(c, LES_ERR_NONFINITE, "non-finite or non-positive state");
  return LES_OK;
}

// ---- one step in phases (axial slabs: the driver exchanges ghost planes and
// takes the global step between them)
int les_step_begin(les_ctx* c, double* Q, double* dt_local, les_stream_t stream) {
  int rc = ready(c);
  if (rc != LES_OK) return rc;
  if (!Q || !dt_local) return fail(c, LES_ERR_INVALID_ARG, "null pointer");
  if (!aligned16(Q)) return fail(c, LES_ERR_ALIGN, "unaligned device pointer");
  cudaStream_t s = (cudaStream_t)stream;
  lesjet::Launch L{s, &c->launches};
  DevScalars* sc = at<DevScalars>(c, c->off_sc);
  if (is_mixed(c)) {
    prestep32(c, at<float>(c, c->off_hi), sc, L);
    ProfScope ps(c, PK_DT, s);
    lesjet::launch_dt_finalize(c->p, at<double>(c, c->off_part), sc, 0, L);
  } else {
    // node quantities (with the CFL minima), dt, viscosity of Q^n; stage 1
    // reuses them
    lesjet::StageIO64 io = io64(c, Q);
    {
      ProfScope ps(c, PK_NODE, s);
      lesjet::launch_node64(c->g, c->p, io, true, L);
    }
    {
      ProfScope ps(c, PK_DT, s);
      lesjet::launch_dt_finalize(c->p, io.partials, io.sc, 0, L);
    }
    ProfScope ps(c, PK_MU, s);
    lesjet::launch_mu64(c->g, c->p, io, L);
  }
  if ((rc = cuda_check(c, "les_step_begin")) != LES_OK) return rc;
  DevScalars h;
  if ((rc = read_scalars(c, &h, s)) != LES_OK) return rc;
  *dt_local = h.dt;
  if (h.status != 0) return fail(c, LES_ERR_NONFINITE, "non-finite or non-positive state");
  return LES_OK;
}

int les_step_set_dt(les_ctx* c, double dt, les_stream_t stream) {
  int rc = ready(c);
  if (rc != LES_OK) return rc;
  if (!(dt > 0.0) || !(dt < 1.0e300)) return fail(c, LES_ERR_INVALID_ARG, "dt must be positive and finite");
  lesjet::Launch L{(cudaStream_t)stream, &c->launches};
  lesjet::launch_set_dt(at<DevScalars>(c, c->off_sc), dt, L);
  return cuda_check(c, "les_step_set_dt");
}

int les_step_stage(les_ctx* c, int l, double* Q, les_stream_t stream) {
  int rc = ready(c);
  if (rc != LES_OK) return rc;
  if (!Q || l < 1 || l > 5) return fail(c, LES_ERR_INVALID_ARG, "null pointer or stage outside 1..5");
  if (!aligned16(Q)) return fail(c, LES_ERR_ALIGN, "unaligned device pointer");
  cudaStream_t s = (cudaStream_t)stream;
  lesjet::Launch L{s, &c->launches};
  if (!is_mixed(c)) {
    double* SA = at<double>(c, c->off_sa);
    double* SB = at<double>(c, c->off_sb);
    const double* in = (l == 1) ? Q : ((l % 2 == 0) ? SA : SB);
    double* out = (l == 5) ? Q : ((l % 2 == 1) ? SA : SB);
    lesjet::StageIO64 io = io64(c, in);
    if (l == 1) {
      // node quantities and viscosity of Q^n come from les_step_begin
      ProfScope ps(c, PK_FLUX, s);
      lesjet::launch_sensor64(c->g, io, L);
      for (int d = 0; d < 3; ++d) lesjet::launch_flux64(c->g, c->p, io, d, L);
    } else {
      residual64(c, io, !c->p.freeze_visc, false, 0, L);
    }
    ProfScope ps(c, PK_UPDATE, s);
    lesjet::launch_update64(c->g, io, Q, kAlpha[l - 1], l == 5 ? 2 : 1, out, L);
  } else {
    float* hi = at<float>(c, c->off_hi);
    float* SA = at<float>(c, c->off_sa);
    float* SB = at<float>(c, c->off_sb);
    const float* in = (l == 1) ? hi : ((l % 2 == 0) ? SA : SB);
    float* out = (l == 5) ? nullptr : ((l % 2 == 1) ? SA : SB);
    if (l > 1 && !c->p.freeze_visc) prestep32(c, in, nullptr, L);  // Reading A17, unfrozen
    ProfScope ps(c, PK_STAGE, s);
    lesjet::launch_stage_fused(l == 5 ? 2 : 1, c->g, c->p, fused_io(c, in, out), kAlpha[l - 1], L);
  }
  return cuda_check(c, "les_step_stage");
}

int les_step_end(les_ctx* c, double* Q, les_stream_t stream) {
  int rc = ready(c);
  if (rc != LES_OK) return rc;
  if (!Q) return fail(c, LES_ERR_INVALID_ARG, "null pointer");
  cudaStream_t s = (cudaStream_t)stream;
  lesjet::Launch L{s, &c->launches};
  if (jet_bc(c)) {
    ProfScope ps(c, PK_BC, s);
    DevScalars* sc = at<DevScalars>(c, c->off_sc);
    if (!is_mixed(c))
      lesjet::launch_bc_jet(c->g, c->p, Q, at<double>(c, c->off_m64), at<double>(c, c->off_rth), sc,
                            0, 0.0, L);
    else if (has_m64(c))
      lesjet::launch_bc_jet_hl(c->g, c->p, at<float>(c, c->off_hi), at<float>(c, c->off_lo),
                               at<double>(c, c->off_m64), at<double>(c, c->off_rth), sc, L);
    else
      lesjet::launch_bc_jet_hl(c->g, c->p, at<float>(c, c->off_hi), at<float>(c, c->off_lo),
                               at<float>(c, c->off_m32), at<double>(c, c->off_rth), sc, L);
  }
  return cuda_check(c, "les_step_end");
}

int les_state_load(les_ctx* c, const double* Q, les_stream_t stream) {
  int rc = ready(c);
  if (rc != LES_OK) return rc;
  if (!Q) return fail(c, LES_ERR_INVALID_ARG, "null pointer");
  if (!aligned16(Q)) return fail(c, LES_ERR_ALIGN, "unaligned device pointer");
  lesjet::Launch L{(cudaStream_t)stream, &c->launches};
  if (is_mixed(c)) split_state(c, Q, L);
  return cuda_check(c, "les_state_load");
}

int les_state_store(les_ctx* c, double* Q, les_stream_t stream) {
  int rc = ready(c);
  if (rc != LES_OK) return rc;
  if (!Q) return fail(c, LES_ERR_INVALID_ARG, "null pointer");
  if (!aligned16(Q)) return fail(c, LES_ERR_ALIGN, "unaligned device pointer");
  lesjet::Launch L{(cudaStream_t)stream, &c->launches};
  if (is_mixed(c)) join_state(c, Q, L);
  return cuda_check(c, "les_state_store");
}

int les_state_buffer(les_ctx* c, int l, void** a, void** b, int* elem_bytes) {
  int rc = ready(c);
  if (rc != LES_OK) return rc;
  if (!a || !b || !elem_bytes || l < 0 || l > 5)
    return fail(c, LES_ERR_INVALID_ARG, "null pointer or stage outside 0..5");
  *b = nullptr;
  if (l >= 1 && l <= 4) {
    *a = c->ws + ((l % 2 == 1) ? c->off_sa : c->off_sb);
    *elem_bytes = is_mixed(c) ? 4 : 8;
  } else if (!is_mixed(c)) {
    *a = nullptr;  // the caller's Q
    *elem_bytes = 8;
  } else {
    *a = c->ws + c->off_hi;
    *b = c->ws + c->off_lo;
    *elem_bytes = 4;
  }
  return LES_OK;
}

int les_halo_copy(les_ctx* dst, double* Qdst, les_ctx* src, const double* Qsrc, int l, int side,
                  les_stream_t stream) {
  int rc = ready(dst);
  if (rc != LES_OK) return rc;
  if ((rc = ready(src)) != LES_OK) return rc;
  if (side != 0 && side != 1) return fail(dst, LES_ERR_INVALID_ARG, "side must be 0 or 1");
  if (dst->g.n[1] != src->g.n[1] || dst->g.n[2] != src->g.n[2] || is_mixed(dst) != is_mixed(src))
    return fail(dst, LES_ERR_INVALID_ARG, "slabs differ in nj, nk or precision");
  // side 0: dst lies above src (dst's low ghosts from src's top own planes)
  if (side == 0 ? (dst->g.glo != 2 || src->g.ghi != 2) : (dst->g.ghi != 2 || src->g.glo != 2))
    return fail(dst, LES_ERR_INVALID_ARG, "the slabs have no ghost planes at this cut");
  void *da, *db, *sa, *sb;
  int de, se;
  if ((rc = les_state_buffer(dst, l, &da, &db, &de)) != LES_OK) return rc;
  if ((rc = les_state_buffer(src, l, &sa, &sb, &se)) != LES_OK) return fail(dst, rc, "source buffers");
  if (!da) da = Qdst;
  if (!sa) sa = const_cast<double*>(Qsrc);
  if (!da || !sa) return fail(dst, LES_ERR_INVALID_ARG, "null state pointer");
  const size_t e = (size_t)de;
  const size_t plane = (size_t)dst->g.n[1] * dst->g.n[2] * e;
  const size_t dp = (size_t)dst->g.N * e, sp = (size_t)src->g.N * e;
  const size_t doff = (side == 0) ? 0 : (size_t)(dst->g.n[0] - 2) * plane;
  const size_t soff = (side == 0) ? (size_t)(src->g.n[0] - 4) * plane : 2 * plane;
  cudaStream_t s = (cudaStream_t)stream;
  void* dsts[2] = {da, db};
  void* srcs[2] = {sa, sb};
  for (int k = 0; k < 2; ++k) {
    if (!dsts[k]) continue;
    if (cudaMemcpy2DAsync((char*)dsts[k] + doff, dp, (const char*)srcs[k] + soff, sp, 2 * plane, 5,
                          cudaMemcpyDefault, s) != cudaSuccess)
      return cuda_check(dst, "les_halo_copy");
  }
  return LES_OK;
}

int les_run_n_steps(les_ctx* c, int n, double* Q, les_diag* diag, les_stream_t stream) {
  int rc = ready(c);
  if (rc != LES_OK) return rc;
  if (!Q || n < 0) return fail(c, LES_ERR_INVALID_ARG, "null pointer or negative n");
  if (!aligned16(Q)) return fail(c, LES_ERR_ALIGN, "unaligned device pointer");
  cudaStream_t s = (cudaStream_t)stream;
  lesjet::Launch L{s, &c->launches};
  if (is_mixed(c)) {
    split_state(c, Q, L);
    mixed_steps(c, n, s);
    join_state(c, Q, L);
  } else {
    for (int i = 0; i < n; ++i) rk_step(c, Q, s);
  }
  {
    ProfScope ps(c, PK_TOTALS, s);
    totals(c, Q, L);
  }
  return finish_run(c, n, diag, s);
}

// True when the pinned host range [host, host + bytes) lies inside one
// allocation or registration known to the driver (cuPointerGetAttribute's
// range start and size, fetched through the runtime); false when it does not
// or the driver cannot tell.
bool host_range_covers(const void* host, size_t bytes) {
  typedef CUresult (*PfnPointerGetAttribute)(void*, CUpointer_attribute, CUdeviceptr);
  static PfnPointerGetAttribute get_attr = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* f = nullptr;
    cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
    if (cudaGetDriverEntryPointByVersion("cuPointerGetAttribute", &f, 12000, cudaEnableDefault,
                                         &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      get_attr = (PfnPointerGetAttribute)f;
  });
  if (!get_attr) return false;
  CUdeviceptr start = 0;
  size_t size = 0;
  const CUdeviceptr p = (CUdeviceptr)(uintptr_t)host;
  if (get_attr(&start, CU_POINTER_ATTRIBUTE_RANGE_START_ADDR, p) != CUDA_SUCCESS ||
      get_attr(&size, CU_POINTER_ATTRIBUTE_RANGE_SIZE, p) != CUDA_SUCCESS)
    return false;
  return start <= p && (unsigned long long)(p - start) + bytes <= (unsigned long long)size;
}

// Device-side address of a host buffer of `bytes` bytes when all of it is
// pinned host memory that the driver maps into this device's address space;
// nullptr otherwise (pageable, partly registered or unknown memory goes
// through the staging copy).
const void* mapped_host(const void* host, size_t bytes) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, host) != cudaSuccess) {
    cudaGetLastError();  // clear the query's error state
    return nullptr;
  }
  if (a.type != cudaMemoryTypeHost || a.devicePointer == nullptr) return nullptr;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || (a.device >= 0 && a.device != dev)) {
    cudaGetLastError();
    return nullptr;
  }
  if (!host_range_covers(host, bytes)) return nullptr;
  return a.devicePointer;
}

int les_run_host(les_ctx* c, int n, double* Q_host, double* Q_dev, les_diag* diag,
                 les_stream_t stream) {
  int rc = ready(c);
  if (rc != LES_OK) return rc;
  if (!Q_host || !Q_dev || n < 0) return fail(c, LES_ERR_INVALID_ARG, "null pointer or negative n");
  if (!aligned16(Q_dev)) return fail(c, LES_ERR_ALIGN, "unaligned device pointer");
  cudaStream_t s = (cudaStream_t)stream;
  const size_t bytes = 5 * (size_t)c->g.N * sizeof(double);
  if (is_mixed(c)) {
    // mapped pinned memory: the split kernel reads the host state and the
    // join kernel writes it back over the host link, with no FP64 staging
    // copy (the float pair state lives in the workspace in between)
    double* Qm = const_cast<double*>(static_cast<const double*>(mapped_host(Q_host, bytes)));
    if (Qm && aligned16(Qm)) {
      lesjet::Launch L{s, &c->launches};
      split_state(c, Qm, L);
      mixed_steps(c, n, s);
      {
        // one pass joins the state into the host buffer and sums the totals:
        // their FP64 arithmetic hides under the write-back over the host link
        ProfScope ps(c, PK_CONVERT, s);
        if (has_m64(c))
          lesjet::launch_join_totals_hl(c->g, at<float>(c, c->off_hi), at<float>(c, c->off_lo),
                                        at<double>(c, c->off_m64), Qm, at<double>(c, c->off_part),
                                        at<DevScalars>(c, c->off_sc), L);
        else
          lesjet::launch_join_totals_hl(c->g, at<float>(c, c->off_hi), at<float>(c, c->off_lo),
                                        at<float>(c, c->off_m32), Qm, at<double>(c, c->off_part),
                                        at<DevScalars>(c, c->off_sc), L);
      }
      return finish_run(c, n, diag, s);
    }
  }
  if (cudaMemcpyAsync(Q_dev, Q_host, bytes, cudaMemcpyHostToDevice, s) != cudaSuccess)
    return cuda_check(c, "les_run_host upload");
  rc = les_run_n_steps(c, n, Q_dev, diag, stream);
  if (rc != LES_OK && rc != LES_ERR_NONFINITE) return rc;
  if (cudaMemcpyAsync(Q_host, Q_dev, bytes, cudaMemcpyDeviceToHost, s) != cudaSuccess)
    return cuda_check(c, "les_run_host download");
  if (cudaStreamSynchronize(s) != cudaSuccess) return cuda_check(c, "les_run_host sync");
  return rc;
}

int les_totals(les_ctx* c, const double* Q, double out[5], les_stream_t stream) {
  int rc = ready(c);
  if (rc != LES_OK) return rc;
  if (!Q || !out) return fail(c, LES_ERR_INVALID_ARG, "null pointer");
  cudaStream_t s = (cudaStream_t)stream;
  lesjet::Launch L{s, &c->launches};
  totals(c, Q, L);
  if ((rc = cuda_check(c, "les_totals")) != LES_OK) return rc;
  DevScalars h;
  if ((rc = read_scalars(c, &h, s)) != LES_OK) return rc;
  for (int q = 0; q < 5; ++q) out[q] = h.totals[q];
  return LES_OK;
}

uint64_t les_launch_count(const les_ctx* c) { return c ? c->launches : 0; }

int les_profile(les_ctx* c, int enable) {
  if (!c) return LES_ERR_INVALID_ARG;
  c->prof_on = enable != 0;
  drop_step_graph(c);
  if (enable) {
    for (int k = 0; k < PK_COUNT; ++k) {
      c->prof_ms[k] = 0.0;
      c->prof_n[k] = 0;
    }
  }
  return LES_OK;
}

int les_profile_read(les_ctx* c, double ms[16], uint64_t counts[16], les_stream_t stream) {
  if (!c || !ms || !counts) return LES_ERR_INVALID_ARG;
  if (cudaStreamSynchronize((cudaStream_t)stream) != cudaSuccess)
    return cuda_check(c, "les_profile_read");
  for (auto& r : c->prof_pending) {
    float t = 0.f;
    if (cudaEventSynchronize(r.b) == cudaSuccess && cudaEventElapsedTime(&t, r.a, r.b) == cudaSuccess) {
      c->prof_ms[r.kind] += t;
      c->prof_n[r.kind] += 1;
    }
    c->prof_pool.push_back(r.a);
    c->prof_pool.push_back(r.b);
  }
  c->prof_pending.clear();
  for (int k = 0; k < 16; ++k) {
    ms[k] = k < PK_COUNT ? c->prof_ms[k] : 0.0;
    counts[k] = k < PK_COUNT ? c->prof_n[k] : 0;
  }
  return cuda_check(c, "les_profile_read");
}

const char* les_profile_name(int kind) {
  return (kind >= 0 && kind < PK_COUNT) ? kProfNames[kind] : "";
}

}  // extern "C"

// ------------------------------------------------------------ adjoint
namespace {

struct AdjLayout {
  size_t acc, node, mk, lamMK, S, lamS, lamR, lamQ0, work, lam, Qnext, E, partials, scal;
  size_t qd, mkd, noded, fluxd, rd, ckpt, segS, segMK, segN, total;
  int nckpt, K;
};

AdjLayout adj_layout(const les_ctx* c, int nsteps, int K) {
  const size_t N = (size_t)c->g.N, d = sizeof(double), dd = sizeof(lesjet::Dual);
  AdjLayout L;
  size_t o = 0;
  auto take = [&](size_t bytes) {
    const size_t at_ = o;
    o = align256(o + bytes);
    return at_;
  };
  L.acc = take((18 + 3 * 45) * N * d);  // accumulators, then the interface records
  L.node = take(8 * N * d);
  L.mk = take(2 * N * d);
  L.lamMK = take(2 * N * d);
  L.S = take(6 * 5 * N * d);
  L.lamS = take(5 * N * d);
  L.lamR = take(5 * N * d);
  L.lamQ0 = take(5 * N * d);
  L.work = take(5 * N * d);
  L.lam = take(5 * N * d);
  L.Qnext = take(5 * N * d);
  L.E = take(5 * (size_t)c->g.n[1] * c->g.n[2] * d);
  L.partials = take(((size_t)lesjet::kRedBlocks * 16 + 64) * d);
  L.scal = take(64 * d);
  L.qd = take(5 * N * dd);
  L.mkd = take(2 * N * dd);
  L.noded = take(8 * N * dd);
  L.fluxd = take(15 * N * dd);
  L.rd = take(5 * N * dd);
  L.K = K > 0 ? K : 1;
  L.nckpt = nsteps > 0 ? (nsteps + L.K - 1) / L.K + 1 : 1;
  L.ckpt = take((size_t)L.nckpt * 5 * N * d);
  // one segment of the window: the six stage states and the frozen viscosity
  // of each of its K steps, kept from the recompute for the reverse sweep
  const int ks = nsteps > 0 ? L.K : 0;
  L.segS = take((size_t)ks * 6 * 5 * N * d);
  L.segMK = take((size_t)ks * 2 * N * d);
  L.segN = take((size_t)ks * 5 * 8 * N * d);  // node quantities of the five stage inputs
  L.total = o;
  return L;
}

int adj_check(les_ctx* c) {
  int rc = ready(c);
  if (rc != LES_OK) return rc;
  if (c->p.precision != LES_PREC_FP64)
    return fail(c, LES_ERR_UNSUPPORTED, "the adjoint is provided for the FP64 form");
  if (c->p.sgs_model != LES_SGS_NONE)
    return fail(c, LES_ERR_UNSUPPORTED, "the adjoint supports sgs_model = LES_SGS_NONE");
  if (c->p.bc == LES_BC_JET_CHAR)
    return fail(c, LES_ERR_UNSUPPORTED, "the adjoint supports bc = LES_BC_FROZEN or LES_BC_JET");
  if (c->p.dt_mode != LES_DT_FIXED)
    return fail(c, LES_ERR_UNSUPPORTED, "the adjoint needs dt_mode = LES_DT_FIXED");
  if (!c->p.freeze_visc)
    return fail(c, LES_ERR_UNSUPPORTED, "the adjoint needs freeze_visc = 1");
  if (c->p.axis)
    return fail(c, LES_ERR_UNSUPPORTED, "the adjoint is provided for grids without an axis");
  if (c->g.glo || c->g.ghi)
    return fail(c, LES_ERR_UNSUPPORTED, "the adjoint is provided for undivided grids");
  return LES_OK;
}

template <typename T>
T* aw_at(void* aw, size_t off) {
  return reinterpret_cast<T*>(reinterpret_cast<char*>(aw) + off);
}

lesjet::StageIO64 adj_io(les_ctx* c, void* aw, const AdjLayout& Ly, const double* Qin) {
  lesjet::StageIO64 io;
  io.Qin = Qin;
  io.M = at<double>(c, c->off_m64);
  io.gn = at<double>(c, c->off_gn);
  io.nu = at<double>(c, c->off_nu);
  io.node = aw_at<double>(aw, Ly.node);
  io.mk = aw_at<double>(aw, Ly.mk);
  io.flux = at<double>(c, c->off_flux);
  io.partials = at<double>(c, c->off_part);
  io.sc = at<DevScalars>(c, c->off_sc);
  return io;
}

// Forward recompute of one step from S[0] = Q^n: frozen viscosity mk of Q^n
// and the stage states S[1..5] (S[5] before the boundary conditions).  With
// nodes != nullptr ([5][8][N]) the node quantities of the five stage inputs
// are kept there for the reverse sweep.
void adj_forward(les_ctx* c, void* aw, const AdjLayout& Ly, double* const S[6], double* mk,
                 double* nodes, cudaStream_t s) {
  lesjet::Launch L{s, &c->launches};
  const Grid& g = c->g;
  lesjet::StageIO64 io = adj_io(c, aw, Ly, S[0]);
  io.mk = mk;
  auto node_of = [&](int l) { return nodes ? nodes + (size_t)(l - 1) * 8 * g.N : io.node; };
  lesjet::launch_dt_finalize(c->p, at<double>(c, c->off_part), at<DevScalars>(c, c->off_sc), 0, L);
  io.node = node_of(1);
  lesjet::launch_node64(g, c->p, io, false, L);  // node quantities of Q^n = stage-1 input
  lesjet::launch_mu64(g, c->p, io, L);
  for (int l = 1; l <= 5; ++l) {
    io.Qin = S[l - 1];
    io.node = node_of(l);
    if (l > 1) lesjet::launch_node64(g, c->p, io, false, L);
    lesjet::launch_sensor64(g, io, L);
    for (int d = 0; d < 3; ++d) lesjet::launch_flux64(g, c->p, io, d, L);
    lesjet::launch_update64(g, io, S[0], kAlpha[l - 1], 1, S[l], L);
  }
}

// Reverse of one step whose forward states S[0..5] and viscosity mk are
// stored: lam_out = (dQ^{n+1}/dQ^n)^T lam_next; grad_dev[16] +=
// (dQ^{n+1}/da)^T lam_next.  lam_out may alias lam_next.
void adj_reverse(les_ctx* c, void* aw, const AdjLayout& Ly, double* const S[6], const double* mk,
                 const double* nodes, double t_n, const double* lam_next, double* lam_out,
                 double* grad_dev, cudaStream_t s) {
  lesjet::Launch L{s, &c->launches};
  const Grid& g = c->g;
  const size_t bytes = 5 * (size_t)g.N * sizeof(double);
  const double dt = c->p.dt_fixed;
  const double* M = at<double>(c, c->off_m64);
  DevScalars* sc = at<DevScalars>(c, c->off_sc);
  double* lamS = aw_at<double>(aw, Ly.lamS);
  double* lamR = aw_at<double>(aw, Ly.lamR);
  double* lamQ0 = aw_at<double>(aw, Ly.lamQ0);
  double* lamMK = aw_at<double>(aw, Ly.lamMK);
  double* Qnext = aw_at<double>(aw, Ly.Qnext);
  lesjet::StageIO64 io = adj_io(c, aw, Ly, S[0]);
  io.mk = const_cast<double*>(mk);
  // boundary conditions at t^{n+1}
  if (jet_bc(c)) {
    cudaMemcpyAsync(Qnext, S[5], bytes, cudaMemcpyDeviceToDevice, s);
    lesjet::launch_bc_jet(g, c->p, Qnext, M, at<double>(c, c->off_rth), sc, 1, t_n + dt, L);
    lesjet::launch_bc_vjp(g, c->p, M, at<double>(c, c->off_rth), S[5], Qnext, lam_next, t_n + dt,
                          lamS, aw_at<double>(aw, Ly.E), aw_at<double>(aw, Ly.partials), grad_dev, L);
  } else {
    cudaMemcpyAsync(lamS, lam_next, bytes, cudaMemcpyDeviceToDevice, s);
  }
  // stages 5 .. 1
  cudaMemsetAsync(lamQ0, 0, bytes, s);
  cudaMemsetAsync(lamMK, 0, 2 * (size_t)g.N * sizeof(double), s);
  for (int l = 5; l >= 1; --l) {
    lesjet::launch_stage_prep(g, M, kAlpha[l - 1] * dt, lamS, lamR, lamQ0, L);
    io.Qin = S[l - 1];
    if (nodes)
      io.node = const_cast<double*>(nodes) + (size_t)(l - 1) * 8 * g.N;  // kept by adj_forward
    else
      lesjet::launch_node64(g, c->p, io, false, L);
    lesjet::launch_sensor64(g, io, L);
    lesjet::launch_rhs_vjp(g, c->p, S[l - 1], M, io.gn, io.node, io.mk, lamR, aw_at<double>(aw, Ly.acc),
                           lamS, lamMK, L, io.nu);
  }
  lesjet::launch_axpy(5 * g.N, 1.0, lamS, lamQ0, L);
  lesjet::launch_mu_vjp(g, c->p, S[0], lamMK, lamQ0, L);
  cudaMemcpyAsync(lam_out, lamQ0, bytes, cudaMemcpyDeviceToDevice, s);
}

}  // namespace

extern "C" {

size_t les_adjoint_workspace_bytes(const les_ctx* c, int nsteps, int ckpt_every) {
  return c ? adj_layout(c, nsteps, ckpt_every).total : 0;
}

int les_rhs_jvp(les_ctx* c, const double* Q, const double* dQ, const double* dMK, double* R,
                double* dR, void* aw, les_stream_t stream) {
  int rc = ready(c);
  if (rc != LES_OK) return rc;
  if (c->p.precision != LES_PREC_FP64) return fail(c, LES_ERR_UNSUPPORTED, "FP64 contexts only");
  if (!Q || !dQ || !dR || !aw) return fail(c, LES_ERR_INVALID_ARG, "null pointer");
  if (!aligned16(Q) || !aligned16(dQ) || !aligned16(dR) || !aligned16(aw) || (R && !aligned16(R)) ||
      (dMK && !aligned16(dMK)))
    return fail(c, LES_ERR_ALIGN, "unaligned device pointer");
  lesjet::Launch L{(cudaStream_t)stream, &c->launches};
  const AdjLayout Ly = adj_layout(c, 0, 1);
  const long long N = c->g.N;
  lesjet::StageIO64 io = adj_io(c, aw, Ly, Q);
  lesjet::launch_node64(c->g, c->p, io, false, L);
  lesjet::launch_mu64(c->g, c->p, io, L);
  lesjet::Dual* qd = aw_at<lesjet::Dual>(aw, Ly.qd);
  lesjet::Dual* mkd = aw_at<lesjet::Dual>(aw, Ly.mkd);
  lesjet::Dual* rd = aw_at<lesjet::Dual>(aw, Ly.rd);
  lesjet::launch_pack_dual(5 * N, Q, dQ, qd, L);
  lesjet::launch_pack_dual(2 * N, io.mk, dMK, mkd, L);
  lesjet::launch_rhs_jvp(c->g, c->p, qd, io.M, mkd, aw_at<lesjet::Dual>(aw, Ly.noded),
                         aw_at<lesjet::Dual>(aw, Ly.fluxd), rd, L);
  lesjet::launch_unpack_dual(5 * N, rd, R, dR, L);
  return cuda_check(c, "les_rhs_jvp");
}

int les_rhs_vjp(les_ctx* c, const double* Q, const double* lamR, double* lamQ, double* lamMK,
                void* aw, les_stream_t stream) {
  int rc = ready(c);
  if (rc != LES_OK) return rc;
  if (c->p.precision != LES_PREC_FP64) return fail(c, LES_ERR_UNSUPPORTED, "FP64 contexts only");
  if (!Q || !lamR || !lamQ || !lamMK || !aw) return fail(c, LES_ERR_INVALID_ARG, "null pointer");
  if (!aligned16(Q) || !aligned16(lamR) || !aligned16(lamQ) || !aligned16(lamMK) || !aligned16(aw))
    return fail(c, LES_ERR_ALIGN, "unaligned device pointer");
  cudaStream_t s = (cudaStream_t)stream;
  lesjet::Launch L{s, &c->launches};
  const AdjLayout Ly = adj_layout(c, 0, 1);
  lesjet::StageIO64 io = adj_io(c, aw, Ly, Q);
  lesjet::launch_node64(c->g, c->p, io, false, L);
  lesjet::launch_mu64(c->g, c->p, io, L);
  cudaMemsetAsync(lamMK, 0, 2 * (size_t)c->g.N * sizeof(double), s);
  lesjet::launch_sensor64(c->g, io, L);
  lesjet::launch_rhs_vjp(c->g, c->p, Q, io.M, io.gn, io.node, io.mk, lamR, aw_at<double>(aw, Ly.acc), lamQ,
                         lamMK, L, io.nu);
  return cuda_check(c, "les_rhs_vjp");
}

int les_adjoint_step(les_ctx* c, const double* Qn, double t_n, const double* lam_next,
                     double* lam_out, double grad[16], void* aw, les_stream_t stream) {
  int rc = adj_check(c);
  if (rc != LES_OK) return rc;
  if (!Qn || !lam_next || !lam_out || !aw) return fail(c, LES_ERR_INVALID_ARG, "null pointer");
  if (!aligned16(Qn) || !aligned16(lam_next) || !aligned16(lam_out) || !aligned16(aw))
    return fail(c, LES_ERR_ALIGN, "unaligned device pointer");
  cudaStream_t s = (cudaStream_t)stream;
  const AdjLayout Ly = adj_layout(c, 0, 1);
  double* gdev = aw_at<double>(aw, Ly.scal) + 1;
  cudaMemsetAsync(gdev, 0, 16 * sizeof(double), s);
  double* S[6];
  for (int l = 0; l < 6; ++l) S[l] = aw_at<double>(aw, Ly.S) + (size_t)l * 5 * c->g.N;
  cudaMemcpyAsync(S[0], Qn, 5 * (size_t)c->g.N * sizeof(double), cudaMemcpyDeviceToDevice, s);
  double* mk = aw_at<double>(aw, Ly.mk);
  adj_forward(c, aw, Ly, S, mk, nullptr, s);
  adj_reverse(c, aw, Ly, S, mk, nullptr, t_n, lam_next, lam_out, gdev, s);
  if ((rc = cuda_check(c, "les_adjoint_step")) != LES_OK) return rc;
  double h[16];
  cudaMemcpyAsync(h, gdev, sizeof(h), cudaMemcpyDeviceToHost, s);
  if (cudaStreamSynchronize(s) != cudaSuccess) return cuda_check(c, "les_adjoint_step sync");
  if (grad)
    for (int m = 0; m < 16; ++m) grad[m] += h[m];
  return cuda_check(c, "les_adjoint_step");
}

int les_adjoint_window(les_ctx* c, const double* Q_start, double t0, int nsteps, int ckpt_every,
                       int j_surface, void* aw, double* J_out, double grad[16],
                       les_stream_t stream) {
  int rc = adj_check(c);
  if (rc != LES_OK) return rc;
  if (!Q_start || !aw || nsteps < 1 || ckpt_every < 1)
    return fail(c, LES_ERR_INVALID_ARG, "null pointer, nsteps < 1 or ckpt_every < 1");
  if (j_surface < 0 || j_surface >= c->g.n[1]) return fail(c, LES_ERR_INVALID_ARG, "j_surface out of range");
  if (!aligned16(Q_start) || !aligned16(aw)) return fail(c, LES_ERR_ALIGN, "unaligned device pointer");
  cudaStream_t s = (cudaStream_t)stream;
  lesjet::Launch L{s, &c->launches};
  const AdjLayout Ly = adj_layout(c, nsteps, ckpt_every);
  const int K = Ly.K;
  const Grid& g = c->g;
  const size_t bytes = 5 * (size_t)g.N * sizeof(double);
  const double dt = c->p.dt_fixed;
  const double* M = at<double>(c, c->off_m64);
  double* scal = aw_at<double>(aw, Ly.scal);
  double* Jdev = scal;            // J
  double* gdev = scal + 1;        // gradient [16]
  double* Jscratch = scal + 17;   // discarded J of the reverse pass
  double* part = aw_at<double>(aw, Ly.partials);
  double* work = aw_at<double>(aw, Ly.work);
  double* lam = aw_at<double>(aw, Ly.lam);
  auto ckpt = [&](int k) { return aw_at<double>(aw, Ly.ckpt) + (size_t)k * 5 * g.N; };
  auto segS = [&](int m, int l) {
    return aw_at<double>(aw, Ly.segS) + ((size_t)m * 6 + l) * 5 * g.N;
  };
  auto segMK = [&](int m) { return aw_at<double>(aw, Ly.segMK) + (size_t)m * 2 * g.N; };
  auto segN = [&](int m) { return aw_at<double>(aw, Ly.segN) + (size_t)m * 5 * 8 * g.N; };
  cudaMemsetAsync(scal, 0, 64 * sizeof(double), s);
  DevScalars* sc = at<DevScalars>(c, c->off_sc);
  const int last = (nsteps - 1) / K;  // the last segment is kept by the forward sweep
  // one step from segS(m, 0), keeping its stage states; Q^{n+1} goes to dst
  auto kept_step = [&](int m, int n, double* dst) {
    double* S[6];
    for (int l = 0; l < 6; ++l) S[l] = segS(m, l);
    adj_forward(c, aw, Ly, S, segMK(m), segN(m), s);
    cudaMemcpyAsync(dst, S[5], bytes, cudaMemcpyDeviceToDevice, s);
    if (jet_bc(c))
      lesjet::launch_bc_jet(g, c->p, dst, M, at<double>(c, c->off_rth), sc, 1, t0 + (n + 1) * dt, L);
  };
  // forward window, checkpoints every K steps
  cudaMemcpyAsync(ckpt(0), Q_start, bytes, cudaMemcpyDeviceToDevice, s);
  cudaMemcpyAsync(work, Q_start, bytes, cudaMemcpyDeviceToDevice, s);
  lesjet::launch_set_time(sc, t0, L);
  for (int n = 1; n <= nsteps; ++n) {
    const int m = n - 1 - last * K;
    const double* Qn = work;
    if (m < 0) {
      rk_step(c, work, s);
    } else {
      if (m == 0) cudaMemcpyAsync(segS(0, 0), work, bytes, cudaMemcpyDeviceToDevice, s);
      double* dst = (n == nsteps) ? work : segS(m + 1, 0);
      kept_step(m, n - 1, dst);
      Qn = dst;
    }
    lesjet::launch_functional(g, c->p, j_surface, dt, M, Qn, nullptr, part, Jdev, L);
    if (n % K == 0 && n < nsteps) cudaMemcpyAsync(ckpt(n / K), work, bytes, cudaMemcpyDeviceToDevice, s);
  }
  // reverse sweep, segment by segment, recomputing the segment's states
  cudaMemsetAsync(lam, 0, bytes, s);
  for (int sg = last; sg >= 0; --sg) {
    const int n0 = sg * K, n1 = (n0 + K < nsteps) ? n0 + K : nsteps;
    // recompute the segment from its checkpoint, keeping every stage state
    // and viscosity (Q^{n1} itself is the next checkpoint)
    if (sg != last) {
      cudaMemcpyAsync(segS(0, 0), ckpt(sg), bytes, cudaMemcpyDeviceToDevice, s);
      for (int m = 0; m < n1 - n0; ++m) {
        if (m + 1 < n1 - n0) {
          kept_step(m, n0 + m, segS(m + 1, 0));
        } else {
          double* S[6];
          for (int l = 0; l < 6; ++l) S[l] = segS(m, l);
          adj_forward(c, aw, Ly, S, segMK(m), segN(m), s);
        }
      }
    }
    for (int n = n1; n >= n0 + 1; --n) {
      const int m = n - 1 - n0;
      const double* Qn = (n == nsteps) ? work : ((n == n1) ? ckpt(sg + 1) : segS(m + 1, 0));
      lesjet::launch_functional(g, c->p, j_surface, dt, M, Qn, lam, part, Jscratch, L);
      double* S[6];
      for (int l = 0; l < 6; ++l) S[l] = segS(m, l);
      adj_reverse(c, aw, Ly, S, segMK(m), segN(m), t0 + (n - 1) * dt, lam, lam, gdev, s);
    }
  }
  if ((rc = cuda_check(c, "les_adjoint_window")) != LES_OK) return rc;
  double h[17];
  cudaMemcpyAsync(h, scal, sizeof(h), cudaMemcpyDeviceToHost, s);
  if (cudaStreamSynchronize(s) != cudaSuccess) return cuda_check(c, "les_adjoint_window sync");
  if (J_out) *J_out = h[0];
  if (grad)
    for (int m = 0; m < 16; ++m) grad[m] = h[1 + m];
  return cuda_check(c, "les_adjoint_window");
}

int les_grid_jet(int ni, int nj, int nk, const les_jet_grid* gp, double* xyz, les_stream_t stream) {
  if (!gp || !xyz) return LES_ERR_INVALID_ARG;
  if (ni < 2 || nj < 2 || nk < 2) return LES_ERR_SHAPE;
  const long long N = (long long)ni * nj * nk;
  if (N >= (1LL << 40)) return LES_ERR_SHAPE;
  const les_jet_grid G = *gp;
  if (!(G.length > 0.0) || !(G.r0 >= 0.0) || !(G.r0 < G.r_c) || !(G.r_c < G.r1) || !(G.A >= 0.0) ||
      !(G.A < 1.0) || !(G.beta > 0.0))
    return LES_ERR_INVALID_ARG;
  if (!aligned16(xyz)) return LES_ERR_ALIGN;
  const double q = G.ratio > 0.0 ? G.ratio : (ni <= 288 ? 1.01 : std::pow(1.01, 288.0 / ni));
  // s_c: the point the map r(s; s_c) sends to r_c (bisection on the monotone r(s_c; s_c))
  auto gmap = [&](double s, double sc) {
    return s - (G.A / G.beta) * (std::tanh(G.beta * (s - sc)) + std::tanh(G.beta * sc));
  };
  double lo = 0.0, hi = 1.0;
  for (int it = 0; it < 200; ++it) {
    const double mid = 0.5 * (lo + hi);
    const double r = G.r0 + (G.r1 - G.r0) * gmap(mid, mid) / gmap(1.0, mid);
    if (r < G.r_c)
      lo = mid;
    else
      hi = mid;
  }
  Grid g;
  g.n[0] = ni;
  g.n[1] = nj;
  g.n[2] = nk;
  g.per[0] = g.per[1] = 0;
  g.per[2] = 1;
  g.N = N;
  g.stride[0] = (long long)nj * nk;
  g.stride[1] = nk;
  g.stride[2] = 1;
  unsigned long long launches = 0;
  lesjet::Launch L{(cudaStream_t)stream, &launches};
  lesjet::launch_grid_jet(g, G.length, q, G.r0, G.r1, G.A, G.beta, 0.5 * (lo + hi), xyz, L);
  return cudaGetLastError() == cudaSuccess ? LES_OK : LES_ERR_CUDA;
}

int les_surface_functional(les_ctx* c, const double* Q, int j_surface, double w, double* J_out,
                           les_stream_t stream) {
  int rc = ready(c);
  if (rc != LES_OK) return rc;
  if (!Q || !J_out) return fail(c, LES_ERR_INVALID_ARG, "null pointer");
  if (!aligned16(Q)) return fail(c, LES_ERR_ALIGN, "unaligned device pointer");
  if (j_surface < 0 || j_surface >= c->g.n[1]) return fail(c, LES_ERR_INVALID_ARG, "j_surface out of range");
  cudaStream_t s = (cudaStream_t)stream;
  lesjet::Launch L{s, &c->launches};
  double* part = at<double>(c, c->off_part);
  double* out = part + 4 * (size_t)lesjet::kMaxPartials;  // past the block partials
  cudaMemsetAsync(out, 0, sizeof(double), s);
  if (has_m64(c))
    lesjet::launch_functional(c->g, c->p, j_surface, w, at<double>(c, c->off_m64), Q, nullptr, part,
                              out, L);
  else
    lesjet::launch_functional(c->g, c->p, j_surface, w, at<float>(c, c->off_m32), Q, part, out, L);
  if ((rc = cuda_check(c, "les_surface_functional")) != LES_OK) return rc;
  double h = 0.0;
  cudaMemcpyAsync(&h, out, sizeof(double), cudaMemcpyDeviceToHost, s);
  if (cudaStreamSynchronize(s) != cudaSuccess) return cuda_check(c, "les_surface_functional sync");
  *J_out = h;
  return cuda_check(c, "les_surface_functional");
}

}  // extern "C"

// Read-only views of a context for other translation units of the library
// (not exported from the shared object).
namespace lesjet {
__attribute__((visibility("hidden"))) const les_params* ctx_params(const les_ctx* c) {
  return &c->p;
}
__attribute__((visibility("hidden"))) void ctx_shape(const les_ctx* c, int shape[3]) {
  shape[0] = c->g.n[0];
  shape[1] = c->g.n[1];
  shape[2] = c->g.n[2];
}
__attribute__((visibility("hidden"))) void ctx_set_error(les_ctx* c, const char* msg) {
  c->err = msg;
}
}  // namespace lesjet
