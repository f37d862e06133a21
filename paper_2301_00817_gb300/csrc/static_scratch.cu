// static_scratch.cu -- les_time_step_static: the global CFL time step of a
// state computed with NO device allocation by the library or the caller.
//
// Who needs it: code that holds a solver state and its metrics but may not
// call cudaMalloc or grow a device memory pool -- for example a monitoring or
// steering hook that an application calls between solver steps after it has
// committed all device memory to its own fixed pool, or a plain-C tool that
// receives only raw device pointers and has no allocator of its own.  Such a
// caller cannot provide the workspace that les_time_step uses.
//
// Its scratch is the file-scope array g_static_scratch below: per-axial-plane
// minima and flags plus the result.  Every GPU that loads the library holds
// it until the process exits.  All calls share it and it keeps the last
// call's contents, so calls that overlap on the GPU (on different streams or
// host threads) race; each call overwrites every slot it reads, so nothing
// has to be cleared between calls.
//
// Set-up: the device address of the array is looked up with
// cudaGetSymbolAddress with the caller's device current, once per CUDA
// context (the module holding the array is loaded afresh, at another
// address, into every context: a second context on the same device, or the
// primary context re-created after cudaDeviceReset).  The first call in a
// context does this lookup, so it should come before any stream capture.
#include <cuda.h>  // driver types only: the two entry points below come through the runtime
#include <cuda_runtime.h>

#include <mutex>

#include "../../include/lesjet.h"
#include "lesjet_dev.cuh"

// [0, max_ni): plane minima of 1/(lambda_xi + lambda_eta + lambda_zeta);
// [max_ni, 2 max_ni): plane flags (1.0 = non-finite or non-positive state);
// [2 max_ni]: dt; [2 max_ni + 1]: flag of the whole state.  256 KiB.
static __device__ __align__(256) double g_static_scratch[2 * LES_STATIC_MAX_NI + 2];

namespace {

constexpr int kStaticMaxNi = LES_STATIC_MAX_NI;
constexpr int kMaxDevices = 64;

// Address of g_static_scratch as seen in one context of a device.
struct ScratchSlot {
  double* ptr = nullptr;
  unsigned long long ctx_id = 0;  // cuCtxGetId of the context the address belongs to
  bool keyed = false;             // ctx_id is valid
};
ScratchSlot g_slots[kMaxDevices];
std::mutex g_setup_mutex;

typedef CUresult (*PfnCtxGetCurrent)(CUcontext*);
typedef CUresult (*PfnCtxGetId)(CUcontext, unsigned long long*);

// Unique id of the context current to this thread (ids are never reused,
// unlike context handles); false if the driver cannot tell.
bool current_context_id(unsigned long long* id) {
  static PfnCtxGetCurrent get_current = nullptr;
  static PfnCtxGetId get_id = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    cudaDriverEntryPointQueryResult q1 = cudaDriverEntryPointSymbolNotFound, q2 = q1;
    void* f1 = nullptr;
    void* f2 = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f1, 12000, cudaEnableDefault, &q1) ==
            cudaSuccess &&
        q1 == cudaDriverEntryPointSuccess &&
        cudaGetDriverEntryPointByVersion("cuCtxGetId", &f2, 12000, cudaEnableDefault, &q2) ==
            cudaSuccess &&
        q2 == cudaDriverEntryPointSuccess) {
      get_current = (PfnCtxGetCurrent)f1;
      get_id = (PfnCtxGetId)f2;
    }
  });
  if (!get_current || !get_id) return false;
  CUcontext c = nullptr;
  if (get_current(&c) != CUDA_SUCCESS || c == nullptr) return false;
  return get_id(c, id) == CUDA_SUCCESS;
}

// One block per axial plane i: FP64 spectral radii of every node of the plane
// (same formulas as the time step of les_time_step) and the plane minimum.
__global__ void k_static_plane_min(lesjet::Grid g, double gamma, const double* __restrict__ Q,
                                   const double* __restrict__ M, double* __restrict__ scratch) {
  const int i = blockIdx.x;
  const long long N = g.N;
  const long long plane = (long long)g.n[1] * g.n[2];
  const long long base = (long long)i * plane;
  double local_min = 1.0e300;
  int bad = 0;
  for (long long e = threadIdx.x; e < plane; e += blockDim.x) {
    const long long n = base + e;
    const double rho = Q[n];
    const double inv_rho = 1.0 / rho;
    const double u = Q[N + n] * inv_rho, v = Q[2 * N + n] * inv_rho, w = Q[3 * N + n] * inv_rho;
    const double p = (gamma - 1.0) * (Q[4 * N + n] - 0.5 * rho * (u * u + v * v + w * w));
    const double a = sqrt(gamma * p * inv_rho);
    double lsum = 0.0;
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      const double mx = M[(3 * d) * N + n], my = M[(3 * d + 1) * N + n], mz = M[(3 * d + 2) * N + n];
      lsum += fabs(mx * u + my * v + mz * w) + a * sqrt(mx * mx + my * my + mz * mz);
    }
    const double inv = 1.0 / lsum;
    if (!(rho > 0.0) || !(p > 0.0) || !(inv > 0.0) || !(inv < 1.0e300)) bad = 1;
    local_min = inv < local_min ? inv : local_min;
  }
  __shared__ double smin[32];
  __shared__ int sbad[32];
  for (int off = 16; off > 0; off >>= 1) {
    local_min = fmin(local_min, __shfl_xor_sync(0xffffffffu, local_min, off));
    bad |= __shfl_xor_sync(0xffffffffu, bad, off);
  }
  if ((threadIdx.x & 31) == 0) {
    smin[threadIdx.x >> 5] = local_min;
    sbad[threadIdx.x >> 5] = bad;
  }
  __syncthreads();
  if (threadIdx.x < 32) {
    const bool live = threadIdx.x < (blockDim.x >> 5);
    double m = live ? smin[threadIdx.x] : 1.0e300;
    int b = live ? sbad[threadIdx.x] : 0;
    for (int off = 16; off > 0; off >>= 1) {
      m = fmin(m, __shfl_xor_sync(0xffffffffu, m, off));
      b |= __shfl_xor_sync(0xffffffffu, b, off);
    }
    if (threadIdx.x == 0) {
      scratch[i] = m;
      scratch[kStaticMaxNi + i] = b ? 1.0 : 0.0;
    }
  }
}

// Minimum over the ni plane minima (fixed order), then dt and the flag.
__global__ void k_static_final(int ni, int mode, double cfl, double dt_fixed,
                               double* __restrict__ scratch) {
  __shared__ double smin[32];
  __shared__ double sbad[32];
  double m = 1.0e300, b = 0.0;
  for (int i = threadIdx.x; i < ni; i += blockDim.x) {
    m = fmin(m, scratch[i]);
    b = fmax(b, scratch[kStaticMaxNi + i]);
  }
  for (int off = 16; off > 0; off >>= 1) {
    m = fmin(m, __shfl_xor_sync(0xffffffffu, m, off));
    b = fmax(b, __shfl_xor_sync(0xffffffffu, b, off));
  }
  if ((threadIdx.x & 31) == 0) {
    smin[threadIdx.x >> 5] = m;
    sbad[threadIdx.x >> 5] = b;
  }
  __syncthreads();
  if (threadIdx.x < 32) {
    const bool live = threadIdx.x < (blockDim.x >> 5);
    m = live ? smin[threadIdx.x] : 1.0e300;
    b = live ? sbad[threadIdx.x] : 0.0;
    for (int off = 16; off > 0; off >>= 1) {
      m = fmin(m, __shfl_xor_sync(0xffffffffu, m, off));
      b = fmax(b, __shfl_xor_sync(0xffffffffu, b, off));
    }
    if (threadIdx.x == 0) {
      double dt = (mode == LES_DT_FIXED) ? dt_fixed : cfl * m;
      if (!(dt > 0.0) || !(dt < 1.0e300)) b = 1.0;
      scratch[2 * kStaticMaxNi] = dt;
      scratch[2 * kStaticMaxNi + 1] = b;
    }
  }
}

// Device address of g_static_scratch in the context current to this thread
// (the runtime's primary context of the current device unless the caller
// made another one current), looked up once per context.
cudaError_t scratch_for_current_context(double** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_setup_mutex);
  ScratchSlot& slot = g_slots[dev];
  unsigned long long id = 0;
  bool keyed = current_context_id(&id);
  if (keyed && slot.keyed && slot.ptr && slot.ctx_id == id) {
    *out = slot.ptr;
    return cudaSuccess;
  }
  double* ptr = nullptr;
  e = cudaGetSymbolAddress((void**)&ptr, g_static_scratch);
  if (e != cudaSuccess) return e;
  // the lookup makes the runtime's context current if none was: key on it
  if (!keyed) keyed = current_context_id(&id);
  slot.ptr = ptr;
  slot.ctx_id = id;
  slot.keyed = keyed;  // unkeyed: looked up again on every call
  *out = ptr;
  return cudaSuccess;
}

}  // namespace

// Read-only views of the host-side context (defined in api.cu).
namespace lesjet {
const les_params* ctx_params(const les_ctx* c);
void ctx_shape(const les_ctx* c, int shape[3]);
void ctx_set_error(les_ctx* c, const char* msg);
}  // namespace lesjet

extern "C" int les_time_step_static(les_ctx* ctx, const double* Q, const double* M,
                                    double* dt_out, les_stream_t stream) {
  if (!ctx || !Q || !M || !dt_out) return LES_ERR_INVALID_ARG;
  if ((reinterpret_cast<uintptr_t>(Q) & 15u) || (reinterpret_cast<uintptr_t>(M) & 15u)) {
    lesjet::ctx_set_error(ctx, "les_time_step_static: device pointers must be 16-byte aligned");
    return LES_ERR_ALIGN;
  }
  const les_params* p = lesjet::ctx_params(ctx);
  int shape[3];
  lesjet::ctx_shape(ctx, shape);
  if (shape[0] > kStaticMaxNi) {
    lesjet::ctx_set_error(ctx, "les_time_step_static: ni exceeds LES_STATIC_MAX_NI (16384 axial "
                                "planes), the size of its static scratch; use les_time_step");
    return LES_ERR_SHAPE;
  }
  double* scratch = nullptr;
  cudaError_t e = scratch_for_current_context(&scratch);
  if (e != cudaSuccess) {
    lesjet::ctx_set_error(ctx, cudaGetErrorString(e));
    return LES_ERR_CUDA;
  }
  lesjet::Grid g;
  g.n[0] = shape[0];
  g.n[1] = shape[1];
  g.n[2] = shape[2];
  for (int d = 0; d < 3; ++d) g.per[d] = p->periodic[d] ? 1 : 0;
  g.N = (long long)shape[0] * shape[1] * shape[2];
  g.stride[0] = (long long)shape[1] * shape[2];
  g.stride[1] = shape[2];
  g.stride[2] = 1;
  cudaStream_t s = (cudaStream_t)stream;
  // cudaLaunchKernel returns each launch's own error: the thread's sticky
  // last-error state (which may hold another component's error) is neither
  // read nor cleared here
  double gamma = p->gamma;
  void* args1[] = {&g, &gamma, (void*)&Q, (void*)&M, &scratch};
  e = cudaLaunchKernel((const void*)k_static_plane_min, dim3(shape[0]), dim3(256), args1, 0, s);
  int ni = shape[0], mode = p->dt_mode;
  double cfl = p->cfl, dt_fixed = p->dt_fixed;
  void* args2[] = {&ni, &mode, &cfl, &dt_fixed, &scratch};
  if (e == cudaSuccess)
    e = cudaLaunchKernel((const void*)k_static_final, dim3(1), dim3(1024), args2, 0, s);
  double host[2] = {0.0, 0.0};
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(host, scratch + 2 * kStaticMaxNi, sizeof(host), cudaMemcpyDeviceToHost, s);
  // errors raised while the kernels run surface here
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) {
    lesjet::ctx_set_error(ctx, cudaGetErrorString(e));
    return LES_ERR_CUDA;
  }
  *dt_out = host[0];
  if (host[1] != 0.0) {
    lesjet::ctx_set_error(ctx, "les_time_step_static: non-finite or non-positive state");
    return LES_ERR_NONFINITE;
  }
  return LES_OK;
}
