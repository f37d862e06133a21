// stage.cu -- time-step finalisation and small helpers of the stepping
// path (the residual and stage update live in fused.cu).
#include "lesjet_dev.cuh"
#include "lesjet_host.h"

namespace lesjet {

static int blocks_for(long long count, int threads, long long cap = 0) {
  if (cap <= 0) cap = 64LL * sm_count();
  long long b = (count + threads - 1) / threads;
  if (b > cap) b = cap;
  if (b < 1) b = 1;
  return (int)b;
}

// Fixed-order minimum over the block partials, then dt and t^{n+1}.
__global__ void k_dt_finalize(const double* __restrict__ partials, int nparts, int mode,
                              double cfl, double dt_fixed, int advance, DevScalars* sc) {
  __shared__ double sm[32];
  double m = 1.0e300;
  for (int i = threadIdx.x; i < nparts; i += blockDim.x) m = fmin(m, partials[i]);
  for (int off = 16; off > 0; off >>= 1) m = fmin(m, __shfl_xor_sync(0xffffffffu, m, off));
  if ((threadIdx.x & 31) == 0) sm[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x < 32) {
    m = threadIdx.x < (blockDim.x >> 5) ? sm[threadIdx.x] : 1.0e300;
    for (int off = 16; off > 0; off >>= 1) m = fmin(m, __shfl_xor_sync(0xffffffffu, m, off));
    if (threadIdx.x == 0) {
      double dt = (mode == LES_DT_FIXED) ? dt_fixed : cfl * m;
      if (!(dt > 0.0) || !(dt < 1.0e300)) {
        sc->status = LES_ERR_NONFINITE;
        dt = 0.0;
      } else if (sc->status != 0) {
        sc->status = LES_ERR_NONFINITE;
      }
      sc->dt = dt;
      if (advance) {
        sc->t += dt;
        sc->steps += 1;
      }
    }
  }
}

__global__ void k_set_dt(DevScalars* sc, double dt) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    sc->dt = dt;
    sc->t += dt;
    sc->steps += 1;
  }
}

void launch_set_dt(DevScalars* sc, double dt, const Launch& L) {
  k_set_dt<<<1, 32, 0, L.s>>>(sc, dt);
  ++*L.counter;
}

template <typename R>
__global__ void k_cast_to_double(long long count, const R* __restrict__ a, double* __restrict__ b) {
  for (long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x; n < count;
       n += (long long)gridDim.x * blockDim.x)
    b[n] = (double)a[n];
}

// ------------------------------------------------------------- launchers

void launch_dt_finalize(const les_params& p, double* partials, DevScalars* sc, int advance,
                        const Launch& L) {
  k_dt_finalize<<<1, 1024, 0, L.s>>>(partials, kRedBlocks, p.dt_mode, p.cfl, p.dt_fixed, advance,
                                     sc);
  ++*L.counter;
}

void launch_mk_to_double(int precision, const Grid& g, const void* mk, int fields, double* out,
                         const Launch& L) {
  const long long count = fields * g.N;
  if (precision == LES_PREC_FP64) {
    cudaMemcpyAsync(out, mk, count * sizeof(double), cudaMemcpyDeviceToDevice, L.s);
  } else {
    k_cast_to_double<float><<<blocks_for(count, 256), 256, 0, L.s>>>(count, (const float*)mk, out);
    ++*L.counter;
  }
}

}  // namespace lesjet
