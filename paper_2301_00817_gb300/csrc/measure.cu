// measure.cu -- FMA throughput of the device's CUDA cores (FP64 and FP32),
// the arithmetic roof of the ALU-bound kernels.  Every thread advances
// kChains independent FMA chains, so the pipe is limited by issue rate, not
// by dependent-instruction latency; the grid fills every SM several times.
#include <cuda_runtime.h>

#include "lesjet.h"

namespace {

constexpr int kChains = 16;
constexpr int kThreads = 256;

template <typename T>
__global__ void __launch_bounds__(kThreads) k_fma_chains(T* __restrict__ out, int iters, T a, T b) {
  T x[kChains];
#pragma unroll
  for (int j = 0; j < kChains; ++j) x[j] = (T)(threadIdx.x + j) * (T)1e-3;
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int j = 0; j < kChains; ++j) x[j] = x[j] * a + b;
  }
  T s = 0;
#pragma unroll
  for (int j = 0; j < kChains; ++j) s += x[j];
  if (s == (T)-12345.0) out[blockIdx.x] = s;  // keeps the chains live
}

template <typename T>
int run(int iters, double* tflops, cudaStream_t s) {
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return LES_ERR_CUDA;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int blocks = (sms > 0 ? sms : 152) * 8;
  T* out = nullptr;  // never written (the guard value is not reached)
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  // the multiplier is 1 - 2^-20 and the addend small: the chains stay finite
  const T a = (T)0.99999904632568359375, b = (T)1e-7;
  k_fma_chains<T><<<blocks, kThreads, 0, s>>>(out, iters / 8, a, b);  // warm-up
  cudaEventRecord(e0, s);
  k_fma_chains<T><<<blocks, kThreads, 0, s>>>(out, iters, a, b);
  cudaEventRecord(e1, s);
  int rc = LES_OK;
  float ms = 0.f;
  if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess ||
      cudaGetLastError() != cudaSuccess || !(ms > 0.f))
    rc = LES_ERR_CUDA;
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (rc != LES_OK) return rc;
  const double flops = 2.0 * kChains * (double)iters * (double)blocks * kThreads;
  *tflops = flops / ((double)ms * 1e-3) / 1e12;
  return LES_OK;
}

}  // namespace

extern "C" int les_measure_fma_peak(int precision, double* tflops, les_stream_t stream) {
  if (!tflops) return LES_ERR_INVALID_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  if (precision == LES_PREC_FP64) return run<double>(1 << 12, tflops, s);
  if (precision == LES_PREC_MIXED || precision == LES_PREC_MIXED_COMPACT)
    return run<float>(1 << 16, tflops, s);
  return LES_ERR_INVALID_ARG;
}
