// lesjet_dev.cuh -- device-side types and helpers shared by the CUDA
// translation units of liblesjet (sm_103a).  Nothing here is shared with the
// CPU oracle.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/lesjet.h"

namespace lesjet {

// Structured grid, k fastest: node n = (i*nj + j)*nk + k.
struct Grid {
  int n[3];
  int per[3];
  long long N;
  long long stride[3];  // {nj*nk, nk, 1}
  // ghost planes at the low / high xi end of an axial slab (0 at a physical
  // face): those planes belong to the neighbouring slab, which refreshes
  // them between the stages; this grid updates, reduces and sums only its
  // own planes [glo, n[0] - ghi)
  int glo = 0, ghi = 0;
};

// Own planes of a slab (every plane of an undivided grid).
__host__ __device__ inline bool owned_plane(const Grid& g, int i) {
  return i >= g.glo && i < g.n[0] - g.ghi;
}

// Scheme constants in the compute precision R.
template <typename R>
struct Consts {
  R gamma, gm1;      // gamma, gamma - 1
  R k2, k4;          // dissipation constants
  R mu_scale;        // M_j / Re (0 when inviscid)
  R S_suth;          // 110.4 K / T_ref
  R cs2;             // Cs^2 (Smagorinsky) or 2.5 Cs^2 (Vreman)
  R inv_gm1_pr;      // 1/((gamma-1) Pr)
  R inv_gm1_prs;     // 1/((gamma-1) Pr_sgs)
  int sgs;           // LES_SGS_*
  int axis;          // 1: ring j = 0 on the axis (J^-1 = 0 there), Reading A27
};

// Device-resident scalars of a context (inside the workspace).
struct DevScalars {
  double t;          // simulation time (t^{n+1} once a step's dt is known)
  double dt;         // current step
  int status;        // LES_OK or LES_ERR_NONFINITE (sticky)
  int steps;
  unsigned int ticket;  // blocks of a reduction that have finished (its last
                        // block finalises and resets it to 0)
  int pad_;
  double totals[5];
  double dyn[9];     // dynamic SGS procedure: 6 averaged terms, C_ds, C_I, Pr_sgs
};

// Reductions run on a fixed grid (whatever the GPU's SM count), so their
// block partials and summation order, hence their bits, never change.
constexpr int kRedBlocks = 1216;
constexpr int kRedThreads = 256;
constexpr int kMaxPartials = kRedBlocks;

// Multiprocessor count of the current device (cached per device), for
// sizing grid-stride launches in whole waves.
inline int sm_count() {
  static int cache[64] = {0};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 152;
  if (cache[dev] == 0) {
    int sms = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms <= 0)
      sms = 152;
    cache[dev] = sms;
  }
  return cache[dev];
}

__host__ __device__ inline long long idx3(const Grid& g, int i, int j, int k) {
  return ((long long)i * g.n[1] + j) * g.n[2] + k;
}

__device__ __forceinline__ void decompose(const Grid& g, long long n, int c[3]) {
  if (g.N <= 0x7fffffffLL) {  // every index fits 32 bits: the cheaper division
    const unsigned u = (unsigned)n, nk = (unsigned)g.n[2], nj = (unsigned)g.n[1];
    const unsigned r = u / nk;
    c[2] = (int)(u - r * nk);
    c[0] = (int)(r / nj);
    c[1] = (int)(r - (unsigned)c[0] * nj);
    return;
  }
  long long r = n / g.n[2];
  c[2] = (int)(n - r * g.n[2]);
  c[0] = (int)(r / g.n[1]);
  c[1] = (int)(r - (long long)c[0] * g.n[1]);
}

// Node 'off' steps from node n (coordinates c) along direction d; -1 when it
// falls outside a non-periodic direction.  Periodic directions wrap.
__device__ __forceinline__ long long step(const Grid& g, long long n, const int c[3],
                                          int d, int off) {
  int nd = g.n[d];
  int v = c[d] + off;
  if (g.per[d]) {
    if (v >= nd) v -= nd;
    else if (v < 0) v += nd;
  } else if (v < 0 || v >= nd) {
    return -1;
  }
  return n + (long long)(v - c[d]) * g.stride[d];
}

// Coordinate along d of the node step(g, n, c, d, off) returned (valid only
// when that node exists): c[d] + off, wrapped like step().
__device__ __forceinline__ int coord_step(const Grid& g, const int c[3], int d, int off) {
  int v = c[d] + off;
  if (v >= g.n[d]) v -= g.n[d];
  else if (v < 0) v += g.n[d];
  return v;
}

// A node the stages update: inside every non-periodic face, and along xi
// inside the slab's own planes (a ghost plane is refreshed by the exchange).
__device__ __forceinline__ bool is_interior(const Grid& g, const int c[3]) {
#pragma unroll
  for (int d = 0; d < 3; ++d)
    if (!g.per[d] && (c[d] == 0 || c[d] == g.n[d] - 1)) return false;
  return c[0] >= g.glo && c[0] < g.n[0] - g.ghi;
}

template <typename T>
__device__ __forceinline__ T dev_sqrt(T x);
template <>
__device__ __forceinline__ double dev_sqrt<double>(double x) { return sqrt(x); }
template <>
__device__ __forceinline__ float dev_sqrt<float>(float x) { return sqrtf(x); }

template <typename T>
__device__ __forceinline__ T dev_abs(T x) { return x < T(0) ? -x : x; }

template <typename T>
__device__ __forceinline__ T dev_max(T a, T b) { return a > b ? a : b; }

// ----------------------------------------------------------------- Philox
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): ten rounds of two
// 32x32->64 multiplies with the round multipliers, word swap, xor with the
// key; the key advances by the two Weyl increments between rounds.
__device__ inline void philox4x32_10(uint32_t x[4], uint32_t k0, uint32_t k1) {
  const uint32_t A = 0xD2511F53u, B = 0xCD9E8D57u;
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    uint32_t hiA = __umulhi(A, x[0]), loA = A * x[0];
    uint32_t hiB = __umulhi(B, x[2]), loB = B * x[2];
    uint32_t y0 = hiB ^ x[1] ^ k0;
    uint32_t y2 = hiA ^ x[3] ^ k1;
    x[0] = y0;
    x[1] = loB;
    x[2] = y2;
    x[3] = loA;
    k0 += 0x9E3779B9u;
    k1 += 0xBB67AE85u;
  }
}

}  // namespace lesjet

// Host-side launch helpers implemented in the .cu files.
namespace lesjet {

struct Launch {
  cudaStream_t s;
  unsigned long long* counter;
};

// On a grid with an axis (Reading A27) an axis node's SGS viscosity is the
// azimuthal mean of ring 1's at its plane, summed in increasing k; its
// laminar part is its own.  One block per plane i, after k_mu (or the mixed
// prestep) has written mk for every node: ring 1's SGS part is mk minus its
// laminar part.  T(n) gives a node's temperature.
template <typename R>
__device__ __forceinline__ R mu_laminar(const Consts<R>& K, R T) {
  return K.mu_scale * T * dev_sqrt(T) * (R(1) + K.S_suth) / (T + K.S_suth);
}

template <typename R, class TempOf>
__global__ void k_mu_axis(Grid g, Consts<R> K, TempOf T, R* __restrict__ mk) {
  extern __shared__ __align__(16) unsigned char smu_raw[];
  R* smu = reinterpret_cast<R*>(smu_raw);
  const int nk = g.n[2];
  const long long N = g.N;
  const long long base0 = (long long)blockIdx.x * g.stride[0];  // (i, 0, 0)
  const long long base1 = base0 + g.stride[1];                  // (i, 1, 0)
  for (int k = threadIdx.x; k < nk; k += blockDim.x)
    smu[k] = mk[base1 + k] - mu_laminar(K, T(base1 + k));
  __syncthreads();
  __shared__ R mean;
  if (threadIdx.x == 0) {
    R s = R(0);
    for (int k = 0; k < nk; ++k) s += smu[k];
    mean = s / R(nk);
  }
  __syncthreads();
  for (int k = threadIdx.x; k < nk; k += blockDim.x) {
    const long long n = base0 + k;
    const R ml = mu_laminar(K, T(n));
    mk[n] = ml + mean;
    mk[N + n] = ml * K.inv_gm1_pr + mean * K.inv_gm1_prs;
  }
}

// Temperature of a node from a node array (FP64 form: node[4 N + n]).
template <typename R>
struct TempFromNode {
  const R* node;
  long long N;
  __device__ R operator()(long long n) const { return node[4 * N + n]; }
};

// Temperature of a node recovered from the conserved state (System I
// energy), as the mixed prestep does.
template <typename R, typename TQ>
struct TempFromState {
  const TQ* Q;
  long long N;
  R gamma, gm1;
  __device__ R operator()(long long n) const {
    const R rho = (R)Q[n];
    const R ir = R(1) / rho;
    const R u = (R)Q[N + n] * ir, v = (R)Q[2 * N + n] * ir, w = (R)Q[3 * N + n] * ir;
    const R p = gm1 * ((R)Q[4 * N + n] - R(0.5) * rho * (u * u + v * v + w * w));
    return gamma * p * ir;
  }
};


}  // namespace lesjet
