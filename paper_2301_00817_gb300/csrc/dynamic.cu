// dynamic.cu -- the dynamic Smagorinsky procedure (Sec. "Dynamic Smagorinsky
// Model", Eqs. yoshizawa, av_ci, av_cd, av_Pr_sgs), for the FP64 form and,
// with FP32 node fields, products, filter and per-node terms (the sums
// still in FP64, fixed order), for the mixed forms.
//
// Once per viscosity evaluation, from the node primitives of the state:
//   k_dyn_products  per node: the 25 fields the test filter acts on (rho,
//                   rho u_i, rho T, rho u_i u_j, rho|S| S_ij, rho|S| S_mm,
//                   rho|S|^2, rho u_j T, rho|S| dT/dx_j);
//   k_dyn_filter3   the test filter (a tensor product of 3-point filters,
//                   applied along zeta, eta, xi in that order) in one pass
//                   over the FP32 fields; k_dyn_filter1, one direction per
//                   pass, for the FP64 fields;
//   k_dyn_favre     the Favre-filtered velocity and temperature per node;
//   k_dyn_sums      per interior node: the strain of the Favre-filtered
//                   velocity, the Leonard-type terms, and the six
//                   J^-1-weighted sums of the numerators and denominators;
//                   fixed-grid block partials (deterministic);
//   k_dyn_final     one block: fixed-order totals and the coefficients
//                   C_ds, C_I (clipped at 0) and Pr_sgs (the configured
//                   value when the dynamic one is not positive).
// The viscosity pass (k_mu) then forms mu_sgs = C_ds rho Delta^2 |S|, the
// dynamic kappa_sgs and the Yoshizawa sigma_ll = 2 C_I rho Delta^2 |S|^2.
// Test filter: the (1/4, 1/2, 1/4) trapezoidal filter along each direction
// (width 2 Delta), identity along a non-periodic direction at its faces.
#include "stage64_kernels.cuh"

namespace lesjet {

namespace {

constexpr int kDynFields = 25;
constexpr int kDynSums = 7;  // six weighted sums and the sum of the weights

// Cartesian gradient of a node field through the node's metrics.
template <typename R, typename TM>
__device__ __forceinline__ void grad_of(const Grid& g, const TM* __restrict__ M,
                                        const R* __restrict__ f, long long n, const int c[3],
                                        R out[3]) {
  const long long N = g.N;
  R dd[3];
#pragma unroll
  for (int d = 0; d < 3; ++d) dd[d] = node_deriv(g, f, n, c, d);
#pragma unroll
  for (int x = 0; x < 3; ++x)
    out[x] = (R)M[x * N + n] * dd[0] + (R)M[(3 + x) * N + n] * dd[1] + (R)M[(6 + x) * N + n] * dd[2];
}

// S_ij from a velocity gradient gr[i][x] = d u_i/d x_x; returns |S|.
template <typename R>
__device__ __forceinline__ R strain(const R gr[3][3], R S[3][3]) {
  R ss = R(0);
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      S[i][j] = R(0.5) * (gr[i][j] + gr[j][i]);
      ss += S[i][j] * S[i][j];
    }
  return dev_sqrt(R(2) * ss);
}

__constant__ int kI6[6] = {0, 1, 2, 0, 0, 1};
__constant__ int kJ6[6] = {0, 1, 2, 1, 2, 2};

// Register bounds (here and on k_dyn_sums): left free, the compiler gave
// these kernels 230-254 registers, one 256-thread block per SM for a
// latency-bound pass; the FP32 forms fit 64 (80 for the sums) registers.
template <typename R, typename TQ, typename TM>
__global__ void __launch_bounds__(256, sizeof(R) == 4 ? 4 : 2) k_dyn_products(Grid g, const TQ* __restrict__ Q,
                                                      const TM* __restrict__ M,
                                                      const R* __restrict__ node,
                                                      R* __restrict__ D) {
  const long long N = g.N;
  for (long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x; n < N;
       n += (long long)gridDim.x * blockDim.x) {
    int c[3];
    decompose(g, n, c);
    const R rho = (R)Q[n];
    const R vel[3] = {node[n], node[N + n], node[2 * N + n]};
    const R T = node[4 * N + n];
    R gr[3][3], S[3][3], dT[3];
#pragma unroll
    for (int q = 0; q < 3; ++q) grad_of(g, M, node + q * N, n, c, gr[q]);
    grad_of(g, M, node + 4 * N, n, c, dT);
    const R Sm = strain(gr, S);
    D[n] = rho;
#pragma unroll
    for (int i = 0; i < 3; ++i) D[(1 + i) * N + n] = rho * vel[i];
    D[4 * N + n] = rho * T;
#pragma unroll
    for (int k = 0; k < 6; ++k) {
      const int i = kI6[k], j = kJ6[k];
      D[(5 + k) * N + n] = rho * vel[i] * vel[j];
      D[(11 + k) * N + n] = rho * Sm * S[i][j];
    }
    D[17 * N + n] = rho * Sm * (S[0][0] + S[1][1] + S[2][2]);
    D[18 * N + n] = rho * Sm * Sm;
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      D[(19 + j) * N + n] = rho * vel[j] * T;
      D[(22 + j) * N + n] = rho * Sm * dT[j];
    }
  }
}

// One pass of the test filter along direction D for `count` fields:
// dst = (src_{-1} + 2 src_0 + src_{+1})/4 along D (periodic wrap), the
// identity at the faces of a non-periodic D.
template <int D, typename R>
__global__ void __launch_bounds__(256) k_dyn_filter1(Grid g, const R* __restrict__ src,
                                                     int count, R* __restrict__ dst) {
  const long long N = g.N;
  const long long s = g.stride[D];
  const int nd = g.n[D];
  for (long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x; n < N;
       n += (long long)gridDim.x * blockDim.x) {
    int c[3];
    decompose(g, n, c);
    const bool face = !g.per[D] && (c[D] == 0 || c[D] == nd - 1);
    if (face) {
      for (int q = 0; q < count; ++q) dst[q * N + n] = src[q * N + n];
      continue;
    }
    const long long np = (c[D] == nd - 1) ? n - (long long)(nd - 1) * s : n + s;
    const long long nm = (c[D] == 0) ? n + (long long)(nd - 1) * s : n - s;
#pragma unroll 5
    for (int q = 0; q < count; ++q)
      dst[q * N + n] = R(0.25) * src[q * N + nm] + R(0.5) * src[q * N + n] + R(0.25) * src[q * N + np];
  }
}

// The test filter's three directions in one kernel.  A CTA owns a tile of
// kF3J x kF3K (eta, zeta) columns and a range of planes [i0, i1), and takes
// the fields NB at a time.  For each group it marches along xi over planes
// i0 - 1 .. i1: it stages the plane's tile with a one-node halo in shared
// memory, filters along zeta over the halo rows, then along eta, and keeps
// the last three of its column's 2-D-filtered values in registers to
// filter along xi.  Each output takes the same operations in the same order
// as three one-direction passes would (zeta, eta, xi; identity at the faces
// of a non-periodic direction).  Traffic: each field read once (with the
// tile and chunk halos) and written once, against three reads and three
// writes for separate passes; the NB fields of a group share the barriers
// and keep several loads in flight per thread (one field at a time was
// latency-bound: 40% slower than three passes).
constexpr int kF3J = 8, kF3K = 32;  // tile rows (eta) x columns (zeta); 256 threads

template <typename R, int NB>
__global__ void __launch_bounds__(kF3J * kF3K) k_dyn_filter3(Grid g, const R* __restrict__ src,
                                                             int count, int nch,
                                                             R* __restrict__ dst) {
  __shared__ R S[NB][kF3J + 2][kF3K + 2];  // the plane's tile with a one-node halo
  __shared__ R Z[NB][kF3J + 2][kF3K];      // filtered along zeta, rows -1 .. kF3J
  const long long N = g.N;
  const int ni = g.n[0], nj = g.n[1], nk = g.n[2];
  const int tx = threadIdx.x % kF3K, ty = threadIdx.x / kF3K;
  const int k0 = blockIdx.x * kF3K, j0 = blockIdx.y * kF3J;
  const int i0 = (int)((long long)blockIdx.z * ni / nch);
  const int i1 = (int)((long long)(blockIdx.z + 1) * ni / nch);
  const int j = j0 + ty, k = k0 + tx;
  const bool own = j < nj && k < nk;
  auto wrap = [](int v, int n, int per) {  // -1 outside a non-periodic range
    if (per) return ((v % n) + n) % n;     // (a tile may span several periods)
    return (v >= 0 && v < n) ? v : -1;
  };
  const bool jface = !g.per[1] && (j == 0 || j == nj - 1);
  for (int f0 = 0; f0 < count; f0 += NB) {  // NB fields at a time (count % NB == 0)
    R em[NB], ec[NB];  // 2-D-filtered values of planes x - 2, x - 1
#pragma unroll
    for (int b = 0; b < NB; ++b) em[b] = ec[b] = R(0);
    for (int x = i0 - 1; x <= i1; ++x) {
      const int ig = wrap(x, ni, g.per[0]);
      R e[NB];
#pragma unroll
      for (int b = 0; b < NB; ++b) e[b] = R(0);
      if (ig >= 0) {  // (uniform over the CTA)
        const long long pbase = (long long)ig * nj * nk;
        for (int q = threadIdx.x; q < (kF3J + 2) * (kF3K + 2); q += blockDim.x) {
          const int r = q / (kF3K + 2), c = q - r * (kF3K + 2);
          const int jg = wrap(j0 - 1 + r, nj, g.per[1]), kg = wrap(k0 - 1 + c, nk, g.per[2]);
          const bool in = jg >= 0 && kg >= 0;
          const long long off = pbase + (long long)jg * nk + kg;
#pragma unroll
          for (int b = 0; b < NB; ++b) S[b][r][c] = in ? src[(long long)(f0 + b) * N + off] : R(0);
        }
        __syncthreads();
        for (int q = threadIdx.x; q < (kF3J + 2) * kF3K; q += blockDim.x) {
          const int r = q / kF3K, c = q - r * kF3K;
          const int kk = k0 + c;
          const bool face = !g.per[2] && (kk == 0 || kk == nk - 1);
#pragma unroll
          for (int b = 0; b < NB; ++b)
            Z[b][r][c] = face ? S[b][r][c + 1]
                              : R(0.25) * S[b][r][c] + R(0.5) * S[b][r][c + 1] + R(0.25) * S[b][r][c + 2];
        }
        __syncthreads();
#pragma unroll
        for (int b = 0; b < NB; ++b)
          e[b] = jface ? Z[b][ty + 1][tx]
                       : R(0.25) * Z[b][ty][tx] + R(0.5) * Z[b][ty + 1][tx] + R(0.25) * Z[b][ty + 2][tx];
      }
      // plane x - 1 has both xi neighbours now
      const int xo = x - 1;
      if (xo >= i0 && xo < i1 && own) {
        const bool face = !g.per[0] && (xo == 0 || xo == ni - 1);
        const long long o = (long long)xo * nj * nk + (long long)j * nk + k;
#pragma unroll
        for (int b = 0; b < NB; ++b)
          dst[(long long)(f0 + b) * N + o] = face ? ec[b] : R(0.25) * em[b] + R(0.5) * ec[b] + R(0.25) * e[b];
      }
#pragma unroll
      for (int b = 0; b < NB; ++b) {
        em[b] = ec[b];
        ec[b] = e[b];
      }
    }
  }
}

// Favre-filtered velocity and temperature u^_i = (rho u_i)^/rho^,
// T^ = (rho T)^/rho^ at every node, from the filtered fields F.
template <typename R>
__global__ void __launch_bounds__(256) k_dyn_favre(long long N, const R* __restrict__ F,
                                                   R* __restrict__ H) {
  for (long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x; n < N;
       n += (long long)gridDim.x * blockDim.x) {
    const R r = F[n];
#pragma unroll
    for (int q = 0; q < 4; ++q) H[q * N + n] = F[(1 + q) * N + n] / r;
  }
}

// Per interior node the six terms (numerators and denominators of the
// three coefficients), in R; their J^-1-weighted sums in FP64.
template <typename R, typename TM>
__global__ void __launch_bounds__(256, sizeof(R) == 4 ? 3 : 1) k_dyn_sums(Grid g, const TM* __restrict__ M,
                                                  const R* __restrict__ node,
                                                  const R* __restrict__ Fh,
                                                  const R* __restrict__ H,
                                                  double* __restrict__ partials) {
  const long long N = g.N;
  double acc[kDynSums] = {0, 0, 0, 0, 0, 0, 0};
  for (long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x; n < N;
       n += (long long)gridDim.x * blockDim.x) {
    int c[3];
    decompose(g, n, c);
    if (!is_interior(g, c)) continue;
    const double wgt = (double)M[9 * N + n];
    const R Delta = cbrt((R)M[9 * N + n]);
    const R D2 = Delta * Delta, Dh2 = R(4) * D2;
    R gr[3][3], S[3][3], dT[3], grh[3][3], Sh[3][3], dTh[3];
#pragma unroll
    for (int q = 0; q < 3; ++q) grad_of(g, M, node + q * N, n, c, gr[q]);
    grad_of(g, M, node + 4 * N, n, c, dT);
    strain(gr, S);
#pragma unroll
    for (int q = 0; q < 3; ++q) grad_of(g, M, H + q * N, n, c, grh[q]);
    grad_of(g, M, H + 3 * N, n, c, dTh);
    const R Shm = strain(grh, Sh);
    // the filtered fields at this node (Fh holds all 25)
    R fh[kDynFields];
#pragma unroll
    for (int q = 5; q < kDynFields; ++q) fh[q] = Fh[q * N + n];
    const R rh = Fh[n];
    const R mh[3] = {Fh[N + n], Fh[2 * N + n], Fh[3 * N + n]};
    R L[3][3], Fs[3][3];
#pragma unroll
    for (int k = 0; k < 6; ++k) {
      const int i = kI6[k], j = kJ6[k];
      L[i][j] = L[j][i] = fh[5 + k] - mh[i] * mh[j] / rh;
      Fs[i][j] = Fs[j][i] = fh[11 + k];
    }
    const R trS = S[0][0] + S[1][1] + S[2][2];
    const R trSh = Sh[0][0] + Sh[1][1] + Sh[2][2];
    R LS = R(0), FS = R(0), ShS = R(0);
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int j = 0; j < 3; ++j) {
        LS += L[i][j] * S[i][j];
        FS += Fs[i][j] * S[i][j];
        ShS += Sh[i][j] * S[i][j];
      }
    const R Lkk = L[0][0] + L[1][1] + L[2][2];
    const R numC = LS - Lkk * trS / R(3);
    const R denC = R(2) * D2 * (FS - fh[17] * trS / R(3)) -
                   R(2) * Dh2 * (rh * Shm * ShS - rh * Shm * trSh * trS / R(3));
    const R denI = R(2) * Dh2 * rh * Shm * Shm - R(2) * D2 * fh[18];
    R numP = R(0), denP = R(0);
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      const R K = fh[19 + j] - mh[j] * Fh[4 * N + n] / rh;
      numP += D2 * fh[22 + j] * dT[j] - Dh2 * rh * Shm * dTh[j] * dT[j];
      denP += K * dT[j];
    }
    acc[0] += wgt * (double)numC;
    acc[1] += wgt * (double)denC;
    acc[2] += wgt * (double)Lkk;
    acc[3] += wgt * (double)denI;
    acc[4] += wgt * (double)numP;
    acc[5] += wgt * (double)denP;
    acc[6] += wgt;
  }
  __shared__ double red[kDynSums][32];
#pragma unroll
  for (int q = 0; q < kDynSums; ++q)
    for (int off = 16; off > 0; off >>= 1) acc[q] += __shfl_xor_sync(0xffffffffu, acc[q], off);
  if ((threadIdx.x & 31) == 0)
#pragma unroll
    for (int q = 0; q < kDynSums; ++q) red[q][threadIdx.x >> 5] = acc[q];
  __syncthreads();
  if (threadIdx.x < 32) {
#pragma unroll
    for (int q = 0; q < kDynSums; ++q) {
      double v = threadIdx.x < (blockDim.x >> 5) ? red[q][threadIdx.x] : 0.0;
      for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
      if (threadIdx.x == 0) partials[q * kRedBlocks + blockIdx.x] = v;
    }
  }
}

// One block of kDynSums warps: warp q totals partial array q in a fixed order.
__global__ void k_dyn_final(const double* __restrict__ partials, double pr_default,
                            DevScalars* __restrict__ sc) {
  __shared__ double tot[kDynSums];
  const int q = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (q < kDynSums) {
    double v = 0.0;
    for (int b = lane; b < kRedBlocks; b += 32) v += partials[q * kRedBlocks + b];
    for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
    if (lane == 0) tot[q] = v;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double* out = sc->dyn;
    for (int k = 0; k < 6; ++k) out[k] = tot[k] / tot[6];
    double Cd = out[1] != 0.0 ? out[0] / out[1] : 0.0;
    if (!(Cd > 0.0)) Cd = 0.0;
    double CI = out[3] != 0.0 ? out[2] / out[3] : 0.0;
    if (!(CI > 0.0)) CI = 0.0;
    double Pr = out[5] != 0.0 ? Cd * out[4] / out[5] : 0.0;
    if (!(Pr > 0.0) || !(Pr < 1e300)) Pr = pr_default;
    out[6] = Cd;
    out[7] = CI;
    out[8] = Pr;
  }
}

}  // namespace

template <typename R, typename TQ, typename TM>
static void dynamic_t(const Grid& g, const les_params& p, const TQ* Q, const TM* M, const R* node,
                      R* scratch, double* partials, DevScalars* sc, const Launch& L) {
  const int th = 256, nb = blocks_for(g.N, th);
  R* D = scratch;                                 // products, then the eta pass
  R* T = scratch + (long long)kDynFields * g.N;  // zeta pass, then the filtered fields
  k_dyn_products<R, TQ, TM><<<nb, th, 0, L.s>>>(g, Q, M, node, D);
  if constexpr (sizeof(R) == 4) {
    // FP32 fields: the test filter in one pass (k_dyn_filter3), with enough
    // axial chunks for about eight CTAs per SM
    const int tk = (g.n[2] + kF3K - 1) / kF3K, tj = (g.n[1] + kF3J - 1) / kF3J;
    const long long want = 8LL * sm_count();
    int nch = (int)((want + (long long)tk * tj - 1) / ((long long)tk * tj));
    nch = nch < 1 ? 1 : (nch > g.n[0] ? g.n[0] : nch);
    static_assert(kDynFields % 5 == 0, "the filter takes the fields five at a time");
    k_dyn_filter3<R, 5><<<dim3(tk, tj, nch), kF3J * kF3K, 0, L.s>>>(g, D, kDynFields, nch, T);
    *L.counter += 1;
  } else {
    // FP64 fields: three one-direction passes (the one-pass kernel is bound
    // by its FP64 work and latency there: 1.24 against 0.86 ms on 1.97M points)
    k_dyn_filter1<2, R><<<nb, th, 0, L.s>>>(g, D, kDynFields, T);
    k_dyn_filter1<1, R><<<nb, th, 0, L.s>>>(g, T, kDynFields, D);
    k_dyn_filter1<0, R><<<nb, th, 0, L.s>>>(g, D, kDynFields, T);
    *L.counter += 3;
  }
  k_dyn_favre<R><<<nb, th, 0, L.s>>>(g.N, T, D);  // D is free again: u^, v^, w^, T^
  k_dyn_sums<R, TM><<<kRedBlocks, kRedThreads, 0, L.s>>>(g, M, node, T, D, partials);
  k_dyn_final<<<1, 32 * kDynSums, 0, L.s>>>(partials, p.Pr_sgs, sc);
  *L.counter += 4;
}

void launch_dynamic64(const Grid& g, const les_params& p, const StageIO64& io, double* scratch,
                      const Launch& L) {
  dynamic_t<double, double, double>(g, p, io.Qin, io.M, io.node, scratch, io.partials, io.sc, L);
}

void launch_dynamic32(const Grid& g, const les_params& p, const float* Q, const float* M,
                      float* node, float* scratch, double* partials, DevScalars* sc,
                      const Launch& L) {
  // the FP32 node fields (u v w p T; the radii are not used) of the float state
  const int th = 256, nb = blocks_for(g.N, th);
  k_node<float, float, float, false><<<nb, th, 0, L.s>>>(g, make_consts<float>(p), Q, M, nullptr, node,
                                                        partials, sc);
  ++*L.counter;
  dynamic_t<float, float, float>(g, p, Q, M, node, scratch, partials, sc, L);
}

}  // namespace lesjet
