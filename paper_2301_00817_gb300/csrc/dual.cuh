// dual.cuh -- forward-mode dual numbers (value + one tangent) for device
// code.  Instantiating the FP64 residual kernels on Dual yields the exact
// Jacobian-vector product of the discrete residual, with the same branch
// choices as the FP64 kernels (|x| = x < 0 ? -x : x has derivative +1 at 0;
// max passes the tangent of the operand the comparison selects).
#pragma once

#include <cuda_runtime.h>

#include "lesjet_dev.cuh"

namespace lesjet {

// keep the double overloads visible next to the Dual ones below
using ::cbrt;
using ::cos;
using ::exp;
using ::pow;
using ::sqrt;
using ::tanh;

struct Dual {
  double v, d;
  __host__ __device__ Dual() : v(0.0), d(0.0) {}
  __host__ __device__ Dual(double x) : v(x), d(0.0) {}
  __host__ __device__ Dual(double x, double dx) : v(x), d(dx) {}
  __host__ __device__ explicit operator double() const { return v; }
  __host__ __device__ Dual& operator+=(const Dual& o) { v += o.v; d += o.d; return *this; }
  __host__ __device__ Dual& operator-=(const Dual& o) { v -= o.v; d -= o.d; return *this; }
  __host__ __device__ Dual& operator*=(const Dual& o) { d = d * o.v + v * o.d; v *= o.v; return *this; }
};

__host__ __device__ inline Dual operator-(const Dual& a) { return Dual(-a.v, -a.d); }
__host__ __device__ inline Dual operator+(const Dual& a, const Dual& b) { return Dual(a.v + b.v, a.d + b.d); }
__host__ __device__ inline Dual operator-(const Dual& a, const Dual& b) { return Dual(a.v - b.v, a.d - b.d); }
__host__ __device__ inline Dual operator*(const Dual& a, const Dual& b) { return Dual(a.v * b.v, a.d * b.v + a.v * b.d); }
__host__ __device__ inline Dual operator/(const Dual& a, const Dual& b) {
  const double q = a.v / b.v;
  return Dual(q, (a.d - q * b.d) / b.v);
}
__host__ __device__ inline Dual operator+(const Dual& a, double b) { return Dual(a.v + b, a.d); }
__host__ __device__ inline Dual operator+(double a, const Dual& b) { return Dual(a + b.v, b.d); }
__host__ __device__ inline Dual operator-(const Dual& a, double b) { return Dual(a.v - b, a.d); }
__host__ __device__ inline Dual operator-(double a, const Dual& b) { return Dual(a - b.v, -b.d); }
__host__ __device__ inline Dual operator*(const Dual& a, double b) { return Dual(a.v * b, a.d * b); }
__host__ __device__ inline Dual operator*(double a, const Dual& b) { return Dual(a * b.v, a * b.d); }
__host__ __device__ inline Dual operator/(const Dual& a, double b) { return Dual(a.v / b, a.d / b); }
__host__ __device__ inline Dual operator/(double a, const Dual& b) {
  const double q = a / b.v;
  return Dual(q, -q * b.d / b.v);
}
__host__ __device__ inline bool operator<(const Dual& a, const Dual& b) { return a.v < b.v; }
__host__ __device__ inline bool operator>(const Dual& a, const Dual& b) { return a.v > b.v; }
__host__ __device__ inline bool operator<=(const Dual& a, const Dual& b) { return a.v <= b.v; }
__host__ __device__ inline bool operator>=(const Dual& a, const Dual& b) { return a.v >= b.v; }
__host__ __device__ inline bool operator==(const Dual& a, const Dual& b) { return a.v == b.v; }
__host__ __device__ inline bool operator<(const Dual& a, double b) { return a.v < b; }
__host__ __device__ inline bool operator>(const Dual& a, double b) { return a.v > b; }
__host__ __device__ inline bool operator<=(const Dual& a, double b) { return a.v <= b; }
__host__ __device__ inline bool operator>=(const Dual& a, double b) { return a.v >= b; }

__device__ inline Dual sqrt(const Dual& a) {
  const double s = ::sqrt(a.v);
  return Dual(s, s > 0.0 ? a.d / (2.0 * s) : 0.0);
}
__device__ inline Dual cbrt(const Dual& a) {
  const double c = ::cbrt(a.v);
  return Dual(c, c != 0.0 ? a.d / (3.0 * c * c) : 0.0);
}
__device__ inline Dual pow(const Dual& a, double e) {
  const double p = ::pow(a.v, e);
  return Dual(p, a.v != 0.0 ? e * p / a.v * a.d : 0.0);
}
__device__ inline Dual exp(const Dual& a) {
  const double e = ::exp(a.v);
  return Dual(e, e * a.d);
}
__device__ inline Dual tanh(const Dual& a) {
  const double t = ::tanh(a.v);
  return Dual(t, (1.0 - t * t) * a.d);
}
__device__ inline Dual cos(const Dual& a) { return Dual(::cos(a.v), -::sin(a.v) * a.d); }

template <>
__device__ __forceinline__ Dual dev_sqrt<Dual>(Dual x) {
  return sqrt(x);
}

}  // namespace lesjet
