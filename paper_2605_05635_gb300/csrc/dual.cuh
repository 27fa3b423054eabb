// dual.cuh -- forward-mode dual numbers (value + N tangents) for the
// Jacobian products of the adjoint kernel.  Only the operations the
// right-hand side, the lapses and the emitter/emissivity formulas use.
#pragma once
#include <cuda_runtime.h>

namespace bhrt {
// A nested namespace keeps these overloads from hiding the global double
// math functions inside bhrt; argument-dependent lookup finds them for duals.
namespace ad {

template <int N>
struct Dual {
  double v;
  double d[N];
  __host__ __device__ Dual() : v(0.0) {
#pragma unroll
    for (int i = 0; i < N; ++i) d[i] = 0.0;
  }
  __host__ __device__ Dual(double x) : v(x) {  // NOLINT: implicit constant
#pragma unroll
    for (int i = 0; i < N; ++i) d[i] = 0.0;
  }
  __host__ __device__ static Dual var(double x, int k) {
    Dual r(x);
    r.d[k] = 1.0;
    return r;
  }
};

#define BH_DUAL_UNARY(name, fv, fd)                                      \
  template <int N>                                                       \
  __host__ __device__ inline Dual<N> name(const Dual<N>& a) {            \
    Dual<N> r;                                                           \
    const double x = a.v;                                                \
    r.v = fv;                                                            \
    const double g = fd;                                                 \
    for (int i = 0; i < N; ++i) r.d[i] = g * a.d[i];                     \
    return r;                                                            \
  }

template <int N>
__host__ __device__ inline Dual<N> operator+(const Dual<N>& a, const Dual<N>& b) {
  Dual<N> r;
  r.v = a.v + b.v;
  for (int i = 0; i < N; ++i) r.d[i] = a.d[i] + b.d[i];
  return r;
}
template <int N>
__host__ __device__ inline Dual<N> operator-(const Dual<N>& a, const Dual<N>& b) {
  Dual<N> r;
  r.v = a.v - b.v;
  for (int i = 0; i < N; ++i) r.d[i] = a.d[i] - b.d[i];
  return r;
}
template <int N>
__host__ __device__ inline Dual<N> operator-(const Dual<N>& a) {
  Dual<N> r;
  r.v = -a.v;
  for (int i = 0; i < N; ++i) r.d[i] = -a.d[i];
  return r;
}
template <int N>
__host__ __device__ inline Dual<N> operator*(const Dual<N>& a, const Dual<N>& b) {
  Dual<N> r;
  r.v = a.v * b.v;
  for (int i = 0; i < N; ++i) r.d[i] = a.d[i] * b.v + a.v * b.d[i];
  return r;
}
template <int N>
__host__ __device__ inline Dual<N> operator/(const Dual<N>& a, const Dual<N>& b) {
  Dual<N> r;
  const double ib = 1.0 / b.v;
  r.v = a.v * ib;
  for (int i = 0; i < N; ++i) r.d[i] = (a.d[i] - r.v * b.d[i]) * ib;
  return r;
}
template <int N>
__host__ __device__ inline Dual<N> operator+(const Dual<N>& a, double b) {
  Dual<N> r = a;
  r.v += b;
  return r;
}
template <int N>
__host__ __device__ inline Dual<N> operator+(double b, const Dual<N>& a) { return a + b; }
template <int N>
__host__ __device__ inline Dual<N> operator-(const Dual<N>& a, double b) { return a + (-b); }
template <int N>
__host__ __device__ inline Dual<N> operator-(double b, const Dual<N>& a) { return -a + b; }
template <int N>
__host__ __device__ inline Dual<N> operator*(const Dual<N>& a, double b) {
  Dual<N> r;
  r.v = a.v * b;
  for (int i = 0; i < N; ++i) r.d[i] = a.d[i] * b;
  return r;
}
template <int N>
__host__ __device__ inline Dual<N> operator*(double b, const Dual<N>& a) { return a * b; }
template <int N>
__host__ __device__ inline Dual<N> operator/(const Dual<N>& a, double b) { return a * (1.0 / b); }
template <int N>
__host__ __device__ inline Dual<N> operator/(double b, const Dual<N>& a) { return Dual<N>(b) / a; }

BH_DUAL_UNARY(exp, ::exp(x), r.v)
BH_DUAL_UNARY(log1p, ::log1p(x), 1.0 / (1.0 + x))
BH_DUAL_UNARY(sqrt, ::sqrt(x), 0.5 / r.v)
BH_DUAL_UNARY(sin, ::sin(x), ::cos(x))
BH_DUAL_UNARY(cos, ::cos(x), -::sin(x))
BH_DUAL_UNARY(tanh, ::tanh(x), 1.0 - r.v * r.v)
#undef BH_DUAL_UNARY

template <int N>
__host__ __device__ inline Dual<N> log(const Dual<N>& a) {
  Dual<N> r;
  r.v = ::log(a.v);
  for (int i = 0; i < N; ++i) r.d[i] = a.d[i] / a.v;
  return r;
}

// a^b for a > 0, both arguments carrying tangents.
template <int N>
__host__ __device__ inline Dual<N> pow(const Dual<N>& a, const Dual<N>& b) {
  return exp(b * log(a));
}

// Overloads used by the generic lapse and right-hand side (found by
// argument-dependent lookup when they are instantiated on duals).
template <int N>
__host__ __device__ inline Dual<N> d_exp(const Dual<N>& x) { return exp(x); }
template <int N>
__host__ __device__ inline Dual<N> d_log1p(const Dual<N>& x) { return log1p(x); }
template <int N>
__host__ __device__ inline void d_sincos(const Dual<N>& x, Dual<N>* s, Dual<N>* c) {
  *s = sin(x);
  *c = cos(x);
}
template <int N>
__host__ __device__ inline Dual<N> d_rcp(const Dual<N>& x) { return Dual<N>(1.0) / x; }
template <int N>
__host__ __device__ inline bool operator>(const Dual<N>& a, const Dual<N>& b) { return a.v > b.v; }

}  // namespace ad
using ad::Dual;
}  // namespace bhrt
