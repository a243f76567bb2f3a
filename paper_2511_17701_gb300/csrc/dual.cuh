// dual.cuh -- forward-mode dual numbers in FP64: a value and its derivatives along N seeded
// input directions. The pusher templates of pusher.cuh evaluated with R = Dual<N> give the
// directional derivatives of every intermediate, which the adjoint assembles into the
// Jacobian of one step. Only the operations those templates use are defined.
#pragma once
#include <cuda_runtime.h>

namespace {

template <int N>
struct Dual {
  double v;
  double d[N];
  __device__ __forceinline__ Dual() {}
  __device__ __forceinline__ Dual(double x) : v(x) {
#pragma unroll
    for (int i = 0; i < N; ++i) d[i] = 0.0;
  }
};

template <int N>
__device__ __forceinline__ Dual<N> operator+(const Dual<N> &a, const Dual<N> &b) {
  Dual<N> r;
  r.v = a.v + b.v;
#pragma unroll
  for (int i = 0; i < N; ++i) r.d[i] = a.d[i] + b.d[i];
  return r;
}
template <int N>
__device__ __forceinline__ Dual<N> operator-(const Dual<N> &a, const Dual<N> &b) {
  Dual<N> r;
  r.v = a.v - b.v;
#pragma unroll
  for (int i = 0; i < N; ++i) r.d[i] = a.d[i] - b.d[i];
  return r;
}
template <int N>
__device__ __forceinline__ Dual<N> operator-(const Dual<N> &a) {
  Dual<N> r;
  r.v = -a.v;
#pragma unroll
  for (int i = 0; i < N; ++i) r.d[i] = -a.d[i];
  return r;
}
template <int N>
__device__ __forceinline__ Dual<N> operator*(const Dual<N> &a, const Dual<N> &b) {
  Dual<N> r;
  r.v = a.v * b.v;
#pragma unroll
  for (int i = 0; i < N; ++i) r.d[i] = fma(a.d[i], b.v, a.v * b.d[i]);
  return r;
}
template <int N>
__device__ __forceinline__ Dual<N> operator/(const Dual<N> &a, const Dual<N> &b) {
  Dual<N> r;
  const double ib = 1.0 / b.v;
  r.v = a.v * ib;
#pragma unroll
  for (int i = 0; i < N; ++i) r.d[i] = (a.d[i] - r.v * b.d[i]) * ib;
  return r;
}
template <int N>
__device__ __forceinline__ Dual<N> operator+(const Dual<N> &a, double b) { return a + Dual<N>(b); }
template <int N>
__device__ __forceinline__ Dual<N> operator+(double a, const Dual<N> &b) { return Dual<N>(a) + b; }
template <int N>
__device__ __forceinline__ Dual<N> operator-(const Dual<N> &a, double b) { return a - Dual<N>(b); }
template <int N>
__device__ __forceinline__ Dual<N> operator-(double a, const Dual<N> &b) { return Dual<N>(a) - b; }
template <int N>
__device__ __forceinline__ Dual<N> operator*(const Dual<N> &a, double b) {
  Dual<N> r;
  r.v = a.v * b;
#pragma unroll
  for (int i = 0; i < N; ++i) r.d[i] = a.d[i] * b;
  return r;
}
template <int N>
__device__ __forceinline__ Dual<N> operator*(double a, const Dual<N> &b) { return b * a; }
template <int N>
__device__ __forceinline__ Dual<N> operator/(const Dual<N> &a, double b) { return a * (1.0 / b); }
template <int N>
__device__ __forceinline__ Dual<N> operator/(double a, const Dual<N> &b) { return Dual<N>(a) / b; }

template <int N>
__device__ __forceinline__ Dual<N> fma_(const Dual<N> &a, const Dual<N> &b, const Dual<N> &c) {
  Dual<N> r;
  r.v = fma(a.v, b.v, c.v);
#pragma unroll
  for (int i = 0; i < N; ++i) r.d[i] = fma(a.d[i], b.v, fma(a.v, b.d[i], c.d[i]));
  return r;
}
template <int N>
__device__ __forceinline__ Dual<N> fma_(double a, const Dual<N> &b, const Dual<N> &c) {
  Dual<N> r;
  r.v = fma(a, b.v, c.v);
#pragma unroll
  for (int i = 0; i < N; ++i) r.d[i] = fma(a, b.d[i], c.d[i]);
  return r;
}
template <int N>
__device__ __forceinline__ Dual<N> fma_(const Dual<N> &a, double b, const Dual<N> &c) {
  return fma_(b, a, c);
}
// 1/sqrt(a): derivative -a'/(2 a^{3/2})
template <int N>
__device__ __forceinline__ Dual<N> rsqrt_(const Dual<N> &a) {
  Dual<N> r;
  r.v = rsqrt(a.v);
  const double k = -0.5 * r.v * r.v * r.v;
#pragma unroll
  for (int i = 0; i < N; ++i) r.d[i] = k * a.d[i];
  return r;
}
template <int N>
__device__ __forceinline__ Dual<N> exp_(const Dual<N> &a) {
  Dual<N> r;
  r.v = exp(a.v);
#pragma unroll
  for (int i = 0; i < N; ++i) r.d[i] = r.v * a.d[i];
  return r;
}
template <int N>
__device__ __forceinline__ void sincos_(const Dual<N> &a, Dual<N> &s, Dual<N> &c) {
  double sv, cv;
  sincos(a.v, &sv, &cv);
  s.v = sv;
  c.v = cv;
#pragma unroll
  for (int i = 0; i < N; ++i) {
    s.d[i] = cv * a.d[i];
    c.d[i] = -sv * a.d[i];
  }
}
__device__ __forceinline__ double exp_(double a) { return exp(a); }
__device__ __forceinline__ void sincos_(double a, double &s, double &c) { sincos(a, &s, &c); }

// the value part, for branch decisions and cell indices
__device__ __forceinline__ double val(double a) { return a; }
template <int N>
__device__ __forceinline__ double val(const Dual<N> &a) { return a.v; }

}  // namespace
