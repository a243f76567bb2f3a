// dfloat.cuh -- unevaluated sums of two floats ("double-float", about 48 significant bits)
// for the FP64 pusher's predictor: GB300's FP64 pipe bounds that kernel while its FP32 pipe
// and instruction issue are mostly idle, so a predictor step carried in pairs of FP32 numbers
// (Dekker's and Knuth's error-free transformations: the rounding error of an FP32 sum is
// recovered with two-sum, that of a product with one fused multiply-add) lands within about
// 1e-14 of the FP64 fixed point at FP32-pipe cost. Only start points come from here: every
// result the pusher stores is an FP64 evaluation checked in FP64.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace {

struct DF {
  float hi, lo;  // value hi + lo, |lo| <= ulp(hi) / 2
  DF() = default;
  __host__ __device__ constexpr DF(float h, float l) : hi(h), lo(l) {}
  // from a float or an integer constant (exact for |i| < 2^24)
  __host__ __device__ constexpr DF(float f) : hi(f), lo(0.0f) {}
  __host__ __device__ constexpr DF(int i) : hi((float)i), lo(0.0f) {}
  // from a double: meant for literal constants, which the compiler folds (a runtime double
  // would cost FP64 conversions: df_of splits those on the integer pipe)
  __host__ __device__ constexpr DF(double d) : hi((float)d), lo((float)(d - (double)(float)d)) {}
};

// a double constant as a pair, at compile time (literals only: used for the series
// coefficients)
__host__ __device__ constexpr DF dfc(double x) {
  return DF((float)x, (float)(x - (double)(float)x));
}

// s + e = a + b exactly (Knuth's two-sum)
__device__ __forceinline__ DF two_sum(float a, float b) {
  const float s = a + b, bb = s - a;
  return DF(s, (a - (s - bb)) + (b - bb));
}
// s + e = a + b exactly when |a| >= |b| (or a = 0)
__device__ __forceinline__ DF fast_two_sum(float a, float b) {
  const float s = a + b;
  return DF(s, b - (s - a));
}

__device__ __forceinline__ DF operator+(DF a, DF b) {
  const DF s = two_sum(a.hi, b.hi);
  const DF t = two_sum(a.lo, b.lo);
  const DF u = fast_two_sum(s.hi, s.lo + t.hi);
  return fast_two_sum(u.hi, u.lo + t.lo);
}
__device__ __forceinline__ DF operator-(DF a) { return DF(-a.hi, -a.lo); }
__device__ __forceinline__ DF operator-(DF a, DF b) { return a + (-b); }
__device__ __forceinline__ DF operator*(DF a, DF b) {
  const float p = a.hi * b.hi;
  float e = fmaf(a.hi, b.hi, -p);  // the product's rounding error, exactly
  e = fmaf(a.hi, b.lo, fmaf(a.lo, b.hi, e));
  return fast_two_sum(p, e);
}
__device__ __forceinline__ DF fma_(DF a, DF b, DF c) { return a * b + c; }

// 1/b: the FP32 reciprocal refined by one Newton step in pairs (the error squares: 2^-44)
__device__ __forceinline__ DF df_rcp(DF b) {
  const DF r(__fdividef(1.0f, b.hi));
  const DF e = DF(1.0f) - b * r;
  return r + r * e;
}
__device__ __forceinline__ DF operator/(DF a, DF b) { return a * df_rcp(b); }
// 1/sqrt(x): the FP32 value refined by one Newton step in pairs, r + r (1 - x r^2) / 2
__device__ __forceinline__ DF df_rsqrt(DF x) {
  const DF r(rsqrtf(x.hi));
  const DF e = DF(1.0f) - x * (r * r);
  return r + r * DF(0.5f * e.hi, 0.5f * e.lo);
}
__device__ __forceinline__ DF rsqrt_(DF x) { return df_rsqrt(x); }

// a double split into a pair on the integer pipe: hi its leading 24 bits (truncated), lo
// the next 24 of the remaining 29 (rounded by the integer-to-float conversion), so the pair
// holds the double to about 2^-48 of itself; zero, subnormals, values below about 2^-100 in
// the low part and non-finite values keep only hi (the predictor needs their leading bits
// only)
__device__ __forceinline__ DF df_of(double x) {
  const unsigned hi32 = (unsigned)__double2hiint(x), lo32 = (unsigned)__double2loint(x);
  const unsigned sign = hi32 & 0x80000000u, ex = (hi32 >> 20) & 0x7ffu;
  const int e = (int)ex - 896;  // rebias 1023 -> 127
  float h;
  if (e <= 0) h = __uint_as_float(sign);
  else if (e >= 255) h = __uint_as_float(sign | 0x7f800000u);
  else h = __uint_as_float(sign | ((unsigned)e << 23) | ((hi32 & 0xfffffu) << 3) | (lo32 >> 29));
  float l = 0.0f;
  const int es = (int)ex - 1075 + 127;  // biased FP32 exponent of the low part's unit 2^(ex - 1075)
  if (e > 0 && e < 255 && es >= 1) {
    const unsigned m = lo32 & 0x1fffffffu;  // the 29 bits below hi
    l = (float)m * __uint_as_float((unsigned)es << 23);
    if (sign) l = -l;
  }
  return DF(h, l);
}

}  // namespace
