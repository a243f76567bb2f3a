// sum.cu -- exact, order-independent sums of doubles (no counterpart in the paper). The
// adjoint's gradient with respect to the field amplitude is a sum over particles; when the
// particles are split across GPUs these sums make it the same bits for every split.
//
// A finite double v is M 2^(b - 1075) with b its biased exponent field (b = 1 for
// subnormals, which carry no implicit bit) and M a signed integer, |M| < 2^53. Per b the bins
// hold the int64 sums of M's high part (M >> 32, arithmetic) and low part (M & 0xffffffff),
// so adding values, or adding bins element by element (an all-reduce of int64 sums across
// processes), is exact integer arithmetic whose result does not depend on the order. The
// host routine rounds the binned total to the nearest double (ties to even) once.
#include <stdint.h>
#include <string.h>

#include <cmath>

#include "grpic_internal.cuh"

namespace {

constexpr int NB = GRPIC_SUM_BINS;
constexpr int SUM_TPB = 256;

__global__ void __launch_bounds__(SUM_TPB) k_sum_bins(const double *__restrict__ x, int64_t n,
                                                      unsigned long long *bins) {
  __shared__ unsigned long long sb[2 * NB];  // 32 KB
  for (int t = threadIdx.x; t < 2 * NB; t += blockDim.x) sb[t] = 0ull;
  __syncthreads();
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n;
       k += (int64_t)gridDim.x * blockDim.x) {
    const unsigned long long u = (unsigned long long)__double_as_longlong(x[k]);
    const int b = (int)((u >> 52) & 0x7ff);
    if (b == 0x7ff) continue;  // inf and NaN carry nothing
    const long long f = (long long)(u & ((1ull << 52) - 1));
    long long M = b ? (f | (1ll << 52)) : f;
    if (u >> 63) M = -M;
    const long long hi = M >> 32;                 // arithmetic shift: floor(M / 2^32)
    const long long lo = M - (hi << 32);          // in [0, 2^32)
    const int bb = b ? b : 1;
    // two's complement: unsigned addition of the bit patterns is signed addition
    if (hi) atomicAdd(&sb[2 * bb], (unsigned long long)hi);
    if (lo) atomicAdd(&sb[2 * bb + 1], (unsigned long long)lo);
  }
  __syncthreads();
  for (int t = threadIdx.x; t < 2 * NB; t += blockDim.x)
    if (sb[t]) atomicAdd(&bins[t], sb[t]);
}

}  // namespace

extern "C" GRPIC_API grpic_status grpic_sum_bins_add(const double *x, int64_t n, int64_t *bins,
                                                     void *stream) {
  if (n < 0 || !bins || (n > 0 && !x)) return GRPIC_EINVAL;
  if (cudaPeekAtLastError() != cudaSuccess) return GRPIC_ECUDA;  // not this call's error
  if (n == 0) return GRPIC_OK;
  int64_t blocks = (n + SUM_TPB - 1) / SUM_TPB;
  if (blocks > 4 * 152) blocks = 4 * 152;
  k_sum_bins<<<(int)blocks, SUM_TPB, 0, static_cast<cudaStream_t>(stream)>>>(
      x, n, reinterpret_cast<unsigned long long *>(bins));
  COUNT_LAUNCH(1);
  return cudaGetLastError() == cudaSuccess ? GRPIC_OK : GRPIC_ECUDA;
}

// Host: the binned total as a fixed-point integer of 32-bit digits (digit i weighs
// 2^(32 i - 1074)), normalised, then rounded to 53 significant bits.
extern "C" GRPIC_API grpic_status grpic_sum_bins_value(const int64_t *bins, double *out) {
  if (!bins || !out) return GRPIC_EINVAL;
  // bits: bin b's term (H 2^32 + L) 2^(b - 1) above 2^-1074, |H| < 2^52 and L < 2^63 for at
  // most 2^31 values, so below 2^(2046 + 86); a few digits more for the carries and sign
  constexpr int ND = (2047 + 96) / 32 + 4;
  int64_t d[ND];
  memset(d, 0, sizeof(d));
  for (int b = 1; b < NB; ++b) {
    const int64_t H = bins[2 * b], L = bins[2 * b + 1];
    if (!H && !L) continue;
    if (H > ((int64_t)1 << 52) || H < -((int64_t)1 << 52) || L < 0) return GRPIC_EINVAL;
    const int p = b - 1, q = p / 32, r = p % 32;
    // (H 2^32 + L) 2^r as 32-bit digits from position q: L 2^r spans up to three digits,
    // H 2^(32 + r) up to three digits from q + 1
    const unsigned __int128 lr = (unsigned __int128)(uint64_t)L << r;
    for (int k = 0; k < 3; ++k) d[q + k] += (int64_t)((uint64_t)(lr >> (32 * k)) & 0xffffffffu);
    const __int128 hr = (__int128)H * ((__int128)1 << r);  // signed, |hr| < 2^84
    const bool neg = hr < 0;
    unsigned __int128 mag = neg ? (unsigned __int128)(-hr) : (unsigned __int128)hr;
    for (int k = 0; k < 3; ++k) {
      const int64_t dig = (int64_t)((uint64_t)(mag >> (32 * k)) & 0xffffffffu);
      d[q + 1 + k] += neg ? -dig : dig;
    }
  }
  // carries: every digit to [0, 2^32), the sign left in the top digit
  for (int i = 0; i < ND - 1; ++i) {
    const int64_t c = d[i] >> 32;  // floor division by 2^32
    d[i] -= c * ((int64_t)1 << 32);
    d[i + 1] += c;
  }
  const bool negative = d[ND - 1] < 0;
  if (negative) {  // magnitude: two's complement of the digit string
    int64_t carry = 1;
    for (int i = 0; i < ND; ++i) {
      int64_t v = (~d[i] & 0xffffffffll) + carry;
      carry = v >> 32;
      d[i] = v & 0xffffffffll;
    }
  }
  int top = -1;  // highest set bit
  for (int i = ND - 1; i >= 0 && top < 0; --i)
    if (d[i]) {
      int h = 31;
      while (!((d[i] >> h) & 1)) --h;
      top = 32 * i + h;
    }
  auto bit = [&](int k) -> uint64_t { return k < 0 ? 0 : (uint64_t)((d[k / 32] >> (k % 32)) & 1); };
  double v = 0.0;
  if (top >= 0) {
    if (top <= 52) {  // below 2^53 units of 2^-1074: exact (subnormal or the smallest normals)
      uint64_t m = 0;
      for (int k = top; k >= 0; --k) m = (m << 1) | bit(k);
      v = std::ldexp((double)m, -1074);
    } else {
      uint64_t m = 0;
      for (int k = top; k >= top - 52; --k) m = (m << 1) | bit(k);
      const uint64_t guard = bit(top - 53);
      bool sticky = false;
      for (int k = top - 54; k >= 0 && !sticky; --k) sticky = bit(k) != 0;
      int e = top - 52;
      if (guard && (sticky || (m & 1))) {
        if (++m == ((uint64_t)1 << 53)) {
          m >>= 1;
          ++e;
        }
      }
      v = std::ldexp((double)m, e - 1074);
    }
  }
  *out = negative ? -v : v;
  return GRPIC_OK;
}
