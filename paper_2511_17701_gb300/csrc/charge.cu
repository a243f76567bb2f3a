// charge.cu -- the charge-conservation check of the deposit (Sec. 3.2, Eq.
// charge-conservation-disc), in FP64 for both precisions: the discrete continuity equation
//   (J^1(i+1/2, j) - J^1(i-1/2, j)) + (J^2(i, j+1/2) - J^2(i, j-1/2))
//       + (rho^{n+1}(i, j) - rho^n(i, j)) / dt = 0
// at every node i in [-1, n_r + 1], j in [0, n_theta], where rho is the charge q w of every
// live massive particle shared over the four nodes of its cell with linear weights, at the
// previous and at the current position. The zigzag deposit satisfies it to rounding. With
// n_f current-filter passes the charge planes get the same passes as the currents.
#include "grpic_internal.cuh"

namespace {

constexpr int TPB_Q = 256;

// rho at the previous and current positions, and the charge magnitude sum |q w| S over both
// (the scale of their rounding: charges of opposite sign cancel in rho, not in rho_abs)
template <typename T>
__global__ void __launch_bounds__(TPB_Q) k_rho(GridP g, SpeciesDevT<T> s, double *rho_prev,
                                              double *rho_new, double *rho_abs) {
  const int64_t n = *s.n;
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n;
       k += (int64_t)gridDim.x * blockDim.x) {
    if (s.tag[k] == 0) continue;
    const double q = s.qc * (double)s.w[k], qa = fabs(q);
    for (int which = 0; which < 2; ++which) {
      const int i = which ? s.i1[k] : s.i1p[k], j = which ? s.i2[k] : s.i2p[k];
      const double w1 = which ? (double)s.dx1[k] : (double)s.dx1p[k];
      const double w2 = which ? (double)s.dx2[k] : (double)s.dx2p[k];
      const double c00 = (1.0 - w1) * (1.0 - w2), c10 = w1 * (1.0 - w2);
      const double c01 = (1.0 - w1) * w2, c11 = w1 * w2;
      const int64_t o = sidx(g, i, j);
      double *r = (which ? rho_new : rho_prev) + o, *ra = rho_abs + o;
      atomicAdd(r, q * c00);
      atomicAdd(r + 1, q * c10);
      atomicAdd(r + g.NX, q * c01);
      atomicAdd(r + g.NX + 1, q * c11);
      atomicAdd(ra, qa * c00);
      atomicAdd(ra + 1, qa * c10);
      atomicAdd(ra + g.NX, qa * c01);
      atomicAdd(ra + g.NX + 1, qa * c11);
    }
  }
}

// max of non-negative doubles through their bit patterns (monotone for v >= 0)
__device__ __forceinline__ void max_pos(double *p, double v) {
  atomicMax(reinterpret_cast<unsigned long long *>(p), (unsigned long long)__double_as_longlong(v));
}

// out[0] = max |residual|, out[1] = max |drho/dt|, out[2] = max |residual| / (|J terms| +
// |drho/dt|), out[3] = max rho_abs / dt over the nodes (the scale of the rounding)
template <typename T>
__global__ void __launch_bounds__(TPB_Q) k_continuity(GridP g, const T *J1, const T *J2,
                                                     const double *rho_prev,
                                                     const double *rho_new,
                                                     const double *rho_abs, double *out) {
  // nodes i in [-1, n_r + 1], j in [0, n_th]; with n_f filter passes the zero fill beyond the
  // stored x1 range (columns -G .. n_r + G) changes values up to n_f - G - 2 columns in from
  // either edge, and the divergence at node i reads column i - 1, so nodes i < n_f - G and
  // i > n_r + G + 1 - n_f are left out
  const int ilo = max(-1, g.n_f - G_);
  const int ihi = min(g.n_r + 1, g.n_r + G_ + 1 - g.n_f);
  const int ni = ihi - ilo + 1, nj = g.n_th + 1;
  double m0 = 0.0, m1 = 0.0, m2 = 0.0, m3 = 0.0;
  const double idt = 1.0 / g.dt;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < (int64_t)ni * nj;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(t % ni) + ilo, j = (int)(t / ni);
    const int64_t k = sidx(g, i, j);
    const double a = (double)J1[k], b = (double)J1[k - 1];
    const double c = (double)J2[k], d = (double)J2[k - g.NX];
    const double dr = (rho_new[k] - rho_prev[k]) * idt;
    const double res = fabs((a - b) + (c - d) + dr);
    const double sc = fabs(a) + fabs(b) + fabs(c) + fabs(d) + fabs(dr);
    m0 = fmax(m0, res);
    m1 = fmax(m1, fabs(dr));
    if (sc > 0.0) m2 = fmax(m2, res / sc);
    m3 = fmax(m3, rho_abs[k] * idt);
  }
  for (int o = 16; o > 0; o >>= 1) {
    m0 = fmax(m0, __shfl_xor_sync(0xffffffffu, m0, o));
    m1 = fmax(m1, __shfl_xor_sync(0xffffffffu, m1, o));
    m2 = fmax(m2, __shfl_xor_sync(0xffffffffu, m2, o));
    m3 = fmax(m3, __shfl_xor_sync(0xffffffffu, m3, o));
  }
  if ((threadIdx.x & 31) == 0) {
    max_pos(out, m0);
    max_pos(out + 1, m1);
    max_pos(out + 2, m2);
    max_pos(out + 3, m3);
  }
}

}  // namespace

template <typename T>
cudaError_t launch_charge_rho(const GridP &g, SpeciesDevT<T> s, int64_t n_bound,
                              double *rho_prev, double *rho_new, double *rho_abs,
                              cudaStream_t st) {
  if (n_bound <= 0) return cudaGetLastError();
  int64_t b = (n_bound + TPB_Q - 1) / TPB_Q;
  if (b > 152 * 32) b = 152 * 32;
  k_rho<T><<<(int)b, TPB_Q, 0, st>>>(g, s, rho_prev, rho_new, rho_abs);
  COUNT_LAUNCH(1);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_continuity(const GridP &g, const T *J1, const T *J2, const double *rho_prev,
                              const double *rho_new, const double *rho_abs, double *out,
                              cudaStream_t st) {
  cudaError_t e = cudaMemsetAsync(out, 0, 4 * sizeof(double), st);
  if (e != cudaSuccess) return e;
  const int64_t nodes = (int64_t)(g.n_r + 3) * (g.n_th + 1);
  int64_t b = (nodes + TPB_Q - 1) / TPB_Q;
  if (b > 152 * 8) b = 152 * 8;
  k_continuity<T><<<(int)b, TPB_Q, 0, st>>>(g, J1, J2, rho_prev, rho_new, rho_abs, out);
  COUNT_LAUNCH(1);
  return cudaGetLastError();
}

#define INSTANTIATE_CHARGE(T)                                                                  \
  template cudaError_t launch_charge_rho<T>(const GridP &, SpeciesDevT<T>, int64_t, double *,   \
                                            double *, double *, cudaStream_t);                  \
  template cudaError_t launch_continuity<T>(const GridP &, const T *, const T *,               \
                                            const double *, const double *, const double *,     \
                                            double *, cudaStream_t);
INSTANTIATE_CHARGE(double)
INSTANTIATE_CHARGE(float)
