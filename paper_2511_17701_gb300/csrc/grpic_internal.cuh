// grpic_internal.cuh -- device helpers and kernel launch interfaces shared by the
// translation units of libgrpic (not installed, not part of the C ABI).
//
// Geometry follows Appendix A of arXiv:2511.17701 in code units: the quasi-spherical
// Kerr-Schild map r = r0 + exp(xi), xi = log(r_min - r0) + x1 dxi, theta = eta +
// 2 h0 eta (pi - 2 eta)(pi - eta) / pi^2 with eta = x2 deta (deta = pi / n_theta, called dth
// here), dphi = 1; r0 = h0 = 0 is the plain log-r grid with uniform theta. Mass M = 1
// (Kerr-Schild) or M = 0 and a = 0 (kerr_schild_0, flat).
#pragma once
#include <cuda.h>  // CUtensorMap (the tensor-map descriptor of the TMA-staged tiled push)
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/grpic.h"

#define G_ GRPIC_GHOSTS
#define GRPIC_PI 3.14159265358979323846

// Grid and step parameters passed by value to every kernel.
struct GridP {
  int n_r, n_th, NX, NY, n_iter, n_f;
  int stop_on_repeat;  // stop an implicit iteration once its iterate repeats exactly
  double iter_tol;     // > 0: FP64 implicit iterations start from an FP32 predictor and stop
                       // once the update is at most iter_tol max(1, |value|)
  double r_min, r_max, dxi, dth, a, M, dt, small_angle, r_absorb, absorb_coef;
  double idt;       // 1 / dt
  double pi_small;  // pi - small_angle
  double a2, M2;    // a^2 and 2 M
  // the same constants as pairs of floats (value hi + lo, about 48 bits) for the FP64
  // pusher's double-float predictor: a, M, dxi, dth, 1/dth^2, dt, a^2, 2M
  float d_a[2], d_M[2], d_dxi[2], d_dth[2], d_ig2[2], d_dt[2], d_a2[2], d_M2[2], d_r0[2],
      d_c3[2];
  double ig2;  // 1 / dth^2
  // quasi-spherical map: radial offset, equatorial concentration, qks = (r0 != 0 || h0 != 0),
  // c3 = 4 h0 / pi^2 (the cubic coefficient of theta(eta_j + d) - theta(eta_j))
  double r0, h0, c3;
  double e_min;  // r_min - r0 = exp(xi) at x1 = 0
  int qks;
  // FP32 copies for the mixed path (read from the kernel parameters, no conversions)
  float f_a, f_M, f_dxi, f_dth, f_ig2, f_dt, f_idt, f_r0, f_c3, f_iter_tol, f_a2, f_M2;
  // cells of x1 over which the coordinate velocities vary by order one: 1 / (4 dxi)
  float f_x1_scale;
};

// Fill the FP32 copies once a, M, dxi, dth and dt are set.
inline void grid_float_copies(GridP &g) {
  g.idt = g.dt > 0.0 ? 1.0 / g.dt : 0.0;
  g.pi_small = GRPIC_PI - g.small_angle;
  g.a2 = g.a * g.a;
  g.M2 = 2.0 * g.M;
  g.f_a2 = g.f_a * g.f_a;
  g.f_M2 = 2.0f * g.f_M;
  const double dv[10] = {g.a, g.M, g.dxi, g.dth, g.ig2, g.dt, g.a2, g.M2, g.r0, g.c3};
  float *dp[10] = {g.d_a, g.d_M, g.d_dxi, g.d_dth, g.d_ig2, g.d_dt, g.d_a2, g.d_M2, g.d_r0, g.d_c3};
  for (int k = 0; k < 10; ++k) {
    dp[k][0] = (float)dv[k];
    dp[k][1] = (float)(dv[k] - (double)dp[k][0]);
  }
  g.f_iter_tol = (float)g.iter_tol;
  g.f_a = (float)g.a; g.f_M = (float)g.M; g.f_dxi = (float)g.dxi; g.f_dth = (float)g.dth;
  g.f_ig2 = (float)g.ig2; g.f_dt = (float)g.dt; g.f_idt = g.dt > 0.0 ? (float)(1.0 / g.dt) : 0.0f;
  g.f_r0 = (float)g.r0; g.f_c3 = (float)g.c3;
  g.f_x1_scale = g.dxi > 0.0 ? (float)(0.25 / g.dxi) : 1.0f;
}

// The quasi-spherical map at a point (App. A): r with e = exp(xi) = r - r0 and f = dr/dx1 =
// dxi e; theta, g = dtheta/dx2 and gp = dg/dx2. theta is formed in the operation order of
// the plain definition, each operation rounded (no contraction): near theta = pi sin(theta)
// is ill-conditioned in theta and every other rounding of it shows at ~1e-13.
__host__ __device__ inline double map_e(const GridP &g, double x1) {
  return g.e_min * exp(x1 * g.dxi);
}
// Q = false: the plain grid is known at compile time (the hot kernels' instantiation for
// it); Q = true decides at run time
template <bool Q = true>
__device__ __forceinline__ double map_theta(const GridP &g, double x2) {
  const double eta = __dmul_rn(x2, g.dth);
  if (!(Q && g.qks)) return eta;
  const double q = __dmul_rn(__dmul_rn(__dmul_rn(__dmul_rn(2.0, g.h0), eta),
                                       __dadd_rn(GRPIC_PI, -__dmul_rn(2.0, eta))),
                             __dadd_rn(GRPIC_PI, -eta));
  return __dadd_rn(eta, __ddiv_rn(q, __dmul_rn(GRPIC_PI, GRPIC_PI)));
}
// g = deta (1 + 2 h0 + 12 h0 (eta/pi)(eta/pi - 1)), gp = deta^2 12 h0 (2 eta/pi^2 - 1/pi)
template <bool Q = true>
__device__ __forceinline__ void map_g(const GridP &g, double x2, double &gg, double &gp) {
  if (!(Q && g.qks)) {
    gg = g.dth;
    gp = 0.0;
    return;
  }
  constexpr double inv_pi = 1.0 / GRPIC_PI;  // multiplications only: no FP64 division
  const double eta = x2 * g.dth, u = eta * inv_pi;
  gg = g.dth * (1.0 + 2.0 * g.h0 + 12.0 * g.h0 * u * (u - 1.0));
  gp = g.dth * g.dth * 12.0 * g.h0 * (2.0 * u - 1.0) * inv_pi;
}

// The grid constants in the arithmetic type R.
// (a2 = a a and M2 = 2 M, rounded as the products the metric would form)
template <typename R>
struct Cst {
  R a, M, dxi, dth, ig2, dt, a2, M2;
};
template <typename R>
__device__ __forceinline__ Cst<R> cst(const GridP &g) {  // other arithmetic types (duals)
  return {R(g.a), R(g.M), R(g.dxi), R(g.dth), R(g.ig2), R(g.dt), R(g.a2), R(g.M2)};
}
template <>
__device__ __forceinline__ Cst<double> cst<double>(const GridP &g) {
  return {g.a, g.M, g.dxi, g.dth, g.ig2, g.dt, g.a2, g.M2};
}
template <>
__device__ __forceinline__ Cst<float> cst<float>(const GridP &g) {
  return {g.f_a, g.f_M, g.f_dxi, g.f_dth, g.f_ig2, g.f_dt, g.f_a2, g.f_M2};
}

// Yee point classes of the metric tables: (i, j), (i+1/2, j), (i, j+1/2), (i+1/2, j+1/2).
enum { CLS_NN = 0, CLS_HN = 1, CLS_NH = 2, CLS_HH = 3 };
// Quantities tabulated per class (Eq. discretized-auxE/auxH and the curls).
enum { T_ALPHA = 0, T_H11, T_H22, T_H33, T_IHT2, T_WT13, T_WB1, T_ISH, T_NQ };

__host__ __device__ inline int64_t plane_size(const GridP &g) { return (int64_t)g.NX * g.NY; }
__host__ __device__ inline int64_t sidx(const GridP &g, int i, int j) {
  return (int64_t)(j + G_) * g.NX + (i + G_);
}

// Device view of one species' arrays; T is double (FP64 path) or float (mixed path).
template <typename T>
struct SpeciesDevT {
  int32_t *i1, *i2;
  T *dx1, *dx2, *u1, *u2, *u3, *phi, *w;
  uint8_t *tag;
  int32_t *i1p, *i2p;
  T *dx1p, *dx2p;
  const int64_t *n;  // live count, on the device
  double qm, qc;
  float f_qm, f_qc;  // FP32 copies
  // mass term of gamma = sqrt(m2 + h^ij u_i u_j) (Sec. 2.3): 1 for massive particles, 0 for
  // massless ones, which skip the EM push (Sec. 3.1) and, being neutral, deposit nothing
  double m2;
  float f_m2;
};
using SpeciesDev = SpeciesDevT<double>;

// Diagnostics counters on the device (unsigned long long for atomicAdd).
enum { DG_LEFT_INNER = 0, DG_LEFT_OUTER, DG_REFLECT, DG_NONFINITE, DG_INJECTED,
       DG_INJECT_DROPPED, DG_STAGE_TIMEOUT, DG_N };

// ---------------------------------------------------------------------------------
// Metric of Appendix A, written directly in the code-unit (xi, eta) form of the
// quasi-spherical Kerr-Schild section, with the mass M kept explicit.
// ---------------------------------------------------------------------------------
struct MetricV {
  double h11, h22, h33, h13, H11, H22, H33, H13, alpha, beta1, sqrt_h, sqrt_ht;
};
struct MetricD {
  double d1H11, d1H22, d1H33, d1H13, d1alpha, d1beta1;
  double d2H11, d2H22, d2H33, d2H13, d2alpha, d2beta1;
};

template <bool DERIV>
__device__ __forceinline__ void metric_eval(const GridP &g, double x1, double x2, bool clamp,
                                            MetricV &m, MetricD *d) {
  const double a = g.a, M = g.M, a2 = a * a;
  const double e = map_e(g, x1), r = g.r0 + e;
  double th = map_theta(g, x2);
  if (clamp) th = fmin(fmax(th, g.small_angle), GRPIC_PI - g.small_angle);
  double gg, gp;
  map_g(g, x2, gg, gp);
  double s, c;
  sincos(th, &s, &c);
  const double s2 = s * s, r2 = r * r;
  const double Sig = r2 + a2 * c * c;
  const double Del = r2 - 2.0 * M * r + a2;
  const double A = (r2 + a2) * (r2 + a2) - a2 * Del * s2;
  const double iSig = 1.0 / Sig;
  const double z = 2.0 * M * r * iSig;
  const double al2 = 1.0 / (1.0 + z);          // alpha^2 = 1/(1+z)
  const double f = g.dxi * e, fi = 1.0 / f;     // d xi e^xi and its inverse
  m.alpha = sqrt(al2);
  m.h11 = f * f * (1.0 + z);
  m.h13 = -f * a * (1.0 + z) * s2;
  m.h22 = gg * gg * Sig;
  m.h33 = A * s2 * iSig;
  m.H11 = A * iSig * iSig * al2 * fi * fi;      // A / (Sigma (Sigma + 2 M r)) / f^2
  m.H13 = a * iSig * fi;
  m.H22 = iSig / (gg * gg);
  m.H33 = iSig / s2;
  m.beta1 = z * al2 * fi;
  m.sqrt_ht = f * gg * Sig / m.alpha;
  m.sqrt_h = m.sqrt_ht * s;
  if (DERIV) {
    const double dxS = 2.0 * r * f, deS = -2.0 * a2 * s * c * gg;
    const double dxD = 2.0 * (r - M) * f;
    const double dxA = 4.0 * r * f * (r2 + a2) - a2 * s2 * dxD;
    const double deA = -2.0 * a2 * s * c * Del * gg;
    const double P = Sig * Sig * (1.0 + z);     // Sigma (Sigma + 2 M r)
    const double iP2 = 1.0 / (P * P);
    const double iS2 = iSig * iSig;
    const double al3 = m.alpha * al2;
    d->d1H11 = (P * dxA - 2.0 * A * (M * r * dxS + Sig * (dxS + M * f))) * iP2 * fi * fi -
               2.0 * g.dxi * m.H11;
    d->d2H11 = (P * deA - 2.0 * A * deS * (M * r + Sig)) * iP2 * fi * fi;
    d->d1H22 = -dxS * iS2 / (gg * gg);
    d->d2H22 = -deS * iS2 / (gg * gg) - 2.0 * m.H22 * gp / gg;  // dg/dx2 = gp (h0 != 0)
    d->d1H33 = -dxS * iS2 / s2;
    d->d2H33 = -(deS + 2.0 * (c / s) * Sig * gg) * iS2 / s2;
    d->d1H13 = -a * iS2 * dxS * fi - g.dxi * a * iSig * fi;
    d->d2H13 = -a * iS2 * deS * fi;
    d->d1alpha = -M * (f * Sig - r * dxS) * iS2 * al3;
    d->d2alpha = M * r * deS * iS2 * al3;
    d->d1beta1 = fi * 2.0 * M * (f * Sig - r * dxS) * iS2 * al2 * al2 - g.dxi * m.beta1;
    d->d2beta1 = -fi * 2.0 * M * r * deS * iS2 * al2 * al2;
  }
}

// ---------------------------------------------------------------------------------
// Stationary potentials: Wald (Eq. Wald) and its zero-spin limit, and their
// derivatives in code coordinates, written from the physical (r, theta) closed forms.
// ---------------------------------------------------------------------------------
struct Pot {
  double A0, A1, A3;              // A_0, A_1 (code), A_3
  double d1A0, d2A0, d1A3, d2A1;  // the derivatives the fields need
};

__device__ __forceinline__ void potential(const GridP &g, int kind, double B0, double x1, double x2, bool derivs,
                          Pot &p) {
  const double a = g.a, M = g.M, a2 = a * a;
  const double e = map_e(g, x1), r = g.r0 + e, th = map_theta(g, x2);
  double s, c;
  sincos(th, &s, &c);
  double gg, gp;
  map_g(g, x2, gg, gp);
  const double s2 = s * s, f = g.dxi * e;
  if (kind == GRPIC_FIELD_VERTICAL) {
    p.A0 = 0.0; p.A1 = 0.0; p.A3 = 0.5 * B0 * r * r * s2;
    p.d1A0 = p.d2A0 = p.d2A1 = 0.0;
    p.d1A3 = f * B0 * r * s2;
    return;
  }
  if (kind == GRPIC_FIELD_MONOPOLE) {  // A_phi = -B0 cos(theta), Sec. 4.5
    p.A0 = 0.0; p.A1 = 0.0; p.A3 = -B0 * c;
    p.d1A0 = p.d2A0 = p.d2A1 = 0.0;
    p.d1A3 = 0.0;
    return;
  }
  const double Sig = r * r + a2 * c * c, Del = r * r - 2.0 * M * r + a2;
  const double A = (r * r + a2) * (r * r + a2) - a2 * Del * s2;
  const double z = 2.0 * M * r / Sig;
  // physical Wald potential: A_t = (B0 a / 2)(z (2 - s^2) - 2), A_r = (B0 a / 2)(2 z - (1+z) s^2),
  // A_phi = (B0 / 2)(A s^2 / Sigma - 2 a^2 z s^2)
  const double hb = 0.5 * B0;
  p.A0 = hb * a * (z * (2.0 - s2) - 2.0);
  p.A1 = f * hb * a * (2.0 * z - (1.0 + z) * s2);
  p.A3 = hb * (A * s2 / Sig - 2.0 * a2 * z * s2);
  if (!derivs) return;
  const double drS = 2.0 * r, dtS = -2.0 * a2 * s * c;
  const double drz = 2.0 * M * (Sig - r * drS) / (Sig * Sig);
  const double dtz = -2.0 * M * r * dtS / (Sig * Sig);
  const double drA = 4.0 * r * (r * r + a2) - a2 * s2 * (2.0 * r - 2.0 * M);
  const double dts2 = 2.0 * s * c;
  p.d1A0 = f * hb * a * drz * (2.0 - s2);
  p.d2A0 = gg * hb * a * (dtz * (2.0 - s2) - z * dts2);
  p.d1A3 = f * hb * (s2 * (drA * Sig - A * drS) / (Sig * Sig) - 2.0 * a2 * s2 * drz);
  p.d2A1 = gg * f * hb * a * (2.0 * dtz - dtz * s2 - (1.0 + z) * dts2);
}

// Tetrad maps of Appendix A (matrix form).
__device__ __forceinline__ void t_vec_to_hat(const MetricV &m, const double A[3], double Ah[3]) {
  const double s11 = sqrt(m.H11), s33 = sqrt(m.h33);
  Ah[0] = A[0] / s11;
  Ah[1] = sqrt(m.h22) * A[1];
  Ah[2] = m.h13 / s33 * A[0] + s33 * A[2];
}
__device__ __forceinline__ void t_cov_to_hat(const MetricV &m, const double a[3], double ah[3]) {
  const double s11 = sqrt(m.H11);
  ah[0] = s11 * (a[0] - m.h13 / m.h33 * a[2]);
  ah[1] = a[1] / sqrt(m.h22);
  ah[2] = a[2] / sqrt(m.h33);
}
__device__ __forceinline__ void t_hat_to_cov(const MetricV &m, const double ah[3], double a[3]) {
  const double s33 = sqrt(m.h33);
  a[0] = ah[0] / sqrt(m.H11) + m.h13 / s33 * ah[2];
  a[1] = sqrt(m.h22) * ah[1];
  a[2] = s33 * ah[2];
}

// gamma = sqrt(m2 + h^ij u_i u_j), m2 = 1 (massive) or 0 (massless), Sec. 2.3
__device__ __forceinline__ double gamma_of(const MetricV &m, const double u[3], double m2) {
  return sqrt(m2 + m.H11 * u[0] * u[0] + m.H22 * u[1] * u[1] + m.H33 * u[2] * u[2] +
              2.0 * m.H13 * u[0] * u[2]);
}

// Boris step over coordinate time dt/2 in the tetrad frame, hq = qm alpha dt / 2.
__device__ __forceinline__ void boris_step(double u[3], const double D[3], const double B[3],
                                           double hq) {
  const double e = 0.5 * hq;
  const double m0 = u[0] + e * D[0], m1 = u[1] + e * D[1], m2 = u[2] + e * D[2];
  const double ig = rsqrt(1.0 + m0 * m0 + m1 * m1 + m2 * m2);
  const double t0 = e * B[0] * ig, t1 = e * B[1] * ig, t2 = e * B[2] * ig;
  const double sf = 2.0 / (1.0 + t0 * t0 + t1 * t1 + t2 * t2);
  const double p0 = m0 + (m1 * t2 - m2 * t1);
  const double p1 = m1 + (m2 * t0 - m0 * t2);
  const double p2 = m2 + (m0 * t1 - m1 * t0);
  u[0] = m0 + sf * (p1 * t2 - p2 * t1) + e * D[0];
  u[1] = m1 + sf * (p2 * t0 - p0 * t2) + e * D[1];
  u[2] = m2 + sf * (p0 * t1 - p1 * t0) + e * D[2];
}

// Bilinear interpolation of a plane at code position (x1, x2) for a component whose Yee
// location is offset by (s1, s2); ghost rows across the axes hold the mirrored values.
__device__ __forceinline__ double interp_plane(const double *__restrict__ pl, int NX, double x1,
                                               double x2, double s1, double s2) {
  const double y1 = x1 - s1, y2 = x2 - s2;
  const double f1 = floor(y1), f2 = floor(y2);
  const int i0 = (int)f1, j0 = (int)f2;
  const double w1 = y1 - f1, w2 = y2 - f2;
  const double *p = pl + (int64_t)(j0 + G_) * NX + (i0 + G_);
  return (1.0 - w1) * (1.0 - w2) * __ldg(p) + w1 * (1.0 - w2) * __ldg(p + 1) +
         (1.0 - w1) * w2 * __ldg(p + NX) + w1 * w2 * __ldg(p + NX + 1);
}

// Kernels launched by the library (host counter, reset by grpic_get_timing).
extern long long grpic_launches;
#define COUNT_LAUNCH(n) (grpic_launches += (n))

// ---------------------------------------------------------------------------------
// Launchers (host functions defined in fields.cu, particles.cu, sort.cu).
// Every launcher returns cudaGetLastError() of its launches.
// ---------------------------------------------------------------------------------
template <typename T>
struct FieldPtrsT {
  T *B[3], *D[3], *B0[3], *D0[3], *J[3], *J0[3], *Bn[3], *Bi[3], *Di[3];
  T *E[3], *H[3], *Dh[3];
  const T *tab;    // [4 classes][T_NQ][plane]
  const T *polar;  // [3][NX]: the polar area at x1 = i + 1/2, then the absorber factor
                   // absorb_coef x^3 at x1 = i and at x1 = i + 1/2 (stored at i)
};
using FieldPtrs = FieldPtrsT<double>;

// Per-cell tables of the FP32 pusher (mixed precision), computed in FP64: r at x1 = i,
// sin and cos of theta at x2 = j, for stored i, j.
struct PushTables {
  const float *r, *s, *c;           // e = r - r0 at cell corners i, sin/cos(theta) at corners j
  const double *r64, *s64, *c64;    // the same in FP64, for the guard zones
  // quasi-spherical theta: per corner row j, theta(eta_j + d) - theta(eta_j) =
  // d (t1_j + d (t2_j + d c3)) for an offset d in eta (t1 = dtheta/deta, t2 = its half
  // derivative); 1 and 0 on the plain grid
  const float *t1, *t2;
  const double *t1_64, *t2_64;
  const double *th64;  // theta at corner row j, formed as map_theta forms it
  // exp(xi) at corner column i and sin, cos(theta) at corner row j as float pairs (hi, lo)
  const float2 *r_df, *s_df, *c_df;
  const float2 *t1_df, *t2_df;  // the quasi-spherical theta offset's t1, t2 as pairs
  int guard_ilo, guard_ihi;  // cells guard_ilo <= i1 < guard_ihi (around the horizon) and
  int guard_j;               // within guard_j of an axis evaluate the metric in FP64
};

// The guard particles of one species for the current push (mixed path): zone 1 (FP64
// metric) indices ascending from idx[0], zone 2 (the cell rows on the axes, FP64 routine)
// descending from idx[cap - 1], counted in count[0], count[1]; bit k of mask marks particle
// k as listed (written only by the classification, read by the FP32 kernel).
struct GuardList {
  uint32_t *idx;
  uint32_t *mask;
  int64_t cap;
  unsigned long long *count;
};

// The particle range of every sort tile (mixed path): particles tile_start[t] ..
// tile_start[t+1] - 1 were in tile t at the last sort (start is null when no sort has run
// since the particles were last set, and the push does not use tiles).
// tma: the window comes from `pad` (the 6 planes B^n, D with rows padded to NXp floats, a
// multiple of 4) by the tensor copies of `map` (a 3D map over [6][NY][NXp] with a box of
// one window plane); the kernel takes it as a __grid_constant__ parameter.
struct TileInfo {
  CUtensorMap map;
  const uint32_t *start;
  float *pad;
  int tr, tt, ntr, n_tiles, tma, NXp;
};
constexpr int TILE_HALO = 6;  // cells of the window beyond the tile on every side

// Streams of one push: the classification and the FP64-pipe-bound guard kernels run on
// `side`, forked from `main` by `fork`; `done` is recorded on `side` after them and the
// caller makes `main` wait on it before anything reads the currents or the particles.
// which part of a push to launch: the mixed path's guard stage (classify, then the FP64
// guard kernels, all on `side`) and its main FP32 kernel (on `main`, after the classify) can
// be issued separately, so that the guard stages of all species start before the first FP32
// kernel
// stages of a mixed push: PUSH_GUARD = PUSH_CLASSIFY then PUSH_GUARD_KERNELS (side stream),
// PUSH_MAIN the FP32 kernel; PUSH_ALL all of them (the FP64 path has the main stage only)
enum { PUSH_ALL = 0, PUSH_GUARD = 1, PUSH_MAIN = 2, PUSH_CLASSIFY = 3, PUSH_GUARD_KERNELS = 4 };
__host__ __device__ inline bool push_main_stage(int s) { return s == PUSH_ALL || s == PUSH_MAIN; }
__host__ __device__ inline bool push_classify_stage(int s) {
  return s == PUSH_ALL || s == PUSH_GUARD || s == PUSH_CLASSIFY;
}
__host__ __device__ inline bool push_guard_kernels_stage(int s) {
  return s == PUSH_ALL || s == PUSH_GUARD || s == PUSH_GUARD_KERNELS;
}
struct PushStreams {
  cudaStream_t main, side;
  cudaEvent_t fork, done, classified;  // side after main; guard kernels done; classify done
  cudaEvent_t t0, t1;  // when not null: recorded on `main` around the main push kernel
  int stage = PUSH_ALL;
};

template <typename T>
cudaError_t launch_metric_tables(const GridP &g, T *tab, T *polar, cudaStream_t st);
cudaError_t launch_dt_min(const GridP &g, double *scratch, int nscratch, double *out,
                          cudaStream_t st);
template <typename T>
cudaError_t launch_init_fields(const GridP &g, const FieldPtrsT<T> &F, int kind, double B0,
                               cudaStream_t st);
template <typename T>
cudaError_t launch_field_finish_init(const GridP &g, const FieldPtrsT<T> &F, int user,
                                     cudaStream_t st);
template <typename T>
cudaError_t launch_predict(const GridP &g, const FieldPtrsT<T> &F, cudaStream_t st);
template <typename T>
cudaError_t launch_advance(const GridP &g, const FieldPtrsT<T> &F, cudaStream_t st);
template <typename T>
cudaError_t launch_aux_fields(const GridP &g, const FieldPtrsT<T> &F, cudaStream_t st);
// current filter (filter.cu): n passes on n_comp planes a (scratch s; in_s: see filter.cu),
// and the n_f passes on J (may trade the J and E plane pointers of F)
template <typename T>
cudaError_t launch_filter(const GridP &g, T *const a[3], T *const s[3], const int half[3],
                          const double parity[3], int n_comp, int n, cudaStream_t st,
                          bool *in_s);
template <typename T>
cudaError_t launch_filter_currents(const GridP &g, FieldPtrsT<T> &F, cudaStream_t st);
// pair injection (inject.cu): scratch bytes it needs, its cell-centre metric table (once per
// grid), and the launch
size_t inject_scratch_bytes(const GridP &g);
cudaError_t launch_inject_tables(const GridP &g, unsigned char *scratch, cudaStream_t st);
template <typename T>
cudaError_t launch_inject(const GridP &g, const FieldPtrsT<T> &F, SpeciesDevT<T> se,
                          SpeciesDevT<T> sp, int64_t n_bound_e, int64_t n_bound_p,
                          int64_t cap_e, int64_t cap_p, double sigma0, double sigma_th,
                          double B0, const double *pool, int64_t pool_n, int64_t pool_offset,
                          unsigned char *scratch, unsigned long long *diag, cudaStream_t st);
template <typename T>
cudaError_t launch_zero(T *p, int64_t n, cudaStream_t st);

cudaError_t launch_push_tables(const GridP &g, const PushTables &tb, cudaStream_t st);
template <typename T>
cudaError_t launch_charge_rho(const GridP &g, SpeciesDevT<T> s, int64_t n_bound,
                              double *rho_prev, double *rho_new, double *rho_abs,
                              cudaStream_t st);
template <typename T>
cudaError_t launch_continuity(const GridP &g, const T *J1, const T *J2, const double *rho_prev,
                              const double *rho_new, const double *rho_abs, double *out,
                              cudaStream_t st);
cudaError_t launch_adjoint_forward(const GridP &g, const FieldPtrsT<double> &F, int64_t n,
                                   double qm, double scale, int n_steps, int every, int n_iter,
                                   const double *st0, double *out, double *ckpt,
                                   cudaStream_t st);
cudaError_t launch_adjoint_backward(const GridP &g, const FieldPtrsT<double> &F, int64_t n,
                                    double qm, double scale, double gfac, int n_steps, int every,
                                    int n_iter,
                                    const double *ckpt, const double *gout, double *gin,
                                    double *gscale_pp, double *gscale_sum, double *scratch,
                                    cudaStream_t st);
template <typename T>
cudaError_t launch_load(const GridP &g, SpeciesDevT<T> s, int64_t k0, int64_t n,
                        const grpic_particle_init &in, double density_power, cudaStream_t st);
template <typename T>
cudaError_t launch_push(const GridP &g, const FieldPtrsT<T> &F, SpeciesDevT<T> s,
                        const PushTables &tb, const GuardList &gl, const TileInfo &ti,
                        int64_t n_bound, bool deposit, unsigned long long *diag,
                        const PushStreams &ps);
template <typename T>
cudaError_t launch_deposit(const GridP &g, const FieldPtrsT<T> &F, SpeciesDevT<T> s,
                           const PushTables &tb, int64_t n_bound, cudaStream_t st);
template <typename T>
cudaError_t launch_invariants(const GridP &g, SpeciesDevT<T> s, int kind, double B0,
                              double *E, double *L, int64_t n_bound, cudaStream_t st);

struct SortScratch {
  uint32_t *keys[2], *vals[2];
  uint32_t *hist;     // [256][nblocks]
  uint32_t *bsum;     // block sums of the scan
  unsigned long long *alive;  // alive count of the species being sorted
  int64_t max_n;
  int max_blocks;
};
int64_t sort_hist_entries(int64_t max_n);
int64_t sort_bsum_entries(int64_t max_n);
// with_prev false: the previous-position arrays are left out of the gather (the caller
// pushes the species next, and the push rewrites them first)
template <typename T>
cudaError_t launch_sort(const GridP &g, int tile_r, int tile_t, SpeciesDevT<T> in,
                        SpeciesDevT<T> out, int64_t n_bound, int64_t *n_dev, const SortScratch &S,
                        uint32_t *tile_start, cudaStream_t st, bool with_prev = true);
