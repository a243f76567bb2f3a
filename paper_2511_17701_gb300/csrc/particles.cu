// particles.cu -- the GR particle pusher (Sec. 3.1 of arXiv:2511.17701) and the
// charge-conserving conformal current deposit (Sec. 3.2), one thread per particle.
//
// FP64 path: the double-precision pipe, not HBM, bounds the kernel on GB300 (every
// particle-step evaluates the metric up to n_iter + 2 times). Mixed path: FP32 state,
// fields and arithmetic; for particles within a few cells of the horizon or an axis the
// metric, lapse and shift are evaluated in FP64 (and rounded), in a second kernel. Particle state is SoA; consecutive threads read consecutive elements,
// and field gathers hit L1/L2 because the particles are kept sorted by cell.
#include "grpic_internal.cuh"
#include "pusher.cuh"

namespace {

constexpr int TPB = 128;

__device__ __forceinline__ void count(unsigned long long *diag, int which) {
  atomicAdd(diag + which, 1ull);
}

// x is neither infinite nor NaN
__device__ __forceinline__ bool finite64(double x) {
  return ((unsigned)__double2hiint(x) & 0x7ff00000u) != 0x7ff00000u;
}
// |x| <= c and |x| < c for a constant c >= 0 (x NaN: false): the ordering of non-negative
// doubles is the ordering of their bit patterns
__device__ __forceinline__ bool abs_le(double x, double c) {
  return ((unsigned long long)__double_as_longlong(x) & 0x7fffffffffffffffull) <=
         (unsigned long long)__double_as_longlong(c);
}
__device__ __forceinline__ bool abs_lt(double x, double c) {
  return ((unsigned long long)__double_as_longlong(x) & 0x7fffffffffffffffull) <
         (unsigned long long)__double_as_longlong(c);
}
// x < c and x > c for a constant c > 0 (x NaN: false): as signed integers, negative doubles
// order below every positive one and positive doubles order as their bit patterns
__device__ __forceinline__ bool lt_pos(double x, double c) {
  return __double_as_longlong(x) < __double_as_longlong(c) && finite64(x);
}
__device__ __forceinline__ bool gt_pos(double x, double c) {
  return __double_as_longlong(x) > __double_as_longlong(c) && finite64(x);
}

// =================================================================================
// FP64 routine. r and sin/cos at the iterates follow from their values at x^n by the
// exponential and angle-addition formulas with short Taylor series of the small offsets
// (|eps| <= 0.02: truncation below 1e-18); CUDA's exp/sincos beyond that and in the
// SMALL_ANGLE_GR clamp. theta at every point is formed as the oracle forms it (map_theta:
// x2 dtheta, then the quasi-spherical cubic, each operation rounded), and its offset from
// theta(x^n) is exact (Sterbenz): near theta = pi sin(theta) is ill-conditioned in theta,
// so any other way of forming theta would move the result by ~1e-12 relative.
// =================================================================================
struct Base {
  double x1, th0;     // x^n and theta(x^n) (not clamped)
  double e0, s0, c0;  // exp(xi) = r - r0, sin(theta), cos(theta) at x^n
};

__device__ __forceinline__ double exp_small(double e) {  // exp(e), |e| <= 0.02
  double p = 1.0 / 5040.0;
  p = fma(p, e, 1.0 / 720.0);
  p = fma(p, e, 1.0 / 120.0);
  p = fma(p, e, 1.0 / 24.0);
  p = fma(p, e, 1.0 / 6.0);
  p = fma(p, e, 0.5);
  p = fma(p, e, 1.0);
  return fma(p, e, 1.0);
}

template <bool Q = true>
__device__ __forceinline__ Base make_base(const GridP &g, double x1, double x2) {
  Base b;
  b.x1 = x1;
  b.th0 = map_theta<Q>(g, x2);
  b.e0 = map_e(g, x1);
  sincos(b.th0, &b.s0, &b.c0);
  return b;
}

// x^n from the per-corner tables (rows away from the axes): exp(xi) = r64[i] exp(dx1 dxi) and
// sin/cos(theta) by the angle-addition formulas from corner row j, with Taylor series of the
// offsets (|dx1 dxi| <= 0.02: truncation below 1e-18; |d| <= 0.1, d = theta - theta_j exact by
// Sterbenz since theta_j >= 2 dtheta there: below 3e-19). One FP64 exp and sincos fewer per
// particle; beyond those offsets the library functions as make_base.
template <bool Q = true>
__device__ __forceinline__ Base make_base_tab(const GridP &g, const PushTables &tb, int i1, int i2,
                                              double dx1, double x1, double x2) {
  Base b;
  b.x1 = x1;
  b.th0 = map_theta<Q>(g, x2);
  const double e = dx1 * g.dxi;
  b.e0 = abs_le(e, 0.02) ? __ldg(tb.r64 + i1 + G_) * exp_small(e) : map_e(g, x1);
  const double d = b.th0 - __ldg(tb.th64 + i2 + G_);
  if (abs_le(d, 0.1)) {
    const double q = d * d;
    double sp = 1.0 / 362880.0;
    sp = fma(sp, q, -1.0 / 5040.0);
    sp = fma(sp, q, 1.0 / 120.0);
    sp = fma(sp, q, -1.0 / 6.0);
    const double se = fma(sp * q, d, d);
    double cp = -1.0 / 3628800.0;
    cp = fma(cp, q, 1.0 / 40320.0);
    cp = fma(cp, q, -1.0 / 720.0);
    cp = fma(cp, q, 1.0 / 24.0);
    cp = fma(cp, q, -0.5);
    const double ce = fma(cp, q, 1.0);
    const double s0 = __ldg(tb.s64 + i2 + G_), c0 = __ldg(tb.c64 + i2 + G_);
    b.s0 = fma(s0, ce, c0 * se);
    b.c0 = fma(c0, ce, -s0 * se);
  } else {
    sincos(b.th0, &b.s0, &b.c0);
  }
  return b;
}

// x^n itself: r, sin and cos are the base's (local_rsc with zero offsets gives the same bits),
// theta clamped to [small_angle, pi - small_angle]
template <bool Q = true>
__device__ __forceinline__ void local_at_base(const GridP &g, const Base &b, double x2,
                                              Pt<double> &p) {
  p.r = Q ? g.r0 + b.e0 : b.e0;
  p.f = g.dxi * b.e0;
  if (Q && g.qks) {
    map_g<Q>(g, x2, p.gg, p.gp);
  } else {
    p.gg = g.dth;
    p.igg = g.ig2;
    p.gp = 0.0;
  }
  const double th = b.th0;
  if (lt_pos(th, g.small_angle) || gt_pos(th, g.pi_small)) {
    sincos(fmin(fmax(th, g.small_angle), GRPIC_PI - g.small_angle), &p.s, &p.c);
  } else {
    p.s = b.s0;
    p.c = b.c0;
  }
}

// the point (x1t, x2t): r, sin(theta), cos(theta) with theta clamped to [small_angle,
// pi - small_angle], and the map's factors
template <bool Q = true>
__device__ __forceinline__ void local_rsc(const GridP &g, const Base &b, double x1t, double x2t,
                                          Pt<double> &p) {
  const double e1 = (x1t - b.x1) * g.dxi;
  const double ex = abs_le(e1, 0.02) ? b.e0 * exp_small(e1) : map_e(g, x1t);
  p.r = Q ? g.r0 + ex : ex;
  p.f = g.dxi * ex;
  if (Q && g.qks) {
    map_g<Q>(g, x2t, p.gg, p.gp);
  } else {
    p.gg = g.dth;
    p.igg = g.ig2;
    p.gp = 0.0;
  }
  const double th = map_theta<Q>(g, x2t);
  const double e2 = th - b.th0;
  if (lt_pos(th, g.small_angle) || gt_pos(th, g.pi_small)) {
    sincos(fmin(fmax(th, g.small_angle), GRPIC_PI - g.small_angle), &p.s, &p.c);
  } else if (abs_le(e2, 0.02)) {
    const double q = e2 * e2;
    double sp = -1.0 / 5040.0;
    sp = fma(sp, q, 1.0 / 120.0);
    sp = fma(sp, q, -1.0 / 6.0);
    const double se = fma(sp * q, e2, e2);  // sin(e2)
    double cp = 1.0 / 40320.0;
    cp = fma(cp, q, -1.0 / 720.0);
    cp = fma(cp, q, 1.0 / 24.0);
    cp = fma(cp, q, -0.5);
    const double ce = fma(cp, q, 1.0);      // cos(e2)
    p.s = fma(b.s0, ce, b.c0 * se);
    p.c = fma(b.c0, ce, -b.s0 * se);
  } else {
    sincos(th, &p.s, &p.c);
  }
}

// dphi/dt = alpha/gamma h^{3j} u_j at (x1t, x2t) (Eq. discretized-geodesic-x-phi; q times
// it is J^3 / sqrt(h) w, Sec. 3.2); alpha/gamma = 1/sqrt((1+z) gamma^2).
template <bool Q = true>
__device__ __forceinline__ double phi_rate64(const GridP &g, const Base &b, double x1t,
                                             double x2t, const double u[3], double m2) {
  Pt<double> p;
  local_rsc<Q>(g, b, x1t, x2t, p);
  Geo<double> o;
  geo_from_rsc<Q>(g, p, o);
  const double q = fma(o.H11 * u[0], u[0], fma(o.H22 * u[1], u[1], fma(o.H33 * u[2], u[2],
                   fma(2.0 * o.H13 * u[0], u[2], m2))));
  return rsqrt(o.opz * q) * fma(o.H13, u[0], o.H33 * u[2]);
}

// Bilinear interpolation at code position (x1, x2) of planes whose Yee location is offset by
// 0 or 1/2 in each direction. The cells and weights of the two offsets per direction are
// formed once for all six gathers (absolute coordinates, rounded as the oracle rounds them:
// y = x - s, cell floor(y), weight y - floor(y)).
struct Lerp64 {
  int i[2], j[2];
  double w1[2], w2[2];
};
__device__ __forceinline__ void lerp_setup(double x1, double x2, Lerp64 &L) {
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    const double y1 = h ? x1 - 0.5 : x1, y2 = h ? x2 - 0.5 : x2;
    const double f1 = floor(y1), f2 = floor(y2);
    L.i[h] = (int)f1;
    L.j[h] = (int)f2;
    L.w1[h] = y1 - f1;
    L.w2[h] = y2 - f2;
  }
}
template <typename T>
__device__ __forceinline__ double interp64(const T *__restrict__ pl, int NX, const Lerp64 &L,
                                           int h1, int h2) {
  const T *p = pl + (int64_t)(L.j[h2] + G_) * NX + (L.i[h1] + G_);
  const double p00 = __ldg(p), p10 = __ldg(p + 1), p01 = __ldg(p + NX), p11 = __ldg(p + NX + 1);
  // nested linear interpolations: the same bilinear value in 3 DADD + 3 DFMA
  const double w1 = L.w1[h1];
  const double a = fma(w1, p10 - p00, p00), c = fma(w1, p11 - p01, p01);
  return fma(L.w2[h2], c - a, a);
}

template <typename T>
__device__ __forceinline__ void add_(T *p, double v) {
  atomicAdd(p, (T)v);
}

// Charge-conserving deposit of one move (Sec. 3.2, Eq. charge-conservation-disc): the zigzag
// split of Umeda et al. (2003) with area weighting, plus J^3 = q alpha u^3 / gamma at the
// midpoint, in absolute coordinates as the oracle.
template <typename T>
__device__ __forceinline__ void deposit64(const GridP &g, const FieldPtrsT<T> &F, double q,
                                          int ia, int ja, double xa1, double xa2, int ib, int jb,
                                          double xb1, double xb2, double v3) {
  const double idt = g.idt;
  // the relay point: min/max of the cell indices taken on integers (the same values)
  const double xr1 = fmin((double)(min(ia, ib) + 1), fmax((double)max(ia, ib), 0.5 * (xa1 + xb1)));
  const double xr2 = fmin((double)(min(ja, jb) + 1), fmax((double)max(ja, jb), 0.5 * (xa2 + xb2)));
  T *J1 = F.J[0], *J2 = F.J[1], *J3 = F.J[2];
  const int NX = g.NX;
  {
    const double F1 = q * (xr1 - xa1) * idt, F2 = q * (xr2 - xa2) * idt;
    const double W1 = 0.5 * (xa1 + xr1) - ia, W2 = 0.5 * (xa2 + xr2) - ja;
    const int64_t k = sidx(g, ia, ja);
    add_(J1 + k, F1 * (1.0 - W2));
    add_(J1 + k + NX, F1 * W2);
    add_(J2 + k, F2 * (1.0 - W1));
    add_(J2 + k + 1, F2 * W1);
  }
  {
    const double F1 = q * (xb1 - xr1) * idt, F2 = q * (xb2 - xr2) * idt;
    const double W1 = 0.5 * (xr1 + xb1) - ib, W2 = 0.5 * (xr2 + xb2) - jb;
    const int64_t k = sidx(g, ib, jb);
    add_(J1 + k, F1 * (1.0 - W2));
    add_(J1 + k + NX, F1 * W2);
    add_(J2 + k, F2 * (1.0 - W1));
    add_(J2 + k + 1, F2 * W1);
  }
  const double xm1 = 0.5 * (xa1 + xb1), xm2 = 0.5 * (xa2 + xb2);
  const double f1 = floor(xm1), f2 = floor(xm2);
  const int i0 = (int)f1, j0 = (int)f2;
  const double w1 = xm1 - f1, w2 = xm2 - f2, qv = q * v3;
  const int64_t k = sidx(g, i0, j0);
  add_(J3 + k, qv * (1.0 - w1) * (1.0 - w2));
  add_(J3 + k + 1, qv * w1 * (1.0 - w2));
  add_(J3 + k + NX, qv * (1.0 - w1) * w2);
  add_(J3 + k + NX + 1, qv * w1 * w2);
}

// Stop rule of the FP32 implicit iterations: the update within ITER_TOL32 max(1, |value|),
// two FP32 ulps at 1. The remaining error, rho / (1 - rho) of that update (rho the
// contraction), is then below the rounding of the stored values.
constexpr float ITER_TOL32 = 0x1p-22f;
__device__ __forceinline__ bool settled32(float n0, float t0, float n1, float t1) {
  return fabsf(n0 - t0) <= ITER_TOL32 * fmaxf(1.0f, fabsf(n0)) &&
         fabsf(n1 - t1) <= ITER_TOL32 * fmaxf(1.0f, fabsf(n1));
}
// The coordinate iteration may also stop on an estimate of its remaining error: two successive
// updates d_prev, d of a linearly converging iteration give its rate as about d / d_prev, so
// the error left after the latest one is about d^2 / d_prev. Stop when sixteen times that is
// below ITER_TOL32 (cell units). After the first metric evaluation at the midpoint, d_prev is
// the particle's whole move and d about rho times it (rho ~ dt |dV/dx|, 1e-3 or less off the
// guard zones), so most warps stop there instead of running a third evaluation for the few
// lanes whose update is still above the plain rule's bound.
__device__ __forceinline__ bool settled32_rate(float d, float d_prev) {
  return 16.0f * d * d <= ITER_TOL32 * d_prev;
}

// Refined form of the two implicit substeps (iter_tol > 0): an FP32 predictor iterates the
// same map to an exact FP32 repeat (metric from the FP32 cell tables; the coordinate
// substep's also stops on the rate estimate above, which puts it within the rounding of its
// FP32 values as well) and gives the map's Jacobian J there (FP32, analytic). The FP64 map
// is evaluated at the predictor's point; one Newton step with J on that residual lands
// within about |J error| times the predictor's rounding of the FP64 fixed point, and a
// second FP64 evaluation there verifies it: the result is taken once an FP64 update is at
// most iter_tol max(1, |value|), with plain FP64 iterations after the second evaluation
// while it is not (at most n_iter evaluations in all). The result is the FP64 fixed point to about rho iter_tol, rho < 1 the contraction,
// whatever the start: J and the predictor only save FP64 work (mixed-precision refinement).
// |n - t| <= tol max(1, |n|): the difference in FP64 (n and t agree to about tol), the test
// in FP32 on truncated values (the bound moves by less than 2^-22 of itself)
__device__ __forceinline__ bool converged(double n, double t, float tol) {
  return fabsf(f32_trunc(n - t)) <= tol * fmaxf(1.0f, fabsf(f32_trunc(n)));
}
// the largest eigenvalue modulus of a 2 x 2 matrix: the asymptotic contraction of a map
// with that Jacobian
__device__ __forceinline__ float spectral_radius(const float J[2][2]) {
  const float tr = J[0][0] + J[1][1], det = fmaf(J[0][0], J[1][1], -J[0][1] * J[1][0]);
  const float disc = fmaf(tr, tr, -4.0f * det);
  return disc >= 0.0f ? 0.5f * (fabsf(tr) + sqrtf(disc)) : sqrtf(fmaxf(det, 0.0f));
}
// Whether the method's n_iter iterations from its start come within a tenth of tol of the
// fixed point, so that the refined result stands for the method's n_iter result: d1 is the
// method's first update (from the FP32 predictor's first step), rho the contraction (the
// spectral radius of J), the remainder d1 rho^n_iter.
__device__ __forceinline__ bool method_converges(float d1, float rho, int n_iter, float tol,
                                                 double s0, double s1) {
  if (!(rho < 0.5f)) return false;
  if (!(rho > 0.0f)) return true;
  const float scale = fmaxf(1.0f, fmaxf(fabsf(f32_trunc(s0)), fabsf(f32_trunc(s1))));
  return d1 * exp2f((float)n_iter * log2f(rho)) <= 0.1f * tol * scale;
}
// t + (I - J)^{-1} (n - t): the Newton step of t = G(t) from the residual n - t; the plain
// iteration step (n itself) when the result is not finite
__device__ __forceinline__ void newton_step(const float J[2][2], double t0, double t1, double n0,
                                            double n1, double &s0, double &s1) {
  const float a = 1.0f - J[0][0], d = 1.0f - J[1][1];
  const float idet = 1.0f / fmaf(a, d, -J[0][1] * J[1][0]);
  const double r0 = n0 - t0, r1 = n1 - t1;
  s0 = t0 + fma(f64_widen(idet * d), r0, f64_widen(idet * J[0][1]) * r1);
  s1 = t1 + fma(f64_widen(idet * J[1][0]), r0, f64_widen(idet * a) * r1);
  if (!(finite64(s0) && finite64(s1))) {
    s0 = n0;
    s1 = n1;
  }
}

// ---------------------------------------------------------------------------------
// Double-float predictor step of the refined iterations (plain grid). The implicit map is
// evaluated once in float pairs (about 48 bits, dfloat.cuh) at the FP32 predictor's point,
// and one Newton step with the FP32 Jacobian there lands within about 1e-14 of the FP64
// fixed point (the predictor's 1e-7 error times the Jacobian's 1e-7 relative error, plus the
// pairs' rounding): the FP64 evaluation that follows then usually meets the stop rule at
// once, one FP64 map evaluation per substep instead of two. The arithmetic runs on the FP32
// pipe, which the FP64 kernel otherwise leaves idle; the result is still the FP64 map's.
// ---------------------------------------------------------------------------------
// r, sin(theta), cos(theta) and the map's factors as pairs at x1 = i + o1, x2 = j + o2: the
// corner tables and Taylor series of the offsets (|o1 dxi|, |theta offset| <= 0.12: the
// series' truncation below 1e-19), on a quasi-spherical grid with the theta offset's cubic in
// the offset in eta and its derivatives
template <bool Q>
__device__ __forceinline__ void rsc_df(const GridP &g, const PushTables &tb, int i, int j, DF o1,
                                       DF o2, Pt<DF> &p) {
  const Cst<DF> k = cst<DF>(g);
  const DF e = o1 * k.dxi;
  DF x = dfc(1.0 / 362880.0);
  x = fma_(x, e, dfc(1.0 / 40320.0));
  x = fma_(x, e, dfc(1.0 / 5040.0));
  x = fma_(x, e, dfc(1.0 / 720.0));
  x = fma_(x, e, dfc(1.0 / 120.0));
  x = fma_(x, e, dfc(1.0 / 24.0));
  x = fma_(x, e, dfc(1.0 / 6.0));
  x = fma_(x, e, DF(0.5f));
  x = fma_(x, e, DF(1.0f));
  x = fma_(x, e, DF(1.0f));  // exp(e)
  const float2 rt = __ldg(tb.r_df + i + G_);
  const DF ex = DF(rt.x, rt.y) * x;
  p.r = Q ? DF(g.d_r0[0], g.d_r0[1]) + ex : ex;
  p.f = k.dxi * ex;
  DF d = o2 * k.dth;  // the offset in eta, then in theta
  if (Q && g.qks) {
    const float2 a1 = __ldg(tb.t1_df + j + G_), a2 = __ldg(tb.t2_df + j + G_);
    const DF t1(a1.x, a1.y), t2(a2.x, a2.y), c3(g.d_c3[0], g.d_c3[1]);
    const DF t22 = t2 + t2, c33 = DF(3) * c3;
    p.gg = k.dth * fma_(d, fma_(c33, d, t22), t1);
    p.gp = k.dth * k.dth * fma_(c33 + c33, d, t22);
    p.igg = DF(0.0f);
    d = d * fma_(d, fma_(c3, d, t2), t1);
  } else {
    p.gg = k.dth;
    p.igg = k.ig2;
    p.gp = DF(0.0f);
  }
  const DF q = d * d;
  DF sp = dfc(1.0 / 362880.0);
  sp = fma_(sp, q, dfc(-1.0 / 5040.0));
  sp = fma_(sp, q, dfc(1.0 / 120.0));
  sp = fma_(sp, q, dfc(-1.0 / 6.0));
  const DF se = fma_(sp * q, d, d);
  DF cp = dfc(-1.0 / 3628800.0);
  cp = fma_(cp, q, dfc(1.0 / 40320.0));
  cp = fma_(cp, q, dfc(-1.0 / 720.0));
  cp = fma_(cp, q, dfc(1.0 / 24.0));
  cp = fma_(cp, q, DF(-0.5f));
  const DF ce = fma_(cp, q, DF(1.0f));
  const float2 st = __ldg(tb.s_df + j + G_), ct = __ldg(tb.c_df + j + G_);
  const DF s0(st.x, st.y), c0(ct.x, ct.y);
  p.s = s0 * ce + c0 * se;
  p.c = c0 * ce - s0 * se;
}
__device__ __forceinline__ DF df_half(DF a) { return DF(0.5f * a.hi, 0.5f * a.lo); }

// the coordinate map t -> dx + dt V((x^n + t)/2) of Eq. (discretized-geodesic-x) in pairs
template <bool Q>
__device__ __forceinline__ void coord_map_df(const GridP &g, const PushTables &tb, int i1, int i2,
                                             DF dx1, DF dx2, const DF u[3], DF m2, DF t1, DF t2,
                                             DF &n1, DF &n2) {
  Pt<DF> p;
  rsc_df<Q>(g, tb, i1, i2, df_half(dx1 + t1), df_half(dx2 + t2), p);
  Geo<DF> o;
  geo_from_rsc<Q>(g, p, o);
  const DF uu = DF(2) * u[0] * u[2];
  const DF q = fma_(o.H11 * u[0], u[0], fma_(o.H22 * u[1], u[1],
               fma_(o.H33 * u[2], u[2], fma_(o.H13, uu, m2))));
  const DF ag = rsqrt_(o.opz * q);
  const DF dt = cst<DF>(g).dt;
  n1 = fma_(dt, fma_(ag, fma_(o.H11, u[0], o.H13 * u[2]), -o.beta1), dx1);
  n2 = fma_(dt, ag * o.H22 * u[1], dx2);
}

// t + (I - J)^{-1} (n - t) in pairs, the matrix from the FP32 Jacobian
__device__ __forceinline__ void newton_df(const float J[2][2], DF t0, DF t1, DF n0, DF n1,
                                          DF &s0, DF &s1) {
  const float a = 1.0f - J[0][0], d = 1.0f - J[1][1];
  const float idet = 1.0f / fmaf(a, d, -J[0][1] * J[1][0]);
  const DF r0 = n0 - t0, r1 = n1 - t1;
  s0 = t0 + (DF(idet * d) * r0 + DF(idet * J[0][1]) * r1);
  s1 = t1 + (DF(idet * J[1][0]) * r0 + DF(idet * a) * r1);
}

// the metric pieces the momentum map reads, as pairs
__device__ __forceinline__ void df_local(const Local<double> &L, Local<DF> &D) {
  D.alpha = df_of(L.alpha);
  D.G.H11 = df_of(L.G.H11);
  D.G.H13 = df_of(L.G.H13);
  D.G.H22 = df_of(L.G.H22);
  D.G.H33 = df_of(L.G.H33);
  D.d1H11 = df_of(L.d1H11); D.d1H22 = df_of(L.d1H22); D.d1H33 = df_of(L.d1H33);
  D.d1H13 = df_of(L.d1H13); D.d1alpha = df_of(L.d1alpha); D.d1beta1 = df_of(L.d1beta1);
  D.d2H11 = df_of(L.d2H11); D.d2H22 = df_of(L.d2H22); D.d2H33 = df_of(L.d2H33);
  D.d2H13 = df_of(L.d2H13); D.d2alpha = df_of(L.d2alpha); D.d2beta1 = df_of(L.d2beta1);
}

template <bool Q = true>
__device__ __forceinline__ void geodesic_refined(const GridP &g, const PushTables &tb, int i1,
                                                 int i2, float o1, float o2,
                                                 const Local<double> &L, double u[3],
                                                 double m2) {
  Pt<float> pf;
  rsc32<Q>(g, tb, i1, i2, o1, o2, pf);
  Local<float> Lf;
  local_full<Q>(g, pf, Lf);
  const float uf[3] = {f32_trunc(u[0]), f32_trunc(u[1]), f32_trunc(u[2])};
  const GeoMap<float> mf(g, Lf, uf, f32_trunc(m2));
  float p0 = uf[0], p1 = uf[1], d1 = 0.0f;
  for (int it = 0; it < g.n_iter; ++it) {
    float n0, n1;
    mf.apply(p0, p1, n0, n1);
    if (it == 0) d1 = fmaxf(fabsf(n0 - p0), fabsf(n1 - p1));
    const bool fixed = n0 == p0 && n1 == p1;
    p0 = n0;
    p1 = n1;
    if (fixed) break;
  }
  const GeoMap<double> m(g, L, u, m2);
  double t0 = u[0], t1 = u[1];
  float J[2][2] = {{0.0f, 0.0f}, {0.0f, 0.0f}};
  double n0, n1, s0, s1;
  bool df_start = false;
  if (isfinite(p0) && isfinite(p1)) {
    mf.jacobian(p0, p1, J);
    {  // the double-float predictor step
      if (g.n_iter >= 2) {
        Local<DF> Ld;
        df_local(L, Ld);
        const DF ud[3] = {df_of(u[0]), df_of(u[1]), df_of(u[2])};
        const GeoMap<DF> md(g, Ld, ud, DF(f32_trunc(m2)));
        DF n0d, n1d, s0d, s1d;
        md.apply(DF(p0), DF(p1), n0d, n1d);
        newton_df(J, DF(p0), DF(p1), n0d, n1d, s0d, s1d);
        s0 = df_to_double(s0d);
        s1 = df_to_double(s1d);
        df_start = finite64(s0) && finite64(s1);
      }
    }
    t0 = f64_widen(p0);
    t1 = f64_widen(p1);
  }
  if (!df_start) {
    m.apply(t0, t1, n0, n1);
    newton_step(J, t0, t1, n0, n1, s0, s1);
  }
  bool conv = false;
  for (int it = 1; it < g.n_iter && !conv; ++it) {
    m.apply(s0, s1, n0, n1);
    conv = converged(n0, s0, g.f_iter_tol) && converged(n1, s1, g.f_iter_tol);
    s0 = n0;
    s1 = n1;
  }
  if (!method_converges(d1, spectral_radius(J), g.n_iter, g.f_iter_tol, s0, s1)) {
    geodesic_momentum(g, L, u, m2);  // the method's n_iter iterations from u
    return;
  }
  u[0] = s0;
  u[1] = s1;
}

// dt/2 times the derivative of the coordinate velocity V of Eq. (discretized-geodesic-x) at
// the point of L for the momentum u: the Jacobian of the map t -> x^n + dt V((x^n + t)/2).
// V^1 = (alpha/gamma) (h^11 u_1 + h^13 u_3) - beta^1, V^2 = (alpha/gamma) h^22 u_2, with
// alpha/gamma = (q / alpha^2)^(-1/2), q = m2 + h^ij u_i u_j.
__device__ __forceinline__ void coord_jacobian(const GridP &g, const Local<float> &L,
                                               const float u[3], float m2, float J[2][2]) {
  const Geo<float> &o = L.G;
  const float uu = 2.0f * u[0] * u[2], u00 = u[0] * u[0], u11 = u[1] * u[1], u22 = u[2] * u[2];
  const float q = fmaf(o.H11, u00, fmaf(o.H22, u11, fmaf(o.H33, u22, fmaf(o.H13, uu, m2))));
  const float ag = rsqrtf(o.opz * q);
  const float w1 = fmaf(o.H11, u[0], o.H13 * u[2]), w2 = o.H22 * u[1];
  const float ia = L.alpha * o.opz;           // 1 / alpha
  const float hq = 0.5f * ag * ag * o.opz;    // 1 / (2 q)
  const float hdt = 0.5f * g.f_dt;
  const float dH11[2] = {L.d1H11, L.d2H11}, dH22[2] = {L.d1H22, L.d2H22};
  const float dH33[2] = {L.d1H33, L.d2H33}, dH13[2] = {L.d1H13, L.d2H13};
  const float dal[2] = {L.d1alpha, L.d2alpha}, dbe[2] = {L.d1beta1, L.d2beta1};
#pragma unroll
  for (int j = 0; j < 2; ++j) {
    const float dq = fmaf(dH11[j], u00, fmaf(dH22[j], u11, fmaf(dH33[j], u22, dH13[j] * uu)));
    const float dag = ag * fmaf(dal[j], ia, -dq * hq);
    J[0][j] = hdt * (fmaf(dag, w1, ag * fmaf(dH11[j], u[0], dH13[j] * u[2])) - dbe[j]);
    J[1][j] = hdt * fmaf(dag, w2, ag * dH22[j] * u[1]);
  }
}

// The FP64 routine on FP32 storage (the mixed path's axis rows) stops its iterations once the
// update is within SETTLE32 max(1, |value|), far below what the stored FP32 result resolves;
// the FP64 path (settle 0) stops at an exact repeat only.
constexpr double SETTLE32 = 0x1p-26;
__device__ __forceinline__ bool settled64(double n0, double t0, double n1, double t1,
                                          double settle) {
  return fabs(n0 - t0) <= settle * fmax(1.0, fabs(n0)) &&
         fabs(n1 - t1) <= settle * fmax(1.0, fabs(n1));
}
// the geodesic momentum substep with that stop rule (settle 0: geodesic_momentum itself)
__device__ __forceinline__ void geodesic_momentum_settle(const GridP &g, const Local<double> &L,
                                                         double u[3], double m2, double settle) {
  if (settle == 0.0) {
    geodesic_momentum(g, L, u, m2);
    return;
  }
  const GeoMap<double> m(g, L, u, m2);
  double t0 = u[0], t1 = u[1];
  for (int it = 0; it < g.n_iter; ++it) {
    double n0, n1;
    m.apply(t0, t1, n0, n1);
    const bool fixed = settled64(n0, t0, n1, t1, settle);
    t0 = n0;
    t1 = n1;
    if (fixed && g.stop_on_repeat) break;
  }
  u[0] = t0;
  u[1] = t1;
}

// The coordinate substep, Eq. (discretized-geodesic-x), as the method iterates it: metric at
// x_bar = (x^n + x~)/2, the first iterate x^n itself (metric L.G), n_iter iterations or
// until an exact repeat. t1, t2: the new offsets from cell (i1, i2).
template <bool Q = true>
__device__ __forceinline__ void coord_exact(const GridP &g, const Base &b, const Local<double> &L,
                                            int i1, int i2, double dx1, double dx2,
                                            const double u[3], double m2, double &t1,
                                            double &t2, double settle = 0.0) {
  const double uu0 = 2.0 * u[0] * u[2];
  t1 = dx1;
  t2 = dx2;
  for (int it = 0; it < g.n_iter; ++it) {
    Geo<double> o;
    if (it == 0) {
      o = L.G;
    } else {
      Pt<double> p;
      // x_bar = i + (dx + x~)/2, rounded in that order
      local_rsc<Q>(g, b, __dadd_rn((double)i1, 0.5 * __dadd_rn(dx1, t1)),
                   __dadd_rn((double)i2, 0.5 * __dadd_rn(dx2, t2)), p);
      geo_from_rsc<Q>(g, p, o);
    }
    const double q = fma(o.H11 * u[0], u[0], fma(o.H22 * u[1], u[1],
                     fma(o.H33 * u[2], u[2], fma(o.H13, uu0, m2))));
    const double ag = rsqrt(o.opz * q);  // alpha / gamma
    const double n1 = fma(g.dt, fma(ag, fma(o.H11, u[0], o.H13 * u[2]), -o.beta1), dx1);
    const double n2 = fma(g.dt, ag * o.H22 * u[1], dx2);
    // exact repeat: later iterations are no-ops; or (settle > 0) an update below settle
    const bool fixed = settle > 0.0 ? settled64(n1, t1, n2, t2, settle)
                                    : (n1 == t1) && (n2 == t2);
    t1 = n1;
    t2 = n2;
    if (fixed && g.stop_on_repeat) break;
  }
}

// One FP64 evaluation of the coordinate map at the iterate (t1, t2): the new offsets (n1, n2)
// and dphi/dt (v3) at its midpoint x_bar = i + (dx + t)/2
template <bool Q = true>
__device__ __forceinline__ void coord_map64(const GridP &g, const Base &b, int i1, int i2,
                                            double dx1, double dx2, const double u[3],
                                            double m2, double t1, double t2, double &n1,
                                            double &n2, double &v3) {
  Pt<double> p;
  local_rsc<Q>(g, b, __dadd_rn((double)i1, 0.5 * __dadd_rn(dx1, t1)),
               __dadd_rn((double)i2, 0.5 * __dadd_rn(dx2, t2)), p);
  Geo<double> o;
  geo_from_rsc<Q>(g, p, o);
  const double q = fma(o.H11 * u[0], u[0], fma(o.H22 * u[1], u[1],
                   fma(o.H33 * u[2], u[2], fma(o.H13, 2.0 * u[0] * u[2], m2))));
  const double ag = rsqrt(o.opz * q);
  n1 = fma(g.dt, fma(ag, fma(o.H11, u[0], o.H13 * u[2]), -o.beta1), dx1);
  n2 = fma(g.dt, ag * o.H22 * u[1], dx2);
  v3 = ag * fma(o.H13, u[0], o.H33 * u[2]);  // Eq. (discretized-geodesic-x-phi) at x_bar
}

// the coordinate substep's refined iterations; t1, t2: the new offsets from cell (i1, i2)
// v3 (dphi/dt) comes back from the metric of the last FP64 evaluation, whose midpoint is
// within iter_tol of the final one (or is NaN when the method's iteration ran instead).
template <bool Q = true>
__device__ __forceinline__ void coord_refined(const GridP &g, const PushTables &tb, const Base &b,
                                              const Local<double> &L, int i1, int i2,
                                              double dx1, double dx2, const double u[3],
                                              double m2, double &t1, double &t2, double &v3) {
  const float uf[3] = {f32_trunc(u[0]), f32_trunc(u[1]), f32_trunc(u[2])};
  const float a1 = f32_trunc(dx1), a2 = f32_trunc(dx2), dt = g.f_dt, m2f = f32_trunc(m2);
  const float uuf = 2.0f * uf[0] * uf[2];
  float p1 = a1, p2 = a2, d1 = 0.0f, d_prev = 0.0f;
  for (int it = 0; it < g.n_iter; ++it) {
    Pt<float> pf;
    rsc32<Q>(g, tb, i1, i2, 0.5f * (a1 + p1), 0.5f * (a2 + p2), pf);
    Geo<float> o;
    geo_from_rsc<Q>(g, pf, o);
    const float q = fmaf(o.H11 * uf[0], uf[0], fmaf(o.H22 * uf[1], uf[1],
                    fmaf(o.H33 * uf[2], uf[2], fmaf(o.H13, uuf, m2f))));
    const float ag = rsqrtf(o.opz * q);
    const float n1 = fmaf(dt, fmaf(ag, fmaf(o.H11, uf[0], o.H13 * uf[2]), -o.beta1), a1);
    const float n2 = fmaf(dt, ag * o.H22 * uf[1], a2);
    const float d = fmaxf(fabsf(n1 - p1), fabsf(n2 - p2));
    if (it == 0) d1 = d;
    const bool fixed = (n1 == p1 && n2 == p2) || settled32_rate(d, d_prev);
    d_prev = d;
    p1 = n1;
    p2 = n2;
    if (fixed) break;
  }
  t1 = dx1;
  t2 = dx2;
  float J[2][2] = {{0.0f, 0.0f}, {0.0f, 0.0f}};
  double n1, n2, s1, s2;
  bool df_start = false;
  if (isfinite(p1) && isfinite(p2) && fabsf(p1) < 4.0f && fabsf(p2) < 4.0f) {
    t1 = f64_widen(p1);
    t2 = f64_widen(p2);
    Pt<float> pf;  // the Jacobian at the predictor's midpoint
    rsc32<Q>(g, tb, i1, i2, 0.5f * (a1 + p1), 0.5f * (a2 + p2), pf);
    Local<float> Lf;
    local_full<Q>(g, pf, Lf);
    coord_jacobian(g, Lf, uf, m2f, J);
    {  // the double-float predictor step
      if (g.n_iter >= 2) {
        const DF ud[3] = {df_of(u[0]), df_of(u[1]), df_of(u[2])};
        const DF d1d = df_of(dx1), d2d = df_of(dx2);
        DF n1d, n2d, s1d, s2d;
        coord_map_df<Q>(g, tb, i1, i2, d1d, d2d, ud, DF(m2f), DF(p1), DF(p2), n1d, n2d);
        newton_df(J, DF(p1), DF(p2), n1d, n2d, s1d, s2d);
        s1 = df_to_double(s1d);
        s2 = df_to_double(s2d);
        df_start = finite64(s1) && finite64(s2);
      }
    }
  }
  if (!df_start) {
    coord_map64<Q>(g, b, i1, i2, dx1, dx2, u, m2, t1, t2, n1, n2, v3);
    newton_step(J, t1, t2, n1, n2, s1, s2);
  }
  bool conv = false;
  for (int it = 1; it < g.n_iter && !conv; ++it) {
    coord_map64<Q>(g, b, i1, i2, dx1, dx2, u, m2, s1, s2, n1, n2, v3);
    conv = converged(n1, s1, g.f_iter_tol) && converged(n2, s2, g.f_iter_tol);
    s1 = n1;
    s2 = n2;
  }
  t1 = s1;
  t2 = s2;
  if (!method_converges(d1, spectral_radius(J), g.n_iter, g.f_iter_tol, t1, t2)) {
    coord_exact<Q>(g, b, L, i1, i2, dx1, dx2, u, m2, t1, t2);  // the method's iterations
    v3 = NAN;
  }
}

// One particle in FP64: steps 2-11 of Sec. 3.1, the boundaries of Sec. 3.3.3, and
// (DEPOSIT) the deposit of its move. T is the storage type of state and fields. REFINE
// false compiles the refined iterations out (a caller whose particles all sit in the two
// cell rows next to an axis, where they never apply).
template <bool Q, typename T, bool DEPOSIT, bool REFINE = true>
__device__ __forceinline__ void push64(const GridP &g, const FieldPtrsT<T> &F,
                                       const PushTables &tb, const SpeciesDevT<T> &s,
                                       int64_t k, unsigned long long *diag) {
  const int i1 = s.i1[k], i2 = s.i2[k];
  const double dx1 = (double)s.dx1[k], dx2 = (double)s.dx2[k];
  const double x1 = i1 + dx1, x2 = i2 + dx2;
  const bool em = s.m2 != 0.0;  // massless particles skip the EM push (Sec. 3.1)
  const double settle = sizeof(T) == 4 ? SETTLE32 : 0.0;  // FP32 storage: see SETTLE32
  // the refined iterations keep two cell rows away from the axes: there the coordinate map
  // (metric terms ~ 1/sin^2(theta)) has more than one fixed point within reach, and the
  // method's answer is the one its iteration from x^n finds
  const bool refine = REFINE && g.iter_tol > 0.0 && i2 >= 2 && i2 < g.n_th - 2;
  const Base b = refine ? make_base_tab<Q>(g, tb, i1, i2, dx1, x1, x2) : make_base<Q>(g, x1, x2);
  Pt<double> p0;
  local_at_base<Q>(g, b, x2, p0);  // clamps theta near the axes
  Local<double> L;
  local_full<Q>(g, p0, L);
  double Bh[3], Dh[3], uh[3], u[3] = {(double)s.u1[k], (double)s.u2[k], (double)s.u3[k]};
  const double hq = s.qm * L.alpha * 0.5 * g.dt;
  if (em) {
    // step 2: fields at x^n
    double Bv[3], Dv[3];
    Lerp64 lw;
    lerp_setup(x1, x2, lw);
    Bv[0] = interp64(F.Bn[0], g.NX, lw, 0, 1);
    Bv[1] = interp64(F.Bn[1], g.NX, lw, 1, 0);
    Bv[2] = interp64(F.Bn[2], g.NX, lw, 1, 1);
    Dv[0] = interp64(F.D[0], g.NX, lw, 1, 0);
    Dv[1] = interp64(F.D[1], g.NX, lw, 0, 1);
    Dv[2] = interp64(F.D[2], g.NX, lw, 0, 0);
    // step 3: to the tetrad basis
    vec_hat(L, Bv, Bh);
    vec_hat(L, Dv, Dh);
    cov_hat(L, u, uh);
    boris(uh, Dh, Bh, hq);     // step 4
    hat_cov(L, uh, u);         // step 5
  }
  if (refine) geodesic_refined<Q>(g, tb, i1, i2, f32_trunc(dx1), f32_trunc(dx2), L, u, s.m2);
  else geodesic_momentum_settle(g, L, u, s.m2, settle);  // step 6
  if (em) {
    cov_hat(L, u, uh);         // step 7
    boris(uh, Dh, Bh, hq);     // step 8
    hat_cov(L, uh, u);         // step 9
  }
  // step 10: implicit coordinate push, Eq. (discretized-geodesic-x)
  double t1 = dx1, t2 = dx2, v3r = NAN;
  if (refine) coord_refined<Q>(g, tb, b, L, i1, i2, dx1, dx2, u, s.m2, t1, t2, v3r);
  else coord_exact<Q>(g, b, L, i1, i2, dx1, dx2, u, s.m2, t1, t2, settle);
  if (!(finite64(u[0]) && finite64(u[1]) && finite64(u[2]) && abs_lt(t1, 1e6) &&
        abs_lt(t2, 1e6))) {
    s.tag[k] = 0;
    count(diag, DG_NONFINITE);
    return;
  }
  const double f1 = floor(t1), f2 = floor(t2);
  int j1 = i1 + (int)f1, j2 = i2 + (int)f2;
  double e1 = t1 - f1, e2 = t2 - f2;
  // boundaries (Sec. 3.3.3): reflection off the axes, removal into the ghost zone
  if (j2 < 0) { j2 = 0; e2 = 1.0 - e2; u[1] = -u[1]; count(diag, DG_REFLECT); }
  else if (j2 >= g.n_th) { j2 = g.n_th - 1; e2 = 1.0 - e2; u[1] = -u[1]; count(diag, DG_REFLECT); }
  if (j2 < 0 || j2 >= g.n_th) {
    s.tag[k] = 0;
    count(diag, DG_NONFINITE);
    return;
  }
  s.i1[k] = j1; s.i2[k] = j2; s.dx1[k] = (T)e1; s.dx2[k] = (T)e2;
  s.u1[k] = (T)u[0]; s.u2[k] = (T)u[1]; s.u3[k] = (T)u[2];
  if (j1 < 0) { s.tag[k] = 2; count(diag, DG_LEFT_INNER); }
  else if (j1 >= g.n_r) { s.tag[k] = 2; count(diag, DG_LEFT_OUTER); }
  // step 11: phi at x^{n+1/2}, the midpoint of the stored x^n and the final x^{n+1}
  const double xb1 = j1 + e1, xb2 = j2 + e2;
  const double v3 = isnan(v3r)
      ? phi_rate64<Q>(g, b, 0.5 * __dadd_rn(x1, xb1), 0.5 * __dadd_rn(x2, xb2), u, s.m2) : v3r;
  s.phi[k] = (T)((double)s.phi[k] + g.dt * v3);
  if (DEPOSIT) deposit64(g, F, s.qc * (double)s.w[k], i1, i2, x1, x2, j1, j2, xb1, xb2, v3);
}

// =================================================================================
// FP32 routine (mixed precision, particles off the horizon and axis guard zones).
// Positions stay cell + offset: every coordinate is handled relative to the start cell,
// r and sin/cos(theta) come from FP64-computed per-cell tables and short Taylor series
// of the offset from the cell corner, so FP32 keeps its relative accuracy at any cell
// index and next to theta = pi.
// =================================================================================
// The guard-zone form of rsc32: r, sin and cos in FP64 from the FP64 corner tables, with
// theta clamped to [small_angle, pi - small_angle] as in the FP64 routine.
template <bool Q = true>
__device__ __forceinline__ void rsc64(const GridP &g, const PushTables &tb, int i, int j,
                                      float o1, float o2, Pt<double> &p) {
  const double e = (double)o1 * g.dxi;
  const double ex = fabs(e) <= 0.05 ? __ldg(tb.r64 + i + G_) * exp_small(e)  // < 1e-15
                                    : map_e(g, (double)i + (double)o1);
  p.r = Q ? g.r0 + ex : ex;
  p.f = g.dxi * ex;
  double d = (double)o2 * g.dth;  // the offset in eta, then in theta
  double th;
  if (Q && g.qks) {
    const double x2 = (double)j + (double)o2;
    map_g<Q>(g, x2, p.gg, p.gp);
    th = map_theta<Q>(g, x2);
    const double t1 = __ldg(tb.t1_64 + j + G_), t2 = __ldg(tb.t2_64 + j + G_);
    d = d * fma(d, fma(g.c3, d, t2), t1);
  } else {
    p.gg = g.dth;
    p.igg = g.ig2;
    p.gp = 0.0;
    th = ((double)j + (double)o2) * g.dth;
  }
  double &s = p.s, &c = p.c;
  if (th < g.small_angle || th > GRPIC_PI - g.small_angle) {
    sincos(fmin(fmax(th, g.small_angle), GRPIC_PI - g.small_angle), &s, &c);
  } else if (fabs(d) <= 0.1) {
    const double q = d * d;  // Taylor series to d^9 and d^10: truncation below 3e-17
    double sp = 1.0 / 362880.0;
    sp = fma(sp, q, -1.0 / 5040.0);
    sp = fma(sp, q, 1.0 / 120.0);
    sp = fma(sp, q, -1.0 / 6.0);
    const double se = fma(sp * q, d, d);
    double cp = -1.0 / 3628800.0;
    cp = fma(cp, q, 1.0 / 40320.0);
    cp = fma(cp, q, -1.0 / 720.0);
    cp = fma(cp, q, 1.0 / 24.0);
    cp = fma(cp, q, -0.5);
    const double ce = fma(cp, q, 1.0);
    const double s0 = __ldg(tb.s64 + j + G_), c0 = __ldg(tb.c64 + j + G_);
    s = fma(s0, ce, c0 * se);
    c = fma(c0, ce, -s0 * se);
  } else {
    sincos(th, &s, &c);
  }
}

// FP64 metric values rounded for the FP32 arithmetic of the guard zones
__device__ __forceinline__ void narrow(const Geo<double> &a, Geo<float> &b) {
  b.H11 = (float)a.H11; b.H13 = (float)a.H13; b.H22 = (float)a.H22; b.H33 = (float)a.H33;
  b.beta1 = (float)a.beta1; b.opz = (float)a.opz;
}
__device__ __forceinline__ void narrow(const Local<double> &a, Local<float> &b) {
  b.alpha = (float)a.alpha;
  narrow(a.G, b.G);
  b.d1H11 = (float)a.d1H11; b.d1H22 = (float)a.d1H22; b.d1H33 = (float)a.d1H33;
  b.d1H13 = (float)a.d1H13; b.d1alpha = (float)a.d1alpha; b.d1beta1 = (float)a.d1beta1;
  b.d2H11 = (float)a.d2H11; b.d2H22 = (float)a.d2H22; b.d2H33 = (float)a.d2H33;
  b.d2H13 = (float)a.d2H13; b.d2alpha = (float)a.d2alpha; b.d2beta1 = (float)a.d2beta1;
  b.rH11 = (float)a.rH11; b.sH11 = (float)a.sH11; b.rh22 = (float)a.rh22;
  b.sh22 = (float)a.sh22; b.rh33 = (float)a.rh33; b.sh33 = (float)a.sh33;
  b.k13 = (float)a.k13; b.m13 = (float)a.m13;
}

// The contravariant metric, shift and 1 + z at a cell-relative point, evaluated in FP64
// (G64: guard zones) or in FP32, as FP32 values.
template <bool Q, bool G64>
__device__ __forceinline__ void geo_at(const GridP &g, const PushTables &tb, int i, int j,
                                       float o1, float o2, Geo<float> &o) {
  if constexpr (G64) {
    Pt<double> p;
    rsc64<Q>(g, tb, i, j, o1, o2, p);
    Geo<double> od;
    geo_from_rsc<Q>(g, p, od);
    narrow(od, o);
  } else {
    Pt<float> p;
    rsc32<Q>(g, tb, i, j, o1, o2, p);
    geo_from_rsc<Q>(g, p, o);
  }
}

// bilinear interpolation from the cell-relative position (i, o) for a Yee offset (s1, s2),
// in a plane of row stride `stride` whose element (0, 0) is cell (0, 0) of the indices given
// (read through the read-only data path from global memory, or plainly from shared memory)
template <bool SMEM>
__device__ __forceinline__ float interp_gen(const float *__restrict__ pl, int stride, int i1,
                                            int i2, float o1, float o2, float s1, float s2) {
  const float y1 = o1 - s1, y2 = o2 - s2;
  const float f1 = floorf(y1), f2 = floorf(y2);
  const int i0 = i1 + (int)f1, j0 = i2 + (int)f2;
  const float w1 = y1 - f1, w2 = y2 - f2;
  const float *p = pl + (int64_t)j0 * stride + i0;
  float p00, p10, p01, p11;
  if constexpr (SMEM) {
    p00 = p[0]; p10 = p[1]; p01 = p[stride]; p11 = p[stride + 1];
  } else {
    p00 = __ldg(p); p10 = __ldg(p + 1); p01 = __ldg(p + stride); p11 = __ldg(p + stride + 1);
  }
  const float a = fmaf(w1, p10 - p00, p00);
  const float b = fmaf(w1, p11 - p01, p01);
  return fmaf(w2, b - a, a);
}

// The fields of the push: B^n and D planes in global memory ...
struct GlobalFields {
  const float *pl[6];  // Bn1..3, D1..3, shifted so that index (j, i) is cell (i, j)
  int NX;
  __device__ __forceinline__ GlobalFields(const GridP &g, const FieldPtrsT<float> &F) : NX(g.NX) {
    const int64_t o = (int64_t)G_ * g.NX + G_;
    for (int c = 0; c < 3; ++c) {
      pl[c] = F.Bn[c] + o;
      pl[3 + c] = F.D[c] + o;
    }
  }
  __device__ __forceinline__ float at(int c, int i1, int i2, float o1, float o2, float s1,
                                      float s2) const {
    return interp_gen<false>(pl[c], NX, i1, i2, o1, o2, s1, s2);
  }
};
// ... or a shared-memory window of W1 x W2 nodes whose node (0, 0) is cell (iw0, jw0)
struct WindowFields {
  const float *win;  // 6 planes of W1 * W2
  int W1, plane, iw0, jw0;
  __device__ __forceinline__ float at(int c, int i1, int i2, float o1, float o2, float s1,
                                      float s2) const {
    return interp_gen<true>(win + c * plane, W1, i1 - iw0, i2 - jw0, o1, o2, s1, s2);
  }
};

// One move of the mixed path, relative to its start cell (ia, ja): from (a1, a2) in [0, 1]^2
// to (b1, b2) in cell (ia + di, ja + dj), charge weight q and dphi/dt v3 at the midpoint.
struct Move32 {
  int ia, ja, di, dj;
  float a1, a2, b1, b2, q, v3;
};

// The zigzag deposit of a move (Sec. 3.2, Eq. charge-conservation-disc; Umeda et al. 2003)
// as three groups of four contributions, each group belonging to one cell: the segment in
// the start cell and the segment in the end cell (J1 at (i, j) and (i, j+1), J2 at (i, j) and
// (i+1, j) of that cell, as the plane stores edges), and J3 = q v3 at the four corners
// around the midpoint. cell[g] is the plane index of group g's cell.
__device__ __forceinline__ void zigzag32(const GridP &g, const Move32 &m, float c[3][4],
                                         int cell[3]) {
  const float idt = g.f_idt, q = m.q;
  const float r1 = fminf((float)min(0, m.di) + 1.0f, fmaxf((float)max(0, m.di), 0.5f * (m.a1 + m.b1)));
  const float r2 = fminf((float)min(0, m.dj) + 1.0f, fmaxf((float)max(0, m.dj), 0.5f * (m.a2 + m.b2)));
  {
    const float F1 = q * (r1 - m.a1) * idt, F2 = q * (r2 - m.a2) * idt;
    const float W1 = 0.5f * (m.a1 + r1), W2 = 0.5f * (m.a2 + r2);
    c[0][0] = F1 * (1.0f - W2); c[0][1] = F1 * W2; c[0][2] = F2 * (1.0f - W1); c[0][3] = F2 * W1;
    cell[0] = (int)sidx(g, m.ia, m.ja);
  }
  {
    const float F1 = q * (m.b1 - r1) * idt, F2 = q * (m.b2 - r2) * idt;
    const float W1 = 0.5f * (r1 + m.b1) - (float)m.di, W2 = 0.5f * (r2 + m.b2) - (float)m.dj;
    c[1][0] = F1 * (1.0f - W2); c[1][1] = F1 * W2; c[1][2] = F2 * (1.0f - W1); c[1][3] = F2 * W1;
    cell[1] = (int)sidx(g, m.ia + m.di, m.ja + m.dj);
  }
  const float m1 = 0.5f * (m.a1 + m.b1), m2 = 0.5f * (m.a2 + m.b2);
  const float f1 = floorf(m1), f2 = floorf(m2);
  const float w1 = m1 - f1, w2 = m2 - f2, qv = q * m.v3;
  c[2][0] = qv * (1.0f - w1) * (1.0f - w2); c[2][1] = qv * w1 * (1.0f - w2);
  c[2][2] = qv * (1.0f - w1) * w2;          c[2][3] = qv * w1 * w2;
  cell[2] = (int)sidx(g, m.ia + (int)f1, m.ja + (int)f2);
}

// Where the deposit goes: the current planes in global memory ...
struct GlobalSink {
  float *J[3];
  int NX;
  __device__ __forceinline__ GlobalSink(const GridP &g, const FieldPtrsT<float> &F) : NX(g.NX) {
    for (int c = 0; c < 3; ++c) J[c] = F.J[c];
  }
  __device__ __forceinline__ void add(int grp, int k, const float c[4]) const {
    if (grp < 2) {
      atomicAdd(J[0] + k, c[0]);
      atomicAdd(J[0] + k + NX, c[1]);
      atomicAdd(J[1] + k, c[2]);
      atomicAdd(J[1] + k + 1, c[3]);
    } else {
      atomicAdd(J[2] + k, c[0]);
      atomicAdd(J[2] + k + 1, c[1]);
      atomicAdd(J[2] + k + NX, c[2]);
      atomicAdd(J[2] + k + NX + 1, c[3]);
    }
  }
};
// ... or a shared-memory window (as WindowFields) flushed to global memory by the caller;
// a group whose four targets are not all inside it goes to global memory directly
struct WindowSink {
  GlobalSink glob;
  float *win;  // 3 planes of W1 * W2
  int W1, W2, plane, iw0, jw0;
  __device__ __forceinline__ void add(int grp, int k, const float c[4]) const {
    const int j = k / glob.NX - G_, i = k - (j + G_) * glob.NX - G_;
    const int wi = i - iw0, wj = j - jw0;
    if (wi < 0 || wj < 0 || wi > W1 - 2 || wj > W2 - 2) {
      glob.add(grp, k, c);
      return;
    }
    float *w = win + wj * W1 + wi;
    if (grp < 2) {
      atomicAdd(w, c[0]);
      atomicAdd(w + W1, c[1]);
      atomicAdd(w + plane, c[2]);
      atomicAdd(w + plane + 1, c[3]);
    } else {
      w += 2 * plane;
      atomicAdd(w, c[0]);
      atomicAdd(w + 1, c[1]);
      atomicAdd(w + W1, c[2]);
      atomicAdd(w + W1 + 1, c[3]);
    }
  }
};

// Sums of v over runs of equal keys in consecutive lanes (all 32 lanes call it): a suffix
// scan bounded by the next run head, so the first lane of each run ends with the run's sum.
// Returns whether this lane heads a run.
__device__ __forceinline__ bool run_sums(int key, float v[4]) {
  constexpr unsigned FULL = 0xffffffffu;
  const int lane = threadIdx.x & 31;
  const int kp = __shfl_up_sync(FULL, key, 1);
  const bool head = lane == 0 || kp != key;
  const unsigned H = __ballot_sync(FULL, head);
  if (H == FULL) return true;  // no two neighbouring lanes share a cell
  const unsigned above = lane == 31 ? 0u : (H & (FULL << (lane + 1)));
  const int nh = above ? __ffs(above) - 1 : 32;  // first lane of the next run
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const float o = __shfl_down_sync(FULL, v[q], d);
      if (lane + d < nh) v[q] += o;
    }
  }
  return head;
}

// Warp-cooperative deposit (every lane of the warp calls it; on = false where a lane has no
// move): per group, contributions to the same cell from consecutive lanes are summed with
// shuffles (particles are kept sorted by cell, so a warp holds few runs) and the first lane
// of each run issues the four atomics. A move that stays in its cell has both segments in
// that cell; they are added before the reduction.
template <class Sink>
__device__ __forceinline__ void deposit32_warp(const GridP &g, const Sink &sink,
                                               const Move32 &m, bool on) {
  float c[3][4];
  int cell[3] = {-1, -1, -1};
  if (on) {
    zigzag32(g, m, c, cell);
    if (cell[1] == cell[0]) {
#pragma unroll
      for (int q = 0; q < 4; ++q) c[0][q] += c[1][q];
      cell[1] = -1;
    }
  } else {
#pragma unroll
    for (int grp = 0; grp < 3; ++grp)
#pragma unroll
      for (int q = 0; q < 4; ++q) c[grp][q] = 0.0f;
  }
#pragma unroll
  for (int grp = 0; grp < 3; ++grp) {
    if (!__any_sync(0xffffffffu, cell[grp] >= 0)) continue;
    const bool head = run_sums(cell[grp], c[grp]);
    if (head && cell[grp] >= 0) sink.add(grp, cell[grp], c[grp]);
  }
}


// The FP32 momentum substep: n_iter applications of the geodesic map, or fewer under the
// stop rule above.
__device__ __forceinline__ void geodesic_momentum32(const GridP &g, const Local<float> &L,
                                                    float u[3], float m2) {
  const GeoMap<float> m(g, L, u, m2);
  float t0 = u[0], t1 = u[1];
  for (int it = 0; it < g.n_iter; ++it) {
    float n0, n1;
    m.apply(t0, t1, n0, n1);
    const bool done = settled32(n0, t0, n1, t1);
    t0 = n0;
    t1 = n1;
    if (done && g.stop_on_repeat) break;
  }
  u[0] = t0;
  u[1] = t1;
}

template <bool Q, bool G64>
__device__ __forceinline__ float phi_rate32(const GridP &g, const PushTables &tb, int i, int j,
                                            float o1, float o2, const float u[3], float m2) {
  Geo<float> o;
  geo_at<Q, G64>(g, tb, i, j, o1, o2, o);
  const float q = fmaf(o.H11 * u[0], u[0], fmaf(o.H22 * u[1], u[1],
                  fmaf(o.H33 * u[2], u[2], fmaf(o.H13, 2.0f * u[0] * u[2], m2))));
  return rsqrtf(o.opz * q) * fmaf(o.H13, u[0], o.H33 * u[2]);
}

// One particle of the mixed path: steps 2-11 of Sec. 3.1 in FP32 with the metric, lapse
// and shift evaluated in FP32 (G64 false: off the guard zones) or in FP64 (G64 true: guard
// zone 1). Returns false when the particle was dropped, else its move (for the deposit). The cell rows on the axes (zone 2) take the
// FP64 routine instead: there the FP32 rounding of the tetrad-frame momentum, about eps |u|,
// enters dphi/dt divided by r sin(theta), which has no lower bound in those rows; one row
// or more away sin(theta) >= dtheta and dt <= CFL r dtheta bound the phi error per step
// by about eps CFL.
template <bool Q, bool G64, class Fields>
__device__ __forceinline__ bool push32(const GridP &g, const Fields &F, const PushTables &tb,
                                       const SpeciesDevT<float> &s, int64_t k,
                                       unsigned long long *diag, Move32 &mv) {
  const int i1 = s.i1[k], i2 = s.i2[k];
  const float dx1 = s.dx1[k], dx2 = s.dx2[k];
  const bool em = s.f_m2 != 0.0f;  // massless particles skip the EM push (Sec. 3.1)
  Local<float> L;
  if constexpr (G64) {
    Pt<double> p;
    rsc64<Q>(g, tb, i1, i2, dx1, dx2, p);
    Local<double> Ld;
    local_full<Q>(g, p, Ld);
    narrow(Ld, L);
  } else {
    Pt<float> p;
    rsc32<Q>(g, tb, i1, i2, dx1, dx2, p);
    local_full<Q>(g, p, L);
  }
  float Bh[3], Dh[3], uh[3], u[3] = {s.u1[k], s.u2[k], s.u3[k]};
  const float hq = s.f_qm * L.alpha * 0.5f * g.f_dt;
  if (em) {
    float Bv[3], Dv[3];
    Bv[0] = F.at(0, i1, i2, dx1, dx2, 0.0f, 0.5f);
    Bv[1] = F.at(1, i1, i2, dx1, dx2, 0.5f, 0.0f);
    Bv[2] = F.at(2, i1, i2, dx1, dx2, 0.5f, 0.5f);
    Dv[0] = F.at(3, i1, i2, dx1, dx2, 0.5f, 0.0f);
    Dv[1] = F.at(4, i1, i2, dx1, dx2, 0.0f, 0.5f);
    Dv[2] = F.at(5, i1, i2, dx1, dx2, 0.0f, 0.0f);
    vec_hat(L, Bv, Bh);
    vec_hat(L, Dv, Dh);
    cov_hat(L, u, uh);
    boris(uh, Dh, Bh, hq);
    hat_cov(L, uh, u);
  }
  geodesic_momentum32(g, L, u, s.f_m2);
  if (em) {
    cov_hat(L, u, uh);
    boris(uh, Dh, Bh, hq);
    hat_cov(L, uh, u);
  }
  const float dt = g.f_dt;
  const float uu0 = 2.0f * u[0] * u[2];
  // the coordinate iteration under the FP32 stop rules; dphi/dt then comes from the metric of
  // its last iteration, whose midpoint is within half the final update of the final one. So
  // the rate rule also wants that update below ITER_TOL32 times the cells over which dphi/dt
  // changes by order one: the distance to the nearer axis in theta (dphi/dt ~ 1/sin^2(theta))
  // and 1/(4 dxi) in x1 (~ 1/r^2), which keeps its relative error at FP32 rounding
  const float d_cap = ITER_TOL32 * fminf((float)min(i2, g.n_th - 1 - i2), g.f_x1_scale);
  float t1 = dx1, t2 = dx2, v3 = NAN, d_prev = 0.0f;
  for (int it = 0; it < g.n_iter; ++it) {
    Geo<float> o;
    if (it == 0) o = L.G;
    else geo_at<Q, G64>(g, tb, i1, i2, 0.5f * (dx1 + t1), 0.5f * (dx2 + t2), o);
    const float q = fmaf(o.H11 * u[0], u[0], fmaf(o.H22 * u[1], u[1],
                    fmaf(o.H33 * u[2], u[2], fmaf(o.H13, uu0, s.f_m2))));
    const float ag = rsqrtf(o.opz * q);
    const float n1 = fmaf(dt, fmaf(ag, fmaf(o.H11, u[0], o.H13 * u[2]), -o.beta1), dx1);
    const float n2 = fmaf(dt, ag * o.H22 * u[1], dx2);
    const float d = fmaxf(fabsf(n1 - t1), fabsf(n2 - t2));
    const bool done = settled32(n1, t1, n2, t2) || (settled32_rate(d, d_prev) && d <= d_cap);
    d_prev = d;
    t1 = n1;
    t2 = n2;
    if (done && g.stop_on_repeat) {
      v3 = ag * fmaf(o.H13, u[0], o.H33 * u[2]);
      break;
    }
  }
  if (!(isfinite(u[0]) && isfinite(u[1]) && isfinite(u[2]) && isfinite(t1) && isfinite(t2) &&
        fabsf(t1) < 1e6f && fabsf(t2) < 1e6f)) {
    s.tag[k] = 0;
    count(diag, DG_NONFINITE);
    return false;
  }
  const float f1 = floorf(t1), f2 = floorf(t2);
  const int di = (int)f1;
  const int j1 = i1 + di;
  const int j2 = i2 + (int)f2;
  const float e1 = t1 - f1, e2 = t2 - f2;
  // off the axis rows a particle is at least one cell from either axis and moves less than
  // a cell per step (CFL), so no reflection happens here; guard anyway
  if (j2 < 0 || j2 >= g.n_th) {
    s.tag[k] = 0;
    count(diag, DG_NONFINITE);
    return false;
  }
  const int dj = j2 - i2;
  s.i1[k] = j1; s.i2[k] = j2; s.dx1[k] = e1; s.dx2[k] = e2;
  s.u1[k] = u[0]; s.u2[k] = u[1]; s.u3[k] = u[2];
  if (j1 < 0) { s.tag[k] = 2; count(diag, DG_LEFT_INNER); }
  else if (j1 >= g.n_r) { s.tag[k] = 2; count(diag, DG_LEFT_OUTER); }
  // phi at the midpoint, relative to the start cell (when the iteration ran to n_iter)
  const float b1 = (float)di + e1, b2 = (float)dj + e2;
  if (isnan(v3))
    v3 = phi_rate32<Q, G64>(g, tb, i1, i2, 0.5f * (dx1 + b1), 0.5f * (dx2 + b2), u, s.f_m2);
  s.phi[k] = fmaf(dt, v3, s.phi[k]);
  mv = Move32{i1, i2, di, dj, dx1, dx2, b1, b2, s.f_qc * s.w[k], v3};
  return true;
}

// 0: FP32 metric; 1: FP64 metric (within guard_j rows of an axis or guard cells of the
// horizon); 2: the cell rows on the axes, FP64 routine
__device__ __forceinline__ int guard_zone(const PushTables &tb, const GridP &g, int i1, int i2) {
  if (i2 == 0 || i2 == g.n_th - 1) return 2;
  return ((i1 >= tb.guard_ilo && i1 < tb.guard_ihi) || i2 < tb.guard_j ||
          i2 >= g.n_th - tb.guard_j) ? 1 : 0;
}

// FP64 path: one thread per particle, step 1 (previous location) then the FP64 routine.
// Bound by the FP64 pipe; on 67 M particles of the 2048^2 workload 3 resident blocks per SM
// (166 registers, no spills) measured 85.4 ms per launch against 86.9 ms with 4 (128
// registers, spills) and 89.3 ms with 5 (96 registers).
template <bool DEPOSIT, bool Q>
#ifndef GRPIC_PUSH64_MIN_BLOCKS  // resident blocks per SM the fused FP64 kernel is built for
#define GRPIC_PUSH64_MIN_BLOCKS 3
#endif
__global__ void __launch_bounds__(TPB, DEPOSIT ? GRPIC_PUSH64_MIN_BLOCKS : 3) k_push(GridP g, FieldPtrsT<double> F, PushTables tb,
                                              SpeciesDevT<double> s, unsigned long long *diag) {
  const int64_t n = *s.n;
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n;
       k += (int64_t)gridDim.x * blockDim.x) {
    if (s.i1p) {  // step 1: the previous position, when a later call reads it
      s.i1p[k] = s.i1[k]; s.i2p[k] = s.i2[k]; s.dx1p[k] = s.dx1[k]; s.dx2p[k] = s.dx2[k];
    }
    const uint8_t tag = s.tag[k];
    if (tag != 1) {
      if (tag != 0) s.tag[k] = 0;
      continue;
    }
    push64<Q, double, DEPOSIT>(g, F, tb, s, k, diag);
  }
}

// Mixed path, classification: zone 1 and zone 2 particles are appended to their lists
// (warp-aggregated) and marked in the mask, one word per 32 consecutive particles (bit k & 31
// of word k >> 5; a warp's 32 lanes cover one word). The kernel is bound by load latency, so
// each thread takes CL_U particles a grid stride apart and issues all their loads before
// using any; the loop is uniform over the warp (its first particle decides).
constexpr int CL_U = 8;
// one-warp blocks per SM of the zone-1 and zone-2 guard kernels (launch shape)
#ifndef GRPIC_GUARD_BLOCKS_PER_SM
#define GRPIC_GUARD_BLOCKS_PER_SM 8
#endif
#ifndef GRPIC_AXIS_BLOCKS_PER_SM
#define GRPIC_AXIS_BLOCKS_PER_SM 4
#endif
// their register caps as resident one-warp blocks per SM (65536 / (32 x this) registers):
// the registers they hold while resident are taken from the concurrent FP32 kernel. The
// zone-1 kernel capped at 80 (a few spills) left the FP32 kernel enough to make the mixed
// step 2% faster on GB300 than uncapped (119) or at 64; capping the zone-2 kernel cost more
// than it gave.
#ifndef GRPIC_GUARD_MIN_BLOCKS
#define GRPIC_GUARD_MIN_BLOCKS 24
#endif
#ifndef GRPIC_AXIS_MIN_BLOCKS
#define GRPIC_AXIS_MIN_BLOCKS 1
#endif
__global__ void __launch_bounds__(TPB) k_classify(GridP g, SpeciesDevT<float> s, PushTables tb,
                                                  GuardList gl) {
  const int64_t n = *s.n;
  const int lane = threadIdx.x & 31;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t w0 = blockIdx.x * (int64_t)blockDim.x + (threadIdx.x & ~31); w0 < n;
       w0 += CL_U * stride) {
    uint8_t tag[CL_U];
    int a[CL_U], b[CL_U];
#pragma unroll
    for (int q = 0; q < CL_U; ++q) {
      const int64_t k = w0 + q * stride + lane;
      tag[q] = 0;
      a[q] = b[q] = 0;
      if (k < n) {
        tag[q] = s.tag[k];
        a[q] = s.i1[k];
        b[q] = s.i2[k];
      }
    }
#pragma unroll
    for (int q = 0; q < CL_U; ++q) {
      const int64_t kw = w0 + q * stride;  // the warp's first particle
      if (kw >= n) break;
      const int zone = tag[q] == 1 ? guard_zone(tb, g, a[q], b[q]) : 0;
      const unsigned m1 = __ballot_sync(0xffffffffu, zone == 1);
      const unsigned m2 = __ballot_sync(0xffffffffu, zone == 2);
      if (lane == 0) gl.mask[kw >> 5] = m1 | m2;
      if (m1 | m2) {
        unsigned long long b1 = 0, b2 = 0;
        if (lane == 0) {
          if (m1) b1 = atomicAdd(gl.count, (unsigned long long)__popc(m1));
          if (m2) b2 = atomicAdd(gl.count + 1, (unsigned long long)__popc(m2));
        }
        b1 = __shfl_sync(0xffffffffu, b1, 0);
        b2 = __shfl_sync(0xffffffffu, b2, 0);
        const unsigned below = (1u << lane) - 1u;
        const uint32_t k = (uint32_t)(kw + lane);
        if (zone == 1) gl.idx[b1 + __popc(m1 & below)] = k;
        if (zone == 2) gl.idx[gl.cap - 1 - (int64_t)(b2 + __popc(m2 & below))] = k;
      }
    }
  }
}

// Mixed path, FP32 kernel: step 1 and the FP32 routine for every unlisted particle (it runs
// concurrently with the guard kernels, which own the listed ones). The loop runs while the
// warp's first particle exists, so the whole warp reaches the cooperative deposit. Its
// gathers and atomics need many resident warps to hide their latency: 12 blocks per SM (40
// registers, spills) measured 0.60 ms per 8.4 M particles against 0.71 ms with 6 (80
// registers, no spills) on GB300, and on 67 M particles of the 2048^2 workload 10 blocks
// (48 registers, fewer spills) 3.22 ms against 3.29 ms with 12, 3.28 with 9 and 3.35 with
// 8; it is bound by instruction issue.
#ifndef GRPIC_PUSH32_MIN_BLOCKS  // resident blocks per SM the FP32 kernel is built for
#define GRPIC_PUSH32_MIN_BLOCKS 10
#endif
template <bool DEPOSIT, bool Q>
__global__ void __launch_bounds__(TPB, GRPIC_PUSH32_MIN_BLOCKS) k_push32(GridP g, FieldPtrsT<float> F,
                                                SpeciesDevT<float> s, PushTables tb,
                                                GuardList gl, unsigned long long *diag) {
  const int64_t n = *s.n;
  const int lane = threadIdx.x & 31;
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k - lane < n;
       k += (int64_t)gridDim.x * blockDim.x) {
    Move32 mv;
    bool on = false;
    if (k < n && !((__ldg(gl.mask + (k >> 5)) >> lane) & 1u)) {
      if (s.i1p) {
        s.i1p[k] = s.i1[k]; s.i2p[k] = s.i2[k]; s.dx1p[k] = s.dx1[k]; s.dx2p[k] = s.dx2[k];
      }
      const uint8_t tag = s.tag[k];
      if (tag == 1) on = push32<Q, false>(g, GlobalFields(g, F), tb, s, k, diag, mv);
      else if (tag != 0) s.tag[k] = 0;
    }
    if (DEPOSIT) deposit32_warp(g, GlobalSink(g, F), mv, on);
  }
}

// Mixed path, FP32 kernel on sort tiles: one CTA per tile pushes the particles that were in
// the tile at the last sort. The B^n and D planes of the tile and a halo of TILE_HALO cells
// are staged in shared memory; the deposit (after the warp reduction) accumulates in a
// shared-memory window of the same extent, flushed to global memory at the end. A particle
// whose cell has drifted out of the window gathers from, and deposits to, global memory.
// The window is loaded by the CTA's threads, or (TMA) by the tensor memory accelerator: one
// thread issues one bulk tensor copy per field plane, the others wait on an mbarrier.
constexpr int TILE_TPB = 256;

// floats per window plane in shared memory: W1 x W2 rounded up to 128 bytes (the tensor
// copies' destinations)
__host__ __device__ inline int window_plane(int W1, int W2) { return (W1 * W2 + 31) / 32 * 32; }

// The padded copy the tensor copies read: B^n and D ([NY][NX] each) into [6][NY][NXp], rows
// padded with zeros to NXp (a multiple of 4 floats, so every row starts on 16 bytes).
__global__ void __launch_bounds__(256) k_pad_fields(FieldPtrsT<float> F, float *pad, int NX,
                                                   int NY, int NXp) {
  const int64_t per = (int64_t)NY * NXp, n = 6 * per;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int c = (int)(t / per);
    const int64_t r = t - c * per;
    const int j = (int)(r / NXp), i = (int)(r - (int64_t)j * NXp);
    pad[t] = i < NX ? __ldg((c < 3 ? F.Bn[c] : F.D[c - 3]) + (int64_t)j * NX + i) : 0.0f;
  }
}

// The tile window by the tensor memory accelerator: thread 0 initialises the barrier, arms it
// with the window's bytes and issues one 3D tensor copy per field plane (a box of W1 x W2 x 1
// at column x0, row y0 of plane c of the padded copy; zeros outside it). Every thread then
// polls the barrier's phase 0 for at most about a second of clock cycles. Returns false when
// the copies did not complete (counted in the diagnostics, after a second bounded wait for
// them); the CTA then leaves its tile.
constexpr long long STAGE_WAIT_CYCLES = 2000000000ll;
__device__ __forceinline__ bool wait_phase0(uint32_t bar) {
  uint32_t done = 0;
  const long long t0 = clock64();
  while (!done && clock64() - t0 < STAGE_WAIT_CYCLES) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], 0;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(bar)
        : "memory");
  }
  return done != 0;
}
__device__ __forceinline__ bool stage_tma(const TileInfo &ti, float *fwin, int PL, int x0, int y0,
                                          int W1, int W2, uint64_t *barp,
                                          unsigned long long *diag) {
  const uint32_t bar = (uint32_t)__cvta_generic_to_shared(barp);
  if (threadIdx.x == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    const uint32_t bytes = 6u * (uint32_t)W1 * (uint32_t)W2 * 4u;
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes)
                 : "memory");
    const uint64_t map = reinterpret_cast<uint64_t>(&ti.map);
#pragma unroll
    for (int c = 0; c < 6; ++c) {
      const uint32_t dst = (uint32_t)__cvta_generic_to_shared(fwin + c * PL);
      asm volatile(
          "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
          " [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(dst),
          "l"(map), "r"(x0), "r"(y0), "r"(c), "r"(bar)
          : "memory");
    }
  }
  const bool ok = wait_phase0(bar);
  if (__syncthreads_or(!ok)) {
    if (threadIdx.x == 0) atomicAdd(diag + DG_STAGE_TIMEOUT, 1ull);
    wait_phase0(bar);  // the copies may still land: a second bounded wait before leaving
    return false;
  }
  return true;
}

template <bool DEPOSIT, bool Q, bool TMA>
__global__ void __launch_bounds__(TILE_TPB) k_push32_tiled(GridP g, FieldPtrsT<float> F,
                                                          SpeciesDevT<float> s, PushTables tb,
                                                          GuardList gl,
                                                          const __grid_constant__ TileInfo ti,
                                                          unsigned long long *diag) {
  extern __shared__ float sm_raw[];
  __shared__ __align__(8) uint64_t bar;
  // 128-byte aligned window planes (the launch adds the slack)
  float *sm = reinterpret_cast<float *>(
      (reinterpret_cast<uintptr_t>(sm_raw) + 127) & ~static_cast<uintptr_t>(127));
  const int t = blockIdx.x;
  const int tx = t % ti.ntr, ty = t / ti.ntr;
  const int W1 = ti.tr + 2 * TILE_HALO, W2 = ti.tt + 2 * TILE_HALO;
  const int plane = window_plane(W1, W2);
  const int iw0 = tx * ti.tr - TILE_HALO, jw0 = ty * ti.tt - TILE_HALO;
  float *fwin = sm, *jwin = sm + 6 * plane;
  if (DEPOSIT)
    for (int e = threadIdx.x; e < 3 * plane; e += blockDim.x) jwin[e] = 0.0f;
  if constexpr (TMA) {
    // window node (0, 0) is storage column iw0 + G, row jw0 + G (a multiple of 4 columns)
    if (!stage_tma(ti, fwin, plane, iw0 + G_, jw0 + G_, W1, W2, &bar, diag)) return;
  } else {
    // stage the fields (zero outside the stored planes)
    for (int e = threadIdx.x; e < 6 * W1 * W2; e += blockDim.x) {
      const int c = e / (W1 * W2), r = e - c * (W1 * W2), wj = r / W1, wi = r - wj * W1;
      const int i = iw0 + wi, j = jw0 + wj;
      float v = 0.0f;
      if (i >= -G_ && i < g.NX - G_ && j >= -G_ && j < g.NY - G_)
        v = __ldg((c < 3 ? F.Bn[c] : F.D[c - 3]) + sidx(g, i, j));
      fwin[c * plane + r] = v;
    }
  }
  __syncthreads();
  const WindowFields wf{fwin, W1, plane, iw0, jw0};
  const GlobalFields gf(g, F);
  const WindowSink ws{GlobalSink(g, F), jwin, W1, W2, plane, iw0, jw0};
  const int64_t begin = ti.start[t], end = ti.start[t + 1];
  const int lane = threadIdx.x & 31;
  for (int64_t k = begin + threadIdx.x; k - lane < end; k += blockDim.x) {
    Move32 mv;
    bool on = false;
    if (k < end && !((__ldg(gl.mask + (k >> 5)) >> (k & 31)) & 1u)) {
      if (s.i1p) {
        s.i1p[k] = s.i1[k]; s.i2p[k] = s.i2[k]; s.dx1p[k] = s.dx1[k]; s.dx2p[k] = s.dx2[k];
      }
      const uint8_t tag = s.tag[k];
      if (tag == 1) {
        // the interpolation reads cells i +- 1, j +- 1
        const int i1 = s.i1[k], i2 = s.i2[k];
        const bool inside = i1 - 1 >= iw0 && i1 + 1 < iw0 + W1 && i2 - 1 >= jw0 && i2 + 1 < jw0 + W2;
        on = inside ? push32<Q, false>(g, wf, tb, s, k, diag, mv)
                    : push32<Q, false>(g, gf, tb, s, k, diag, mv);
      } else if (tag != 0) {
        s.tag[k] = 0;
      }
    }
    if (DEPOSIT) deposit32_warp(g, ws, mv, on);
  }
  if (DEPOSIT) {
    __syncthreads();
    for (int e = threadIdx.x; e < 3 * plane; e += blockDim.x) {
      const int c = e / plane, r = e - c * plane;
      const float v = jwin[e];
      if (v != 0.0f && r < W1 * W2) {
        const int wj = r / W1, wi = r - wj * W1;
        atomicAdd(F.J[c] + sidx(g, iw0 + wi, jw0 + wj), v);
      }
    }
  }
}

size_t tiled_smem_bytes(const TileInfo &ti) {
  return (size_t)9 * window_plane(ti.tr + 2 * TILE_HALO, ti.tt + 2 * TILE_HALO) * sizeof(float) +
         128;
}

// Mixed path, guard kernels (side stream): step 1 and the routine of the listed particles,
// zone 1 with the metric in FP64, zone 2 with the FP64 routine.
template <bool DEPOSIT, bool Q>
__global__ void __launch_bounds__(32, GRPIC_GUARD_MIN_BLOCKS) k_push_guard(GridP g, FieldPtrsT<float> F,
                                                    SpeciesDevT<float> s, PushTables tb,
                                                    GuardList gl, unsigned long long *diag) {
  const int64_t n = (int64_t)gl.count[0];
  const int lane = threadIdx.x & 31;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t - lane < n;
       t += (int64_t)gridDim.x * blockDim.x) {
    Move32 mv;
    bool on = false;
    if (t < n) {
      const int64_t k = gl.idx[t];
      if (s.i1p) {
        s.i1p[k] = s.i1[k]; s.i2p[k] = s.i2[k]; s.dx1p[k] = s.dx1[k]; s.dx2p[k] = s.dx2[k];
      }
      on = push32<Q, true>(g, GlobalFields(g, F), tb, s, k, diag, mv);
    }
    if (DEPOSIT) deposit32_warp(g, GlobalSink(g, F), mv, on);
  }
}

template <bool DEPOSIT, bool Q>
__global__ void __launch_bounds__(32, GRPIC_AXIS_MIN_BLOCKS) k_push_axis(GridP g, FieldPtrsT<float> F,
                                                   SpeciesDevT<float> s, PushTables tb,
                                                   GuardList gl, unsigned long long *diag) {
  const int64_t n = (int64_t)gl.count[1];
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t k = gl.idx[gl.cap - 1 - t];
    if (s.i1p) {
      s.i1p[k] = s.i1[k]; s.i2p[k] = s.i2[k]; s.dx1p[k] = s.dx1[k]; s.dx2p[k] = s.dx2[k];
    }
    push64<Q, float, DEPOSIT, false>(g, F, tb, s, k, diag);  // axis rows: never refined
  }
}

// Deposit from stored previous and new positions (grpic_deposit).
template <typename T>
__global__ void __launch_bounds__(TPB) k_deposit(GridP g, FieldPtrsT<T> F, SpeciesDevT<T> s,
                                                 PushTables tb) {
  const int64_t n = *s.n;
  const int lane = threadIdx.x & 31;
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k - lane < n;
       k += (int64_t)gridDim.x * blockDim.x) {
    const bool live = k < n && s.tag[k] != 0;
    int ia = 0, ja = 0, ib = 0, jb = 0, zone = 2;
    if (live) {
      ia = s.i1p[k]; ja = s.i2p[k]; ib = s.i1[k]; jb = s.i2[k];
      if constexpr (sizeof(T) == 4) zone = guard_zone(tb, g, ia, ja);
    }
    if constexpr (sizeof(T) == 4) {  // zones 0 and 1: the FP32 deposit of the mixed path
      Move32 mv;
      const bool on = live && zone < 2;
      if (on) {
        const float a1 = s.dx1p[k], a2 = s.dx2p[k];
        const float b1 = (float)(ib - ia) + s.dx1[k], b2 = (float)(jb - ja) + s.dx2[k];
        const float u[3] = {s.u1[k], s.u2[k], s.u3[k]};
        const float m1 = 0.5f * (a1 + b1), m2 = 0.5f * (a2 + b2);
        const float v3 = zone ? phi_rate32<true, true>(g, tb, ia, ja, m1, m2, u, s.f_m2)
                              : phi_rate32<true, false>(g, tb, ia, ja, m1, m2, u, s.f_m2);
        mv = Move32{ia, ja, ib - ia, jb - ja, a1, a2, b1, b2, s.f_qc * s.w[k], v3};
      }
      deposit32_warp(g, GlobalSink(g, F), mv, on);
    }
    if (live && zone == 2) {  // FP64 path, and the axis rows of the mixed path
      const double xa1 = ia + (double)s.dx1p[k], xa2 = ja + (double)s.dx2p[k];
      const double xb1 = ib + (double)s.dx1[k], xb2 = jb + (double)s.dx2[k];
      const double u[3] = {(double)s.u1[k], (double)s.u2[k], (double)s.u3[k]};
      const Base b = make_base(g, xa1, xa2);
      const double v3 = phi_rate64(g, b, 0.5 * __dadd_rn(xa1, xb1), 0.5 * __dadd_rn(xa2, xb2), u,
                                   s.m2);
      deposit64(g, F, s.qc * (double)s.w[k], ia, ja, xa1, xa2, ib, jb, xb1, xb2, v3);
    }
  }
}

// Loading of particles [k0, k0 + n) from FP64 device inputs (cell indices already in
// place): u_i = e_i^j u_j^ at the particle (App. A), w = w0 r^{-k} sqrt(h)(x_p); FP64.
template <typename T>
__global__ void k_load(GridP g, SpeciesDevT<T> s, int64_t k0, int64_t n, const double *dx1,
                       const double *dx2, const double *uh1, const double *uh2,
                       const double *uh3, const double *w0, double dpow) {
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t k = k0 + t;
    const double x1 = s.i1[k] + dx1[t], x2 = s.i2[k] + dx2[t];
    MetricV m;
    metric_eval<false>(g, x1, x2, true, m, nullptr);
    const double uh[3] = {uh1[t], uh2[t], uh3[t]};
    double u[3];
    t_hat_to_cov(m, uh, u);
    s.dx1[k] = (T)dx1[t]; s.dx2[k] = (T)dx2[t];
    s.u1[k] = (T)u[0]; s.u2[k] = (T)u[1]; s.u3[k] = (T)u[2];
    MetricV m0;
    metric_eval<false>(g, x1, x2, false, m0, nullptr);
    const double r = g.r0 + map_e(g, x1);
    s.w[k] = (T)(w0[t] * pow(r, -dpow) * m0.sqrt_h);
    s.phi[k] = (T)0;
    s.tag[k] = 1;
    s.i1p[k] = s.i1[k]; s.i2p[k] = s.i2[k]; s.dx1p[k] = s.dx1[k]; s.dx2p[k] = s.dx2[k];
  }
}

// Conserved energy and angular momentum per unit mass (Sec. 2.3), E = -u_0 - qm A_0,
// L = u_3 + qm A_3, u_0 = -alpha gamma + beta^1 u_1, at the midpoint of the previous and
// current positions (Sec. 4.1 takes the position at the velocity time level); FP64.
template <typename T>
__global__ void k_invariants(GridP g, SpeciesDevT<T> s, int kind, double B0, double *E,
                             double *Lout) {
  const int64_t n = *s.n;
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n;
       k += (int64_t)gridDim.x * blockDim.x) {
    const double x1 = 0.5 * ((s.i1[k] + (double)s.dx1[k]) + (s.i1p[k] + (double)s.dx1p[k]));
    const double x2 = 0.5 * ((s.i2[k] + (double)s.dx2[k]) + (s.i2p[k] + (double)s.dx2p[k]));
    MetricV m;
    metric_eval<false>(g, x1, x2, true, m, nullptr);
    const double u[3] = {(double)s.u1[k], (double)s.u2[k], (double)s.u3[k]};
    const double u0 = -m.alpha * gamma_of(m, u, s.m2) + m.beta1 * u[0];
    Pot p;
    p.A0 = p.A3 = 0.0;
    if (kind == GRPIC_FIELD_WALD || kind == GRPIC_FIELD_VERTICAL || kind == GRPIC_FIELD_MONOPOLE)
      potential(g, kind, B0, x1, x2, false, p);
    E[k] = -u0 - s.qm * p.A0;
    Lout[k] = u[2] + s.qm * p.A3;
  }
}

__global__ void k_push_tables(GridP g, PushTables tb) {
  const int n = max(g.NX, g.NY);
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < n; t += gridDim.x * blockDim.x) {
    if (t < g.NX) {  // exp(xi) = r - r0 at the corner column
      const double e = map_e(g, t - G_);
      const_cast<double *>(tb.r64)[t] = e;
      const_cast<float *>(tb.r)[t] = (float)e;
      const_cast<float2 *>(tb.r_df)[t] = make_float2((float)e, (float)(e - (double)(float)e));
    }
    if (t < g.NY) {
      double s, c;
      const double th = map_theta(g, t - G_);
      const_cast<double *>(tb.th64)[t] = th;
      sincos(th, &s, &c);
      const_cast<double *>(tb.s64)[t] = s;
      const_cast<double *>(tb.c64)[t] = c;
      const_cast<float2 *>(tb.s_df)[t] = make_float2((float)s, (float)(s - (double)(float)s));
      const_cast<float2 *>(tb.c_df)[t] = make_float2((float)c, (float)(c - (double)(float)c));
      const_cast<float *>(tb.s)[t] = (float)s;
      const_cast<float *>(tb.c)[t] = (float)c;
      // theta(eta_j + d) - theta(eta_j) = d (t1 + d (t2 + d c3)): t1 = dtheta/deta at eta_j,
      // t2 = k (6 eta_j - 3 pi), k = 2 h0 / pi^2 (1 and 0 on the plain grid)
      const double eta = (t - G_) * g.dth, k = 2.0 * g.h0 / (GRPIC_PI * GRPIC_PI);
      const double t1 = 1.0 + k * (GRPIC_PI * GRPIC_PI - 6.0 * GRPIC_PI * eta + 6.0 * eta * eta);
      const double t2 = k * (6.0 * eta - 3.0 * GRPIC_PI);
      const_cast<double *>(tb.t1_64)[t] = t1;
      const_cast<double *>(tb.t2_64)[t] = t2;
      const_cast<float *>(tb.t1)[t] = (float)t1;
      const_cast<float *>(tb.t2)[t] = (float)t2;
      const_cast<float2 *>(tb.t1_df)[t] = make_float2((float)t1, (float)(t1 - (double)(float)t1));
      const_cast<float2 *>(tb.t2_df)[t] = make_float2((float)t2, (float)(t2 - (double)(float)t2));
    }
  }
}

int blocks_for(int64_t n) {
  int64_t b = (n + TPB - 1) / TPB;
  const int64_t cap = 152 * 64;
  if (b > cap) b = cap;
  return (int)(b < 1 ? 1 : b);
}

}  // namespace

cudaError_t launch_push_tables(const GridP &g, const PushTables &tb, cudaStream_t st) {
  k_push_tables<<<8, 256, 0, st>>>(g, tb);
  COUNT_LAUNCH(1);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_load(const GridP &g, SpeciesDevT<T> s, int64_t k0, int64_t n,
                        const grpic_particle_init &in, double dpow, cudaStream_t st) {
  if (n <= 0) return cudaGetLastError();
  k_load<T><<<blocks_for(n), TPB, 0, st>>>(g, s, k0, n, in.dx1, in.dx2, in.uh1, in.uh2, in.uh3,
                                           in.w0, dpow);
  COUNT_LAUNCH(1);
  return cudaGetLastError();
}

// the push kernels for a grid kind known at compile time (Q: quasi-spherical)
template <typename T, bool Q>
cudaError_t push_impl(const GridP &g, const FieldPtrsT<T> &F, SpeciesDevT<T> s,
                      const PushTables &tb, const GuardList &gl, const TileInfo &ti,
                      int64_t n_bound, bool deposit, unsigned long long *diag,
                      const PushStreams &ps) {
  const bool main_stage = push_main_stage(ps.stage);
  const bool classify_stage = push_classify_stage(ps.stage);
  const bool kernels_stage = push_guard_kernels_stage(ps.stage);
  if (n_bound <= 0) {  // keep a requested event pair recorded (zero duration)
    if (main_stage && ps.t0) cudaEventRecord(ps.t0, ps.main);
    if (main_stage && ps.t1) cudaEventRecord(ps.t1, ps.main);
    return cudaGetLastError();
  }
  if constexpr (sizeof(T) == 8) {
    if (!main_stage) return cudaSuccess;  // the FP64 path has no guard stage
    if (ps.t0) cudaEventRecord(ps.t0, ps.main);
    if (deposit) k_push<true, Q><<<blocks_for(n_bound), TPB, 0, ps.main>>>(g, F, tb, s, diag);
    else k_push<false, Q><<<blocks_for(n_bound), TPB, 0, ps.main>>>(g, F, tb, s, diag);
    if (ps.t1) cudaEventRecord(ps.t1, ps.main);
    COUNT_LAUNCH(1);
  } else {
    cudaError_t e;
    const int nb = blocks_for(n_bound);
    if (classify_stage || kernels_stage) {
      // each part runs on the side stream after everything issued so far on main (the
      // classify reads only the particles, so a step may issue it before the field predict;
      // the guard kernels read the predicted fields and add to the zeroed currents)
      if ((e = cudaEventRecord(ps.fork, ps.main)) != cudaSuccess) return e;
      if ((e = cudaStreamWaitEvent(ps.side, ps.fork, 0)) != cudaSuccess) return e;
    }
    if (classify_stage) {
      if ((e = cudaMemsetAsync(gl.count, 0, 2 * sizeof(unsigned long long), ps.side)) != cudaSuccess)
        return e;
      k_classify<<<blocks_for((n_bound + CL_U - 1) / CL_U), TPB, 0, ps.side>>>(g, s, tb, gl);
      if ((e = cudaEventRecord(ps.classified, ps.side)) != cudaSuccess) return e;
      COUNT_LAUNCH(1);
    }
    if (kernels_stage) {
      // the guard kernels are FP64-pipe bound: a few one-warp blocks per SM reach every SM
      // sub-partition's FP64 unit and leave the registers to the concurrent FP32 kernel
      constexpr int gb = 152 * GRPIC_GUARD_BLOCKS_PER_SM, ab = 152 * GRPIC_AXIS_BLOCKS_PER_SM;
      if (deposit) {
        k_push_guard<true, Q><<<gb, 32, 0, ps.side>>>(g, F, s, tb, gl, diag);
        k_push_axis<true, Q><<<ab, 32, 0, ps.side>>>(g, F, s, tb, gl, diag);
      } else {
        k_push_guard<false, Q><<<gb, 32, 0, ps.side>>>(g, F, s, tb, gl, diag);
        k_push_axis<false, Q><<<ab, 32, 0, ps.side>>>(g, F, s, tb, gl, diag);
      }
      if ((e = cudaEventRecord(ps.done, ps.side)) != cudaSuccess) return e;
      COUNT_LAUNCH(2);
    }
    if (!main_stage) return cudaGetLastError();
    // the FP32 kernel reads the mask the classify writes
    if ((e = cudaStreamWaitEvent(ps.main, ps.classified, 0)) != cudaSuccess) return e;
    // the tiled kernel needs the tile ranges of a sort and a window that fits in shared memory
    const size_t smem = tiled_smem_bytes(ti);
    const bool tiled = ti.start != nullptr && smem <= 200 * 1024;
    if (tiled && smem > 48 * 1024) {
      void (*const kern[4])(GridP, FieldPtrsT<float>, SpeciesDevT<float>, PushTables, GuardList,
                            const TileInfo, unsigned long long *) = {
          k_push32_tiled<true, Q, false>, k_push32_tiled<false, Q, false>,
          k_push32_tiled<true, Q, true>, k_push32_tiled<false, Q, true>};
      for (auto *f : kern)
        if ((e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)smem)) != cudaSuccess) return e;
    }
    if (tiled && ti.tma) {  // the padded copy the tensor copies read
      k_pad_fields<<<152 * 8, 256, 0, ps.main>>>(F, ti.pad, g.NX, g.NY, ti.NXp);
      COUNT_LAUNCH(1);
    }
    if (ps.t0) cudaEventRecord(ps.t0, ps.main);
    if (tiled && ti.tma) {
      if (deposit)
        k_push32_tiled<true, Q, true><<<ti.n_tiles, TILE_TPB, smem, ps.main>>>(g, F, s, tb, gl, ti, diag);
      else
        k_push32_tiled<false, Q, true><<<ti.n_tiles, TILE_TPB, smem, ps.main>>>(g, F, s, tb, gl, ti, diag);
    } else if (tiled) {
      if (deposit)
        k_push32_tiled<true, Q, false><<<ti.n_tiles, TILE_TPB, smem, ps.main>>>(g, F, s, tb, gl, ti, diag);
      else
        k_push32_tiled<false, Q, false><<<ti.n_tiles, TILE_TPB, smem, ps.main>>>(g, F, s, tb, gl, ti, diag);
    } else {
      if (deposit) k_push32<true, Q><<<nb, TPB, 0, ps.main>>>(g, F, s, tb, gl, diag);
      else k_push32<false, Q><<<nb, TPB, 0, ps.main>>>(g, F, s, tb, gl, diag);
    }
    if (ps.t1) cudaEventRecord(ps.t1, ps.main);
    COUNT_LAUNCH(1);
  }
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_push(const GridP &g, const FieldPtrsT<T> &F, SpeciesDevT<T> s,
                        const PushTables &tb, const GuardList &gl, const TileInfo &ti,
                        int64_t n_bound, bool deposit, unsigned long long *diag,
                        const PushStreams &ps) {
  return g.qks ? push_impl<T, true>(g, F, s, tb, gl, ti, n_bound, deposit, diag, ps)
               : push_impl<T, false>(g, F, s, tb, gl, ti, n_bound, deposit, diag, ps);
}

template <typename T>
cudaError_t launch_deposit(const GridP &g, const FieldPtrsT<T> &F, SpeciesDevT<T> s,
                           const PushTables &tb, int64_t n_bound, cudaStream_t st) {
  if (n_bound <= 0) return cudaGetLastError();
  k_deposit<T><<<blocks_for(n_bound), TPB, 0, st>>>(g, F, s, tb);
  COUNT_LAUNCH(1);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_invariants(const GridP &g, SpeciesDevT<T> s, int kind, double B0, double *E,
                              double *L, int64_t n_bound, cudaStream_t st) {
  if (n_bound <= 0) return cudaGetLastError();
  k_invariants<T><<<blocks_for(n_bound), TPB, 0, st>>>(g, s, kind, B0, E, L);
  COUNT_LAUNCH(1);
  return cudaGetLastError();
}

#define INSTANTIATE_PARTICLES(T)                                                               \
  template cudaError_t launch_load<T>(const GridP &, SpeciesDevT<T>, int64_t, int64_t,        \
                                      const grpic_particle_init &, double, cudaStream_t);     \
  template cudaError_t launch_push<T>(const GridP &, const FieldPtrsT<T> &, SpeciesDevT<T>,    \
                                      const PushTables &, const GuardList &, const TileInfo &, \
                                      int64_t, bool, unsigned long long *,                     \
                                      const PushStreams &);                                    \
  template cudaError_t launch_deposit<T>(const GridP &, const FieldPtrsT<T> &, SpeciesDevT<T>, \
                                         const PushTables &, int64_t, cudaStream_t);           \
  template cudaError_t launch_invariants<T>(const GridP &, SpeciesDevT<T>, int, double,        \
                                            double *, double *, int64_t, cudaStream_t);
INSTANTIATE_PARTICLES(double)
INSTANTIATE_PARTICLES(float)
