// pusher.cuh -- the pieces of the GR pusher (Sec. 3.1 and App. A of arXiv:2511.17701)
// written once for an arithmetic type R: double (FP64 path, adjoint), float (mixed path) and
// the forward-mode dual numbers of the adjoint (dual.cuh). Included by particles.cu and
// adjoint.cu; everything is inline device code.
#pragma once
#include "dfloat.cuh"
#include "grpic_internal.cuh"

namespace {

// precision-generic math
__device__ __forceinline__ double fma_(double a, double b, double c) { return fma(a, b, c); }
__device__ __forceinline__ float fma_(float a, float b, float c) { return fmaf(a, b, c); }
__device__ __forceinline__ double rsqrt_(double a) { return rsqrt(a); }
__device__ __forceinline__ float rsqrt_(float a) { return rsqrtf(a); }
// ---------------------------------------------------------------------------------
// Conversions and tests on the integer pipe. GB300's FP64 pipe bounds the FP64 kernel and
// also executes the FP64 conversion, compare and min/max instructions; these bit-level forms
// keep such work off it where the exact FP64 semantics are not needed.
// ---------------------------------------------------------------------------------
// A double in FP32's normal range truncated toward zero to 24 significant bits; a signed
// zero below that range, a signed infinity above it, NaN kept. For the FP32 predictor's
// inputs and for stop tests, where a start point or a bound moves by less than 2^-23 of itself.
__device__ __forceinline__ float f32_trunc(double x) {
  const unsigned hi = (unsigned)__double2hiint(x), lo = (unsigned)__double2loint(x);
  const unsigned sign = hi & 0x80000000u, ex = (hi >> 20) & 0x7ffu;
  const int e = (int)ex - 896;  // rebias 1023 -> 127
  const unsigned m = ((hi & 0xfffffu) << 3) | (lo >> 29);
  unsigned r = sign | ((unsigned)e << 23) | m;
  if (e <= 0) r = sign;
  if (e >= 255) r = sign | 0x7f800000u | ((ex == 0x7ffu && (m | (lo & 0x1fffffffu))) ? 0x400000u : 0u);
  return __uint_as_float(r);
}
// The exact double of a normal float; zero and subnormals become a signed zero, inf and NaN
// are kept. For the FP32 predictor's results (FP64 start points) and the FP32 Newton
// coefficients, which only steer FP64 iterations that are checked in FP64.
__device__ __forceinline__ double f64_widen(float f) {
  const unsigned v = __float_as_uint(f);
  const unsigned sign = v & 0x80000000u, e = (v >> 23) & 0xffu, m = v & 0x7fffffu;
  unsigned hi = sign | ((e + 896u) << 20) | (m >> 3), lo = m << 29;
  if (e == 0u) hi = sign, lo = 0u;
  if (e == 255u) hi = sign | 0x7ff00000u | (m ? 0x80000u : 0u), lo = 0u;
  return __hiloint2double((int)hi, (int)lo);
}
// 1/b in FP64 by Newton-Raphson iteration on the reciprocal (y <- y + y (1 - b y), each
// step squaring the relative error) from an FP32 seed: b truncated to FP32 on the integer
// pipe, CUDA's fast FP32 reciprocal (within 2 ulp, so a seed error below 2^-21), two FP64
// steps (2^-42, then below the FP64 rounding): within about one ulp of the correctly rounded
// quotient in four FMAs. A b outside FP32's normal range takes the IEEE division.
__device__ __forceinline__ double rcp_nr(double b) {
  const unsigned ex = ((unsigned)__double2hiint(b) >> 20) & 0x7ffu;
  if (ex < 1023u - 125u || ex > 1023u + 126u) return 1.0 / b;
  const double y0 = f64_widen(__fdividef(1.0f, f32_trunc(b)));
  const double y1 = fma(y0, fma(-b, y0, 1.0), y0);
  return fma(y1, fma(-b, y1, 1.0), y1);
}

// a / b for the pusher's quotients (a = 1 or 2): in FP64 a times rcp_nr(b) (a power of two:
// exact); exact division for the adjoint's dual numbers; CUDA's fast FP32 division (within
// 2 ulp) in FP32, whose arithmetic carries ~1e-7 relative errors anyway
template <typename R>
__device__ __forceinline__ R div_(R a, R b) { return a / b; }
template <>
__device__ __forceinline__ double div_<double>(double a, double b) { return a * rcp_nr(b); }
template <>
__device__ __forceinline__ float div_<float>(float a, float b) { return __fdividef(a, b); }

}  // namespace

// the grid constants as float pairs (split on the host)
template <>
__device__ __forceinline__ Cst<DF> cst<DF>(const GridP &g) {
  return {DF(g.d_a[0], g.d_a[1]),     DF(g.d_M[0], g.d_M[1]),     DF(g.d_dxi[0], g.d_dxi[1]),
          DF(g.d_dth[0], g.d_dth[1]), DF(g.d_ig2[0], g.d_ig2[1]), DF(g.d_dt[0], g.d_dt[1]),
          DF(g.d_a2[0], g.d_a2[1]),   DF(g.d_M2[0], g.d_M2[1])};
}

namespace {
// a pair as a double: both parts widen exactly on the integer pipe, one FP64 add
__device__ __forceinline__ double df_to_double(DF a) { return f64_widen(a.hi) + f64_widen(a.lo); }

// =================================================================================
// Metric pieces shared by both precisions (App. A, quasi-spherical Kerr-Schild, mass M
// explicit). All reciprocals of one evaluation come from one division.
// =================================================================================

// A point of the grid: r, sin(theta), cos(theta) and the map's factors f = dr/dx1 =
// dxi (r - r0), gg = dtheta/dx2, gp = dgg/dx2, and igg = 1/gg^2 on the plain grid (gg =
// dtheta, gp = 0 there; on a quasi-spherical grid 1/gg^2 shares the metric's one division).
template <typename R>
struct Pt {
  R r, s, c, f, gg, igg, gp;
};

// The contravariant metric, shift and 1 + z = 1/alpha^2 at a point.
template <typename R>
struct Geo {
  R H11, H13, H22, H33, beta1, opz;
};
template <bool Q = true, typename R>
__device__ __forceinline__ void geo_from_rsc(const GridP &g, const Pt<R> &p, Geo<R> &o) {
  const Cst<R> k = cst<R>(g);
  const R a = k.a, a2 = k.a2, M2 = k.M2;
  const R r = p.r, s2 = p.s * p.s, r2 = r * r;
  const R Sig = fma_(a2, p.c * p.c, r2);
  const R S2 = fma_(M2, r, Sig);  // Sigma + 2 M r
  const R A = (r2 + a2) * (r2 + a2) - a2 * (r2 - M2 * r + a2) * s2;
  const R f = p.f;
  const R u = Sig * S2 * f;
  R iQ, igg;
  if (Q && g.qks) {
    const R g2 = p.gg * p.gg;
    const R iX = div_((R)1, u * s2 * g2);  // the one division
    iQ = iX * g2;
    igg = iX * u * s2;
  } else {
    iQ = div_((R)1, u * s2);               // the one division
    igg = p.igg;
  }
  const R iu = iQ * s2;                 // 1 / (Sigma S2 f)
  const R iSig = iu * S2 * f, iS2 = iu * Sig * f, fi = iu * Sig * S2;
  o.opz = S2 * iSig;
  o.H11 = A * iSig * iS2 * fi * fi;
  o.H13 = a * iSig * fi;
  o.H22 = iSig * igg;
  o.H33 = iQ * u * iSig;                // 1 / (Sigma s^2)
  o.beta1 = M2 * r * iS2 * fi;
}

// The metric at x^n with the derivatives the momentum push needs, and the tetrad
// coefficients; one division, four reciprocal square roots.
template <typename R>
struct Local {
  R alpha;
  Geo<R> G;
  R d1H11, d1H22, d1H33, d1H13, d1alpha, d1beta1;
  R d2H11, d2H22, d2H33, d2H13, d2alpha, d2beta1;
  R rH11, sH11, rh22, sh22, rh33, sh33, k13, m13;
};
template <bool Q = true, typename R>
__device__ __forceinline__ void local_full(const GridP &g, const Pt<R> &p, Local<R> &L) {
  const Cst<R> k = cst<R>(g);
  const R a = k.a, M = k.M, a2 = k.a2, M2 = k.M2, gg = p.gg, dxi = k.dxi;
  const R r = p.r, s = p.s, c = p.c, r2 = r * r, s2 = s * s;
  const R Sig = fma_(a2, c * c, r2);
  const R S2 = fma_(M2, r, Sig);
  const R Del = r2 - M2 * r + a2;
  const R A = (r2 + a2) * (r2 + a2) - a2 * Del * s2;
  const R f = p.f;
  const R u = Sig * S2 * f;
  R iQ, igg;
  if (Q && g.qks) {
    const R g2 = gg * gg;
    const R iX = div_((R)1, u * s2 * g2);
    iQ = iX * g2;
    igg = iX * u * s2;
  } else {
    iQ = div_((R)1, u * s2);
    igg = p.igg;
  }
  const R iu = iQ * s2;
  const R iSig = iu * S2 * f, iS2 = iu * Sig * f, fi = iu * Sig * S2;
  const R is2 = iQ * u;
  Geo<R> &o = L.G;
  o.opz = S2 * iSig;
  o.H11 = A * iSig * iS2 * fi * fi;
  o.H13 = a * iSig * fi;
  o.H22 = iSig * igg;
  o.H33 = iSig * is2;
  o.beta1 = M2 * r * iS2 * fi;
  const R al2 = Sig * iS2;
  L.alpha = rsqrt_(o.opz);
  const R dxS = (R)2 * r * f, deS = (R)-2 * a2 * s * c * gg;
  const R dxA = (R)4 * r * f * (r2 + a2) - a2 * s2 * (R)2 * (r - M) * f;
  const R deA = (R)-2 * a2 * s * c * Del * gg;
  const R P = Sig * S2;
  const R iP = iSig * iS2, iP2 = iP * iP, fi2 = fi * fi;
  const R iSg2 = iSig * iSig;
  const R al3 = L.alpha * al2;
  L.d1H11 = (P * dxA - (R)2 * A * (M * r * dxS + Sig * (dxS + M * f))) * iP2 * fi2 -
            (R)2 * dxi * o.H11;
  L.d2H11 = (P * deA - (R)2 * A * deS * (M * r + Sig)) * iP2 * fi2;
  L.d1H22 = -dxS * iSg2 * igg;
  L.d2H22 = -deS * iSg2 * igg;
  if (Q && g.qks) L.d2H22 = L.d2H22 - (R)2 * o.H22 * p.gp * gg * igg;  // h^22 = h^tt/gg^2
  L.d1H33 = -dxS * iSg2 * is2;
  L.d2H33 = -(deS + (R)2 * c * s * is2 * Sig * gg) * iSg2 * is2;
  L.d1H13 = -a * fi * iSig * (iSig * dxS + dxi);
  L.d2H13 = -a * iSg2 * deS * fi;
  const R fsr = f * Sig - r * dxS;
  L.d1alpha = -M * fsr * iSg2 * al3;
  L.d2alpha = M * r * deS * iSg2 * al3;
  L.d1beta1 = M2 * fi * fsr * iS2 * iS2 - dxi * o.beta1;
  L.d2beta1 = (R)-2 * M * fi * r * deS * iS2 * iS2;
  const R h22 = gg * gg * Sig, h33 = A * s2 * iSig, h13 = -f * a * o.opz * s2;
  L.rH11 = rsqrt_(o.H11);
  L.sH11 = o.H11 * L.rH11;
  L.rh22 = rsqrt_(h22);
  L.sh22 = h22 * L.rh22;
  L.rh33 = rsqrt_(h33);
  L.sh33 = h33 * L.rh33;
  L.k13 = h13 * L.rh33;    // h_13 / sqrt(h_33)
  L.m13 = L.k13 * L.rh33;  // h_13 / h_33
}

// App. A tetrad maps with the precomputed coefficients (M: type of the metric values, R: of
// the vectors; the same type everywhere except in the adjoint's momentum derivatives)
template <typename M, typename R>
__device__ __forceinline__ void vec_hat(const Local<M> &L, const R A[3], R o[3]) {
  o[0] = A[0] * L.rH11;
  o[1] = L.sh22 * A[1];
  o[2] = fma_(L.k13, A[0], L.sh33 * A[2]);
}
template <typename M, typename R>
__device__ __forceinline__ void cov_hat(const Local<M> &L, const R a[3], R o[3]) {
  o[0] = L.sH11 * fma_(-L.m13, a[2], a[0]);
  o[1] = a[1] * L.rh22;
  o[2] = a[2] * L.rh33;
}
template <typename M, typename R>
__device__ __forceinline__ void hat_cov(const Local<M> &L, const R h[3], R o[3]) {
  o[0] = fma_(h[0], L.rH11, L.k13 * h[2]);
  o[1] = L.sh22 * h[1];
  o[2] = L.sh33 * h[2];
}

// Boris step over coordinate time dt/2 in the tetrad frame (Sec. 3.1), hq = qm alpha dt/2.
template <typename R>
__device__ __forceinline__ void boris(R u[3], const R D[3], const R B[3], R hq) {
  const R e = (R)0.5 * hq;
  const R m0 = fma_(e, D[0], u[0]), m1 = fma_(e, D[1], u[1]), m2 = fma_(e, D[2], u[2]);
  const R ig = rsqrt_(fma_(m0, m0, fma_(m1, m1, fma_(m2, m2, (R)1))));
  const R t0 = e * B[0] * ig, t1 = e * B[1] * ig, t2 = e * B[2] * ig;
  const R sf = div_((R)2, fma_(t0, t0, fma_(t1, t1, fma_(t2, t2, (R)1))));
  const R p0 = m0 + (m1 * t2 - m2 * t1);
  const R p1 = m1 + (m2 * t0 - m0 * t2);
  const R p2 = m2 + (m0 * t1 - m1 * t0);
  u[0] = m0 + sf * (p1 * t2 - p2 * t1) + e * D[0];
  u[1] = m1 + sf * (p2 * t0 - p0 * t2) + e * D[1];
  u[2] = m2 + sf * (p0 * t1 - p1 * t0) + e * D[2];
}

// Eq. (discretized-geodesic-u): the map t -> G(t) whose fixed point is the new covariant
// (u_1, u_2): implicit midpoint with the metric and its derivatives at x^n, u_3 unchanged
// (the substep conserves it). m2: the mass term of gamma (1 massive, 0 massless). Everything that does not depend on the iterate t is
// precomputed; apply() evaluates G once.
template <typename R>
struct GeoMap {
  R u0, u1, hu0, hu1, c0, c1, e1, e2, f1, f2, D1a, D1b, D2a, D2b, hdt;
  R H11, H22, d1H11, d1H22, d2H11, d2H22;
  GeoMap() = default;
  template <typename M>
  __device__ __forceinline__ GeoMap(const GridP &g, const Local<M> &L, const R u[3], R m2) {
    const R u3 = u[2];
    const Geo<M> &o = L.G;
    const R dt = cst<R>(g).dt;
    u0 = u[0];
    u1 = u[1];
    c0 = fma_(o.H33 * u3, u3, m2);
    c1 = (R)2 * o.H13 * u3;
    e1 = L.d1H33 * u3 * u3;
    e2 = (R)2 * L.d1H13 * u3;
    f1 = L.d2H33 * u3 * u3;
    f2 = (R)2 * L.d2H13 * u3;
    D1a = dt * L.d1alpha;
    D1b = dt * L.d1beta1;
    D2a = dt * L.d2alpha;
    D2b = dt * L.d2beta1;
    hdt = (R)0.5 * dt * L.alpha;
    hu0 = (R)0.5 * u0;
    hu1 = (R)0.5 * u1;
    H11 = o.H11;
    H22 = o.H22;
    d1H11 = L.d1H11;
    d1H22 = L.d1H22;
    d2H11 = L.d2H11;
    d2H22 = L.d2H22;
  }
  __device__ __forceinline__ void apply(R t0, R t1, R &n0, R &n1) const {
    const R b0 = fma_((R)0.5, t0, hu0), b1 = fma_((R)0.5, t1, hu1);
    const R b1s = b1 * b1;
    const R q = fma_(b0, fma_(H11, b0, c1), fma_(H22, b1s, c0));  // gamma_bar^2
    const R ig = rsqrt_(q);
    const R gb = q * ig;                                          // gamma_bar
    const R ha = hdt * ig;                                        // dt / (2 u^0)
    const R k1 = fma_(b0, fma_(d1H11, b0, e2), fma_(d1H22, b1s, e1));
    const R k2 = fma_(b0, fma_(d2H11, b0, f2), fma_(d2H22, b1s, f1));
    n0 = fma_(b0, D1b, fma_(-gb, D1a, fma_(-ha, k1, u0)));
    n1 = fma_(b0, D2b, fma_(-gb, D2a, fma_(-ha, k2, u1)));
  }
  // J[i][j] = d n_i / d t_j of apply at t (the map depends on t through b = (t + u)/2)
  __device__ __forceinline__ void jacobian(R t0, R t1, R J[2][2]) const {
    const R b0 = fma_((R)0.5, t0, hu0), b1 = fma_((R)0.5, t1, hu1);
    const R b1s = b1 * b1;
    const R q = fma_(b0, fma_(H11, b0, c1), fma_(H22, b1s, c0));
    const R ig = rsqrt_(q);
    const R ha = hdt * ig;
    const R k1 = fma_(b0, fma_(d1H11, b0, e2), fma_(d1H22, b1s, e1));
    const R k2 = fma_(b0, fma_(d2H11, b0, f2), fma_(d2H22, b1s, f1));
    const R q0 = fma_((R)2 * H11, b0, c1), q1 = (R)2 * H22 * b1;  // dq/db
    const R hg = (R)0.5 * ig, hh = (R)-0.5 * ha * ig * ig;       // d gamma/dq, d ha/dq
    const R g0 = hg * q0, g1 = hg * q1, a0 = hh * q0, a1 = hh * q1;
    const R k10 = fma_((R)2 * d1H11, b0, e2), k11 = (R)2 * d1H22 * b1;
    const R k20 = fma_((R)2 * d2H11, b0, f2), k21 = (R)2 * d2H22 * b1;
    J[0][0] = (R)0.5 * (D1b - g0 * D1a - a0 * k1 - ha * k10);
    J[0][1] = (R)0.5 * (-g1 * D1a - a1 * k1 - ha * k11);
    J[1][0] = (R)0.5 * (D2b - g0 * D2a - a0 * k2 - ha * k20);
    J[1][1] = (R)0.5 * (-g1 * D2a - a1 * k2 - ha * k21);
  }
};

// The geodesic substep: n_iter applications of G from t = u.
template <typename R>
__device__ __forceinline__ void geodesic_momentum(const GridP &g, const Local<R> &L, R u[3],
                                                  R m2) {
  const GeoMap<R> m(g, L, u, m2);
  R t0 = u[0], t1 = u[1];
  for (int it = 0; it < g.n_iter; ++it) {
    R n0, n1;
    m.apply(t0, t1, n0, n1);
    // once the iterate repeats exactly, every later iteration repeats it too (same inputs,
    // deterministic arithmetic): stopping here returns bit for bit the n_iter result
    const bool fixed = (n0 == t0) && (n1 == t1);
    t0 = n0;
    t1 = n1;
    if (fixed && g.stop_on_repeat) break;
  }
  u[0] = t0;
  u[1] = t1;
}

// FP32 r, sin(theta), cos(theta) and the map's factors from FP64-computed per-cell tables and
// short Taylor series of the offset from the cell corner (mixed path; and the FP32 predictor
// of the FP64 path's refined implicit iterations), at x1 = i + o1, x2 = j + o2.
template <bool Q = true>
__device__ __forceinline__ void rsc32(const GridP &g, const PushTables &tb, int i, int j,
                                      float o1, float o2, Pt<float> &pt) {
  const float e = o1 * g.f_dxi;  // |e| <= 2 dxi
  float p = 1.0f / 720.0f;
  p = fmaf(p, e, 1.0f / 120.0f);
  p = fmaf(p, e, 1.0f / 24.0f);
  p = fmaf(p, e, 1.0f / 6.0f);
  p = fmaf(p, e, 0.5f);
  p = fmaf(p, e, 1.0f);
  const float ex = __ldg(tb.r + i + G_) * fmaf(p, e, 1.0f);  // r - r0
  pt.r = Q ? g.f_r0 + ex : ex;
  pt.f = g.f_dxi * ex;
  float d = o2 * g.f_dth;  // |d| <= 2 dtheta: the offset in eta, then in theta
  if (Q && g.qks) {
    const float t1 = __ldg(tb.t1 + j + G_), t2 = __ldg(tb.t2 + j + G_), c3 = g.f_c3;
    pt.gg = g.f_dth * fmaf(d, fmaf(3.0f * c3, d, 2.0f * t2), t1);
    pt.gp = g.f_dth * g.f_dth * fmaf(6.0f * c3, d, 2.0f * t2);
    d = d * fmaf(d, fmaf(c3, d, t2), t1);
  } else {
    pt.gg = g.f_dth;
    pt.igg = g.f_ig2;
    pt.gp = 0.0f;
  }
  const float q = d * d;
  const float se = fmaf(fmaf(fmaf(-1.0f / 5040.0f, q, 1.0f / 120.0f), q, -1.0f / 6.0f) * q, d, d);
  const float ce = fmaf(fmaf(fmaf(fmaf(1.0f / 40320.0f, q, -1.0f / 720.0f), q, 1.0f / 24.0f), q,
                             -0.5f), q, 1.0f);
  const float s0 = __ldg(tb.s + j + G_), c0 = __ldg(tb.c + j + G_);
  pt.s = fmaf(s0, ce, c0 * se);
  pt.c = fmaf(c0, ce, -s0 * se);
}

}  // namespace
