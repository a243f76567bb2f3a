// particles.cu -- the GR particle pusher (Sec. 3.1 of arXiv:2511.17701) and the
// charge-conserving conformal current deposit (Sec. 3.2), one thread per particle.
//
// FP64 throughout. On GB300 the double-precision pipe, not HBM, bounds this kernel:
// every particle-step evaluates the metric 2 n_iter + 2 times. Particle state is SoA;
// consecutive threads read consecutive elements (coalesced), and field gathers hit L1/L2
// because the particles are kept sorted by cell.
#include "grpic_internal.cuh"

namespace {

constexpr int TPB = 128;

// Yee offsets (Fig. 1): B^1 (0, 1/2), B^2 (1/2, 0), B^3 (1/2, 1/2); D^1 (1/2, 0),
// D^2 (0, 1/2), D^3 (0, 0).
__device__ __forceinline__ void gather_fields(const GridP &g, const FieldPtrs &F, double x1,
                                              double x2, double B[3], double D[3]) {
  B[0] = interp_plane(F.Bn[0], g.NX, x1, x2, 0.0, 0.5);
  B[1] = interp_plane(F.Bn[1], g.NX, x1, x2, 0.5, 0.0);
  B[2] = interp_plane(F.Bn[2], g.NX, x1, x2, 0.5, 0.5);
  D[0] = interp_plane(F.D[0], g.NX, x1, x2, 0.5, 0.0);
  D[1] = interp_plane(F.D[1], g.NX, x1, x2, 0.0, 0.5);
  D[2] = interp_plane(F.D[2], g.NX, x1, x2, 0.0, 0.0);
}

// ---------------------------------------------------------------------------------
// Metric at the iterates. The implicit pushes evaluate the metric at points within a
// fraction of a cell of x^n. r, sin(theta), cos(theta) there follow from their values at
// x^n by the exponential and the angle-addition formulas with short Taylor series of the
// small offsets (|eps| <= 0.02: truncation below 1e-18 relative); larger offsets and the
// SMALL_ANGLE_GR clamp fall back to CUDA's exp and sincos. All reciprocals of one
// evaluation come from a single division.
// ---------------------------------------------------------------------------------
struct Base {
  double x1, th0;     // x^n and theta(x^n) = x2 dtheta (not clamped)
  double r0, s0, c0;  // r, sin(theta), cos(theta) at x^n
};

// exp(e) for |e| <= 0.02 (Taylor to e^7)
__device__ __forceinline__ double exp_small(double e) {
  double p = 1.0 / 5040.0;
  p = fma(p, e, 1.0 / 720.0);
  p = fma(p, e, 1.0 / 120.0);
  p = fma(p, e, 1.0 / 24.0);
  p = fma(p, e, 1.0 / 6.0);
  p = fma(p, e, 0.5);
  p = fma(p, e, 1.0);
  return fma(p, e, 1.0);
}

// r, sin(theta), cos(theta) at the code position (x1t, x2t), theta clamped to
// [small_angle, pi - small_angle]. theta = x2t dtheta is formed with one rounded product,
// and its offset from theta(x^n) is exact (Sterbenz), so the result is sin and cos of
// exactly that double: near theta = pi, where sin(theta) is ill-conditioned in theta, any
// other way of forming theta would move the result by ~1e-12 relative.
__device__ __forceinline__ void local_rsc(const GridP &g, const Base &b, double x1t, double x2t,
                                          double &r, double &s, double &c) {
  const double e1 = (x1t - b.x1) * g.dxi;
  r = fabs(e1) <= 0.02 ? b.r0 * exp_small(e1) : g.r_min * exp(x1t * g.dxi);
  const double th = __dmul_rn(x2t, g.dth);
  const double e2 = th - b.th0;
  if (th < g.small_angle || th > GRPIC_PI - g.small_angle) {
    sincos(fmin(fmax(th, g.small_angle), GRPIC_PI - g.small_angle), &s, &c);
  } else if (fabs(e2) <= 0.02) {
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
    s = fma(b.s0, ce, b.c0 * se);
    c = fma(b.c0, ce, -b.s0 * se);
  } else {
    sincos(th, &s, &c);
  }
}

// The contravariant metric, shift and 1 + z = 1/alpha^2 from r, sin, cos (App. A, code units).
struct Geo {
  double H11, H13, H22, H33, beta1, opz;
};
__device__ __forceinline__ void geo_from_rsc(const GridP &g, double r, double s, double c,
                                             Geo &o) {
  const double a = g.a, M = g.M, a2 = a * a;
  const double r2 = r * r, s2 = s * s;
  const double Sig = fma(a2, c * c, r2);
  const double S2 = fma(2.0 * M, r, Sig);                       // Sigma + 2 M r
  const double A = (r2 + a2) * (r2 + a2) - a2 * (r2 - 2.0 * M * r + a2) * s2;
  const double f = g.dxi * r;
  const double u = Sig * S2 * f;
  const double iQ = 1.0 / (u * s2);                            // the one division
  const double iu = iQ * s2;                                   // 1 / (Sigma S2 f)
  const double iSig = iu * S2 * f, iS2 = iu * Sig * f, fi = iu * Sig * S2;
  o.opz = S2 * iSig;
  o.H11 = A * iSig * iS2 * fi * fi;
  o.H13 = a * iSig * fi;
  o.H22 = iSig * g.ig2;
  o.H33 = iQ * u * iSig;                                       // 1 / (Sigma s^2)
  o.beta1 = 2.0 * M * r * iS2 * fi;
}

// The full metric at x^n with the derivatives the momentum push needs, and the tetrad
// coefficients (App. A); one division, four reciprocal square roots.
struct Local {
  double alpha, ialpha;
  Geo G;
  double d1H11, d1H22, d1H33, d1H13, d1alpha, d1beta1;
  double d2H11, d2H22, d2H33, d2H13, d2alpha, d2beta1;
  double rH11, sH11, rh22, sh22, rh33, sh33, k13, m13;  // tetrad coefficients
};
__device__ __forceinline__ void local_full(const GridP &g, double r, double s, double c,
                                           Local &L) {
  const double a = g.a, M = g.M, a2 = a * a, gg = g.dth;
  const double r2 = r * r, s2 = s * s;
  const double Sig = fma(a2, c * c, r2);
  const double S2 = fma(2.0 * M, r, Sig);
  const double Del = r2 - 2.0 * M * r + a2;
  const double A = (r2 + a2) * (r2 + a2) - a2 * Del * s2;
  const double f = g.dxi * r;
  const double u = Sig * S2 * f;
  const double iQ = 1.0 / (u * s2);
  const double iu = iQ * s2;
  const double iSig = iu * S2 * f, iS2 = iu * Sig * f, fi = iu * Sig * S2;
  const double is2 = iQ * u;
  Geo &o = L.G;
  o.opz = S2 * iSig;
  o.H11 = A * iSig * iS2 * fi * fi;
  o.H13 = a * iSig * fi;
  o.H22 = iSig * g.ig2;
  o.H33 = iSig * is2;
  o.beta1 = 2.0 * M * r * iS2 * fi;
  const double al2 = Sig * iS2;
  L.alpha = rsqrt(o.opz);
  L.ialpha = o.opz * L.alpha;
  // derivatives (App. A, quasi-spherical Kerr-Schild, mass M explicit)
  const double dxS = 2.0 * r * f, deS = -2.0 * a2 * s * c * gg;
  const double dxA = 4.0 * r * f * (r2 + a2) - a2 * s2 * 2.0 * (r - M) * f;
  const double deA = -2.0 * a2 * s * c * Del * gg;
  const double P = Sig * S2;
  const double iP = iSig * iS2, iP2 = iP * iP, fi2 = fi * fi;
  const double iSg2 = iSig * iSig;
  const double al3 = L.alpha * al2;
  L.d1H11 = (P * dxA - 2.0 * A * (M * r * dxS + Sig * (dxS + M * f))) * iP2 * fi2 -
            2.0 * g.dxi * o.H11;
  L.d2H11 = (P * deA - 2.0 * A * deS * (M * r + Sig)) * iP2 * fi2;
  L.d1H22 = -dxS * iSg2 * g.ig2;
  L.d2H22 = -deS * iSg2 * g.ig2;
  L.d1H33 = -dxS * iSg2 * is2;
  L.d2H33 = -(deS + 2.0 * c * s * is2 * Sig * gg) * iSg2 * is2;
  L.d1H13 = -a * fi * iSig * (iSig * dxS + g.dxi);
  L.d2H13 = -a * iSg2 * deS * fi;
  const double fsr = f * Sig - r * dxS;
  L.d1alpha = -M * fsr * iSg2 * al3;
  L.d2alpha = M * r * deS * iSg2 * al3;
  L.d1beta1 = 2.0 * M * fi * fsr * iS2 * iS2 - g.dxi * o.beta1;
  L.d2beta1 = -2.0 * M * fi * r * deS * iS2 * iS2;
  // tetrad coefficients
  const double h22 = gg * gg * Sig, h33 = A * s2 * iSig, h13 = -f * a * o.opz * s2;
  L.rH11 = rsqrt(o.H11);
  L.sH11 = o.H11 * L.rH11;
  L.rh22 = rsqrt(h22);
  L.sh22 = h22 * L.rh22;
  L.rh33 = rsqrt(h33);
  L.sh33 = h33 * L.rh33;
  L.k13 = h13 * L.rh33;          // h_13 / sqrt(h_33)
  L.m13 = L.k13 * L.rh33;        // h_13 / h_33
}

// App. A tetrad maps with precomputed coefficients
__device__ __forceinline__ void vec_hat(const Local &L, const double A[3], double o[3]) {
  o[0] = A[0] * L.rH11;
  o[1] = L.sh22 * A[1];
  o[2] = fma(L.k13, A[0], L.sh33 * A[2]);
}
__device__ __forceinline__ void cov_hat(const Local &L, const double a[3], double o[3]) {
  o[0] = L.sH11 * fma(-L.m13, a[2], a[0]);
  o[1] = a[1] * L.rh22;
  o[2] = a[2] * L.rh33;
}
__device__ __forceinline__ void hat_cov(const Local &L, const double h[3], double o[3]) {
  o[0] = fma(h[0], L.rH11, L.k13 * h[2]);
  o[1] = L.sh22 * h[1];
  o[2] = L.sh33 * h[2];
}

// Eq. (discretized-geodesic-u): implicit midpoint with fixed n_iter, metric at x^n.
__device__ __forceinline__ void geodesic_momentum(const GridP &g, const Local &L, double u[3]) {
  const double u0 = u[0], u1 = u[1], u3 = u[2];  // u_3 is not changed by this substep
  const Geo &o = L.G;
  const double c0 = fma(o.H33 * u3, u3, 1.0), c1 = 2.0 * o.H13 * u3;
  const double e1 = L.d1H33 * u3 * u3, e2 = 2.0 * L.d1H13 * u3;
  const double f1 = L.d2H33 * u3 * u3, f2 = 2.0 * L.d2H13 * u3;
  const double D1a = g.dt * L.d1alpha, D1b = g.dt * L.d1beta1;
  const double D2a = g.dt * L.d2alpha, D2b = g.dt * L.d2beta1;
  const double hdt = 0.5 * g.dt * L.alpha;
  const double hu0 = 0.5 * u0, hu1 = 0.5 * u1;
  double t0 = u0, t1 = u1;
  for (int it = 0; it < g.n_iter; ++it) {
    const double b0 = fma(0.5, t0, hu0), b1 = fma(0.5, t1, hu1);
    const double b1s = b1 * b1;
    const double q = fma(b0, fma(o.H11, b0, c1), fma(o.H22, b1s, c0));  // gamma_bar^2
    const double ig = rsqrt(q);
    const double gb = q * ig;                                          // gamma_bar
    const double ha = hdt * ig;                                        // dt / (2 u^0)
    const double k1 = fma(b0, fma(L.d1H11, b0, e2), fma(L.d1H22, b1s, e1));
    const double k2 = fma(b0, fma(L.d2H11, b0, f2), fma(L.d2H22, b1s, f1));
    const double n0 = fma(b0, D1b, fma(-gb, D1a, fma(-ha, k1, u0)));
    const double n1 = fma(b0, D2b, fma(-gb, D2a, fma(-ha, k2, u1)));
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

// Charge-conserving deposit of one move (Sec. 3.2, Eq. charge-conservation-disc): the
// zigzag split of Umeda et al. (2003) with area weighting, plus J^3 = q alpha u^3 / gamma
// at the midpoint with the same theta regularisation as the push.
__device__ __forceinline__ void deposit_move(const GridP &g, const FieldPtrs &F, double q,
                                             int ia, int ja, double xa1, double xa2, int ib,
                                             int jb, double xb1, double xb2, double v3) {
  const double idt = 1.0 / g.dt;
  const double xr1 = fmin(fmin((double)ia, (double)ib) + 1.0,
                          fmax(fmax((double)ia, (double)ib), 0.5 * (xa1 + xb1)));
  const double xr2 = fmin(fmin((double)ja, (double)jb) + 1.0,
                          fmax(fmax((double)ja, (double)jb), 0.5 * (xa2 + xb2)));
  double *J1 = F.J[0], *J2 = F.J[1], *J3 = F.J[2];
  const int NX = g.NX;
  {
    const double F1 = q * (xr1 - xa1) * idt, F2 = q * (xr2 - xa2) * idt;
    const double W1 = 0.5 * (xa1 + xr1) - ia, W2 = 0.5 * (xa2 + xr2) - ja;
    const int64_t k = sidx(g, ia, ja);
    atomicAdd(J1 + k, F1 * (1.0 - W2));
    atomicAdd(J1 + k + NX, F1 * W2);
    atomicAdd(J2 + k, F2 * (1.0 - W1));
    atomicAdd(J2 + k + 1, F2 * W1);
  }
  {
    const double F1 = q * (xb1 - xr1) * idt, F2 = q * (xb2 - xr2) * idt;
    const double W1 = 0.5 * (xr1 + xb1) - ib, W2 = 0.5 * (xr2 + xb2) - jb;
    const int64_t k = sidx(g, ib, jb);
    atomicAdd(J1 + k, F1 * (1.0 - W2));
    atomicAdd(J1 + k + NX, F1 * W2);
    atomicAdd(J2 + k, F2 * (1.0 - W1));
    atomicAdd(J2 + k + 1, F2 * W1);
  }
  const double xm1 = 0.5 * (xa1 + xb1), xm2 = 0.5 * (xa2 + xb2);
  const double f1 = floor(xm1), f2 = floor(xm2);
  const int i0 = (int)f1, j0 = (int)f2;
  const double w1 = xm1 - f1, w2 = xm2 - f2, qv = q * v3;
  const int64_t k = sidx(g, i0, j0);
  atomicAdd(J3 + k, qv * (1.0 - w1) * (1.0 - w2));
  atomicAdd(J3 + k + 1, qv * w1 * (1.0 - w2));
  atomicAdd(J3 + k + NX, qv * (1.0 - w1) * w2);
  atomicAdd(J3 + k + NX + 1, qv * w1 * w2);
}

// dphi/dt = alpha/gamma h^{3j} u_j at (x1t, x2t) (Eq. discretized-geodesic-x-phi; q times
// it is J^3 / sqrt(h) w, Sec. 3.2); alpha/gamma = 1/sqrt((1+z) gamma^2).
__device__ __forceinline__ double phi_rate(const GridP &g, const Base &b, double x1t, double x2t,
                                           const double u[3]) {
  double r, sn, cs;
  local_rsc(g, b, x1t, x2t, r, sn, cs);
  Geo o;
  geo_from_rsc(g, r, sn, cs, o);
  const double q = fma(o.H11 * u[0], u[0], fma(o.H22 * u[1], u[1], fma(o.H33 * u[2], u[2],
                   fma(2.0 * o.H13 * u[0], u[2], 1.0))));
  return rsqrt(o.opz * q) * fma(o.H13, u[0], o.H33 * u[2]);
}

__device__ __forceinline__ Base make_base(const GridP &g, double x1, double x2) {
  Base b;
  b.x1 = x1;
  b.th0 = __dmul_rn(x2, g.dth);
  b.r0 = g.r_min * exp(x1 * g.dxi);
  sincos(b.th0, &b.s0, &b.c0);
  return b;
}

__device__ __forceinline__ void count(unsigned long long *diag, int which) {
  atomicAdd(diag + which, 1ull);
}

// One particle: steps 1-11 of Sec. 3.1, the boundaries of Sec. 3.3.3, and (DEPOSIT) the
// deposit of its move.
template <bool DEPOSIT>
__global__ void __launch_bounds__(TPB) k_push(GridP g, FieldPtrs F, SpeciesDev s,
                                              unsigned long long *diag) {
  const int64_t n = *s.n;
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n;
       k += (int64_t)gridDim.x * blockDim.x) {
    const int i1 = s.i1[k], i2 = s.i2[k];
    const double dx1 = s.dx1[k], dx2 = s.dx2[k];
    // step 1: save the previous location
    s.i1p[k] = i1; s.i2p[k] = i2; s.dx1p[k] = dx1; s.dx2p[k] = dx2;
    const uint8_t tag = s.tag[k];
    if (tag != 1) {
      if (tag != 0) s.tag[k] = 0;
      continue;
    }
    const double x1 = i1 + dx1, x2 = i2 + dx2;
    // step 2: fields at x^n
    double Bv[3], Dv[3];
    gather_fields(g, F, x1, x2, Bv, Dv);
    const Base b = make_base(g, x1, x2);
    double sn, cs;
    {
      double r0;
      local_rsc(g, b, x1, x2, r0, sn, cs);  // clamps theta near the axes
    }
    Local L;
    local_full(g, b.r0, sn, cs, L);
    // step 3: to the tetrad basis
    double Bh[3], Dh[3], uh[3], u[3] = {s.u1[k], s.u2[k], s.u3[k]};
    vec_hat(L, Bv, Bh);
    vec_hat(L, Dv, Dh);
    cov_hat(L, u, uh);
    const double hq = s.qm * L.alpha * 0.5 * g.dt;
    boris_step(uh, Dh, Bh, hq);  // step 4
    hat_cov(L, uh, u);           // step 5
    geodesic_momentum(g, L, u);  // step 6
    cov_hat(L, u, uh);           // step 7
    boris_step(uh, Dh, Bh, hq);  // step 8
    hat_cov(L, uh, u);           // step 9
    // step 10: implicit coordinate push, Eq. (discretized-geodesic-x), metric at
    // x_bar = (x^n + x~)/2; the first iterate is x^n itself
    const double uu0 = 2.0 * u[0] * u[2];
    double t1 = dx1, t2 = dx2;
    for (int it = 0; it < g.n_iter; ++it) {
      Geo o;
      if (it == 0) {
        o = L.G;
      } else {
        double r, s_, c_;
        // x_bar = i + (dx + x~)/2, rounded in that order
        local_rsc(g, b, __dadd_rn((double)i1, 0.5 * __dadd_rn(dx1, t1)),
                  __dadd_rn((double)i2, 0.5 * __dadd_rn(dx2, t2)), r, s_, c_);
        geo_from_rsc(g, r, s_, c_, o);
      }
      const double q = fma(o.H11 * u[0], u[0], fma(o.H22 * u[1], u[1],
                       fma(o.H33 * u[2], u[2], fma(o.H13, uu0, 1.0))));
      const double ag = rsqrt(o.opz * q);  // alpha / gamma
      const double n1 = fma(g.dt, fma(ag, fma(o.H11, u[0], o.H13 * u[2]), -o.beta1), dx1);
      const double n2 = fma(g.dt, ag * o.H22 * u[1], dx2);
      const bool fixed = (n1 == t1) && (n2 == t2);  // exact repeat: later iterations are no-ops
      t1 = n1;
      t2 = n2;
      if (fixed && g.stop_on_repeat) break;
    }
    if (!(isfinite(u[0]) && isfinite(u[1]) && isfinite(u[2]) && isfinite(t1) &&
          isfinite(t2) && fabs(t1) < 1e6 && fabs(t2) < 1e6)) {
      s.tag[k] = 0;
      count(diag, DG_NONFINITE);
      continue;
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
      continue;
    }
    s.i1[k] = j1; s.i2[k] = j2; s.dx1[k] = e1; s.dx2[k] = e2;
    s.u1[k] = u[0]; s.u2[k] = u[1]; s.u3[k] = u[2];
    if (j1 < 0) { s.tag[k] = 2; count(diag, DG_LEFT_INNER); }
    else if (j1 >= g.n_r) { s.tag[k] = 2; count(diag, DG_LEFT_OUTER); }
    // step 11: phi at x^{n+1/2}, the midpoint of the stored x^n and the final x^{n+1}
    const double xb1 = j1 + e1, xb2 = j2 + e2;
    const double v3 = phi_rate(g, b, 0.5 * __dadd_rn(x1, xb1), 0.5 * __dadd_rn(x2, xb2), u);
    s.phi[k] += g.dt * v3;
    if (DEPOSIT) deposit_move(g, F, s.qc * s.w[k], i1, i2, x1, x2, j1, j2, xb1, xb2, v3);
  }
}

// Deposit from stored previous and new positions (grpic_deposit).
__global__ void __launch_bounds__(TPB) k_deposit(GridP g, FieldPtrs F, SpeciesDev s) {
  const int64_t n = *s.n;
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n;
       k += (int64_t)gridDim.x * blockDim.x) {
    if (s.tag[k] == 0) continue;
    const int ia = s.i1p[k], ja = s.i2p[k], ib = s.i1[k], jb = s.i2[k];
    const double xa1 = ia + s.dx1p[k], xa2 = ja + s.dx2p[k];
    const double xb1 = ib + s.dx1[k], xb2 = jb + s.dx2[k];
    const double u[3] = {s.u1[k], s.u2[k], s.u3[k]};
    const Base b = make_base(g, xa1, xa2);
    const double v3 = phi_rate(g, b, 0.5 * __dadd_rn(xa1, xb1), 0.5 * __dadd_rn(xa2, xb2), u);
    deposit_move(g, F, s.qc * s.w[k], ia, ja, xa1, xa2, ib, jb, xb1, xb2, v3);
  }
}

// Loading: u_i = e_i^j u_j^ at the particle (App. A), w = w0 r^{-k} sqrt(h)(x_p).
__global__ void k_load(GridP g, SpeciesDev s, int64_t n, const double *uh1, const double *uh2,
                       const double *uh3, const double *w0, double dpow) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n;
       k += (int64_t)gridDim.x * blockDim.x) {
    const double x1 = s.i1[k] + s.dx1[k], x2 = s.i2[k] + s.dx2[k];
    MetricV m;
    metric_eval<false>(g, x1, x2, true, m, nullptr);
    const double uh[3] = {uh1[k], uh2[k], uh3[k]};
    double u[3];
    t_hat_to_cov(m, uh, u);
    s.u1[k] = u[0]; s.u2[k] = u[1]; s.u3[k] = u[2];
    MetricV m0;
    metric_eval<false>(g, x1, x2, false, m0, nullptr);
    const double r = g.r_min * exp(x1 * g.dxi);
    s.w[k] = w0[k] * pow(r, -dpow) * m0.sqrt_h;
    s.phi[k] = 0.0;
    s.tag[k] = 1;
    s.i1p[k] = s.i1[k]; s.i2p[k] = s.i2[k]; s.dx1p[k] = s.dx1[k]; s.dx2p[k] = s.dx2[k];
  }
}

int blocks_for(int64_t n) {
  int64_t b = (n + TPB - 1) / TPB;
  const int64_t cap = 152 * 64;
  if (b > cap) b = cap;
  return (int)(b < 1 ? 1 : b);
}

}  // namespace

cudaError_t launch_load(const GridP &g, SpeciesDev s, int64_t n, const grpic_particle_init &in,
                        double dpow, cudaStream_t st) {
  if (n <= 0) return cudaGetLastError();
  k_load<<<blocks_for(n), TPB, 0, st>>>(g, s, n, in.uh1, in.uh2, in.uh3, in.w0, dpow);
  COUNT_LAUNCH(1);
  return cudaGetLastError();
}

cudaError_t launch_push(const GridP &g, const FieldPtrs &F, SpeciesDev s, int64_t n_bound,
                        bool deposit, unsigned long long *diag, cudaStream_t st) {
  if (n_bound <= 0) return cudaGetLastError();
  if (deposit)
    k_push<true><<<blocks_for(n_bound), TPB, 0, st>>>(g, F, s, diag);
  else
    k_push<false><<<blocks_for(n_bound), TPB, 0, st>>>(g, F, s, diag);
  COUNT_LAUNCH(1);
  return cudaGetLastError();
}

cudaError_t launch_deposit(const GridP &g, const FieldPtrs &F, SpeciesDev s, int64_t n_bound,
                           cudaStream_t st) {
  if (n_bound <= 0) return cudaGetLastError();
  k_deposit<<<blocks_for(n_bound), TPB, 0, st>>>(g, F, s);
  COUNT_LAUNCH(1);
  return cudaGetLastError();
}
