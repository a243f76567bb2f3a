// adjoint.cu -- adjoint of the GR pusher over frozen fields (Sec. 3.1 of arXiv:2511.17701):
// gradients of the final test-particle state (x1, x2, phi, u_1, u_2, u_3) with respect to the
// initial state and the field amplitude (the Wald field is linear in B0), for massive charged
// test particles.
//
// Forward: every particle is pushed n_steps steps in the em-plane fields times
// scale = B0 / (the amplitude the planes hold), both implicit substeps iterated to an exact
// repeat (at most n_iter times), with the state stored every `every` steps (checkpoints).
// Backward (reverse sweep, one thread per particle): for each checkpoint segment, last to
// first, the segment's states are recomputed into scratch memory, then the steps are
// traversed backwards with lambda <- J^T lambda, where J is the 6 x 7 Jacobian of one step
// (inputs: the state and the scale). J comes from forward-mode dual numbers through the same
// templates the pusher uses (pusher.cuh): one pass seeding x1, x2 (the metric differentiated
// too) and one seeding u_1, u_2, u_3 and the scale (metric values only; it depends on x
// alone). At the two implicit substeps the implicit-function theorem replaces
// differentiation through the iterations: at the fixed point t* = G(t*, p),
// dt* = (I - dG/dt)^{-1} (dG/dp) dp. The Jacobians of a segment are formed while its states
// are recomputed and kept in scratch memory for the reverse sweep.
#include "dual.cuh"
#include "grpic_internal.cuh"
#include "pusher.cuh"

namespace {

constexpr int TPB_ADJ = 64;
using D2 = Dual<2>;
using D4 = Dual<4>;

// the point at absolute code coordinates on the plain log-r grid (the adjoint's entry points
// reject quasi-spherical grids): r, sin(theta), cos(theta) with theta clamped to
// [small_angle, pi - small_angle] for the metric (Sec. 3.3.2), with zero derivative there,
// and the map's factors f = dxi r, gg = dtheta
template <typename R>
__device__ __forceinline__ void rsc_abs(const GridP &g, const R &x1, const R &x2, Pt<R> &p) {
  const R e = g.r_min * exp_(x1 * g.dxi);
  p.r = e;
  p.f = g.dxi * e;
  p.gg = R(g.dth);
  p.igg = R(g.ig2);
  p.gp = R(0.0);
  R &s = p.s, &c = p.c;
  const R th = x2 * g.dth;
  const double tv = val(th);
  if (tv < g.small_angle || tv > GRPIC_PI - g.small_angle) {
    double sv, cv;
    sincos(tv < g.small_angle ? g.small_angle : GRPIC_PI - g.small_angle, &sv, &cv);
    s = R(sv);
    c = R(cv);
  } else {
    sincos_(th, s, c);
  }
}

// bilinear interpolation at absolute code coordinates for a Yee offset (s1, s2)
template <typename R>
__device__ __forceinline__ R interp_abs(const double *__restrict__ pl, int NX, const R &x1,
                                        const R &x2, double s1, double s2) {
  const R y1 = x1 - s1, y2 = x2 - s2;
  const double f1 = floor(val(y1)), f2 = floor(val(y2));
  const int i0 = (int)f1, j0 = (int)f2;
  const R w1 = y1 - f1, w2 = y2 - f2;
  const double *p = pl + (int64_t)(j0 + G_) * NX + (i0 + G_);
  const double p00 = __ldg(p), p10 = __ldg(p + 1), p01 = __ldg(p + NX), p11 = __ldg(p + NX + 1);
  return (1.0 - w1) * (1.0 - w2) * p00 + w1 * (1.0 - w2) * p10 + (1.0 - w1) * w2 * p01 +
         w1 * w2 * p11;
}

// metric with derivatives, tetrad-frame fields (at unit amplitude and at `scale`) and the
// Boris coefficient at x^n
template <typename R>
struct Frame {
  Local<R> L;
  R Bh1[3], Dh1[3];  // unit amplitude
  R Bh[3], Dh[3], hq;
};
template <typename R>
__device__ __forceinline__ void frame_at(const GridP &g, const FieldPtrsT<double> &F,
                                         const R x[2], const R &scale, double qm, Frame<R> &fr) {
  R Bv[3], Dv[3];
  Bv[0] = interp_abs(F.B[0], g.NX, x[0], x[1], 0.0, 0.5);
  Bv[1] = interp_abs(F.B[1], g.NX, x[0], x[1], 0.5, 0.0);
  Bv[2] = interp_abs(F.B[2], g.NX, x[0], x[1], 0.5, 0.5);
  Dv[0] = interp_abs(F.D[0], g.NX, x[0], x[1], 0.5, 0.0);
  Dv[1] = interp_abs(F.D[1], g.NX, x[0], x[1], 0.0, 0.5);
  Dv[2] = interp_abs(F.D[2], g.NX, x[0], x[1], 0.0, 0.0);
  Pt<R> p;
  rsc_abs(g, x[0], x[1], p);
  local_full(g, p, fr.L);
  vec_hat(fr.L, Bv, fr.Bh1);
  vec_hat(fr.L, Dv, fr.Dh1);
  for (int i = 0; i < 3; ++i) {
    fr.Bh[i] = scale * fr.Bh1[i];
    fr.Dh[i] = scale * fr.Dh1[i];
  }
  fr.hq = qm * fr.L.alpha * 0.5 * g.dt;
}

// one EM half step: to the tetrad frame, Boris over dt/2, back (steps 3-5 and 7-9)
template <typename M, typename R>
__device__ __forceinline__ void em_half(const Local<M> &L, const R Dh[3], const R Bh[3],
                                        const R &hq, const R uin[3], R uout[3]) {
  R uh[3];
  cov_hat(L, uin, uh);
  boris(uh, Dh, Bh, hq);
  hat_cov(L, uh, uout);
}

// coordinate velocity dx^i/dt of Eq. (discretized-geodesic-x) from the metric at the point
template <typename M, typename R>
__device__ __forceinline__ void velocity(const Geo<M> &o, const R u[3], R &v1, R &v2) {
  const R q = fma_(o.H11 * u[0], u[0], fma_(o.H22 * u[1], u[1],
              fma_(o.H33 * u[2], u[2], fma_(o.H13, (R)2 * u[0] * u[2], (R)1))));
  const R ag = rsqrt_(o.opz * q);  // alpha / gamma
  v1 = fma_(ag, fma_(o.H11, u[0], o.H13 * u[2]), R(-o.beta1));
  v2 = ag * o.H22 * u[1];
}
template <typename R>
__device__ __forceinline__ void geo_abs(const GridP &g, const R &x1, const R &x2, Geo<R> &o) {
  Pt<R> p;
  rsc_abs(g, x1, x2, p);
  geo_from_rsc(g, p, o);
}

// dphi/dt of Eq. (discretized-geodesic-x-phi) at a point
template <typename R>
__device__ __forceinline__ R phi_rate(const GridP &g, const R &x1, const R &x2, const R u[3]) {
  Geo<R> o;
  geo_abs(g, x1, x2, o);
  const R q = fma_(o.H11 * u[0], u[0], fma_(o.H22 * u[1], u[1],
              fma_(o.H33 * u[2], u[2], fma_(o.H13, (R)2 * u[0] * u[2], (R)1))));
  return rsqrt_(o.opz * q) * fma_(o.H13, u[0], o.H33 * u[2]);
}

// The values of one step from state st = (x1, x2, phi, u1, u2, u3).
struct StepVals {
  double u1[3];  // after the first EM half step
  double t[2];   // converged geodesic iterate (u_1, u_2)
  double un[3];  // u^{n+1}
  double xn[2];  // converged x^{n+1}
  double phin;   // phi^{n+1}
  bool ok;       // finite and inside 0 <= x1 < n_r, 0 <= x2 <= n_th
};

__device__ __forceinline__ void step_values(const GridP &g, const FieldPtrsT<double> &F,
                                            const double st[6], double scale, double qm,
                                            int n_iter, StepVals &sv, Frame<double> &fr) {
  const double x[2] = {st[0], st[1]}, u[3] = {st[3], st[4], st[5]};
  frame_at(g, F, x, scale, qm, fr);
  em_half(fr.L, fr.Dh, fr.Bh, fr.hq, u, sv.u1);
  const GeoMap<double> gm(g, fr.L, sv.u1, 1.0);
  double t0 = sv.u1[0], t1 = sv.u1[1];
  for (int it = 0; it < n_iter; ++it) {
    double n0, n1;
    gm.apply(t0, t1, n0, n1);
    const bool fixed = n0 == t0 && n1 == t1;
    t0 = n0;
    t1 = n1;
    if (fixed) break;
  }
  sv.t[0] = t0;
  sv.t[1] = t1;
  const double u2[3] = {t0, t1, sv.u1[2]};
  em_half(fr.L, fr.Dh, fr.Bh, fr.hq, u2, sv.un);
  double a0 = x[0], a1 = x[1];  // the first iterate is x^n
  for (int it = 0; it < n_iter; ++it) {
    Geo<double> o;
    geo_abs(g, 0.5 * (x[0] + a0), 0.5 * (x[1] + a1), o);
    double v1, v2;
    velocity(o, sv.un, v1, v2);
    const double n0 = fma(g.dt, v1, x[0]), n1 = fma(g.dt, v2, x[1]);
    const bool fixed = n0 == a0 && n1 == a1;
    a0 = n0;
    a1 = n1;
    if (fixed) break;
  }
  sv.xn[0] = a0;
  sv.xn[1] = a1;
  sv.ok = isfinite(a0) && isfinite(a1) && isfinite(sv.un[0]) && isfinite(sv.un[1]) &&
          isfinite(sv.un[2]) && a0 >= 0.0 && a0 < g.n_r && a1 >= 0.0 && a1 <= g.n_th;
  sv.phin = sv.ok ? fma(g.dt, phi_rate(g, 0.5 * (x[0] + a0), 0.5 * (x[1] + a1), sv.un), st[2])
                  : st[2];
}

__device__ __forceinline__ bool inside(const GridP &g, const double st[6]) {
  bool ok = st[0] >= 0.0 && st[0] < g.n_r && st[1] >= 0.0 && st[1] <= g.n_th;
  for (int q = 2; q < 6; ++q) ok = ok && isfinite(st[q]);
  return ok;
}

// inverse of a 2 x 2 matrix I - A
__device__ __forceinline__ void inv_i_minus(const double A[2][2], double M[2][2]) {
  const double a = 1.0 - A[0][0], b = -A[0][1], c = -A[1][0], d = 1.0 - A[1][1];
  const double id = 1.0 / (a * d - b * c);
  M[0][0] = d * id;
  M[0][1] = -b * id;
  M[1][0] = -c * id;
  M[1][1] = a * id;
}

// The step's Jacobian at st: J[r][c] = d(output r)/d(input c), outputs x1, x2, phi, u1, u2,
// u3 after the step, inputs x1, x2, u1, u2, u3, scale (the phi column is the unit vector).
constexpr int JC = 6;  // stored input columns
__device__ void step_jacobian(const GridP &g, const FieldPtrsT<double> &F, const double st[6],
                              double scale, double qm, const StepVals &sv,
                              const Frame<double> &fr, double J[6][JC]) {
  // the implicit-function theorem's matrices: (I - dG/dt)^{-1} of the geodesic map at its fixed
  // point and (I - dt/2 dV/dx_bar)^{-1} at the final coordinate midpoint
  double Mt[2][2], Mx[2][2];
  {
    const GeoMap<double> gv(g, fr.L, sv.u1, 1.0);
    GeoMap<D2> gd;
#define WIDEN(m) gd.m = D2(gv.m);
    WIDEN(u0) WIDEN(u1) WIDEN(hu0) WIDEN(hu1) WIDEN(c0) WIDEN(c1) WIDEN(e1) WIDEN(e2)
    WIDEN(f1) WIDEN(f2) WIDEN(D1a) WIDEN(D1b) WIDEN(D2a) WIDEN(D2b) WIDEN(hdt)
    WIDEN(H11) WIDEN(H22) WIDEN(d1H11) WIDEN(d1H22) WIDEN(d2H11) WIDEN(d2H22)
#undef WIDEN
    D2 t0(sv.t[0]), t1(sv.t[1]), n0, n1;
    t0.d[0] = 1.0;
    t1.d[1] = 1.0;
    gd.apply(t0, t1, n0, n1);
    const double A[2][2] = {{n0.d[0], n0.d[1]}, {n1.d[0], n1.d[1]}};
    inv_i_minus(A, Mt);
    D2 xb1(0.5 * (st[0] + sv.xn[0])), xb2(0.5 * (st[1] + sv.xn[1]));
    xb1.d[0] = 1.0;
    xb2.d[1] = 1.0;
    Geo<D2> ob;
    geo_abs(g, xb1, xb2, ob);
    const D2 un[3] = {D2(sv.un[0]), D2(sv.un[1]), D2(sv.un[2])};
    D2 v1, v2;
    velocity(ob, un, v1, v2);
    const double h = 0.5 * g.dt;
    const double B[2][2] = {{h * v1.d[0], h * v1.d[1]}, {h * v2.d[0], h * v2.d[1]}};
    inv_i_minus(B, Mx);
  }
  // pass A: x1, x2 seeded; the metric, fields and tetrads differentiated
  {
    D2 X[2] = {D2(st[0]), D2(st[1])};
    X[0].d[0] = 1.0;
    X[1].d[1] = 1.0;
    const D2 U[3] = {D2(st[3]), D2(st[4]), D2(st[5])};
    Frame<D2> fd;
    frame_at(g, F, X, D2(scale), qm, fd);
    D2 U1[3], U2[3], U3[3];
    em_half(fd.L, fd.Dh, fd.Bh, fd.hq, U, U1);
    const GeoMap<D2> gm(g, fd.L, U1, D2(1.0));
    D2 n0, n1;
    gm.apply(D2(sv.t[0]), D2(sv.t[1]), n0, n1);
    U2[0] = D2(sv.t[0]);
    U2[1] = D2(sv.t[1]);
    U2[2] = U1[2];
    for (int k = 0; k < 2; ++k) {
      U2[0].d[k] = Mt[0][0] * n0.d[k] + Mt[0][1] * n1.d[k];
      U2[1].d[k] = Mt[1][0] * n0.d[k] + Mt[1][1] * n1.d[k];
    }
    em_half(fd.L, fd.Dh, fd.Bh, fd.hq, U2, U3);
    Geo<D2> ob;
    geo_abs(g, 0.5 * (X[0] + sv.xn[0]), 0.5 * (X[1] + sv.xn[1]), ob);
    D2 v1, v2;
    velocity(ob, U3, v1, v2);
    D2 XN[2] = {D2(sv.xn[0]), D2(sv.xn[1])};
    for (int k = 0; k < 2; ++k) {
      const double r0 = X[0].d[k] + g.dt * v1.d[k], r1 = X[1].d[k] + g.dt * v2.d[k];
      XN[0].d[k] = Mx[0][0] * r0 + Mx[0][1] * r1;
      XN[1].d[k] = Mx[1][0] * r0 + Mx[1][1] * r1;
    }
    const D2 v3 = phi_rate(g, 0.5 * (X[0] + XN[0]), 0.5 * (X[1] + XN[1]), U3);
    for (int k = 0; k < 2; ++k) {
      J[0][k] = XN[0].d[k];
      J[1][k] = XN[1].d[k];
      J[2][k] = g.dt * v3.d[k];
      J[3][k] = U3[0].d[k];
      J[4][k] = U3[1].d[k];
      J[5][k] = U3[2].d[k];
    }
  }
  // pass B: u_1, u_2, u_3 and the scale seeded; the metric at x^n and at the final
  // coordinate midpoint is fixed (values), the fields are linear in the scale
  {
    D4 U[3] = {D4(st[3]), D4(st[4]), D4(st[5])};
    for (int i = 0; i < 3; ++i) U[i].d[i] = 1.0;
    D4 Bh[3], Dh[3];
    for (int i = 0; i < 3; ++i) {
      Bh[i] = D4(fr.Bh[i]);
      Bh[i].d[3] = fr.Bh1[i];
      Dh[i] = D4(fr.Dh[i]);
      Dh[i].d[3] = fr.Dh1[i];
    }
    const D4 hq(fr.hq);
    D4 U1[3], U2[3], U3[3];
    em_half(fr.L, Dh, Bh, hq, U, U1);
    const GeoMap<D4> gm(g, fr.L, U1, D4(1.0));
    D4 n0, n1;
    gm.apply(D4(sv.t[0]), D4(sv.t[1]), n0, n1);
    U2[0] = D4(sv.t[0]);
    U2[1] = D4(sv.t[1]);
    U2[2] = U1[2];
    for (int k = 0; k < 4; ++k) {
      U2[0].d[k] = Mt[0][0] * n0.d[k] + Mt[0][1] * n1.d[k];
      U2[1].d[k] = Mt[1][0] * n0.d[k] + Mt[1][1] * n1.d[k];
    }
    em_half(fr.L, Dh, Bh, hq, U2, U3);
    Geo<double> ob;
    geo_abs(g, 0.5 * (st[0] + sv.xn[0]), 0.5 * (st[1] + sv.xn[1]), ob);
    D4 v1, v2;
    velocity(ob, U3, v1, v2);
    D4 XN[2] = {D4(sv.xn[0]), D4(sv.xn[1])};
    for (int k = 0; k < 4; ++k) {
      const double r0 = g.dt * v1.d[k], r1 = g.dt * v2.d[k];
      XN[0].d[k] = Mx[0][0] * r0 + Mx[0][1] * r1;
      XN[1].d[k] = Mx[1][0] * r0 + Mx[1][1] * r1;
    }
    const D4 v3 = phi_rate(g, 0.5 * (st[0] + XN[0]), 0.5 * (st[1] + XN[1]), U3);
    for (int k = 0; k < 4; ++k) {
      J[0][2 + k] = XN[0].d[k];
      J[1][2 + k] = XN[1].d[k];
      J[2][2 + k] = g.dt * v3.d[k];
      J[3][2 + k] = U3[0].d[k];
      J[4][2 + k] = U3[1].d[k];
      J[5][2 + k] = U3[2].d[k];
    }
  }
}

__global__ void __launch_bounds__(TPB_ADJ) k_adj_forward(GridP g, FieldPtrsT<double> F, int64_t n,
                                                        double qm, double scale, int n_steps,
                                                        int every, int n_iter,
                                                        const double *__restrict__ st0,
                                                        double *__restrict__ out,
                                                        double *__restrict__ ckpt) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n;
       k += (int64_t)gridDim.x * blockDim.x) {
    double st[6];
    for (int q = 0; q < 6; ++q) st[q] = st0[q * n + k];
    bool bad = !inside(g, st);
    for (int step = 0; step < n_steps; ++step) {
      if (step % every == 0) {
        double *c = ckpt + (int64_t)(step / every) * 6 * n;
        for (int q = 0; q < 6; ++q) c[q * n + k] = bad ? NAN : st[q];
      }
      if (bad) continue;
      StepVals sv;
      Frame<double> fr;
      step_values(g, F, st, scale, qm, n_iter, sv, fr);
      if (!sv.ok) {
        bad = true;
        continue;
      }
      st[0] = sv.xn[0]; st[1] = sv.xn[1]; st[2] = sv.phin;
      st[3] = sv.un[0]; st[4] = sv.un[1]; st[5] = sv.un[2];
    }
    for (int q = 0; q < 6; ++q) out[q * n + k] = bad ? NAN : st[q];
  }
}

__global__ void __launch_bounds__(TPB_ADJ) k_adj_backward(
    GridP g, FieldPtrsT<double> F, int64_t n, double qm, double scale, double gfac, int n_steps,
    int every, int n_iter, const double *__restrict__ ckpt, const double *__restrict__ gout,
    double *__restrict__ gin, double *__restrict__ gscale, double *__restrict__ scratch) {
  const int n_seg = (n_steps + every - 1) / every;
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n;
       k += (int64_t)gridDim.x * blockDim.x) {
    double lam[6];
    bool zero = true;
    for (int q = 0; q < 6; ++q) {
      lam[q] = gout[q * n + k];
      zero = zero && lam[q] == 0.0;
    }
    double gs = 0.0;
    bool bad = false;
    for (int seg = n_seg - 1; seg >= 0 && !bad; --seg) {
      const int s0 = seg * every, len = min(n_steps, s0 + every) - s0;
      double st[6];
      const double *c = ckpt + (int64_t)seg * 6 * n;
      for (int q = 0; q < 6; ++q) st[q] = c[q * n + k];
      if (!inside(g, st)) {
        bad = true;
        break;
      }
      // recompute the segment from its checkpoint, keeping each step's Jacobian
      for (int j = 0; j < len; ++j) {
        StepVals sv;
        Frame<double> fr;
        step_values(g, F, st, scale, qm, n_iter, sv, fr);
        if (!sv.ok) {
          bad = true;
          break;
        }
        double J[6][JC];
        step_jacobian(g, F, st, scale, qm, sv, fr, J);
        double *w = scratch + (int64_t)j * 6 * JC * n + k;
        for (int r = 0; r < 6; ++r)
          for (int cc = 0; cc < JC; ++cc) w[(int64_t)(r * JC + cc) * n] = J[r][cc];
        st[0] = sv.xn[0]; st[1] = sv.xn[1]; st[2] = sv.phin;
        st[3] = sv.un[0]; st[4] = sv.un[1]; st[5] = sv.un[2];
      }
      // reverse sweep: lambda_n = J_n^T lambda_{n+1}
      for (int j = len - 1; j >= 0 && !bad; --j) {
        const double *w = scratch + (int64_t)j * 6 * JC * n + k;
        double nl[JC] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
        for (int r = 0; r < 6; ++r)
          for (int cc = 0; cc < JC; ++cc) nl[cc] = fma(w[(int64_t)(r * JC + cc) * n], lam[r], nl[cc]);
        // inputs x1, x2, u1, u2, u3 map to state rows 0, 1, 3, 4, 5; phi passes through
        lam[0] = nl[0];
        lam[1] = nl[1];
        lam[3] = nl[2];
        lam[4] = nl[3];
        lam[5] = nl[4];
        gs += nl[5];
      }
    }
    // a particle that reached a boundary has no gradient: zero where its cotangent was zero
    // (it does not enter the loss), NaN otherwise
    const double fill = zero ? 0.0 : NAN;
    for (int q = 0; q < 6; ++q) gin[q * n + k] = bad ? fill : lam[q];
    gscale[k] = bad ? fill : gs * gfac;
  }
}

// out[0] = sum of x[0..n): one block, fixed order (deterministic)
__global__ void __launch_bounds__(1024) k_sum(const double *__restrict__ x, int64_t n,
                                              double *__restrict__ out) {
  __shared__ double red[1024];
  double a = 0.0;
  for (int64_t i = threadIdx.x; i < n; i += blockDim.x) a += x[i];
  red[threadIdx.x] = a;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) out[0] = red[0];
}

int adj_blocks(int64_t n) {
  int64_t b = (n + TPB_ADJ - 1) / TPB_ADJ;
  const int64_t cap = 152 * 32;
  return (int)(b < 1 ? 1 : (b > cap ? cap : b));
}

}  // namespace

cudaError_t launch_adjoint_forward(const GridP &g, const FieldPtrsT<double> &F, int64_t n,
                                   double qm, double scale, int n_steps, int every, int n_iter,
                                   const double *st0, double *out, double *ckpt,
                                   cudaStream_t st) {
  if (n <= 0) return cudaGetLastError();
  k_adj_forward<<<adj_blocks(n), TPB_ADJ, 0, st>>>(g, F, n, qm, scale, n_steps, every, n_iter,
                                                   st0, out, ckpt);
  COUNT_LAUNCH(1);
  return cudaGetLastError();
}

cudaError_t launch_adjoint_backward(const GridP &g, const FieldPtrsT<double> &F, int64_t n,
                                    double qm, double scale, double gfac, int n_steps, int every,
                                    int n_iter,
                                    const double *ckpt, const double *gout, double *gin,
                                    double *gscale_pp, double *gscale_sum, double *scratch,
                                    cudaStream_t st) {
  if (n <= 0) return cudaMemsetAsync(gscale_sum, 0, sizeof(double), st);
  k_adj_backward<<<adj_blocks(n), TPB_ADJ, 0, st>>>(g, F, n, qm, scale, gfac, n_steps, every,
                                                    n_iter, ckpt, gout, gin, gscale_pp, scratch);
  k_sum<<<1, 1024, 0, st>>>(gscale_pp, n, gscale_sum);
  COUNT_LAUNCH(2);
  return cudaGetLastError();
}
