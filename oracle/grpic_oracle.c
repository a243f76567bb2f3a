/*
 * grpic_oracle.c -- plain, slow FP64 CPU oracle of the 2D-axisymmetric
 * general-relativistic PIC step of arXiv:2511.17701 (Entity, GR module).
 *
 * TEST INFRASTRUCTURE. This file exists to check the CUDA library against the
 * paper. Only tests/, __graft_entry__.smoke() and bench.py's cpu_baseline and
 * reference leg may build, load or call it. It shares no code, header, table
 * or constant generator with paper_2511_17701_gb300/ and imports nothing from it.
 *
 * Written for a reader holding the paper: every routine cites the section or
 * equation it follows and keeps its notation. There is no blocking, fusion or
 * precomputed table: the metric is evaluated from its closed form wherever a
 * value is needed. Built with -O2 -ffp-contract=off.
 *
 * Where the paper is silent or garbled the routine states the reading it takes.
 */
#include "grpic_oracle.h"

#include <complex.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define G ORA_G

static double PI_ = 3.14159265358979323846;

/* ------------------------------------------------------------------------ */
/* grid geometry: code coordinates are uniform (Sec. 3, "code units"); the    */
/* quasi-spherical map of Appendix A:                                          */
/*   r = r0 + exp(xi), xi = log(r_min - r0) + x1 dxi,                          */
/*   theta = eta + 2 h0 eta (pi - 2 eta)(pi - eta) / pi^2, eta = x2 deta,      */
/* with dxi = log((r_max - r0)/(r_min - r0)) / n_r and deta = pi / n_theta.    */
/* r0 = h0 = 0 is the plain log-r grid with uniform theta. The map's          */
/* functions are in pusher_generic.inc (they serve both instances).           */
/* ------------------------------------------------------------------------ */
static double dxi_of(const ora_params *p) {
  return log((p->r_max - p->r0) / (p->r_min - p->r0)) / p->n_r;
}
static double dth_of(const ora_params *p) { return PI_ / p->n_th; } /* deta */
static int NX_of(const ora_params *p) { return p->n_r + 2 * G + 1; }
static int NY_of(const ora_params *p) { return p->n_th + 2 * G + 1; }
static int64_t plane_size(const ora_params *p) { return (int64_t)NX_of(p) * NY_of(p); }

/* element (i, j) of a plane in the storage convention of grpic_oracle.h */
#define AT(pl, i, j) (pl)[(int64_t)((j) + G) * NX + ((i) + G)]

/* Yee offsets (Fig. 1): B^1 (i, j+1/2), B^2 (i+1/2, j), B^3 (i+1/2, j+1/2),
 *                       D^1 (i+1/2, j), D^2 (i, j+1/2), D^3 (i, j).          */
static const double SB[3][2] = {{0.0, 0.5}, {0.5, 0.0}, {0.5, 0.5}};
static const double SD[3][2] = {{0.5, 0.0}, {0.0, 0.5}, {0.0, 0.0}};

/* The metric, tetrads, Boris step, geodesic substep, interpolation and the frozen-field
 * step, in double (the oracle) ... */
#define REAL double
#define FN(name) name
#define METRIC ora_metric
#define RSQRT sqrt
#define REXP exp
#define RSIN sin
#define RCOS cos
#define RE(x) (x)
#include "pusher_generic.inc"
#undef REAL
#undef FN
#undef METRIC
#undef RSQRT
#undef REXP
#undef RSIN
#undef RCOS
#undef RE

/* ... and in double complex, for complex-step derivatives of the frozen-field push */
typedef struct {
  double complex r, th, f, g, h11, h22, h33, h13, H11, H22, H33, H13;
  double complex alpha, beta1, sqrt_h, sqrt_ht;
  double complex d1H11, d1H22, d1H33, d1H13, d1alpha, d1beta1;
  double complex d2H11, d2H22, d2H33, d2H13, d2alpha, d2beta1;
} ora_metric_cs;
#define REAL double complex
#define FN(name) name##_cs
#define METRIC ora_metric_cs
#define RSQRT csqrt
#define REXP cexp
#define RSIN csin
#define RCOS ccos
#define RE(x) creal(x)
#include "pusher_generic.inc"
#undef REAL
#undef FN
#undef METRIC
#undef RSQRT
#undef REXP
#undef RSIN
#undef RCOS
#undef RE
/* Polar area of the half cell next to the axis at radius x1 (Sec. 3.3.2 and the
 * closed form of Appendix A), per unit phi: integral_0^{1/2} sqrt(h) dx2 with Sigma
 * taken at its axis value. Reading: no factor 2 pi (dphi = 1, as the closed form). */
static double polar_area(const ora_params *p, double x1) {
  const double M = p->metric == 1 ? 1.0 : 0.0;
  const double a = p->metric == 1 ? p->a : 0.0;
  double r, f, th, g, gp;
  map_r(p, x1, &r, &f);
  map_th(p, 0.5, &th, &g, &gp); /* theta at the half cell's edge; x2 -> theta is monotone */
  return f * (r * r + a * a) * sqrt(1.0 + 2.0 * M * r / (r * r + a * a)) * (1.0 - cos(th));
}

/* theta(eta_j) + theta(eta_{j+1}) and theta(eta_{j+1}) - theta(eta_j) of the face rows j,
 * j + 1, with the cubic's difference expanded so that nothing cancels:
 * p(eta + d) - p(eta) = d (pi^2 - 6 pi eta + 6 eta^2) + d^2 (6 eta - 3 pi) + 2 d^3 for
 * p(eta) = eta (pi - 2 eta)(pi - eta) = pi^2 eta - 3 pi eta^2 + 2 eta^3. */
static double theta_sum(const ora_params *p, int j) {
  const double de = dth_of(p), e0 = j * de, e1 = (j + 1) * de, k = 2.0 * p->h0 / (PI_ * PI_);
  const double p0 = e0 * (PI_ - 2.0 * e0) * (PI_ - e0), p1 = e1 * (PI_ - 2.0 * e1) * (PI_ - e1);
  return (2 * j + 1) * de + k * (p0 + p1);
}
static double theta_diff(const ora_params *p, int j) {
  const double de = dth_of(p), e0 = j * de, k = 2.0 * p->h0 / (PI_ * PI_);
  return de + k * (de * (PI_ * PI_ - 6.0 * PI_ * e0 + 6.0 * e0 * e0) +
                   de * de * (6.0 * e0 - 3.0 * PI_) + 2.0 * de * de * de);
}

/* ------------------------------------------------------------------------ */
/* Wald vacuum potential, Eq. (Wald), and the vertical field (its a = 0       */
/* limit). Complex arithmetic so that derivatives can be taken by the complex */
/* step, d f/dx = Im f(x + i e)/e, exact to rounding.                         */
/* ------------------------------------------------------------------------ */
typedef double complex cplx;
static void wald_potential_c(const ora_params *p, int kind, double B0, cplx x1, cplx x2,
                             cplx *A0, cplx *A1, cplx *A3) {
  const double M = p->metric == 1 ? 1.0 : 0.0;
  const double a = p->metric == 1 ? p->a : 0.0;
  cplx r, f, th, g, gp;
  map_r_cs(p, x1, &r, &f);
  map_th_cs(p, x2, &th, &g, &gp);
  cplx s = csin(th), c = ccos(th), s2 = s * s;
  if (kind == 2) { /* vertical: A_phi = B0 r^2 sin^2(theta) / 2 */
    *A0 = 0.0; *A1 = 0.0; *A3 = 0.5 * B0 * r * r * s2;
    return;
  }
  if (kind == 4) { /* magnetic monopole of the BZ test (Sec. 4.5): A_phi = -B0 cos(theta) */
    *A0 = 0.0; *A1 = 0.0; *A3 = -B0 * c;
    return;
  }
  cplx Sig = r * r + a * a * c * c;
  cplx Del = r * r - 2.0 * M * r + a * a;
  cplx AA = (r * r + a * a) * (r * r + a * a) - a * a * Del * s2;
  cplx z = 2.0 * M * r / Sig;
  cplx h13 = -f * a * (1.0 + z) * s2;     /* code-unit h_13 (dphi = 1), f = dr/dx1 */
  cplx h11 = f * f * (1.0 + z);
  cplx h33 = AA * s2 / Sig;
  cplx beta1 = z / (1.0 + z) / f;
  cplx g00 = -(1.0 - z);
  *A0 = 0.5 * B0 * (h13 * beta1 + 2.0 * a * g00);
  *A1 = 0.5 * B0 * (h13 + 2.0 * a * h11 * beta1);
  *A3 = 0.5 * B0 * (h33 + 2.0 * a * h13 * beta1);
}

static void wald_potential(const ora_params *p, int kind, double B0, double x1, double x2,
                           double A[3]) {
  cplx A0, A1, A3;
  wald_potential_c(p, kind, B0, x1, x2, &A0, &A1, &A3);
  A[0] = creal(A0); A[1] = creal(A1); A[2] = creal(A3);
}

/* The difference A_1(x1, theta_{j+1}) - A_1(x1, theta_j) of the Wald potential, for the
 * discrete curl that gives B^3. With A_1 = (B0/2) a f (2 M r (1 + cos^2)/Sigma - sin^2) and
 * sin^2(b) - sin^2(a) = sin(b - a) sin(b + a), cos^2(b) - cos^2(a) = -(sin^2(b) - sin^2(a)):
 *   dA_1 = -(B0/2) a f D (1 + 2 M r (r^2 - a^2) / (Sigma_a Sigma_b)),
 *   D = sin(theta_{j+1} - theta_j) sin(theta_{j+1} + theta_j),
 * exact in real arithmetic; the plain difference of the two values loses about 1/dtheta^2
 * of its digits next to the axes, where A_1 varies as theta^2. */
static double wald_dA1_theta(const ora_params *p, int kind, double B0, double x1, int j) {
  if (kind != 1) return 0.0; /* the vertical field has A_1 = 0 */
  const double M = p->metric == 1 ? 1.0 : 0.0;
  const double a = p->metric == 1 ? p->a : 0.0;
  double r, f, tha, thb, g, gp;
  map_r(p, x1, &r, &f);
  map_th(p, j, &tha, &g, &gp);
  map_th(p, j + 1, &thb, &g, &gp);
  const double ca = cos(tha), cb = cos(thb);
  const double Sa = r * r + a * a * ca * ca, Sb = r * r + a * a * cb * cb;
  const double D = sin(theta_diff(p, j)) * sin(theta_sum(p, j));
  return -0.5 * B0 * a * f * D * (1.0 + 2.0 * M * r * (r * r - a * a) / (Sa * Sb));
}

/* The difference A_3(x1, theta_{j+1}) - A_3(x1, theta_j) for the discrete curl that gives
 * B^1. For the monopole, -B0 (cos(theta_{j+1}) - cos(theta_j)) = 2 B0 sin((theta_j +
 * theta_{j+1}) / 2) sin((theta_{j+1} - theta_j) / 2) in product form: the plain difference
 * of the cosines loses about 1/dtheta^2 of its digits next to the axes. Other kinds: the
 * plain difference. */
static double dA3_theta(const ora_params *p, int kind, double B0, double x1, int j) {
  if (kind == 4)
    return 2.0 * B0 * sin(0.5 * theta_sum(p, j)) * sin(0.5 * theta_diff(p, j));
  double A[3], Ab[3];
  wald_potential(p, kind, B0, x1, j, A);
  wald_potential(p, kind, B0, x1, j + 1, Ab);
  return Ab[2] - A[2];
}

/* derivatives of A_0, A_1, A_3 with respect to x1 (dir 0) or x2 (dir 1) */
static void wald_dpotential(const ora_params *p, int kind, double B0, double x1, double x2,
                            int dir, double dA[3]) {
  const double e = 1e-30;
  cplx A0, A1, A3;
  if (dir == 0) wald_potential_c(p, kind, B0, x1 + e * I, x2, &A0, &A1, &A3);
  else wald_potential_c(p, kind, B0, x1, x2 + e * I, &A0, &A1, &A3);
  dA[0] = cimag(A0) / e; dA[1] = cimag(A1) / e; dA[2] = cimag(A3) / e;
}

/* Analytic D^i and B^i of the stationary potential at a point (Sec. 2.2):
 * E_i = F_i0 = d_i A_0, B^i = eps^{ijk} d_j A_k / sqrt(h), and D from the inverse of
 * Eq. (aux): E_i = alpha h_ij D^j + e_ijk beta^j B^k (theta decoupled, so the r-phi block
 * inverts with h^{ij}). sqrt(h) B^2 = -d_1 A_3 and sqrt(h) B^3 = -d_2 A_1 are used as
 * products so that the axis, where sqrt(h) = 0, needs no division. */
static void wald_fields_point(const ora_params *p, int kind, double B0, double x1, double x2,
                              double B[3], double D[3]) {
  ora_metric m;
  metric_eval(p, x1, x2, 0, 0, &m);
  double d1[3], d2[3];
  wald_dpotential(p, kind, B0, x1, x2, 0, d1);
  wald_dpotential(p, kind, B0, x1, x2, 1, d2);
  double E1 = d1[0], E2 = d2[0], E3 = 0.0;
  double shB2 = -d1[2], shB3 = -d2[1];
  B[0] = d2[2] / m.sqrt_h;
  B[1] = shB2 / m.sqrt_h;
  B[2] = shB3 / m.sqrt_h;
  double rhs3 = E3 - m.beta1 * shB2; /* = alpha (h_31 D^1 + h_33 D^3) */
  D[0] = (m.H11 * E1 + m.H13 * rhs3) / m.alpha;
  D[1] = m.H22 * (E2 + m.beta1 * shB3) / m.alpha;
  D[2] = (m.H13 * E1 + m.H33 * rhs3) / m.alpha;
}

/* ------------------------------------------------------------------------ */
/* One particle, the eleven steps of Sec. 3.1, then the boundaries of         */
/* Sec. 3.3.3. field_mode 0: fields from the B^n and D^n planes; 1: analytic  */
/* stationary field of kind `fkind` and amplitude B0 (used by the pins).       */
/* counters: 0 left inner, 1 left outer, 2 axis reflections, 3 non-finite.    */
/* ------------------------------------------------------------------------ */
static void push_one(const ora_params *p, const double *F, ora_species *s, int64_t k,
                     int field_mode, int fkind, double B0, int64_t cnt[4]) {
  const int NX = NX_of(p);
  const int64_t PS = plane_size(p);
  const double dt = p->dt;
  /* step 1: save previous location */
  s->i1p[k] = s->i1[k]; s->i2p[k] = s->i2[k];
  s->dx1p[k] = s->dx1[k]; s->dx2p[k] = s->dx2[k];
  if (s->tag[k] != 1) { s->tag[k] = 0; return; }
  double x1 = s->i1[k] + s->dx1[k], x2 = s->i2[k] + s->dx2[k];
  const double m2 = s->massless ? 0.0 : 1.0;
  /* step 2: fields at x^n (not needed by massless particles) */
  double Dv[3], Bv[3];
  if (s->massless) {
    for (int c = 0; c < 3; ++c) Bv[c] = Dv[c] = 0.0;
  } else if (field_mode == 0) {
    for (int c = 0; c < 3; ++c) {
      Bv[c] = interp(F + (ORA_BN1 + c) * PS, NX, x1, x2, SB[c][0], SB[c][1]);
      Dv[c] = interp(F + (ORA_D1 + c) * PS, NX, x1, x2, SD[c][0], SD[c][1]);
    }
  } else if (fkind != 0) {
    wald_fields_point(p, fkind, B0, x1, x2, Bv, Dv);
  } else {
    for (int c = 0; c < 3; ++c) Bv[c] = Dv[c] = 0.0;
  }
  /* metric (with derivatives) at x^n, theta regularised near the axis */
  ora_metric m;
  metric_eval(p, x1, x2, 1, 1, &m);
  /* step 3: fields and velocity to the tetrad basis */
  double Dh[3], Bh[3], uh[3], u[3] = {s->u1[k], s->u2[k], s->u3[k]};
  vec_to_hat(&m, Dv, Dh);
  vec_to_hat(&m, Bv, Bh);
  cov_to_hat(&m, u, uh);
  double hq = s->qm * m.alpha * 0.5 * dt;
  /* steps 3-5 and 7-9 (the EM push) are skipped for massless particles (Sec. 3.1) */
  if (!s->massless) {
    boris(uh, Dh, Bh, hq);   /* step 4 */
    hat_to_cov(&m, uh, u);   /* step 5 */
  }
  geodesic_u(p, &m, u, m2);  /* step 6 */
  if (!s->massless) {
    cov_to_hat(&m, u, uh);   /* step 7 */
    boris(uh, Dh, Bh, hq);   /* step 8 */
    hat_to_cov(&m, uh, u);   /* step 9 */
  }
  /* step 10: implicit coordinate push, Eq. (discretized-geodesic-x), metric at the
   * midpoint x_bar = (x^n + x~)/2; positions kept as cell + offset */
  double dxt1 = s->dx1[k], dxt2 = s->dx2[k];
  for (int it = 0; it < p->n_iter; ++it) {
    double xb1 = s->i1[k] + 0.5 * (s->dx1[k] + dxt1);
    double xb2 = s->i2[k] + 0.5 * (s->dx2[k] + dxt2);
    ora_metric mb;
    metric_eval(p, xb1, xb2, 1, 0, &mb);
    double gam = gamma_of(&mb, u, m2);
    double v1 = mb.alpha / gam * (mb.H11 * u[0] + mb.H13 * u[2]) - mb.beta1;
    double v2 = mb.alpha / gam * (mb.H22 * u[1]);
    dxt1 = s->dx1[k] + dt * v1;
    dxt2 = s->dx2[k] + dt * v2;
  }
  if (!(isfinite(u[0]) && isfinite(u[1]) && isfinite(u[2]) && isfinite(dxt1) &&
        isfinite(dxt2) && fabs(dxt1) < 1e6 && fabs(dxt2) < 1e6)) {
    s->tag[k] = 0;
    cnt[3] += 1;
    return;
  }
  int i1n = s->i1[k] + (int)floor(dxt1);
  int i2n = s->i2[k] + (int)floor(dxt2);
  double dx1n = dxt1 - floor(dxt1), dx2n = dxt2 - floor(dxt2);
  /* boundaries (Sec. 3.3.3): reflection off the axes, removal through the horizon
   * layer into the ghost zone (reading: i1 < 0) and through the outer edge */
  if (i2n < 0) { i2n = 0; dx2n = 1.0 - dx2n; u[1] = -u[1]; cnt[2] += 1; }
  else if (i2n >= p->n_th) { i2n = p->n_th - 1; dx2n = 1.0 - dx2n; u[1] = -u[1]; cnt[2] += 1; }
  if (i2n < 0 || i2n >= p->n_th) { s->tag[k] = 0; cnt[3] += 1; return; }
  s->i1[k] = i1n; s->i2[k] = i2n; s->dx1[k] = dx1n; s->dx2[k] = dx2n;
  s->u1[k] = u[0]; s->u2[k] = u[1]; s->u3[k] = u[2];
  if (i1n < 0) { s->tag[k] = 2; cnt[0] += 1; }
  else if (i1n >= p->n_r) { s->tag[k] = 2; cnt[1] += 1; }
  /* step 11: out-of-plane coordinate, Eq. (discretized-geodesic-x-phi), at
   * x^{n+1/2}; reading: midpoint of the stored x^n and the final x^{n+1} */
  double xm1 = 0.5 * ((s->i1p[k] + s->dx1p[k]) + (i1n + dx1n));
  double xm2 = 0.5 * ((s->i2p[k] + s->dx2p[k]) + (i2n + dx2n));
  ora_metric mm;
  metric_eval(p, xm1, xm2, 1, 0, &mm);
  double gam = gamma_of(&mm, u, m2);
  s->phi[k] += dt * mm.alpha / gam * (mm.H13 * u[0] + mm.H33 * u[2]);
}

void ora_push(const ora_params *p, const double *F, ora_species *s, int field_mode,
              int fkind, double B0, int64_t *counters) {
  int64_t c0 = 0, c1 = 0, c2 = 0, c3 = 0;
#pragma omp parallel for schedule(static) reduction(+ : c0, c1, c2, c3)
  for (int64_t k = 0; k < s->n; ++k) {
    int64_t cnt[4] = {0, 0, 0, 0};
    push_one(p, F, s, k, field_mode, fkind, B0, cnt);
    c0 += cnt[0]; c1 += cnt[1]; c2 += cnt[2]; c3 += cnt[3];
  }
  counters[0] += c0; counters[1] += c1; counters[2] += c2; counters[3] += c3;
}

/* ------------------------------------------------------------------------ */
/* Charge-conserving deposit, Sec. 3.2, Eq. (charge-conservation-disc).       */
/* Reading of the scheme of paper I: first-order (area-weighting) conformal   */
/* shape in code coordinates and the zigzag split of Umeda et al. (2003):      */
/* the move x_a -> x_b is cut at the relay point                               */
/*   x_r = min(min(i_a, i_b) + 1, max(max(i_a, i_b), (x_a + x_b)/2))           */
/* per dimension, each piece lies in one cell and deposits its flux onto the   */
/* two faces it crosses with linear weights. J^3 = q alpha u^3 / gamma         */
/* (Sec. 3.2) at x^{n+1/2}, u^3 = h^{3j} u_j, with the same theta regularisation*/
/* as the pusher. Real particles only: nothing is deposited across the axis.   */
/* ------------------------------------------------------------------------ */
static void add_dep(double *J, double *Ja, int NX, int i, int j, double v) {
  AT(J, i, j) += v;
  AT(Ja, i, j) += fabs(v);
}

void ora_deposit(const ora_params *p, double *F, ora_species *sp, int ns) {
  const int NX = NX_of(p);
  const int64_t PS = plane_size(p);
  for (int c = 0; c < 3; ++c) {
    memset(F + (ORA_J1 + c) * PS, 0, sizeof(double) * PS);
    memset(F + (ORA_JA1 + c) * PS, 0, sizeof(double) * PS);
  }
  double *J1 = F + ORA_J1 * PS, *J2 = F + ORA_J2 * PS, *J3 = F + ORA_J3 * PS;
  double *A1 = F + ORA_JA1 * PS, *A2 = F + ORA_JA2 * PS, *A3 = F + ORA_JA3 * PS;
  const double dt = p->dt;
  for (int si = 0; si < ns; ++si) {
    ora_species *s = &sp[si];
    if (s->massless) continue; /* reading: massless particles are neutral */
    for (int64_t k = 0; k < s->n; ++k) {
      if (s->tag[k] == 0) continue;
      double q = s->qc * s->w[k];
      int ia = s->i1p[k], ja = s->i2p[k], ib = s->i1[k], jb = s->i2[k];
      double xa1 = ia + s->dx1p[k], xa2 = ja + s->dx2p[k];
      double xb1 = ib + s->dx1[k], xb2 = jb + s->dx2[k];
      double xr1 = fmin(fmin(ia, ib) + 1.0, fmax(fmax(ia, ib), 0.5 * (xa1 + xb1)));
      double xr2 = fmin(fmin(ja, jb) + 1.0, fmax(fmax(ja, jb), 0.5 * (xa2 + xb2)));
      /* piece a: x_a -> x_r inside cell (ia, ja) */
      double F1 = q * (xr1 - xa1) / dt, F2 = q * (xr2 - xa2) / dt;
      double W1 = 0.5 * (xa1 + xr1) - ia, W2 = 0.5 * (xa2 + xr2) - ja;
      add_dep(J1, A1, NX, ia, ja, F1 * (1.0 - W2));
      add_dep(J1, A1, NX, ia, ja + 1, F1 * W2);
      add_dep(J2, A2, NX, ia, ja, F2 * (1.0 - W1));
      add_dep(J2, A2, NX, ia + 1, ja, F2 * W1);
      /* piece b: x_r -> x_b inside cell (ib, jb) */
      F1 = q * (xb1 - xr1) / dt; F2 = q * (xb2 - xr2) / dt;
      W1 = 0.5 * (xr1 + xb1) - ib; W2 = 0.5 * (xr2 + xb2) - jb;
      add_dep(J1, A1, NX, ib, jb, F1 * (1.0 - W2));
      add_dep(J1, A1, NX, ib, jb + 1, F1 * W2);
      add_dep(J2, A2, NX, ib, jb, F2 * (1.0 - W1));
      add_dep(J2, A2, NX, ib + 1, jb, F2 * W1);
      /* out-of-plane component at the midpoint */
      double xm1 = 0.5 * (xa1 + xb1), xm2 = 0.5 * (xa2 + xb2);
      ora_metric mm;
      metric_eval(p, xm1, xm2, 1, 0, &mm);
      double u[3] = {s->u1[k], s->u2[k], s->u3[k]};
      double v3 = mm.alpha / gamma_of(&mm, u, 1.0) * (mm.H13 * u[0] + mm.H33 * u[2]);
      int i0 = (int)floor(xm1), j0 = (int)floor(xm2);
      double w1 = xm1 - i0, w2 = xm2 - j0;
      add_dep(J3, A3, NX, i0, j0, q * v3 * (1.0 - w1) * (1.0 - w2));
      add_dep(J3, A3, NX, i0 + 1, j0, q * v3 * w1 * (1.0 - w2));
      add_dep(J3, A3, NX, i0, j0 + 1, q * v3 * (1.0 - w1) * w2);
      add_dep(J3, A3, NX, i0 + 1, j0 + 1, q * v3 * w1 * w2);
    }
  }
}

/* charge sum_p q S at the grid nodes from x^n (prev = 1) or x^{n+1} (prev = 0):
 * the conformal density sqrt(h) rho of Sec. 3.2 (diagnostic for the pins) */
void ora_charge(const ora_params *p, const ora_species *sp, int ns, int prev, double *rho) {
  const int NX = NX_of(p);
  memset(rho, 0, sizeof(double) * plane_size(p));
  for (int si = 0; si < ns; ++si) {
    const ora_species *s = &sp[si];
    if (s->massless) continue;
    for (int64_t k = 0; k < s->n; ++k) {
      if (s->tag[k] == 0) continue;
      int i = prev ? s->i1p[k] : s->i1[k], j = prev ? s->i2p[k] : s->i2[k];
      double w1 = prev ? s->dx1p[k] : s->dx1[k], w2 = prev ? s->dx2p[k] : s->dx2[k];
      double q = s->qc * s->w[k];
      AT(rho, i, j) += q * (1.0 - w1) * (1.0 - w2);
      AT(rho, i + 1, j) += q * w1 * (1.0 - w2);
      AT(rho, i, j + 1) += q * (1.0 - w1) * w2;
      AT(rho, i + 1, j + 1) += q * w1 * w2;
    }
  }
}

/* ------------------------------------------------------------------------ */
/* Field solver, Sec. 3.3.                                                    */
/* ------------------------------------------------------------------------ */
/* metric at the stored point (i, j) of a Yee class with offsets (s1, s2) */
static void metric_at(const ora_params *p, double s1, double s2, int i, int j, ora_metric *m) {
  metric_eval(p, i + s1, j + s2, 0, 0, m);
}
static double sht_h13(const ora_metric *m) { return m->sqrt_ht * m->h13; }          /* [sqrt(h~) h_13]        */
static double sht_b1(const ora_metric *m) { return m->sqrt_ht * m->sqrt_h * m->beta1; } /* [sqrt(h~ h) beta^1] */

/* Eq. (discretized-auxE) with the volume-weighted averages of
 * Eq. (discretized-auxH): E_i from (B, D) on stored i in [-1, n_r + 1]. */
static void aux_E(const ora_params *p, const double *B[3], const double *D[3], double *E[3]) {
  const int NX = NX_of(p);
  ora_metric m, ma, mb;
  for (int j = 0; j <= p->n_th; ++j)
    for (int i = -1; i <= p->n_r + 1; ++i) {
      /* E_1 at (i+1/2, j) */
      metric_at(p, 0.5, 0.0, i, j, &m);
      metric_at(p, 0.0, 0.0, i, j, &ma);
      metric_at(p, 0.0, 0.0, i + 1, j, &mb);
      double avg = (sht_h13(&ma) * AT(D[2], i, j) + sht_h13(&mb) * AT(D[2], i + 1, j)) /
                   (2.0 * m.sqrt_ht);
      AT(E[0], i, j) = m.alpha * (m.h11 * AT(D[0], i, j) + avg);
      /* E_3 at (i, j); zero on the axes by symmetry */
      if (j == 0 || j == p->n_th) {
        AT(E[2], i, j) = 0.0;
      } else {
        metric_at(p, 0.0, 0.0, i, j, &m);
        metric_at(p, 0.5, 0.0, i - 1, j, &ma);
        metric_at(p, 0.5, 0.0, i, j, &mb);
        double a13 = (sht_h13(&ma) * AT(D[0], i - 1, j) + sht_h13(&mb) * AT(D[0], i, j)) /
                     (2.0 * m.sqrt_ht);
        double ab2 = (sht_b1(&ma) * AT(B[1], i - 1, j) + sht_b1(&mb) * AT(B[1], i, j)) /
                     (2.0 * m.sqrt_ht);
        AT(E[2], i, j) = m.alpha * (m.h33 * AT(D[2], i, j) + a13) + ab2;
      }
    }
  for (int j = 0; j < p->n_th; ++j)
    for (int i = -1; i <= p->n_r + 1; ++i) {
      /* E_2 at (i, j+1/2); reading: beta^1 in <sqrt(h) beta B^3> */
      metric_at(p, 0.0, 0.5, i, j, &m);
      metric_at(p, 0.5, 0.5, i - 1, j, &ma);
      metric_at(p, 0.5, 0.5, i, j, &mb);
      double ab3 = (sht_b1(&ma) * AT(B[2], i - 1, j) + sht_b1(&mb) * AT(B[2], i, j)) /
                   (2.0 * m.sqrt_ht);
      AT(E[1], i, j) = m.alpha * m.h22 * AT(D[1], i, j) - ab3;
    }
}

/* Eq. (discretized-auxE), H part: H_i from (B, D) on stored i in [-1, n_r + 1]. */
static void aux_H(const ora_params *p, const double *B[3], const double *D[3], double *H[3]) {
  const int NX = NX_of(p);
  ora_metric m, ma, mb;
  for (int j = 0; j < p->n_th; ++j)
    for (int i = -1; i <= p->n_r + 1; ++i) {
      /* H_1 at (i, j+1/2) */
      metric_at(p, 0.0, 0.5, i, j, &m);
      metric_at(p, 0.5, 0.5, i - 1, j, &ma);
      metric_at(p, 0.5, 0.5, i, j, &mb);
      double a13 = (sht_h13(&ma) * AT(B[2], i - 1, j) + sht_h13(&mb) * AT(B[2], i, j)) /
                   (2.0 * m.sqrt_ht);
      AT(H[0], i, j) = m.alpha * (m.h11 * AT(B[0], i, j) + a13);
      /* H_3 at (i+1/2, j+1/2) */
      metric_at(p, 0.5, 0.5, i, j, &m);
      metric_at(p, 0.0, 0.5, i, j, &ma);
      metric_at(p, 0.0, 0.5, i + 1, j, &mb);
      double b13 = (sht_h13(&ma) * AT(B[0], i, j) + sht_h13(&mb) * AT(B[0], i + 1, j)) /
                   (2.0 * m.sqrt_ht);
      double d2 = (sht_b1(&ma) * AT(D[1], i, j) + sht_b1(&mb) * AT(D[1], i + 1, j)) /
                  (2.0 * m.sqrt_ht);
      AT(H[2], i, j) = m.alpha * (m.h33 * AT(B[2], i, j) + b13) - d2;
    }
  for (int j = 0; j <= p->n_th; ++j)
    for (int i = -1; i <= p->n_r + 1; ++i) {
      /* H_2 at (i+1/2, j) */
      metric_at(p, 0.5, 0.0, i, j, &m);
      metric_at(p, 0.0, 0.0, i, j, &ma);
      metric_at(p, 0.0, 0.0, i + 1, j, &mb);
      double d3 = (sht_b1(&ma) * AT(D[2], i, j) + sht_b1(&mb) * AT(D[2], i + 1, j)) /
                  (2.0 * m.sqrt_ht);
      AT(H[1], i, j) = m.alpha * m.h22 * AT(B[1], i, j) + d3;
    }
}

/* Eq. (discretized-faraday): Bout = Bin - dt curl E, on the evolved points;
 * B^2 on the axes is not evolved (it vanishes there). */
static void faraday(const ora_params *p, const double *Bin[3], const double *E[3],
                    double *Bout[3]) {
  const int NX = NX_of(p);
  const double dt = p->dt;
  ora_metric m;
  for (int j = 0; j < p->n_th; ++j)
    for (int i = 0; i <= p->n_r; ++i) {
      metric_at(p, 0.0, 0.5, i, j, &m);
      AT(Bout[0], i, j) = AT(Bin[0], i, j) - dt * (AT(E[2], i, j + 1) - AT(E[2], i, j)) / m.sqrt_h;
    }
  for (int j = 1; j < p->n_th; ++j)
    for (int i = 0; i < p->n_r; ++i) {
      metric_at(p, 0.5, 0.0, i, j, &m);
      AT(Bout[1], i, j) = AT(Bin[1], i, j) + dt * (AT(E[2], i + 1, j) - AT(E[2], i, j)) / m.sqrt_h;
    }
  for (int j = 0; j < p->n_th; ++j)
    for (int i = 0; i < p->n_r; ++i) {
      metric_at(p, 0.5, 0.5, i, j, &m);
      double curl = (AT(E[1], i + 1, j) - AT(E[1], i, j)) - (AT(E[0], i, j + 1) - AT(E[0], i, j));
      AT(Bout[2], i, j) = AT(Bin[2], i, j) - dt * curl / m.sqrt_h;
    }
}

/* Eq. (discretized-ampere): Dout = Din + dt (curl H - 4 pi J) / sqrt(h); on the
 * axes D^1 follows the integral form of Sec. 3.3.2 with the polar area and D^3
 * is not evolved. Reading of the axis current term: the deposit gives the axis
 * node the whole radial flux into its half cell, so the coefficient that keeps
 * the discrete Gauss law exact is 4 pi (the printed 2 pi pairs with a current
 * counted over the full dual face). The theta = pi axis takes -H_3(j - 1/2). */
static void ampere(const ora_params *p, const double *Din[3], const double *H[3],
                   const double *J[3], double *Dout[3]) {
  const int NX = NX_of(p);
  const double dt = p->dt, fpi = 4.0 * PI_;
  ora_metric m;
  for (int j = 0; j <= p->n_th; ++j)
    for (int i = 0; i < p->n_r; ++i) {
      if (j == 0) {
        AT(Dout[0], i, j) = AT(Din[0], i, j) +
                            dt * (AT(H[2], i, 0) - fpi * AT(J[0], i, j)) / polar_area(p, i + 0.5);
      } else if (j == p->n_th) {
        AT(Dout[0], i, j) = AT(Din[0], i, j) + dt * (-AT(H[2], i, j - 1) - fpi * AT(J[0], i, j)) /
                                                   polar_area(p, i + 0.5);
      } else {
        metric_at(p, 0.5, 0.0, i, j, &m);
        double curl = AT(H[2], i, j) - AT(H[2], i, j - 1);
        AT(Dout[0], i, j) = AT(Din[0], i, j) + dt * (curl - fpi * AT(J[0], i, j)) / m.sqrt_h;
      }
    }
  for (int j = 0; j < p->n_th; ++j)
    for (int i = 0; i <= p->n_r; ++i) {
      metric_at(p, 0.0, 0.5, i, j, &m);
      double curl = -(AT(H[2], i, j) - AT(H[2], i - 1, j));
      AT(Dout[1], i, j) = AT(Din[1], i, j) + dt * (curl - fpi * AT(J[1], i, j)) / m.sqrt_h;
    }
  for (int j = 1; j < p->n_th; ++j)
    for (int i = 0; i <= p->n_r; ++i) {
      metric_at(p, 0.0, 0.0, i, j, &m);
      double curl = (AT(H[1], i, j) - AT(H[1], i - 1, j)) - (AT(H[0], i, j) - AT(H[0], i, j - 1));
      AT(Dout[2], i, j) = AT(Din[2], i, j) + dt * (curl - fpi * AT(J[2], i, j)) / m.sqrt_h;
    }
}

/* Boundary conditions (Sec. 3.3.3). */
/* MATCH absorbing layer; paper I's form is not available. Reading:
 * F <- F - lambda (F - F_init), lambda = coef * min(1, ((r - r_abs)/(r_max - r_abs))^3)
 * for points with r > r_absorb. */
static void bc_match(const ora_params *p, double *Fc[3], const double *Fi[3], const double S[3][2]) {
  const int NX = NX_of(p);
  if (!(p->r_absorb < p->r_max)) return;
  for (int c = 0; c < 3; ++c)
    for (int j = 0; j <= p->n_th; ++j)
      for (int i = -G; i <= p->n_r + G; ++i) {
        double r, f;
        map_r(p, i + S[c][0], &r, &f);
        if (r <= p->r_absorb) continue;
        double x = (r - p->r_absorb) / (p->r_max - p->r_absorb);
        if (x > 1.0) x = 1.0;
        double lam = p->absorb_coef * x * x * x;
        AT(Fc[c], i, j) = AT(Fc[c], i, j) - lam * (AT(Fc[c], i, j) - AT(Fi[c], i, j));
      }
}

/* horizon layer: cells i1 in [-N_GHOSTS, n_f] copy cell n_f + 1 */
static void bc_horizon(const ora_params *p, double *Fc[3]) {
  const int NX = NX_of(p);
  for (int c = 0; c < 3; ++c)
    for (int j = -G; j <= p->n_th + G; ++j)
      for (int i = -G; i <= p->n_f; ++i) AT(Fc[c], i, j) = AT(Fc[c], p->n_f + 1, j);
}

/* axis ghost rows by reflection symmetry (Fig. 1): r components even, theta and phi
 * components odd. A row class is "node" (x2 = j) or "half" (x2 = j + 1/2). */
static void fill_axis_row(const ora_params *p, double *pl, int half, double par) {
  const int NX = NX_of(p);
  const int N = p->n_th;
  for (int i = -G; i <= p->n_r + G; ++i) {
    if (!half) {
      for (int k = 1; k <= G; ++k) {
        AT(pl, i, -k) = par * AT(pl, i, k);
        AT(pl, i, N + k) = par * AT(pl, i, N - k);
      }
    } else {
      for (int k = 0; k < G; ++k) AT(pl, i, -1 - k) = par * AT(pl, i, k);
      for (int k = 0; k <= G; ++k) AT(pl, i, N + k) = par * AT(pl, i, N - 1 - k);
    }
  }
}
static void fill_axis_B(const ora_params *p, double *B[3]) {
  fill_axis_row(p, B[0], 1, 1.0);
  fill_axis_row(p, B[1], 0, -1.0);
  fill_axis_row(p, B[2], 1, -1.0);
}
static void fill_axis_D(const ora_params *p, double *D[3]) {
  fill_axis_row(p, D[0], 0, 1.0);
  fill_axis_row(p, D[1], 1, -1.0);
  fill_axis_row(p, D[2], 0, -1.0);
}

static double *plane(const ora_params *p, double *F, int k) { return F + k * plane_size(p); }

/* Loop step 2 (Sec. 3.4): B^{n-1} = (B^{n-3/2} + B^{n-1/2})/2,
 * D^{n-1/2} = (D^{n-1} + D^n)/2, E^{n-1/2} from {B^{n-1/2}, D^{n-1/2}},
 * auxiliary Faraday B^{n-1} -> B^n. Output in the BN planes. */
void ora_field_predict(const ora_params *p, double *F) {
  const int64_t PS = plane_size(p);
  double *tmp = malloc(sizeof(double) * PS * 9);
  double *Bm1[3], *Dh[3], *E[3], *Bn[3];
  const double *Bc[3], *Dc[3], *Bmc[3], *Ec[3];
  for (int c = 0; c < 3; ++c) {
    Bm1[c] = tmp + c * PS; Dh[c] = tmp + (3 + c) * PS; E[c] = tmp + (6 + c) * PS;
    Bn[c] = plane(p, F, ORA_BN1 + c);
    for (int64_t q = 0; q < PS; ++q) {
      Bm1[c][q] = 0.5 * (plane(p, F, ORA_B01 + c)[q] + plane(p, F, ORA_B1 + c)[q]);
      Dh[c][q] = 0.5 * (plane(p, F, ORA_D01 + c)[q] + plane(p, F, ORA_D1 + c)[q]);
      E[c][q] = 0.0;
    }
    Bc[c] = plane(p, F, ORA_B1 + c); Dc[c] = Dh[c]; Bmc[c] = Bm1[c]; Ec[c] = E[c];
  }
  aux_E(p, Bc, Dc, E);
  for (int c = 0; c < 3; ++c) memcpy(Bn[c], Bm1[c], sizeof(double) * PS);
  faraday(p, Bmc, Ec, Bn);
  bc_horizon(p, Bn);
  fill_axis_B(p, Bn);
  free(tmp);
}

/* ------------------------------------------------------------------------ */
/* Current filter (Sec. 3.2: the deposit is followed by n_f filter passes;    */
/* Sec. 3.3.3: the horizon layer i1 <= n_f keeps their effect off the         */
/* domain). The filter itself is paper I's and not given here. Reading: one   */
/* pass replaces each value by the binomial stencil (1 2 1)/4 x (1 2 1)/4 of   */
/* its eight neighbours and itself, on the grid extended across each axis by   */
/* the mirror image of the particles (positive weights): node-row quantities   */
/* (J^1, J^3, rho) are even and half-row ones (J^2) odd across an axis, and    */
/* the axis node, which holds the charge of a half cell, holds twice that in   */
/* the extended grid. Values beyond the stored x1 range read as zero. Each     */
/* pass maps the stored values to new stored values; rows outside the         */
/* component's range stay zero. Convolution commutes with the differences of  */
/* the continuity equation, so filtered currents conserve the filtered charge. */
/* ------------------------------------------------------------------------ */
/* the value of the mirror-extended grid at stored column i and row index j (position j for a
 * node row, j + 1/2 for a half row) */
static double filter_ext(const ora_params *p, const double *f, int i, int j, int half,
                         double parity) {
  const int NX = NX_of(p), N = p->n_th;
  if (i < -G || i > p->n_r + G) return 0.0;
  double sgn = 1.0;
  /* reflect the position x = j (+ 1/2) into [0, N]: x -> -x, x -> 2N - x */
  for (;;) {
    if (!half) {
      if (j < 0) { j = -j; sgn *= parity; continue; }
      if (j > N) { j = 2 * N - j; sgn *= parity; continue; }
      break;
    } else {
      if (j < 0) { j = -j - 1; sgn *= parity; continue; }
      if (j > N - 1) { j = 2 * N - j - 1; sgn *= parity; continue; }
      break;
    }
  }
  double v = sgn * AT(f, i, j);
  if (!half && (j == 0 || j == N)) v *= 2.0;
  return v;
}

/* n passes of the filter on one plane; half = 1 for a half-row component. One pass is the
 * plain 3 x 3 binomial stencil (1 2 1) x (1 2 1) / 16 on the mirror-extended grid. */
void ora_filter_plane(const ora_params *p, double *f, int half, double parity, int n) {
  const int NX = NX_of(p), N = p->n_th;
  const int64_t PS = plane_size(p);
  double *src = malloc(sizeof(double) * PS);
  const double w[3] = {1.0, 2.0, 1.0};
  const int jmax = half ? N - 1 : N;
  for (int pass = 0; pass < n; ++pass) {
    memcpy(src, f, sizeof(double) * PS);
    memset(f, 0, sizeof(double) * PS);
    for (int j = 0; j <= jmax; ++j)
      for (int i = -G; i <= p->n_r + G; ++i) {
        double acc = 0.0;
        for (int b = -1; b <= 1; ++b)
          for (int a = -1; a <= 1; ++a)
            acc += w[a + 1] * w[b + 1] * filter_ext(p, src, i + a, j + b, half, parity);
        acc /= 16.0;
        if (!half && (j == 0 || j == N)) acc *= 0.5; /* back to the half cell */
        AT(f, i, j) = acc;
      }
  }
  free(src);
}

/* the n_f passes on the currents J^1 (node rows, even), J^2 (half rows, odd), J^3 (node rows,
 * even); the absolute-term sums JA (a rounding scale for the tests) with even parity */
void ora_filter_currents(const ora_params *p, double *F) {
  if (p->n_f <= 0) return;
  const int64_t PS = plane_size(p);
  const int half[3] = {0, 1, 0};
  const double par[3] = {1.0, -1.0, 1.0};
  for (int c = 0; c < 3; ++c) {
    ora_filter_plane(p, F + (ORA_J1 + c) * PS, half[c], par[c], p->n_f);
    ora_filter_plane(p, F + (ORA_JA1 + c) * PS, half[c], 1.0, p->n_f);
  }
}

/* Loop steps 5-7 (Sec. 3.4), after the deposit wrote J^{n+1/2} into J. */
void ora_field_advance(const ora_params *p, double *F) {
  const int64_t PS = plane_size(p);
  double *tmp = malloc(sizeof(double) * PS * 18);
  double *Jn[3], *E[3], *H[3], *Bnew[3], *Dh[3], *Dnew[3];
  const double *Bn[3], *D[3], *B[3], *J[3], *Jnc[3], *Ec[3], *Hc[3], *Dhc[3], *Bnewc[3];
  const double *Bi[3], *Di[3];
  for (int c = 0; c < 3; ++c) {
    Jn[c] = tmp + c * PS; E[c] = tmp + (3 + c) * PS; H[c] = tmp + (6 + c) * PS;
    Bnew[c] = tmp + (9 + c) * PS; Dh[c] = tmp + (12 + c) * PS; Dnew[c] = tmp + (15 + c) * PS;
    memset(E[c], 0, sizeof(double) * PS);
    memset(H[c], 0, sizeof(double) * PS);
    Bn[c] = plane(p, F, ORA_BN1 + c); D[c] = plane(p, F, ORA_D1 + c);
    B[c] = plane(p, F, ORA_B1 + c); J[c] = plane(p, F, ORA_J1 + c);
    Bi[c] = plane(p, F, ORA_BI1 + c); Di[c] = plane(p, F, ORA_DI1 + c);
    /* step 5: J^n = (J^{n-1/2} + J^{n+1/2}) / 2 */
    for (int64_t q = 0; q < PS; ++q) {
      Jn[c][q] = 0.5 * (plane(p, F, ORA_J01 + c)[q] + J[c][q]);
      Dh[c][q] = 0.5 * (plane(p, F, ORA_D01 + c)[q] + D[c][q]);
    }
    Jnc[c] = Jn[c]; Ec[c] = E[c]; Hc[c] = H[c]; Dhc[c] = Dh[c]; Bnewc[c] = Bnew[c];
  }
  /* step 6: E^n, H^n from {B^n, D^n}; main Faraday B^{n-1/2} -> B^{n+1/2} */
  aux_E(p, Bn, D, E);
  aux_H(p, Bn, D, H);
  for (int c = 0; c < 3; ++c) memcpy(Bnew[c], B[c], sizeof(double) * PS);
  faraday(p, B, Ec, Bnew);
  bc_match(p, Bnew, Bi, SB);
  bc_horizon(p, Bnew);
  fill_axis_B(p, Bnew);
  /* step 7a: auxiliary Ampere D^{n-1/2} -> D^{n+1/2} with H^n, J^n (into Dh, in place) */
  {
    double *Dtmp[3];
    const double *Dtc[3];
    double *tmp2 = malloc(sizeof(double) * PS * 3);
    for (int c = 0; c < 3; ++c) {
      Dtmp[c] = tmp2 + c * PS;
      memcpy(Dtmp[c], Dh[c], sizeof(double) * PS);
      Dtc[c] = Dtmp[c];
    }
    ampere(p, Dtc, Hc, Jnc, Dh);
    free(tmp2);
  }
  bc_horizon(p, Dh);
  /* step 7b: H^{n+1/2} from {B^{n+1/2}, D^{n+1/2}} */
  for (int c = 0; c < 3; ++c) memset(H[c], 0, sizeof(double) * PS);
  aux_H(p, Bnewc, Dhc, H);
  /* step 7c: final Ampere D^n -> D^{n+1} with H^{n+1/2}, J^{n+1/2} */
  for (int c = 0; c < 3; ++c) memcpy(Dnew[c], D[c], sizeof(double) * PS);
  ampere(p, D, Hc, J, Dnew);
  bc_match(p, Dnew, Di, SD);
  bc_horizon(p, Dnew);
  fill_axis_D(p, Dnew);
  /* step 8: em0 <- (B^{n-1/2}, D^n), em <- (B^{n+1/2}, D^{n+1}), cur0 <- J^{n+1/2} */
  for (int c = 0; c < 3; ++c) {
    memcpy(plane(p, F, ORA_B01 + c), B[c], sizeof(double) * PS);
    memcpy(plane(p, F, ORA_D01 + c), D[c], sizeof(double) * PS);
    memcpy(plane(p, F, ORA_B1 + c), Bnew[c], sizeof(double) * PS);
    memcpy(plane(p, F, ORA_D1 + c), Dnew[c], sizeof(double) * PS);
    memcpy(plane(p, F, ORA_J01 + c), J[c], sizeof(double) * PS);
  }
  free(tmp);
}

/* ------------------------------------------------------------------------ */
/* Initial fields (Sec. 4.2; Eq. Wald). Reading: B^1, B^2 from the discrete    */
/* curl of A_3 at the nodes and B^3 from the discrete curl of A_1 at          */
/* (i+1/2, j) (so div B vanishes discretely); D at each of its Yee points from */
/* the pointwise inverse of Eq. (aux) with E_i = d_i A_0 and the analytic B.   */
/* kind: 0 zero, 1 Wald, 2 vertical, 4 monopole (Sec. 4.5). em0 = em, cur0 = 0. */
/* ------------------------------------------------------------------------ */
void ora_init_fields(const ora_params *p, double *F, int kind, double B0) {
  const int NX = NX_of(p);
  const int64_t PS = plane_size(p);
  memset(F, 0, sizeof(double) * PS * ORA_NPLANES);
  if (kind != 0) {
    double *B[3] = {plane(p, F, ORA_B1), plane(p, F, ORA_B2), plane(p, F, ORA_B3)};
    double *D[3] = {plane(p, F, ORA_D1), plane(p, F, ORA_D2), plane(p, F, ORA_D3)};
    ora_metric m;
    double A[3], Ab[3], Bv[3], Dv[3];
    for (int j = 0; j <= p->n_th; ++j)
      for (int i = -G; i <= p->n_r + G; ++i) {
        /* B^1 at (i, j+1/2) and B^3 at (i+1/2, j+1/2) on half rows */
        if (j < p->n_th) {
          metric_at(p, 0.0, 0.5, i, j, &m);
          AT(B[0], i, j) = dA3_theta(p, kind, B0, i, j) / m.sqrt_h;
          metric_at(p, 0.5, 0.5, i, j, &m);
          AT(B[2], i, j) = -wald_dA1_theta(p, kind, B0, i + 0.5, j) / m.sqrt_h;
          wald_fields_point(p, kind, B0, i, j + 0.5, Bv, Dv);
          AT(D[1], i, j) = Dv[1];
        }
        /* B^2 at (i+1/2, j), zero on the axes */
        if (j > 0 && j < p->n_th) {
          metric_at(p, 0.5, 0.0, i, j, &m);
          wald_potential(p, kind, B0, i, j, A);
          wald_potential(p, kind, B0, i + 1, j, Ab);
          AT(B[1], i, j) = -(Ab[2] - A[2]) / m.sqrt_h;
        }
        wald_fields_point(p, kind, B0, i + 0.5, j, Bv, Dv);
        AT(D[0], i, j) = Dv[0];
        if (j > 0 && j < p->n_th) {
          wald_fields_point(p, kind, B0, i, j, Bv, Dv);
          AT(D[2], i, j) = Dv[2];
        }
      }
    bc_horizon(p, B);
    bc_horizon(p, D);
    fill_axis_B(p, B);
    fill_axis_D(p, D);
  }
  for (int c = 0; c < 6; ++c) {
    memcpy(plane(p, F, ORA_B01 + c), plane(p, F, ORA_B1 + c), sizeof(double) * PS);
    memcpy(plane(p, F, ORA_BI1 + c), plane(p, F, ORA_B1 + c), sizeof(double) * PS);
  }
  for (int c = 0; c < 3; ++c) memcpy(plane(p, F, ORA_BN1 + c), plane(p, F, ORA_B1 + c), sizeof(double) * PS);
}

/* ------------------------------------------------------------------------ */
/* Particle loading. The caller gives positions and momenta in the local FIDO */
/* tetrad frame; u_i = e_i^j u_j^ (Appendix A). Weight (reading of "uniform"  */
/* loading with a density profile): w = w0 r^{-k} sqrt(h)(x_p), so that       */
/* sum_p w S approximates n sqrt(h) with n ~ r^{-k}.                          */
/* ------------------------------------------------------------------------ */
void ora_load(const ora_params *p, ora_species *s, const double *uh1, const double *uh2,
              const double *uh3, const double *w0, double density_power) {
#pragma omp parallel for schedule(static)
  for (int64_t k = 0; k < s->n; ++k) {
    double x1 = s->i1[k] + s->dx1[k], x2 = s->i2[k] + s->dx2[k];
    ora_metric m;
    metric_eval(p, x1, x2, 1, 0, &m);
    double uh[3] = {uh1[k], uh2[k], uh3[k]}, u[3];
    hat_to_cov(&m, uh, u);
    s->u1[k] = u[0]; s->u2[k] = u[1]; s->u3[k] = u[2];
    ora_metric m0;
    metric_eval(p, x1, x2, 0, 0, &m0);
    s->w[k] = w0[k] * pow(m0.r, -density_power) * m0.sqrt_h;
    s->phi[k] = 0.0;
    s->tag[k] = 1;
    s->i1p[k] = s->i1[k]; s->i2p[k] = s->i2[k]; s->dx1p[k] = s->dx1[k]; s->dx2p[k] = s->dx2[k];
  }
}

/* ------------------------------------------------------------------------ */
/* Pair injection of the BZ monopole test (Sec. 4.5): plasma is injected where */
/* the local magnetization sigma = B_i B^i / (4 pi n m) exceeds sigma_th. The  */
/* paper gives no more. Reading: per cell (i1 in [0, n_r), i2 in [0, n_th)),   */
/* B at the cell centre from the em planes (B^1 and B^2 averaged over the two  */
/* faces, B^3 as stored), B_i B^i = h_ij B^i B^j with h at the centre; n the   */
/* summed |w| of the live particles of both species in the cell divided by     */
/* sqrt(h) at the centre; sigma = sigma0 (B_i B^i / B0^2) / n in units of the  */
/* fiducial density. Where sigma > sigma_th, one e- e+ pair is added at one    */
/* point of the cell with weights w = dn sqrt(h_centre) / 2 each, dn the       */
/* density that brings sigma down to sigma_th. Offsets and tetrad-frame        */
/* momenta come from a pool of random draws (8 per pair: dx1, dx2, e- u^, e+   */
/* u^), used in cell order (i1 fastest) from entry pool_offset on, cyclically. */
/* Co-located opposite charges of equal weight: the charge density does not   */
/* change.                                                                     */
/* ------------------------------------------------------------------------ */
static void cell_state(const ora_params *p, const double *F, const ora_species *se,
                       const ora_species *sp, double *n_cell, double *b2, double *sqrt_hc) {
  const int NX = NX_of(p);
  const int64_t NC = (int64_t)p->n_r * p->n_th;
  const double *B1 = F + ORA_B1 * plane_size(p), *B2 = F + ORA_B2 * plane_size(p);
  const double *B3 = F + ORA_B3 * plane_size(p);
  memset(n_cell, 0, sizeof(double) * NC);
  const ora_species *both[2] = {se, sp};
  for (int q = 0; q < 2; ++q)
    for (int64_t k = 0; k < both[q]->n; ++k) {
      if (both[q]->tag[k] != 1) continue;
      int i = both[q]->i1[k], j = both[q]->i2[k];
      if (i < 0 || i >= p->n_r || j < 0 || j >= p->n_th) continue;
      n_cell[(int64_t)j * p->n_r + i] += fabs(both[q]->w[k]);
    }
  for (int j = 0; j < p->n_th; ++j)
    for (int i = 0; i < p->n_r; ++i) {
      const int64_t c = (int64_t)j * p->n_r + i;
      ora_metric m;
      metric_eval(p, i + 0.5, j + 0.5, 0, 0, &m);
      const double b1 = 0.5 * (AT(B1, i, j) + AT(B1, i + 1, j));
      const double bb2 = 0.5 * (AT(B2, i, j) + AT(B2, i, j + 1));
      const double b3 = AT(B3, i, j);
      b2[c] = m.h11 * b1 * b1 + m.h22 * bb2 * bb2 + m.h33 * b3 * b3 + 2.0 * m.h13 * b1 * b3;
      sqrt_hc[c] = m.sqrt_h;
      n_cell[c] /= m.sqrt_h;
    }
}

/* the cell densities and B_i B^i the injection sees (for the pins) */
void ora_cell_state(const ora_params *p, const double *F, const ora_species *se,
                    const ora_species *sp, double *n_cell, double *b2) {
  const int64_t NC = (int64_t)p->n_r * p->n_th;
  double *sq = malloc(sizeof(double) * NC);
  cell_state(p, F, se, sp, n_cell, b2, sq);
  free(sq);
}

/* injects into se and sp (room for cap particles each); returns the pairs added */
int64_t ora_inject(const ora_params *p, const double *F, ora_species *se, ora_species *sp,
                   double sigma0, double sigma_th, double B0, const double *pool,
                   int64_t pool_n, int64_t pool_offset, int64_t cap) {
  const int64_t NC = (int64_t)p->n_r * p->n_th;
  double *n_cell = malloc(sizeof(double) * NC), *b2 = malloc(sizeof(double) * NC);
  double *sq = malloc(sizeof(double) * NC);
  cell_state(p, F, se, sp, n_cell, b2, sq);
  /* pairs that fit: the first ones in cell order */
  const int64_t room = cap - (se->n > sp->n ? se->n : sp->n);
  int64_t added = 0;
  for (int j = 0; j < p->n_th; ++j)
    for (int i = 0; i < p->n_r; ++i) {
      const int64_t c = (int64_t)j * p->n_r + i;
      /* sigma > sigma_th without dividing by n (n may be 0) */
      if (!(sigma0 * b2[c] > sigma_th * B0 * B0 * n_cell[c])) continue;
      if (added >= room) continue;
      const double dn = sigma0 * b2[c] / (B0 * B0 * sigma_th) - n_cell[c];
      const double *r = pool + 8 * ((pool_offset + added) % pool_n);
      ora_species *both[2] = {se, sp};
      for (int q = 0; q < 2; ++q) {
        ora_species *s = both[q];
        const int64_t k = s->n++;
        s->i1[k] = i; s->i2[k] = j; s->dx1[k] = r[0]; s->dx2[k] = r[1];
        ora_metric m;
        metric_eval(p, i + r[0], j + r[1], 1, 0, &m);
        double uh[3] = {r[2 + 3 * q], r[3 + 3 * q], r[4 + 3 * q]}, u[3];
        hat_to_cov(&m, uh, u);
        s->u1[k] = u[0]; s->u2[k] = u[1]; s->u3[k] = u[2];
        s->w[k] = 0.5 * dn * sq[c];
        s->phi[k] = 0.0;
        s->tag[k] = 1;
        s->i1p[k] = i; s->i2p[k] = j; s->dx1p[k] = r[0]; s->dx2p[k] = r[1];
      }
      ++added;
    }
  free(n_cell); free(b2); free(sq);
  return added;
}

/* ------------------------------------------------------------------------ */
/* Sort (added by this implementation, not in the paper): stable sort of the   */
/* particles by tile-major cell key, particles not alive last and dropped.     */
/* key = tile * (tr*tt) + (i2 % tt) * tr + (i1 % tr), tile = (i2/tt) * ntr +   */
/* i1/tr, ntr = ceil(n_r / tr). Returns the new particle count.                */
/* ------------------------------------------------------------------------ */
typedef struct { uint64_t key; int64_t idx; } ora_kv;
static int kv_cmp(const void *a, const void *b) {
  const ora_kv *x = a, *y = b;
  if (x->key != y->key) return x->key < y->key ? -1 : 1;
  return x->idx < y->idx ? -1 : (x->idx > y->idx ? 1 : 0);
}
uint32_t ora_sort_key(const ora_params *p, int tr, int tt, int32_t i1, int32_t i2, uint8_t tag) {
  if (tag != 1) return 0xFFFFFFFFu;
  uint32_t ntr = (uint32_t)((p->n_r + tr - 1) / tr);
  uint32_t tile = (uint32_t)(i2 / tt) * ntr + (uint32_t)(i1 / tr);
  return tile * (uint32_t)(tr * tt) + (uint32_t)(i2 % tt) * (uint32_t)tr + (uint32_t)(i1 % tr);
}

#define PERMUTE(T, arr)                                              \
  do {                                                               \
    T *t_ = malloc(sizeof(T) * (n > 0 ? n : 1));                     \
    for (int64_t k = 0; k < n; ++k) t_[k] = (arr)[kv[k].idx];        \
    memcpy((arr), t_, sizeof(T) * n);                                \
    free(t_);                                                        \
  } while (0)

int64_t ora_sort(const ora_params *p, ora_species *s, int tr, int tt, int64_t *perm_out) {
  int64_t n = s->n;
  ora_kv *kv = malloc(sizeof(ora_kv) * (n > 0 ? n : 1));
  for (int64_t k = 0; k < n; ++k) {
    kv[k].key = ora_sort_key(p, tr, tt, s->i1[k], s->i2[k], s->tag[k]);
    kv[k].idx = k;
  }
  qsort(kv, n, sizeof(ora_kv), kv_cmp); /* (key, index) is unique: the order is stable */
  int64_t alive = 0;
  for (int64_t k = 0; k < n; ++k) alive += kv[k].key != 0xFFFFFFFFu;
  if (perm_out)
    for (int64_t k = 0; k < n; ++k) perm_out[k] = kv[k].idx;
  PERMUTE(int32_t, s->i1); PERMUTE(int32_t, s->i2);
  PERMUTE(double, s->dx1); PERMUTE(double, s->dx2);
  PERMUTE(double, s->u1); PERMUTE(double, s->u2); PERMUTE(double, s->u3);
  PERMUTE(double, s->phi); PERMUTE(double, s->w); PERMUTE(uint8_t, s->tag);
  PERMUTE(int32_t, s->i1p); PERMUTE(int32_t, s->i2p);
  PERMUTE(double, s->dx1p); PERMUTE(double, s->dx2p);
  free(kv);
  s->n = alive;
  return alive;
}

/* ------------------------------------------------------------------------ */
/* The PIC loop of Sec. 3.4: predict, (sort), push, deposit, advance.          */
/* ------------------------------------------------------------------------ */
void ora_step(const ora_params *p, double *F, ora_species *sp, int ns, int n_steps,
              int sort_every, int tr, int tt, int64_t step0, int64_t *counters) {
  for (int n = 0; n < n_steps; ++n) {
    ora_field_predict(p, F);
    if (sort_every > 0 && (step0 + n) % sort_every == 0)
      for (int si = 0; si < ns; ++si) ora_sort(p, &sp[si], tr, tt, NULL);
    for (int si = 0; si < ns; ++si) ora_push(p, F, &sp[si], 0, 0, 0.0, counters);
    ora_deposit(p, F, sp, ns);
    ora_filter_currents(p, F);
    ora_field_advance(p, F);
  }
}

/* ------------------------------------------------------------------------ */
/* Helpers exposed to the pins.                                                */
/* ------------------------------------------------------------------------ */
void ora_metric_point(const ora_params *p, double x1, double x2, int clamp, ora_metric *m) {
  metric_eval(p, x1, x2, clamp, 1, m);
}
double ora_polar_area(const ora_params *p, double x1) { return polar_area(p, x1); }
void ora_potential(const ora_params *p, int kind, double B0, double x1, double x2, double A[3]) {
  wald_potential(p, kind, B0, x1, x2, A);
}
void ora_fields_point(const ora_params *p, int kind, double B0, double x1, double x2,
                      double B[3], double D[3]) {
  wald_fields_point(p, kind, B0, x1, x2, B, D);
}
/* dir: 0 contravariant -> hat, 1 hat -> contravariant, 2 covariant -> hat, 3 hat -> covariant */
void ora_tetrad(const ora_params *p, double x1, double x2, int dir, const double in[3],
                double out[3]) {
  ora_metric m;
  metric_eval(p, x1, x2, 1, 0, &m);
  if (dir == 0) vec_to_hat(&m, in, out);
  else if (dir == 1) hat_to_vec(&m, in, out);
  else if (dir == 2) cov_to_hat(&m, in, out);
  else hat_to_cov(&m, in, out);
}
void ora_boris(double u[3], const double Dh[3], const double Bh[3], double hq) { boris(u, Dh, Bh, hq); }
/* u_0 = -alpha gamma + beta^1 u_1 (footnote of Sec. 2.3, reading u^i = h^ij u_j - u^0 beta^i) */
double ora_u_lower0(const ora_params *p, double x1, double x2, const double u[3], int massless) {
  ora_metric m;
  metric_eval(p, x1, x2, 1, 0, &m);
  return -m.alpha * gamma_of(&m, u, massless ? 0.0 : 1.0) + m.beta1 * u[0];
}
/* conserved energy and angular momentum per unit mass (Sec. 2.3) with A of kind/B0 */
void ora_invariants(const ora_params *p, int kind, double B0, double qm, double x1, double x2,
                    const double u[3], double out[2]) {
  double A[3] = {0.0, 0.0, 0.0};
  if (kind != 0) wald_potential(p, kind, B0, x1, x2, A);
  out[0] = -ora_u_lower0(p, x1, x2, u, 0) - qm * A[0];
  out[1] = u[2] + qm * A[2];
}
double ora_time_step(const ora_params *p, double cfl) {
  /* reading of the CFL rule: dt = cfl * min over cell centres of
   * 1 / (alpha sqrt(h^11 + h^22) + |beta^1|) */
  double best = 1e300;
  for (int j = 0; j < p->n_th; ++j)
    for (int i = 0; i < p->n_r; ++i) {
      ora_metric m;
      metric_eval(p, i + 0.5, j + 0.5, 0, 0, &m);
      double v = 1.0 / (m.alpha * sqrt(m.H11 + m.H22) + fabs(m.beta1));
      if (v < best) best = v;
    }
  return cfl * best;
}
/* Frozen-field push of n test particles for n_steps steps (steps 2-11 of Sec. 3.1, no
 * deposit) with the em-plane fields of F times `scale` and both implicit pushes iterated
 * p->n_iter times. state: [6][n] doubles x1, x2, phi, u1, u2, u3 (absolute code
 * coordinates), advanced in place. A particle whose step would leave the domain interior
 * (horizon layer, outer edge, an axis) is set to NaN and stays NaN. */
void ora_push_frozen(const ora_params *p, const double *F, double scale, double qm,
                     int n_steps, int64_t n, double *state) {
#pragma omp parallel for schedule(dynamic, 16)
  for (int64_t k = 0; k < n; ++k) {
    double x[2] = {state[k], state[n + k]}, phi = state[2 * n + k];
    double u[3] = {state[3 * n + k], state[4 * n + k], state[5 * n + k]};
    int bad = !(x[0] == x[0]);
    for (int st = 0; st < n_steps && !bad; ++st) bad = frozen_step(p, F, scale, qm, x, u, &phi);
    const double v[6] = {x[0], x[1], phi, u[0], u[1], u[2]};
    for (int q = 0; q < 6; ++q) state[q * n + k] = bad ? NAN : v[q];
  }
}

/* The same in complex arithmetic: the state is re + i im and the scale scale_re + i scale_im.
 * With the perturbation i e (e ~ 1e-30) on one input, Im(output) / e is the derivative of
 * the double map with respect to that input, exact to rounding (complex step). */
void ora_push_frozen_cs(const ora_params *p, const double *F, double scale_re, double scale_im,
                        double qm, int n_steps, int64_t n, double *re, double *im) {
  const double complex scale = scale_re + scale_im * I;
#pragma omp parallel for schedule(dynamic, 16)
  for (int64_t k = 0; k < n; ++k) {
    double complex x[2], u[3], phi;
    for (int q = 0; q < 2; ++q) x[q] = re[q * n + k] + im[q * n + k] * I;
    phi = re[2 * n + k] + im[2 * n + k] * I;
    for (int q = 0; q < 3; ++q) u[q] = re[(3 + q) * n + k] + im[(3 + q) * n + k] * I;
    int bad = !(creal(x[0]) == creal(x[0]));
    for (int st = 0; st < n_steps && !bad; ++st)
      bad = frozen_step_cs(p, F, scale, qm, x, u, &phi);
    const double complex v[6] = {x[0], x[1], phi, u[0], u[1], u[2]};
    for (int q = 0; q < 6; ++q) {
      re[q * n + k] = bad ? NAN : creal(v[q]);
      im[q * n + k] = bad ? NAN : cimag(v[q]);
    }
  }
}

/* The auxiliary fields E, H of the em planes (B, D) as they stand, Eqs. (discretized-auxE)
 * and (discretized-auxH): E and H each 3 planes (E_1, E_2, E_3), zero where not computed. */
void ora_aux_fields(const ora_params *p, const double *F, double *E, double *H) {
  const int64_t PS = plane_size(p);
  const double *B[3], *D[3];
  double *e[3], *h[3];
  for (int c = 0; c < 3; ++c) {
    B[c] = F + (ORA_B1 + c) * PS;
    D[c] = F + (ORA_D1 + c) * PS;
    e[c] = E + c * PS;
    h[c] = H + c * PS;
    memset(e[c], 0, sizeof(double) * PS);
    memset(h[c], 0, sizeof(double) * PS);
  }
  aux_E(p, B, D, e);
  aux_H(p, B, D, h);
}

int ora_version(void) { return 6; }

/* Threads of the OpenMP loops (the particle push and the charge sums); timing only. */
void ora_set_threads(int n) {
#ifdef _OPENMP
  if (n > 0) omp_set_num_threads(n);
#else
  (void)n;
#endif
}
int ora_max_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}
