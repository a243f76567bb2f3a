// fields.cu -- metric tables, initial fields and the GR field solver of Sec. 3.3 of
// arXiv:2511.17701 (Faraday, Ampere, auxiliary E and H with volume-weighted averages,
// axis treatment, horizon layer and absorbing layer), plus the loop steps 2 and 5-8 of
// Sec. 3.4. Grid work is a small fraction of a step at the particle counts this library
// targets (tens of particles per cell): one thread per grid point, metric from tables.
#include "grpic_internal.cuh"

namespace {

constexpr int TPB = 256;

template <typename T>
__device__ __forceinline__ T tabv(const T *tab, const GridP &g, int cls, int q, int i, int j) {
  return __ldg(tab + ((int64_t)(cls * T_NQ + q)) * plane_size(g) + sidx(g, i, j));
}

// ---------------------------------------------------------------------------------
// Tables: per Yee class, alpha, h_11, h_22, h_33, 1/(2 sqrt(h~)) (the weight of the
// volume-weighted averages, stored as a reciprocal so the field kernels multiply instead of
// dividing), [sqrt(h~) h_13], [sqrt(h~ h) beta^1], 1/sqrt(h) at every stored point; the
// polar area A(x1) = dr (r^2 + a^2) sqrt(1 + 2 M r/(r^2 + a^2)) (1 - cos(theta(x2 = 1/2)))
// (App. A, per unit phi; theta(1/2) = dtheta/2 on the plain grid).
// ---------------------------------------------------------------------------------
// The absorbing layer (MATCH, Sec. 3.3.3): a field value v relaxes towards its initial value
// vi as v - k (v - vi), k = absorb_coef x^3, x = (r - r_absorb) / (r_max - r_absorb) capped at
// 1, beyond r_absorb. k depends on x1 alone, so it is tabulated per column.
__device__ __forceinline__ double absorb_factor(const GridP &g, double x1) {
  if (!(g.r_absorb < g.r_max)) return 0.0;
  const double r = g.r0 + map_e(g, x1);
  if (r <= g.r_absorb) return 0.0;
  double x = (r - g.r_absorb) / (g.r_max - g.r_absorb);
  x = fmin(x, 1.0);
  return g.absorb_coef * x * x * x;
}

template <typename T>
__global__ void k_metric_tables(GridP g, T *tab, T *polar) {
  const int64_t ps = plane_size(g);
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < 4 * ps;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int cls = (int)(t / ps);
    const int64_t q = t - cls * ps;
    const int i = (int)(q % g.NX) - G_, j = (int)(q / g.NX) - G_;
    const double s1 = (cls == CLS_HN || cls == CLS_HH) ? 0.5 : 0.0;
    const double s2 = (cls == CLS_NH || cls == CLS_HH) ? 0.5 : 0.0;
    MetricV m;
    metric_eval<false>(g, i + s1, j + s2, false, m, nullptr);
    T *o = tab + (int64_t)cls * T_NQ * ps + q;
    o[T_ALPHA * ps] = (T)m.alpha;
    o[T_H11 * ps] = (T)m.h11;
    o[T_H22 * ps] = (T)m.h22;
    o[T_H33 * ps] = (T)m.h33;
    o[T_IHT2 * ps] = (T)(0.5 / m.sqrt_ht);
    o[T_WT13 * ps] = (T)(m.sqrt_ht * m.h13);
    o[T_WB1 * ps] = (T)(m.sqrt_ht * m.sqrt_h * m.beta1);
    o[T_ISH * ps] = (T)(1.0 / m.sqrt_h);
    if (cls == CLS_HN && j == 0) {
      const double e = map_e(g, i + 0.5), r = g.r0 + e, a2 = g.a * g.a;
      polar[i + G_] = (T)(g.dxi * e * (r * r + a2) * sqrt(1.0 + 2.0 * g.M * r / (r * r + a2)) *
                          (1.0 - cos(map_theta(g, 0.5))));
      polar[2 * g.NX + i + G_] = (T)absorb_factor(g, i + 0.5);
    }
    if (cls == CLS_NN && j == 0) polar[g.NX + i + G_] = (T)absorb_factor(g, i);
  }
}

// dt = cfl * min over cell centres of 1 / (alpha sqrt(h^11 + h^22) + |beta^1|); positive
// doubles order like their bit patterns, so the minimum is an integer atomicMin.
__global__ void k_dt_min(GridP g, unsigned long long *out) {
  __shared__ unsigned long long sm[TPB];
  unsigned long long best = 0x7FF0000000000000ull;  // +inf
  const int64_t n = (int64_t)g.n_r * g.n_th;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(t % g.n_r), j = (int)(t / g.n_r);
    MetricV m;
    metric_eval<false>(g, i + 0.5, j + 0.5, false, m, nullptr);
    const double v = 1.0 / (m.alpha * sqrt(m.H11 + m.H22) + fabs(m.beta1));
    const unsigned long long b = (unsigned long long)__double_as_longlong(v);
    best = b < best ? b : best;
  }
  sm[threadIdx.x] = best;
  __syncthreads();
  for (int s = TPB / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s && sm[threadIdx.x + s] < sm[threadIdx.x]) sm[threadIdx.x] = sm[threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x == 0) atomicMin(out, sm[0]);
}

// D at a Yee point from the inverse of Eq. (aux) with E_i = d_i A_0, E_3 = 0 and
// sqrt(h) B^2 = -d_1 A_3, sqrt(h) B^3 = -d_2 A_1 (no division by sqrt(h) on the axis).
__device__ void d_from_potential(const GridP &g, int kind, double B0, double x1, double x2,
                                 int comp, double &out) {
  Pot p;
  potential(g, kind, B0, x1, x2, true, p);
  MetricV m;
  metric_eval<false>(g, x1, x2, false, m, nullptr);
  if (comp == 0) out = (m.H11 * p.d1A0 + m.H13 * m.beta1 * p.d1A3) / m.alpha;
  else if (comp == 1) out = m.H22 * (p.d2A0 - m.beta1 * p.d2A1) / m.alpha;
  else out = (m.H13 * p.d1A0 + m.H33 * m.beta1 * p.d1A3) / m.alpha;
}

__device__ double inv_sqrt_h(const GridP &g, double x1, double x2) {
  MetricV m;
  metric_eval<false>(g, x1, x2, false, m, nullptr);
  return 1.0 / m.sqrt_h;
}

// theta_j + theta_{j+1} and theta_{j+1} - theta_j of two face rows; with h0 the cubic's
// difference p(eta + d) - p(eta) = d (pi^2 - 6 pi eta + 6 eta^2) + d^2 (6 eta - 3 pi) + 2 d^3
// (p(eta) = eta (pi - 2 eta)(pi - eta)) is expanded so that nothing cancels
__device__ double theta_sum(const GridP &g, int j) {
  const double de = g.dth, e0 = j * de, e1 = (j + 1) * de, k = 2.0 * g.h0 / (GRPIC_PI * GRPIC_PI);
  const double p0 = e0 * (GRPIC_PI - 2.0 * e0) * (GRPIC_PI - e0);
  const double p1 = e1 * (GRPIC_PI - 2.0 * e1) * (GRPIC_PI - e1);
  return (2 * j + 1) * de + k * (p0 + p1);
}
__device__ double theta_diff(const GridP &g, int j) {
  const double de = g.dth, e0 = j * de, k = 2.0 * g.h0 / (GRPIC_PI * GRPIC_PI);
  return de + k * (de * (GRPIC_PI * GRPIC_PI - 6.0 * GRPIC_PI * e0 + 6.0 * e0 * e0) +
                   de * de * (6.0 * e0 - 3.0 * GRPIC_PI) + 2.0 * de * de * de);
}

// A_1(x1, theta_{j+1}) - A_1(x1, theta_j) of the Wald potential (Eq. Wald) for the discrete
// curl that gives B^3, in product form: with A_1 = (B0/2) a f (2 M r (1 + cos^2)/Sigma -
// sin^2) and sin^2(b) - sin^2(a) = sin(b - a) sin(b + a) = -(cos^2(b) - cos^2(a)),
//   dA_1 = -(B0/2) a f D (1 + 2 M r (r^2 - a^2) / (Sigma_a Sigma_b)),
//   D = sin(theta_{j+1} - theta_j) sin(theta_{j+1} + theta_j);
// the plain difference loses ~1/dth^2 of its digits next to the axes (A_1 ~ theta^2 there).
// A_3(x1, theta_{j+1}) - A_3(x1, theta_j) for the discrete curl that gives B^1; for the
// monopole, -B0 (cos(theta_{j+1}) - cos(theta_j)) = 2 B0 sin((theta_j + theta_{j+1}) / 2)
// sin((theta_{j+1} - theta_j) / 2) in product form (the plain difference of the cosines
// loses ~1/dth^2 of its digits next to the axes)
__device__ double dA3_theta(const GridP &g, int kind, double B0, int i, int j) {
  if (kind == GRPIC_FIELD_MONOPOLE)
    return 2.0 * B0 * sin(0.5 * theta_sum(g, j)) * sin(0.5 * theta_diff(g, j));
  Pot pa, pb;
  potential(g, kind, B0, i, j, false, pa);
  potential(g, kind, B0, i, j + 1, false, pb);
  return pb.A3 - pa.A3;
}

__device__ double dA1_theta(const GridP &g, int kind, double B0, double x1, int j) {
  if (kind != GRPIC_FIELD_WALD) return 0.0;  // the vertical field has A_1 = 0
  const double a = g.a, M = g.M;
  const double e = map_e(g, x1), r = g.r0 + e, f = g.dxi * e;
  const double ca = cos(map_theta(g, j)), cb = cos(map_theta(g, j + 1));
  const double Sa = r * r + a * a * ca * ca, Sb = r * r + a * a * cb * cb;
  const double D = sin(theta_diff(g, j)) * sin(theta_sum(g, j));
  return -0.5 * B0 * a * f * D * (1.0 + 2.0 * M * r * (r * r - a * a) / (Sa * Sb));
}

template <typename T>
__global__ void k_init_fields(GridP g, FieldPtrsT<T> F, int kind, double B0) {
  const int ni = g.n_r + 2 * G_ + 1, nj = g.n_th + 1;
  const int64_t n = (int64_t)ni * nj;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(t % ni) - G_, j = (int)(t / ni);
    const int64_t k = sidx(g, i, j);
    const bool axis = (j == 0 || j == g.n_th);
    Pot pa, pb;
    if (j < g.n_th) {
      F.B[0][k] = (T)(dA3_theta(g, kind, B0, i, j) * inv_sqrt_h(g, i, j + 0.5));
      F.B[2][k] = (T)(-dA1_theta(g, kind, B0, i + 0.5, j) * inv_sqrt_h(g, i + 0.5, j + 0.5));
      double d;
      d_from_potential(g, kind, B0, i, j + 0.5, 1, d);
      F.D[1][k] = (T)d;
    }
    if (!axis) {
      potential(g, kind, B0, i, j, false, pa);
      potential(g, kind, B0, i + 1, j, false, pb);
      F.B[1][k] = (T)(-(pb.A3 - pa.A3) * inv_sqrt_h(g, i + 0.5, j));
      double d;
      d_from_potential(g, kind, B0, i, j, 2, d);
      F.D[2][k] = (T)d;
    } else {
      F.B[1][k] = (T)0;
      F.D[2][k] = (T)0;
    }
    double d0;
    d_from_potential(g, kind, B0, i + 0.5, j, 0, d0);
    F.D[0][k] = (T)d0;
  }
}

// ---------------------------------------------------------------------------------
// Boundary conditions (Sec. 3.3.3).
// ---------------------------------------------------------------------------------
// Horizon layer: cells i1 in [-G, n_f] copy cell n_f + 1, all rows.
template <typename T>
__global__ void k_horizon(GridP g, T *p0, T *p1, T *p2) {
  const int nl = g.n_f + 1 + G_, nj = g.NY;
  const int64_t n = (int64_t)nl * nj * 3;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int c = (int)(t / ((int64_t)nl * nj));
    const int64_t q = t - c * (int64_t)nl * nj;
    const int i = (int)(q % nl) - G_, j = (int)(q / nl) - G_;
    T *p = c == 0 ? p0 : (c == 1 ? p1 : p2);
    p[sidx(g, i, j)] = p[sidx(g, g.n_f + 1, j)];
  }
}

// Axis ghost rows by reflection (Fig. 1): r components even, theta and phi components
// odd; half rows (x2 = j + 1/2) and node rows mirror differently. isB selects the B
// classes (B^1 half, B^2 node, B^3 half) or the D classes (D^1 node, D^2 half, D^3 node).
template <typename T>
__global__ void k_axis(GridP g, T *p0, T *p1, T *p2, int isB) {
  const int ni = g.NX;
  const int nrow = 2 * G_ + 1;  // rows written per component (2 below, 3 above)
  const int64_t n = (int64_t)ni * nrow * 3;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int c = (int)(t / ((int64_t)ni * nrow));
    const int64_t q = t - c * (int64_t)ni * nrow;
    const int i = (int)(q % ni) - G_, rr = (int)(q / ni);
    T *p = c == 0 ? p0 : (c == 1 ? p1 : p2);
    const bool half = isB ? (c != 1) : (c == 1);
    const T par = (c == 0) ? (T)1 : (T)-1;
    const int N = g.n_th;
    if (!half) {
      if (rr < G_) {  // rows -1, -2 from 1, 2
        const int k = rr + 1;
        p[sidx(g, i, -k)] = par * p[sidx(g, i, k)];
      } else if (rr < 2 * G_) {  // rows N+1, N+2 from N-1, N-2
        const int k = rr - G_ + 1;
        p[sidx(g, i, N + k)] = par * p[sidx(g, i, N - k)];
      }
    } else {
      if (rr < G_) {  // rows -1, -2 from 0, 1
        p[sidx(g, i, -1 - rr)] = par * p[sidx(g, i, rr)];
      } else {  // rows N, N+1, N+2 from N-1, N-2, N-3
        const int k = rr - G_;
        p[sidx(g, i, N + k)] = par * p[sidx(g, i, N - 1 - k)];
      }
    }
  }
}

// ---------------------------------------------------------------------------------
// Auxiliary fields, Eq. (discretized-auxE) with the averages of Eq. (discretized-auxH).
// D (and for E also B) may be the mean of two time levels: X = wa Xa + wb Xb.
// Computed on stored i in [-1, n_r + 1], rows [0, n_theta].
// ---------------------------------------------------------------------------------
template <typename T>
struct Pair3 {
  const T *a[3], *b[3];
  T wa, wb;
};
template <typename T>
__device__ __forceinline__ T pv(const Pair3<T> &P, int c, int64_t k) {
  T v = P.wa * __ldg(P.a[c] + k);
  if (P.wb != (T)0) v += P.wb * __ldg(P.b[c] + k);
  return v;
}

template <typename T>
__global__ void k_aux_E(GridP g, Pair3<T> B, Pair3<T> D, const T *tab, T *E1, T *E2, T *E3) {
  const int ni = g.n_r + 3, nj = g.n_th + 1;
  const int64_t n = (int64_t)ni * nj;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(t % ni) - 1, j = (int)(t / ni);
    const int64_t k = sidx(g, i, j);
    // E_1 at (i+1/2, j) = alpha [h_11 D^1 + <h_13 D^3>]
    {
      const T avg = (tabv(tab, g, CLS_NN, T_WT13, i, j) * pv(D, 2, k) +
                     tabv(tab, g, CLS_NN, T_WT13, i + 1, j) * pv(D, 2, k + 1)) *
                    tabv(tab, g, CLS_HN, T_IHT2, i, j);
      E1[k] = tabv(tab, g, CLS_HN, T_ALPHA, i, j) *
              (tabv(tab, g, CLS_HN, T_H11, i, j) * pv(D, 0, k) + avg);
    }
    // E_3 at (i, j) = alpha [h_33 D^3 + <h_13 D^1>] + <sqrt(h) beta^1 B^2>; zero on the axes
    if (j == 0 || j == g.n_th) {
      E3[k] = (T)0;
    } else {
      const T w2 = tabv(tab, g, CLS_NN, T_IHT2, i, j);
      const T a13 = (tabv(tab, g, CLS_HN, T_WT13, i - 1, j) * pv(D, 0, k - 1) +
                     tabv(tab, g, CLS_HN, T_WT13, i, j) * pv(D, 0, k)) * w2;
      const T ab2 = (tabv(tab, g, CLS_HN, T_WB1, i - 1, j) * pv(B, 1, k - 1) +
                     tabv(tab, g, CLS_HN, T_WB1, i, j) * pv(B, 1, k)) * w2;
      E3[k] = tabv(tab, g, CLS_NN, T_ALPHA, i, j) *
                  (tabv(tab, g, CLS_NN, T_H33, i, j) * pv(D, 2, k) + a13) + ab2;
    }
    // E_2 at (i, j+1/2) = alpha h_22 D^2 - <sqrt(h) beta^1 B^3>
    if (j < g.n_th) {
      const T ab3 = (tabv(tab, g, CLS_HH, T_WB1, i - 1, j) * pv(B, 2, k - 1) +
                     tabv(tab, g, CLS_HH, T_WB1, i, j) * pv(B, 2, k)) *
                    tabv(tab, g, CLS_NH, T_IHT2, i, j);
      E2[k] = tabv(tab, g, CLS_NH, T_ALPHA, i, j) * tabv(tab, g, CLS_NH, T_H22, i, j) *
                  pv(D, 1, k) - ab3;
    }
  }
}

template <typename T>
__global__ void k_aux_H(GridP g, Pair3<T> B, Pair3<T> D, const T *tab, T *H1, T *H2, T *H3) {
  const int ni = g.n_r + 3, nj = g.n_th + 1;
  const int64_t n = (int64_t)ni * nj;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(t % ni) - 1, j = (int)(t / ni);
    const int64_t k = sidx(g, i, j);
    if (j < g.n_th) {
      // H_1 at (i, j+1/2) = alpha [h_11 B^1 + <h_13 B^3>]
      const T a13 = (tabv(tab, g, CLS_HH, T_WT13, i - 1, j) * pv(B, 2, k - 1) +
                     tabv(tab, g, CLS_HH, T_WT13, i, j) * pv(B, 2, k)) *
                    tabv(tab, g, CLS_NH, T_IHT2, i, j);
      H1[k] = tabv(tab, g, CLS_NH, T_ALPHA, i, j) *
              (tabv(tab, g, CLS_NH, T_H11, i, j) * pv(B, 0, k) + a13);
      // H_3 at (i+1/2, j+1/2) = alpha [h_33 B^3 + <h_13 B^1>] - <sqrt(h) beta^1 D^2>
      const T w3 = tabv(tab, g, CLS_HH, T_IHT2, i, j);
      const T b13 = (tabv(tab, g, CLS_NH, T_WT13, i, j) * pv(B, 0, k) +
                     tabv(tab, g, CLS_NH, T_WT13, i + 1, j) * pv(B, 0, k + 1)) * w3;
      const T bd2 = (tabv(tab, g, CLS_NH, T_WB1, i, j) * pv(D, 1, k) +
                     tabv(tab, g, CLS_NH, T_WB1, i + 1, j) * pv(D, 1, k + 1)) * w3;
      H3[k] = tabv(tab, g, CLS_HH, T_ALPHA, i, j) *
                  (tabv(tab, g, CLS_HH, T_H33, i, j) * pv(B, 2, k) + b13) - bd2;
    }
    // H_2 at (i+1/2, j) = alpha h_22 B^2 + <sqrt(h) beta^1 D^3>
    const T bd3 = (tabv(tab, g, CLS_NN, T_WB1, i, j) * pv(D, 2, k) +
                   tabv(tab, g, CLS_NN, T_WB1, i + 1, j) * pv(D, 2, k + 1)) *
                  tabv(tab, g, CLS_HN, T_IHT2, i, j);
    H2[k] = tabv(tab, g, CLS_HN, T_ALPHA, i, j) * tabv(tab, g, CLS_HN, T_H22, i, j) *
                pv(B, 1, k) + bd3;
  }
}

// MATCH absorbing layer (reading of paper I's form): F <- F - lambda (F - F_init),
// lambda = coef min(1, ((r - r_abs)/(r_max - r_abs)))^3 for r > r_absorb, rows [0, n_theta].
// The initial value is read only inside the layer (the factor is zero elsewhere).
template <typename T>
__device__ __forceinline__ T match(const GridP &g, T v, const T *init, int64_t idx,
                                   const T *absorb, int i, int j) {
  if (j < 0 || j > g.n_th) return v;
  const T k = __ldg(absorb + i + G_);  // the factor at this column (absorb_factor)
  return k == (T)0 ? v : v - k * (v - __ldg(init + idx));
}

// Faraday, Eq. (discretized-faraday): Bout = Bin - dt curl E / sqrt(h) on the evolved
// points, Bout = Bin elsewhere; B^2 is not evolved on the axes. Covers every stored point.
template <typename T>
__global__ void k_faraday(GridP g, Pair3<T> Bin, const T *E1, const T *E2, const T *E3,
                          const T *tab, const T *absorb, T *B1, T *B2, T *B3, const T *Bi1,
                          const T *Bi2, const T *Bi3, int do_match) {
  const int64_t n = plane_size(g);
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(t % g.NX) - G_, j = (int)(t / g.NX) - G_;
    const int64_t k = t;
    const T dt = (T)g.dt;
    T b1 = pv(Bin, 0, k), b2 = pv(Bin, 1, k), b3 = pv(Bin, 2, k);
    const bool rows_half = (j >= 0 && j < g.n_th);
    if (rows_half && i >= 0 && i <= g.n_r)
      b1 -= dt * (__ldg(E3 + k + g.NX) - __ldg(E3 + k)) * tabv(tab, g, CLS_NH, T_ISH, i, j);
    if (j >= 1 && j < g.n_th && i >= 0 && i < g.n_r)
      b2 += dt * (__ldg(E3 + k + 1) - __ldg(E3 + k)) * tabv(tab, g, CLS_HN, T_ISH, i, j);
    if (rows_half && i >= 0 && i < g.n_r)
      b3 -= dt * ((__ldg(E2 + k + 1) - __ldg(E2 + k)) - (__ldg(E1 + k + g.NX) - __ldg(E1 + k))) *
            tabv(tab, g, CLS_HH, T_ISH, i, j);
    if (do_match) {
      b1 = match(g, b1, Bi1, k, absorb, i, j);
      b2 = match(g, b2, Bi2, k, absorb + g.NX, i, j);
      b3 = match(g, b3, Bi3, k, absorb + g.NX, i, j);
    }
    B1[k] = b1; B2[k] = b2; B3[k] = b3;
  }
}

// Ampere, Eq. (discretized-ampere): Dout = Din + dt (curl H - 4 pi J) / sqrt(h); on the
// axes D^1 follows the integral form of Sec. 3.3.2 with the polar area (reading: the
// whole radial flux into the half cell, coefficient 4 pi; -H_3 at theta = pi) and D^3
// is not evolved. J may be the mean of two time levels.
template <typename T>
__global__ void k_ampere(GridP g, Pair3<T> Din, const T *H1, const T *H2, const T *H3, Pair3<T> J,
                         const T *tab, const T *polar, T *D1, T *D2, T *D3, const T *Di1,
                         const T *Di2, const T *Di3, int do_match) {
  const int64_t n = plane_size(g);
  const T fpi = (T)(4.0 * GRPIC_PI), dt = (T)g.dt;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(t % g.NX) - G_, j = (int)(t / g.NX) - G_;
    const int64_t k = t;
    T d1 = pv(Din, 0, k), d2 = pv(Din, 1, k), d3 = pv(Din, 2, k);
    if (i >= 0 && i < g.n_r && j >= 0 && j <= g.n_th) {
      if (j == 0)
        d1 += dt * (__ldg(H3 + k) - fpi * pv(J, 0, k)) / __ldg(polar + i + G_);
      else if (j == g.n_th)
        d1 += dt * (-__ldg(H3 + k - g.NX) - fpi * pv(J, 0, k)) / __ldg(polar + i + G_);
      else
        d1 += dt * ((__ldg(H3 + k) - __ldg(H3 + k - g.NX)) - fpi * pv(J, 0, k)) *
              tabv(tab, g, CLS_HN, T_ISH, i, j);
    }
    if (i >= 0 && i <= g.n_r && j >= 0 && j < g.n_th)
      d2 += dt * (-(__ldg(H3 + k) - __ldg(H3 + k - 1)) - fpi * pv(J, 1, k)) *
            tabv(tab, g, CLS_NH, T_ISH, i, j);
    if (i >= 0 && i <= g.n_r && j >= 1 && j < g.n_th)
      d3 += dt * ((__ldg(H2 + k) - __ldg(H2 + k - 1)) - (__ldg(H1 + k) - __ldg(H1 + k - g.NX)) -
                  fpi * pv(J, 2, k)) *
            tabv(tab, g, CLS_NN, T_ISH, i, j);
    if (do_match) {
      d1 = match(g, d1, Di1, k, polar + 2 * g.NX, i, j);
      d2 = match(g, d2, Di2, k, polar + g.NX, i, j);
      d3 = match(g, d3, Di3, k, polar + g.NX, i, j);
    }
    D1[k] = d1; D2[k] = d2; D3[k] = d3;
  }
}

template <typename T>
__global__ void k_copy3(int64_t n, const T *a0, const T *a1, const T *a2, T *b0, T *b1, T *b2) {
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n;
       t += (int64_t)gridDim.x * blockDim.x) {
    b0[t] = a0[t]; b1[t] = a1[t]; b2[t] = a2[t];
  }
}

template <typename T>
__global__ void k_zero(T *p, int64_t n) {
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n;
       t += (int64_t)gridDim.x * blockDim.x)
    p[t] = (T)0;
}

int blocks_for(int64_t n) {
  int64_t b = (n + TPB - 1) / TPB;
  if (b > 152 * 32) b = 152 * 32;
  return (int)(b < 1 ? 1 : b);
}

template <typename T>
Pair3<T> one(T *const p[3]) {
  Pair3<T> P;
  for (int c = 0; c < 3; ++c) { P.a[c] = p[c]; P.b[c] = p[c]; }
  P.wa = (T)1; P.wb = (T)0;
  return P;
}
template <typename T>
Pair3<T> mean(T *const p[3], T *const q[3]) {
  Pair3<T> P;
  for (int c = 0; c < 3; ++c) { P.a[c] = p[c]; P.b[c] = q[c]; }
  P.wa = (T)0.5; P.wb = (T)0.5;
  return P;
}

template <typename T>
void horizon(const GridP &g, T *const p[3], cudaStream_t st) {
  const int64_t n = (int64_t)(g.n_f + 1 + G_) * g.NY * 3;
  k_horizon<T><<<blocks_for(n), TPB, 0, st>>>(g, p[0], p[1], p[2]);
  COUNT_LAUNCH(1);
}
template <typename T>
void axis(const GridP &g, T *const p[3], int isB, cudaStream_t st) {
  const int64_t n = (int64_t)g.NX * (2 * G_ + 1) * 3;
  k_axis<T><<<blocks_for(n), TPB, 0, st>>>(g, p[0], p[1], p[2], isB);
  COUNT_LAUNCH(1);
}
template <typename T>
void auxE(const GridP &g, Pair3<T> B, Pair3<T> D, const FieldPtrsT<T> &F, cudaStream_t st) {
  const int64_t n = (int64_t)(g.n_r + 3) * (g.n_th + 1);
  k_aux_E<T><<<blocks_for(n), TPB, 0, st>>>(g, B, D, F.tab, F.E[0], F.E[1], F.E[2]);
  COUNT_LAUNCH(1);
}
template <typename T>
void auxH(const GridP &g, Pair3<T> B, Pair3<T> D, const FieldPtrsT<T> &F, cudaStream_t st) {
  const int64_t n = (int64_t)(g.n_r + 3) * (g.n_th + 1);
  k_aux_H<T><<<blocks_for(n), TPB, 0, st>>>(g, B, D, F.tab, F.H[0], F.H[1], F.H[2]);
  COUNT_LAUNCH(1);
}

}  // namespace

template <typename T>
cudaError_t launch_metric_tables(const GridP &g, T *tab, T *polar, cudaStream_t st) {
  k_metric_tables<T><<<blocks_for(4 * plane_size(g)), TPB, 0, st>>>(g, tab, polar);
  COUNT_LAUNCH(1);
  return cudaGetLastError();
}

cudaError_t launch_dt_min(const GridP &g, double *scratch, int, double *out, cudaStream_t st) {
  unsigned long long *u = reinterpret_cast<unsigned long long *>(scratch);
  const unsigned long long inf = 0x7FF0000000000000ull;
  cudaMemcpyAsync(u, &inf, sizeof(inf), cudaMemcpyHostToDevice, st);
  k_dt_min<<<blocks_for((int64_t)g.n_r * g.n_th), TPB, 0, st>>>(g, u);
  COUNT_LAUNCH(1);
  cudaMemcpyAsync(out, u, sizeof(double), cudaMemcpyDeviceToHost, st);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_zero(T *p, int64_t n, cudaStream_t st) {
  k_zero<T><<<blocks_for(n), TPB, 0, st>>>(p, n);
  COUNT_LAUNCH(1);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_init_fields(const GridP &g, const FieldPtrsT<T> &F, int kind, double B0,
                               cudaStream_t st) {
  const int64_t ps = plane_size(g);
  for (int c = 0; c < 3; ++c) {
    launch_zero(F.B[c], ps, st);
    launch_zero(F.D[c], ps, st);
  }
  if (kind == GRPIC_FIELD_WALD || kind == GRPIC_FIELD_VERTICAL || kind == GRPIC_FIELD_MONOPOLE) {
    const int64_t n = (int64_t)(g.n_r + 2 * G_ + 1) * (g.n_th + 1);
    k_init_fields<T><<<blocks_for(n), TPB, 0, st>>>(g, F, kind, B0);
    COUNT_LAUNCH(1);
  }
  return cudaGetLastError();
}

// After em holds the initial B, D: boundary fills, em0 = em, initial-field copy,
// cur0 = cur = 0, B^n = B.
template <typename T>
cudaError_t launch_field_finish_init(const GridP &g, const FieldPtrsT<T> &F, int, cudaStream_t st) {
  const int64_t ps = plane_size(g);
  horizon(g, F.B, st);
  horizon(g, F.D, st);
  axis(g, F.B, 1, st);
  axis(g, F.D, 0, st);
  k_copy3<T><<<blocks_for(ps), TPB, 0, st>>>(ps, F.B[0], F.B[1], F.B[2], F.B0[0], F.B0[1], F.B0[2]);
  k_copy3<T><<<blocks_for(ps), TPB, 0, st>>>(ps, F.D[0], F.D[1], F.D[2], F.D0[0], F.D0[1], F.D0[2]);
  k_copy3<T><<<blocks_for(ps), TPB, 0, st>>>(ps, F.B[0], F.B[1], F.B[2], F.Bi[0], F.Bi[1], F.Bi[2]);
  k_copy3<T><<<blocks_for(ps), TPB, 0, st>>>(ps, F.D[0], F.D[1], F.D[2], F.Di[0], F.Di[1], F.Di[2]);
  k_copy3<T><<<blocks_for(ps), TPB, 0, st>>>(ps, F.B[0], F.B[1], F.B[2], F.Bn[0], F.Bn[1], F.Bn[2]);
  COUNT_LAUNCH(5);
  for (int c = 0; c < 3; ++c) {
    launch_zero(F.J[c], ps, st);
    launch_zero(F.J0[c], ps, st);
    launch_zero(F.E[c], ps, st);
    launch_zero(F.H[c], ps, st);
    launch_zero(F.Dh[c], ps, st);
  }
  return cudaGetLastError();
}

// Loop step 2 of Sec. 3.4: B^{n-1} = (B^{n-3/2} + B^{n-1/2})/2, D^{n-1/2} = (D^{n-1} + D^n)/2,
// E^{n-1/2} from {B^{n-1/2}, D^{n-1/2}}, auxiliary Faraday B^{n-1} -> B^n (BN planes).
template <typename T>
cudaError_t launch_predict(const GridP &g, const FieldPtrsT<T> &F, cudaStream_t st) {
  auxE(g, one(F.B), mean(F.D0, F.D), F, st);
  const Pair3<T> Bm = mean(F.B0, F.B);
  const int64_t ps = plane_size(g);
  k_faraday<T><<<blocks_for(ps), TPB, 0, st>>>(g, Bm, F.E[0], F.E[1], F.E[2], F.tab, nullptr,
                                               F.Bn[0], F.Bn[1], F.Bn[2], nullptr, nullptr,
                                               nullptr, 0);
  COUNT_LAUNCH(1);
  horizon(g, F.Bn, st);
  axis(g, F.Bn, 1, st);
  return cudaGetLastError();
}

// Loop steps 5-7 of Sec. 3.4 (J holds J^{n+1/2}). Writes B^{n+1/2} into the B0 planes and
// D^{n+1} into the D0 planes; the caller then swaps em/em0 and cur/cur0.
template <typename T>
cudaError_t launch_advance(const GridP &g, const FieldPtrsT<T> &F, cudaStream_t st) {
  const int64_t ps = plane_size(g);
  // step 6: E^n, H^n from {B^n, D^n}; Faraday B^{n-1/2} -> B^{n+1/2}
  auxE(g, one(F.Bn), one(F.D), F, st);
  auxH(g, one(F.Bn), one(F.D), F, st);
  k_faraday<T><<<blocks_for(ps), TPB, 0, st>>>(g, one(F.B), F.E[0], F.E[1], F.E[2], F.tab,
                                               F.polar + g.NX, F.B0[0], F.B0[1], F.B0[2],
                                               F.Bi[0], F.Bi[1], F.Bi[2], 1);
  COUNT_LAUNCH(1);
  horizon(g, F.B0, st);
  axis(g, F.B0, 1, st);
  // step 7: auxiliary Ampere D^{n-1/2} -> D^{n+1/2} with H^n and J^n = (J^{n-1/2} + J^{n+1/2})/2
  k_ampere<T><<<blocks_for(ps), TPB, 0, st>>>(g, mean(F.D0, F.D), F.H[0], F.H[1], F.H[2],
                                              mean(F.J0, F.J), F.tab, F.polar, F.Dh[0], F.Dh[1],
                                              F.Dh[2], nullptr, nullptr, nullptr, 0);
  COUNT_LAUNCH(1);
  horizon(g, F.Dh, st);
  // H^{n+1/2} from {B^{n+1/2}, D^{n+1/2}}; final Ampere D^n -> D^{n+1} with J^{n+1/2}
  auxH(g, one(F.B0), one(F.Dh), F, st);
  k_ampere<T><<<blocks_for(ps), TPB, 0, st>>>(g, one(F.D), F.H[0], F.H[1], F.H[2], one(F.J),
                                              F.tab, F.polar, F.D0[0], F.D0[1], F.D0[2], F.Di[0],
                                              F.Di[1], F.Di[2], 1);
  COUNT_LAUNCH(1);
  horizon(g, F.D0, st);
  axis(g, F.D0, 0, st);
  return cudaGetLastError();
}

// The auxiliary fields E and H (Eqs. discretized-auxE, discretized-auxH) of the em planes as
// they stand (B^{n+1/2} and D^{n+1} after a step), into the E and H scratch planes.
template <typename T>
cudaError_t launch_aux_fields(const GridP &g, const FieldPtrsT<T> &F, cudaStream_t st) {
  auxE(g, one(F.B), one(F.D), F, st);
  auxH(g, one(F.B), one(F.D), F, st);
  return cudaGetLastError();
}

#define INSTANTIATE_FIELDS(T)                                                                    \
  template cudaError_t launch_metric_tables<T>(const GridP &, T *, T *, cudaStream_t);         \
  template cudaError_t launch_zero<T>(T *, int64_t, cudaStream_t);                              \
  template cudaError_t launch_init_fields<T>(const GridP &, const FieldPtrsT<T> &, int, double, \
                                             cudaStream_t);                                     \
  template cudaError_t launch_field_finish_init<T>(const GridP &, const FieldPtrsT<T> &, int,   \
                                                   cudaStream_t);                               \
  template cudaError_t launch_predict<T>(const GridP &, const FieldPtrsT<T> &, cudaStream_t);   \
  template cudaError_t launch_advance<T>(const GridP &, const FieldPtrsT<T> &, cudaStream_t);   \
  template cudaError_t launch_aux_fields<T>(const GridP &, const FieldPtrsT<T> &, cudaStream_t);
INSTANTIATE_FIELDS(double)
INSTANTIATE_FIELDS(float)
