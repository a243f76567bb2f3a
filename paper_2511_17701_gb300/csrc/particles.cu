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

// Eq. (discretized-geodesic-u): implicit midpoint with fixed n_iter, metric at x^n.
__device__ __forceinline__ void geodesic_momentum(const GridP &g, const MetricV &m,
                                                  const MetricD &d, double u[3]) {
  const double u0 = u[0], u1 = u[1];
  double t0 = u0, t1 = u1;
  const double u2 = u[2];  // u_3 is not changed by the geodesic substep
  for (int it = 0; it < g.n_iter; ++it) {
    const double b0 = 0.5 * (u0 + t0), b1 = 0.5 * (u1 + t1);
    const double q = 1.0 + m.H11 * b0 * b0 + m.H22 * b1 * b1 + m.H33 * u2 * u2 +
                     2.0 * m.H13 * b0 * u2;
    const double ig = rsqrt(q);        // 1 / gamma_bar
    const double U0 = q * ig / m.alpha;  // u^0 = gamma / alpha
    const double hU = 0.5 * m.alpha * ig;  // 1 / (2 u^0)
    const double k1 = d.d1H11 * b0 * b0 + d.d1H22 * b1 * b1 + d.d1H33 * u2 * u2 +
                      2.0 * d.d1H13 * b0 * u2;
    const double k2 = d.d2H11 * b0 * b0 + d.d2H22 * b1 * b1 + d.d2H33 * u2 * u2 +
                      2.0 * d.d2H13 * b0 * u2;
    t0 = u0 + g.dt * (-m.alpha * U0 * d.d1alpha + b0 * d.d1beta1 - hU * k1);
    t1 = u1 + g.dt * (-m.alpha * U0 * d.d2alpha + b0 * d.d2beta1 - hU * k2);
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

// dphi/dt = alpha/gamma h^{3j} u_j at a point (Eq. discretized-geodesic-x-phi; also J^3/q).
__device__ __forceinline__ double phi_rate(const GridP &g, double x1, double x2,
                                           const double u[3]) {
  MetricV m;
  metric_eval<false>(g, x1, x2, true, m, nullptr);
  return m.alpha * rsqrt(1.0 + m.H11 * u[0] * u[0] + m.H22 * u[1] * u[1] +
                         m.H33 * u[2] * u[2] + 2.0 * m.H13 * u[0] * u[2]) *
         (m.H13 * u[0] + m.H33 * u[2]);
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
    MetricV m;
    MetricD md;
    metric_eval<true>(g, x1, x2, true, m, &md);
    // step 3: to the tetrad basis
    double Bh[3], Dh[3], uh[3], u[3] = {s.u1[k], s.u2[k], s.u3[k]};
    t_vec_to_hat(m, Bv, Bh);
    t_vec_to_hat(m, Dv, Dh);
    t_cov_to_hat(m, u, uh);
    const double hq = s.qm * m.alpha * 0.5 * g.dt;
    boris_step(uh, Dh, Bh, hq);      // step 4
    t_hat_to_cov(m, uh, u);          // step 5
    geodesic_momentum(g, m, md, u);  // step 6
    t_cov_to_hat(m, u, uh);          // step 7
    boris_step(uh, Dh, Bh, hq);      // step 8
    t_hat_to_cov(m, uh, u);          // step 9
    // step 10: implicit coordinate push, Eq. (discretized-geodesic-x), metric at x_bar
    double t1 = dx1, t2 = dx2;
    for (int it = 0; it < g.n_iter; ++it) {
      MetricV mb;
      metric_eval<false>(g, i1 + 0.5 * (dx1 + t1), i2 + 0.5 * (dx2 + t2), true, mb, nullptr);
      const double ig = rsqrt(1.0 + mb.H11 * u[0] * u[0] + mb.H22 * u[1] * u[1] +
                              mb.H33 * u[2] * u[2] + 2.0 * mb.H13 * u[0] * u[2]);
      const double ag = mb.alpha * ig;
      t1 = dx1 + g.dt * (ag * (mb.H11 * u[0] + mb.H13 * u[2]) - mb.beta1);
      t2 = dx2 + g.dt * (ag * mb.H22 * u[1]);
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
    const double v3 = phi_rate(g, 0.5 * (x1 + xb1), 0.5 * (x2 + xb2), u);
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
    const double v3 = phi_rate(g, 0.5 * (xa1 + xb1), 0.5 * (xa2 + xb2), u);
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
