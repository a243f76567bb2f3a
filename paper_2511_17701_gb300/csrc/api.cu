// api.cu -- the C ABI of include/grpic.h: context, arena layout, argument checks and the
// order of launches for each entry point. No device memory is allocated here: every
// buffer is carved out of the caller's arena.
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <new>
#include <utility>
#include <vector>

#include "grpic_internal.cuh"

namespace {

constexpr size_t ALIGN = 256;

struct SpeciesState {
  int64_t cap = 0, n_bound = 0;
  double qm = 0.0, qc = 0.0;
  bool loaded = false;
  grpic_particles soa[2];
  int live = 0;
  int64_t *n_dev = nullptr;
  size_t off_n = 0, off_soa[2][14] = {};
};

constexpr size_t kElem[14] = {4, 4, 8, 8, 8, 8, 8, 8, 8, 1, 4, 4, 8, 8};

size_t up(size_t x) { return (x + ALIGN - 1) / ALIGN * ALIGN; }

__global__ void k_set_i64(int64_t *p, int64_t v) { *p = v; }

}  // namespace

long long grpic_launches = 0;

enum { PH_PREDICT = 0, PH_SORT, PH_PUSH, PH_DEPOSIT, PH_ADVANCE, PH_N };

struct grpic_ctx {
  grpic_config cfg;
  GridP g;
  size_t need = 0;
  char *arena = nullptr;
  cudaStream_t stream = nullptr;
  bool bound = false, metric_ready = false, fields_ready = false;
  // arena offsets
  size_t off_planes = 0, off_tab = 0, off_polar = 0, off_dt = 0, off_diag = 0;
  size_t off_keys[2] = {}, off_vals[2] = {}, off_hist = 0, off_bsum = 0, off_alive = 0;
  int64_t max_cap = 0;
  FieldPtrs F;
  SpeciesState sp[GRPIC_MAX_SPECIES];
  SortScratch S;
  unsigned long long *diag = nullptr;
  int64_t step = 0;
  // optional per-phase timing with CUDA events on the bound stream
  bool timing = false;
  std::vector<std::pair<cudaEvent_t, cudaEvent_t>> ev[PH_N];
  size_t ev_used[PH_N] = {};
  int64_t push_calls = 0;
  char err[512];
};

namespace {

grpic_status fail(grpic_ctx *c, grpic_status s, const char *fmt, ...) {
  if (c) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(c->err, sizeof(c->err), fmt, ap);
    va_end(ap);
  }
  return s;
}

grpic_status cuda_check(grpic_ctx *c, cudaError_t e, const char *where) {
  if (e == cudaSuccess) return GRPIC_OK;
  return fail(c, GRPIC_ECUDA, "%s: %s", where, cudaGetErrorString(e));
}

#define CK(call)                                                     \
  do {                                                               \
    grpic_status s_ = cuda_check(ctx, (call), #call);                \
    if (s_ != GRPIC_OK) return s_;                                   \
  } while (0)

template <typename T>
T *at(grpic_ctx *c, size_t off) {
  return reinterpret_cast<T *>(c->arena + off);
}

void assign_species_ptrs(grpic_ctx *c, SpeciesState &s) {
  for (int b = 0; b < 2; ++b) {
    grpic_particles &p = s.soa[b];
    const size_t *o = s.off_soa[b];
    p.i1 = at<int32_t>(c, o[0]); p.i2 = at<int32_t>(c, o[1]);
    p.dx1 = at<double>(c, o[2]); p.dx2 = at<double>(c, o[3]);
    p.u1 = at<double>(c, o[4]); p.u2 = at<double>(c, o[5]); p.u3 = at<double>(c, o[6]);
    p.phi = at<double>(c, o[7]); p.w = at<double>(c, o[8]);
    p.tag = at<uint8_t>(c, o[9]);
    p.i1p = at<int32_t>(c, o[10]); p.i2p = at<int32_t>(c, o[11]);
    p.dx1p = at<double>(c, o[12]); p.dx2p = at<double>(c, o[13]);
  }
  s.n_dev = at<int64_t>(c, s.off_n);
}

SpeciesDev dev_view(const SpeciesState &s, int which) {
  const grpic_particles &p = s.soa[which];
  SpeciesDev d;
  d.i1 = p.i1; d.i2 = p.i2; d.dx1 = p.dx1; d.dx2 = p.dx2;
  d.u1 = p.u1; d.u2 = p.u2; d.u3 = p.u3; d.phi = p.phi; d.w = p.w; d.tag = p.tag;
  d.i1p = p.i1p; d.i2p = p.i2p; d.dx1p = p.dx1p; d.dx2p = p.dx2p;
  d.n = s.n_dev; d.qm = s.qm; d.qc = s.qc;
  return d;
}

double *plane_of(grpic_ctx *c, int k) {
  FieldPtrs &F = c->F;
  if (k < 3) return F.B[k];
  if (k < 6) return F.D[k - 3];
  if (k < 9) return F.B0[k - 6];
  if (k < 12) return F.D0[k - 9];
  if (k < 15) return F.J[k - 12];
  if (k < 18) return F.J0[k - 15];
  if (k < 21) return F.Bn[k - 18];
  if (k < 24) return F.Bi[k - 21];
  return F.Di[k - 24];
}

grpic_status need_bound(grpic_ctx *ctx) {
  if (!ctx) return GRPIC_EINVAL;
  if (!ctx->bound) return fail(ctx, GRPIC_ESTATE, "no arena bound (grpic_bind)");
  return GRPIC_OK;
}
grpic_status need_fields(grpic_ctx *ctx) {
  grpic_status s = need_bound(ctx);
  if (s) return s;
  if (!ctx->metric_ready) return fail(ctx, GRPIC_ESTATE, "metric not initialised (grpic_init_metric)");
  if (!ctx->fields_ready) return fail(ctx, GRPIC_ESTATE, "fields not initialised (grpic_init_fields)");
  return GRPIC_OK;
}
grpic_status need_species(grpic_ctx *ctx, int s) {
  if (s < 0 || s >= ctx->cfg.n_species) return fail(ctx, GRPIC_EINVAL, "species %d out of range", s);
  return GRPIC_OK;
}

// Records a start event on construction and a stop event on destruction when the
// context's timing is on.
struct PhaseTimer {
  grpic_ctx *c;
  int ph;
  std::pair<cudaEvent_t, cudaEvent_t> *pr = nullptr;
  PhaseTimer(grpic_ctx *ctx, int phase) : c(ctx), ph(phase) {
    if (!c->timing) return;
    if (c->ev_used[ph] == c->ev[ph].size()) {
      std::pair<cudaEvent_t, cudaEvent_t> e{nullptr, nullptr};
      if (cudaEventCreate(&e.first) != cudaSuccess || cudaEventCreate(&e.second) != cudaSuccess)
        return;
      c->ev[ph].push_back(e);
    }
    pr = &c->ev[ph][c->ev_used[ph]++];
    cudaEventRecord(pr->first, c->stream);
  }
  ~PhaseTimer() {
    if (pr) cudaEventRecord(pr->second, c->stream);
  }
};

cudaError_t copy(void *dst, const void *src, size_t bytes, cudaStream_t st) {
  if (bytes == 0) return cudaSuccess;
  return cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDefault, st);
}

}  // namespace

extern "C" {

grpic_status grpic_create(const grpic_config *cfg, grpic_ctx **out) {
  if (!cfg || !out) return GRPIC_EINVAL;
  *out = nullptr;
  const grpic_config &c = *cfg;
  if (c.metric != GRPIC_METRIC_KS0 && c.metric != GRPIC_METRIC_KS) return GRPIC_EINVAL;
  if (c.n_r < 4 || c.n_theta < 4 || c.n_r > 65536 || c.n_theta > 65536) return GRPIC_EINVAL;
  if (!(c.r_min > 0.0) || !(c.r_max > c.r_min)) return GRPIC_EINVAL;
  if (c.metric == GRPIC_METRIC_KS && !(c.a >= 0.0 && c.a < 1.0)) return GRPIC_EINVAL;
  if (c.n_iter < 1 || c.n_iter > 1000) return GRPIC_EINVAL;
  if (!(c.small_angle > 0.0 && c.small_angle < 0.1)) return GRPIC_EINVAL;
  if (c.n_filter < 0 || c.n_filter + 2 >= c.n_r) return GRPIC_EINVAL;
  if (c.n_species < 1 || c.n_species > GRPIC_MAX_SPECIES) return GRPIC_EINVAL;
  if (c.precision != GRPIC_FP64) return GRPIC_EINVAL;
  if (c.tile_r < 1 || c.tile_theta < 1 || c.sort_every < 0) return GRPIC_EINVAL;
  if (!(c.dt > 0.0) && !(c.cfl > 0.0 && c.cfl <= 1.0)) return GRPIC_EINVAL;
  for (int s = 0; s < c.n_species; ++s)
    if (c.capacity[s] < 0 || c.capacity[s] >= ((int64_t)1 << 31)) return GRPIC_EINVAL;

  grpic_ctx *ctx = new (std::nothrow) grpic_ctx;
  if (!ctx) return GRPIC_ENOMEM;
  ctx->cfg = c;
  ctx->err[0] = 0;
  GridP &g = ctx->g;
  g.n_r = c.n_r; g.n_th = c.n_theta;
  g.NX = c.n_r + 2 * G_ + 1; g.NY = c.n_theta + 2 * G_ + 1;
  g.n_iter = c.n_iter; g.n_f = c.n_filter;
  g.stop_on_repeat = c.full_iterations ? 0 : 1;
  g.r_min = c.r_min; g.r_max = c.r_max;
  g.dxi = log(c.r_max / c.r_min) / c.n_r;
  g.dth = GRPIC_PI / c.n_theta;
  g.ig2 = 1.0 / (g.dth * g.dth);
  g.a = c.metric == GRPIC_METRIC_KS ? c.a : 0.0;
  g.M = c.metric == GRPIC_METRIC_KS ? 1.0 : 0.0;
  g.dt = c.dt;
  g.small_angle = c.small_angle;
  g.r_absorb = c.r_absorb;
  g.absorb_coef = c.absorb_coef;

  // arena layout
  const size_t ps = (size_t)plane_size(g);
  size_t off = 0;
  ctx->off_planes = off; off += up(ps * 8) * 36;
  ctx->off_tab = off;    off += up(ps * 8) * 4 * T_NQ;
  ctx->off_polar = off;  off += up((size_t)g.NX * 8);
  ctx->off_dt = off;     off += up(64);
  ctx->off_diag = off;   off += up(DG_N * 8);
  ctx->max_cap = 1;
  for (int s = 0; s < c.n_species; ++s) {
    SpeciesState &sp = ctx->sp[s];
    sp.cap = c.capacity[s];
    if (sp.cap > ctx->max_cap) ctx->max_cap = sp.cap;
    sp.off_n = off; off += up(8);
    for (int b = 0; b < 2; ++b)
      for (int a = 0; a < 14; ++a) {
        sp.off_soa[b][a] = off;
        off += up((size_t)(sp.cap > 0 ? sp.cap : 1) * kElem[a]);
      }
  }
  for (int b = 0; b < 2; ++b) {
    ctx->off_keys[b] = off; off += up((size_t)ctx->max_cap * 4);
    ctx->off_vals[b] = off; off += up((size_t)ctx->max_cap * 4);
  }
  ctx->off_hist = off;  off += up((size_t)sort_hist_entries(ctx->max_cap) * 4);
  ctx->off_bsum = off;  off += up((size_t)sort_bsum_entries(ctx->max_cap) * 4);
  ctx->off_alive = off; off += up(8);
  ctx->need = off;
  *out = ctx;
  return GRPIC_OK;
}

size_t grpic_arena_bytes(const grpic_ctx *ctx) { return ctx ? ctx->need : 0; }

grpic_status grpic_bind(grpic_ctx *ctx, void *arena, size_t bytes, void *stream) {
  if (!ctx) return GRPIC_EINVAL;
  if (!arena) return fail(ctx, GRPIC_EINVAL, "null arena");
  if (((uintptr_t)arena) % ALIGN) return fail(ctx, GRPIC_EINVAL, "arena not 256-byte aligned");
  if (bytes < ctx->need)
    return fail(ctx, GRPIC_ENOMEM, "arena has %zu bytes, %zu needed", bytes, ctx->need);
  ctx->arena = static_cast<char *>(arena);
  ctx->stream = static_cast<cudaStream_t>(stream);
  const size_t ps = (size_t)plane_size(ctx->g);
  const size_t pb = up(ps * 8);
  double *pl[36];
  for (int k = 0; k < 36; ++k) pl[k] = at<double>(ctx, ctx->off_planes + k * pb);
  FieldPtrs &F = ctx->F;
  for (int c = 0; c < 3; ++c) {
    F.B[c] = pl[c]; F.D[c] = pl[3 + c]; F.B0[c] = pl[6 + c]; F.D0[c] = pl[9 + c];
    F.J[c] = pl[12 + c]; F.J0[c] = pl[15 + c]; F.Bn[c] = pl[18 + c];
    F.Bi[c] = pl[21 + c]; F.Di[c] = pl[24 + c];
    F.E[c] = pl[27 + c]; F.H[c] = pl[30 + c]; F.Dh[c] = pl[33 + c];
  }
  F.tab = at<double>(ctx, ctx->off_tab);
  F.polar = at<double>(ctx, ctx->off_polar);
  ctx->diag = at<unsigned long long>(ctx, ctx->off_diag);
  for (int s = 0; s < ctx->cfg.n_species; ++s) assign_species_ptrs(ctx, ctx->sp[s]);
  SortScratch &S = ctx->S;
  for (int b = 0; b < 2; ++b) {
    S.keys[b] = at<uint32_t>(ctx, ctx->off_keys[b]);
    S.vals[b] = at<uint32_t>(ctx, ctx->off_vals[b]);
  }
  S.hist = at<uint32_t>(ctx, ctx->off_hist);
  S.bsum = at<uint32_t>(ctx, ctx->off_bsum);
  S.alive = at<unsigned long long>(ctx, ctx->off_alive);
  S.max_n = ctx->max_cap;
  S.max_blocks = 0;
  CK(cudaMemsetAsync(ctx->diag, 0, DG_N * 8, ctx->stream));
  for (int s = 0; s < ctx->cfg.n_species; ++s)
    CK(cudaMemsetAsync(ctx->sp[s].n_dev, 0, 8, ctx->stream));
  ctx->bound = true;
  ctx->metric_ready = ctx->fields_ready = false;
  return GRPIC_OK;
}

grpic_status grpic_init_metric(grpic_ctx *ctx) {
  grpic_status s = need_bound(ctx);
  if (s) return s;
  FieldPtrs &F = ctx->F;
  CK(launch_metric_tables(ctx->g, const_cast<double *>(F.tab), const_cast<double *>(F.polar),
                          ctx->stream));
  if (!(ctx->cfg.dt > 0.0)) {
    double dmin = 0.0;
    CK(launch_dt_min(ctx->g, at<double>(ctx, ctx->off_dt), 8, &dmin, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    if (!(dmin > 0.0) || !isfinite(dmin)) return fail(ctx, GRPIC_EINVAL, "bad CFL minimum %g", dmin);
    ctx->g.dt = ctx->cfg.cfl * dmin;
  } else {
    ctx->g.dt = ctx->cfg.dt;
  }
  ctx->metric_ready = true;
  return GRPIC_OK;
}

double grpic_dt(const grpic_ctx *ctx) { return ctx && ctx->metric_ready ? ctx->g.dt : 0.0; }

grpic_status grpic_init_fields(grpic_ctx *ctx, int kind, double B0) {
  grpic_status s = need_bound(ctx);
  if (s) return s;
  if (!ctx->metric_ready) return fail(ctx, GRPIC_ESTATE, "metric not initialised");
  if (kind < GRPIC_FIELD_ZERO || kind > GRPIC_FIELD_USER) return fail(ctx, GRPIC_EINVAL, "bad field kind");
  if (kind != GRPIC_FIELD_USER) CK(launch_init_fields(ctx->g, ctx->F, kind, B0, ctx->stream));
  CK(launch_field_finish_init(ctx->g, ctx->F, kind == GRPIC_FIELD_USER, ctx->stream));
  ctx->fields_ready = true;
  ctx->step = 0;
  return GRPIC_OK;
}

grpic_status grpic_load_particles(grpic_ctx *ctx, int species, int64_t n, double qm, double qc,
                                  double density_power, const grpic_particle_init *in) {
  grpic_status s = need_bound(ctx);
  if (s) return s;
  if ((s = need_species(ctx, species))) return s;
  if (!ctx->metric_ready) return fail(ctx, GRPIC_ESTATE, "metric not initialised");
  SpeciesState &sp = ctx->sp[species];
  if (n < 0 || n > sp.cap) return fail(ctx, GRPIC_ECAPACITY, "%lld particles, capacity %lld", (long long)n, (long long)sp.cap);
  if (n > 0 && (!in || !in->i1 || !in->i2 || !in->dx1 || !in->dx2 || !in->uh1 || !in->uh2 || !in->uh3 || !in->w0))
    return fail(ctx, GRPIC_EINVAL, "null particle array");
  sp.qm = qm; sp.qc = qc;
  const grpic_particles &L = sp.soa[sp.live];
  const grpic_particles &T = sp.soa[1 - sp.live];  // staging for the momenta and weights
  const cudaStream_t st = ctx->stream;
  CK(copy(L.i1, in->i1, n * 4, st));
  CK(copy(L.i2, in->i2, n * 4, st));
  CK(copy(L.dx1, in->dx1, n * 8, st));
  CK(copy(L.dx2, in->dx2, n * 8, st));
  CK(copy(T.u1, in->uh1, n * 8, st));
  CK(copy(T.u2, in->uh2, n * 8, st));
  CK(copy(T.u3, in->uh3, n * 8, st));
  CK(copy(T.w, in->w0, n * 8, st));
  grpic_particle_init dv = *in;
  dv.uh1 = T.u1; dv.uh2 = T.u2; dv.uh3 = T.u3; dv.w0 = T.w;
  CK(launch_load(ctx->g, dev_view(sp, sp.live), n, dv, density_power, st));
  k_set_i64<<<1, 1, 0, st>>>(sp.n_dev, n);
  COUNT_LAUNCH(1);
  CK(cudaGetLastError());
  sp.n_bound = n;
  sp.loaded = true;
  return GRPIC_OK;
}

grpic_status grpic_set_particles(grpic_ctx *ctx, int species, int64_t n, double qm, double qc,
                                 const grpic_particles *in) {
  grpic_status s = need_bound(ctx);
  if (s) return s;
  if ((s = need_species(ctx, species))) return s;
  SpeciesState &sp = ctx->sp[species];
  if (n < 0 || n > sp.cap) return fail(ctx, GRPIC_ECAPACITY, "%lld particles, capacity %lld", (long long)n, (long long)sp.cap);
  if (n > 0 && !in) return fail(ctx, GRPIC_EINVAL, "null particle arrays");
  sp.qm = qm; sp.qc = qc;
  const grpic_particles &L = sp.soa[sp.live];
  const cudaStream_t st = ctx->stream;
  if (n > 0) {
    const void *src[14] = {in->i1, in->i2, in->dx1, in->dx2, in->u1, in->u2, in->u3,
                           in->phi, in->w, in->tag, in->i1p, in->i2p, in->dx1p, in->dx2p};
    void *dst[14] = {L.i1, L.i2, L.dx1, L.dx2, L.u1, L.u2, L.u3,
                     L.phi, L.w, L.tag, L.i1p, L.i2p, L.dx1p, L.dx2p};
    for (int a = 0; a < 14; ++a) {
      if (!src[a]) return fail(ctx, GRPIC_EINVAL, "null particle array %d", a);
      CK(copy(dst[a], src[a], (size_t)n * kElem[a], st));
    }
  }
  k_set_i64<<<1, 1, 0, st>>>(sp.n_dev, n);
  COUNT_LAUNCH(1);
  CK(cudaGetLastError());
  sp.n_bound = n;
  sp.loaded = true;
  return GRPIC_OK;
}

grpic_status grpic_species_arrays(grpic_ctx *ctx, int species, grpic_particles *out, int64_t *n) {
  grpic_status s = need_bound(ctx);
  if (s) return s;
  if ((s = need_species(ctx, species))) return s;
  SpeciesState &sp = ctx->sp[species];
  if (out) *out = sp.soa[sp.live];
  if (n) {
    CK(cudaMemcpyAsync(n, sp.n_dev, 8, cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
  }
  return GRPIC_OK;
}

grpic_status grpic_get_particles(grpic_ctx *ctx, int species, grpic_particles *out, int64_t *n) {
  int64_t cnt = 0;
  grpic_particles L;
  grpic_status s = grpic_species_arrays(ctx, species, &L, &cnt);
  if (s) return s;
  if (n) *n = cnt;
  if (!out) return GRPIC_OK;
  const void *src[14] = {L.i1, L.i2, L.dx1, L.dx2, L.u1, L.u2, L.u3,
                         L.phi, L.w, L.tag, L.i1p, L.i2p, L.dx1p, L.dx2p};
  void *dst[14] = {out->i1, out->i2, out->dx1, out->dx2, out->u1, out->u2, out->u3,
                   out->phi, out->w, out->tag, out->i1p, out->i2p, out->dx1p, out->dx2p};
  for (int a = 0; a < 14; ++a)
    if (dst[a]) CK(copy(dst[a], src[a], (size_t)cnt * kElem[a], ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  return GRPIC_OK;
}

grpic_status grpic_plane_ptr(grpic_ctx *ctx, int plane, double **out) {
  grpic_status s = need_bound(ctx);
  if (s) return s;
  if (plane < 0 || plane >= GRPIC_NPLANES || !out) return fail(ctx, GRPIC_EINVAL, "bad plane %d", plane);
  *out = plane_of(ctx, plane);
  return GRPIC_OK;
}

grpic_status grpic_push(grpic_ctx *ctx, int species) {
  grpic_status s = need_fields(ctx);
  if (s) return s;
  if ((s = need_species(ctx, species))) return s;
  SpeciesState &sp = ctx->sp[species];
  if (!sp.loaded) return fail(ctx, GRPIC_ESTATE, "species %d has no particles", species);
  PhaseTimer t(ctx, PH_PUSH);
  CK(launch_push(ctx->g, ctx->F, dev_view(sp, sp.live), sp.n_bound, false, ctx->diag, ctx->stream));
  ++ctx->push_calls;
  return GRPIC_OK;
}

grpic_status grpic_deposit(grpic_ctx *ctx) {
  grpic_status s = need_fields(ctx);
  if (s) return s;
  const int64_t ps = plane_size(ctx->g);
  PhaseTimer t(ctx, PH_DEPOSIT);
  for (int c = 0; c < 3; ++c) CK(launch_zero(ctx->F.J[c], ps, ctx->stream));
  for (int k = 0; k < ctx->cfg.n_species; ++k) {
    SpeciesState &sp = ctx->sp[k];
    if (!sp.loaded) continue;
    CK(launch_deposit(ctx->g, ctx->F, dev_view(sp, sp.live), sp.n_bound, ctx->stream));
  }
  return GRPIC_OK;
}

static void rotate(grpic_ctx *ctx) {
  FieldPtrs &F = ctx->F;
  for (int c = 0; c < 3; ++c) {
    double *t = F.B[c]; F.B[c] = F.B0[c]; F.B0[c] = t;
    t = F.D[c]; F.D[c] = F.D0[c]; F.D0[c] = t;
    t = F.J[c]; F.J[c] = F.J0[c]; F.J0[c] = t;
  }
}

grpic_status grpic_field_step(grpic_ctx *ctx, int phase) {
  grpic_status s = need_fields(ctx);
  if (s) return s;
  if (phase == GRPIC_PREDICT) {
    PhaseTimer t(ctx, PH_PREDICT);
    CK(launch_predict(ctx->g, ctx->F, ctx->stream));
  } else if (phase == GRPIC_ADVANCE) {
    PhaseTimer t(ctx, PH_ADVANCE);
    CK(launch_advance(ctx->g, ctx->F, ctx->stream));
    rotate(ctx);  // em <- (B^{n+1/2}, D^{n+1}), em0 <- (B^{n-1/2}, D^n), cur0 <- J^{n+1/2}
  } else {
    return fail(ctx, GRPIC_EINVAL, "bad phase %d", phase);
  }
  return GRPIC_OK;
}

grpic_status grpic_sort(grpic_ctx *ctx, int species) {
  grpic_status s = need_bound(ctx);
  if (s) return s;
  if ((s = need_species(ctx, species))) return s;
  SpeciesState &sp = ctx->sp[species];
  if (!sp.loaded) return GRPIC_OK;
  PhaseTimer t(ctx, PH_SORT);
  CK(launch_sort(ctx->g, ctx->cfg.tile_r, ctx->cfg.tile_theta, dev_view(sp, sp.live),
                 dev_view(sp, 1 - sp.live), sp.n_bound, sp.n_dev, ctx->S, ctx->stream));
  sp.live = 1 - sp.live;
  return GRPIC_OK;
}

grpic_status grpic_step(grpic_ctx *ctx, int n_steps) {
  grpic_status s = need_fields(ctx);
  if (s) return s;
  if (n_steps < 0) return fail(ctx, GRPIC_EINVAL, "negative step count");
  const int64_t ps = plane_size(ctx->g);
  for (int n = 0; n < n_steps; ++n) {
    {
      PhaseTimer t(ctx, PH_PREDICT);
      CK(launch_predict(ctx->g, ctx->F, ctx->stream));
    }
    if (ctx->cfg.sort_every > 0 && ctx->step % ctx->cfg.sort_every == 0)
      for (int k = 0; k < ctx->cfg.n_species; ++k)
        if ((s = grpic_sort(ctx, k))) return s;
    {
      PhaseTimer t(ctx, PH_PUSH);  // fused push + deposit of every species
      for (int c = 0; c < 3; ++c) CK(launch_zero(ctx->F.J[c], ps, ctx->stream));
      for (int k = 0; k < ctx->cfg.n_species; ++k) {
        SpeciesState &sp = ctx->sp[k];
        if (!sp.loaded) continue;
        CK(launch_push(ctx->g, ctx->F, dev_view(sp, sp.live), sp.n_bound, true, ctx->diag,
                       ctx->stream));
        ++ctx->push_calls;
      }
    }
    {
      PhaseTimer t(ctx, PH_ADVANCE);
      CK(launch_advance(ctx->g, ctx->F, ctx->stream));
    }
    rotate(ctx);
    ++ctx->step;
  }
  return GRPIC_OK;
}

grpic_status grpic_get_diagnostics(grpic_ctx *ctx, grpic_diag *out) {
  grpic_status s = need_bound(ctx);
  if (s) return s;
  if (!out) return GRPIC_EINVAL;
  unsigned long long h[DG_N];
  CK(cudaMemcpyAsync(h, ctx->diag, sizeof(h), cudaMemcpyDeviceToHost, ctx->stream));
  memset(out, 0, sizeof(*out));
  for (int k = 0; k < ctx->cfg.n_species; ++k)
    CK(cudaMemcpyAsync(&out->alive[k], ctx->sp[k].n_dev, 8, cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  CK(cudaMemsetAsync(ctx->diag, 0, sizeof(h), ctx->stream));
  out->left_inner = (int64_t)h[DG_LEFT_INNER];
  out->left_outer = (int64_t)h[DG_LEFT_OUTER];
  out->reflections = (int64_t)h[DG_REFLECT];
  out->nonfinite = (int64_t)h[DG_NONFINITE];
  return GRPIC_OK;
}

grpic_status grpic_set_timing(grpic_ctx *ctx, int enable) {
  if (!ctx) return GRPIC_EINVAL;
  ctx->timing = enable != 0;
  return GRPIC_OK;
}

grpic_status grpic_get_timing(grpic_ctx *ctx, grpic_timing *out) {
  grpic_status s = need_bound(ctx);
  if (s) return s;
  if (!out) return GRPIC_EINVAL;
  CK(cudaStreamSynchronize(ctx->stream));
  double ms[PH_N] = {};
  for (int ph = 0; ph < PH_N; ++ph) {
    for (size_t k = 0; k < ctx->ev_used[ph]; ++k) {
      float t = 0.f;
      CK(cudaEventElapsedTime(&t, ctx->ev[ph][k].first, ctx->ev[ph][k].second));
      ms[ph] += t;
    }
    ctx->ev_used[ph] = 0;
  }
  out->predict_ms = ms[PH_PREDICT];
  out->sort_ms = ms[PH_SORT];
  out->push_ms = ms[PH_PUSH];
  out->deposit_ms = ms[PH_DEPOSIT];
  out->advance_ms = ms[PH_ADVANCE];
  out->push_calls = ctx->push_calls;
  out->launches = grpic_launches;
  ctx->push_calls = 0;
  grpic_launches = 0;
  return GRPIC_OK;
}

const char *grpic_last_error(const grpic_ctx *ctx) { return ctx ? ctx->err : "null context"; }

void grpic_destroy(grpic_ctx *ctx) {
  if (!ctx) return;
  for (int ph = 0; ph < PH_N; ++ph)
    for (auto &e : ctx->ev[ph]) {
      cudaEventDestroy(e.first);
      cudaEventDestroy(e.second);
    }
  delete ctx;
}

}  // extern "C"
