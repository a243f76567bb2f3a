// api.cu -- the C ABI of include/grpic.h: context, arena layout, argument checks and the
// order of launches for each entry point. No device memory is allocated here: every
// buffer is carved out of the caller's arena. Each entry point dispatches on the
// precision of the context (FP64 or mixed).
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <new>
#include <utility>
#include <vector>

#include <cudaTypedefs.h>  // PFN_cuTensorMapEncodeTiled

#include "grpic_internal.cuh"

namespace {

constexpr size_t ALIGN = 256;
constexpr int NARR = 14;
// integer, floating or byte arrays of a species, in the order of grpic_particles
constexpr int kKind[NARR] = {0, 0, 1, 1, 1, 1, 1, 1, 1, 2, 0, 0, 1, 1};

struct SpeciesState {
  int64_t cap = 0, n_bound = 0;
  double qm = 0.0, qc = 0.0;
  bool massless = false;  // gamma without the mass term, no EM push, no deposit
  bool loaded = false;
  grpic_particles soa[2];
  int live = 0;
  int64_t *n_dev = nullptr;
  size_t off_n = 0, off_soa[2][NARR] = {};
  size_t off_gl = 0;  // guard list, mask and counters (mixed path)
  GuardList gl{};
  size_t off_tiles = 0;       // tile ranges of the last sort (mixed path)
  uint32_t *tile_start = nullptr;
  bool tiles_valid = false;
  // the previous-position arrays hold the positions before the last push (false after a
  // fused push + deposit that did not store them)
  bool prev_valid = true;
};

size_t up(size_t x) { return (x + ALIGN - 1) / ALIGN * ALIGN; }

__global__ void k_set_i64(int64_t *p, int64_t v) { *p = v; }

// the alive particles in each of the ranges [c len, (c + 1) len) of a species holding *n
__global__ void k_chunk_counts(const int64_t *n, int64_t *out, int64_t len, int chunks) {
  const int c = threadIdx.x;
  if (c < chunks) {
    const int64_t m = *n - c * len;
    out[c] = m < 0 ? 0 : (m > len ? len : m);
  }
}

}  // namespace

long long grpic_launches = 0;

enum { PH_PREDICT = 0, PH_SORT, PH_PUSH, PH_DEPOSIT, PH_ADVANCE, PH_KERNEL, PH_INJECT, PH_N };

// grpic_step_host streams each FP64 species in this many particle ranges, so that the copies
// of one range overlap the push of another (the mixed push, with its guard lists, streams
// whole species)
constexpr int HOST_CHUNKS = 4;

struct grpic_ctx {
  grpic_config cfg;
  GridP g;
  bool mixed = false;
  size_t fsz = 8;  // bytes of a floating element of fields and particles
  size_t need = 0;
  char *arena = nullptr;
  cudaStream_t stream = nullptr;
  cudaStream_t side = nullptr;  // guard kernels of the mixed push
  cudaEvent_t ev_fork[GRPIC_MAX_SPECIES] = {}, ev_done[GRPIC_MAX_SPECIES] = {};
  cudaEvent_t ev_class[GRPIC_MAX_SPECIES] = {};
  // grpic_step_host: copy streams, events and pinned counts, created on its first call;
  // device counts of the particle ranges it streams (in the arena)
  cudaStream_t h2d = nullptr, d2h = nullptr;
  cudaEvent_t ev_start = nullptr, ev_in[GRPIC_MAX_SPECIES][HOST_CHUNKS] = {},
              ev_pushed[GRPIC_MAX_SPECIES][HOST_CHUNKS] = {};
  int64_t *host_n = nullptr;
  size_t off_chunk = 0;
  bool bound = false, metric_ready = false, fields_ready = false;
  double field_b0 = 1.0;  // amplitude of the analytic field in the planes (1 for user fields)
  size_t off_planes = 0, off_tab = 0, off_polar = 0, off_dt = 0, off_diag = 0, off_ptab = 0;
  size_t off_keys[2] = {}, off_vals[2] = {}, off_hist = 0, off_bsum = 0, off_alive = 0;
  size_t off_stage = 0, off_rho = 0, off_inj = 0;
  int64_t load_chunk = 0;
  int64_t max_cap = 0;
  FieldPtrsT<double> F64;
  FieldPtrsT<float> F32;
  PushTables tb{};
  SpeciesState sp[GRPIC_MAX_SPECIES];
  SortScratch S;
  unsigned long long *diag = nullptr;
  int64_t step = 0;
  bool timing = false;
  bool keep_prev = true;  // the fused push + deposit stores the previous positions
  // tiled_push = 2: the padded copy of B^n and D the tensor copies read, and its tensor map
  size_t off_pad = 0;
  int NXp = 0;
  CUtensorMap tmap;  // aligned as CUtensorMap requires
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

size_t elem_bytes(const grpic_ctx *c, int a) {
  return kKind[a] == 0 ? 4 : (kKind[a] == 1 ? c->fsz : 1);
}

void **slot(grpic_particles &p, int a) {
  void **v[NARR] = {(void **)&p.i1, (void **)&p.i2, &p.dx1, &p.dx2, &p.u1, &p.u2, &p.u3,
                    &p.phi, &p.w, (void **)&p.tag, (void **)&p.i1p, (void **)&p.i2p, &p.dx1p,
                    &p.dx2p};
  return v[a];
}
const void *cslot(const grpic_particles &p, int a) {
  const void *v[NARR] = {p.i1, p.i2, p.dx1, p.dx2, p.u1, p.u2, p.u3,
                         p.phi, p.w, p.tag, p.i1p, p.i2p, p.dx1p, p.dx2p};
  return v[a];
}

void assign_species_ptrs(grpic_ctx *c, SpeciesState &s) {
  for (int b = 0; b < 2; ++b)
    for (int a = 0; a < NARR; ++a) *slot(s.soa[b], a) = c->arena + s.off_soa[b][a];
  s.n_dev = at<int64_t>(c, s.off_n);
}

template <typename T>
SpeciesDevT<T> dev_view(const SpeciesState &s, int which) {
  const grpic_particles &p = s.soa[which];
  SpeciesDevT<T> d;
  d.i1 = p.i1; d.i2 = p.i2;
  d.dx1 = (T *)p.dx1; d.dx2 = (T *)p.dx2;
  d.u1 = (T *)p.u1; d.u2 = (T *)p.u2; d.u3 = (T *)p.u3;
  d.phi = (T *)p.phi; d.w = (T *)p.w; d.tag = p.tag;
  d.i1p = p.i1p; d.i2p = p.i2p; d.dx1p = (T *)p.dx1p; d.dx2p = (T *)p.dx2p;
  d.n = s.n_dev; d.qm = s.qm; d.qc = s.qc; d.f_qm = (float)s.qm; d.f_qc = (float)s.qc;
  d.m2 = s.massless ? 0.0 : 1.0;
  d.f_m2 = (float)d.m2;
  return d;
}

template <typename T>
T *plane_of(FieldPtrsT<T> &F, int k) {
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

template <typename T>
void assign_fields(grpic_ctx *c, FieldPtrsT<T> &F) {
  const size_t pb = up((size_t)plane_size(c->g) * sizeof(T));
  T *pl[36];
  for (int k = 0; k < 36; ++k) pl[k] = at<T>(c, c->off_planes + k * pb);
  for (int i = 0; i < 3; ++i) {
    F.B[i] = pl[i]; F.D[i] = pl[3 + i]; F.B0[i] = pl[6 + i]; F.D0[i] = pl[9 + i];
    F.J[i] = pl[12 + i]; F.J0[i] = pl[15 + i]; F.Bn[i] = pl[18 + i];
    F.Bi[i] = pl[21 + i]; F.Di[i] = pl[24 + i];
    F.E[i] = pl[27 + i]; F.H[i] = pl[30 + i]; F.Dh[i] = pl[33 + i];
  }
  F.tab = at<T>(c, c->off_tab);
  F.polar = at<T>(c, c->off_polar);
}

template <typename T>
void rotate(FieldPtrsT<T> &F) {
  for (int c = 0; c < 3; ++c) {
    std::swap(F.B[c], F.B0[c]);
    std::swap(F.D[c], F.D0[c]);
    std::swap(F.J[c], F.J0[c]);
  }
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

cudaError_t copy(void *dst, const void *src, size_t bytes, cudaStream_t st) {
  if (bytes == 0) return cudaSuccess;
  return cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDefault, st);
}

// Records a start event on construction and a stop event on destruction when the
// context's timing is on.
// the next unused event pair of a phase (null when timing is off or events run out)
std::pair<cudaEvent_t, cudaEvent_t> *next_events(grpic_ctx *c, int ph) {
  if (!c->timing) return nullptr;
  if (c->ev_used[ph] == c->ev[ph].size()) {
    std::pair<cudaEvent_t, cudaEvent_t> e{nullptr, nullptr};
    if (cudaEventCreate(&e.first) != cudaSuccess || cudaEventCreate(&e.second) != cudaSuccess)
      return nullptr;
    c->ev[ph].push_back(e);
  }
  return &c->ev[ph][c->ev_used[ph]++];
}

struct PhaseTimer {
  grpic_ctx *c;
  int ph;
  std::pair<cudaEvent_t, cudaEvent_t> *pr = nullptr;
  PhaseTimer(grpic_ctx *ctx, int phase) : c(ctx), ph(phase) {
    pr = next_events(c, ph);
    if (pr) cudaEventRecord(pr->first, c->stream);
  }
  ~PhaseTimer() {
    if (pr) cudaEventRecord(pr->second, c->stream);
  }
};

// --- precision-dispatched pieces of the hot path
template <typename T>
cudaError_t do_push(grpic_ctx *c, FieldPtrsT<T> &F, int k, bool deposit, int stage = PUSH_ALL) {
  SpeciesState &sp = c->sp[k];
  const std::pair<cudaEvent_t, cudaEvent_t> *kt =
      push_main_stage(stage) ? next_events(c, PH_KERNEL) : nullptr;
  const PushStreams ps{c->stream, c->side, c->ev_fork[k], c->ev_done[k], c->ev_class[k],
                       kt ? kt->first : nullptr, kt ? kt->second : nullptr, stage};
  const int tr = c->cfg.tile_r, tt = c->cfg.tile_theta;
  const int ntr = (c->g.n_r + tr - 1) / tr, ntt = (c->g.n_th + tt - 1) / tt;
  TileInfo ti{};
  ti.start = sp.tiles_valid && c->cfg.tiled_push ? sp.tile_start : nullptr;
  ti.tr = tr;
  ti.tt = tt;
  ti.ntr = ntr;
  ti.n_tiles = ntr * ntt;
  if (c->cfg.tiled_push == 2) {
    ti.tma = 1;
    ti.map = c->tmap;
    ti.pad = at<float>(c, c->off_pad);
    ti.NXp = c->NXp;
  }
  // step 1 of Sec. 3.1 stores the previous position for the deposit; a push that deposits
  // its own move needs it only when a later call reads it (grpic_set_keep_prev): null
  // previous-position arrays tell the kernels to skip the stores
  SpeciesDevT<T> v = dev_view<T>(sp, sp.live);
  const bool write_prev = !deposit || c->keep_prev;
  if (!write_prev) v.i1p = v.i2p = nullptr, v.dx1p = v.dx2p = nullptr;
  if (push_main_stage(stage)) sp.prev_valid = write_prev;
  // massless particles are neutral: their push deposits nothing
  return launch_push<T>(c->g, F, v, c->tb, sp.gl, ti, sp.n_bound, deposit && !sp.massless,
                        c->diag, ps);
}
// the main stream waits for the guard kernels of species k (mixed path)
cudaError_t join_push(grpic_ctx *c, int k) {
  return c->mixed ? cudaStreamWaitEvent(c->stream, c->ev_done[k], 0) : cudaSuccess;
}
template <typename T>
cudaError_t do_zero_J(grpic_ctx *c, FieldPtrsT<T> &F) {
  const int64_t ps = plane_size(c->g);
  for (int i = 0; i < 3; ++i) {
    cudaError_t e = launch_zero<T>(F.J[i], ps, c->stream);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

template <typename T>
cudaError_t charge_check(grpic_ctx *ctx, FieldPtrsT<T> &F, bool after_step, double *out) {
  const int64_t ps = plane_size(ctx->g);
  double *rp = at<double>(ctx, ctx->off_rho), *rn = at<double>(ctx, ctx->off_rho + up(ps * 8));
  double *ra = at<double>(ctx, ctx->off_rho + 2 * up(ps * 8));
  cudaError_t e = launch_zero<double>(rp, ps, ctx->stream);
  if (e == cudaSuccess) e = launch_zero<double>(rn, ps, ctx->stream);
  if (e == cudaSuccess) e = launch_zero<double>(ra, ps, ctx->stream);
  for (int k = 0; k < ctx->cfg.n_species && e == cudaSuccess; ++k) {
    SpeciesState &sp = ctx->sp[k];
    if (sp.loaded && !sp.massless) e = launch_charge_rho<T>(ctx->g, dev_view<T>(sp, sp.live), sp.n_bound, rp, rn,
                                            ra, ctx->stream);
  }
  // with current filtering the currents conserve the filtered charge
  if (e == cudaSuccess && ctx->g.n_f > 0) {
    double *const a[3] = {rp, rn, ra};
    double *const s[3] = {at<double>(ctx, ctx->off_rho + 3 * up(ps * 8)),
                          at<double>(ctx, ctx->off_rho + 4 * up(ps * 8)),
                          at<double>(ctx, ctx->off_rho + 5 * up(ps * 8))};
    const int half[3] = {0, 0, 0};
    const double par[3] = {1.0, 1.0, 1.0};
    e = launch_filter<double>(ctx->g, a, s, half, par, 3, ctx->g.n_f, ctx->stream, nullptr);
  }
  T *const *J = after_step ? F.J0 : F.J;
  if (e == cudaSuccess)
    e = launch_continuity<T>(ctx->g, J[0], J[1], rp, rn, ra, out, ctx->stream);
  return e;
}

}  // namespace

extern "C" {

grpic_status grpic_create(const grpic_config *cfg, grpic_ctx **out) {
  if (!cfg || !out) return GRPIC_EINVAL;
  *out = nullptr;
  const grpic_config &c = *cfg;
  if (c.metric != GRPIC_METRIC_KS0 && c.metric != GRPIC_METRIC_KS) return GRPIC_EINVAL;
  if (c.n_r < 4 || c.n_theta < 4 || c.n_r > 65536 || c.n_theta > 65536) return GRPIC_EINVAL;
  // plane indices are 32-bit in the deposit
  if ((int64_t)(c.n_r + 2 * G_ + 1) * (c.n_theta + 2 * G_ + 1) >= ((int64_t)1 << 31))
    return GRPIC_EINVAL;
  if (!(c.r_min > 0.0) || !(c.r_max > c.r_min)) return GRPIC_EINVAL;
  // the quasi-spherical map (App. A): r0 below r_min; theta(eta) monotone for -1/2 < h0 < 1
  if (!(c.r0 < c.r_min) || !isfinite(c.r0) || !(c.h0 > -0.5 && c.h0 < 1.0)) return GRPIC_EINVAL;
  if (c.metric == GRPIC_METRIC_KS && !(c.a >= 0.0 && c.a < 1.0)) return GRPIC_EINVAL;
  if (c.n_iter < 1 || c.n_iter > 1000) return GRPIC_EINVAL;
  if (!(c.small_angle > 0.0 && c.small_angle < 0.1)) return GRPIC_EINVAL;
  if (c.n_filter < 0 || c.n_filter + 2 >= c.n_r || c.n_filter > 64) return GRPIC_EINVAL;
  // Sec. 3.3.3: the inner boundary lies at least n_f + 1 cells inside the event horizon
  if (c.metric == GRPIC_METRIC_KS &&
      !(c.r0 + (c.r_min - c.r0) * exp((c.n_filter + 1) * log((c.r_max - c.r0) / (c.r_min - c.r0)) /
                                      c.n_r) <= 1.0 + sqrt(1.0 - c.a * c.a)))
    return GRPIC_EINVAL;
  if (c.n_species < 1 || c.n_species > GRPIC_MAX_SPECIES) return GRPIC_EINVAL;
  if (c.precision != GRPIC_FP64 && c.precision != GRPIC_MIXED) return GRPIC_EINVAL;
  if (c.tile_r < 1 || c.tile_theta < 1 || c.sort_every < 0) return GRPIC_EINVAL;
  // the TMA-staged tiled push: the window's first column (tile start - halo + ghosts) must be
  // a multiple of 4 floats, the 16 bytes a tensor copy's innermost coordinate needs
  if (c.tiled_push < 0 || c.tiled_push > 2) return GRPIC_EINVAL;
  if (c.tiled_push == 2 && (c.precision != GRPIC_MIXED || c.tile_r % 4 != 0 ||
                            (G_ - TILE_HALO) % 4 != 0 || c.tile_r + 2 * TILE_HALO > 256 ||
                            c.tile_theta + 2 * TILE_HALO > 256))
    return GRPIC_EINVAL;
  if (c.tile_r > 65536 || c.tile_theta > 65536) return GRPIC_EINVAL;
  {  // the sort's largest live key (the tile-padded cell count) below the dead key, in int range
    const uint64_t ntr = (uint64_t)((c.n_r + c.tile_r - 1) / c.tile_r);
    const uint64_t ntt = (uint64_t)((c.n_theta + c.tile_theta - 1) / c.tile_theta);
    if (ntr * ntt * (uint64_t)c.tile_r * (uint64_t)c.tile_theta > (uint64_t)INT32_MAX)
      return GRPIC_EINVAL;
  }
  if (!(c.dt > 0.0) && !(c.cfl > 0.0 && c.cfl <= 1.0)) return GRPIC_EINVAL;
  if (c.fp64_guard_cells < 0 || 2 * c.fp64_guard_cells >= c.n_theta) return GRPIC_EINVAL;
  if (!(c.iter_tol >= 0.0 && c.iter_tol < 1e-6)) return GRPIC_EINVAL;
  for (int s = 0; s < c.n_species; ++s) {
    if (c.capacity[s] < 0 || c.capacity[s] >= ((int64_t)1 << 31)) return GRPIC_EINVAL;
    if (c.massless[s] != 0 && c.massless[s] != 1) return GRPIC_EINVAL;
  }

  grpic_ctx *ctx = new (std::nothrow) grpic_ctx;
  if (!ctx) return GRPIC_ENOMEM;
  ctx->cfg = c;
  ctx->err[0] = 0;
  ctx->mixed = c.precision == GRPIC_MIXED;
  ctx->fsz = ctx->mixed ? 4 : 8;
  GridP &g = ctx->g;
  g.n_r = c.n_r; g.n_th = c.n_theta;
  g.NX = c.n_r + 2 * G_ + 1; g.NY = c.n_theta + 2 * G_ + 1;
  g.n_iter = c.n_iter; g.n_f = c.n_filter;
  g.stop_on_repeat = c.full_iterations ? 0 : 1;
  g.iter_tol = c.iter_tol;
  g.r_min = c.r_min; g.r_max = c.r_max;
  g.r0 = c.r0; g.h0 = c.h0;
  g.e_min = c.r_min - c.r0;
  g.qks = (c.r0 != 0.0 || c.h0 != 0.0) ? 1 : 0;
  g.c3 = 4.0 * c.h0 / (GRPIC_PI * GRPIC_PI);
  g.dxi = log((c.r_max - c.r0) / (c.r_min - c.r0)) / c.n_r;
  g.dth = GRPIC_PI / c.n_theta;
  g.ig2 = 1.0 / (g.dth * g.dth);
  g.a = c.metric == GRPIC_METRIC_KS ? c.a : 0.0;
  g.M = c.metric == GRPIC_METRIC_KS ? 1.0 : 0.0;
  g.dt = c.dt;
  g.small_angle = c.small_angle;
  g.r_absorb = c.r_absorb;
  g.absorb_coef = c.absorb_coef;
  grid_float_copies(g);
  // the FP64 guard of the mixed pusher: guard cells on either side of the cell holding the
  // horizon, and guard cells next to each axis
  const int guard = c.fp64_guard_cells > 0 ? c.fp64_guard_cells : 4;
  int ih = -1000000;
  if (g.M > 0.0) {
    const double rh = 1.0 + sqrt(1.0 - g.a * g.a);
    ih = (int)floor(log((rh - g.r0) / (g.r_min - g.r0)) / g.dxi);
  }
  ctx->tb.guard_ilo = ih - guard;
  ctx->tb.guard_ihi = ih + guard + 1;
  ctx->tb.guard_j = guard;

  const size_t ps = (size_t)plane_size(g), fs = ctx->fsz;
  size_t off = 0;
  ctx->off_planes = off; off += up(ps * fs) * 36;
  ctx->off_tab = off;    off += up(ps * fs) * 4 * T_NQ;
  ctx->off_polar = off;  off += up((size_t)3 * g.NX * fs);
  ctx->off_ptab = off;   off += 16 * up((size_t)(g.NX > g.NY ? g.NX : g.NY) * 8);
  ctx->off_dt = off;     off += up(64);
  ctx->off_diag = off;   off += up(DG_N * 8);
  ctx->off_chunk = off;  off += up(GRPIC_MAX_SPECIES * HOST_CHUNKS * 8);
  ctx->max_cap = 1;
  for (int s = 0; s < c.n_species; ++s) {
    SpeciesState &sp = ctx->sp[s];
    sp.cap = c.capacity[s];
    sp.massless = c.massless[s] == 1;
    if (sp.cap > ctx->max_cap) ctx->max_cap = sp.cap;
    sp.off_n = off; off += up(8);
    for (int b = 0; b < 2; ++b)
      for (int a = 0; a < NARR; ++a) {
        sp.off_soa[b][a] = off;
        off += up((size_t)(sp.cap > 0 ? sp.cap : 1) * elem_bytes(ctx, a));
      }
  }
  for (int b = 0; b < 2; ++b) {
    ctx->off_keys[b] = off; off += up((size_t)ctx->max_cap * 4);
    ctx->off_vals[b] = off; off += up((size_t)ctx->max_cap * 4);
  }
  ctx->off_hist = off;  off += up((size_t)sort_hist_entries(ctx->max_cap) * 4);
  ctx->off_bsum = off;  off += up((size_t)sort_bsum_entries(ctx->max_cap) * 4);
  ctx->off_alive = off; off += up(8);
  if (ctx->mixed) {
    const int64_t ntiles = (int64_t)((c.n_r + c.tile_r - 1) / c.tile_r) *
                           ((c.n_theta + c.tile_theta - 1) / c.tile_theta);
    for (int s = 0; s < c.n_species; ++s) {
      const size_t cap = (size_t)(ctx->sp[s].cap > 0 ? ctx->sp[s].cap : 1);
      ctx->sp[s].off_gl = off;
      off += up(cap * 4) + up((cap + 31) / 32 * 4) + up(16);
      ctx->sp[s].off_tiles = off;
      off += up((size_t)(ntiles + 1) * 4);
    }
  }
  ctx->off_rho = off; off += 6 * up(ps * 8) + up(64);  // FP64 charge planes of the check
  ctx->off_inj = off; off += up(inject_scratch_bytes(g));  // pair injection per-cell scratch
  if (c.tiled_push == 2) {  // [6][NY][NXp] floats, rows padded to 16 bytes
    ctx->NXp = (g.NX + 3) / 4 * 4;
    ctx->off_pad = off; off += up((size_t)6 * g.NY * ctx->NXp * 4);
  }
  ctx->load_chunk = ctx->max_cap < ((int64_t)1 << 20) ? ctx->max_cap : ((int64_t)1 << 20);
  ctx->off_stage = off; off += 6 * up((size_t)ctx->load_chunk * 8);
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
  if (ctx->mixed) assign_fields(ctx, ctx->F32);
  else assign_fields(ctx, ctx->F64);
  const size_t tstride = up((size_t)(ctx->g.NX > ctx->g.NY ? ctx->g.NX : ctx->g.NY) * 8);
  ctx->tb.r = at<float>(ctx, ctx->off_ptab);
  ctx->tb.s = at<float>(ctx, ctx->off_ptab + tstride);
  ctx->tb.c = at<float>(ctx, ctx->off_ptab + 2 * tstride);
  ctx->tb.r64 = at<double>(ctx, ctx->off_ptab + 3 * tstride);
  ctx->tb.s64 = at<double>(ctx, ctx->off_ptab + 4 * tstride);
  ctx->tb.c64 = at<double>(ctx, ctx->off_ptab + 5 * tstride);
  ctx->tb.t1 = at<float>(ctx, ctx->off_ptab + 6 * tstride);
  ctx->tb.t2 = at<float>(ctx, ctx->off_ptab + 7 * tstride);
  ctx->tb.t1_64 = at<double>(ctx, ctx->off_ptab + 8 * tstride);
  ctx->tb.t2_64 = at<double>(ctx, ctx->off_ptab + 9 * tstride);
  ctx->tb.th64 = at<double>(ctx, ctx->off_ptab + 10 * tstride);
  ctx->tb.r_df = at<float2>(ctx, ctx->off_ptab + 11 * tstride);
  ctx->tb.s_df = at<float2>(ctx, ctx->off_ptab + 12 * tstride);
  ctx->tb.c_df = at<float2>(ctx, ctx->off_ptab + 13 * tstride);
  ctx->tb.t1_df = at<float2>(ctx, ctx->off_ptab + 14 * tstride);
  ctx->tb.t2_df = at<float2>(ctx, ctx->off_ptab + 15 * tstride);
  if (ctx->cfg.tiled_push == 2) {
    // tensor map of the padded planes [6][NY][NXp] (FP32), box one window plane W1 x W2 x 1;
    // the encoder comes from the driver through the runtime (no link to the driver library)
    void *fn = nullptr;
    cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault,
                                         &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess || !fn)
      return fail(ctx, GRPIC_ECUDA, "cuTensorMapEncodeTiled is not available");
    const auto encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
    const cuuint64_t NXp = (cuuint64_t)ctx->NXp, NY = (cuuint64_t)ctx->g.NY;
    const cuuint64_t dims[3] = {NXp, NY, 6};
    const cuuint64_t strides[2] = {NXp * 4, NXp * NY * 4};
    const cuuint32_t box[3] = {(cuuint32_t)(ctx->cfg.tile_r + 2 * TILE_HALO),
                               (cuuint32_t)(ctx->cfg.tile_theta + 2 * TILE_HALO), 1};
    const cuuint32_t es[3] = {1, 1, 1};
    const CUresult r = encode(&ctx->tmap, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3,
                              at<float>(ctx, ctx->off_pad), dims, strides, box, es,
                              CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                              CU_TENSOR_MAP_L2_PROMOTION_NONE, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return fail(ctx, GRPIC_ECUDA, "tensor map encoding failed (%d)", (int)r);
  }
  if (ctx->mixed) {
    for (int s = 0; s < ctx->cfg.n_species; ++s) {
      SpeciesState &sp = ctx->sp[s];
      const size_t cap = (size_t)(sp.cap > 0 ? sp.cap : 1);
      sp.gl.idx = at<uint32_t>(ctx, sp.off_gl);
      sp.gl.mask = at<uint32_t>(ctx, sp.off_gl + up(cap * 4));
      sp.gl.count = at<unsigned long long>(ctx, sp.off_gl + up(cap * 4) + up((cap + 31) / 32 * 4));
      sp.gl.cap = (int64_t)cap;
      sp.tile_start = at<uint32_t>(ctx, sp.off_tiles);
      sp.tiles_valid = false;
    }
    if (!ctx->side) {  // the guard kernels are the longer chain: higher priority
      int lo = 0, hi = 0;
      CK(cudaDeviceGetStreamPriorityRange(&lo, &hi));
      CK(cudaStreamCreateWithPriority(&ctx->side, cudaStreamNonBlocking, hi));
      for (int s = 0; s < GRPIC_MAX_SPECIES; ++s) {
        CK(cudaEventCreateWithFlags(&ctx->ev_fork[s], cudaEventDisableTiming));
        CK(cudaEventCreateWithFlags(&ctx->ev_done[s], cudaEventDisableTiming));
        CK(cudaEventCreateWithFlags(&ctx->ev_class[s], cudaEventDisableTiming));
      }
    }
  }
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
  if (ctx->mixed) {
    CK(launch_metric_tables<float>(ctx->g, const_cast<float *>(ctx->F32.tab),
                                   const_cast<float *>(ctx->F32.polar), ctx->stream));
  } else {
    CK(launch_metric_tables<double>(ctx->g, const_cast<double *>(ctx->F64.tab),
                                    const_cast<double *>(ctx->F64.polar), ctx->stream));
  }
  CK(launch_push_tables(ctx->g, ctx->tb, ctx->stream));
  CK(launch_inject_tables(ctx->g, reinterpret_cast<unsigned char *>(ctx->arena + ctx->off_inj),
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
  grid_float_copies(ctx->g);
  ctx->metric_ready = true;
  return GRPIC_OK;
}

double grpic_dt(const grpic_ctx *ctx) { return ctx && ctx->metric_ready ? ctx->g.dt : 0.0; }

grpic_status grpic_init_fields(grpic_ctx *ctx, int kind, double B0) {
  grpic_status s = need_bound(ctx);
  if (s) return s;
  if (!ctx->metric_ready) return fail(ctx, GRPIC_ESTATE, "metric not initialised");
  if (kind < GRPIC_FIELD_ZERO || kind > GRPIC_FIELD_MONOPOLE)
    return fail(ctx, GRPIC_EINVAL, "bad field kind");
  if (ctx->mixed) {
    if (kind != GRPIC_FIELD_USER) CK(launch_init_fields<float>(ctx->g, ctx->F32, kind, B0, ctx->stream));
    CK(launch_field_finish_init<float>(ctx->g, ctx->F32, kind == GRPIC_FIELD_USER, ctx->stream));
  } else {
    if (kind != GRPIC_FIELD_USER) CK(launch_init_fields<double>(ctx->g, ctx->F64, kind, B0, ctx->stream));
    CK(launch_field_finish_init<double>(ctx->g, ctx->F64, kind == GRPIC_FIELD_USER, ctx->stream));
  }
  ctx->fields_ready = true;
  ctx->field_b0 = (kind == GRPIC_FIELD_WALD || kind == GRPIC_FIELD_VERTICAL ||
                   kind == GRPIC_FIELD_MONOPOLE) ? B0 : 1.0;
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
  const cudaStream_t st = ctx->stream;
  CK(copy(L.i1, in->i1, n * 4, st));
  CK(copy(L.i2, in->i2, n * 4, st));
  // the FP64 inputs go through a staging region of LOAD_CHUNK particles (host or device
  // sources), then one kernel converts each chunk into the species arrays
  double *stg = at<double>(ctx, ctx->off_stage);
  for (int64_t k0 = 0; k0 < n; k0 += ctx->load_chunk) {
    const int64_t m = n - k0 < ctx->load_chunk ? n - k0 : ctx->load_chunk;
    const double *src[6] = {in->dx1, in->dx2, in->uh1, in->uh2, in->uh3, in->w0};
    for (int a = 0; a < 6; ++a)
      CK(copy(stg + a * ctx->load_chunk, src[a] + k0, (size_t)m * 8, st));
    grpic_particle_init dv = *in;
    dv.dx1 = stg; dv.dx2 = stg + ctx->load_chunk; dv.uh1 = stg + 2 * ctx->load_chunk;
    dv.uh2 = stg + 3 * ctx->load_chunk; dv.uh3 = stg + 4 * ctx->load_chunk;
    dv.w0 = stg + 5 * ctx->load_chunk;
    if (ctx->mixed)
      CK(launch_load<float>(ctx->g, dev_view<float>(sp, sp.live), k0, m, dv, density_power, st));
    else
      CK(launch_load<double>(ctx->g, dev_view<double>(sp, sp.live), k0, m, dv, density_power, st));
  }
  k_set_i64<<<1, 1, 0, st>>>(sp.n_dev, n);
  COUNT_LAUNCH(1);
  CK(cudaGetLastError());
  sp.n_bound = n;
  sp.loaded = true;
  sp.prev_valid = true;
  sp.tiles_valid = false;  // new particles: no tile ranges until the next sort
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
  grpic_particles &L = sp.soa[sp.live];
  const cudaStream_t st = ctx->stream;
  if (n > 0) {
    // i1p, i2p, dx1p, dx2p (the last four arrays) may all be null: the previous position
    // is then the position, copied on the device
    const bool prev = in->i1p || in->i2p || in->dx1p || in->dx2p;
    const int n_in = prev ? NARR : NARR - 4;
    for (int a = 0; a < n_in; ++a) {
      const void *src = cslot(*in, a);
      if (!src) return fail(ctx, GRPIC_EINVAL, "null particle array %d", a);
      CK(copy(*slot(L, a), src, (size_t)n * elem_bytes(ctx, a), st));
    }
    if (!prev) {
      const int from[4] = {0, 1, 2, 3};  // i1, i2, dx1, dx2 -> i1p, i2p, dx1p, dx2p
      for (int q = 0; q < 4; ++q)
        CK(copy(*slot(L, NARR - 4 + q), *slot(L, from[q]), (size_t)n * elem_bytes(ctx, from[q]),
                st));
    }
  }
  k_set_i64<<<1, 1, 0, st>>>(sp.n_dev, n);
  COUNT_LAUNCH(1);
  CK(cudaGetLastError());
  sp.n_bound = n;
  sp.loaded = true;
  sp.prev_valid = true;
  sp.tiles_valid = false;  // new particles: no tile ranges until the next sort
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
  for (int a = 0; a < NARR; ++a) {
    void *dst = *slot(*out, a);
    if (dst) CK(copy(dst, cslot(L, a), (size_t)cnt * elem_bytes(ctx, a), ctx->stream));
  }
  CK(cudaStreamSynchronize(ctx->stream));
  return GRPIC_OK;
}

grpic_status grpic_aux_fields(grpic_ctx *ctx, void *const E[3], void *const H[3]) {
  grpic_status s = need_fields(ctx);
  if (s) return s;
  if (!E || !H) return fail(ctx, GRPIC_EINVAL, "null E or H");
  for (int c = 0; c < 3; ++c)
    if (!E[c] || !H[c]) return fail(ctx, GRPIC_EINVAL, "null plane %d", c);
  const size_t bytes = (size_t)plane_size(ctx->g) * ctx->fsz;
  if (ctx->mixed) {
    CK(launch_aux_fields<float>(ctx->g, ctx->F32, ctx->stream));
    for (int c = 0; c < 3; ++c) {
      CK(copy(E[c], ctx->F32.E[c], bytes, ctx->stream));
      CK(copy(H[c], ctx->F32.H[c], bytes, ctx->stream));
    }
  } else {
    CK(launch_aux_fields<double>(ctx->g, ctx->F64, ctx->stream));
    for (int c = 0; c < 3; ++c) {
      CK(copy(E[c], ctx->F64.E[c], bytes, ctx->stream));
      CK(copy(H[c], ctx->F64.H[c], bytes, ctx->stream));
    }
  }
  CK(cudaStreamSynchronize(ctx->stream));
  return GRPIC_OK;
}

grpic_status grpic_plane_ptr(grpic_ctx *ctx, int plane, void **out) {
  grpic_status s = need_bound(ctx);
  if (s) return s;
  if (plane < 0 || plane >= GRPIC_NPLANES || !out) return fail(ctx, GRPIC_EINVAL, "bad plane %d", plane);
  *out = ctx->mixed ? (void *)plane_of(ctx->F32, plane) : (void *)plane_of(ctx->F64, plane);
  return GRPIC_OK;
}

// the entry points that read the previous positions refuse them when the last push did not
// store them
static grpic_status need_prev(grpic_ctx *ctx, int k) {
  if (ctx->sp[k].loaded && !ctx->sp[k].prev_valid)
    return fail(ctx, GRPIC_ESTATE, "species %d: the last push did not store the previous "
                "positions (grpic_set_keep_prev)", k);
  return GRPIC_OK;
}

grpic_status grpic_invariants(grpic_ctx *ctx, int species, int kind, double B0, double *E,
                              double *L) {
  grpic_status s = need_bound(ctx);
  if (s) return s;
  if ((s = need_species(ctx, species))) return s;
  if ((s = need_prev(ctx, species))) return s;
  if (!ctx->metric_ready) return fail(ctx, GRPIC_ESTATE, "metric not initialised");
  if (!E || !L) return fail(ctx, GRPIC_EINVAL, "null output");
  SpeciesState &sp = ctx->sp[species];
  if (ctx->mixed)
    CK(launch_invariants<float>(ctx->g, dev_view<float>(sp, sp.live), kind, B0, E, L, sp.n_bound,
                                ctx->stream));
  else
    CK(launch_invariants<double>(ctx->g, dev_view<double>(sp, sp.live), kind, B0, E, L,
                                 sp.n_bound, ctx->stream));
  return GRPIC_OK;
}

grpic_status grpic_push(grpic_ctx *ctx, int species) {
  grpic_status s = need_fields(ctx);
  if (s) return s;
  if ((s = need_species(ctx, species))) return s;
  SpeciesState &sp = ctx->sp[species];
  if (!sp.loaded) return fail(ctx, GRPIC_ESTATE, "species %d has no particles", species);
  PhaseTimer t(ctx, PH_PUSH);
  if (ctx->mixed) CK(do_push(ctx, ctx->F32, species, false));
  else CK(do_push(ctx, ctx->F64, species, false));
  CK(join_push(ctx, species));
  ++ctx->push_calls;
  return GRPIC_OK;
}

grpic_status grpic_deposit(grpic_ctx *ctx) {
  grpic_status s = need_fields(ctx);
  if (s) return s;
  for (int k = 0; k < ctx->cfg.n_species; ++k)
    if (!ctx->sp[k].massless && (s = need_prev(ctx, k))) return s;
  PhaseTimer t(ctx, PH_DEPOSIT);
  if (ctx->mixed) CK(do_zero_J(ctx, ctx->F32));
  else CK(do_zero_J(ctx, ctx->F64));
  for (int k = 0; k < ctx->cfg.n_species; ++k) {
    SpeciesState &sp = ctx->sp[k];
    if (!sp.loaded || sp.massless) continue;
    if (ctx->mixed)
      CK(launch_deposit<float>(ctx->g, ctx->F32, dev_view<float>(sp, sp.live), ctx->tb,
                               sp.n_bound, ctx->stream));
    else
      CK(launch_deposit<double>(ctx->g, ctx->F64, dev_view<double>(sp, sp.live), ctx->tb,
                                sp.n_bound, ctx->stream));
  }
  if (ctx->mixed) CK(launch_filter_currents<float>(ctx->g, ctx->F32, ctx->stream));
  else CK(launch_filter_currents<double>(ctx->g, ctx->F64, ctx->stream));
  return GRPIC_OK;
}

grpic_status grpic_field_step(grpic_ctx *ctx, int phase) {
  grpic_status s = need_fields(ctx);
  if (s) return s;
  if (phase == GRPIC_PREDICT) {
    PhaseTimer t(ctx, PH_PREDICT);
    if (ctx->mixed) CK(launch_predict<float>(ctx->g, ctx->F32, ctx->stream));
    else CK(launch_predict<double>(ctx->g, ctx->F64, ctx->stream));
  } else if (phase == GRPIC_ADVANCE) {
    PhaseTimer t(ctx, PH_ADVANCE);
    if (ctx->mixed) {
      CK(launch_advance<float>(ctx->g, ctx->F32, ctx->stream));
      rotate(ctx->F32);
    } else {
      CK(launch_advance<double>(ctx->g, ctx->F64, ctx->stream));
      rotate(ctx->F64);  // em <- (B^{n+1/2}, D^{n+1}), em0 <- (B^{n-1/2}, D^n), cur0 <- J^{n+1/2}
    }
  } else {
    return fail(ctx, GRPIC_EINVAL, "bad phase %d", phase);
  }
  return GRPIC_OK;
}

}  // extern "C"

namespace {
// the cell sort of one species; with_prev false inside grpic_step, whose push of the species
// follows and rewrites the previous positions before anything reads them
grpic_status sort_species(grpic_ctx *ctx, int species, bool with_prev) {
  grpic_status s = need_bound(ctx);
  if (s) return s;
  if ((s = need_species(ctx, species))) return s;
  SpeciesState &sp = ctx->sp[species];
  if (!sp.loaded) return GRPIC_OK;
  PhaseTimer t(ctx, PH_SORT);
  if (ctx->mixed) {
    CK(launch_sort<float>(ctx->g, ctx->cfg.tile_r, ctx->cfg.tile_theta, dev_view<float>(sp, sp.live),
                          dev_view<float>(sp, 1 - sp.live), sp.n_bound, sp.n_dev, ctx->S,
                          sp.tile_start, ctx->stream, with_prev));
    sp.tiles_valid = true;
  } else {
    CK(launch_sort<double>(ctx->g, ctx->cfg.tile_r, ctx->cfg.tile_theta,
                           dev_view<double>(sp, sp.live), dev_view<double>(sp, 1 - sp.live),
                           sp.n_bound, sp.n_dev, ctx->S, nullptr, ctx->stream, with_prev));
  }
  sp.live = 1 - sp.live;
  return GRPIC_OK;
}
}  // namespace

extern "C" {

grpic_status grpic_sort(grpic_ctx *ctx, int species) { return sort_species(ctx, species, true); }

}  // extern "C"

namespace {

// The particle state of grpic_step_host: host arrays per species and the counts they hold.
struct HostIO {
  const grpic_particles *st;
  const int64_t *n_in;
};

int host_chunks(const grpic_ctx *c) { return c->mixed ? 1 : HOST_CHUNKS; }
int64_t chunk_len(int64_t n, int chunks) { return (n + chunks - 1) / chunks; }

// the state arrays of particles [a, b) of species k between host and device
grpic_status host_copy(grpic_ctx *ctx, int k, const HostIO &io, int64_t a, int64_t b, bool in,
                       cudaStream_t st) {
  const grpic_particles &L = ctx->sp[k].soa[ctx->sp[k].live];
  for (int q = 0; q < NARR - 4; ++q) {
    const size_t eb = elem_bytes(ctx, q);
    char *dev = static_cast<char *>(const_cast<void *>(cslot(L, q))) + a * eb;
    char *host = static_cast<char *>(const_cast<void *>(cslot(io.st[k], q))) + a * eb;
    CK(in ? copy(dev, host, (size_t)(b - a) * eb, st) : copy(host, dev, (size_t)(b - a) * eb, st));
  }
  return GRPIC_OK;
}

// FP64 push of particles [a, a + m) of species k, their alive count at n_chunk (device)
cudaError_t push_range(grpic_ctx *c, int k, int64_t a, int64_t m, const int64_t *n_chunk) {
  SpeciesState &sp = c->sp[k];
  SpeciesDevT<double> v = dev_view<double>(sp, sp.live);
  v.i1 += a; v.i2 += a; v.dx1 += a; v.dx2 += a; v.u1 += a; v.u2 += a; v.u3 += a;
  v.phi += a; v.w += a; v.tag += a; v.i1p += a; v.i2p += a; v.dx1p += a; v.dx2p += a;
  v.n = n_chunk;
  const PushStreams ps{c->stream, c->side, c->ev_fork[k], c->ev_done[k], c->ev_class[k],
                       nullptr, nullptr, PUSH_ALL};
  TileInfo ti{};
  ti.tr = c->cfg.tile_r;
  ti.tt = c->cfg.tile_theta;
  return launch_push<double>(c->g, c->F64, v, c->tb, sp.gl, ti, m, !sp.massless, c->diag, ps);
}

// species k of grpic_step_host: range c is pushed once its copies to the device are done and
// goes back to the host arrays on the d2h stream once its push is done (both streams of the
// mixed push). A sort in the step reads the whole species, so it waits for every range; the
// ranges then follow the sorted order, with the alive count of each taken on the device
// (ranges past the count push nothing and bring back stale values the count excludes).
grpic_status host_species(grpic_ctx *ctx, int k, const HostIO &io, bool sort_now) {
  grpic_status s;
  SpeciesState &sp = ctx->sp[k];
  const int C = host_chunks(ctx);
  const int64_t nk = io.n_in[k], len = chunk_len(nk, C);
  if (sort_now)
    for (int c = 0; c < C; ++c) CK(cudaStreamWaitEvent(ctx->stream, ctx->ev_in[k][c], 0));
  k_set_i64<<<1, 1, 0, ctx->stream>>>(sp.n_dev, nk);
  COUNT_LAUNCH(1);
  CK(cudaGetLastError());
  sp.n_bound = nk;
  sp.tiles_valid = false;
  if (sort_now && (s = sort_species(ctx, k, false))) return s;
  int64_t *cn = at<int64_t>(ctx, ctx->off_chunk) + k * HOST_CHUNKS;
  if (C > 1) {
    k_chunk_counts<<<1, 32, 0, ctx->stream>>>(sp.n_dev, cn, len, C);
    COUNT_LAUNCH(1);
    CK(cudaGetLastError());
  }
  for (int c = 0; c < C; ++c) {
    const int64_t a = c * len, b = a + len < nk ? a + len : nk;
    if (b <= a) break;
    CK(cudaStreamWaitEvent(ctx->stream, ctx->ev_in[k][c], 0));
    {
      PhaseTimer t(ctx, PH_PUSH);
      if (ctx->mixed) CK(do_push(ctx, ctx->F32, k, true));
      else if (C == 1) CK(do_push(ctx, ctx->F64, k, true));
      else CK(push_range(ctx, k, a, b - a, cn + c));
      ++ctx->push_calls;
    }
    CK(cudaEventRecord(ctx->ev_pushed[k][c], ctx->stream));
    CK(cudaStreamWaitEvent(ctx->d2h, ctx->ev_pushed[k][c], 0));
    if (ctx->mixed) CK(cudaStreamWaitEvent(ctx->d2h, ctx->ev_done[k], 0));
    if ((s = host_copy(ctx, k, io, a, b, false, ctx->d2h))) return s;
  }
  CK(cudaMemcpyAsync(ctx->host_n + k, sp.n_dev, 8, cudaMemcpyDeviceToHost, ctx->d2h));
  return GRPIC_OK;
}

// the copies of every species' ranges to the device, each range's event after its copies
grpic_status host_in(grpic_ctx *ctx, const HostIO &io) {
  grpic_status s;
  for (int k = 0; k < ctx->cfg.n_species; ++k) {
    if (!ctx->sp[k].loaded) continue;
    const int C = host_chunks(ctx);
    const int64_t nk = io.n_in[k], len = chunk_len(nk, C);
    for (int c = 0; c < C; ++c) {
      const int64_t a = c * len, b = a + len < nk ? a + len : nk;
      if (b > a && (s = host_copy(ctx, k, io, a, b, true, ctx->h2d))) return s;
      CK(cudaEventRecord(ctx->ev_in[k][c], ctx->h2d));
    }
  }
  return GRPIC_OK;
}

// One full PIC step (Sec. 3.4). With io, every species first waits for its state to arrive
// from the host, and is sorted and pushed before the next species is touched, so that the
// copies of one species overlap the work on another.
grpic_status step_once(grpic_ctx *ctx, const HostIO *io) {
  grpic_status s;
  const bool sort_now = ctx->cfg.sort_every > 0 && ctx->step % ctx->cfg.sort_every == 0;
  // mixed, no sort this step: classify every species on the side stream first, beside the
  // field predict (it reads only the particles), so the first FP32 kernel need not wait for it
  const bool early_classify = ctx->mixed && !io && !sort_now;
  if (early_classify)
    for (int k = 0; k < ctx->cfg.n_species; ++k)
      if (ctx->sp[k].loaded) CK(do_push(ctx, ctx->F32, k, true, PUSH_CLASSIFY));
  {
    PhaseTimer t(ctx, PH_PREDICT);
    if (ctx->mixed) CK(launch_predict<float>(ctx->g, ctx->F32, ctx->stream));
    else CK(launch_predict<double>(ctx->g, ctx->F64, ctx->stream));
  }
  if (!io) {
    if (sort_now)
      for (int k = 0; k < ctx->cfg.n_species; ++k)
        if ((s = sort_species(ctx, k, false))) return s;
    PhaseTimer t(ctx, PH_PUSH);  // fused push + deposit of every species
    if (ctx->mixed) CK(do_zero_J(ctx, ctx->F32));
    else CK(do_zero_J(ctx, ctx->F64));
    // mixed: the guard stages of all species first, so that their FP64 kernels (the longer
    // chain, on the side stream) run beside all the FP32 kernels instead of trailing the last
    if (ctx->mixed)
      for (int k = 0; k < ctx->cfg.n_species; ++k)
        if (ctx->sp[k].loaded)
          CK(do_push(ctx, ctx->F32, k, true, early_classify ? PUSH_GUARD_KERNELS : PUSH_GUARD));
    for (int k = 0; k < ctx->cfg.n_species; ++k) {
      SpeciesState &sp = ctx->sp[k];
      if (!sp.loaded) continue;
      if (ctx->mixed) CK(do_push(ctx, ctx->F32, k, true, PUSH_MAIN));
      else CK(do_push(ctx, ctx->F64, k, true));
      ++ctx->push_calls;
    }
    for (int k = 0; k < ctx->cfg.n_species; ++k)
      if (ctx->sp[k].loaded) CK(join_push(ctx, k));
  } else {
    if (ctx->mixed) CK(do_zero_J(ctx, ctx->F32));
    else CK(do_zero_J(ctx, ctx->F64));
    for (int k = 0; k < ctx->cfg.n_species; ++k)
      if (ctx->sp[k].loaded && (s = host_species(ctx, k, *io, sort_now))) return s;
    for (int k = 0; k < ctx->cfg.n_species; ++k)
      if (ctx->sp[k].loaded) CK(join_push(ctx, k));
  }
  if (ctx->g.n_f > 0) {
    PhaseTimer t(ctx, PH_DEPOSIT);  // the current filter, the deposit's last part
    if (ctx->mixed) CK(launch_filter_currents<float>(ctx->g, ctx->F32, ctx->stream));
    else CK(launch_filter_currents<double>(ctx->g, ctx->F64, ctx->stream));
  }
  {
    PhaseTimer t(ctx, PH_ADVANCE);
    if (ctx->mixed) {
      CK(launch_advance<float>(ctx->g, ctx->F32, ctx->stream));
      rotate(ctx->F32);
    } else {
      CK(launch_advance<double>(ctx->g, ctx->F64, ctx->stream));
      rotate(ctx->F64);
    }
  }
  ++ctx->step;
  return GRPIC_OK;
}

}  // namespace

extern "C" {

grpic_status grpic_step(grpic_ctx *ctx, int n_steps) {
  grpic_status s = need_fields(ctx);
  if (s) return s;
  if (n_steps < 0) return fail(ctx, GRPIC_EINVAL, "negative step count");
  for (int n = 0; n < n_steps; ++n)
    if ((s = step_once(ctx, nullptr))) return s;
  return GRPIC_OK;
}

grpic_status grpic_step_host(grpic_ctx *ctx, const grpic_particles *state, int64_t *n) {
  grpic_status s = need_fields(ctx);
  if (s) return s;
  if (!state || !n) return fail(ctx, GRPIC_EINVAL, "null state or counts");
  for (int k = 0; k < ctx->cfg.n_species; ++k) {
    const SpeciesState &sp = ctx->sp[k];
    if (n[k] < 0 || n[k] > sp.cap)
      return fail(ctx, GRPIC_ECAPACITY, "species %d: %lld particles, capacity %lld", k,
                  (long long)n[k], (long long)sp.cap);
    if (n[k] > 0 && !sp.loaded)
      return fail(ctx, GRPIC_ESTATE, "species %d was never loaded or set", k);
    for (int a = 0; a < NARR - 4 && n[k] > 0; ++a)
      if (!cslot(state[k], a)) return fail(ctx, GRPIC_EINVAL, "species %d: null array %d", k, a);
  }
  if (!ctx->h2d) {
    CK(cudaStreamCreateWithFlags(&ctx->h2d, cudaStreamNonBlocking));
    CK(cudaStreamCreateWithFlags(&ctx->d2h, cudaStreamNonBlocking));
    CK(cudaEventCreateWithFlags(&ctx->ev_start, cudaEventDisableTiming));
    for (int k = 0; k < GRPIC_MAX_SPECIES; ++k)
      for (int c = 0; c < HOST_CHUNKS; ++c) {
        CK(cudaEventCreateWithFlags(&ctx->ev_in[k][c], cudaEventDisableTiming));
        CK(cudaEventCreateWithFlags(&ctx->ev_pushed[k][c], cudaEventDisableTiming));
      }
    void *hn = nullptr;
    CK(cudaMallocHost(&hn, GRPIC_MAX_SPECIES * sizeof(int64_t)));
    ctx->host_n = static_cast<int64_t *>(hn);
  }
  // the copies in start after everything issued before on the context's stream
  CK(cudaEventRecord(ctx->ev_start, ctx->stream));
  CK(cudaStreamWaitEvent(ctx->h2d, ctx->ev_start, 0));
  const HostIO io{state, n};
  s = host_in(ctx, io);
  if (!s) s = step_once(ctx, &io);
  // on an error the copies already issued finish before the caller's arrays are released
  const cudaError_t e1 = cudaStreamSynchronize(ctx->d2h), e2 = cudaStreamSynchronize(ctx->h2d);
  if (s) return s;
  CK(e1);
  CK(e2);
  CK(cudaStreamSynchronize(ctx->stream));
  for (int k = 0; k < ctx->cfg.n_species; ++k)
    if (ctx->sp[k].loaded) n[k] = ctx->host_n[k];
  return GRPIC_OK;
}

grpic_status grpic_inject(grpic_ctx *ctx, int species_e, int species_p, double sigma0,
                          double sigma_th, double B0, const double *pool, int64_t pool_n,
                          int64_t pool_offset) {
  grpic_status s = need_fields(ctx);
  if (s) return s;
  if ((s = need_species(ctx, species_e)) || (s = need_species(ctx, species_p))) return s;
  if (species_e == species_p) return fail(ctx, GRPIC_EINVAL, "one species for both members");
  SpeciesState &se = ctx->sp[species_e], &sp = ctx->sp[species_p];
  if (se.massless || sp.massless) return fail(ctx, GRPIC_EINVAL, "massless species");
  if (!pool || pool_n <= 0) return fail(ctx, GRPIC_EINVAL, "empty pool");
  if (!(sigma0 > 0.0) || !(sigma_th > 0.0) || !(B0 != 0.0) || !isfinite(sigma0) ||
      !isfinite(sigma_th) || !isfinite(B0))
    return fail(ctx, GRPIC_EINVAL, "bad sigma0, sigma_th or B0");
  PhaseTimer t(ctx, PH_INJECT);
  unsigned char *scratch = reinterpret_cast<unsigned char *>(ctx->arena + ctx->off_inj);
  if (ctx->mixed)
    CK(launch_inject<float>(ctx->g, ctx->F32, dev_view<float>(se, se.live),
                            dev_view<float>(sp, sp.live), se.loaded ? se.n_bound : 0,
                            sp.loaded ? sp.n_bound : 0, se.cap, sp.cap, sigma0, sigma_th, B0,
                            pool, pool_n, pool_offset, scratch, ctx->diag, ctx->stream));
  else
    CK(launch_inject<double>(ctx->g, ctx->F64, dev_view<double>(se, se.live),
                             dev_view<double>(sp, sp.live), se.loaded ? se.n_bound : 0,
                             sp.loaded ? sp.n_bound : 0, se.cap, sp.cap, sigma0, sigma_th, B0,
                             pool, pool_n, pool_offset, scratch, ctx->diag, ctx->stream));
  // counts stay on the device; the host keeps upper bounds for the launch sizes
  const int64_t nc = (int64_t)ctx->g.n_r * ctx->g.n_th;
  for (SpeciesState *q : {&se, &sp}) {
    const int64_t b = (q->loaded ? q->n_bound : 0) + nc;
    q->n_bound = b < q->cap ? b : q->cap;
    q->loaded = true;
    q->tiles_valid = false;
  }
  return GRPIC_OK;
}

grpic_status grpic_charge_check(grpic_ctx *ctx, int after_step, double out[4]) {
  grpic_status s = need_fields(ctx);
  if (s) return s;
  if (!out) return GRPIC_EINVAL;
  for (int k = 0; k < ctx->cfg.n_species; ++k)
    if (!ctx->sp[k].massless && (s = need_prev(ctx, k))) return s;
  double *dev = at<double>(ctx, ctx->off_rho + 6 * up((size_t)plane_size(ctx->g) * 8));
  if (ctx->mixed) CK(charge_check(ctx, ctx->F32, after_step != 0, dev));
  else CK(charge_check(ctx, ctx->F64, after_step != 0, dev));
  CK(cudaMemcpyAsync(out, dev, 4 * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  return GRPIC_OK;
}

static grpic_status adjoint_args(grpic_ctx *ctx, int64_t n, double b0, int n_steps,
                                 int ckpt_every, int n_iter) {
  grpic_status s = need_fields(ctx);
  if (s) return s;
  if (ctx->mixed) return fail(ctx, GRPIC_ESTATE, "the adjoint needs an FP64 context");
  if (n < 0 || n_steps < 0 || ckpt_every < 1 || n_iter < 1 || n_iter > 1000)
    return fail(ctx, GRPIC_EINVAL, "bad adjoint sizes");
  if (!(ctx->field_b0 != 0.0) || !isfinite(b0))
    return fail(ctx, GRPIC_EINVAL, "field amplitude %g against planes of %g", b0, ctx->field_b0);
  if (ctx->g.qks) return fail(ctx, GRPIC_EINVAL, "the adjoint takes the plain log-r grid (r0 = h0 = 0)");
  return GRPIC_OK;
}

grpic_status grpic_adjoint_forward(grpic_ctx *ctx, int64_t n, double qm, double b0, int n_steps,
                                   int ckpt_every, int n_iter, const double *state0,
                                   double *state_out, double *ckpt) {
  grpic_status s = adjoint_args(ctx, n, b0, n_steps, ckpt_every, n_iter);
  if (s) return s;
  if (n > 0 && (!state0 || !state_out || (n_steps > 0 && !ckpt)))
    return fail(ctx, GRPIC_EINVAL, "null adjoint buffer");
  CK(launch_adjoint_forward(ctx->g, ctx->F64, n, qm, b0 / ctx->field_b0, n_steps, ckpt_every,
                            n_iter, state0, state_out, ckpt, ctx->stream));
  return GRPIC_OK;
}

grpic_status grpic_adjoint_backward(grpic_ctx *ctx, int64_t n, double qm, double b0, int n_steps,
                                    int ckpt_every, int n_iter, const double *ckpt,
                                    const double *grad_out, double *grad_state0,
                                    double *grad_b0_pp, double *grad_b0, double *scratch) {
  grpic_status s = adjoint_args(ctx, n, b0, n_steps, ckpt_every, n_iter);
  if (s) return s;
  if (!grad_b0 || (n > 0 && (!grad_out || !grad_state0 || !grad_b0_pp ||
                             (n_steps > 0 && (!ckpt || !scratch)))))
    return fail(ctx, GRPIC_EINVAL, "null adjoint buffer");
  // the kernels differentiate with respect to the field scale b0 / field_b0
  CK(launch_adjoint_backward(ctx->g, ctx->F64, n, qm, b0 / ctx->field_b0, 1.0 / ctx->field_b0,
                             n_steps, ckpt_every, n_iter, ckpt, grad_out, grad_state0,
                             grad_b0_pp, grad_b0, scratch, ctx->stream));
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
  out->injected = (int64_t)h[DG_INJECTED];
  out->inject_dropped = (int64_t)h[DG_INJECT_DROPPED];
  out->stage_timeouts = (int64_t)h[DG_STAGE_TIMEOUT];
  return GRPIC_OK;
}

grpic_status grpic_set_keep_prev(grpic_ctx *ctx, int keep) {
  if (!ctx) return GRPIC_EINVAL;
  ctx->keep_prev = keep != 0;
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
  out->kernel_ms = ms[PH_KERNEL];
  out->inject_ms = ms[PH_INJECT];
  out->push_calls = ctx->push_calls;
  out->launches = grpic_launches;
  ctx->push_calls = 0;
  grpic_launches = 0;
  return GRPIC_OK;
}

const char *grpic_last_error(const grpic_ctx *ctx) { return ctx ? ctx->err : "null context"; }

size_t grpic_config_bytes(void) { return sizeof(grpic_config); }

void grpic_destroy(grpic_ctx *ctx) {
  if (!ctx) return;
  if (ctx->h2d) {
    cudaStreamSynchronize(ctx->h2d);
    cudaStreamSynchronize(ctx->d2h);
    cudaStreamDestroy(ctx->h2d);
    cudaStreamDestroy(ctx->d2h);
    cudaEventDestroy(ctx->ev_start);
    for (int k = 0; k < GRPIC_MAX_SPECIES; ++k)
      for (int c = 0; c < HOST_CHUNKS; ++c) {
        cudaEventDestroy(ctx->ev_in[k][c]);
        cudaEventDestroy(ctx->ev_pushed[k][c]);
      }
    cudaFreeHost(ctx->host_n);
  }
  for (int ph = 0; ph < PH_N; ++ph)
    for (auto &e : ctx->ev[ph]) {
      cudaEventDestroy(e.first);
      cudaEventDestroy(e.second);
    }
  if (ctx->side) {
    cudaStreamSynchronize(ctx->side);
    cudaStreamDestroy(ctx->side);
    for (int s = 0; s < GRPIC_MAX_SPECIES; ++s) {
      cudaEventDestroy(ctx->ev_fork[s]);
      cudaEventDestroy(ctx->ev_done[s]);
      cudaEventDestroy(ctx->ev_class[s]);
    }
  }
  delete ctx;
}

}  // extern "C"
