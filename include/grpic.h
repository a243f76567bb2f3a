/*
 * grpic.h -- C ABI of the GB300 (sm_103a) library for the per-step hot path of
 * the 2D-axisymmetric general-relativistic particle-in-cell method of
 * arXiv:2511.17701 (Entity, GR module): GR pusher -> charge-conserving current
 * deposit -> GR Maxwell update of D and B through the auxiliary E and H.
 *
 * Conventions common to every entry point
 *  - Errors are returned as grpic_status; grpic_last_error() gives a one-line
 *    message. Nothing traps, aborts or throws.
 *  - All work is queued on the stream given to grpic_bind() and is asynchronous,
 *    except where an entry point says it synchronises.
 *  - Device memory: the library allocates none. The caller allocates one arena of
 *    grpic_arena_bytes() bytes (any allocator: cudaMalloc, a torch tensor, ...),
 *    passes it to grpic_bind() and keeps it alive until grpic_destroy(). The
 *    library carves every table, field plane, particle array and scratch buffer
 *    out of it. Host memory for the context itself comes from malloc.
 *  - A context is not thread safe; use one per host thread and stream.
 *  - Calling an entry point before its prerequisites (bind, init_metric,
 *    init_fields, particles) returns GRPIC_ESTATE.
 *
 * Field storage (same convention as the CPU oracle, so planes compare element by
 * element): every plane is a row-major [NY][NX] array of doubles,
 * NX = n_r + 2*GRPIC_GHOSTS + 1, NY = n_theta + 2*GRPIC_GHOSTS + 1; the grid
 * point x1 = i or i+1/2, x2 = j or j+1/2 is stored at [j + G][i + G] (a half
 * integer position is stored at its lower integer). Yee locations (Fig. 1 of the
 * paper): B^1 (i, j+1/2), B^2 (i+1/2, j), B^3 (i+1/2, j+1/2), D^1 (i+1/2, j),
 * D^2 (i, j+1/2), D^3 (i, j); currents as D.
 */
#ifndef GRPIC_H
#define GRPIC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#if defined(__GNUC__)
#define GRPIC_API __attribute__((visibility("default")))
#else
#define GRPIC_API
#endif

#define GRPIC_GHOSTS 2
#define GRPIC_MAX_SPECIES 8

typedef struct grpic_ctx grpic_ctx;

typedef enum {
  GRPIC_OK = 0,
  GRPIC_EINVAL = 1,      /* bad argument or configuration                       */
  GRPIC_ENOMEM = 2,      /* arena smaller than grpic_arena_bytes()              */
  GRPIC_ECUDA = 3,       /* a CUDA call failed (message in grpic_last_error)    */
  GRPIC_ESTATE = 4,      /* prerequisites missing                               */
  GRPIC_ECAPACITY = 5,   /* more particles than the species capacity           */
  GRPIC_ENONFINITE = 6   /* non-finite particle state was found (diagnostics)   */
} grpic_status;

typedef enum { GRPIC_METRIC_KS0 = 0, GRPIC_METRIC_KS = 1 } grpic_metric_kind;
typedef enum {
  GRPIC_FP64 = 0,  /* FP64 state, fields and arithmetic                                  */
  GRPIC_MIXED = 1  /* FP32 fields, momenta, offsets and currents (int32 cells); FP32
                      arithmetic, with the metric, lapse and shift evaluated in FP64 for
                      particles within fp64_guard_cells of the horizon or an axis, and
                      the whole push in FP64 for particles in the cell rows on the axes */
} grpic_precision;
typedef enum {
  GRPIC_FIELD_ZERO = 0,     /* all fields zero                                    */
  GRPIC_FIELD_WALD = 1,     /* Wald vacuum field, Eq. (Wald), Sec. 4.1.2          */
  GRPIC_FIELD_VERTICAL = 2, /* its zero-spin limit, A_phi = B0 r^2 sin^2(theta)/2 */
  GRPIC_FIELD_USER = 3,     /* caller wrote em (B, D); the library derives the rest */
  GRPIC_FIELD_MONOPOLE = 4  /* magnetic monopole of the BZ test, A_phi = -B0 cos(theta),
                               B^r = B0 sin(theta)/sqrt(h), Sec. 4.5                 */
} grpic_field_kind;
typedef enum { GRPIC_PREDICT = 0, GRPIC_ADVANCE = 1 } grpic_field_phase;

/* field planes, in the order of the CPU oracle's planes */
typedef enum {
  GRPIC_B1 = 0, GRPIC_B2, GRPIC_B3, GRPIC_D1, GRPIC_D2, GRPIC_D3,        /* em  : B^{n-1/2}, D^n     */
  GRPIC_B01, GRPIC_B02, GRPIC_B03, GRPIC_D01, GRPIC_D02, GRPIC_D03,      /* em0 : B^{n-3/2}, D^{n-1} */
  GRPIC_J1, GRPIC_J2, GRPIC_J3,                                          /* cur : J^{n+1/2}          */
  GRPIC_J01, GRPIC_J02, GRPIC_J03,                                       /* cur0: J^{n-1/2}          */
  GRPIC_BN1, GRPIC_BN2, GRPIC_BN3,                                       /* B^n from PREDICT         */
  GRPIC_BI1, GRPIC_BI2, GRPIC_BI3, GRPIC_DI1, GRPIC_DI2, GRPIC_DI3,      /* initial field            */
  GRPIC_NPLANES
} grpic_plane;

/* Everything the paper makes a parameter of the step. */
typedef struct {
  int metric;          /* grpic_metric_kind: kerr_schild_0 (flat) or Kerr-Schild, App. A   */
  double a;            /* black-hole spin, 0 <= a < 1 (ignored for KS0)                     */
  int n_r, n_theta;    /* cells along x1 (radial) and x2 (polar), Sec. 3                    */
  double r_min, r_max; /* x1 in [0, n_r] maps to r = r0 + (r_min - r0) exp(x1 dxi), dxi =
                          ln((r_max - r0)/(r_min - r0))/n_r (quasi-spherical map of App. A;
                          r0, h0 below); x2 in [0, n_theta] maps to eta = x2 pi / n_theta and
                          theta(eta) (theta = eta when h0 = 0)                                */
  double cfl;          /* used when dt <= 0: dt = cfl * min over cells of
                          1 / (alpha sqrt(h^11 + h^22) + |beta^1|)                           */
  double dt;           /* time step; > 0 overrides cfl                                       */
  int n_iter;          /* fixed iteration count of both implicit geodesic pushes, Sec. 3.1   */
  double small_angle;  /* SMALL_ANGLE_GR, Sec. 3.3.2 (1e-5)                                  */
  int n_filter;        /* n_f, Sec. 3.2 and 3.3.3: the deposit is followed by n_f passes of the
                          current filter (binomial (1 2 1) x (1 2 1)/16 on the grid extended
                          across the axes by mirror images: J^1, J^3 even, J^2 odd, axis nodes
                          holding half cells), and the fields in cells i1 <= n_f copy cell
                          n_f + 1. 0 .. 64; with the Kerr metric the grid must start at least
                          n_f + 1 cells inside the horizon, r(x1 = n_f + 1) <= r_h (else
                          GRPIC_EINVAL)                                                        */
  double r_absorb;     /* absorbing (MATCH) layer for r > r_absorb, Sec. 3.3.3               */
  double absorb_coef;  /* its strength                                                       */
  int n_species;       /* 1 .. GRPIC_MAX_SPECIES                                             */
  int64_t capacity[GRPIC_MAX_SPECIES]; /* particles per species the arena holds              */
  int sort_every;      /* grpic_step sorts particles by cell every k steps (0: never)        */
  int tile_r, tile_theta; /* sort tile, in cells: 1 .. 65536, with the tile-padded cell count
                             ceil(n_r/tile_r) ceil(n_theta/tile_theta) tile_r tile_theta at most
                             2^31 - 1 (else GRPIC_EINVAL)                                      */
  int precision;       /* grpic_precision                                                     */
  int full_iterations; /* 0: the implicit pushes stop once an iterate repeats bit for bit (every
                          later iteration would return the same bits, so the result equals the
                          n_iter result exactly), except in GRPIC_MIXED: its FP32 iterations
                          stop once the update is within 2^-22 max(1, |value|), the FP64
                          iterations of its axis rows (stored in FP32) within 2^-26 max(1,
                          |value|) (the remaining error, a fraction rho / (1 - rho) of that,
                          is below the rounding of the stored values); 1: always run n_iter
                          iterations                                                         */
  int fp64_guard_cells; /* GRPIC_MIXED: cells from the horizon and from each axis where the
                           metric is evaluated in FP64 (default 4 when 0)                     */
  int tiled_push;       /* GRPIC_MIXED: 1 = after a sort, push each sort tile in one CTA with
                           the fields of the tile and a 6-cell halo staged in shared memory and
                           the currents accumulated there (the window loaded by the CTA's
                           threads); 2 = the same with the window loaded by the tensor memory
                           accelerator (one thread issues one bulk tensor copy per field plane
                           from a copy of the planes with rows padded to 16 bytes, made before
                           each push; needs tile_r a multiple of 4, else GRPIC_EINVAL);
                           0 (default) = one thread per particle over the whole species with
                           gathers through L1/L2, which measures faster on GB300 for this
                           pusher                                                             */
  double iter_tol;      /* the implicit pushes (steps 6 and 10 of Sec. 3.1): 0 (default) = the
                           stop rule of full_iterations; > 0 = an FP32 predictor iterates each
                           to an exact FP32 repeat and gives the map's Jacobian there; one FP64
                           evaluation at that point, one Newton step, then FP64 iterations
                           until the update is at most iter_tol max(1, |value|) (at most n_iter
                           evaluations in all): the FP64 fixed point to about rho iter_tol
                           (rho < 1 the contraction of the iteration), in fewer FP64
                           operations. Must be below 1e-6                                      */
  double r0, h0;        /* quasi-spherical Kerr-Schild grid (App. A): r = r0 + exp(xi), xi
                           uniform in x1 (r0 < r_min); theta = eta + 2 h0 eta (pi - 2 eta)
                           (pi - eta) / pi^2, eta uniform in x2 (-1/2 < h0 < 1; h0 > 0 puts
                           cells toward the equator). 0, 0: the plain log-r grid with uniform
                           theta. The adjoint entry points need 0, 0                          */
  int massless[GRPIC_MAX_SPECIES]; /* 1: a species of massless particles (photons): gamma =
                           sqrt(h^ij u_i u_j) (Sec. 2.3), no field interpolation and no EM
                           push (Sec. 3.1), only the two geodesic substeps and phi; they are
                           neutral, so the deposit, the charge check and grpic_deposit skip
                           them. 0: massive (gamma = sqrt(1 + h^ij u_i u_j)). Other values:
                           GRPIC_EINVAL                                                        */
} grpic_config;

/* Pointers to one species' particle arrays (SoA, length >= n). Positions are a cell
 * index plus an offset in [0, 1] (Sec. 3: i1, dx1, i2, dx2); u are covariant code-unit
 * momenta u_i; phi the out-of-plane angle (Eq. discretized-geodesic-x-phi); w the
 * weight; tag 1 alive, 2 left the domain in the last push (its move is still
 * deposited), 0 dead. i1p..dx2p is the previous position (Sec. 3.2). The floating
 * arrays (dx1, dx2, u1, u2, u3, phi, w, dx1p, dx2p) hold double for GRPIC_FP64 and
 * float for GRPIC_MIXED. */
typedef struct {
  int32_t *i1, *i2;
  void *dx1, *dx2, *u1, *u2, *u3, *phi, *w;
  uint8_t *tag;
  int32_t *i1p, *i2p;
  void *dx1p, *dx2p;
} grpic_particles;

/* Initial particles for grpic_load_particles: position, momentum in the local
 * orthonormal FIDO tetrad frame (App. A) and a base weight. */
typedef struct {
  const int32_t *i1, *i2;
  const double *dx1, *dx2;
  const double *uh1, *uh2, *uh3;
  const double *w0;
} grpic_particle_init;

typedef struct {
  int64_t left_inner;    /* particles removed through the horizon layer            */
  int64_t left_outer;    /* particles removed through r = r_max                     */
  int64_t reflections;   /* axis reflections, Sec. 3.3.3                           */
  int64_t nonfinite;     /* particles dropped for non-finite or runaway state       */
  int64_t alive[GRPIC_MAX_SPECIES];
  int64_t injected;      /* pairs added by grpic_inject                             */
  int64_t inject_dropped; /* pairs grpic_inject found no room for                   */
  int64_t stage_timeouts; /* tile windows whose tensor copies did not complete within the
                             kernel's bounded wait (tiled_push = 2; the tile's particles were
                             left unpushed); 0 in a healthy run                            */
} grpic_diag;

/* --- set-up ----------------------------------------------------------------------- */

/* Validates cfg (the problem parameters of Secs. 3.1-3.4 and App. A: spin, grid map, time
 * step rule, iterations, boundaries; see grpic_config) and creates a host context (no CUDA
 * work). *out owns host memory only; release it with grpic_destroy. Errors: GRPIC_EINVAL
 * (bad sizes, spin, radii, species counts). */
GRPIC_API grpic_status grpic_create(const grpic_config *cfg, grpic_ctx **out);

/* Bytes of device memory the context needs (256-byte aligned sub-buffers): field planes,
 * metric tables, particle arrays (two copies for the sort), scratch. Memory management,
 * with no counterpart in the paper. No CUDA work; 0 for a null context. */
GRPIC_API size_t grpic_arena_bytes(const grpic_ctx *ctx);

/* (Memory and stream management, no counterpart in the paper.)
 * Binds the caller-owned device arena (>= grpic_arena_bytes, 256-byte aligned)
 * and the CUDA stream (cudaStream_t, NULL = legacy default) on the current device.
 * With GRPIC_MIXED the first bind also creates one internal stream and event pairs
 * (no device memory): the push forks the FP64 guard-zone kernels onto it and joins
 * them back to the bound stream before returning, so callers see one stream.
 * Errors: GRPIC_ENOMEM (too small), GRPIC_EINVAL (misaligned), GRPIC_ECUDA. */
GRPIC_API grpic_status grpic_bind(grpic_ctx *ctx, void *arena, size_t bytes, void *stream);

/* Tabulates the code-unit metric of App. A (alpha, h_ij, sqrt(h), sqrt(h~),
 * [sqrt(h~) h_13], [sqrt(h~ h) beta^1], 1/sqrt(h)) at the four Yee point classes, the
 * polar areas of Sec. 3.3.2 and the FP64 cell-centre metric of grpic_inject, and fixes dt
 * (cfl rule when cfg.dt <= 0).
 * Synchronises the stream once (dt is read back). */
GRPIC_API grpic_status grpic_init_metric(grpic_ctx *ctx);

/* The time step in use after grpic_init_metric (0 before): cfg.dt, or cfl times the
 * smallest light-crossing time of a cell, min over cell centres of 1 / (alpha sqrt(h^11 +
 * h^22) + |beta^1|) in code units (Sec. 3 fixes the time step of the leap-frog scheme but
 * gives no rule for it: this Courant rule is a reading). No CUDA work. */
GRPIC_API double grpic_dt(const grpic_ctx *ctx);

/* Initial fields (Sec. 4.1.2, 4.2): B^1, B^2 from the discrete curl of A_3 at the nodes,
 * B^3 from the discrete curl of A_1; D at each Yee point from the inverse of Eq. (aux)
 * with E_i = d_i A_0. Then em0 = em (stationary start), cur0 = 0, and the initial field
 * is kept as the absorbing-layer target. kind GRPIC_FIELD_USER keeps em as written by
 * the caller and only does the copies and boundary fills. */
GRPIC_API grpic_status grpic_init_fields(grpic_ctx *ctx, int kind, double B0);

/* --- particles -------------------------------------------------------------------- */

/* Loads n particles of a species from positions and tetrad-frame momenta: u_i =
 * e_i^j u_j^ (App. A) at the particle, w = w0 r^{-density_power} sqrt(h)(x_p),
 * phi = 0, tag = 1, previous position = position. qm is the Lorentz coefficient
 * (q/m) per unit stored field; qc the deposit coefficient (sign of q included).
 * Pointers may be host or device memory (copied with cudaMemcpyDefault).
 * Errors: GRPIC_ECAPACITY when n > capacity. */
GRPIC_API grpic_status grpic_load_particles(grpic_ctx *ctx, int species, int64_t n, double qm, double qc,
                                  double density_power, const grpic_particle_init *in);

/* Sets the full state of a species (every array of grpic_particles), host or device
 * pointers. Used for restarts and to feed identical states to parity checks. The four
 * previous-position arrays (i1p, i2p, dx1p, dx2p) may all be null: the previous position is
 * then set to the position on the device (the push writes it anyway, Sec. 3.2); either all
 * four or none. Errors: GRPIC_ECAPACITY (n > capacity), GRPIC_EINVAL (a null array among the
 * first ten, or some but not all of the last four). */
GRPIC_API grpic_status grpic_set_particles(grpic_ctx *ctx, int species, int64_t n, double qm, double qc,
                                 const grpic_particles *in);

/* Copies a species' state out into caller arrays (host or device; null array pointers
 * are skipped), in the layout of grpic_particles, and its count into *n. State I/O, with no
 * counterpart in the paper. Synchronises the stream. Errors: GRPIC_ESTATE (not bound),
 * GRPIC_EINVAL (species out of range). */
GRPIC_API grpic_status grpic_get_particles(grpic_ctx *ctx, int species, grpic_particles *out,
                                 int64_t *n);

/* Device pointers of a species' arrays inside the arena (valid until the next sort, which
 * moves the species to the other copy) and its live count (synchronises when n is given).
 * No counterpart in the paper. Errors: GRPIC_ESTATE (not bound), GRPIC_EINVAL (species). */
GRPIC_API grpic_status grpic_species_arrays(grpic_ctx *ctx, int species, grpic_particles *out,
                                  int64_t *n);

/* The auxiliary fields of Sec. 2 (Eqs. discretized-auxE and discretized-auxH: E_i =
 * alpha h_ij D^j + ... and H_i = alpha h_ij B^j - ..., with the spatial averages of those
 * equations) of the em planes as they stand (B^{n+1/2}, D^{n+1} after a step), copied into
 * E[c], H[c] (c = 0, 1, 2: the x1, x2, x3 covariant components), each a full plane in the
 * plane layout of grpic_plane_ptr, host or device memory; the values are defined on the
 * stored columns -1 .. n_r + 1 and rows 0 .. n_theta (the half-row components on rows
 * 0 .. n_theta - 1), the rest of each plane is scratch. For diagnostics such as the
 * field-line angular velocity and the Poynting flux of Sec. 4.5; synchronises. Errors:
 * GRPIC_ESTATE (fields not initialised), GRPIC_EINVAL (a null pointer). */
GRPIC_API grpic_status grpic_aux_fields(grpic_ctx *ctx, void *const E[3], void *const H[3]);

/* Device pointer of a field plane inside the arena (valid until the next ADVANCE,
 * which rotates em/em0 and cur/cur0); elements are double (GRPIC_FP64) or float
 * (GRPIC_MIXED). The planes are the state of the loop of Sec. 3.4 (em, em0, cur, cur0,
 * B^n) and the initial field the absorbing layer relaxes to (Sec. 3.3.3), GRPIC_NPLANES in
 * all, each [n_theta + 5][n_r + 5] with 2 ghost cells per side. Errors: GRPIC_ESTATE (not
 * bound), GRPIC_EINVAL (plane out of range, null out). */
GRPIC_API grpic_status grpic_plane_ptr(grpic_ctx *ctx, int plane, void **out);

/* Conserved energy and angular momentum per unit mass of each particle of a species
 * (Sec. 2.3): E = -u_0 - (q/m) A_0, L = u_3 + (q/m) A_3 with u_0 = -alpha gamma + beta^1 u_1,
 * A of the stationary field `kind` (GRPIC_FIELD_WALD, _VERTICAL or _MONOPOLE, amplitude B0;
 * ZERO gives the geodesic values), evaluated in FP64 at the midpoint of the previous and current
 * positions (the velocity time level, as Sec. 4.1 does). E and L are device arrays of at
 * least the species' count. */
GRPIC_API grpic_status grpic_invariants(grpic_ctx *ctx, int species, int kind, double B0,
                                        double *E, double *L);

/* --- the hot path ---------------------------------------------------------------- */

/* One particle push of a species, steps 1-11 of Sec. 3.1 with the boundaries of
 * Sec. 3.3.3: saves x^n as the previous position, interpolates B^n (BN planes) and D^n,
 * Boris in the tetrad frame for dt/2, implicit geodesic momentum push (Eq.
 * discretized-geodesic-u), Boris for dt/2, implicit coordinate push (Eq.
 * discretized-geodesic-x), axis reflection, removal, phi update. */
GRPIC_API grpic_status grpic_push(grpic_ctx *ctx, int species);

/* Conformal current deposit of all species from previous and new positions, Sec. 3.2,
 * Eq. (charge-conservation-disc): zeroes J, then deposits J^{n+1/2} and applies the n_f
 * current-filter passes (config n_filter). */
GRPIC_API grpic_status grpic_deposit(grpic_ctx *ctx);

/* GRPIC_PREDICT: loop step 2 of Sec. 3.4 (B^{n-1}, D^{n-1/2}, E^{n-1/2}, auxiliary
 * Faraday B^{n-1} -> B^n into the BN planes). GRPIC_ADVANCE: loop steps 5-8 (J^n, E^n,
 * H^n, Faraday B^{n-1/2} -> B^{n+1/2}, auxiliary Ampere D^{n-1/2} -> D^{n+1/2},
 * H^{n+1/2}, Ampere D^n -> D^{n+1}, boundaries, rotation of em0/em and cur0/cur). */
GRPIC_API grpic_status grpic_field_step(grpic_ctx *ctx, int phase);

/* Stable sort of a species by tile-major cell key; particles not alive go last and
 * are dropped (the count shrinks). Integer work: the permutation is unique. The paper has
 * no sort; it keeps the particles of a cell together for the gathers and the deposit.
 * Errors: GRPIC_ESTATE (not bound), GRPIC_EINVAL (species out of range). */
GRPIC_API grpic_status grpic_sort(grpic_ctx *ctx, int species);

/* n_steps full PIC steps (Sec. 3.4): PREDICT, sort every cfg.sort_every steps, fused
 * push + deposit of all species, ADVANCE. */
GRPIC_API grpic_status grpic_step(grpic_ctx *ctx, int n_steps);

/* One full PIC step (Sec. 3.4, as grpic_step with n_steps = 1) with the particle state
 * streamed through host memory; the paper has no counterpart to the streaming. state[k]
 * (k < n_species) holds host arrays i1, i2, dx1, dx2, u1, u2, u3, phi, w, tag in the
 * context's precision (as in grpic_set_particles; i1p .. dx2p are not used), n[k] the
 * particles they hold. Species k's arrays go to the device on a copy stream, and the step
 * waits for them only before it sorts or pushes that species; its state comes back into
 * the same arrays on a second copy stream as soon as its push is done, so the copies of
 * one species overlap the work on another. An FP64 context streams each species as four
 * particle ranges, each pushed once its copies are in and copied back once pushed (a sort
 * in the step waits for all four). Returns when all is done, with n[k] = the count
 * after the step (a sort in the step drops the particles that left); the arrays hold n[k]
 * elements on entry and at most that many are written. Page-locked host memory lets the
 * copies run asynchronously (pageable memory works, serialised). Each species with
 * n[k] > 0 must have been loaded or set before: its q/m and deposit coefficient are kept.
 * Errors: GRPIC_ESTATE (fields not initialised, a species never loaded), GRPIC_ECAPACITY
 * (n[k] > capacity), GRPIC_EINVAL (null state, counts or array). */
GRPIC_API grpic_status grpic_step_host(grpic_ctx *ctx, const grpic_particles *state,
                                       int64_t *n);

/* --- allocation-free sort ------------------------------------------------------- */

/* Largest particle count grpic_sort_permutation_noalloc accepts. */
#define GRPIC_NOALLOC_SORT_MAX (1 << 20)

/* The paper has no counterpart to this entry point. It computes the same stable
 * tile-major cell order as grpic_sort, but needs neither a context nor an arena: it is
 * for callers that may not allocate device memory at all and cannot hand over scratch
 * space either -- for example a host program whose memory manager owns every byte of the
 * GPU through its own pool, or a time-critical loop that must not pay for the device-wide
 * synchronisation a cudaMalloc can cause. The caller passes device arrays i1, i2, tag of
 * n particles (as in grpic_particles, cells in [0, n_r) x [0, n_theta)) and receives on the
 * device perm[k] = input index of the k-th particle in the sorted order (alive particles,
 * tag 1, first and in key order, ties in input order; then the others in input order) and
 * *n_alive, the number of alive particles. Work is queued on `stream` (cudaStream_t).
 * Scratch lives in one file-scope device array of about 16.3 MiB, sized for
 * GRPIC_NOALLOC_SORT_MAX particles, that every GPU using this entry point holds until the
 * process exits. The first call on a device looks up that array's device address
 * (cudaGetSymbolAddress); make that first call before any stream capture. All calls on a
 * device share the array, so calls whose work overlaps on the GPU (other streams, other
 * host threads) race; serialise them. The entry point calls no cudaMalloc or cudaFree.
 * Errors: GRPIC_ECAPACITY when n > GRPIC_NOALLOC_SORT_MAX; GRPIC_EINVAL for sizes below 1,
 * n_r, n_theta, tile_r or tile_theta above 65536, a tile-padded cell count
 * ceil(n_r/tile_r) ceil(n_theta/tile_theta) tile_r tile_theta above 2^31 - 1 (the keys would
 * reach the key of dead particles), or null pointers; GRPIC_ECUDA when a CUDA call of this
 * entry point fails. A CUDA error already pending on the calling thread when the call starts
 * (cudaPeekAtLastError) is not cleared: the call returns GRPIC_ECUDA at once, queues nothing
 * and leaves that error for its owner to read. n = 0 queues one kernel that sets *n_alive
 * to 0. */
GRPIC_API grpic_status grpic_sort_permutation_noalloc(int n_r, int n_theta, int tile_r,
                                                      int tile_theta, const int32_t *i1,
                                                      const int32_t *i2, const uint8_t *tag,
                                                      int64_t n, uint32_t *perm,
                                                      int64_t *n_alive, void *stream);

/* --- exact sums --------------------------------------------------------------------- */

/* Bins of an exact, order-independent sum of doubles (2 int64 per bin). */
#define GRPIC_SUM_BINS 2048

/* No counterpart in the paper: the adjoint's gradient with respect to the field amplitude is
 * a sum over particles, and these two calls make that sum the same bits however the
 * particles are split between calls, streams or GPUs. A finite double v equals
 * M 2^(b - 1075), b its biased exponent field (1 for subnormals, which have no implicit
 * bit) and M a signed integer, |M| < 2^53. bins: 2 x GRPIC_SUM_BINS int64, element 2b the sum
 * of M >> 32 (arithmetic shift) and element 2b + 1 the sum of M & 0xffffffff over the values
 * of exponent b. Being integer sums, bins can be added element by element (an int64
 * all-reduce across processes) without changing the result. Capacity: at most 2^31 values
 * in all per set of bins.
 *
 * grpic_sum_bins_add adds the finite values of the device array x[0 .. n) (NaN and inf are
 * skipped) into the device bins (the caller zeroes them first) with one kernel on `stream`
 * (cudaStream_t). Allocates nothing. Errors: GRPIC_EINVAL (n < 0, null bins, null x with
 * n > 0), GRPIC_ECUDA (a CUDA error pending before the call, left in place, or a failed
 * launch).
 *
 * grpic_sum_bins_value rounds the binned total, read from HOST memory, to the nearest double
 * (ties to even) in *out: the correctly rounded sum of every value added. Host code only, no
 * CUDA call. Errors: GRPIC_EINVAL (null pointers, bins beyond the capacity). */
GRPIC_API grpic_status grpic_sum_bins_add(const double *x, int64_t n, int64_t *bins,
                                          void *stream);
GRPIC_API grpic_status grpic_sum_bins_value(const int64_t *bins, double *out);

/* --- pair injection ----------------------------------------------------------------- */

/* Pair injection of the BZ monopole test (Sec. 4.5: plasma is injected wherever the local
 * magnetization exceeds sigma_th). Per cell (i1 in [0, n_r), i2 in [0, n_theta)): B at the
 * cell centre from the em planes (B^1, B^2 averaged over the two faces, B^3 as stored),
 * B_i B^i = h_ij B^i B^j with h at the centre, n = (sum of |w| of the live particles of both
 * species in the cell) / sqrt(h) at the centre, sigma = sigma0 (B_i B^i / B0^2) / n. Where
 * sigma > sigma_th one pair is added at one point of the cell: a particle of species_e and
 * one of species_p, co-located, each of weight dn sqrt(h_centre) / 2 with dn the density
 * that brings sigma to sigma_th. pool: device-accessible FP64 [pool_n][8] random draws per
 * pair (dx1, dx2 in [0, 1); the tetrad-frame momenta u^ of the species_e and species_p
 * particle), used cyclically in cell order (i1 fastest) from a cursor the library keeps:
 * pool_offset >= 0 sets the cursor first, < 0 continues. The k-th pair goes to slot
 * n + k of both species (n each species' count before the call): where the room of either
 * species runs out, the remaining pairs are dropped and counted (grpic_diag). Counts stay
 * on the device; no synchronisation. The new particles are unsorted (the next sort orders
 * them). Errors: GRPIC_EINVAL (same or massless species, null pool, pool_n <= 0, sigma0 or
 * sigma_th <= 0, B0 = 0), GRPIC_ESTATE (fields not initialised). */
GRPIC_API grpic_status grpic_inject(grpic_ctx *ctx, int species_e, int species_p, double sigma0,
                                    double sigma_th, double B0, const double *pool,
                                    int64_t pool_n, int64_t pool_offset);

/* --- charge conservation ------------------------------------------------------------ */

/* The discrete continuity equation of the deposit (Sec. 3.2, Eq. charge-conservation-disc),
 * evaluated in FP64 for either precision at every node i in [-1, n_r + 1], j in [0, n_theta]
 * (with n_f > 0 filter passes: i in [max(-1, n_f - 2), min(n_r + 1, n_r + 3 - n_f)], and rho
 * filtered by the same passes as the currents):
 *   res = J^1(i+1/2, j) - J^1(i-1/2, j) + J^2(i, j+1/2) - J^2(i, j-1/2)
 *         + (rho^{n+1} - rho^n)(i, j) / dt,
 * with rho the charge q w of every live particle shared over its cell's four nodes by
 * linear weights at the previous (i1p, dx1p, ...) and the current position. The currents
 * are those of the last deposit: after grpic_push + grpic_deposit pass after_step = 0;
 * after grpic_step (whose field advance rotates the currents) pass 1. Writes out[0] =
 * max |res|, out[1] = max |drho/dt|, out[2] = max over nodes of |res| / (|J terms| +
 * |drho/dt|), out[3] = max over nodes of sum |q w| S / dt at both positions (the scale of
 * the rounding: charges of opposite sign cancel in rho but not here, so a rounded residual
 * is a small multiple of eps * out[3]). Uses six FP64 planes of the arena; synchronises the
 * stream.
 * Errors: GRPIC_ESTATE (fields not initialised), GRPIC_EINVAL (null out). */
GRPIC_API grpic_status grpic_charge_check(grpic_ctx *ctx, int after_step, double out[4]);

/* --- adjoint of the pusher over frozen fields ---------------------------------------- */

/* Test particles pushed through the fields the context holds, frozen (steps 2-11 of
 * Sec. 3.1, no deposit, no field update), and the gradients of their final state with
 * respect to the initial state and the field amplitude. FP64 contexts only.
 *
 * State layout (device, caller-owned): [6][n] doubles, rows x1, x2 (absolute code
 * coordinates), phi, u_1, u_2, u_3 (covariant momenta per unit mass). The fields are the
 * em planes (B, D) times b0 / field_b0, where field_b0 is the amplitude given to
 * grpic_init_fields (1 for GRPIC_FIELD_USER); the Wald, vertical and monopole fields are
 * linear in B0, so b0 is the field amplitude. Both implicit substeps iterate to an exact repeat of the
 * iterate, at most n_iter times. A particle whose step would leave 0 <= x1 < n_r,
 * 0 <= x2 <= n_theta (the horizon layer, the outer edge or an axis, where the boundary rules
 * of Sec. 3.3.3 act) is frozen and reported as NaN.
 *
 * grpic_adjoint_forward: state_out = the state after n_steps steps; ckpt receives the state
 * at steps 0, ckpt_every, 2 ckpt_every, ... < n_steps: ceil(n_steps / ckpt_every) x 6 x n
 * doubles (may be null when n_steps == 0).
 * Errors: GRPIC_ESTATE (mixed context, fields not initialised), GRPIC_EINVAL (n < 0,
 * n_steps < 0, ckpt_every < 1, n_iter outside [1, 1000], field_b0 = 0, null buffers, a
 * quasi-spherical grid with r0 or h0 != 0). */
GRPIC_API grpic_status grpic_adjoint_forward(grpic_ctx *ctx, int64_t n, double qm, double b0,
                                             int n_steps, int ckpt_every, int n_iter,
                                             const double *state0, double *state_out,
                                             double *ckpt);

/* The reverse sweep of the same push (the push of Sec. 3.1 over frozen fields; the paper
 * has no adjoint) (same n, qm, b0, n_steps, ckpt_every, n_iter and the
 * ckpt written by grpic_adjoint_forward): given grad_out = dL/d(final state) ([6][n]),
 * writes grad_state0 = dL/d(initial state) ([6][n]), grad_b0_pp[k] = particle k's part of
 * dL/db0 ([n]) and grad_b0[0] = their sum (deterministic order). Each checkpoint segment is
 * recomputed and the Jacobians of its steps are kept in scratch (min(ckpt_every, n_steps) x
 * 36 x n doubles); they use the implicit-function theorem at the implicit substeps, so the
 * result does not depend on ckpt_every (to the bit). Particles reported NaN by the forward
 * get zero gradients where their grad_out is zero, NaN otherwise. Errors: as the forward. */
GRPIC_API grpic_status grpic_adjoint_backward(grpic_ctx *ctx, int64_t n, double qm, double b0,
                                              int n_steps, int ckpt_every, int n_iter,
                                              const double *ckpt, const double *grad_out,
                                              double *grad_state0, double *grad_b0_pp,
                                              double *grad_b0, double *scratch);

/* --- diagnostics ------------------------------------------------------------------ */

/* Per-phase device time of the hot path, measured with CUDA events recorded on the
 * bound stream around each phase of grpic_step / grpic_push / grpic_deposit /
 * grpic_field_step / grpic_sort while timing is enabled, and the number of kernels
 * the library launched (process-wide). In grpic_step the deposit is fused into the push
 * (push_ms) and deposit_ms holds the current filter. */
typedef struct {
  double predict_ms, sort_ms, push_ms, deposit_ms, advance_ms;
  int64_t push_calls;   /* particle-kernel launches timed in push_ms                 */
  int64_t launches;     /* kernels launched by the library since the last reset      */
  double kernel_ms;     /* the main push kernel alone (FP64: k_push; mixed: the FP32
                           kernel, which runs beside the guard kernels), summed over
                           push_calls launches                                        */
  double inject_ms;     /* grpic_inject                                               */
} grpic_timing;

/* Step 1 of Sec. 3.1 saves each particle's previous position for the deposit. A push that
 * deposits its own move (the fused push + deposit of grpic_step and grpic_step_host) reads
 * it from registers, so storing it only serves later calls that read the previous positions
 * (grpic_deposit, grpic_invariants, grpic_charge_check). keep = 1 (the default): the fused
 * push stores them (i1p, i2p, dx1p, dx2p, 16 or 24 bytes per particle); keep = 0: it skips
 * the stores, and until the next grpic_push, grpic_load_particles or grpic_set_particles of a
 * species those three calls return GRPIC_ESTATE and the previous-position arrays returned by
 * grpic_get_particles are stale. grpic_push (no deposit) always stores them. Errors:
 * GRPIC_EINVAL (null ctx). */
GRPIC_API grpic_status grpic_set_keep_prev(grpic_ctx *ctx, int keep);

/* Throughput probe of the arithmetic pipes that bound the pusher kernels; no counterpart in
 * the paper (it supplies the measured denominator of their rooflines). Queues on `stream`
 * (cudaStream_t; null: the default stream) one kernel of blocks_per_sm x (SM count) blocks of
 * 256 threads on the current device, each thread running 8 independent chains of 32 x iters
 * operations op (0: fused multiply-add, 1: multiply, 2: add): precision GRPIC_FP64 in double
 * (the FP64 pipe's rate for that operation), GRPIC_MIXED in float (the FP32 pipe, at one warp
 * instruction per clock per SM sub-partition, i.e. the instruction-issue peak). *ops
 * receives the operations the launch performs; time it with events on the stream. sink: one
 * device double, never written in practice (it keeps the chains live). Allocates nothing.
 * Errors: GRPIC_EINVAL (iters < 1, blocks_per_sm not in 1 .. 64, op not in 0 .. 2, null sink
 * or ops, other precision), GRPIC_ECUDA (a CUDA error pending before the call, which it
 * leaves in place, or a failed launch). */
GRPIC_API grpic_status grpic_probe_alu(int precision, int op, int64_t iters, int blocks_per_sm,
                                       double *sink, void *stream, int64_t *ops);

/* Enables (1) or disables (0) the per-phase events. Off by default. Instrumentation, with
 * no counterpart in the paper (as the timing and diagnostics calls below). */
GRPIC_API grpic_status grpic_set_timing(grpic_ctx *ctx, int enable);

/* Sums the recorded phases and resets the sums and the launch counter.
 * Synchronises the stream. */
GRPIC_API grpic_status grpic_get_timing(grpic_ctx *ctx, grpic_timing *out);

/* Counters accumulated since the last call, and live counts. Synchronises the stream. */
GRPIC_API grpic_status grpic_get_diagnostics(grpic_ctx *ctx, grpic_diag *out);

/* A one-line description of the last error returned on this context (empty when none),
 * owned by the context and valid until its next call. No counterpart in the paper. */
GRPIC_API const char *grpic_last_error(const grpic_ctx *ctx);

/* Waits for the context's streams and frees what it owns on the host and its streams and
 * events; the arena stays the caller's. A null context is ignored. No counterpart in the
 * paper. */
GRPIC_API void grpic_destroy(grpic_ctx *ctx);

/* sizeof(grpic_config) as this library was compiled: bindings compare it with their own
 * layout of the struct before the first grpic_create. No CUDA work; no counterpart in the
 * paper. */
GRPIC_API size_t grpic_config_bytes(void);

#ifdef __cplusplus
}
#endif
#endif
