"""ctypes binding of libgrpic (include/grpic.h): argument marshalling only.

Every step of the hot path runs in the library's CUDA kernels. PyTorch provides the
device arena (one uint8 tensor) and the stream; views into the arena are torch
tensors that alias the library's buffers.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import _build

GHOSTS = 2
MAX_SPECIES = 8

OK, EINVAL, ENOMEM, ECUDA, ESTATE, ECAPACITY, ENONFINITE = range(7)
FP64, MIXED = 0, 1
METRIC_KS0, METRIC_KS = 0, 1
FIELD_ZERO, FIELD_WALD, FIELD_VERTICAL, FIELD_USER, FIELD_MONOPOLE = range(5)
PREDICT, ADVANCE = 0, 1
(B1, B2, B3, D1, D2, D3, B01, B02, B03, D01, D02, D03, J1, J2, J3, J01, J02, J03,
 BN1, BN2, BN3, BI1, BI2, BI3, DI1, DI2, DI3, NPLANES) = range(28)

EXPORTS = ["grpic_create", "grpic_arena_bytes", "grpic_bind", "grpic_init_metric", "grpic_dt",
           "grpic_init_fields", "grpic_load_particles", "grpic_set_particles",
           "grpic_get_particles", "grpic_species_arrays", "grpic_plane_ptr", "grpic_push",
           "grpic_deposit", "grpic_field_step", "grpic_sort", "grpic_step",
           "grpic_get_diagnostics", "grpic_set_timing", "grpic_get_timing", "grpic_last_error",
           "grpic_destroy", "grpic_sort_permutation_noalloc", "grpic_invariants",
           "grpic_adjoint_forward", "grpic_adjoint_backward", "grpic_charge_check",
           "grpic_config_bytes", "grpic_inject", "grpic_step_host", "grpic_aux_fields",
           "grpic_set_keep_prev", "grpic_probe_alu", "grpic_sum_bins_add",
           "grpic_sum_bins_value"]


ADJOINT_SCRATCH_PER_STEP = 36  # doubles per particle and step of grpic_adjoint_backward


class GrpicError(RuntimeError):
    pass


class Config(C.Structure):
    _fields_ = [("metric", C.c_int), ("a", C.c_double), ("n_r", C.c_int), ("n_theta", C.c_int),
                ("r_min", C.c_double), ("r_max", C.c_double), ("cfl", C.c_double),
                ("dt", C.c_double), ("n_iter", C.c_int), ("small_angle", C.c_double),
                ("n_filter", C.c_int), ("r_absorb", C.c_double), ("absorb_coef", C.c_double),
                ("n_species", C.c_int), ("capacity", C.c_int64 * MAX_SPECIES),
                ("sort_every", C.c_int), ("tile_r", C.c_int), ("tile_theta", C.c_int),
                ("precision", C.c_int), ("full_iterations", C.c_int),
                ("fp64_guard_cells", C.c_int), ("tiled_push", C.c_int), ("iter_tol", C.c_double),
                ("r0", C.c_double), ("h0", C.c_double), ("massless", C.c_int * MAX_SPECIES)]


_VP = C.c_void_p
PARTICLE_ARRAYS = [("i1", np.int32), ("i2", np.int32), ("dx1", np.float64), ("dx2", np.float64),
                   ("u1", np.float64), ("u2", np.float64), ("u3", np.float64),
                   ("phi", np.float64), ("w", np.float64), ("tag", np.uint8),
                   ("i1p", np.int32), ("i2p", np.int32), ("dx1p", np.float64),
                   ("dx2p", np.float64)]


class Particles(C.Structure):
    _fields_ = [(k, _VP) for k, _ in PARTICLE_ARRAYS]


class ParticleInit(C.Structure):
    _fields_ = [(k, _VP) for k in ("i1", "i2", "dx1", "dx2", "uh1", "uh2", "uh3", "w0")]


class Timing(C.Structure):
    _fields_ = [("predict_ms", C.c_double), ("sort_ms", C.c_double), ("push_ms", C.c_double),
                ("deposit_ms", C.c_double), ("advance_ms", C.c_double),
                ("push_calls", C.c_int64), ("launches", C.c_int64), ("kernel_ms", C.c_double),
                ("inject_ms", C.c_double)]


class Diag(C.Structure):
    _fields_ = [("left_inner", C.c_int64), ("left_outer", C.c_int64),
                ("reflections", C.c_int64), ("nonfinite", C.c_int64),
                ("alive", C.c_int64 * MAX_SPECIES), ("injected", C.c_int64),
                ("inject_dropped", C.c_int64), ("stage_timeouts", C.c_int64)]


_lib = None


def lib(build: bool = True):
    """Load libgrpic.so (building it first when it is missing or stale). Raises if the
    library cannot be built or loaded: there is no fallback."""
    global _lib
    if _lib is None:
        path = _build.build() if build else _build.LIB
        if not os.path.exists(path):
            raise GrpicError("libgrpic.so not found at %s" % path)
        L = C.CDLL(path)
        L.grpic_config_bytes.restype = C.c_size_t
        if L.grpic_config_bytes() != C.sizeof(Config):
            raise GrpicError("grpic_config layout mismatch: library %d bytes, binding %d"
                             % (L.grpic_config_bytes(), C.sizeof(Config)))
        P = C.c_void_p
        L.grpic_create.argtypes = [C.POINTER(Config), C.POINTER(P)]
        L.grpic_arena_bytes.argtypes = [P]
        L.grpic_arena_bytes.restype = C.c_size_t
        L.grpic_bind.argtypes = [P, P, C.c_size_t, P]
        L.grpic_init_metric.argtypes = [P]
        L.grpic_dt.argtypes = [P]
        L.grpic_dt.restype = C.c_double
        L.grpic_init_fields.argtypes = [P, C.c_int, C.c_double]
        L.grpic_load_particles.argtypes = [P, C.c_int, C.c_int64, C.c_double, C.c_double,
                                           C.c_double, C.POINTER(ParticleInit)]
        L.grpic_set_particles.argtypes = [P, C.c_int, C.c_int64, C.c_double, C.c_double,
                                          C.POINTER(Particles)]
        L.grpic_get_particles.argtypes = [P, C.c_int, C.POINTER(Particles), C.POINTER(C.c_int64)]
        L.grpic_species_arrays.argtypes = [P, C.c_int, C.POINTER(Particles), C.POINTER(C.c_int64)]
        L.grpic_plane_ptr.argtypes = [P, C.c_int, C.POINTER(C.c_void_p)]
        L.grpic_invariants.argtypes = [P, C.c_int, C.c_int, C.c_double, P, P]
        L.grpic_push.argtypes = [P, C.c_int]
        L.grpic_deposit.argtypes = [P]
        L.grpic_field_step.argtypes = [P, C.c_int]
        L.grpic_sort.argtypes = [P, C.c_int]
        L.grpic_step.argtypes = [P, C.c_int]
        L.grpic_step_host.argtypes = [P, C.POINTER(Particles), C.POINTER(C.c_int64)]
        L.grpic_aux_fields.argtypes = [P, C.c_void_p * 3, C.c_void_p * 3]
        L.grpic_get_diagnostics.argtypes = [P, C.POINTER(Diag)]
        L.grpic_set_timing.argtypes = [P, C.c_int]
        L.grpic_set_keep_prev.argtypes = [P, C.c_int]
        L.grpic_probe_alu.argtypes = [C.c_int, C.c_int, C.c_int64, C.c_int, P, P,
                                      C.POINTER(C.c_int64)]
        L.grpic_sum_bins_add.argtypes = [P, C.c_int64, P, P]
        L.grpic_sum_bins_value.argtypes = [P, C.POINTER(C.c_double)]
        L.grpic_get_timing.argtypes = [P, C.POINTER(Timing)]
        L.grpic_last_error.argtypes = [P]
        L.grpic_last_error.restype = C.c_char_p
        L.grpic_sort_permutation_noalloc.argtypes = [C.c_int, C.c_int, C.c_int, C.c_int, P, P,
                                                     P, C.c_int64, P, P, P]
        L.grpic_destroy.argtypes = [P]
        L.grpic_destroy.restype = None
        L.grpic_charge_check.argtypes = [P, C.c_int, C.POINTER(C.c_double)]
        L.grpic_inject.argtypes = [P, C.c_int, C.c_int, C.c_double, C.c_double, C.c_double,
                                   C.c_void_p, C.c_int64, C.c_int64]
        L.grpic_adjoint_forward.argtypes = [P, C.c_int64, C.c_double, C.c_double, C.c_int,
                                            C.c_int, C.c_int, P, P, P]
        L.grpic_adjoint_backward.argtypes = [P, C.c_int64, C.c_double, C.c_double, C.c_int,
                                             C.c_int, C.c_int, P, P, P, P, P, P]
        _lib = L
    return _lib


def make_config(cfg: dict, capacities) -> Config:
    c = Config()
    c.metric = METRIC_KS if cfg.get("metric", "ks") == "ks" else METRIC_KS0
    c.a = float(cfg.get("a", 0.0))
    c.n_r, c.n_theta = int(cfg["n_r"]), int(cfg["n_theta"])
    c.r_min, c.r_max = float(cfg["r_min"]), float(cfg["r_max"])
    c.cfl = float(cfg.get("cfl", 0.5))
    c.dt = float(cfg.get("dt", 0.0))
    c.n_iter = int(cfg.get("n_iter", 10))
    c.small_angle = float(cfg.get("small_angle", 1e-5))
    c.n_filter = int(cfg.get("n_filter", 0))
    c.r_absorb = float(cfg.get("r_absorb", 1e300))
    c.absorb_coef = float(cfg.get("absorb_coef", 1.0))
    c.n_species = len(capacities)
    for i, n in enumerate(list(capacities)[:MAX_SPECIES]):
        c.capacity[i] = int(n)
    c.sort_every = int(cfg.get("sort_every", 0))
    c.tile_r = int(cfg.get("tile_r", 16))
    c.tile_theta = int(cfg.get("tile_theta", 16))
    c.precision = MIXED if cfg.get("precision", "fp64") == "mixed" else FP64
    c.full_iterations = int(cfg.get("full_iterations", 0))
    c.fp64_guard_cells = int(cfg.get("fp64_guard_cells", 0))
    c.tiled_push = int(cfg.get("tiled_push", 0))
    c.iter_tol = float(cfg.get("iter_tol", 0.0))
    c.r0 = float(cfg.get("r0", 0.0))
    c.h0 = float(cfg.get("h0", 0.0))
    # species indices of massless particles (photons)
    for i in cfg.get("massless", ()):
        c.massless[int(i)] = 1
    return c


def particle_dtypes(precision: str) -> list:
    """(name, numpy dtype) of each particle array for a precision ("fp64" or "mixed")."""
    f = np.float32 if precision == "mixed" else np.float64
    return [(k, f if t == np.float64 else t) for k, t in PARTICLE_ARRAYS]


def _ptr(a):
    """Data pointer of a numpy array or torch tensor (host or device), or None."""
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        assert a.flags["C_CONTIGUOUS"]
        return a.ctypes.data
    return a.data_ptr()


class Sim:
    """One simulation context bound to a torch-allocated arena on a CUDA device."""

    def __init__(self, cfg: dict, capacities, device="cuda:0"):
        import torch
        self.torch = torch
        self.cfg = dict(cfg)
        self.L = lib()
        self.ctx = C.c_void_p()
        self._check(self.L.grpic_create(C.byref(make_config(cfg, capacities)),
                                        C.byref(self.ctx)), "create")
        self.nbytes = self.L.grpic_arena_bytes(self.ctx)
        self.device = torch.device(device)
        self.arena_t = torch.empty(self.nbytes + 256, dtype=torch.uint8, device=self.device)
        base = self.arena_t.data_ptr()
        self.off0 = (-base) % 256
        self.stream = torch.cuda.current_stream(self.device)
        self._check(self.L.grpic_bind(self.ctx, base + self.off0, self.nbytes,
                                      self.stream.cuda_stream), "bind")
        self.NX = int(cfg["n_r"]) + 2 * GHOSTS + 1
        self.NY = int(cfg["n_theta"]) + 2 * GHOSTS + 1
        self.n_species = len(capacities)
        self.precision = cfg.get("precision", "fp64")
        self.ptypes = particle_dtypes(self.precision)
        self.fdtype = np.float32 if self.precision == "mixed" else np.float64
        self.tfdtype = torch.float32 if self.precision == "mixed" else torch.float64
        self.qm = [0.0] * self.n_species
        self.qc = [0.0] * self.n_species

    def _check(self, st, what):
        if st != OK:
            msg = self.L.grpic_last_error(self.ctx) if self.ctx else b""
            raise GrpicError("grpic %s failed (status %d): %s" % (what, st, (msg or b"").decode()))

    def close(self):
        if self.ctx:
            self.L.grpic_destroy(self.ctx)
            self.ctx = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # --- set-up ---------------------------------------------------------------------
    def init_metric(self):
        self._check(self.L.grpic_init_metric(self.ctx), "init_metric")

    @property
    def dt(self) -> float:
        return self.L.grpic_dt(self.ctx)

    def init_fields(self, kind: int, B0: float = 1.0):
        self._check(self.L.grpic_init_fields(self.ctx, kind, B0), "init_fields")

    def load_particles(self, s, pos, uhat, w0, qm, qc, density_power=0.0):
        keep = [np.ascontiguousarray(pos["i1"], np.int32), np.ascontiguousarray(pos["i2"], np.int32),
                np.ascontiguousarray(pos["dx1"], np.float64), np.ascontiguousarray(pos["dx2"], np.float64),
                np.ascontiguousarray(uhat[0], np.float64), np.ascontiguousarray(uhat[1], np.float64),
                np.ascontiguousarray(uhat[2], np.float64), np.ascontiguousarray(w0, np.float64)]
        pi = ParticleInit(*[_ptr(a) for a in keep])
        n = keep[0].size
        self._check(self.L.grpic_load_particles(self.ctx, s, n, qm, qc, density_power,
                                                C.byref(pi)), "load_particles")
        self.qm[s], self.qc[s] = qm, qc
        self.sync()

    def set_particles(self, s, arrays: dict, qm, qc):
        """Full species state from host (numpy) or device (torch) arrays. Without i1p, i2p,
        dx1p, dx2p the previous position is set to the position on the device."""
        keep = []
        for k, t in self.ptypes:
            if k not in arrays and k in ("i1p", "i2p", "dx1p", "dx2p"):
                keep.append(None)
                continue
            a = arrays[k]
            if isinstance(a, np.ndarray) or not hasattr(a, "data_ptr"):
                a = np.ascontiguousarray(a, dtype=t)
            keep.append(a)
        n = len(keep[0])
        p = Particles(*[None if a is None else _ptr(a) for a in keep])
        self._check(self.L.grpic_set_particles(self.ctx, s, n, qm, qc, C.byref(p)), "set_particles")
        self.qm[s], self.qc[s] = qm, qc
        self.sync()

    def get_particles(self, s) -> dict:
        """Copy of a species' state as numpy arrays (synchronises)."""
        n = C.c_int64()
        self._check(self.L.grpic_species_arrays(self.ctx, s, None, C.byref(n)), "species_arrays")
        out = {k: np.empty(n.value, dtype=t) for k, t in self.ptypes}
        p = Particles(*[_ptr(out[k]) for k, _ in PARTICLE_ARRAYS])
        self._check(self.L.grpic_get_particles(self.ctx, s, C.byref(p), C.byref(n)), "get_particles")
        return out

    def count(self, s) -> int:
        n = C.c_int64()
        self._check(self.L.grpic_species_arrays(self.ctx, s, None, C.byref(n)), "species_arrays")
        return n.value

    def species_views(self, s) -> dict:
        """Torch views of a species' device arrays (valid until the next sort)."""
        torch = self.torch
        p, n = Particles(), C.c_int64()
        self._check(self.L.grpic_species_arrays(self.ctx, s, C.byref(p), C.byref(n)), "species_arrays")
        dt = {np.int32: torch.int32, np.float64: torch.float64, np.float32: torch.float32,
              np.uint8: torch.uint8}
        out = {}
        base = self.arena_t.data_ptr()
        for k, t in self.ptypes:
            off = getattr(p, k) - base
            size = np.dtype(t).itemsize
            out[k] = self.arena_t[off: off + n.value * size].view(dt[t])
        return out

    def plane(self, k):
        """Torch view [NY, NX] of a field plane (valid until the next ADVANCE)."""
        ptr = C.c_void_p()
        self._check(self.L.grpic_plane_ptr(self.ctx, k, C.byref(ptr)), "plane_ptr")
        off = ptr.value - self.arena_t.data_ptr()
        nb = self.NX * self.NY * np.dtype(self.fdtype).itemsize
        return self.arena_t[off: off + nb].view(self.tfdtype).view(self.NY, self.NX)

    def planes(self) -> np.ndarray:
        """Host copy of all field planes as float64, shape (NPLANES, NY, NX) (synchronises)."""
        self.sync()
        return np.stack([self.plane(k).cpu().numpy().astype(np.float64) for k in range(NPLANES)])

    def aux_fields(self):
        """Host copies of the auxiliary E and H planes (grpic_aux_fields) of the em planes as
        they stand, float64 arrays of shape (3, NY, NX) each."""
        NY, NX = self.NY, self.NX
        E = np.zeros((3, NY, NX), dtype=self.fdtype)
        H = np.zeros((3, NY, NX), dtype=self.fdtype)
        pe = (C.c_void_p * 3)(*[E[c].ctypes.data for c in range(3)])
        ph = (C.c_void_p * 3)(*[H[c].ctypes.data for c in range(3)])
        self._check(self.L.grpic_aux_fields(self.ctx, pe, ph), "aux_fields")
        return E.astype(np.float64), H.astype(np.float64)

    def set_planes(self, F: np.ndarray, which=range(NPLANES)):
        for k in which:
            self.plane(k).copy_(self.torch.from_numpy(
                np.ascontiguousarray(F[k]).astype(self.fdtype)))
        self.sync()

    def invariants(self, s, kind: int, B0: float):
        """Conserved E and L per particle (FP64, computed on the device)."""
        torch = self.torch
        n = self.count(s)
        E = torch.empty(max(n, 1), dtype=torch.float64, device=self.device)
        L = torch.empty(max(n, 1), dtype=torch.float64, device=self.device)
        self._check(self.L.grpic_invariants(self.ctx, s, kind, B0, E.data_ptr(), L.data_ptr()),
                    "invariants")
        self.sync()
        return E[:n].cpu().numpy(), L[:n].cpu().numpy()

    def charge_check(self, after_step: bool):
        """grpic_charge_check: (max |residual|, max |drho/dt|, max node-relative residual,
        max absolute charge per node / dt, the rounding scale)."""
        out = (C.c_double * 4)()
        self._check(self.L.grpic_charge_check(self.ctx, 1 if after_step else 0, out),
                    "charge_check")
        return tuple(float(v) for v in out)

    def inject(self, sigma0, sigma_th, B0, pool, pool_offset=-1, se=0, sp=1):
        """grpic_inject: pairs where the magnetization exceeds sigma_th. pool: a float64
        (pool_n, 8) tensor on the device (kept alive by the caller until the stream has run
        the call); pool_offset >= 0 sets the library's pool cursor, < 0 continues."""
        torch = self.torch
        if (pool.dtype != torch.float64 or pool.device != self.device or pool.dim() != 2 or
                pool.shape[1] != 8 or not pool.is_contiguous()):
            raise GrpicError("inject: expected a contiguous (n, 8) float64 tensor on %s"
                             % self.device)
        self._check(self.L.grpic_inject(self.ctx, se, sp, float(sigma0), float(sigma_th),
                                        float(B0), pool.data_ptr(), pool.shape[0],
                                        int(pool_offset)), "inject")

    # --- adjoint of the pusher over frozen fields -------------------------------------
    def _adjoint_state(self, t, what):
        torch = self.torch
        if t.dtype != torch.float64 or t.device != self.device or t.dim() != 2 or t.shape[0] != 6:
            raise GrpicError("%s: expected a (6, n) float64 tensor on %s" % (what, self.device))
        return t.contiguous()

    def adjoint_forward(self, state0, qm, b0, n_steps, ckpt_every, n_iter):
        """grpic_adjoint_forward: returns (final state (6, n), checkpoints)."""
        torch = self.torch
        state0 = self._adjoint_state(state0, "adjoint_forward")
        n = state0.shape[1]
        out = torch.empty_like(state0)
        n_ck = (n_steps + ckpt_every - 1) // ckpt_every if n_steps > 0 else 0
        ckpt = torch.empty((n_ck, 6, n), dtype=torch.float64, device=self.device)
        self._check(self.L.grpic_adjoint_forward(self.ctx, n, qm, b0, n_steps, ckpt_every, n_iter,
                                                 state0.data_ptr(), out.data_ptr(),
                                                 ckpt.data_ptr() if n_ck else None),
                    "adjoint_forward")
        return out, ckpt

    def adjoint_backward(self, ckpt, grad_out, qm, b0, n_steps, ckpt_every, n_iter):
        """grpic_adjoint_backward: returns (d/d state0 (6, n), d/d b0 per particle (n,),
        d/d b0 (1,))."""
        torch = self.torch
        grad_out = self._adjoint_state(grad_out, "adjoint_backward")
        n = grad_out.shape[1]
        gin = torch.empty_like(grad_out)
        gpp = torch.empty(max(n, 1), dtype=torch.float64, device=self.device)
        gsum = torch.empty(1, dtype=torch.float64, device=self.device)
        scratch = torch.empty((min(ckpt_every, max(n_steps, 1)), ADJOINT_SCRATCH_PER_STEP, n),
                              dtype=torch.float64, device=self.device) if n_steps > 0 else None
        self._check(self.L.grpic_adjoint_backward(
            self.ctx, n, qm, b0, n_steps, ckpt_every, n_iter,
            ckpt.data_ptr() if ckpt.numel() else None, grad_out.data_ptr(), gin.data_ptr(),
            gpp.data_ptr(), gsum.data_ptr(), scratch.data_ptr() if scratch is not None else None),
            "adjoint_backward")
        return gin, gpp[:n], gsum

    # --- hot path -------------------------------------------------------------------
    def push(self, s):
        self._check(self.L.grpic_push(self.ctx, s), "push")

    def deposit(self):
        self._check(self.L.grpic_deposit(self.ctx), "deposit")

    def predict(self):
        self._check(self.L.grpic_field_step(self.ctx, PREDICT), "field_step(PREDICT)")

    def advance(self):
        self._check(self.L.grpic_field_step(self.ctx, ADVANCE), "field_step(ADVANCE)")

    def sort(self, s):
        self._check(self.L.grpic_sort(self.ctx, s), "sort")

    def step(self, n=1):
        self._check(self.L.grpic_step(self.ctx, n), "step")

    def step_host(self, states, counts):
        """One step with the particle state streamed through host memory (grpic_step_host).
        states[k]: dict of host arrays (numpy, or torch tensors in page-locked memory) i1, i2,
        dx1, dx2, u1, u2, u3, phi, w, tag of the context's types, read and then overwritten in
        place; counts[k]: the particles they hold. Returns the counts after the step."""
        ns = len(self.qm)
        P = (Particles * ns)()
        keep = []
        for k in range(ns):
            ptrs = []
            for name, t in self.ptypes:
                a = states[k].get(name) if name not in ("i1p", "i2p", "dx1p", "dx2p") else None
                if a is None:
                    ptrs.append(None)
                    continue
                if isinstance(a, np.ndarray):
                    if a.dtype != np.dtype(t) or not a.flags.c_contiguous:
                        raise GrpicError("step_host: %s must be a contiguous %s array" % (name, t))
                keep.append(a)
                ptrs.append(_ptr(a))
            P[k] = Particles(*ptrs)
        n = (C.c_int64 * ns)(*[int(c) for c in counts])
        self._check(self.L.grpic_step_host(self.ctx, P, n), "step_host")
        return [int(x) for x in n]

    def diagnostics(self) -> dict:
        d = Diag()
        self._check(self.L.grpic_get_diagnostics(self.ctx, C.byref(d)), "get_diagnostics")
        return {"left_inner": d.left_inner, "left_outer": d.left_outer,
                "reflections": d.reflections, "nonfinite": d.nonfinite,
                "alive": [d.alive[i] for i in range(self.n_species)],
                "injected": d.injected, "inject_dropped": d.inject_dropped,
                "stage_timeouts": d.stage_timeouts}

    def set_keep_prev(self, keep: bool):
        """grpic_set_keep_prev: whether the fused push + deposit stores previous positions."""
        self._check(self.L.grpic_set_keep_prev(self.ctx, int(bool(keep))), "set_keep_prev")

    def set_timing(self, on: bool):
        self._check(self.L.grpic_set_timing(self.ctx, int(bool(on))), "set_timing")

    def timing(self) -> dict:
        t = Timing()
        self._check(self.L.grpic_get_timing(self.ctx, C.byref(t)), "get_timing")
        return {k: getattr(t, k) for k, _ in Timing._fields_}

    def sync(self):
        self.stream.synchronize()


PROBE_OPS = {"fma": 0, "mul": 1, "add": 2}


def probe_alu(precision: str, op: str, iters: int, blocks_per_sm: int, sink, stream) -> int:
    """grpic_probe_alu: queue the arithmetic-throughput probe kernel on `stream` (a torch
    stream); precision "fp64" or "fp32", op "fma", "mul" or "add"; sink: a float64 device
    tensor of at least one element. Returns the operations the launch performs."""
    ops = C.c_int64()
    st = lib().grpic_probe_alu(MIXED if precision == "fp32" else FP64, PROBE_OPS[op], int(iters),
                               int(blocks_per_sm), sink.data_ptr(), stream.cuda_stream,
                               C.byref(ops))
    if st != OK:
        raise GrpicError("grpic_probe_alu failed (status %d)" % st)
    return ops.value


SUM_BINS = 2048  # GRPIC_SUM_BINS


def sum_bins_add(x, bins, stream):
    """grpic_sum_bins_add: add the finite values of the float64 CUDA tensor x into the int64
    CUDA tensor bins (2 x SUM_BINS elements) on `stream` (a torch stream)."""
    if x.dtype.itemsize != 8 or not x.is_contiguous() or bins.numel() != 2 * SUM_BINS:
        raise GrpicError("sum_bins_add: expected a contiguous float64 tensor and 2 x %d bins"
                         % SUM_BINS)
    st = lib().grpic_sum_bins_add(x.data_ptr(), x.numel(), bins.data_ptr(), stream.cuda_stream)
    if st != OK:
        raise GrpicError("grpic_sum_bins_add failed (status %d)" % st)


def sum_bins_value(bins) -> float:
    """grpic_sum_bins_value: the correctly rounded total of host bins (an int64 numpy array or
    CPU tensor of 2 x SUM_BINS elements)."""
    a = np.ascontiguousarray(bins.numpy() if hasattr(bins, "numpy") else bins, dtype=np.int64)
    if a.size != 2 * SUM_BINS:
        raise GrpicError("sum_bins_value: expected 2 x %d bins" % SUM_BINS)
    out = C.c_double()
    st = lib().grpic_sum_bins_value(a.ctypes.data, C.byref(out))
    if st != OK:
        raise GrpicError("grpic_sum_bins_value failed (status %d)" % st)
    return out.value
