"""Python access to the FP64 CPU oracle (grpic_oracle.c) through ctypes.

TEST INFRASTRUCTURE. Only tests/, ``__graft_entry__.smoke()`` and bench.py's
cpu_baseline / reference leg may import this module. It does not import the
CUDA package and the CUDA package does not import it.

``OracleSim`` holds one simulation's state in numpy arrays in the storage
convention of ``grpic_oracle.h`` (planes [NY][NX], G = 2 ghost cells per side,
half-integer positions stored at their lower integer) and calls the C routines,
each of which cites the passage of arXiv:2511.17701 it follows.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "grpic_oracle.c")
LIB = os.path.join(HERE, "libgrpic_oracle.so")
G = 2

# plane indices, as the enum in grpic_oracle.h
(B1, B2, B3, D1, D2, D3, B01, B02, B03, D01, D02, D03, J1, J2, J3, J01, J02, J03,
 BN1, BN2, BN3, BI1, BI2, BI3, DI1, DI2, DI3, JA1, JA2, JA3, NPLANES) = range(31)

FIELD_ZERO, FIELD_WALD, FIELD_VERTICAL = 0, 1, 2
FIELD_MONOPOLE = 4  # A_phi = -B0 cos(theta), the BZ monopole test (Sec. 4.5)


def build(force: bool = False) -> str:
    """Compile the oracle (plain C, -O2 -ffp-contract=off, OpenMP over particles)."""
    if force or not os.path.exists(LIB) or os.path.getmtime(LIB) < max(
            os.path.getmtime(SRC), os.path.getmtime(os.path.join(HERE, "grpic_oracle.h")),
            os.path.getmtime(os.path.join(HERE, "pusher_generic.inc"))):
        tmp = LIB + ".tmp%d" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-fopenmp", "-fPIC",
                               "-shared", "-o", tmp, SRC, "-lm"])
        os.replace(tmp, LIB)
    return LIB


class Params(C.Structure):
    _fields_ = [("metric", C.c_int), ("a", C.c_double), ("n_r", C.c_int), ("n_th", C.c_int),
                ("r_min", C.c_double), ("r_max", C.c_double), ("dt", C.c_double),
                ("n_iter", C.c_int), ("small_angle", C.c_double), ("n_f", C.c_int),
                ("r_absorb", C.c_double), ("absorb_coef", C.c_double), ("r0", C.c_double),
                ("h0", C.c_double)]


_MFIELDS = ["r", "th", "f", "g", "h11", "h22", "h33", "h13", "H11", "H22", "H33", "H13",
            "alpha", "beta1", "sqrt_h", "sqrt_ht",
            "d1H11", "d1H22", "d1H33", "d1H13", "d1alpha", "d1beta1",
            "d2H11", "d2H22", "d2H33", "d2H13", "d2alpha", "d2beta1"]


class Metric(C.Structure):
    _fields_ = [(n, C.c_double) for n in _MFIELDS]

    def as_dict(self):
        return {n: getattr(self, n) for n in _MFIELDS}


_PD = C.POINTER(C.c_double)
_PI32 = C.POINTER(C.c_int32)
_PU8 = C.POINTER(C.c_uint8)


class Species(C.Structure):
    _fields_ = [("n", C.c_int64), ("i1", _PI32), ("i2", _PI32), ("dx1", _PD), ("dx2", _PD),
                ("u1", _PD), ("u2", _PD), ("u3", _PD), ("phi", _PD), ("w", _PD),
                ("tag", _PU8), ("i1p", _PI32), ("i2p", _PI32), ("dx1p", _PD), ("dx2p", _PD),
                ("qm", C.c_double), ("qc", C.c_double), ("massless", C.c_int)]


PARTICLE_FIELDS = {"i1": np.int32, "i2": np.int32, "dx1": np.float64, "dx2": np.float64,
                   "u1": np.float64, "u2": np.float64, "u3": np.float64, "phi": np.float64,
                   "w": np.float64, "tag": np.uint8, "i1p": np.int32, "i2p": np.int32,
                   "dx1p": np.float64, "dx2p": np.float64}

_lib = None


def lib():
    global _lib
    if _lib is None:
        L = C.CDLL(build())
        P, PP = C.POINTER(Params), C.POINTER(Species)
        L.ora_metric_point.argtypes = [P, C.c_double, C.c_double, C.c_int, C.POINTER(Metric)]
        L.ora_polar_area.argtypes = [P, C.c_double]
        L.ora_polar_area.restype = C.c_double
        L.ora_potential.argtypes = [P, C.c_int, C.c_double, C.c_double, C.c_double, _PD]
        L.ora_fields_point.argtypes = [P, C.c_int, C.c_double, C.c_double, C.c_double, _PD, _PD]
        L.ora_tetrad.argtypes = [P, C.c_double, C.c_double, C.c_int, _PD, _PD]
        L.ora_boris.argtypes = [_PD, _PD, _PD, C.c_double]
        L.ora_u_lower0.argtypes = [P, C.c_double, C.c_double, _PD, C.c_int]
        L.ora_u_lower0.restype = C.c_double
        L.ora_invariants.argtypes = [P, C.c_int, C.c_double, C.c_double, C.c_double, C.c_double,
                                     _PD, _PD]
        L.ora_set_threads.argtypes = [C.c_int]
        L.ora_set_threads.restype = None
        L.ora_max_threads.restype = C.c_int
        L.ora_time_step.argtypes = [P, C.c_double]
        L.ora_time_step.restype = C.c_double
        L.ora_init_fields.argtypes = [P, _PD, C.c_int, C.c_double]
        L.ora_load.argtypes = [P, PP, _PD, _PD, _PD, _PD, C.c_double]
        L.ora_push.argtypes = [P, _PD, PP, C.c_int, C.c_int, C.c_double, C.POINTER(C.c_int64)]
        L.ora_deposit.argtypes = [P, _PD, PP, C.c_int]
        L.ora_charge.argtypes = [P, PP, C.c_int, C.c_int, _PD]
        L.ora_field_predict.argtypes = [P, _PD]
        L.ora_field_advance.argtypes = [P, _PD]
        L.ora_aux_fields.argtypes = [P, _PD, _PD, _PD]
        L.ora_sort.argtypes = [P, PP, C.c_int, C.c_int, C.POINTER(C.c_int64)]
        L.ora_sort.restype = C.c_int64
        L.ora_sort_key.argtypes = [P, C.c_int, C.c_int, C.c_int32, C.c_int32, C.c_uint8]
        L.ora_sort_key.restype = C.c_uint32
        L.ora_step.argtypes = [P, _PD, PP, C.c_int, C.c_int, C.c_int, C.c_int, C.c_int,
                               C.c_int64, C.POINTER(C.c_int64)]
        L.ora_filter_plane.argtypes = [P, _PD, C.c_int, C.c_double, C.c_int]
        L.ora_filter_currents.argtypes = [P, _PD]
        L.ora_cell_state.argtypes = [P, _PD, PP, PP, _PD, _PD]
        L.ora_inject.argtypes = [P, _PD, PP, PP, C.c_double, C.c_double, C.c_double, _PD,
                                 C.c_int64, C.c_int64, C.c_int64]
        L.ora_inject.restype = C.c_int64
        L.ora_push_frozen.argtypes = [P, _PD, C.c_double, C.c_double, C.c_int, C.c_int64, _PD]
        L.ora_push_frozen_cs.argtypes = [P, _PD, C.c_double, C.c_double, C.c_double, C.c_int,
                                         C.c_int64, _PD, _PD]
        _lib = L
    return _lib


def _dp(a):
    return a.ctypes.data_as(_PD)


def make_params(cfg: dict) -> Params:
    """cfg keys: metric ('ks' | 'ks0'), a, n_r, n_theta, r_min, r_max, dt, n_iter,
    small_angle, n_filter, r_absorb, absorb_coef, r0, h0 (quasi-spherical map)."""
    return Params(1 if cfg.get("metric", "ks") == "ks" else 0, float(cfg.get("a", 0.0)),
                  int(cfg["n_r"]), int(cfg["n_theta"]), float(cfg["r_min"]), float(cfg["r_max"]),
                  float(cfg.get("dt", 0.0)), int(cfg.get("n_iter", 10)),
                  float(cfg.get("small_angle", 1e-5)), int(cfg.get("n_filter", 0)),
                  float(cfg.get("r_absorb", 1e300)), float(cfg.get("absorb_coef", 1.0)),
                  float(cfg.get("r0", 0.0)), float(cfg.get("h0", 0.0)))


def metric_point(cfg, x1, x2, clamp=False):
    m = Metric()
    lib().ora_metric_point(C.byref(make_params(cfg)), x1, x2, int(clamp), C.byref(m))
    return m.as_dict()


def polar_area(cfg, x1):
    return lib().ora_polar_area(C.byref(make_params(cfg)), x1)


def potential(cfg, kind, B0, x1, x2):
    A = np.zeros(3)
    lib().ora_potential(C.byref(make_params(cfg)), kind, B0, x1, x2, _dp(A))
    return A


def fields_point(cfg, kind, B0, x1, x2):
    B, D = np.zeros(3), np.zeros(3)
    lib().ora_fields_point(C.byref(make_params(cfg)), kind, B0, x1, x2, _dp(B), _dp(D))
    return B, D


def tetrad(cfg, x1, x2, direction, v):
    """direction: 'vec2hat', 'hat2vec', 'cov2hat', 'hat2cov'."""
    d = {"vec2hat": 0, "hat2vec": 1, "cov2hat": 2, "hat2cov": 3}[direction]
    vi, vo = np.ascontiguousarray(v, dtype=np.float64), np.zeros(3)
    lib().ora_tetrad(C.byref(make_params(cfg)), x1, x2, d, _dp(vi), _dp(vo))
    return vo


def boris(u, Dh, Bh, hq):
    u = np.array(u, dtype=np.float64)
    lib().ora_boris(_dp(u), _dp(np.asarray(Dh, np.float64)), _dp(np.asarray(Bh, np.float64)), hq)
    return u


def u_lower0(cfg, x1, x2, u, massless=False):
    """u_0 = -alpha gamma + beta^1 u_1, gamma = sqrt(m2 + h^ij u_i u_j), m2 = 0 if massless."""
    return lib().ora_u_lower0(C.byref(make_params(cfg)), x1, x2, _dp(np.asarray(u, np.float64)),
                              int(bool(massless)))


def invariants(cfg, kind, B0, qm, x1, x2, u):
    out = np.zeros(2)
    lib().ora_invariants(C.byref(make_params(cfg)), kind, B0, qm, x1, x2,
                         _dp(np.asarray(u, np.float64)), _dp(out))
    return out


def set_threads(n: int):
    """Threads of the oracle's OpenMP loops (for timing it on 1 or all host cores)."""
    lib().ora_set_threads(int(n))


def max_threads() -> int:
    return int(lib().ora_max_threads())


def time_step(cfg, cfl):
    return lib().ora_time_step(C.byref(make_params(cfg)), cfl)


def sort_key(cfg, tr, tt, i1, i2, tag):
    return lib().ora_sort_key(C.byref(make_params(cfg)), tr, tt, i1, i2, tag)


def sort_keys(cfg, tr, tt, i1, i2, tag=None):
    """ora_sort_key for whole arrays: tile-major cell key (tile = (i2 // tt) * ntr + i1 // tr,
    ntr = ceil(n_r / tr); key = tile * tr * tt + (i2 % tt) * tr + i1 % tr), 0xFFFFFFFF for
    particles not alive, for cells inside the grid (i1, i2 >= 0, as every live particle's).
    A stable argsort of the keys is the sort's permutation."""
    i1 = np.asarray(i1, dtype=np.int64)
    i2 = np.asarray(i2, dtype=np.int64)
    ntr = (int(cfg["n_r"]) + tr - 1) // tr
    key = ((i2 // tt) * ntr + i1 // tr) * (tr * tt) + (i2 % tt) * tr + i1 % tr
    if tag is not None:
        key = np.where(np.asarray(tag) == 1, key, 0xFFFFFFFF)
    return key.astype(np.uint32)


class OracleSpecies:
    """Particle arrays of one species (numpy), mirrored into the C struct on use."""

    def __init__(self, n: int, qm: float, qc: float, massless: bool = False):
        self.qm, self.qc = float(qm), float(qc)
        self.massless = bool(massless)
        self.n = int(n)
        self.a = {k: np.zeros(max(n, 1), dtype=t) for k, t in PARTICLE_FIELDS.items()}

    def struct(self) -> Species:
        a = self.a
        return Species(self.n, a["i1"].ctypes.data_as(_PI32), a["i2"].ctypes.data_as(_PI32),
                       _dp(a["dx1"]), _dp(a["dx2"]), _dp(a["u1"]), _dp(a["u2"]), _dp(a["u3"]),
                       _dp(a["phi"]), _dp(a["w"]), a["tag"].ctypes.data_as(_PU8),
                       a["i1p"].ctypes.data_as(_PI32), a["i2p"].ctypes.data_as(_PI32),
                       _dp(a["dx1p"]), _dp(a["dx2p"]), self.qm, self.qc, int(self.massless))

    def view(self) -> dict:
        return {k: v[: self.n] for k, v in self.a.items()}

    def reserve(self, cap: int):
        """Grow the arrays to hold at least cap particles."""
        if cap > len(self.a["i1"]):
            for k, v in self.a.items():
                g = np.zeros(cap, dtype=v.dtype)
                g[: len(v)] = v
                self.a[k] = g

    def copy(self) -> "OracleSpecies":
        o = OracleSpecies(self.n, self.qm, self.qc, self.massless)
        o.a = {k: v.copy() for k, v in self.a.items()}
        return o


class OracleSim:
    """One grid + fields + species, advanced by the oracle."""

    def __init__(self, cfg: dict):
        self.cfg = dict(cfg)
        if float(self.cfg.get("dt", 0.0)) <= 0.0:
            self.cfg["dt"] = time_step(self.cfg, float(self.cfg.get("cfl", 0.5)))
        self.p = make_params(self.cfg)
        self.NX = self.cfg["n_r"] + 2 * G + 1
        self.NY = self.cfg["n_theta"] + 2 * G + 1
        self.F = np.zeros((NPLANES, self.NY, self.NX))
        self.species: list[OracleSpecies] = []
        self.counters = np.zeros(4, dtype=np.int64)
        self.step_index = 0

    @property
    def dt(self):
        return self.p.dt

    def plane(self, k):
        return self.F[k]

    def init_fields(self, kind: int, B0: float):
        lib().ora_init_fields(C.byref(self.p), _dp(self.F), kind, B0)

    def add_species(self, pos: dict, uhat, w0, qm, qc, density_power=0.0,
                    massless=False) -> OracleSpecies:
        """pos: i1, i2, dx1, dx2 arrays; uhat: (3, n) tetrad-frame momenta; w0: base weights.
        massless: photons (gamma = |u|, no EM push, nothing deposited)."""
        n = len(pos["i1"])
        s = OracleSpecies(n, qm, qc, massless)
        for k in ("i1", "i2", "dx1", "dx2"):
            s.a[k][:n] = pos[k]
        uh = [np.ascontiguousarray(uhat[c], dtype=np.float64) for c in range(3)]
        w0 = np.ascontiguousarray(w0, dtype=np.float64)
        st = s.struct()
        lib().ora_load(C.byref(self.p), C.byref(st), _dp(uh[0]), _dp(uh[1]), _dp(uh[2]),
                       _dp(w0), float(density_power))
        self.species.append(s)
        return s

    def add_raw_species(self, arrays: dict, qm, qc, massless=False) -> OracleSpecies:
        """A species from complete particle arrays (every key of PARTICLE_FIELDS)."""
        n = len(arrays["i1"])
        s = OracleSpecies(n, qm, qc, massless)
        for k in PARTICLE_FIELDS:
            s.a[k][:n] = arrays[k]
        self.species.append(s)
        return s

    def _structs(self):
        arr = (Species * max(len(self.species), 1))()
        for i, s in enumerate(self.species):
            arr[i] = s.struct()
        return arr

    def _sync_n(self, arr):
        for i, s in enumerate(self.species):
            s.n = arr[i].n

    def predict(self):
        lib().ora_field_predict(C.byref(self.p), _dp(self.F))

    def push(self, si: int, field_mode=0, fkind=0, B0=0.0):
        st = self.species[si].struct()
        cnt = np.zeros(4, dtype=np.int64)
        lib().ora_push(C.byref(self.p), _dp(self.F), C.byref(st), field_mode, fkind, B0,
                       cnt.ctypes.data_as(C.POINTER(C.c_int64)))
        self.counters += cnt
        return cnt

    def deposit(self):
        arr = self._structs()
        lib().ora_deposit(C.byref(self.p), _dp(self.F), arr, len(self.species))

    def charge(self, prev: bool):
        rho = np.zeros((self.NY, self.NX))
        arr = self._structs()
        lib().ora_charge(C.byref(self.p), arr, len(self.species), int(prev), _dp(rho))
        return rho

    def filter_currents(self):
        """n_filter passes of the current filter on J (and on the rounding scales JA)."""
        lib().ora_filter_currents(C.byref(self.p), _dp(self.F))

    def filter_plane(self, plane, half: bool, parity: float, n: int):
        """n passes of the current filter on a [NY][NX] array (returns a filtered copy);
        half: a half-row (x2 = j + 1/2) quantity; parity: +1 even, -1 odd across the axes."""
        f = np.ascontiguousarray(plane, dtype=np.float64).copy()
        lib().ora_filter_plane(C.byref(self.p), _dp(f), int(half), float(parity), int(n))
        return f

    def aux_fields(self):
        """E and H (each (3, NY, NX)) of the em planes as they stand (Eqs. discretized-auxE,
        discretized-auxH), zero where the solver does not compute them."""
        E = np.zeros((3, self.NY, self.NX))
        H = np.zeros((3, self.NY, self.NX))
        lib().ora_aux_fields(C.byref(self.p), _dp(self.F), _dp(E), _dp(H))
        return E, H

    def advance(self):
        lib().ora_field_advance(C.byref(self.p), _dp(self.F))

    def cell_state(self, se=0, sp=1):
        """(n, B_i B^i) per cell [n_th][n_r] as the pair injection sees them."""
        nc = np.zeros((self.cfg["n_theta"], self.cfg["n_r"]))
        b2 = np.zeros_like(nc)
        a, b = self.species[se].struct(), self.species[sp].struct()
        lib().ora_cell_state(C.byref(self.p), _dp(self.F), C.byref(a), C.byref(b), _dp(nc),
                             _dp(b2))
        return nc, b2

    def inject(self, sigma0, sigma_th, B0, pool, pool_offset=0, cap=None, se=0, sp=1):
        """Pair injection where sigma > sigma_th (pool: [pool_n, 8] random draws); returns
        the pairs added. cap: room per species (default: every cell can take one pair)."""
        pool = np.ascontiguousarray(pool, dtype=np.float64)
        ncell = self.cfg["n_r"] * self.cfg["n_theta"]
        if cap is None:
            cap = max(self.species[se].n, self.species[sp].n) + ncell
        for k in (se, sp):
            self.species[k].reserve(cap)
        a, b = self.species[se].struct(), self.species[sp].struct()
        added = lib().ora_inject(C.byref(self.p), _dp(self.F), C.byref(a), C.byref(b),
                                 float(sigma0), float(sigma_th), float(B0), _dp(pool),
                                 pool.shape[0], int(pool_offset), int(cap))
        self.species[se].n, self.species[sp].n = int(a.n), int(b.n)
        return int(added)

    def sort(self, si: int, tr: int, tt: int):
        s = self.species[si]
        st = s.struct()
        perm = np.zeros(max(s.n, 1), dtype=np.int64)
        n = lib().ora_sort(C.byref(self.p), C.byref(st), tr, tt,
                           perm.ctypes.data_as(C.POINTER(C.c_int64)))
        old_n = s.n
        s.n = int(n)
        return perm[:old_n]

    def step(self, n_steps=1, sort_every=0, tr=16, tt=16):
        arr = self._structs()
        cnt = np.zeros(4, dtype=np.int64)
        lib().ora_step(C.byref(self.p), _dp(self.F), arr, len(self.species), n_steps, sort_every,
                       tr, tt, self.step_index, cnt.ctypes.data_as(C.POINTER(C.c_int64)))
        self._sync_n(arr)
        self.counters += cnt
        self.step_index += n_steps


# ---------------------------------------------------------------------------------------
# Frozen-field test particles and their exact FP64 Jacobian (complex step)
# ---------------------------------------------------------------------------------------
FROZEN_STATE = ("x1", "x2", "phi", "u1", "u2", "u3")
CS_STEP = 1e-30


def _frozen_params(osim, n_iter):
    p = make_params(dict(osim.cfg, dt=osim.dt))
    if n_iter:
        p.n_iter = int(n_iter)
    return p


def frozen_push(osim, state, scale, qm, n_steps, n_iter=None):
    """Push test particles n_steps steps in osim's em-plane fields times `scale` (steps 2-11
    of Sec. 3.1, no deposit). state: (6, n) array x1, x2, phi, u1, u2, u3 (absolute code
    coordinates). Both implicit pushes run n_iter times (default: the configuration's).
    Returns the new state; particles that reached a boundary are NaN."""
    st = np.array(state, dtype=np.float64, order="C").reshape(6, -1).copy()
    lib().ora_push_frozen(C.byref(_frozen_params(osim, n_iter)), _dp(osim.F), float(scale),
                          float(qm), int(n_steps), st.shape[1], _dp(st))
    return st


def frozen_jacobian(osim, state, scale, qm, n_steps, n_iter=None, inputs=None):
    """d(final state)/d(inputs) of frozen_push by the complex step (exact to rounding).

    inputs: names among FROZEN_STATE and "scale" (default all seven). Returns the final
    state (6, n) and J with shape (n, 6, len(inputs))."""
    inputs = list(inputs or (list(FROZEN_STATE) + ["scale"]))
    st0 = np.array(state, dtype=np.float64, order="C").reshape(6, -1)
    n = st0.shape[1]
    p = _frozen_params(osim, n_iter)
    J = np.zeros((n, 6, len(inputs)))
    final = None
    for c, name in enumerate(inputs):
        re = st0.copy()
        im = np.zeros_like(re)
        s_im = 0.0
        if name == "scale":
            s_im = CS_STEP
        else:
            im[FROZEN_STATE.index(name)] = CS_STEP
        lib().ora_push_frozen_cs(C.byref(p), _dp(osim.F), float(scale), s_im, float(qm),
                                 int(n_steps), n, _dp(re), _dp(im))
        J[:, :, c] = (im / CS_STEP).T
        final = re
    return final, J
