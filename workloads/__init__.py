"""Seeded synthetic inputs for the GR PIC hot path.

This module serves both the CUDA library's users (bench, tests) and the CPU
oracle's tests. It holds none of the method's arithmetic: it only defines the
workload shapes (grid, spin, radii, particles per cell, temperature, seeds) and
draws random numbers: particle positions in code coordinates, momenta in the
local orthonormal (FIDO tetrad) frame from a Maxwell-Juttner distribution, and
base weights. Turning those into covariant momenta and conformal weights is the
method's job and is done separately by the library and by the oracle.

The workloads stand in for the paper's runs (Sec. 4.2 Wald vacuum; Sec. 3.5
performance test, 2048^2 log-r grid): no dataset is read.
"""
from __future__ import annotations

import math
import numpy as np


def horizon_radius(a: float) -> float:
    """Outer horizon of a Kerr black hole, r_h = 1 + sqrt(1 - a^2) (units r_g)."""
    return 1.0 + math.sqrt(1.0 - a * a)


_A = 0.9
_RMIN = 0.95 * horizon_radius(_A)

# Workload definitions. ppc is per species; e+- pairs are co-located. The absorbing
# layer starts at 0.9 r_max (the paper's runs use layers of 10-20% of r_max).
CONFIGS = {
    # Kerr a = 0.9, Wald field, 64^2, r in [0.95 r_h, 10], theta_T = 0.1, 200 steps, CFL 0.5
    "wald64": dict(metric="ks", a=_A, n_r=64, n_theta=64, r_min=_RMIN, r_max=10.0, ppc=8,
                   theta_T=0.1, density_power=0.0, steps=200, cfl=0.5, seed=1, B0=1.0,
                   r_absorb=9.0),
    # same physics on 512^2, r_max = 50, 32 ppc per species (16,777,216 particles), 1000 steps
    "wald512": dict(metric="ks", a=_A, n_r=512, n_theta=512, r_min=_RMIN, r_max=50.0, ppc=32,
                    theta_T=1.0, density_power=0.0, steps=1000, cfl=0.5, seed=2, B0=1.0,
                    r_absorb=45.0),
    # wald64 with 4 current-filter passes: the grid reaches 0.7 r_h (9.9 cells inside the
    # horizon), so the horizon layer i1 <= n_f lies inside it
    "wald64f": dict(metric="ks", a=_A, n_r=64, n_theta=64, r_min=0.7 * horizon_radius(_A),
                    r_max=10.0, ppc=8, theta_T=0.3, density_power=0.0, steps=200, cfl=0.5,
                    seed=4, B0=1.0, r_absorb=9.0, n_filter=4),
    # the BZ monopole test (Sec. 4.5): a = 0.2, r in [r_g, 10 r_g], absorbing layer 1 r_g
    # thick, 1024^2, pairs with theta_T = 0.5 and density ~ r^-2, fiducial rho0 = 5e-5 and
    # d0 = 2.5e-3 r_g (sigma0 = 2500); 45 ppc per species (90 per cell, the paper's
    # performance setting)
    "bz1024": dict(metric="ks", a=0.2, n_r=1024, n_theta=1024, r_min=1.0, r_max=10.0, ppc=45,
                   theta_T=0.5, density_power=2.0, steps=200, cfl=0.5, seed=5, B0=1.0,
                   r_absorb=9.0, rho0=5e-5, d0=2.5e-3, field="monopole", sigma0=2500.0,
                   sigma_th=2000.0, theta_inj=0.5),
    # the pusher benchmark of Sec. 3.5: the monopole test on a 2048^2 log-r grid with 90
    # particles per cell (45 per species, 377,487,360 particles)
    "bz2048": dict(metric="ks", a=0.2, n_r=2048, n_theta=2048, r_min=1.0, r_max=10.0, ppc=45,
                   theta_T=0.5, density_power=2.0, steps=100, cfl=0.5, seed=6, B0=1.0,
                   r_absorb=9.0, rho0=5e-5, d0=2.5e-3, field="monopole", sigma0=2500.0,
                   sigma_th=2000.0, theta_inj=0.5),
    # 2048^2, r_max = 200, 16 ppc per species (134,217,728 particles), density ~ 1/r, 500 steps
    "wald2048": dict(metric="ks", a=_A, n_r=2048, n_theta=2048, r_min=_RMIN, r_max=200.0,
                     ppc=16, theta_T=1.0, density_power=1.0, steps=500, cfl=0.5, seed=3,
                     B0=1.0, r_absorb=180.0),
}

# plasma parameters (code units): fiducial Larmor radius rho0 and skin depth d0 of r_g
RHO0 = 1.0
D0 = 1.0


def species_coefficients(sign: float, rho0: float = RHO0, d0: float = D0):
    """(q/m) B0 = sign / rho0 for the Lorentz force; the deposit coefficient
    sign * rho0 / (4 pi d0^2) gives omega_p = 1/d0 per species at unit density."""
    return sign / rho0, sign * rho0 / (4.0 * math.pi * d0 * d0)


def grid_config(name: str, **over) -> dict:
    c = dict(CONFIGS[name])
    c.update(over)
    return c


def _mj_inverse_cdf(theta: float, npts: int = 200001):
    """Tabulated inverse CDF of the Maxwell-Juttner momentum magnitude,
    f(u) ~ u^2 exp(-(gamma - 1)/theta), gamma = sqrt(1 + u^2)."""
    gmax = 1.0 + 60.0 * theta
    umax = math.sqrt(gmax * gmax - 1.0)
    u = np.linspace(0.0, umax, npts)
    f = u * u * np.exp(-(np.sqrt(1.0 + u * u) - 1.0) / theta)
    cdf = np.concatenate([[0.0], np.cumsum(0.5 * (f[1:] + f[:-1]) * np.diff(u))])
    cdf /= cdf[-1]
    return cdf, u


def maxwell_juttner(rng: np.random.Generator, n: int, theta: float) -> np.ndarray:
    """(3, n) isotropic Maxwell-Juttner momenta (units of m c) in an orthonormal frame."""
    cdf, u = _mj_inverse_cdf(theta)
    mag = np.interp(rng.random(n), cdf, u)
    mu = 2.0 * rng.random(n) - 1.0
    ph = 2.0 * math.pi * rng.random(n)
    st = np.sqrt(np.maximum(0.0, 1.0 - mu * mu))
    return np.stack([mag * st * np.cos(ph), mag * st * np.sin(ph), mag * mu])


def uniform_positions(rng: np.random.Generator, n_r: int, n_theta: int, ppc: int,
                      cells: np.ndarray | None = None) -> dict:
    """ppc particles per cell at uniform random offsets, cell-major order
    (x2 index outer, x1 index inner). `cells` optionally restricts to a list of
    flat cell indices j * n_r + i."""
    if cells is None:
        cells = np.arange(n_r * n_theta, dtype=np.int64)
    cells = np.asarray(cells, dtype=np.int64)
    c = np.repeat(cells, ppc)
    n = c.size
    return {"i1": (c % n_r).astype(np.int32), "i2": (c // n_r).astype(np.int32),
            "dx1": rng.random(n), "dx2": rng.random(n)}


def pair_plasma(cfg: dict, seed: int | None = None, cells: np.ndarray | None = None) -> dict:
    """e+- pair plasma of a workload: shared positions, independent momenta.

    Returns dict(pos=..., uhat=[electrons (3,n), positrons (3,n)], w0=(n,),
    qm=[...], qc=[...], density_power=...)."""
    rng = np.random.Generator(np.random.PCG64(cfg["seed"] if seed is None else seed))
    pos = uniform_positions(rng, cfg["n_r"], cfg["n_theta"], cfg["ppc"], cells)
    n = pos["i1"].size
    ue = maxwell_juttner(rng, n, cfg["theta_T"])
    up = maxwell_juttner(rng, n, cfg["theta_T"])
    rho0, d0 = cfg.get("rho0", RHO0), cfg.get("d0", D0)
    qe, ce = species_coefficients(-1.0, rho0, d0)
    qp, cp = species_coefficients(+1.0, rho0, d0)
    return {"pos": pos, "uhat": [ue, up], "w0": np.full(n, 1.0 / cfg["ppc"]),
            "qm": [qe, qp], "qc": [ce, cp], "density_power": cfg.get("density_power", 0.0)}


def injection_pool(cfg: dict, n: int, seed: int) -> np.ndarray:
    """Random draws for pair injection, [n, 8]: cell offsets dx1, dx2 (uniform), then the
    tetrad-frame momenta of the electron and of the positron (Maxwell-Juttner at the
    workload's injection temperature, theta_inj, else theta_T)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    th = cfg.get("theta_inj", cfg["theta_T"])
    out = np.empty((n, 8))
    out[:, 0] = rng.random(n)
    out[:, 1] = rng.random(n)
    out[:, 2:5] = maxwell_juttner(rng, n, th).T
    out[:, 5:8] = maxwell_juttner(rng, n, th).T
    return out


def random_cells(cfg: dict, n_cells: int, seed: int) -> np.ndarray:
    """A seeded random subset of cells (flat indices), for bounded samples."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return np.sort(rng.choice(cfg["n_r"] * cfg["n_theta"], size=n_cells, replace=False))


def probe_particles(cfg: dict, n: int, seed: int, x1_range, x2_range, u_scale: float) -> dict:
    """n test particles at uniform random code positions inside the given
    ranges with isotropic tetrad-frame momenta of uniform magnitude in [0, u_scale]."""
    rng = np.random.Generator(np.random.PCG64(seed))
    x1 = x1_range[0] + (x1_range[1] - x1_range[0]) * rng.random(n)
    x2 = x2_range[0] + (x2_range[1] - x2_range[0]) * rng.random(n)
    i1 = np.floor(x1).astype(np.int32)
    i2 = np.floor(x2).astype(np.int32)
    mag = u_scale * rng.random(n)
    mu = 2.0 * rng.random(n) - 1.0
    ph = 2.0 * math.pi * rng.random(n)
    st = np.sqrt(np.maximum(0.0, 1.0 - mu * mu))
    uhat = np.stack([mag * st * np.cos(ph), mag * st * np.sin(ph), mag * mu])
    return {"pos": {"i1": i1, "i2": i2, "dx1": x1 - i1, "dx2": x2 - i2}, "uhat": uhat,
            "w0": np.ones(n)}
