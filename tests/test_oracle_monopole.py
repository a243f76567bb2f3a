"""Pins of the oracle's monopole field, the initial field of the BZ monopole test (Sec. 4.5:
A_phi = -B0 cos(theta), B^r = B0 sin(theta) / sqrt(h), every other component zero).

* the discrete curl puts exactly the flux of B0 sin(theta) through each cell face: compared
  with the cosine difference in extended precision;
* the flux through any sphere is 2 B0 (the telescoping sum of the face fluxes);
* D, B^2, B^3 vanish (E = 0 and the shift is parallel to B);
* with a = 0 the monopole is a stationary vacuum solution, and the discrete scheme keeps it
  to rounding over many steps (B^1 is independent of theta cell by cell, so every curl of
  the auxiliary field vanishes);
* with a != 0 it is not stationary: the field lines start to rotate (D^3, B^3 grow).
"""
import math

import numpy as np
import pytest

import workloads as W
from oracle import oracle as O

G = O.G


def bz(n=64, a=0.2, **over):
    return dict(W.grid_config("bz1024", n_r=n, n_theta=n, a=a), **over)


@pytest.mark.parametrize("a", [0.0, 0.2, 0.9])
def test_face_flux_is_exact(a):
    cfg = bz(a=a, r_min=1.0 if a < 0.5 else 0.95 * W.horizon_radius(a))
    sim = O.OracleSim(cfg)
    sim.init_fields(O.FIELD_MONOPOLE, 1.3)
    N = cfg["n_theta"]
    # the grid's theta_j = j dtheta with the FP64 dtheta, in extended precision
    dth = np.longdouble(math.pi / N)
    js = np.arange(N)
    exact = np.array([np.longdouble(1.3) * (np.cos(dth * j) - np.cos(dth * (j + 1)))
                      for j in js], dtype=np.longdouble).astype(np.float64)
    # the FP64 face angle (j + 1/2) dtheta is rounded to half an ulp; near theta = pi that is
    # a relative error of up to 2^-53 pi / sin(theta) in the sine
    mid = (js + 0.5) * math.pi / N
    tol = 4e-16 + np.where(mid > math.pi / 2, 2.0 ** -52 * math.pi / np.sin(mid), 0.0)
    for i in (1, 17, cfg["n_r"] - 1):  # i <= n_f is the horizon layer (copies cell n_f + 1)
        sqrt_h = np.array([O.metric_point(cfg, i, j + 0.5)["sqrt_h"] for j in js])
        flux = sim.F[O.B1][G:G + N, i + G] * sqrt_h
        rel = np.abs((flux - exact) / exact)
        assert np.all(rel <= tol), (i, float(rel.max()))
        assert abs(flux.sum() - 2.6) < 1e-14
    for k in (O.B2, O.B3, O.D1, O.D2, O.D3):
        assert not sim.F[k].any(), k


def run_vacuum(cfg, steps):
    sim = O.OracleSim(cfg)
    sim.init_fields(O.FIELD_MONOPOLE, 1.0)
    F0 = sim.F.copy()
    for _ in range(steps):
        sim.predict()
        sim.deposit()
        sim.advance()
    return F0, sim.F


def test_schwarzschild_monopole_is_stationary():
    cfg = bz(a=0.0, r_absorb=1e300)
    F0, F = run_vacuum(cfg, 100)
    b = np.abs(F0[O.B1]).max()
    assert np.abs(F[O.B1] - F0[O.B1]).max() < 1e-13 * b
    for k in (O.B2, O.B3, O.D1, O.D2, O.D3):
        assert np.abs(F[k]).max() < 1e-13 * b, k


def test_spinning_monopole_starts_to_rotate():
    cfg = bz(a=0.2, r_absorb=1e300)
    F0, F = run_vacuum(cfg, 20)
    b = np.abs(F0[O.B1]).max()
    assert np.abs(F[O.D3]).max() > 1e-6 * b or np.abs(F[O.B3]).max() > 1e-6 * b
