"""Pins of the oracle's time step (ora_time_step): the CFL rule of reading R18,
dt = CFL * min over cell centres of 1 / (alpha sqrt(h^11 + h^22) + |beta^1|) in code units.

The checks do not use the oracle's 3+1 closed forms:
* flat space on the log-r grid (kerr_schild_0): alpha = 1, beta = 0, h^11 = 1/(dxi r)^2,
  h^22 = 1/(dtheta r)^2, so the minimum sits on the innermost column and has a closed form;
* Kerr: the 3+1 quantities are taken from the inverse of the Appendix A 4-metric, retyped in
  physical Kerr-Schild coordinates (alpha = (-g^00)^(-1/2), beta^i = -g^0i / g^00,
  h^ij = g^ij - g^0i g^0j / g^00) and mapped to code units by dr/dx1 = dxi r, dtheta/dx2 =
  dtheta;
* what the rule means: at the cell the minimum selects, alpha sqrt(h^11 + h^22) + beta^1 is the
  fastest coordinate speed -(dx^1/dt + dx^2/dt) of a future null ray (the light cone read off
  the covariant 4-metric by brute force over directions), so dt is CFL times the time light
  needs to cross one cell diagonal inwards.
"""
import math

import numpy as np
import pytest

from oracle import oracle as O
from test_oracle_metric import kerr_schild_4metric

import workloads as W


def _grid(cfg):
    dxi = math.log(cfg["r_max"] / cfg["r_min"]) / cfg["n_r"]
    dth = math.pi / cfg["n_theta"]
    return dxi, dth


@pytest.mark.parametrize("n_r,n_th,r_min,r_max", [(64, 64, 1.0, 10.0), (50, 40, 1.0, 20.0),
                                                  (37, 91, 2.5, 7.0)])
def test_flat_closed_form(n_r, n_th, r_min, r_max):
    cfg = dict(metric="ks0", a=0.0, n_r=n_r, n_theta=n_th, r_min=r_min, r_max=r_max)
    dxi, dth = _grid(cfg)
    r_c = r_min * math.exp(0.5 * dxi)  # centre of the innermost column
    want = 0.5 * r_c / math.sqrt(dxi ** -2 + dth ** -2)
    assert math.isclose(O.time_step(cfg, 0.5), want, rel_tol=1e-13)
    assert math.isclose(O.time_step(cfg, 0.25), 0.5 * want, rel_tol=1e-13)


def _split_code(a, r, th, dxi, dth):
    """alpha, beta^1 and h^11, h^22 in code units from the inverse 4-metric."""
    _, gi = kerr_schild_4metric(a, 1.0, r, th)
    alpha = (-gi[0, 0]) ** -0.5
    beta_r = -gi[0, 1] / gi[0, 0]
    h_rr = gi[1, 1] - gi[0, 1] ** 2 / gi[0, 0]
    h_tt = gi[2, 2] - gi[0, 2] ** 2 / gi[0, 0]
    f = dxi * r
    return alpha, beta_r / f, h_rr / f ** 2, h_tt / dth ** 2


def _speed_from_split(a, r, th, dxi, dth):
    al, b1, H11, H22 = _split_code(a, r, th, dxi, dth)
    return al * math.sqrt(H11 + H22) + abs(b1)


@pytest.mark.parametrize("name,cols", [("wald64", None), ("wald512", 4)])
def test_kerr_against_appendix_4metric(name, cols):
    """Every cell of the 64^2 grid; on the 512^2 grid every row of the four innermost columns
    and of every 16th column (the minimum sits on the innermost column)."""
    cfg = W.grid_config(name)
    dxi, dth = _grid(cfg)
    n_r = cfg["n_r"]
    cols = range(n_r) if cols is None else sorted(set(range(cols)) | set(range(0, n_r, 16)))
    best, arg = math.inf, None
    for ii in cols:
        r = cfg["r_min"] * math.exp((ii + 0.5) * dxi)
        for jj in range(cfg["n_theta"]):
            v = 1.0 / _speed_from_split(cfg["a"], r, (jj + 0.5) * dth, dxi, dth)
            if v < best:
                best, arg = v, (ii, jj)
    dt = O.time_step(cfg, 0.5)
    assert math.isclose(dt, 0.5 * best, rel_tol=1e-12), (dt, 0.5 * best, arg)
    assert arg[0] == 0


def _max_null_speed(a, r, th, dxi, dth):
    """max over future null rays of -(dx^1/dt + dx^2/dt) in code coordinates, by brute force
    over spatial directions: for a direction d, k = (1, l d) is null for the positive root l
    of g_00 + 2 l g_0i d^i + l^2 g_ij d^i d^j = 0."""
    g, _ = kerr_schild_4metric(a, 1.0, r, th)
    J = np.diag([1.0, dxi * r, dth, 1.0])  # physical = J code
    gc = J.T @ g @ J

    def speed(u, v):
        # every null k = (1, k^i) is l d for d = k / |k| and a root l > 0; inside the
        # ergoregion (g_00 > 0) both roots of a direction can be positive, or none real
        d = np.array([math.cos(u) * math.cos(v), math.cos(u) * math.sin(v), math.sin(u)])
        A = d @ gc[1:, 1:] @ d
        B = 2.0 * (gc[0, 1:] @ d)
        Cc = gc[0, 0]
        disc = B * B - 4.0 * A * Cc
        if disc < 0.0:
            return -math.inf
        best = -math.inf
        for lam in ((-B + math.sqrt(disc)) / (2.0 * A), (-B - math.sqrt(disc)) / (2.0 * A)):
            if lam > 0.0:
                best = max(best, -(lam * d[0] + lam * d[1]))
        return best

    best, arg = -math.inf, None
    for u in np.linspace(-1.5, 1.5, 61):
        for v in np.linspace(0.0, 2.0 * math.pi, 121):
            s = speed(u, v)
            if s > best:
                best, arg = s, (u, v)
    from scipy.optimize import minimize
    res = minimize(lambda x: -speed(x[0], x[1]) if math.isfinite(speed(x[0], x[1])) else 1e300,
                   np.array(arg), method="Nelder-Mead",
                   options={"xatol": 1e-12, "fatol": 1e-15, "maxiter": 20000})
    return -res.fun


@pytest.mark.parametrize("a,r,th", [(0.9, 1.45, 0.5 * math.pi), (0.9, 1.4, 0.05),
                                    (0.0, 3.0, 1.0), (0.5, 7.0, 2.7)])
def test_rule_is_the_fastest_inward_null_speed(a, r, th):
    dxi, dth = 0.01, math.pi / 128
    want = _speed_from_split(a, r, th, dxi, dth)
    got = _max_null_speed(a, r, th, dxi, dth)
    assert math.isclose(got, want, rel_tol=1e-8), (got, want)


def test_selected_cell_is_a_null_crossing_time():
    """The cell the oracle's minimum selects on the wald64 grid: CFL over the brute-force
    null speed there equals the oracle's dt."""
    cfg = W.grid_config("wald64")
    dxi, dth = _grid(cfg)
    dt = O.time_step(cfg, 0.5)
    r0 = cfg["r_min"] * math.exp(0.5 * dxi)
    cands = [(j + 0.5) * dth for j in range(cfg["n_theta"])]
    vals = [0.5 / _speed_from_split(cfg["a"], r0, th, dxi, dth) for th in cands]
    th = cands[int(np.argmin(vals))]
    assert math.isclose(dt, 0.5 / _max_null_speed(cfg["a"], r0, th, dxi, dth), rel_tol=1e-8)


def test_schwarzschild_radial_light_speed_is_one():
    """a = 0: alpha sqrt(h^rr) + beta^r = 1/(1+z) + z/(1+z) = 1 in physical units at every r,
    so with a huge theta cell the rule gives dt = CFL dxi r_c on the innermost column."""
    cfg = dict(metric="ks", a=0.0, n_r=40, n_theta=1, r_min=1.8, r_max=20.0)
    dxi = math.log(cfg["r_max"] / cfg["r_min"]) / cfg["n_r"]
    dth = math.pi
    for r in (1.9, 3.0, 11.0):
        al, b1, H11, _ = _split_code(0.0, r, 1.0, dxi, dth)
        assert math.isclose(al * math.sqrt(H11) + b1, 1.0 / (dxi * r), rel_tol=1e-14)
