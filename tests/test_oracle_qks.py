"""Pins of the quasi-spherical Kerr-Schild grid (App. A): r = r0 + exp(xi) with xi uniform in
x1, theta = eta + 2 h0 eta (pi - 2 eta)(pi - eta) / pi^2 with eta uniform in x2.

* the map: endpoints r_min, r_max, 0, pi; theta(pi - eta) = pi - theta(eta); cells at the
  equator 1 - h0 and at the axes 1 + 2 h0 times the uniform size; dr/dx1 and dtheta/dx2
  against finite differences of r and theta;
* the code-unit metric is the Kerr-Schild metric in the new coordinates: at every point the
  physical components equal those of the plain grid at the same (r, theta);
* a circular equatorial geodesic (Bardeen, Press & Teukolsky) stays a fixed point of the
  implicit push in the new coordinates, with phi advancing at its angular frequency;
* the Wald vacuum stays stationary with second-order convergence, and the discrete Gauss law
  holds through full PIC steps with particles, on the new grid.
(The derivative, inverse, 4-metric and polar-area pins of test_oracle_metric.py include two
quasi-spherical grids.)
"""
import math

import numpy as np
import pytest
from scipy.optimize import brentq

import workloads as W
from oracle import oracle as O
from test_oracle_pusher import bl_state, bpt_circular

G = O.G
QKS = W.grid_config("wald64", r0=0.4, h0=0.45)


def eta_of_theta(cfg, th):
    h0 = cfg.get("h0", 0.0)
    f = lambda e: e + 2 * h0 * e * (math.pi - 2 * e) * (math.pi - e) / math.pi ** 2 - th
    return brentq(f, 0.0, math.pi, xtol=1e-15, rtol=1e-15)


def x_of(cfg, r, th):
    r0 = cfg.get("r0", 0.0)
    dxi = math.log((cfg["r_max"] - r0) / (cfg["r_min"] - r0)) / cfg["n_r"]
    x1 = math.log((r - r0) / (cfg["r_min"] - r0)) / dxi
    x2 = eta_of_theta(cfg, th) / (math.pi / cfg["n_theta"])
    return x1, x2


def test_map_endpoints_symmetry_and_concentration():
    n, N = QKS["n_r"], QKS["n_theta"]
    assert O.metric_point(QKS, 0.0, 10.0)["r"] == pytest.approx(QKS["r_min"], rel=1e-15)
    assert O.metric_point(QKS, n, 10.0)["r"] == pytest.approx(QKS["r_max"], rel=1e-14)
    assert O.metric_point(QKS, 5.0, 0.0)["th"] == 0.0
    assert O.metric_point(QKS, 5.0, N)["th"] == pytest.approx(math.pi, rel=1e-15)
    assert O.metric_point(QKS, 5.0, N / 2)["th"] == pytest.approx(math.pi / 2, rel=1e-15)
    for x2 in (0.3, 7.7, 19.2):
        a, b = O.metric_point(QKS, 5.0, x2)["th"], O.metric_point(QKS, 5.0, N - x2)["th"]
        assert a + b == pytest.approx(math.pi, rel=1e-15)
    de, h0 = math.pi / N, QKS["h0"]
    assert O.metric_point(QKS, 5.0, N / 2)["g"] == pytest.approx(de * (1 - h0), rel=1e-14)
    assert O.metric_point(QKS, 5.0, 0.0)["g"] == pytest.approx(de * (1 + 2 * h0), rel=1e-14)


def test_map_derivatives_against_finite_differences():
    e = 1e-3
    for x1, x2 in ((0.5, 0.5), (20.2, 13.7), (55.0, 32.0), (63.1, 60.9)):
        m = O.metric_point(QKS, x1, x2)
        r = [O.metric_point(QKS, x1 + k * e, x2)["r"] for k in (-2, -1, 1, 2)]
        t = [O.metric_point(QKS, x1, x2 + k * e)["th"] for k in (-2, -1, 1, 2)]
        fd_r = (r[0] - 8 * r[1] + 8 * r[2] - r[3]) / (12 * e)
        fd_t = (t[0] - 8 * t[1] + 8 * t[2] - t[3]) / (12 * e)
        assert fd_r == pytest.approx(m["f"], rel=1e-10)
        assert fd_t == pytest.approx(m["g"], rel=1e-10)


@pytest.mark.parametrize("a", [0.0, 0.9])
def test_metric_is_kerr_schild_in_the_new_coordinates(a):
    q = dict(QKS, a=a)
    k = dict(W.grid_config("wald64", a=a), r_min=q["r_min"] - 0.2)
    for x1, x2 in ((3.3, 2.2), (20.2, 13.7), (41.0, 33.3), (60.5, 61.4)):
        mq = O.metric_point(q, x1, x2)
        y1, y2 = x_of(k, mq["r"], mq["th"])
        mk = O.metric_point(k, y1, y2)
        assert mk["r"] == pytest.approx(mq["r"], rel=1e-13)
        assert mk["th"] == pytest.approx(mq["th"], rel=1e-12)
        fq, gq, fk, gk = mq["f"], mq["g"], mk["f"], mk["g"]
        pairs = [("h11", fq * fq, fk * fk), ("h13", fq, fk), ("h22", gq * gq, gk * gk),
                 ("h33", 1.0, 1.0), ("H11", 1 / fq ** 2, 1 / fk ** 2), ("H13", 1 / fq, 1 / fk),
                 ("H22", 1 / gq ** 2, 1 / gk ** 2), ("H33", 1.0, 1.0), ("alpha", 1.0, 1.0),
                 ("beta1", 1 / fq, 1 / fk), ("sqrt_h", fq * gq, fk * gk)]
        for key, sq, sk in pairs:
            assert mq[key] / sq == pytest.approx(mk[key] / sk, rel=1e-11, abs=1e-14), key


@pytest.mark.parametrize("a,r,pro", [(0.9, 8.0, True), (0.5, 6.5, False)])
def test_circular_geodesic_is_a_fixed_point_on_the_new_grid(a, r, pro):
    cfg = dict(QKS, a=a, n_r=256, n_theta=256, r_max=30.0, dt=0.05, n_iter=10,
               small_angle=1e-5)
    E, L = bpt_circular(a, r, pro)
    u_t, u_r, _ = bl_state(a, r, math.pi / 2, L)
    x1, x2 = x_of(cfg, r, math.pi / 2)
    m = O.metric_point(cfg, x1, x2)
    u = np.array([m["f"] * u_r, 0.0, L])
    sim = O.OracleSim(cfg)
    i1, i2 = int(x1), int(x2)
    arr = {k: np.zeros(1, dtype=t) for k, t in O.PARTICLE_FIELDS.items()}
    arr.update(i1=[i1], i2=[i2], dx1=[x1 - i1], dx2=[x2 - i2], u1=[u[0]], u2=[0.0], u3=[L],
               tag=[1], w=[1.0])
    for k in ("i1", "i2", "dx1", "dx2"):
        arr[k + "p"] = arr[k]
    sim.add_raw_species(arr, 0.0, 0.0)
    for _ in range(400):
        sim.push(0, field_mode=1, fkind=0)
    s = sim.species[0].view()
    assert abs(s["i1"][0] + s["dx1"][0] - x1) < 1e-9 * x1
    assert abs(s["i2"][0] + s["dx2"][0] - x2) < 1e-9
    assert np.allclose([s["u1"][0], s["u2"][0], s["u3"][0]], u, rtol=1e-10, atol=1e-12)
    Om = (1.0 if pro else -1.0) / (r ** 1.5 + (a if pro else -a))
    assert s["phi"][0] == pytest.approx(400 * 0.05 * Om, rel=1e-9)


def test_wald_vacuum_converges_on_the_new_grid():
    errs = {}
    for n in (32, 64):
        cfg = dict(QKS, n_r=n, n_theta=n, r_absorb=1e300)
        sim = O.OracleSim(cfg)
        sim.init_fields(O.FIELD_WALD, 1.0)
        F0 = sim.F.copy()
        for _ in range(int(round(4.0 / sim.dt))):
            sim.predict()
            sim.deposit()
            sim.advance()
        r = np.array([O.metric_point(cfg, i, 1.0)["r"] for i in range(-G, n + G + 1)])
        mask = (r > 2.5) & (r < 6.0)
        errs[n] = np.array([
            np.abs(sim.F[c] - F0[c])[G:G + n + 1][:, mask].max()
            / np.abs(F0[c])[G:G + n + 1][:, mask].max() for c in range(6)])
    ratio = errs[32] / errs[64]
    assert np.all(ratio > 2.4), ratio
    assert np.all(errs[64] < 0.05), errs[64]


def test_gauss_law_through_full_steps_on_the_new_grid():
    from test_oracle_fields import gauss_div
    cfg = dict(QKS, n_r=40, n_theta=24, ppc=4, r_absorb=8.0)
    sim = O.OracleSim(cfg)
    sim.init_fields(O.FIELD_WALD, 1.0)
    pl = W.pair_plasma(cfg)
    for s in range(2):
        sim.add_species(pl["pos"], pl["uhat"][s], pl["w0"], pl["qm"][s], pl["qc"][s])
    i_hi = int(x_of(cfg, cfg["r_absorb"], 1.0)[0]) - 2
    for step in range(3):
        sim.predict()
        sim.push(0)
        sim.push(1)
        sim.deposit()
        rho0, rho1 = sim.charge(prev=True), sim.charge(prev=False)
        D0 = [sim.F[O.D1 + c].copy() for c in range(3)]
        sim.advance()
        D1 = [sim.F[O.D1 + c] for c in range(3)]
        lhs = gauss_div(sim, cfg, D1) - gauss_div(sim, cfg, D0)
        rhs = 4 * math.pi * (rho1 - rho0)[G:G + cfg["n_theta"] + 1, G:G + cfg["n_r"] + 1]
        err = np.abs(lhs - rhs)[:, 2:i_hi]
        scale = np.abs(rhs)[:, 2:i_hi].max()
        assert scale > 0 and err.max() < 1e-11 * scale, (step, err.max(), scale)
