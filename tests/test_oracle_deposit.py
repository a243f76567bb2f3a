"""Pins of the oracle's charge-conserving deposit (Sec. 3.2 of arXiv:2511.17701).

* Eq. (charge-conservation-disc): at every node the discrete divergence of the
  deposited conformal current balances the change of sum q S, to rounding;
* single-cell moves: the flux through each face equals the path integral of
  q v S along the straight move, computed here by brute-force quadrature;
* the sum of all fluxes is q times the displacement (zigzag identity);
* J^3 = q alpha u^3 / gamma (Sec. 3.2) in flat spacetime, where u^3 and gamma have
  textbook closed forms.
"""
import math

import numpy as np
import pytest

from oracle import oracle as O

G = O.G


def sim_with_moves(cfg, prev, new, u, w, qc, dt=0.02):
    sim = O.OracleSim(dict(cfg, dt=dt))
    n = len(prev[0])
    arr = {k: np.zeros(n, dtype=t) for k, t in O.PARTICLE_FIELDS.items()}
    for (a, b), x in ((("i1p", "dx1p"), prev[0]), (("i2p", "dx2p"), prev[1]),
                      (("i1", "dx1"), new[0]), (("i2", "dx2"), new[1])):
        i = np.floor(x).astype(np.int32)
        arr[a], arr[b] = i, x - i
    arr["u1"], arr["u2"], arr["u3"] = u
    arr["w"] = w
    arr["tag"][:] = 1
    sim.add_raw_species(arr, 1.0, qc)
    return sim


def random_moves(rng, cfg, n, margin=0.0):
    x1 = rng.uniform(-0.5, cfg["n_r"] + 0.5, n)
    x2 = rng.uniform(0.0, cfg["n_theta"], n)
    d1 = rng.uniform(-0.95, 0.95, n)
    d2 = rng.uniform(-0.95, 0.95, n)
    y1 = x1 + d1
    y2 = np.clip(x2 + d2, 0.0, cfg["n_theta"] - 1e-12)
    return (x1, x2), (y1, y2)


CFG = dict(metric="ks", a=0.9, n_r=40, n_theta=24, r_min=1.3641, r_max=10.0)


def test_discrete_continuity_every_node():
    rng = np.random.default_rng(7)
    n = 3000
    prev, new = random_moves(rng, CFG, n)
    u = rng.normal(size=(3, n))
    sim = sim_with_moves(CFG, prev, new, u, rng.uniform(0.5, 2.0, n), -0.37)
    sim.deposit()
    J1, J2, J3 = sim.F[O.J1], sim.F[O.J2], sim.F[O.J3]
    A1, A2 = sim.F[O.JA1], sim.F[O.JA2]
    r0, r1 = sim.charge(prev=True), sim.charge(prev=False)
    dt = sim.dt
    j0, j1 = G, G + CFG["n_theta"]           # node rows 0 .. n_theta
    i0, i1 = G - 1, G + CFG["n_r"] + 1       # node columns -1 .. n_r + 1
    div = (J1[j0:j1 + 1, i0:i1 + 1] - J1[j0:j1 + 1, i0 - 1:i1]
           + J2[j0:j1 + 1, i0:i1 + 1] - J2[j0 - 1:j1, i0:i1 + 1])
    drho = (r1 - r0)[j0:j1 + 1, i0:i1 + 1] / dt
    scale = (A1[j0:j1 + 1, i0:i1 + 1] + A1[j0:j1 + 1, i0 - 1:i1] + A2[j0:j1 + 1, i0:i1 + 1]
             + A2[j0 - 1:j1, i0:i1 + 1] + 1e-300)
    assert np.max(np.abs(div + drho) / scale) < 1e-13
    assert np.abs(drho).max() > 1.0  # the test moved real charge
    # nothing is deposited across the axes
    assert np.all(J2[:G, :] == 0) and np.all(J2[G + CFG["n_theta"]:, :] == 0)
    # zigzag identity: all radial fluxes add up to q w (x1_b - x1_a) / dt
    qw = -0.37 * sim.species[0].view()["w"]
    assert math.isclose(J1.sum(), np.sum(qw * (new[0] - prev[0])) / dt, rel_tol=1e-12)
    assert math.isclose(J2.sum(), np.sum(qw * (new[1] - prev[1])) / dt, rel_tol=1e-12)


def hat(x):
    return np.maximum(0.0, 1.0 - np.abs(x))


def test_single_cell_moves_equal_path_integral():
    rng = np.random.default_rng(3)
    for _ in range(40):
        i, j = rng.integers(2, 30), rng.integers(1, 20)
        a = np.array([i, j]) + rng.uniform(0.0, 1.0, 2)
        b = np.array([i, j]) + rng.uniform(0.0, 1.0, 2)
        sim = sim_with_moves(CFG, ([a[0]], [a[1]]), ([b[0]], [b[1]]), np.zeros((3, 1)), [1.0],
                             1.0, dt=0.1)
        sim.deposit()
        # brute force: flux through the dual face between nodes (k, l) and (k+1, l) is
        # integral q v1 S(x2(t) - l) dt over the move, divided by dt
        K = 20000
        t = (np.arange(K) + 0.5) / K
        x1 = a[0] + (b[0] - a[0]) * t
        x2 = a[1] + (b[1] - a[1]) * t
        for l in (j, j + 1):
            want = (b[0] - a[0]) * np.mean(hat(x2 - l)) / 0.1
            assert math.isclose(sim.F[O.J1][l + G, i + G], want, rel_tol=1e-9, abs_tol=1e-12)
        for k in (i, i + 1):
            want = (b[1] - a[1]) * np.mean(hat(x1 - k)) / 0.1
            assert math.isclose(sim.F[O.J2][j + G, k + G], want, rel_tol=1e-9, abs_tol=1e-12)


def test_out_of_plane_current_flat():
    """Flat spacetime: u^3 = u_3 / (r^2 sin^2 theta) (dphi = 1), alpha = 1,
    gamma = sqrt(1 + u_r^2 + u_theta^2 / r^2 + u_phi^2 / (r sin theta)^2)."""
    cfg = dict(metric="ks0", a=0.0, n_r=30, n_theta=20, r_min=1.0, r_max=20.0)
    dxi = math.log(cfg["r_max"] / cfg["r_min"]) / cfg["n_r"]
    dth = math.pi / cfg["n_theta"]
    a, b = np.array([11.3, 7.6]), np.array([11.9, 8.2])
    u = np.array([[0.4], [0.3], [2.5]])
    sim = sim_with_moves(cfg, ([a[0]], [a[1]]), ([b[0]], [b[1]]), u, [1.7], 0.5)
    sim.deposit()
    xm = 0.5 * (a + b)
    r, th = cfg["r_min"] * math.exp(xm[0] * dxi), xm[1] * dth
    ur, uth, uph = u[0, 0] / (dxi * r), u[1, 0] / dth, u[2, 0]
    gam = math.sqrt(1 + ur ** 2 + (uth / r) ** 2 + (uph / (r * math.sin(th))) ** 2)
    v3 = uph / (r * math.sin(th)) ** 2 / gam
    q = 0.5 * 1.7
    i0, j0 = 11, 7
    w1, w2 = xm[0] - i0, xm[1] - j0
    want = {(i0, j0): (1 - w1) * (1 - w2), (i0 + 1, j0): w1 * (1 - w2),
            (i0, j0 + 1): (1 - w1) * w2, (i0 + 1, j0 + 1): w1 * w2}
    for (i, j), s in want.items():
        assert math.isclose(sim.F[O.J3][j + G, i + G], q * v3 * s, rel_tol=1e-12)
    assert math.isclose(sim.F[O.J3].sum(), q * v3, rel_tol=1e-12)
