"""Pins of the oracle's charge-conserving deposit (Sec. 3.2 of arXiv:2511.17701).

* Eq. (charge-conservation-disc): at every node the discrete divergence of the
  deposited conformal current balances the change of sum q S, to rounding;
* single-cell moves: the flux through each face equals the path integral of
  q v S along the straight move, computed here by brute-force quadrature;
* the sum of all fluxes is q times the displacement (zigzag identity);
* the deposit test of Sec. 4.3: the flux of D through r ~ 10 around an a = 0.95 black hole
  is 4 pi times the charge inside while one particle of a pair is inside, and returns to
  zero once both have crossed the horizon;
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


def gauss_areas(cfg, i):
    """The face areas of the surface x1 = i + 1/2 at the node rows: sqrt(h) at (i + 1/2, j),
    the polar areas of the half cells at the axis rows."""
    N = cfg["n_theta"]
    return np.array([O.polar_area(cfg, i + 0.5) if j in (0, N) else
                     O.metric_point(cfg, i + 0.5, j)["sqrt_h"] for j in range(N + 1)])


def gauss_flux(osim, areas, i):
    """The flux of sqrt(h) D^1 through the surface x1 = i + 1/2: the discrete divergence of
    sqrt(h) D summed over the nodes inside telescopes to it."""
    return float(areas @ osim.F[O.D1][G:G + len(areas), i + G])


def test_pair_falling_into_a_spinning_black_hole_leaves_no_flux():
    """The deposit test of Sec. 4.3: an e- e+ pair starts at r = 17, theta = pi/2 around an
    a = 0.95 black hole with no field. Here both move inward (tetrad-frame u_r = -1 and -3;
    the paper reflects the outgoing electron at the outer boundary, which is not a boundary
    of the method). The flux of D^1 through r ~ 10 is 4 pi times the charge inside while
    exactly one particle is inside (Gauss, discrete and exact), and returns to zero, to
    rounding, once both have crossed the horizon and been removed."""
    import workloads as W
    a = 0.95
    cfg = dict(metric="ks", a=a, n_r=56, n_theta=36, r_min=0.85 * W.horizon_radius(a),
               r_max=24.0, r_absorb=21.0, cfl=0.5)
    osim = O.OracleSim(cfg)
    osim.init_fields(O.FIELD_ZERO, 0.0)
    dxi = math.log(cfg["r_max"] / cfg["r_min"]) / cfg["n_r"]
    x1 = math.log(17.0 / cfg["r_min"]) / dxi
    x2 = cfg["n_theta"] / 2 + 0.5
    pos = {"i1": np.array([int(x1)], np.int32), "i2": np.array([int(x2)], np.int32),
           "dx1": np.array([x1 - int(x1)]), "dx2": np.array([x2 - int(x2)])}
    # a weakly coupled pair (skin depth 10 r_g): its own attraction does not keep it together
    qe, ce = W.species_coefficients(-1.0, 1.0, 10.0)
    qp, cp = W.species_coefficients(+1.0, 1.0, 10.0)
    osim.add_species(pos, np.array([[-1.0], [0.0], [0.0]]), np.array([1.0]), qe, ce)
    osim.add_species(pos, np.array([[-3.0], [0.0], [0.0]]), np.array([1.0]), qp, cp)
    i10 = int(math.log(10.0 / cfg["r_min"]) / dxi)
    areas = gauss_areas(cfg, i10)
    flux, checked = [], 0
    for _ in range(int(50.0 / osim.dt)):
        osim.step(1)
        f = gauss_flux(osim, areas, i10)
        flux.append(f)
        e, p = osim.species[0].view(), osim.species[1].view()
        xe, xp = e["i1"][0] + e["dx1"][0], p["i1"][0] + p["dx1"][0]
        if p["tag"][0] == 1 and e["tag"][0] == 1 and xp < i10 and xe >= i10 + 1:
            # the positron's charge is all on nodes i <= i10, the electron's on nodes above:
            # the flux is 4 pi qc w of the positron
            assert f == pytest.approx(4 * math.pi * cp * p["w"][0], rel=1e-10)
            checked += 1
    assert checked > 5
    assert osim.counters[0] == 2  # both removed through the horizon layer
    flux = np.abs(np.array(flux))
    assert flux.max() > 0.1
    assert flux[-50:].max() < 1e-12 * flux.max()
