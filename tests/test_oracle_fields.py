"""Pins of the oracle's field solver and PIC loop (Secs. 3.3-3.4 of arXiv:2511.17701).

* div B = 0: the discrete curl of the potential initialises B^1, B^2 without
  divergence and Faraday's discrete curl keeps it (round-off);
* Gauss's law with the deposit: after a full step the change of the discrete
  divergence of sqrt(h) D equals 4 pi times the change of the deposited charge at
  every interior node, the axis nodes included (round-off);
* the Wald vacuum solution (Sec. 4.2) stays stationary, with a departure that
  falls with resolution at second order.
"""
import math

import numpy as np

import workloads as W
from oracle import oracle as O

G = O.G


def sqrt_h_plane(cfg, s1, s2, rows, cols):
    out = np.zeros((len(rows), len(cols)))
    for a, j in enumerate(rows):
        for b, i in enumerate(cols):
            out[a, b] = O.metric_point(cfg, i + s1, j + s2)["sqrt_h"]
    return out


def div_B(sim, cfg):
    n_r, n_t = cfg["n_r"], cfg["n_theta"]
    # cells (i + 1/2, j + 1/2) with i in [1, n_r - 1]: off the horizon layer (i <= n_f = 0,
    # copied from i = 1) and off the outer ghost cells (held at the initial field)
    rows, cols = np.arange(0, n_t), np.arange(1, n_r)
    sh1 = sqrt_h_plane(cfg, 0.0, 0.5, rows, np.arange(1, n_r + 1))
    sh2 = sqrt_h_plane(cfg, 0.5, 0.0, np.arange(0, n_t + 1), cols)
    B1 = sim.F[O.B1][G:G + n_t, G + 1:G + n_r + 1] * sh1
    B2 = sim.F[O.B2][G:G + n_t + 1, G + 1:G + n_r] * sh2
    div = (B1[:, 1:] - B1[:, :-1]) + (B2[1:, :] - B2[:-1, :])
    scale = np.abs(B1[:, 1:]) + np.abs(B1[:, :-1]) + np.abs(B2[1:, :]) + np.abs(B2[:-1, :])
    return np.max(np.abs(div) / (scale + 1e-300))


def test_div_B_vanishes_initially_and_after_steps():
    # no absorbing layer: its per-component damping does not keep div B = 0
    cfg = W.grid_config("wald64", n_r=40, n_theta=24, r_absorb=1e300)
    sim = O.OracleSim(cfg)
    sim.init_fields(O.FIELD_WALD, 1.0)
    assert div_B(sim, cfg) < 1e-13
    for _ in range(20):
        sim.predict()
        sim.deposit()
        sim.advance()
    assert div_B(sim, cfg) < 1e-12


def gauss_div(sim, cfg, D):
    """div(sqrt(h) D) at nodes (i, j); on the axes the half cell uses the polar area."""
    n_r, n_t = cfg["n_r"], cfg["n_theta"]
    out = np.zeros((n_t + 1, n_r + 1))
    for j in range(n_t + 1):
        for i in range(1, n_r):
            if j in (0, n_t):
                Ap, Am = O.polar_area(cfg, i + 0.5), O.polar_area(cfg, i - 0.5)
                sgn = 1.0 if j == 0 else -1.0
                jj = 0 if j == 0 else n_t - 1
                d2 = sgn * O.metric_point(cfg, i, jj + 0.5)["sqrt_h"] * D[1][jj + G, i + G]
                out[j, i] = Ap * D[0][j + G, i + G] - Am * D[0][j + G, i - 1 + G] + d2
            else:
                m1p = O.metric_point(cfg, i + 0.5, j)["sqrt_h"]
                m1m = O.metric_point(cfg, i - 0.5, j)["sqrt_h"]
                m2p = O.metric_point(cfg, i, j + 0.5)["sqrt_h"]
                m2m = O.metric_point(cfg, i, j - 0.5)["sqrt_h"]
                out[j, i] = (m1p * D[0][j + G, i + G] - m1m * D[0][j + G, i - 1 + G]
                             + m2p * D[1][j + G, i + G] - m2m * D[1][j - 1 + G, i + G])
    return out


def test_gauss_law_holds_through_a_full_step():
    cfg = W.grid_config("wald64", n_r=40, n_theta=24, ppc=4, r_absorb=8.0)
    sim = O.OracleSim(cfg)
    sim.init_fields(O.FIELD_WALD, 1.0)
    pl = W.pair_plasma(cfg)
    for s in range(2):
        sim.add_species(pl["pos"], pl["uhat"][s], pl["w0"], pl["qm"][s], pl["qc"][s])
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
        dxi = math.log(cfg["r_max"] / cfg["r_min"]) / cfg["n_r"]
        i_hi = int(math.log(cfg["r_absorb"] / cfg["r_min"]) / dxi) - 2  # stay off MATCH
        sl = (slice(None), slice(cfg["n_filter"] + 2 if "n_filter" in cfg else 2, i_hi))
        err = np.abs(lhs - rhs)[sl]
        scale = np.abs(rhs)[sl].max()
        assert scale > 0
        assert err.max() < 1e-11 * scale, (step, err.max(), scale)
        assert np.abs(rhs[0]).max() > 0 and np.abs(rhs[-1]).max() > 0  # axes carry charge


def test_wald_vacuum_stays_stationary_second_order():
    errs = {}
    for n in (32, 64):
        cfg = W.grid_config("wald64", n_r=n, n_theta=n, r_absorb=1e300)
        sim = O.OracleSim(cfg)
        sim.init_fields(O.FIELD_WALD, 1.0)
        F0 = sim.F.copy()
        for _ in range(int(round(4.0 / sim.dt))):
            sim.predict()
            sim.deposit()
            sim.advance()
        dxi = math.log(cfg["r_max"] / cfg["r_min"]) / n
        r = cfg["r_min"] * np.exp(np.arange(-G, n + G + 1) * dxi)
        mask = (r > 2.5) & (r < 6.0)
        errs[n] = np.array([
            np.abs(sim.F[c] - F0[c])[G:G + n + 1][:, mask].max()
            / np.abs(F0[c])[G:G + n + 1][:, mask].max() for c in range(6)])
    ratio = errs[32] / errs[64]
    assert np.all(ratio > 2.4), ratio
    assert ratio[0] > 3.5 and ratio[3] > 3.5, ratio  # B^r and D^r: clean second order
    assert np.all(errs[64] < 0.05), errs[64]


def test_initial_B3_equals_the_plain_curl_in_extended_precision():
    """B^3 = -(A_1(j+1) - A_1(j)) / sqrt(h) at (i+1/2, j+1/2): the oracle takes the cell
    difference of the Wald A_1 in product form; here the plain difference of the potential's
    closed form (Eq. Wald, A_r = (B0 a / 2)(2 z - (1 + z) sin^2), A_1 = f A_r) is evaluated in
    extended precision, where its cancellation next to the axes costs nothing at this
    resolution. Rows at both axes and in the middle, 2048 cells in theta."""
    cfg = W.grid_config("wald64", n_r=16, n_theta=2048, r_max=200.0, r_absorb=1e300)
    osim = O.OracleSim(cfg)
    osim.init_fields(O.FIELD_WALD, 1.0)
    L = np.longdouble
    a, M, B0 = L(cfg["a"]), L(1), L(1)
    dxi = L(math.log(cfg["r_max"] / cfg["r_min"]) / cfg["n_r"])
    dth = L(np.pi) / L(cfg["n_theta"])   # np.pi rounded to double, as the oracle's pi
    nt = cfg["n_theta"]

    def A1(x1, j):
        r = L(cfg["r_min"]) * np.exp(L(x1) * dxi)
        s, c = np.sin(L(j) * dth), np.cos(L(j) * dth)
        z = 2 * M * r / (r * r + a * a * c * c)
        return dxi * r * B0 * a / 2 * (2 * z - (1 + z) * s * s)

    rows = list(range(0, 6)) + list(range(nt // 2 - 3, nt // 2 + 3)) + list(range(nt - 6, nt))
    worst = 0.0
    for i in range(1, cfg["n_r"], 3):  # i <= 0 is the horizon layer (a copy of cell 1)
        for j in rows:
            m = O.metric_point(cfg, i + 0.5, j + 0.5)
            ref = float(-(A1(i + 0.5, j + 1) - A1(i + 0.5, j))) / m["sqrt_h"]
            got = osim.F[O.B3][j + G, i + G]
            worst = max(worst, abs(got - ref) / abs(ref))
    # next to theta = pi the rounding of the argument (2j + 1) dtheta ~ pi leaves ~1e-13 of
    # sin(theta_a + theta_b); the plain double difference is off by ~5e-11 there
    assert worst < 5e-13, worst
