"""Pins of the oracle's metric and tetrads (Appendix A of arXiv:2511.17701).

The oracle builds the 3+1 quantities from physical closed forms and the chain
rule. Here they are checked against things the oracle does not compute: the
4-metric matrices of Appendix A retyped in physical coordinates (the 3+1 split
must reproduce them), the textbook Schwarzschild and flat limits, numerical
determinants, finite differences and orthonormality of the tetrad.
"""
import math

import numpy as np
import pytest

from oracle import oracle as O

CASES = [
    dict(metric="ks", a=0.9, n_r=64, n_theta=64, r_min=1.3641, r_max=10.0),
    dict(metric="ks", a=0.995, n_r=512, n_theta=512, r_min=1.0, r_max=15.0),
    dict(metric="ks", a=0.0, n_r=100, n_theta=80, r_min=1.8, r_max=20.0),
    dict(metric="ks0", a=0.0, n_r=50, n_theta=40, r_min=1.0, r_max=20.0),
    # quasi-spherical grids of App. A: radial offset r0 and equatorial concentration h0
    dict(metric="ks", a=0.9, n_r=64, n_theta=64, r_min=1.3641, r_max=10.0, r0=0.4, h0=0.45),
    dict(metric="ks", a=0.5, n_r=80, n_theta=60, r_min=1.2, r_max=30.0, r0=-1.0, h0=0.8),
]
PTS = [(0.3, 0.7), (10.5, 3.25), (33.3, 17.9), (40.0, 31.5), (47.9, 5.1)]


def kerr_schild_4metric(a, M, r, th):
    """g_{mu nu} and g^{mu nu} of Appendix A (physical KS coordinates t, r, theta, phi)."""
    s, c = math.sin(th), math.cos(th)
    Sig = r * r + a * a * c * c
    Del = r * r - 2 * M * r + a * a
    A = (r * r + a * a) ** 2 - a * a * Del * s * s
    z = 2 * M * r / Sig
    g = np.array([[-(1 - z), z, 0, -a * z * s * s],
                  [z, 1 + z, 0, -a * (1 + z) * s * s],
                  [0, 0, Sig, 0],
                  [-a * z * s * s, -a * (1 + z) * s * s, 0, A * s * s / Sig]])
    gi = np.array([[-(1 + z), z, 0, 0],
                   [z, Del / Sig, 0, a / Sig],
                   [0, 0, 1 / Sig, 0],
                   [0, a / Sig, 0, 1 / (Sig * s * s)]])
    return g, gi


def physical(m):
    """3+1 quantities of the oracle, converted from code units to physical (r, theta)."""
    f, g = m["f"], m["g"]
    h = np.array([[m["h11"] / f ** 2, 0, m["h13"] / f], [0, m["h22"] / g ** 2, 0],
                  [m["h13"] / f, 0, m["h33"]]])
    H = np.array([[m["H11"] * f ** 2, 0, m["H13"] * f], [0, m["H22"] * g ** 2, 0],
                  [m["H13"] * f, 0, m["H33"]]])
    beta = np.array([m["beta1"] * f, 0.0, 0.0])
    return h, H, m["alpha"], beta


@pytest.mark.parametrize("cfg", CASES)
@pytest.mark.parametrize("pt", PTS)
def test_inverse_and_determinant(cfg, pt):
    x1 = pt[0] * cfg["n_r"] / 50.0
    x2 = pt[1] * cfg["n_theta"] / 32.0
    m = O.metric_point(cfg, x1, x2)
    h = np.array([[m["h11"], 0, m["h13"]], [0, m["h22"], 0], [m["h13"], 0, m["h33"]]])
    H = np.array([[m["H11"], 0, m["H13"]], [0, m["H22"], 0], [m["H13"], 0, m["H33"]]])
    assert np.allclose(h @ H, np.eye(3), rtol=0, atol=1e-13)
    assert math.isclose(math.sqrt(np.linalg.det(h)), m["sqrt_h"], rel_tol=1e-12)
    assert math.isclose(m["sqrt_h"], m["sqrt_ht"] * math.sin(m["th"]), rel_tol=1e-14)


@pytest.mark.parametrize("cfg", CASES[:3] + CASES[4:])
@pytest.mark.parametrize("pt", PTS)
def test_split_reproduces_appendix_4metric(cfg, pt):
    """g^00 = -1/alpha^2, g^0i = beta^i/alpha^2, g^ij = h^ij - beta^i beta^j/alpha^2,
    g_00 = -alpha^2 + beta_k beta^k, g_0i = h_ij beta^j, g_ij = h_ij (Sec. 2.1)."""
    x1 = pt[0] * cfg["n_r"] / 50.0
    x2 = pt[1] * cfg["n_theta"] / 32.0
    m = O.metric_point(cfg, x1, x2)
    g4, gi4 = kerr_schild_4metric(cfg["a"], 1.0, m["r"], m["th"])
    assert np.allclose(g4 @ gi4, np.eye(4), atol=1e-12)  # the retyped matrices themselves
    h, H, al, be = physical(m)
    gi = np.zeros((4, 4))
    gi[0, 0] = -1 / al ** 2
    gi[0, 1:] = gi[1:, 0] = be / al ** 2
    gi[1:, 1:] = H - np.outer(be, be) / al ** 2
    bl = h @ be
    g = np.zeros((4, 4))
    g[0, 0] = -al ** 2 + bl @ be
    g[0, 1:] = g[1:, 0] = bl
    g[1:, 1:] = h
    assert np.allclose(gi, gi4, rtol=1e-12, atol=1e-12)
    assert np.allclose(g, g4, rtol=1e-12, atol=1e-12)
    # sqrt(-g) = alpha sqrt(h) = Sigma sin(theta) (Sec. 2.1 and Appendix A)
    Sig = m["r"] ** 2 + cfg["a"] ** 2 * math.cos(m["th"]) ** 2
    assert math.isclose(al * m["sqrt_h"] / (m["f"] * m["g"]), Sig * math.sin(m["th"]),
                        rel_tol=1e-13)


def test_schwarzschild_and_flat_limits():
    cfg = CASES[2]
    m = O.metric_point(cfg, 37.0, 23.0)
    r = m["r"]
    h, H, al, be = physical(m)
    assert math.isclose(H[0, 0], r / (r + 2), rel_tol=1e-14)
    assert math.isclose(al, math.sqrt(r / (r + 2)), rel_tol=1e-14)
    assert math.isclose(be[0], 2 / (r + 2), rel_tol=1e-14)
    assert H[0, 2] == 0.0 and h[0, 2] == 0.0
    cfg0 = CASES[3]
    m = O.metric_point(cfg0, 17.0, 9.0)
    h, H, al, be = physical(m)
    r, s = m["r"], math.sin(m["th"])
    assert np.allclose(np.diag(h), [1.0, r * r, r * r * s * s], rtol=1e-14)
    assert al == 1.0 and be[0] == 0.0
    for k in ("d1alpha", "d2alpha", "d1beta1", "d2beta1", "d1H13", "d2H13", "d2H11"):
        assert m[k] == 0.0


@pytest.mark.parametrize("cfg", CASES)
def test_derivatives_against_finite_differences(cfg):
    keys = ["H11", "H22", "H33", "H13", "alpha", "beta1"]
    for pt in PTS:
        x1 = pt[0] * cfg["n_r"] / 50.0
        x2 = pt[1] * cfg["n_theta"] / 32.0
        m = O.metric_point(cfg, x1, x2)
        for d, (e1, e2) in ((1, (1e-3, 0)), (2, (0, 1e-3))):
            f = [O.metric_point(cfg, x1 + k * e1, x2 + k * e2) for k in (-2, -1, 1, 2)]
            for k in keys:
                fd = (f[0][k] - 8 * f[1][k] + 8 * f[2][k] - f[3][k]) / (12e-3)
                an = m["d%d%s" % (d, k)]
                scale = max(abs(m[k]), abs(an), 1e-300)
                assert abs(fd - an) <= 1e-8 * scale + 1e-14, (cfg, pt, d, k, fd, an)


@pytest.mark.parametrize("cfg", [CASES[0], CASES[2], CASES[3], CASES[4], CASES[5]])
def test_polar_area(cfg):
    """A(x1) = integral_0^{1/2} sqrt(h) dx2 (Sec. 3.3.2). Exact for a = 0 or flat; with
    spin the closed form takes Sigma on the axis, so it agrees to O(a^2 dtheta^2)."""
    for x1 in (3.5, 20.5, cfg["n_r"] - 0.5):
        xs = np.linspace(0.0, 0.5, 4001)
        vals = np.array([O.metric_point(cfg, x1, x)["sqrt_h"] for x in xs])
        integral = np.sum(0.5 * (vals[1:] + vals[:-1]) * np.diff(xs))
        A = O.polar_area(cfg, x1)
        r = O.metric_point(cfg, x1, 0.25)["r"]
        th_half = O.metric_point(cfg, x1, 0.5)["th"]  # the half cell's polar extent
        tol = cfg["a"] ** 2 * th_half ** 2 / r ** 2 + 1e-7
        assert abs(A - integral) <= tol * integral


@pytest.mark.parametrize("cfg", [CASES[0], CASES[1], CASES[3]])
def test_tetrad_orthonormal_and_inverse(cfg):
    rng = np.random.default_rng(0)
    for pt in PTS:
        x1 = pt[0] * cfg["n_r"] / 50.0
        x2 = pt[1] * cfg["n_theta"] / 32.0
        m = O.metric_point(cfg, x1, x2, clamp=True)
        h = np.array([[m["h11"], 0, m["h13"]], [0, m["h22"], 0], [m["h13"], 0, m["h33"]]])
        E = np.array([O.tetrad(cfg, x1, x2, "hat2vec", e) for e in np.eye(3)]).T
        assert np.allclose(E.T @ h @ E, np.eye(3), atol=1e-12)  # h_ij e^i_a e^j_b = delta_ab
        for _ in range(3):
            v = rng.normal(size=3)
            a = rng.normal(size=3)
            assert np.allclose(O.tetrad(cfg, x1, x2, "vec2hat", O.tetrad(cfg, x1, x2, "hat2vec", v)), v)
            assert np.allclose(O.tetrad(cfg, x1, x2, "hat2cov", O.tetrad(cfg, x1, x2, "cov2hat", a)), a)
            # a scalar is frame independent: a_i A^i = a_hat . A_hat
            vh = O.tetrad(cfg, x1, x2, "vec2hat", v)
            ah = O.tetrad(cfg, x1, x2, "cov2hat", a)
            assert math.isclose(a @ v, ah @ vh, rel_tol=1e-12, abs_tol=1e-12)
            # lowering with h_ij commutes with the change of frame
            assert np.allclose(O.tetrad(cfg, x1, x2, "cov2hat", h @ v), vh, atol=1e-12)
