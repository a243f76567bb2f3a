"""Pin of the oracle's loading weight rule, w = w0 r^-k sqrt(h) at the particle (the input
recipe: unit density has summed weight sqrt(h) per cell), against the proper volume of the
Kerr-Schild grid computed independently here.

The spatial volume element of Kerr-Schild coordinates is sqrt(gamma) = sin(theta)
sqrt(Sigma (Sigma + 2 M r)), Sigma = r^2 + a^2 cos^2(theta) (sqrt(-g) = Sigma sin(theta) as in
Boyer-Lindquist, divided by the lapse 1/sqrt(1 + 2 M r / Sigma)). Particles placed at the
m x m Gauss-Legendre nodes of each cell in the code coordinates (x1, x2), with w0 the node
weights, sum per cell to that rule's value of the integral of r^-k sqrt(gamma) over the
cell (per radian of phi); Gauss-Legendre quadrature in the physical r and theta gives it
here independently. The two rules agree to ~3e-15 on these smooth integrands. A dropped
sin(theta), a Boyer-Lindquist volume (no 2 M r term), a missing dr/dx1 or dtheta/dx2, or
r^+k fails it.
"""
import math

import numpy as np
import pytest

import workloads as W
from oracle import oracle as O

M_SUB = 8  # Gauss-Legendre nodes per cell and direction


def grid_maps(cfg):
    """x1 -> r and x2 -> theta of the grid (App. A): r = r0 + (r_min - r0) exp(x1 dxi), theta
    = eta + 2 h0 eta (pi - 2 eta)(pi - eta)/pi^2 with eta = pi x2 / n_theta."""
    r0, h0 = cfg.get("r0", 0.0), cfg.get("h0", 0.0)
    dxi = math.log((cfg["r_max"] - r0) / (cfg["r_min"] - r0)) / cfg["n_r"]

    def r_of(x1):
        return r0 + (cfg["r_min"] - r0) * np.exp(x1 * dxi)

    def th_of(x2):
        eta = math.pi * np.asarray(x2, dtype=np.float64) / cfg["n_theta"]
        return eta + 2.0 * h0 * eta * (math.pi - 2.0 * eta) * (math.pi - eta) / math.pi ** 2

    return r_of, th_of


def cell_volumes(cfg, k):
    """Integral of r^-k sqrt(gamma) over each cell, [n_theta, n_r], Gauss-Legendre 12 x 12 in
    r and theta (the maps are monotonic, so each cell is [r(i), r(i+1)] x [th(j), th(j+1)])."""
    a, M = cfg["a"], 1.0 if cfg.get("metric", "ks") == "ks" else 0.0
    r_of, th_of = grid_maps(cfg)
    xg, wg = np.polynomial.legendre.leggauss(12)
    ra, rb = r_of(np.arange(cfg["n_r"])), r_of(np.arange(1, cfg["n_r"] + 1))
    ta, tb = th_of(np.arange(cfg["n_theta"])), th_of(np.arange(1, cfg["n_theta"] + 1))
    r = 0.5 * (ra + rb)[None, :, None, None] + 0.5 * (rb - ra)[None, :, None, None] * xg[None, None, :, None]
    t = 0.5 * (ta + tb)[:, None, None, None] + 0.5 * (tb - ta)[:, None, None, None] * xg[None, None, None, :]
    sig = r * r + a * a * np.cos(t) ** 2
    f = r ** (-k) * np.sin(t) * np.sqrt(sig * (sig + 2.0 * M * r))
    jac = (0.25 * (rb - ra)[None, :] * (tb - ta)[:, None])
    return np.einsum("jipq,p,q->ji", f, wg, wg) * jac


def node_plasma(cfg):
    """Particles at the Gauss-Legendre nodes of every cell, and their base weights."""
    n_r, n_t = cfg["n_r"], cfg["n_theta"]
    xg, wg = np.polynomial.legendre.leggauss(M_SUB)
    off, wo = 0.5 * (xg + 1.0), 0.5 * wg
    o1, o2 = np.meshgrid(off, off, indexing="ij")
    w1, w2 = np.meshgrid(wo, wo, indexing="ij")
    i2, i1 = np.meshgrid(np.arange(n_t), np.arange(n_r), indexing="ij")
    nc = n_r * n_t
    pos = {"i1": np.repeat(i1.ravel(), M_SUB * M_SUB).astype(np.int32),
           "i2": np.repeat(i2.ravel(), M_SUB * M_SUB).astype(np.int32),
           "dx1": np.tile(o1.ravel(), nc), "dx2": np.tile(o2.ravel(), nc)}
    return pos, np.tile((w1 * w2).ravel(), nc)


@pytest.mark.parametrize("k", [0.0, 1.0, 2.0])
@pytest.mark.parametrize("grid", ["plain", "quasi_spherical"])
def test_loaded_weights_sum_to_the_proper_volume(k, grid):
    cfg = W.grid_config("wald64", n_r=12, n_theta=10)
    if grid == "quasi_spherical":
        cfg.update(r0=0.4, h0=0.45)
    osim = O.OracleSim(cfg)
    pos, w0 = node_plasma(cfg)
    n = len(w0)
    sp = osim.add_species(pos, np.zeros((3, n)), w0, -1.0, -1.0, density_power=k)
    w = sp.view()["w"]
    summed = np.zeros((cfg["n_theta"], cfg["n_r"]))
    np.add.at(summed, (pos["i2"], pos["i1"]), w)
    vol = cell_volumes(cfg, k)
    assert np.max(np.abs(summed / vol - 1.0)) < 1e-10
    # the unit-density convention: the summed weight of the whole grid is its volume
    assert abs(summed.sum() / vol.sum() - 1.0) < 1e-12
