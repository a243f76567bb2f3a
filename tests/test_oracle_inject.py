"""Pins of the oracle's pair injection (Sec. 4.5: plasma is injected where the local
magnetization exceeds sigma_th). Reading: per cell, sigma = sigma0 (B_i B^i / B0^2) / n
with B at the cell centre and n the pair density; where sigma > sigma_th one co-located
e- e+ pair with weights that bring sigma down to sigma_th, offsets and tetrad-frame
momenta from a pool of random draws used in cell order.

* every cell above the threshold gets exactly one pair, and afterwards its sigma equals
  sigma_th; every other cell keeps its density bit for bit;
* the charge density does not change (co-located opposite charges of equal weight);
* the k-th pair in cell order takes pool entry (offset + k) mod pool_n: positions and the
  tetrad-frame momenta recovered from the covariant ones match it;
* with limited room, the first pairs in cell order are the ones added.
"""
import numpy as np
import pytest

import workloads as W
from oracle import oracle as O
from parity import oracle_state

CFG = W.grid_config("bz1024", n_r=48, n_theta=40, ppc=2)
SIGMA0, B0 = CFG["sigma0"], CFG["B0"]


def state():
    osim = oracle_state(CFG, kind=O.FIELD_MONOPOLE, B0=B0)
    return osim


def sigma(osim):
    n, b2 = osim.cell_state()
    with np.errstate(divide="ignore"):
        return SIGMA0 * b2 / (B0 * B0 * n), n


@pytest.mark.parametrize("sigma_th", [300.0, 2000.0])
def test_injection_brings_sigma_to_the_threshold(sigma_th):
    osim = state()
    s0, n0 = sigma(osim)
    hot = s0 > sigma_th
    assert hot.sum() > 0 and (~hot).sum() > 0
    pool = W.injection_pool(CFG, 5000, seed=3)
    ne, npos = osim.species[0].n, osim.species[1].n
    added = osim.inject(SIGMA0, sigma_th, B0, pool)
    assert added == hot.sum()
    assert osim.species[0].n == ne + added and osim.species[1].n == npos + added
    s1, n1 = sigma(osim)
    assert np.allclose(s1[hot], sigma_th, rtol=1e-12, atol=0)
    assert np.array_equal(n1[~hot], n0[~hot])
    # a second call finds nothing above the threshold (up to rounding at sigma_th)
    assert osim.inject(SIGMA0, sigma_th * (1 + 1e-9), B0, pool) == 0


def test_charge_density_does_not_change():
    osim = state()
    rho0 = osim.charge(prev=False)
    osim.inject(SIGMA0, 300.0, B0, W.injection_pool(CFG, 5000, seed=4))
    rho1 = osim.charge(prev=False)
    # the scale of the cancelling charges: the largest single-species charge in a cell
    v = osim.species[0].view()
    per_cell = np.bincount(v["i2"] * CFG["n_r"] + v["i1"], weights=v["w"])
    scale = abs(osim.species[0].qc) * per_cell.max()
    assert np.abs(rho0).max() <= 1e-14 * scale  # the pairs were co-located before, too
    assert np.abs(rho1 - rho0).max() <= 1e-14 * scale


def test_pool_entries_in_cell_order_with_wraparound():
    osim = state()
    s0, _ = sigma(osim)
    hot = np.argwhere(s0 > 300.0)  # (j, i) rows in cell order (j outer, i inner)
    pool = W.injection_pool(CFG, 7, seed=5)
    off = 5
    ne = osim.species[0].n
    added = osim.inject(SIGMA0, 300.0, B0, pool, pool_offset=off)
    for s_idx, q in ((0, 0), (1, 1)):
        v = osim.species[s_idx].view()
        for k in range(added):
            j, i = hot[k]
            r = pool[(off + k) % 7]
            p = ne + k
            assert (v["i1"][p], v["i2"][p]) == (i, j)
            assert v["dx1"][p] == r[0] and v["dx2"][p] == r[1]
            assert (v["i1p"][p], v["i2p"][p], v["dx1p"][p], v["dx2p"][p]) == (i, j, r[0], r[1])
            assert v["tag"][p] == 1 and v["phi"][p] == 0.0
            uh = O.tetrad(CFG, i + r[0], j + r[1], "cov2hat", [v["u1"][p], v["u2"][p], v["u3"][p]])
            assert np.allclose(uh, r[2 + 3 * q:5 + 3 * q], rtol=1e-13, atol=1e-13)
    we = osim.species[0].view()["w"][ne:]
    assert np.array_equal(we, osim.species[1].view()["w"][ne:]) and np.all(we > 0)


def test_limited_room_takes_the_first_cells():
    a, b = state(), state()
    pool = W.injection_pool(CFG, 5000, seed=6)
    n = a.species[0].n
    full = a.inject(SIGMA0, 300.0, B0, pool)
    part = b.inject(SIGMA0, 300.0, B0, pool, cap=n + 10)
    assert full > 10 and part == 10
    for s in range(2):
        va, vb = a.species[s].view(), b.species[s].view()
        for k in vb:
            assert np.array_equal(va[k][: n + 10], vb[k]), k
