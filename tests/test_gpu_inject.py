"""GPU vs oracle parity of the pair injection of the BZ monopole test (Sec. 4.5; the reading:
sigma per cell from the cell-centre B and the pair density, one co-located pair with the
weight that brings sigma to sigma_th in every cell above it, random draws from a pool in
cell order). The decision compares two FP64 numbers that both sides compute with different
roundings, so the thresholds are chosen with no cell within 1e-9 of them (checked on the
oracle's values): then the injected set is unique and compared exactly, the particles to
the parity bound.
"""
import numpy as np
import pytest

import workloads as W
from oracle import oracle as O
from parity import (assert_particles, assert_planes, gpu_from_oracle, oracle_state,
                    particle_errors, round_state_fp32)

pytestmark = pytest.mark.gpu

CFG = W.grid_config("bz1024", n_r=48, n_theta=40, ppc=2)
SIGMA0, B0 = CFG["sigma0"], CFG["B0"]
AFTER_ADVANCE = list(range(12)) + [15, 16, 17, 18, 19, 20]


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def safe_threshold(osim, want):
    """A threshold near `want` with no cell's sigma within 1e-9 relative of it."""
    n, b2 = osim.cell_state()
    with np.errstate(divide="ignore", invalid="ignore"):
        s = SIGMA0 * b2 / (B0 * B0 * n)
    th = want
    for _ in range(50):
        if not np.any(np.abs(s / th - 1.0) < 1e-9):
            return th
        th *= 1.0 + 1e-6
    raise AssertionError("no safe threshold")


def pool_tensor(torch, pool):
    return torch.tensor(pool, dtype=torch.float64, device="cuda")


def assert_injected(g, osim, n_before, b2, th, rtol=1e-12):
    """Particle parity after an injection. The weight of a pair added near the threshold is
    a difference of two nearly equal densities (the target and the one already there), so
    its error is bounded relative to the target weight n_target sqrt(h) / 2, not to itself;
    every other quantity (and the weights of the particles that were there) to rtol."""
    for s in range(2):
        pg, po = g.get_particles(s), osim.species[s].view()
        nb = n_before[s]
        assert len(pg["w"]) == len(po["w"])
        assert np.allclose(pg["w"][:nb], po["w"][:nb], rtol=rtol, atol=0)
        for p in range(nb, len(po["w"])):
            i, j = int(po["i1"][p]), int(po["i2"][p])
            sq = O.metric_point(CFG, i + 0.5, j + 0.5)["sqrt_h"]
            target = 0.5 * SIGMA0 * b2[j, i] / (B0 * B0 * th) * sq
            assert abs(pg["w"][p] - po["w"][p]) <= rtol * target, (s, p)
        pg = dict(pg, w=po["w"])
        assert_particles(pg, po, rtol=rtol)


@pytest.mark.parametrize("want", [300.0, 2000.0])
def test_injection_matches_the_oracle(torch_cuda, want):
    osim = oracle_state(CFG, kind=O.FIELD_MONOPOLE, B0=B0)
    th = safe_threshold(osim, want)
    nc = CFG["n_r"] * CFG["n_theta"]
    g = gpu_from_oracle(osim, extra_capacity=2 * nc)
    pool = W.injection_pool(CFG, 997, seed=7)
    pt = pool_tensor(torch_cuda, pool)
    g.inject(SIGMA0, th, B0, pt, pool_offset=11)
    nb = [sp.n for sp in osim.species]
    b2 = osim.cell_state()[1]
    added = osim.inject(SIGMA0, th, B0, pool, pool_offset=11)
    assert added > 0
    d = g.diagnostics()
    assert d["injected"] == added and d["inject_dropped"] == 0
    assert_injected(g, osim, nb, b2, th)
    # the cursor continues: a lower threshold injects again from entry 11 + added
    th2 = safe_threshold(osim, 0.5 * th)
    g.inject(SIGMA0, th2, B0, pt)
    nb = [sp.n for sp in osim.species]
    b2 = osim.cell_state()[1]
    added2 = osim.inject(SIGMA0, th2, B0, pool, pool_offset=11 + added)
    assert added2 > 0 and g.diagnostics()["injected"] == added2
    assert_injected(g, osim, nb, b2, th2)


def test_injection_with_limited_room(torch_cuda):
    osim = oracle_state(CFG, kind=O.FIELD_MONOPOLE, B0=B0)
    th = safe_threshold(osim, 300.0)
    g = gpu_from_oracle(osim, extra_capacity=25)
    pool = W.injection_pool(CFG, 500, seed=8)
    g.inject(SIGMA0, th, B0, pool_tensor(torch_cuda, pool), pool_offset=0)
    full = oracle_state(CFG, kind=O.FIELD_MONOPOLE, B0=B0).inject(SIGMA0, th, B0, pool)
    nb = [sp.n for sp in osim.species]
    b2 = osim.cell_state()[1]
    added = osim.inject(SIGMA0, th, B0, pool, cap=osim.species[0].n + 25)
    assert added == 25 and full > 25
    d = g.diagnostics()
    assert d["injected"] == 25 and d["inject_dropped"] == full - 25
    assert_injected(g, osim, nb, b2, th)


def test_steps_after_injection_and_charge(torch_cuda):
    cfg = dict(CFG, sort_every=1, tile_r=8, tile_theta=8)
    osim = oracle_state(cfg, kind=O.FIELD_MONOPOLE, B0=B0)
    th = safe_threshold(osim, 500.0)
    g = gpu_from_oracle(osim, extra_capacity=CFG["n_r"] * CFG["n_theta"])
    pool = W.injection_pool(CFG, 3000, seed=9)
    g.inject(SIGMA0, th, B0, pool_tensor(torch_cuda, pool), pool_offset=0)
    nb = [sp.n for sp in osim.species]
    b2 = osim.cell_state()[1]
    assert osim.inject(SIGMA0, th, B0, pool) > 0
    assert_injected(g, osim, nb, b2, th)
    # from the same state on both sides the steps are compared at the parity bound
    for s in range(2):
        g.set_particles(s, osim.species[s].view(), osim.species[s].qm, osim.species[s].qc)
    g.step(2)
    osim.step(2, sort_every=1, tr=8, tt=8)
    assert_planes(g.planes(), osim.F, planes=AFTER_ADVANCE, rtol=1e-11, what="after injection")
    for s in range(2):
        assert_particles(g.get_particles(s), osim.species[s].view(), rtol=1e-11)
    res, drho, _, scale = g.charge_check(after_step=True)
    assert drho > 0 and res <= 1e-13 * scale


def test_mixed_injection(torch_cuda):
    osim = oracle_state(CFG, kind=O.FIELD_MONOPOLE, B0=B0)
    round_state_fp32(osim)
    th = safe_threshold(osim, 300.0)
    g = gpu_from_oracle(osim, precision="mixed", extra_capacity=CFG["n_r"] * CFG["n_theta"])
    pool = W.injection_pool(CFG, 997, seed=10)
    g.inject(SIGMA0, th, B0, pool_tensor(torch_cuda, pool), pool_offset=0)
    added = osim.inject(SIGMA0, th, B0, pool)
    assert added > 0 and g.diagnostics()["injected"] == added
    for s in range(2):
        e = particle_errors(g.get_particles(s), osim.species[s].view())
        assert max(e.values()) <= 1e-6, e
