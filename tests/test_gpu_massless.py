"""GPU vs oracle parity of massless particles: gamma = sqrt(h^ij u_i u_j) (Sec. 2.3), no
field interpolation and no EM push (Sec. 3.1), only the geodesic momentum and coordinate
substeps and phi; neutral, so nothing is deposited.

The photon species gets the electrons' q/m and deposit coefficient on purpose: a path that
pushed or deposited it as a charge would fail the comparison. Workloads: the a = 0.9 Wald
grid at 64^2 with e+- pairs and one photon per pair member's position (FP64 and mixed
precision, plain and refined implicit iterations, fused steps with a sort), a ragged grid,
photons placed at the axes and the horizon, photons alone (zero current and charge).
"""
import numpy as np
import pytest

import workloads as W
from oracle import oracle as O
from parity import (assert_particles, assert_planes, gpu_from_oracle, oracle_state,
                    particle_errors, plane_errors, round_state_fp32)

pytestmark = pytest.mark.gpu

BASE = W.grid_config("wald64")
RAGGED = W.grid_config("wald64", n_r=37, n_theta=23, a=0.5, ppc=3, r_max=12.0, r_absorb=10.5)
AFTER_ADVANCE = list(range(12)) + [15, 16, 17, 18, 19, 20]
REFINED = 1e-12
MIXED_RTOL = 1e-5


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def with_photons(cfg, seed=11):
    """e+ and e- of the pair plasma (species 0, 1) and photons (species 2) at the same
    positions with their own Maxwell-Juttner momenta."""
    osim = oracle_state(cfg)
    pl = W.pair_plasma(cfg)
    n = pl["pos"]["i1"].size
    uh = W.maxwell_juttner(np.random.default_rng(seed), n, 2.0)
    osim.add_species(pl["pos"], uh, pl["w0"], pl["qm"][1], pl["qc"][1], pl["density_power"],
                     massless=True)
    return osim


def edge_photons(cfg, n=4000, seed=23):
    """Photons in the cell rows at both axes, in the horizon layer, at the outer edge and in
    the bulk, with fast momenta."""
    osim = O.OracleSim(cfg)
    osim.init_fields(O.FIELD_WALD, 1.0)
    rng = np.random.default_rng(seed)
    nt, nr = cfg["n_theta"], cfg["n_r"]
    x2 = np.concatenate([rng.uniform(0.0, 0.3, n // 4), rng.uniform(nt - 0.3, nt, n // 4),
                         rng.uniform(0.0, nt, n // 2)])
    x1 = np.concatenate([rng.uniform(1.0, nr - 4.0, n // 2), rng.uniform(0.0, 0.4, n // 4),
                         rng.uniform(nr - 0.4, nr, n // 4)])
    pos = {"i1": np.floor(x1).astype(np.int32), "i2": np.floor(x2).astype(np.int32)}
    pos["dx1"], pos["dx2"] = x1 - pos["i1"], x2 - pos["i2"]
    uh = W.maxwell_juttner(rng, n, 3.0)
    qm, qc = W.species_coefficients(-1.0)
    osim.add_species(pos, uh, np.full(n, 0.1), qm, qc, massless=True)
    return osim


@pytest.mark.parametrize("iter_tol", [0.0, REFINED])
@pytest.mark.parametrize("cfg", [BASE, RAGGED])
def test_massless_push(torch_cuda, cfg, iter_tol):
    osim = with_photons(cfg)
    osim.predict()
    g = gpu_from_oracle(osim, massless=[2], iter_tol=iter_tol)
    for s in range(3):
        g.push(s)
        osim.push(s)
    for s in range(3):
        assert_particles(g.get_particles(s), osim.species[s].view())
    d = g.diagnostics()
    assert [d["left_inner"], d["left_outer"], d["reflections"], d["nonfinite"]] == \
        [int(x) for x in osim.counters]


@pytest.mark.parametrize("iter_tol", [0.0, REFINED])
def test_massless_edge_particles(torch_cuda, iter_tol):
    osim = edge_photons(BASE)
    osim.predict()
    sp = osim.species[0]
    g = gpu_from_oracle(osim, massless=[0], iter_tol=iter_tol)
    for _ in range(3):
        g.set_particles(0, sp.view(), sp.qm, sp.qc)
        g.push(0)
        osim.push(0)
        assert_particles(g.get_particles(0), sp.view())
    assert osim.counters[0] > 0 and osim.counters[1] > 0 and osim.counters[2] > 0


@pytest.mark.parametrize("iter_tol", [0.0, REFINED])
def test_massless_full_steps_with_sort(torch_cuda, iter_tol):
    cfg = dict(BASE, sort_every=2, tile_r=8, tile_theta=8)
    osim = with_photons(cfg)
    g = gpu_from_oracle(osim, massless=[2], iter_tol=iter_tol)
    g.step(3)
    osim.step(3, sort_every=2, tr=8, tt=8)
    assert_planes(g.planes(), osim.F, planes=AFTER_ADVANCE, rtol=1e-11, what="3 steps")
    for s in range(3):
        assert_particles(g.get_particles(s), osim.species[s].view(), rtol=1e-11)


def test_photons_deposit_nothing(torch_cuda):
    osim = edge_photons(BASE)
    osim.predict()
    sp = osim.species[0]
    g = gpu_from_oracle(osim, massless=[0])
    g.push(0)
    g.deposit()
    F = g.planes()
    for k in (O.J1, O.J2, O.J3):
        assert not F[k].any(), k
    res, drho, _, scale = g.charge_check(after_step=False)
    assert res == 0.0 and drho == 0.0 and scale == 0.0
    # the fused step: the field update sees no current from them
    g2 = gpu_from_oracle(osim, massless=[0])
    g2.step(1)
    osim.step(1)
    assert_planes(g2.planes(), osim.F, planes=AFTER_ADVANCE, what="photon-only step")
    assert_particles(g2.get_particles(0), sp.view())


@pytest.mark.parametrize("cfg", [BASE, RAGGED])
def test_massless_mixed_step(torch_cuda, cfg):
    """Mixed precision: photons in all three zones (FP32, FP64 metric, FP64 routine)."""
    osim = with_photons(cfg)
    round_state_fp32(osim)
    g = gpu_from_oracle(osim, massless=[2], precision="mixed")
    g.step(1)
    osim.step(1)
    for s in range(3):
        e = particle_errors(g.get_particles(s), osim.species[s].view())
        assert max(e.values()) <= MIXED_RTOL, (s, e)
    pe = plane_errors(g.planes(), osim.F, AFTER_ADVANCE)
    assert max(pe.values()) <= MIXED_RTOL, pe


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_photon_orbit_independent_of_energy_on_gpu(torch_cuda, precision):
    """A null geodesic does not depend on the photon's energy: momenta scaled by 1024 give
    the same positions and phases (to the rounding of the scaled sums) and scaled momenta."""
    osim = edge_photons(BASE, seed=5)
    osim.predict()
    sp = osim.species[0]
    big = sp.copy()
    for k in ("u1", "u2", "u3"):
        big.a[k] *= 1024.0
    a = gpu_from_oracle(osim, massless=[0], precision=precision)
    b = gpu_from_oracle(osim, massless=[0], precision=precision)
    b.set_particles(0, big.view(), sp.qm, sp.qc)
    for _ in range(5):
        a.push(0)
        b.push(0)
    pa, pb = a.get_particles(0), b.get_particles(0)
    assert np.array_equal(pa["tag"], pb["tag"])
    live = pa["tag"] != 0
    tol = 1e-13 if precision == "fp64" else 1e-6
    for i, d in (("i1", "dx1"), ("i2", "dx2")):
        xa = pa[i][live] + pa[d][live].astype(np.float64)
        xb = pb[i][live] + pb[d][live].astype(np.float64)
        assert np.max(np.abs(xa - xb) / np.maximum(1.0, np.abs(xa))) <= tol, d
    assert np.max(np.abs(pa["phi"][live] - pb["phi"][live])) <= tol * 10
    for c in ("u1", "u2", "u3"):
        ua = pa[c][live].astype(np.float64) * 1024.0
        ub = pb[c][live].astype(np.float64)
        sc = np.abs(ub) + np.median(np.abs(ub))
        assert np.max(np.abs(ua - ub) / sc) <= tol, c
