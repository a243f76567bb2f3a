"""GPU vs oracle parity on quasi-spherical Kerr-Schild grids (App. A: r = r0 + exp(xi),
theta(eta) concentrated toward the equator by h0): the metric tables and time step, the
Wald and monopole initial fields, loading, the push (plain and refined implicit
iterations, with particles at the axes and the horizon), the deposit, the field advance and
full steps with a sort, in FP64 (1e-12 per step) and mixed precision (1e-5); the adjoint
refuses these grids."""
import math

import numpy as np
import pytest

import workloads as W
from oracle import oracle as O
from parity import (assert_currents, assert_particles, assert_planes, gpu_from_oracle,
                    oracle_state, particle_errors, plane_errors, round_state_fp32)

pytestmark = pytest.mark.gpu

QKS = W.grid_config("wald64", r0=0.4, h0=0.45)
QKS_RAGGED = W.grid_config("wald64", n_r=41, n_theta=27, a=0.5, ppc=3, r_min=1.2, r_max=30.0,
                           r_absorb=26.0, r0=-1.0, h0=0.8)
AFTER_ADVANCE = list(range(12)) + [15, 16, 17, 18, 19, 20]


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


@pytest.mark.parametrize("cfg", [QKS, QKS_RAGGED])
@pytest.mark.parametrize("kind", ["wald", "monopole"])
def test_dt_and_initial_fields(torch_cuda, cfg, kind):
    from paper_2511_17701_gb300 import FIELD_MONOPOLE, FIELD_WALD, Sim
    ok = O.FIELD_WALD if kind == "wald" else O.FIELD_MONOPOLE
    gk = FIELD_WALD if kind == "wald" else FIELD_MONOPOLE
    osim = O.OracleSim(cfg)
    osim.init_fields(ok, 1.3)
    g = Sim(dict(cfg), [1])
    g.init_metric()
    assert math.isclose(g.dt, osim.dt, rel_tol=1e-13)
    g.init_fields(gk, 1.3)
    assert_planes(g.planes(), osim.F, what="qks init")


@pytest.mark.parametrize("cfg", [QKS, QKS_RAGGED])
def test_load_push_deposit_advance(torch_cuda, cfg):
    from paper_2511_17701_gb300 import Sim
    cfg = dict(cfg, density_power=1.0)
    osim = oracle_state(cfg)
    pl = W.pair_plasma(cfg)
    g = Sim(dict(cfg, dt=osim.dt), [osim.species[0].n, osim.species[1].n])
    g.init_metric()
    for s in range(2):
        g.load_particles(s, pl["pos"], pl["uhat"][s], pl["w0"], pl["qm"][s], pl["qc"][s], 1.0)
        assert_particles(g.get_particles(s), osim.species[s].view())
    osim.predict()
    for iter_tol in (0.0, 1e-12):
        o = oracle_state(cfg)
        o.predict()
        g = gpu_from_oracle(o, iter_tol=iter_tol)
        for s in range(2):
            g.push(s)
            o.push(s)
            assert_particles(g.get_particles(s), o.species[s].view())
        g.deposit()
        o.deposit()
        assert_currents(g.planes(), o.F)
        g2 = gpu_from_oracle(o)
        g2.advance()
        o.advance()
        assert_planes(g2.planes(), o.F, planes=AFTER_ADVANCE, what="qks advance")


def test_edge_particles(torch_cuda):
    cfg = QKS
    osim = O.OracleSim(cfg)
    osim.init_fields(O.FIELD_WALD, 1.0)
    n = 4000
    rng = np.random.default_rng(31)
    nt = cfg["n_theta"]
    x2 = np.concatenate([rng.uniform(0.0, 0.3, n // 4), rng.uniform(nt - 0.3, nt, n // 4),
                         rng.uniform(0.0, nt, n // 2)])
    x1 = np.concatenate([rng.uniform(1.0, 60.0, n // 2), rng.uniform(0.0, 0.4, n // 4),
                         rng.uniform(63.6, 64.0, n // 4)])
    pos = {"i1": np.floor(x1).astype(np.int32), "i2": np.floor(x2).astype(np.int32)}
    pos["dx1"], pos["dx2"] = x1 - pos["i1"], x2 - pos["i2"]
    uh = W.maxwell_juttner(rng, n, 3.0)
    qm, qc = W.species_coefficients(-1.0)
    osim.add_species(pos, uh, np.full(n, 0.1), qm, qc)
    osim.predict()
    for iter_tol in (0.0, 1e-12):
        o = O.OracleSim(cfg)
        o.F[:] = osim.F
        o.add_raw_species(osim.species[0].view(), qm, qc)
        g = gpu_from_oracle(o, iter_tol=iter_tol)
        for _ in range(3):
            g.set_particles(0, o.species[0].view(), qm, qc)
            g.push(0)
            o.push(0)
            assert_particles(g.get_particles(0), o.species[0].view())


@pytest.mark.parametrize("cfg", [QKS, QKS_RAGGED])
def test_full_steps_with_sort(torch_cuda, cfg):
    cfg = dict(cfg, sort_every=2, tile_r=8, tile_theta=8)
    osim = oracle_state(cfg)
    g = gpu_from_oracle(osim, iter_tol=1e-12)
    g.step(3)
    osim.step(3, sort_every=2, tr=8, tt=8)
    assert_planes(g.planes(), osim.F, planes=AFTER_ADVANCE, rtol=1e-11, what="qks steps")
    for s in range(2):
        assert_particles(g.get_particles(s), osim.species[s].view(), rtol=1e-11)
    res, drho, _, scale = g.charge_check(after_step=True)
    assert drho > 0 and res <= 1e-13 * scale


@pytest.mark.parametrize("cfg", [QKS, QKS_RAGGED])
def test_mixed_step(torch_cuda, cfg):
    osim = oracle_state(cfg)
    round_state_fp32(osim)
    g = gpu_from_oracle(osim, precision="mixed")
    g.step(1)
    osim.step(1)
    for s in range(2):
        e = particle_errors(g.get_particles(s), osim.species[s].view())
        assert max(e.values()) <= 1e-5, e
    pe = plane_errors(g.planes(), osim.F, AFTER_ADVANCE)
    assert max(pe.values()) <= 1e-5, pe


def test_adjoint_refuses_quasi_spherical_grids(torch_cuda):
    from paper_2511_17701_gb300 import FIELD_WALD, GrpicError, Sim
    torch = torch_cuda
    g = Sim(dict(QKS), [1])
    g.init_metric()
    g.init_fields(FIELD_WALD, 1.0)
    st = torch.zeros((6, 4), dtype=torch.float64, device="cuda")
    st[0] += 30.0
    st[1] += 20.0
    with pytest.raises(GrpicError):
        g.adjoint_forward(st, qm=1.0, b0=1.0, n_steps=2, ckpt_every=1, n_iter=10)


def test_filter_and_photons_on_a_quasi_spherical_grid(torch_cuda):
    """The widened rows together: n_f = 2 current-filter passes, a photon species beside the
    pairs, on the quasi-spherical grid; full steps in FP64 against the oracle."""
    cfg = dict(QKS, r_min=1.2, n_filter=2, sort_every=2, tile_r=8, tile_theta=8)
    osim = oracle_state(cfg)
    pl = W.pair_plasma(cfg)
    uh = W.maxwell_juttner(np.random.default_rng(4), pl["pos"]["i1"].size, 2.0)
    osim.add_species(pl["pos"], uh, pl["w0"], pl["qm"][1], pl["qc"][1], pl["density_power"],
                     massless=True)
    g = gpu_from_oracle(osim, massless=[2])
    g.step(2)
    osim.step(2, sort_every=2, tr=8, tt=8)
    assert_planes(g.planes(), osim.F, planes=AFTER_ADVANCE, rtol=1e-11, what="qks+filter")
    for s in range(3):
        assert_particles(g.get_particles(s), osim.species[s].view(), rtol=1e-11)
