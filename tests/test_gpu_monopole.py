"""GPU vs oracle parity on the BZ monopole workload (Sec. 4.5: A_phi = -B0 cos(theta),
a = 0.2, r in [r_g, 10 r_g], pairs with theta_T = 0.5, density ~ r^-2, rho0 = 5e-5,
d0 = 2.5e-3): the initial field on square and ragged grids, pushes, and full steps with a
sort in FP64 (1e-12 per step) and mixed precision (1e-5), at reduced grid sizes; and the
stationary a = 0 monopole in vacuum."""
import numpy as np
import pytest

import workloads as W
from oracle import oracle as O
from parity import (assert_particles, assert_planes, gpu_from_oracle, oracle_state,
                    particle_errors, plane_errors, round_state_fp32)

pytestmark = pytest.mark.gpu

BZ64 = W.grid_config("bz1024", n_r=64, n_theta=64, ppc=4)
BZ_RAGGED = W.grid_config("bz1024", n_r=41, n_theta=27, ppc=3)
AFTER_ADVANCE = list(range(12)) + [15, 16, 17, 18, 19, 20]


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


@pytest.mark.parametrize("cfg", [BZ64, BZ_RAGGED, dict(BZ64, a=0.0), dict(BZ64, n_r=512,
                                                                           n_theta=512)])
def test_monopole_initial_field(torch_cuda, cfg):
    from paper_2511_17701_gb300 import FIELD_MONOPOLE, Sim
    osim = O.OracleSim(cfg)
    osim.init_fields(O.FIELD_MONOPOLE, 1.7)
    g = Sim(dict(cfg), [1])
    g.init_metric()
    g.init_fields(FIELD_MONOPOLE, 1.7)
    assert_planes(g.planes(), osim.F, what="monopole init")


@pytest.mark.parametrize("cfg", [BZ64, BZ_RAGGED])
def test_monopole_push_and_steps(torch_cuda, cfg):
    cfg = dict(cfg, sort_every=2, tile_r=8, tile_theta=8)
    osim = oracle_state(cfg, kind=O.FIELD_MONOPOLE, B0=cfg["B0"])
    osim.predict()
    g = gpu_from_oracle(osim)
    for s in range(2):
        g.push(s)
        osim.push(s)
        assert_particles(g.get_particles(s), osim.species[s].view())
    osim = oracle_state(cfg, kind=O.FIELD_MONOPOLE, B0=cfg["B0"])
    g = gpu_from_oracle(osim, iter_tol=1e-12)
    g.step(2)
    osim.step(2, sort_every=2, tr=8, tt=8)
    assert_planes(g.planes(), osim.F, planes=AFTER_ADVANCE, rtol=1e-11, what="BZ steps")
    for s in range(2):
        assert_particles(g.get_particles(s), osim.species[s].view(), rtol=1e-11)


def test_monopole_mixed_step(torch_cuda):
    osim = oracle_state(BZ64, kind=O.FIELD_MONOPOLE, B0=BZ64["B0"])
    round_state_fp32(osim)
    g = gpu_from_oracle(osim, precision="mixed")
    g.step(1)
    osim.step(1)
    for s in range(2):
        e = particle_errors(g.get_particles(s), osim.species[s].view())
        assert max(e.values()) <= 1e-5, e
    pe = plane_errors(g.planes(), osim.F, AFTER_ADVANCE)
    assert max(pe.values()) <= 1e-5, pe


def test_schwarzschild_monopole_stays_on_gpu(torch_cuda):
    from paper_2511_17701_gb300 import FIELD_MONOPOLE, Sim
    cfg = dict(BZ64, a=0.0, r_absorb=1e300)
    g = Sim(cfg, [1])
    g.init_metric()
    g.init_fields(FIELD_MONOPOLE, 1.0)
    F0 = g.planes()
    for _ in range(100):
        g.predict()
        g.deposit()
        g.advance()
    F = g.planes()
    b = np.abs(F0[O.B1]).max()
    assert np.abs(F[O.B1] - F0[O.B1]).max() < 1e-13 * b
    for k in (O.B2, O.B3, O.D1, O.D2, O.D3):
        assert np.abs(F[k]).max() < 1e-13 * b, k


def aux_region(cfg):
    """Stored rows and columns where both sides compute every auxiliary component: rows
    j in [0, n_theta - 1], columns i in [-1, n_r + 1]."""
    G = O.G
    return slice(G, G + cfg["n_theta"]), slice(G - 1, G + cfg["n_r"] + 2)


@pytest.mark.parametrize("cfg", [BZ64, BZ_RAGGED])
def test_aux_fields_match_the_oracle(torch_cuda, cfg):
    """grpic_aux_fields: E and H (Eqs. discretized-auxE, discretized-auxH) of the em planes, on
    the same state to rounding, and after two full steps with plasma to the per-step bound."""
    osim = oracle_state(cfg, kind=O.FIELD_MONOPOLE)
    g = gpu_from_oracle(osim)
    J, I = aux_region(cfg)
    for when in ("initial", "after two steps"):
        E, H = g.aux_fields()
        Eo, Ho = osim.aux_fields()
        tol = 1e-13 if when == "initial" else 1e-11
        for name, a, b in (("E", E, Eo), ("H", H, Ho)):
            for c in range(3):
                scale = np.abs(b[c][J, I]).max() + 1e-300
                err = np.abs(a[c][J, I] - b[c][J, I]).max() / scale
                assert err <= tol, (when, name, c, err)
        g.step(2)
        osim.step(2)


def test_aux_fields_mixed(torch_cuda):
    osim = oracle_state(BZ64, kind=O.FIELD_MONOPOLE)
    round_state_fp32(osim)
    g = gpu_from_oracle(osim, precision="mixed")
    J, I = aux_region(BZ64)
    E, H = g.aux_fields()
    Eo, Ho = osim.aux_fields()
    for a, b in ((E, Eo), (H, Ho)):
        for c in range(3):
            scale = np.abs(b[c][J, I]).max() + 1e-300
            assert np.abs(a[c][J, I] - b[c][J, I]).max() / scale <= 1e-5
