"""GPU vs oracle parity of the current filter (n_f passes after the deposit, Sec. 3.2; horizon
layer of n_f cells, Sec. 3.3.3), through grpic_deposit, the fused grpic_step and the charge
check. Grids start far enough inside the horizon for the filter (r(n_f + 1) <= r_h).

* deposit + filter for n_f = 1, 3, 8 (one launch, result copied back from the scratch
  planes), 9 and 12 (two launches), on the 64^2 Kerr grid and a ragged 37 x 23 grid;
* full steps with a sort, FP64 (1e-12 per step) and mixed precision (1e-5);
* the charge check: the filtered currents conserve the filtered charge to rounding.
"""
import pytest

import workloads as W
from oracle import oracle as O
from parity import (assert_currents, assert_particles, assert_planes, gpu_from_oracle,
                    oracle_state, particle_errors, plane_errors, round_state_fp32)

pytestmark = pytest.mark.gpu

R_H = W.horizon_radius(0.9)
DEEP = W.grid_config("wald64f", r_min=0.6 * R_H)  # 13.3 cells inside the horizon
RAGGED = W.grid_config("wald64", n_r=37, n_theta=23, a=0.5, ppc=3, r_max=12.0, r_absorb=10.5,
                       n_filter=3)
AFTER_ADVANCE = list(range(12)) + [15, 16, 17, 18, 19, 20]


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


@pytest.mark.parametrize("cfg,n_f", [(DEEP, 1), (DEEP, 3), (DEEP, 8), (DEEP, 9), (DEEP, 12),
                                     (RAGGED, 3)])
def test_deposit_and_filter(torch_cuda, cfg, n_f):
    cfg = dict(cfg, n_filter=n_f)
    osim = oracle_state(cfg)
    osim.predict()
    for s in range(2):
        osim.push(s)
    g = gpu_from_oracle(osim)
    g.deposit()
    osim.deposit()
    osim.filter_currents()
    assert_currents(g.planes(), osim.F)
    F = g.planes()
    for k in (O.J1, O.J2, O.J3):  # ghost rows stay zero
        assert not F[k][:O.G].any() and not F[k][-O.G:].any()


@pytest.mark.parametrize("cfg", [DEEP, RAGGED])
def test_full_steps_with_filter(torch_cuda, cfg):
    cfg = dict(cfg, sort_every=2, tile_r=8, tile_theta=8)
    osim = oracle_state(cfg)
    g = gpu_from_oracle(osim)
    g.step(1)
    osim.step(1, sort_every=2, tr=8, tt=8)
    assert_planes(g.planes(), osim.F, planes=AFTER_ADVANCE, what="filtered step")
    for s in range(2):
        assert_particles(g.get_particles(s), osim.species[s].view())
    g.step(2)
    osim.step(2, sort_every=2, tr=8, tt=8)
    assert_planes(g.planes(), osim.F, planes=AFTER_ADVANCE, rtol=1e-11, what="3 steps")
    for s in range(2):
        assert_particles(g.get_particles(s), osim.species[s].view(), rtol=1e-11)


def test_mixed_step_with_filter(torch_cuda):
    osim = oracle_state(DEEP)
    round_state_fp32(osim)
    g = gpu_from_oracle(osim, precision="mixed")
    g.step(1)
    osim.step(1)
    for s in range(2):
        e = particle_errors(g.get_particles(s), osim.species[s].view())
        assert max(e.values()) <= 1e-5, e
    pe = plane_errors(g.planes(), osim.F, AFTER_ADVANCE)
    assert max(pe.values()) <= 1e-5, pe


@pytest.mark.parametrize("precision,bound", [("fp64", 1e-13), ("mixed", 1e-6)])
def test_charge_check_with_filter(torch_cuda, precision, bound):
    osim = oracle_state(DEEP)
    g = gpu_from_oracle(osim, precision=precision)
    g.step(2)
    res, drho, _, scale = g.charge_check(after_step=True)
    assert drho > 1e-3
    assert res <= bound * scale, (res, scale)
