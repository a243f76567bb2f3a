"""The FP64 charge-conservation check of the deposit (grpic_charge_check) on the GPU: the
discrete continuity equation of Sec. 3.2 holds to rounding for the FP64 path, and to the
FP32 accumulation of the currents for the mixed path, after separate push + deposit calls
and after full steps; a deliberately inconsistent current plane is reported. Residuals are
measured against the rounding scale: the absolute charge per node over the time step
(e+- charges cancel in rho itself)."""
import numpy as np
import pytest

import workloads as W
from parity import gpu_from_oracle, oracle_state

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


@pytest.mark.parametrize("precision,bound", [("fp64", 1e-13), ("mixed", 1e-6)])
def test_continuity_after_push_and_deposit(torch_cuda, precision, bound):
    osim = oracle_state(W.grid_config("wald64"))
    g = gpu_from_oracle(osim, precision=precision)
    g.predict()
    for s in range(2):
        g.push(s)
    g.deposit()
    res, drho, node, scale = g.charge_check(after_step=False)
    print(precision, "push + deposit: max residual %.3e, max drho/dt %.3e, node-relative %.3e,"
          " rho/dt %.3e" % (res, drho, node, scale))
    assert drho > 1e-3           # charge moved
    assert res / scale < bound, (res, drho, node, scale)


@pytest.mark.parametrize("precision,bound", [("fp64", 1e-13), ("mixed", 1e-6)])
def test_continuity_after_full_steps(torch_cuda, precision, bound):
    osim = oracle_state(W.grid_config("wald64"))
    g = gpu_from_oracle(osim, precision=precision)
    for _ in range(5):
        g.step(1)
        res, drho, node, scale = g.charge_check(after_step=True)
        print(precision, "step: max residual %.3e, max drho/dt %.3e, node-relative %.3e,"
              " rho/dt %.3e" % (res, drho, node, scale))
        assert drho > 1e-3
        assert res / scale < bound, (res, drho, node, scale)


def test_check_reports_a_broken_current(torch_cuda):
    from paper_2511_17701_gb300.binding import J1
    osim = oracle_state(W.grid_config("wald64"))
    g = gpu_from_oracle(osim)
    g.predict()
    for s in range(2):
        g.push(s)
    g.deposit()
    F = g.planes()
    F[J1] *= 1.01                # scale J^1 by 1%: continuity must fail visibly
    g.set_planes(F)
    res, drho, node, scale = g.charge_check(after_step=False)
    # far above the rounding of either precision (~1e-15 and ~1e-9 of the scale)
    assert res / scale > 1e-7 and res / drho > 1e-3


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_pair_falling_into_a_spinning_black_hole_on_gpu(torch_cuda, precision):
    """The deposit test of Sec. 4.3 (as the oracle's pin, both particles moving inward): on
    the GPU the flux of D^1 through r ~ 10 follows the oracle's to 1e-9 of its maximum in
    FP64 (1e-4 mixed) over the whole fall, and returns to zero (1e-12 of the maximum in FP64,
    1e-6 mixed) once both particles have crossed the horizon."""
    import math

    from oracle import oracle as O
    from paper_2511_17701_gb300 import FIELD_ZERO, Sim
    from test_oracle_deposit import gauss_areas
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
    qe, ce = W.species_coefficients(-1.0, 1.0, 10.0)
    qp, cp = W.species_coefficients(+1.0, 1.0, 10.0)
    uh = [np.array([[-1.0], [0.0], [0.0]]), np.array([[-3.0], [0.0], [0.0]])]
    for s, (q, c) in enumerate(((qe, ce), (qp, cp))):
        osim.add_species(pos, uh[s], np.array([1.0]), q, c)
    g = Sim(dict(cfg, dt=osim.dt, precision=precision), [1, 1])
    g.init_metric()
    g.init_fields(FIELD_ZERO)
    for s, (q, c) in enumerate(((qe, ce), (qp, cp))):
        g.load_particles(s, pos, uh[s], np.array([1.0]), q, c, 0.0)
    i10 = int(math.log(10.0 / cfg["r_min"]) / dxi)
    areas = gauss_areas(cfg, i10)
    fo, fg = [], []
    for _ in range(int(50.0 / osim.dt)):
        osim.step(1)
        g.step(1)
        fo.append(float(areas @ osim.F[O.D1][O.G:O.G + len(areas), i10 + O.G]))
        d1 = g.plane(O.D1).cpu().numpy().astype(np.float64)
        fg.append(float(areas @ d1[O.G:O.G + len(areas), i10 + O.G]))
    fo, fg = np.array(fo), np.array(fg)
    peak = np.abs(fo).max()
    assert peak > 0.1
    assert np.abs(fg - fo).max() <= (1e-9 if precision == "fp64" else 1e-4) * peak
    assert np.abs(fg[-50:]).max() <= (1e-12 if precision == "fp64" else 1e-6) * peak
    assert g.diagnostics()["left_inner"] == 2
