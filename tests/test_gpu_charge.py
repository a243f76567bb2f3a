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
