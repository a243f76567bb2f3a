"""The FP64 charge-conservation check of the deposit (grpic_charge_check) on the GPU: the
discrete continuity equation of Sec. 3.2 holds to rounding for the FP64 path, and to the
FP32 accumulation of the currents for the mixed path, after separate push + deposit calls
and after full steps; a deliberately inconsistent current plane is reported."""
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


@pytest.mark.parametrize("precision,bound", [("fp64", 1e-12), ("mixed", 2e-6)])
def test_continuity_after_push_and_deposit(torch_cuda, precision, bound):
    osim = oracle_state(W.grid_config("wald64"))
    g = gpu_from_oracle(osim, precision=precision)
    g.predict()
    for s in range(2):
        g.push(s)
    g.deposit()
    res, drho, node = g.charge_check(after_step=False)
    print(precision, "push + deposit: max residual %.3e, max drho/dt %.3e, node-relative %.3e"
          % (res, drho, node))
    assert drho > 1e-3           # charge moved
    assert res / drho < bound, (res, drho, node)


@pytest.mark.parametrize("precision,bound", [("fp64", 1e-12), ("mixed", 2e-6)])
def test_continuity_after_full_steps(torch_cuda, precision, bound):
    osim = oracle_state(W.grid_config("wald64"))
    g = gpu_from_oracle(osim, precision=precision)
    for _ in range(5):
        g.step(1)
        res, drho, node = g.charge_check(after_step=True)
        print(precision, "step: max residual %.3e, max drho/dt %.3e, node-relative %.3e"
              % (res, drho, node))
        assert drho > 1e-3
        assert res / drho < bound, (res, drho, node)


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
    res, drho, node = g.charge_check(after_step=False)
    assert res / drho > 1e-4
