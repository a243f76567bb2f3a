"""The mixed path's tiled FP32 kernel (fields of a sort tile and its halo staged in shared
memory, currents accumulated there) against the untiled kernel on the same particles in
the same order: the particle state after a fused step is the same bits (the window holds
copies of the field values); the currents differ only in the order of the FP32 sums. Over
many steps without a sort, particles drift out of their tile's window and take the global
path."""
import numpy as np
import pytest

import workloads as W
from parity import gpu_from_oracle, oracle_state

pytestmark = pytest.mark.gpu

J_PLANES = (12, 13, 14)


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def twin_sims(cfg):
    """A: sorted (tile ranges valid, tiled kernel); B: the same particles in the same order
    set afresh (no tile ranges, untiled kernel)."""
    osim = oracle_state(cfg)
    over = dict(precision="mixed", tile_r=cfg["tile_r"], tile_theta=cfg["tile_theta"],
                sort_every=0, tiled_push=1)
    a = gpu_from_oracle(osim, **over)
    for s in range(2):
        a.sort(s)
    b = gpu_from_oracle(osim, **over)
    for s in range(2):
        b.set_particles(s, a.get_particles(s), a.qm[s], a.qc[s])
    return a, b


def rel_norm(x, y):
    return float(np.abs(x - y).max() / max(np.abs(y).max(), 1e-300))


@pytest.mark.parametrize("tile", [8, 16])
def test_tiled_step_matches_untiled(torch_cuda, tile):
    cfg = dict(W.grid_config("wald64"), tile_r=tile, tile_theta=tile)
    a, b = twin_sims(cfg)
    a.step(1)
    b.step(1)
    for s in range(2):
        pa, pb = a.get_particles(s), b.get_particles(s)
        for k in pa:
            assert np.array_equal(pa[k], pb[k]), (s, k)
    Fa, Fb = a.planes(), b.planes()
    for k in (15, 16, 17):  # after the step's rotation cur0 holds the step's currents
        assert rel_norm(Fa[k], Fb[k]) < 1e-5, k


def test_tiled_kernel_after_drift(torch_cuda):
    """30 steps of relativistic particles (theta_T = 1) without a sort: a part of them
    leaves its tile's window (tile 4 + halo 6 cells); the two kernels stay together to the
    FP32 accumulation order."""
    cfg = dict(W.grid_config("wald64", theta_T=1.0), tile_r=4, tile_theta=4)
    a, b = twin_sims(cfg)
    home = [a.get_particles(s) for s in range(2)]
    for _ in range(30):
        a.step(1)
        b.step(1)
    drifted = 0
    for s in range(2):
        pa, pb = a.get_particles(s), b.get_particles(s)
        assert np.array_equal(pa["tag"], pb["tag"])
        alive = pa["tag"] == 1
        for k in ("dx1", "dx2", "u1", "u2", "u3"):
            xa = pa[k][alive].astype(np.float64)
            xb = pb[k][alive].astype(np.float64)
            if k.startswith("dx"):
                ik = "i1" if k == "dx1" else "i2"
                xa = xa + pa[ik][alive]
                xb = xb + pb[ik][alive]
            assert np.max(np.abs(xa - xb) / np.maximum(1.0, np.abs(xb))) < 1e-4, (s, k)
        # home tiles of the sort against the current cells: window = tile +- 6 cells
        h = home[s]
        ti, tj = h["i1"] // 4, h["i2"] // 4
        out = ((pa["i1"] - 1 < ti * 4 - 6) | (pa["i1"] + 1 >= ti * 4 + 10) |
               (pa["i2"] - 1 < tj * 4 - 6) | (pa["i2"] + 1 >= tj * 4 + 10)) & (pa["tag"] == 1)
        drifted += int(out.sum())
    assert drifted > 0
    Fa, Fb = a.planes(), b.planes()
    for k in range(6):
        assert rel_norm(Fa[k], Fb[k]) < 1e-4, k
