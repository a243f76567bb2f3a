"""The mixed path's tiled FP32 kernel (fields of a sort tile and its halo staged in shared
memory, currents accumulated there) against the untiled kernel on the same particles in
the same order: the particle state after a fused step is the same bits (the window holds
copies of the field values); the currents differ only in the order of the FP32 sums. Over
many steps without a sort, particles drift out of their tile's window and take the global
path. Both ways of loading the window are covered: the CTA's threads (tiled_push = 1) and the
tensor memory accelerator (tiled_push = 2: one bulk tensor copy per field plane from a
row-padded copy of the planes, completed on an mbarrier)."""
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


def twin_sims(cfg, tiled=1):
    """A: sorted (tile ranges valid, tiled kernel); B: the same particles in the same order
    set afresh (no tile ranges, untiled kernel)."""
    osim = oracle_state(cfg)
    over = dict(precision="mixed", tile_r=cfg["tile_r"], tile_theta=cfg["tile_theta"],
                sort_every=0, tiled_push=tiled)
    a = gpu_from_oracle(osim, **over)
    for s in range(2):
        a.sort(s)
    b = gpu_from_oracle(osim, **over)
    for s in range(2):
        b.set_particles(s, a.get_particles(s), a.qm[s], a.qc[s])
    return a, b


def rel_norm(x, y):
    return float(np.abs(x - y).max() / max(np.abs(y).max(), 1e-300))


@pytest.mark.parametrize("tiled", [1, 2])
@pytest.mark.parametrize("tile", [8, 16])
def test_tiled_step_matches_untiled(torch_cuda, tile, tiled):
    cfg = dict(W.grid_config("wald64"), tile_r=tile, tile_theta=tile)
    a, b = twin_sims(cfg, tiled)
    a.step(1)
    b.step(1)
    assert a.diagnostics()["stage_timeouts"] == 0
    for s in range(2):
        pa, pb = a.get_particles(s), b.get_particles(s)
        for k in pa:
            assert np.array_equal(pa[k], pb[k]), (s, k)
    Fa, Fb = a.planes(), b.planes()
    for k in (15, 16, 17):  # after the step's rotation cur0 holds the step's currents
        assert rel_norm(Fa[k], Fb[k]) < 1e-5, k


@pytest.mark.parametrize("tiled", [1, 2])
def test_tiled_kernel_after_drift(torch_cuda, tiled):
    """30 steps of relativistic particles (theta_T = 1) without a sort: a part of them
    leaves its tile's window (tile 4 + halo 6 cells); the two kernels stay together to the
    FP32 accumulation order."""
    cfg = dict(W.grid_config("wald64", theta_T=1.0), tile_r=4, tile_theta=4)
    a, b = twin_sims(cfg, tiled)
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


def test_tma_window_on_a_ragged_grid(torch_cuda):
    """A 37 x 23 grid (rows of 42 floats, padded to 44 for the tensor copies; windows that
    run past every edge of the planes) with 12-cell tiles: the TMA-loaded window gives the
    untiled kernel's particle bits."""
    cfg = dict(W.grid_config("wald64", n_r=37, n_theta=23, a=0.5, ppc=3, r_max=12.0,
                             r_absorb=10.5), tile_r=12, tile_theta=12)
    a, b = twin_sims(cfg, 2)
    for _ in range(2):
        a.step(1)
        b.step(1)
    for s in range(2):
        pa, pb = a.get_particles(s), b.get_particles(s)
        for k in ("i1", "i2", "tag"):
            assert np.array_equal(pa[k], pb[k]), (s, k)
    assert a.diagnostics()["stage_timeouts"] == 0
