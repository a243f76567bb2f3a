"""GPU vs oracle parity of every row of the hot path, through the C ABI.

Workloads: the Kerr a = 0.9 Wald configuration at 64^2 with 8 particles per cell per
species (65,536 particles), ragged grids (37 x 23) with odd particle counts, the flat
kerr_schild_0 metric, empty species, particles placed at the axes and the horizon.
Each test starts both sides from the same oracle-built state.
"""
import math

import numpy as np
import pytest

import workloads as W
from oracle import oracle as O
from parity import (assert_currents, assert_particles, assert_planes, gpu_from_oracle,
                    oracle_state)

pytestmark = pytest.mark.gpu

BASE = W.grid_config("wald64")
# after ADVANCE the GPU rotates cur/cur0 by swapping buffers, so J then holds J^{n-1/2}
# while the oracle keeps J^{n+1/2} there; both hold J^{n+1/2} in cur0
AFTER_ADVANCE = list(range(12)) + [15, 16, 17, 18, 19, 20]
RAGGED = W.grid_config("wald64", n_r=37, n_theta=23, a=0.5, ppc=3, r_max=12.0, r_absorb=10.5)
FLAT = dict(W.grid_config("wald64", n_r=40, n_theta=30, ppc=2), metric="ks0", r_min=1.0,
            r_max=20.0, r_absorb=18.0)


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def odd_cells(cfg, frac=0.37, seed=5):
    n = cfg["n_r"] * cfg["n_theta"]
    return W.random_cells(cfg, int(n * frac) | 1, seed)


@pytest.mark.parametrize("cfg", [BASE, RAGGED, FLAT])
def test_dt_and_initial_fields(torch_cuda, cfg):
    from paper_2511_17701_gb300 import FIELD_VERTICAL, FIELD_WALD, Sim
    for kind in (FIELD_WALD, FIELD_VERTICAL):
        osim = O.OracleSim(cfg)
        osim.init_fields(kind, 1.3)
        g = Sim(dict(cfg), [1])
        g.init_metric()
        assert math.isclose(g.dt, osim.dt, rel_tol=1e-13)
        g.init_fields(kind, 1.3)
        assert_planes(g.planes(), osim.F, what="init kind %d" % kind)


@pytest.mark.parametrize("cfg", [BASE, RAGGED, FLAT])
def test_load_particles(torch_cuda, cfg):
    from paper_2511_17701_gb300 import Sim
    cfg = dict(cfg, density_power=1.0)
    osim = oracle_state(cfg, cells=odd_cells(cfg))
    pl = W.pair_plasma(cfg, cells=odd_cells(cfg))
    g = Sim(dict(cfg, dt=osim.dt), [osim.species[0].n, osim.species[1].n + 3])
    g.init_metric()
    for s in range(2):
        g.load_particles(s, pl["pos"], pl["uhat"][s], pl["w0"], pl["qm"][s], pl["qc"][s], 1.0)
        assert_particles(g.get_particles(s), osim.species[s].view())


@pytest.mark.parametrize("cfg", [BASE, RAGGED, FLAT])
def test_predict(torch_cuda, cfg):
    osim = oracle_state(cfg, species=0)
    # perturb em0 so that the time average and the auxiliary Faraday both matter
    rng = np.random.default_rng(1)
    for k in range(O.B01, O.D03 + 1):
        osim.F[k] *= 1.0 + 0.01 * rng.standard_normal(osim.F[k].shape)
    g = gpu_from_oracle(osim)
    g.predict()
    osim.predict()
    assert_planes(g.planes(), osim.F, what="predict")


@pytest.mark.parametrize("cfg", [BASE, RAGGED, FLAT])
def test_push(torch_cuda, cfg):
    osim = oracle_state(cfg, cells=None if cfg is BASE else odd_cells(cfg))
    osim.predict()
    g = gpu_from_oracle(osim)
    for s in range(2):
        g.push(s)
        osim.push(s)
    for s in range(2):
        assert_particles(g.get_particles(s), osim.species[s].view())
    d = g.diagnostics()
    assert [d["left_inner"], d["left_outer"], d["reflections"], d["nonfinite"]] == \
        [int(x) for x in osim.counters]


@pytest.mark.parametrize("cfg", [BASE, RAGGED, FLAT])
def test_deposit(torch_cuda, cfg):
    osim = oracle_state(cfg, cells=None if cfg is BASE else odd_cells(cfg))
    osim.predict()
    for s in range(2):
        osim.push(s)
    g = gpu_from_oracle(osim)
    g.deposit()
    osim.deposit()
    assert_currents(g.planes(), osim.F)


@pytest.mark.parametrize("cfg", [BASE, RAGGED, FLAT])
def test_advance(torch_cuda, cfg):
    osim = oracle_state(cfg, cells=None if cfg is BASE else odd_cells(cfg))
    osim.predict()
    for s in range(2):
        osim.push(s)
    osim.deposit()
    g = gpu_from_oracle(osim)
    g.advance()
    osim.advance()
    assert_planes(g.planes(), osim.F, planes=AFTER_ADVANCE, what="advance")


def random_particle_state(cfg, n, seed):
    rng = np.random.default_rng(seed)
    a = {k: np.zeros(n, dtype=t) for k, t in O.PARTICLE_FIELDS.items()}
    a["i1"] = rng.integers(0, cfg["n_r"], n).astype(np.int32)
    a["i2"] = rng.integers(0, cfg["n_theta"], n).astype(np.int32)
    a["tag"] = rng.choice([0, 1, 1, 1, 1, 2], n).astype(np.uint8)
    for k in ("dx1", "dx2", "u1", "u2", "u3", "phi", "w", "dx1p", "dx2p"):
        a[k] = rng.random(n)
    a["i1p"], a["i2p"] = a["i1"].copy(), a["i2"].copy()
    return a


@pytest.mark.parametrize("n,tiles", [(1, (16, 16)), (4097, (16, 16)), (100003, (8, 4)),
                                     (70001, (37, 23)), (0, (16, 16))])
def test_sort_bit_exact(torch_cuda, n, tiles):
    cfg = dict(RAGGED, tile_r=tiles[0], tile_theta=tiles[1])
    osim = O.OracleSim(dict(cfg, dt=0.01))
    arr = random_particle_state(cfg, n, 3)
    osim.add_raw_species(arr, 1.0, 1.0)
    g = gpu_from_oracle(osim, extra_capacity=5)
    g.sort(0)
    if n:
        osim.sort(0, *tiles)
    pg, po = g.get_particles(0), osim.species[0].view()
    assert len(pg["i1"]) == len(po["i1"]) == int(np.sum(arr["tag"] == 1))
    for k in po:
        assert np.array_equal(pg[k], po[k]), k


def test_sort_beyond_one_chunk_of_the_total_scan(torch_cuda):
    """68,000,000 particles: more segment totals of the digit histogram (one per four blocks
    of 4096 keys) than the 4096 one pass of the totals' block scan covers, so the scan carries
    its running total across chunks (a species of the 2048^2 workloads, 67,108,864 particles,
    fills exactly one). The weight carries each particle's input index (exact in FP64): after
    the sort the weights are the input indices in the stable order of the oracle's keys, the
    dead particles dropped, and the cells follow them."""
    from paper_2511_17701_gb300 import Sim
    n, tiles = 68_000_000, (16, 16)
    cfg = dict(BASE, tile_r=tiles[0], tile_theta=tiles[1], dt=0.01)
    rng = np.random.default_rng(17)
    i1 = rng.integers(0, cfg["n_r"], n, dtype=np.int32)
    i2 = rng.integers(0, cfg["n_theta"], n, dtype=np.int32)
    tag = (rng.random(n) < 0.9).astype(np.uint8)
    arrays = {"i1": i1, "i2": i2, "tag": tag, "w": np.arange(n, dtype=np.float64)}
    zero = np.zeros(n)
    for k in ("dx1", "dx2", "u1", "u2", "u3", "phi"):
        arrays[k] = zero
    g = Sim(cfg, [n])
    g.init_metric()
    g.set_particles(0, arrays, 1.0, 1.0)
    g.sort(0)
    p = g.get_particles(0)
    del g
    keys = O.sort_keys(cfg, tiles[0], tiles[1], i1, i2, tag)
    order = np.argsort(keys, kind="stable")
    order = order[: int(np.count_nonzero(tag == 1))]  # dead keys (0xFFFFFFFF) sort last
    assert len(p["w"]) == len(order)
    assert np.array_equal(p["w"], order.astype(np.float64))
    assert np.array_equal(p["i1"], i1[order]) and np.array_equal(p["i2"], i2[order])


def test_full_step_with_sort(torch_cuda):
    cfg = dict(BASE, sort_every=1, tile_r=8, tile_theta=8)
    osim = oracle_state(cfg)
    g = gpu_from_oracle(osim)
    g.step(1)
    osim.step(1, sort_every=1, tr=8, tt=8)
    F = g.planes()
    assert_planes(F, osim.F, planes=AFTER_ADVANCE, what="step")
    for s in range(2):
        assert_particles(g.get_particles(s), osim.species[s].view())


@pytest.mark.parametrize("cfg", [BASE, RAGGED])
def test_fused_step_equals_separate_calls(torch_cuda, cfg):
    osim = oracle_state(cfg, cells=None if cfg is BASE else odd_cells(cfg))
    g1 = gpu_from_oracle(osim)
    g2 = gpu_from_oracle(osim)
    g1.step(2)
    for _ in range(2):
        g2.predict()
        g2.push(0)
        g2.push(1)
        g2.deposit()
        g2.advance()
    F1, F2 = g1.planes(), g2.planes()
    # the two deposit orders differ only in the order of the atomic sums
    assert_planes(F1, F2, planes=AFTER_ADVANCE, rtol=1e-13, what="fused vs separate")
    for s in range(2):
        assert_particles(g1.get_particles(s), g2.get_particles(s), rtol=1e-13)


def test_ten_step_trajectory(torch_cuda):
    """Ten full steps on both sides: differences grow from rounding, so the bound is
    looser than the per-step one."""
    cfg = BASE
    osim = oracle_state(cfg)
    g = gpu_from_oracle(osim)
    g.step(10)
    osim.step(10)
    assert_planes(g.planes(), osim.F, planes=range(12), rtol=1e-9, what="10 steps")
    for s in range(2):
        assert_particles(g.get_particles(s), osim.species[s].view(), rtol=1e-9)


def test_axis_and_horizon_edge_particles(torch_cuda):
    """Fast particles placed to reflect off both axes, to fall through the horizon layer
    and to leave through the outer edge; three pushes in frozen fields, each from the
    oracle's state."""
    cfg = BASE
    osim = O.OracleSim(cfg)
    osim.init_fields(O.FIELD_WALD, 1.0)
    n = 4000
    rng = np.random.default_rng(9)
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
    g = gpu_from_oracle(osim)
    for _ in range(3):
        g.set_particles(0, osim.species[0].view(), qm, qc)
        g.push(0)
        osim.push(0)
        assert_particles(g.get_particles(0), osim.species[0].view())
    d = g.diagnostics()
    assert min(osim.counters[:3]) > 0
    assert [d["left_inner"], d["left_outer"], d["reflections"], d["nonfinite"]] == \
        [int(x) for x in osim.counters]


def test_empty_species(torch_cuda):
    osim = oracle_state(BASE, species=0)
    osim.add_raw_species({k: np.zeros(0, dtype=t) for k, t in O.PARTICLE_FIELDS.items()},
                         1.0, 1.0)
    g = gpu_from_oracle(osim)
    g.step(2)
    osim.step(2)
    assert_planes(g.planes(), osim.F, planes=range(12), what="empty")
    assert g.count(0) == 0


@pytest.mark.parametrize("cfg", [BASE, RAGGED, FLAT])
def test_stop_on_exact_repeat_is_bit_identical(torch_cuda, cfg):
    """The implicit pushes stop once an iterate repeats bit for bit; forcing all n_iter
    iterations must give the same bits (three pushes in frozen fields: no atomics feed
    back, so both runs are deterministic)."""
    osim = oracle_state(cfg, cells=None if cfg is BASE else odd_cells(cfg))
    osim.predict()
    g1 = gpu_from_oracle(osim)
    g2 = gpu_from_oracle(osim, full_iterations=1)
    for _ in range(3):
        for s in range(2):
            g1.push(s)
            g2.push(s)
    for s in range(2):
        p1, p2 = g1.get_particles(s), g2.get_particles(s)
        for k in p1:
            assert np.array_equal(p1[k], p2[k]), k


REFINED = 1e-12  # iter_tol of the refined implicit iterations (the bench's setting)


@pytest.mark.parametrize("cfg", [BASE, RAGGED, FLAT])
def test_refined_iterations_push(torch_cuda, cfg):
    """FP32 predictor + FP64 iterations to iter_tol: the same FP64 fixed point as the oracle's
    n_iter iterations, within the per-step parity bound."""
    osim = oracle_state(cfg, cells=None if cfg is BASE else odd_cells(cfg))
    osim.predict()
    g = gpu_from_oracle(osim, iter_tol=REFINED)
    for s in range(2):
        g.push(s)
        osim.push(s)
    for s in range(2):
        assert_particles(g.get_particles(s), osim.species[s].view())


def test_refined_iterations_full_step_and_trajectory(torch_cuda):
    cfg = dict(BASE, sort_every=1, tile_r=8, tile_theta=8)
    osim = oracle_state(cfg)
    g = gpu_from_oracle(osim, iter_tol=REFINED)
    g.step(1)
    osim.step(1, sort_every=1, tr=8, tt=8)
    assert_planes(g.planes(), osim.F, planes=AFTER_ADVANCE, what="refined step")
    for s in range(2):
        assert_particles(g.get_particles(s), osim.species[s].view())
    g.step(9)
    osim.step(9, sort_every=1, tr=8, tt=8)
    assert_planes(g.planes(), osim.F, planes=range(12), rtol=1e-9, what="refined 10 steps")
    for s in range(2):
        assert_particles(g.get_particles(s), osim.species[s].view(), rtol=1e-9)


def test_refined_iterations_edge_particles(torch_cuda):
    """Axis reflections, horizon and outer removals with the refined iterations."""
    cfg = BASE
    osim = O.OracleSim(cfg)
    osim.init_fields(O.FIELD_WALD, 1.0)
    n = 4000
    rng = np.random.default_rng(19)
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
    g = gpu_from_oracle(osim, iter_tol=REFINED)
    for _ in range(3):
        g.set_particles(0, osim.species[0].view(), qm, qc)
        g.push(0)
        osim.push(0)
        assert_particles(g.get_particles(0), osim.species[0].view())


def test_set_particles_without_previous_position(torch_cuda):
    """grpic_set_particles with null i1p, i2p, dx1p, dx2p sets the previous position to the
    position; a push from there is the push of the full state."""
    osim = oracle_state(BASE)
    osim.predict()
    sp = osim.species[0]
    g = gpu_from_oracle(osim)
    state = {k: v for k, v in sp.view().items() if k not in ("i1p", "i2p", "dx1p", "dx2p")}
    g.set_particles(0, state, sp.qm, sp.qc)
    got = g.get_particles(0)
    for a, b in (("i1p", "i1"), ("i2p", "i2"), ("dx1p", "dx1"), ("dx2p", "dx2")):
        assert np.array_equal(got[a], got[b]), a
    g.push(0)
    osim.push(0)
    assert_particles(g.get_particles(0), sp.view())


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_fused_step_without_previous_positions(torch_cuda, precision):
    """grpic_set_keep_prev(0): the fused push + deposit skips the previous-position stores.
    From the same state the particles come out with the same bits (only the stores differ),
    the fields within the parity bound (atomic order), and the calls that read the previous
    positions refuse them until a separate push stores them again."""
    from paper_2511_17701_gb300 import FIELD_WALD, GrpicError
    cfg = dict(BASE, precision=precision, sort_every=1, tile_r=8, tile_theta=8)
    osim = oracle_state(cfg)
    if precision == "mixed":
        from parity import round_state_fp32
        round_state_fp32(osim)
    a, b = gpu_from_oracle(osim), gpu_from_oracle(osim)
    b.set_keep_prev(False)
    a.step(1)
    b.step(1)
    for s in range(2):
        pa, pb = a.get_particles(s), b.get_particles(s)
        for k in ("i1", "i2", "dx1", "dx2", "u1", "u2", "u3", "phi", "w", "tag"):
            assert np.array_equal(pa[k], pb[k]), (s, k)
    rt = 1e-12 if precision == "fp64" else 1e-5
    assert_planes(b.planes(), a.planes(), planes=AFTER_ADVANCE, rtol=rt, what="keep_prev")
    for call in (lambda: b.deposit(), lambda: b.invariants(0, FIELD_WALD, 1.0),
                 lambda: b.charge_check(after_step=True)):
        with pytest.raises(GrpicError, match="status 4"):
            call()
    b.predict()
    for s in range(2):
        b.push(s)  # a separate push stores them
    b.deposit()
    b.charge_check(after_step=False)
    b.invariants(0, FIELD_WALD, 1.0)
