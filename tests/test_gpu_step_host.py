"""grpic_step_host: one PIC step (Sec. 3.4) with the particle state streamed through host
memory, the copies of each species overlapping the work on the other.

The step runs the same kernels as grpic_step, so the particle state it leaves (the push reads
only the fields and the state, never the atomically summed currents of the same step) must
equal grpic_step's to the bit after one step, and the FP64 run must follow the oracle over
several steps with sorts that drop the particles that left. Host arrays are numpy (pageable)
or torch tensors in page-locked memory.
"""
import numpy as np
import pytest

import workloads as W
from oracle import oracle as O
from parity import (assert_particles, assert_planes, gpu_from_oracle, oracle_state,
                    particle_errors, round_state_fp32)

pytestmark = pytest.mark.gpu

BASE = W.grid_config("wald64")
STATE = ("i1", "i2", "dx1", "dx2", "u1", "u2", "u3", "phi", "w", "tag")
AFTER_ADVANCE = list(range(12)) + [15, 16, 17, 18, 19, 20]


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def host_state(g, pinned=False):
    """The context's particle state copied into host arrays of its own types."""
    import torch
    states, counts = [], []
    for s in range(g.n_species):
        p = g.get_particles(s)
        if pinned:
            d = {}
            for k in STATE:
                t = torch.empty(p[k].shape, dtype=getattr(torch, p[k].dtype.name), pin_memory=True)
                t.numpy()[:] = p[k]
                d[k] = t
        else:
            d = {k: np.ascontiguousarray(p[k]) for k in STATE}
        states.append(d)
        counts.append(len(p["i1"]))
    return states, counts


def as_numpy(d, n):
    return {k: (v.numpy() if hasattr(v, "numpy") else v)[:n].copy() for k, v in d.items()}


def edge_plasma(cfg, n=6000, seed=29):
    """Pairs in the bulk and in the horizon layer (some leave through the inner boundary)."""
    osim = O.OracleSim(cfg)
    osim.init_fields(O.FIELD_WALD, 1.0)
    rng = np.random.default_rng(seed)
    nr, nt = cfg["n_r"], cfg["n_theta"]
    x1 = np.concatenate([rng.uniform(0.0, 1.5, n // 2), rng.uniform(2.0, nr - 2.0, n - n // 2)])
    x2 = rng.uniform(0.0, nt, n)
    pos = {"i1": np.floor(x1).astype(np.int32), "i2": np.floor(x2).astype(np.int32)}
    pos["dx1"], pos["dx2"] = x1 - pos["i1"], x2 - pos["i2"]
    for q in (1.0, -1.0):
        uh = W.maxwell_juttner(rng, n, 2.0)
        qm, qc = W.species_coefficients(q)
        osim.add_species(pos, uh, np.full(n, 0.1), qm, qc)
    return osim


@pytest.mark.parametrize("pinned", [False, True])
def test_step_host_matches_step_fp64(torch_cuda, pinned):
    cfg = dict(BASE, sort_every=1, tile_r=8, tile_theta=8)
    osim = oracle_state(cfg)
    a = gpu_from_oracle(osim)
    b = gpu_from_oracle(osim)
    states, counts = host_state(b, pinned)
    a.step(1)
    counts = b.step_host(states, counts)
    for s in range(2):
        pa = a.get_particles(s)
        assert counts[s] == len(pa["i1"])
        hb = as_numpy(states[s], counts[s])
        for k in STATE:
            assert np.array_equal(pa[k], hb[k]), (s, k)
    assert_planes(b.planes(), a.planes(), planes=AFTER_ADVANCE, rtol=1e-13, what="fields")


@pytest.mark.parametrize("n_keep", [3, 1001])
def test_step_host_ranges_fp64(torch_cuda, n_keep):
    """An FP64 context streams each species as four ranges: counts that four does not
    divide, fewer particles than ranges, steps without a sort."""
    osim = oracle_state(dict(BASE, sort_every=0))
    a, b = gpu_from_oracle(osim), gpu_from_oracle(osim)
    for g in (a, b):
        for s in range(2):
            sp = osim.species[s]
            g.set_particles(s, {k: v[:n_keep] for k, v in sp.view().items()}, sp.qm, sp.qc)
    states, counts = host_state(b, pinned=True)
    assert counts == [n_keep, n_keep]
    a.step(1)
    counts = b.step_host(states, counts)
    for s in range(2):
        pa = a.get_particles(s)
        assert counts[s] == len(pa["i1"]) == n_keep
        hb = as_numpy(states[s], counts[s])
        for k in STATE:
            assert np.array_equal(pa[k], hb[k]), (s, k)
    a.step(1)
    counts = b.step_host(states, counts)
    for s in range(2):
        assert_particles(b.get_particles(s), a.get_particles(s), rtol=1e-13)


def test_step_host_follows_the_oracle_with_removals(torch_cuda):
    """Three streamed steps with a sort each: particles that fell through the inner boundary
    are dropped by the next sort, on both sides, in the same order."""
    cfg = dict(BASE, sort_every=1, tile_r=8, tile_theta=8)
    osim = edge_plasma(cfg)
    g = gpu_from_oracle(osim)
    states, counts = host_state(g, pinned=True)
    n0 = list(counts)
    for _ in range(3):
        counts = g.step_host(states, counts)
    osim.step(3, sort_every=1, tr=8, tt=8)
    for s in range(2):
        po = osim.species[s].view()
        assert counts[s] == len(po["i1"])
        hb = as_numpy(states[s], counts[s])
        gp = g.get_particles(s)
        for k in STATE:
            assert np.array_equal(gp[k], hb[k]), (s, k)
        assert_particles(gp, po)
    assert counts[0] < n0[0] and counts[1] < n0[1]
    assert_planes(g.planes(), osim.F, planes=AFTER_ADVANCE, what="3 streamed steps")


def test_step_host_mixed(torch_cuda):
    cfg = dict(BASE, precision="mixed", sort_every=2, tile_r=8, tile_theta=8)
    osim = oracle_state(cfg)
    round_state_fp32(osim)
    a = gpu_from_oracle(osim, precision="mixed")
    b = gpu_from_oracle(osim, precision="mixed")
    states, counts = host_state(b, pinned=True)
    a.step(1)
    counts = b.step_host(states, counts)
    osim.step(1, sort_every=2, tr=8, tt=8)
    for s in range(2):
        pa = a.get_particles(s)
        hb = as_numpy(states[s], counts[s])
        for k in STATE:
            assert np.array_equal(pa[k], hb[k]), (s, k)
        e = particle_errors(b.get_particles(s), osim.species[s].view())
        assert max(e.values()) <= 1e-5, (s, e)


def test_step_host_errors(torch_cuda):
    from paper_2511_17701_gb300 import GrpicError
    osim = oracle_state(BASE)
    g = gpu_from_oracle(osim)
    states, counts = host_state(g)
    with pytest.raises(GrpicError):
        g.step_host(states, [counts[0], 10 ** 9])  # above the capacity
    bad = [dict(states[0]), states[1]]
    bad[0]["u2"] = None
    with pytest.raises(GrpicError):
        g.step_host(bad, counts)  # a null array
    # nothing ran: a valid call afterwards still matches grpic_step
    ref = gpu_from_oracle(osim)
    ref.step(1)
    counts = g.step_host(states, counts)
    for s in range(2):
        pr = ref.get_particles(s)
        hb = as_numpy(states[s], counts[s])
        for k in STATE:
            assert np.array_equal(pr[k], hb[k]), (s, k)


def test_step_host_empty_species(torch_cuda):
    """A species holding no particles streams nothing and stays empty."""
    osim = oracle_state(BASE)
    g = gpu_from_oracle(osim)
    states, counts = host_state(g)
    counts = g.step_host(states, [counts[0], 0])
    assert counts[1] == 0
    ref = gpu_from_oracle(osim)
    ref.set_particles(1, {k: v[:0] for k, v in osim.species[1].view().items()},
                      osim.species[1].qm, osim.species[1].qc)
    ref.step(1)
    pr = ref.get_particles(0)
    hb = as_numpy(states[0], counts[0])
    for k in STATE:
        assert np.array_equal(pr[k], hb[k]), k
