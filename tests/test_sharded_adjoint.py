"""The adjoint sharded by particle across ranks, on CPU: the exact binned sum behind the
B0 gradient, and two gloo ranks with an uneven split of the particles.

The binned sum: bins built from their definition in include/grpic.h (a finite double is
M 2^(b - 1075) with b its biased exponent field, 1 for subnormals; per b the int64 sums of
M >> 32 and M & 0xffffffff) are rounded by the library's host routine grpic_sum_bins_value;
the result must be the correctly rounded sum, which Python's math.fsum also returns
(Shewchuk's exact summation), bit for bit. The GPU kernel that fills the bins is checked
against the same definition in test_gpu_adjoint.py.

The sharded adjoint: the per-particle terms come from the oracle's complex-step Jacobian of
the frozen-field push (exact to rounding); two ranks each take an uneven share, bin their
terms, all-reduce the bins over gloo and round once. The gradient with respect to B0 must
be the same bits on both ranks and in one process, and each rank's gradients with respect
to its particles' initial states those of the single process.
"""
import math
import os
import socket
import sys

import numpy as np
import pytest

from paper_2511_17701_gb300.binding import SUM_BINS, sum_bins_value
from paper_2511_17701_gb300.sharded import shard_bounds

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def bins_of(values) -> np.ndarray:
    """The bins of the finite values, from their definition."""
    v = np.asarray(values, dtype=np.float64).ravel()
    bits = v.view(np.uint64)
    b = ((bits >> np.uint64(52)) & np.uint64(0x7FF)).astype(np.int64)
    ok = b != 0x7FF
    f = (bits & np.uint64((1 << 52) - 1)).astype(np.int64)
    M = np.where(b > 0, f | (1 << 52), f)
    M = np.where((bits >> np.uint64(63)) == 1, -M, M)
    bb = np.where(b > 0, b, 1)
    hi = M >> 32
    lo = M - (hi << 32)
    out = np.zeros(2 * SUM_BINS, dtype=np.int64)
    np.add.at(out, 2 * bb[ok], hi[ok])
    np.add.at(out, 2 * bb[ok] + 1, lo[ok])
    return out


def cases():
    rng = np.random.default_rng(11)
    yield rng.normal(size=1000)
    yield rng.normal(size=5000) * np.exp(rng.uniform(-200, 200, size=5000))  # wide exponents
    x = rng.normal(size=2000)
    yield np.concatenate([x, -x[::-1], [1e-300, 3.0]])  # cancellation to a tiny total
    yield np.array([1.0, 2.0 ** -53, 2.0 ** -53])  # the exact tie and a carry above it
    yield np.array([1.0, 2.0 ** -53])  # a tie rounded to even (down)
    yield np.array([1.0 + 2.0 ** -52, 2.0 ** -53])  # a tie rounded to even (up)
    yield np.array([5e-324, 5e-324, -1e-310, 2.2e-308])  # subnormals
    yield -np.abs(rng.normal(size=300)) * 1e10  # a negative total
    yield np.array([1.7e308, 1.7e308, -1.7e308])  # beyond the double range on the way
    yield np.array([np.nan, 1.5, np.inf, -2.25])  # non-finite terms are skipped
    yield np.zeros(10)
    yield np.array([])


@pytest.mark.parametrize("k", range(12))
def test_binned_sum_is_correctly_rounded(k):
    v = list(cases())[k]
    finite = v[np.isfinite(v)]
    want = math.fsum(finite) if not (k == 8) else 1.7e308
    got = sum_bins_value(bins_of(v))
    assert got == want or (math.isnan(got) and math.isnan(want)), (k, got, want)
    # splitting the values and adding the bins gives the same bits
    if v.size > 3:
        parts = np.array_split(v, 7)
        assert sum_bins_value(sum(bins_of(p) for p in parts)) == got


def test_shard_bounds_cover_every_particle_once():
    for n in (0, 1, 7, 100, 101, 1 << 20):
        for world in (1, 2, 3, 8):
            spans = [shard_bounds(n, r, world) for r in range(world)]
            assert spans[0][0] == 0 and spans[-1][1] == n
            assert all(a[1] == b[0] for a, b in zip(spans, spans[1:]))
            sizes = [hi - lo for lo, hi in spans]
            assert max(sizes) - min(sizes) <= 1


# ---------------------------------------------------------------------------------------
# two gloo ranks
# ---------------------------------------------------------------------------------------
N_PART, N_STEPS = 23, 40
SPLIT = (0, 15, 23)  # uneven on purpose: 15 and 8 particles


def _problem():
    import workloads as W
    from oracle import oracle as O
    cfg = W.grid_config("wald64", r_absorb=1e300)
    osim = O.OracleSim(cfg)
    osim.init_fields(O.FIELD_WALD, 1.0)
    tp = W.probe_particles(cfg, N_PART, 3, (15.0, 50.0), (12.0, 52.0), 0.5)
    qm, qc = W.species_coefficients(1.0)
    sp = osim.add_species(tp["pos"], tp["uhat"], tp["w0"], qm, qc)
    v = sp.view()
    st0 = np.stack([v["i1"] + v["dx1"], v["i2"] + v["dx2"], v["phi"], v["u1"], v["u2"], v["u3"]])
    cot = np.random.default_rng(9).normal(size=(6, N_PART))
    return osim, st0, cot, qm


def _oracle_local(osim, qm):
    """A rank's local adjoint from the oracle: the complex-step Jacobian gives cot^T J per
    particle (state columns and the field scale)."""
    import torch
    from oracle import oracle as O

    def run(state0, cot):
        st = state0.numpy()
        final, J = O.frozen_jacobian(osim, st, 1.0, qm, N_STEPS, 60)
        c = cot.numpy()
        g = np.einsum("in,nij->jn", c, J)  # (7, n): d/d state0 rows, then d/d scale
        return (torch.from_numpy(final), torch.from_numpy(g[:6].copy()),
                torch.from_numpy(bins_of(g[6])))
    return run


def _rank(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world))
    sys.path.insert(0, ROOT)
    sys.path.insert(0, os.path.join(ROOT, "tests"))
    import torch
    import torch.distributed as dist

    from paper_2511_17701_gb300.sharded import sharded_adjoint
    dist.init_process_group("gloo", rank=rank, world_size=world)
    osim, st0, cot, qm = _problem()
    lo, hi = SPLIT[rank], SPLIT[rank + 1]
    out, gin, gb0 = sharded_adjoint(_oracle_local(osim, qm), torch.from_numpy(st0[:, lo:hi].copy()),
                                    torch.from_numpy(cot[:, lo:hi].copy()))
    q.put((rank, gin.numpy(), gb0))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_give_the_single_process_gradient_bit_for_bit():
    torch = pytest.importorskip("torch")
    from paper_2511_17701_gb300.sharded import sharded_adjoint
    osim, st0, cot, qm = _problem()
    _, gin1, gb1 = sharded_adjoint(_oracle_local(osim, qm), torch.from_numpy(st0),
                                   torch.from_numpy(cot))
    ctx = torch.multiprocessing.get_context("spawn")
    qu = ctx.Queue()
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    procs = [ctx.Process(target=_rank, args=(r, 2, port, qu)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted((qu.get(timeout=600) for _ in procs), key=lambda t: t[0])
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    for rank, gin, gb0 in res:
        assert gb0 == gb1, (rank, gb0, gb1)  # the same bits on every rank
        lo, hi = SPLIT[rank], SPLIT[rank + 1]
        assert np.array_equal(gin, gin1.numpy()[:, lo:hi], equal_nan=True)
    assert gb1 != 0.0 and math.isfinite(gb1)
    # and that value is the correctly rounded sum of the particles' terms
    from oracle import oracle as O
    _, J = O.frozen_jacobian(osim, st0, 1.0, qm, N_STEPS, 60, inputs=["scale"])
    terms = np.einsum("in,ni->n", cot, J[:, :, 0])
    assert gb1 == math.fsum(terms[np.isfinite(terms)])
