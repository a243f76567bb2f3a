"""The allocation-free sort entry point agrees with the arena-based one.

grpic_sort_permutation_noalloc serves callers that may not allocate device memory and
cannot lend scratch space (a host program whose own pool owns the GPU's memory, or a
time-critical loop that cannot afford the synchronisation of a cudaMalloc): its scratch
is a fixed device array inside the library. This test feeds it the cell indices and tags
of a species held by an ordinary context, sorts the same species with grpic_sort, and
checks that the returned permutation reproduces grpic_sort's result exactly (the order
is unique, so the comparison is bit-exact), on two calls in a row with different sizes
so that nothing left in the shared scratch by the first call leaks into the second.
"""

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


CFG = dict(metric="ks", a=0.9, n_r=37, n_theta=23, r_min=1.3, r_max=12.0, dt=0.01,
           tile_r=8, tile_theta=4)


def random_state(n, seed):
    from paper_2511_17701_gb300.binding import PARTICLE_ARRAYS
    rng = np.random.default_rng(seed)
    a = {k: np.zeros(n, dtype=t) for k, t in PARTICLE_ARRAYS}
    a["i1"] = rng.integers(0, CFG["n_r"], n).astype(np.int32)
    a["i2"] = rng.integers(0, CFG["n_theta"], n).astype(np.int32)
    a["tag"] = rng.choice([0, 1, 1, 1, 1, 2], n).astype(np.uint8)
    for k in ("dx1", "dx2", "u1", "u2", "u3", "phi", "w", "dx1p", "dx2p"):
        a[k] = rng.random(n)
    a["i1p"], a["i2p"] = a["i1"].copy(), a["i2"].copy()
    return a


def noalloc_permutation(torch, sim, n):
    from paper_2511_17701_gb300 import binding as B
    v = sim.species_views(0)
    perm = torch.full((max(n, 1),), -1, dtype=torch.int32, device=sim.device)
    n_alive = torch.full((1,), -1, dtype=torch.int64, device=sim.device)
    st = B.lib().grpic_sort_permutation_noalloc(
        CFG["n_r"], CFG["n_theta"], CFG["tile_r"], CFG["tile_theta"], v["i1"].data_ptr(),
        v["i2"].data_ptr(), v["tag"].data_ptr(), n, perm.data_ptr(), n_alive.data_ptr(),
        sim.stream.cuda_stream)
    assert st == B.OK
    sim.sync()
    return perm.cpu().numpy()[:n].astype(np.int64), int(n_alive.item())


def test_noalloc_sort_matches_grpic_sort_twice(torch_cuda):
    from paper_2511_17701_gb300 import Sim
    for n, seed in ((300007, 1), (70001, 2)):
        sim = Sim(CFG, [n])
        state = random_state(n, seed)
        sim.set_particles(0, state, 1.0, 1.0)
        perm, n_alive = noalloc_permutation(torch_cuda, sim, n)
        sim.sort(0)
        after = sim.get_particles(0)
        assert n_alive == len(after["i1"]) == int(np.sum(state["tag"] == 1))
        assert sorted(perm.tolist()) == list(range(n))
        for k, v in after.items():
            assert np.array_equal(v, state[k][perm[:n_alive]]), k
        # the particles that are not alive follow in input order
        rest = perm[n_alive:]
        assert np.all(np.diff(rest) > 0) and np.all(state["tag"][rest] != 1)
        sim.close()


def test_noalloc_sort_rejects_too_many(torch_cuda):
    from paper_2511_17701_gb300 import binding as B
    lib = B.lib()
    big = (1 << 20) + 1
    dummy = torch_cuda.zeros(8, dtype=torch_cuda.int64, device="cuda:0")
    p = dummy.data_ptr()
    assert lib.grpic_sort_permutation_noalloc(37, 23, 8, 4, p, p, p, big, p, p, None) == B.ECAPACITY
    assert lib.grpic_sort_permutation_noalloc(37, 23, 0, 4, p, p, p, 10, p, p, None) == B.EINVAL


def test_noalloc_sort_at_its_maximum_size(torch_cuda):
    """n = GRPIC_NOALLOC_SORT_MAX, where the fixed scratch (digit histograms, scan sums) is
    full: the permutation reproduces grpic_sort's result."""
    from paper_2511_17701_gb300 import Sim
    n = 1 << 20
    sim = Sim(CFG, [n])
    state = random_state(n, 3)
    sim.set_particles(0, state, 1.0, 1.0)
    perm, n_alive = noalloc_permutation(torch_cuda, sim, n)
    sim.sort(0)
    after = sim.get_particles(0)
    assert n_alive == len(after["i1"]) == int(np.sum(state["tag"] == 1))
    assert np.array_equal(np.sort(perm), np.arange(n))
    for k, v in after.items():
        assert np.array_equal(v, state[k][perm[:n_alive]]), k
    sim.close()


def test_noalloc_sort_of_nothing_sets_zero_alive(torch_cuda):
    from paper_2511_17701_gb300 import binding as B
    lib = B.lib()
    n_alive = torch_cuda.full((1,), -7, dtype=torch_cuda.int64, device="cuda:0")
    st = lib.grpic_sort_permutation_noalloc(37, 23, 8, 4, None, None, None, 0, None,
                                            n_alive.data_ptr(), None)
    assert st == B.OK
    torch_cuda.cuda.synchronize()
    assert int(n_alive.item()) == 0


def test_noalloc_sort_rejects_keys_beyond_the_dead_key(torch_cuda):
    """A tile-padded cell count above 2^31 - 1 would let live keys reach the key of dead
    particles: refused before any work."""
    from paper_2511_17701_gb300 import binding as B
    lib = B.lib()
    dummy = torch_cuda.zeros(8, dtype=torch_cuda.int64, device="cuda:0")
    p = dummy.data_ptr()
    assert lib.grpic_sort_permutation_noalloc(65536, 65536, 1, 1, p, p, p, 4, p, p, None) == B.EINVAL
    assert lib.grpic_sort_permutation_noalloc(65537, 8, 1, 1, p, p, p, 4, p, p, None) == B.EINVAL
    assert lib.grpic_sort_permutation_noalloc(37, 23, 65537, 4, p, p, p, 4, p, p, None) == B.EINVAL
    assert lib.grpic_sort_permutation_noalloc(50000, 50000, 1, 1, p, p, p, 4, p, p, None) == B.EINVAL
