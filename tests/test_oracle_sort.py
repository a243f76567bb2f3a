"""Pins of the oracle's particle sort (an addition of this implementation; the
paper's loop has no sort). Checked against its definition: keys in tile-major
cell order, stability (equal keys keep their input order), removal of particles
that are not alive, and a bijective permutation."""
import numpy as np

from oracle import oracle as O

CFG = dict(metric="ks", a=0.9, n_r=37, n_theta=21, r_min=1.3641, r_max=10.0)


def test_key_layout_by_hand():
    # n_r = 37, tiles 8 x 4: 5 tiles per row of tiles
    assert O.sort_key(CFG, 8, 4, 0, 0, 1) == 0
    assert O.sort_key(CFG, 8, 4, 7, 0, 1) == 7
    assert O.sort_key(CFG, 8, 4, 0, 1, 1) == 8
    assert O.sort_key(CFG, 8, 4, 8, 0, 1) == 32          # second tile
    assert O.sort_key(CFG, 8, 4, 36, 3, 1) == 4 * 32 + 3 * 8 + 4
    assert O.sort_key(CFG, 8, 4, 1, 4, 1) == 5 * 32 + 1  # second row of tiles
    assert O.sort_key(CFG, 8, 4, 3, 3, 0) == 0xFFFFFFFF
    assert O.sort_key(CFG, 8, 4, 3, 3, 2) == 0xFFFFFFFF


def test_sort_is_stable_and_drops_dead():
    rng = np.random.default_rng(11)
    n = 5000
    sim = O.OracleSim(dict(CFG, dt=0.01))
    arr = {k: np.zeros(n, dtype=t) for k, t in O.PARTICLE_FIELDS.items()}
    arr["i1"] = rng.integers(0, CFG["n_r"], n).astype(np.int32)
    arr["i2"] = rng.integers(0, CFG["n_theta"], n).astype(np.int32)
    arr["tag"] = rng.choice([0, 1, 1, 1, 2], n).astype(np.uint8)
    arr["dx1"] = np.arange(n, dtype=np.float64)  # carries the input index
    s = sim.add_raw_species(arr, 1.0, 1.0)
    keys = np.array([O.sort_key(CFG, 8, 4, int(a), int(b), int(t))
                     for a, b, t in zip(arr["i1"], arr["i2"], arr["tag"])], dtype=np.uint64)
    perm = sim.sort(0, 8, 4)
    alive = int(np.sum(arr["tag"] == 1))
    assert s.n == alive
    assert sorted(perm.tolist()) == list(range(n))
    want = np.lexsort((np.arange(n), keys))  # by key, ties by input position
    assert np.array_equal(perm, want)
    v = s.view()
    assert np.array_equal(v["dx1"], want[:alive].astype(np.float64))
    assert np.all(v["tag"] == 1)
    assert np.all(np.diff(keys[want[:alive]].astype(np.int64)) >= 0)


def test_vectorised_keys_equal_the_c_key():
    """oracle.sort_keys (numpy, for the full-size tests) against ora_sort_key element by
    element, on ragged tiles with dead and leaving particles."""
    cfg = CFG
    rng = np.random.default_rng(17)
    n = 4000
    i1 = rng.integers(0, CFG["n_r"], n)  # cells of the domain (live particles have no other)
    i2 = rng.integers(0, CFG["n_theta"], n)
    tag = rng.choice([0, 1, 1, 2], n)
    for tr, tt in ((16, 16), (5, 7), (1, 1)):
        got = O.sort_keys(cfg, tr, tt, i1, i2, tag)
        want = np.array([O.sort_key(cfg, tr, tt, int(a), int(b), int(c))
                         for a, b, c in zip(i1, i2, tag)], dtype=np.uint32)
        assert np.array_equal(got, want), (tr, tt)
