"""The seeded input generators (workloads/) that feed both the oracle and the CUDA path,
checked against what the input recipe fixes: the isotropic Maxwell-Juttner momenta have the
closed-form mean Lorentz factor <gamma> = 3 theta + K_1(1/theta) / K_2(1/theta) (K the
modified Bessel functions of the second kind) and zero mean momentum with equal variances
along the three axes; a pair plasma holds ppc particles in every cell, electrons and
positrons at the same positions with independent momenta and weight 1/ppc; the same seed
gives the same arrays."""
import math

import numpy as np
import pytest

import workloads as W

special = pytest.importorskip("scipy.special")


@pytest.mark.parametrize("theta", [0.1, 0.5, 1.0, 2.0])
def test_maxwell_juttner_mean_gamma_and_isotropy(theta):
    n = 400_000
    u = W.maxwell_juttner(np.random.default_rng(7), n, theta)
    gamma = np.sqrt(1.0 + np.sum(u * u, axis=0))
    mean = 3.0 * theta + special.kn(1, 1.0 / theta) / special.kn(2, 1.0 / theta)
    sigma = gamma.std() / math.sqrt(n)
    assert abs(gamma.mean() - mean) < 5.0 * sigma + 1e-4 * mean, (gamma.mean(), mean)
    var = u.var(axis=1)
    assert np.all(np.abs(u.mean(axis=1)) < 5.0 * np.sqrt(var / n))
    assert np.max(var) / np.min(var) - 1.0 < 0.02


def test_pair_plasma_layout():
    cfg = W.grid_config("wald64", n_r=16, n_theta=12, ppc=5)
    a = W.pair_plasma(cfg)
    b = W.pair_plasma(cfg)
    pos = a["pos"]
    counts = np.zeros((cfg["n_theta"], cfg["n_r"]), dtype=int)
    np.add.at(counts, (pos["i2"], pos["i1"]), 1)
    assert np.all(counts == cfg["ppc"])
    assert np.all((pos["dx1"] >= 0.0) & (pos["dx1"] < 1.0))
    assert np.all((pos["dx2"] >= 0.0) & (pos["dx2"] < 1.0))
    assert np.array_equal(a["w0"], np.full(pos["i1"].size, 1.0 / cfg["ppc"]))
    assert not np.array_equal(a["uhat"][0], a["uhat"][1])  # independent momenta
    assert a["qm"][0] == -a["qm"][1] and a["qc"][0] == -a["qc"][1]
    for k in pos:
        assert np.array_equal(pos[k], b["pos"][k])
    for s in range(2):
        assert np.array_equal(a["uhat"][s], b["uhat"][s])


def test_injection_pool_draws():
    """[n, 8]: uniform cell offsets, then the e- and e+ tetrad-frame momenta, Maxwell-Juttner
    at the injection temperature (theta = 0.5 on the monopole workload, Sec. 4.5)."""
    cfg = W.grid_config("bz1024")
    n = 200_000
    pool = W.injection_pool(cfg, n, seed=3)
    assert pool.shape == (n, 8)
    assert np.array_equal(pool, W.injection_pool(cfg, n, seed=3))
    for c in (0, 1):
        assert np.all((pool[:, c] >= 0.0) & (pool[:, c] < 1.0))
        assert abs(pool[:, c].mean() - 0.5) < 5.0 * math.sqrt(1.0 / 12.0 / n)
    theta = cfg["theta_inj"]
    mean = 3.0 * theta + special.kn(1, 1.0 / theta) / special.kn(2, 1.0 / theta)
    for lo in (2, 5):
        u = pool[:, lo:lo + 3]
        gamma = np.sqrt(1.0 + np.sum(u * u, axis=1))
        assert abs(gamma.mean() - mean) < 5.0 * gamma.std() / math.sqrt(n) + 1e-4 * mean
