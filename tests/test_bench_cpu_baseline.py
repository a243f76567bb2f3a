"""bench.py's CPU baseline (the oracle timed on the host cores), on CPU: the projection of a
bounded sample to the whole workload, and the unprojected run over all particles.

The baseline times the field phases on the whole grid and the particle phases on the
particles of a seeded fraction of the cells; only the particle phases are scaled up to the
workload's particle count. With --cpu-frac 1 every particle is pushed and nothing is scaled.
"""
import argparse
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def test_projection_scales_the_particle_phases_only():
    import bench
    # 1e6 particles; fields 2 s per step, particles 3 s per 1e5 sampled particles
    assert bench.projected_rate(1_000_000, 2.0, 3.0, 100_000) == pytest.approx(1e6 / 32.0)
    # no sample: the measured step itself
    assert bench.projected_rate(1_000_000, 2.0, 3.0, 1_000_000) == pytest.approx(1e6 / 5.0)


def test_full_particle_set_is_not_projected():
    import bench
    import workloads as W
    cfg = W.grid_config("wald64")
    n_total = 2 * cfg["n_r"] * cfg["n_theta"] * cfg["ppc"]
    a = argparse.Namespace(workload="wald64", ppc=0, cpu_frac=1.0, cpu_steps=2,
                           cpu_steps_1core=2)
    r = bench.cpu_baseline(a)
    assert r["sample_particles"] == n_total
    assert "no projection" in r["sample"] and "2 more step(s) on 1 core" in r["sample"]
    # the rates are the workload's particle-steps over the measured step times
    assert r["value"] == pytest.approx(
        n_total / (r["field_s_per_step"] + r["particle_s_per_sample_step"]))
    assert r["one_core"]["value"] == pytest.approx(
        n_total / (r["field_s_per_step"] + r["particle_s_per_sample_step_1core"]))
    assert r["cores"] >= 1 and r["kind"] == "oracle"


def test_sample_is_projected_and_says_so():
    import bench
    import workloads as W
    cfg = W.grid_config("wald64")
    n_total = 2 * cfg["n_r"] * cfg["n_theta"] * cfg["ppc"]
    a = argparse.Namespace(workload="wald64", ppc=0, cpu_frac=0.25, cpu_steps=2,
                           cpu_steps_1core=1)
    r = bench.cpu_baseline(a)
    n_s = r["sample_particles"]
    # a quarter of the cells (rounded down), both species, ppc particles per cell
    assert n_s == 2 * int(cfg["n_r"] * cfg["n_theta"] * 0.25) * cfg["ppc"]
    assert "scaled to the %d particles" % n_total in r["sample"]
    assert r["value"] == pytest.approx(
        bench.projected_rate(n_total, r["field_s_per_step"], r["particle_s_per_sample_step"], n_s))
