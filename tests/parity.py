"""Shared set-up and comparisons for the GPU-vs-oracle parity tests.

The oracle builds and owns every input state; the CUDA library receives copies of
it (the reverse never happens: no value computed on the GPU feeds the oracle).

Tolerances (FP64): particle state and fields agree to 1e-12 relative per step. The two
sides differ only in rounding (fused multiply-adds on the GPU, a different but equivalent
formulation of the metric, CUDA's vs glibc's transcendentals), i.e. ~1e-16 per operation
along chains of a few hundred operations with condition numbers of at most ~1e2 near the
horizon, which stays below 1e-12. Currents are summed by atomics in arbitrary order, so
each cell is compared against 1e-12 times the sum of the absolute values of its
contributions, plus 1e-15 of the largest such sum on the plane: a zigzag segment is a
difference of two positions, and a segment much shorter than a cell keeps their absolute
rounding, not a relative one.
"""
from __future__ import annotations

import numpy as np

import workloads as W
from oracle import oracle as O

RTOL = 1e-12
G = O.G
STATE_PLANES = list(range(27))  # em, em0, cur, cur0, B^n, initial field


def oracle_state(cfg: dict, cells=None, kind=O.FIELD_WALD, B0=1.0, species=2):
    osim = O.OracleSim(cfg)
    osim.init_fields(kind, B0)
    if species:
        pl = W.pair_plasma(cfg, cells=cells)
        for s in range(species):
            osim.add_species(pl["pos"], pl["uhat"][s], pl["w0"], pl["qm"][s], pl["qc"][s],
                             pl["density_power"])
    return osim


def gpu_from_oracle(osim, extra_capacity=0, **over):
    """A GPU context holding a copy of the oracle's full state."""
    from paper_2511_17701_gb300 import FIELD_USER, Sim
    cfg = dict(osim.cfg, dt=osim.dt, **over)
    caps = [max(s.n + extra_capacity, 1) for s in osim.species] or [1]
    g = Sim(cfg, caps)
    g.init_metric()
    g.init_fields(FIELD_USER)
    g.set_planes(osim.F)
    for k, s in enumerate(osim.species):
        g.set_particles(k, s.view(), s.qm, s.qc)
    return g


def max_rel_plane(a, b):
    scale = max(np.abs(b).max(), 1e-300)
    return float(np.abs(a - b).max() / scale)


def assert_planes(Fg, Fo, planes=STATE_PLANES, rtol=RTOL, what=""):
    bad = []
    for k in planes:
        e = max_rel_plane(Fg[k], Fo[k])
        if e > rtol:
            bad.append((k, e))
    assert not bad, "%s planes above %g: %s" % (what, rtol, bad)


def assert_currents(Fg, Fo, rtol=RTOL):
    for c in range(3):
        d = np.abs(Fg[O.J1 + c] - Fo[O.J1 + c])
        lim = rtol * (Fo[O.JA1 + c] + 1e-3 * Fo[O.JA1 + c].max()) + 1e-300
        assert np.all(d <= lim), ("J%d" % (c + 1), float((d / (Fo[O.JA1 + c] + 1e-300)).max()))


def assert_particles(pg: dict, po: dict, rtol=RTOL, exact_order=True, prev=True):
    """prev: also compare the previous positions (False after a fused step that skipped
    storing them, grpic_set_keep_prev(0))."""
    n = len(po["i1"])
    assert len(pg["i1"]) == n
    assert np.array_equal(pg["tag"], po["tag"])
    pairs = (("i1", "dx1"), ("i2", "dx2")) + ((("i1p", "dx1p"), ("i2p", "dx2p")) if prev else ())
    for a, b in pairs:
        xg = pg[a].astype(np.float64) + pg[b]
        xo = po[a].astype(np.float64) + po[b]
        err = np.abs(xg - xo) / np.maximum(1.0, np.abs(xo))
        assert err.max(initial=0.0) <= rtol, (b, float(err.max()), int(err.argmax()))
    for c in ("u1", "u2", "u3"):
        scale = np.median(np.abs(po[c])) if n else 1.0
        err = np.abs(pg[c] - po[c]) / (np.abs(po[c]) + scale + 1e-300)
        assert err.max(initial=0.0) <= rtol, (c, float(err.max()), int(err.argmax()))
    err = np.abs(pg["phi"] - po["phi"]) / np.maximum(1.0, np.abs(po["phi"]))
    assert err.max(initial=0.0) <= rtol, ("phi", float(err.max()))
    assert np.array_equal(pg["w"], po["w"]) or np.allclose(pg["w"], po["w"], rtol=rtol, atol=0)


def round_state_fp32(osim):
    """Round the oracle's floating state (fields and particles) to FP32 values in place, so
    that both sides of a mixed-precision comparison start from the same numbers."""
    osim.F[:] = osim.F.astype(np.float32).astype(np.float64)
    for sp in osim.species:
        for k in ("dx1", "dx2", "u1", "u2", "u3", "phi", "w", "dx1p", "dx2p"):
            sp.a[k][:] = sp.a[k].astype(np.float32).astype(np.float64)


def particle_errors(pg, po):
    """Max relative errors per quantity (positions relative to max(1, |x|), momentum
    components relative to |u_c| + median |u_c|)."""
    out = {}
    assert len(pg["i1"]) == len(po["i1"])
    assert np.array_equal(pg["tag"], po["tag"])
    for a, b in (("i1", "dx1"), ("i2", "dx2")):
        xg = pg[a].astype(np.float64) + pg[b].astype(np.float64)
        xo = po[a].astype(np.float64) + po[b]
        out[b] = float(np.max(np.abs(xg - xo) / np.maximum(1.0, np.abs(xo)), initial=0.0))
    for c in ("u1", "u2", "u3"):
        sc = np.median(np.abs(po[c])) if len(po[c]) else 1.0
        out[c] = float(np.max(np.abs(pg[c] - po[c]) / (np.abs(po[c]) + sc + 1e-300), initial=0.0))
    out["phi"] = float(np.max(np.abs(pg["phi"] - po["phi"]) / np.maximum(1.0, np.abs(po["phi"])),
                              initial=0.0))
    return out


def plane_errors(Fg, Fo, planes):
    return {k: float(np.abs(Fg[k] - Fo[k]).max() / max(np.abs(Fo[k]).max(), 1e-300))
            for k in planes}
