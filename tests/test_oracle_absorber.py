"""Pin of the oracle's absorbing layer (MATCH, Sec. 3.3.3: F relaxes towards the initial
field F_init beyond r_absorb) by what the layer is for: an outgoing electromagnetic pulse
leaves the domain through it instead of reflecting off the outer boundary.

Flat spacetime (M = 0) on the log-r grid r in [3, 30]. The initial field is an outgoing
magnetic-dipole pulse: A_phi-hat = sin(theta) G(r) / r with G(r) = exp(-(r - 9)^2), i.e. the
covariant A_3 = sin^2(theta) G(r) at the nodes, B the discrete curl of A on the staggered
grid (so div B = 0 to rounding) and E_phi = -d_t A_phi with the dependence G(r - t),
D^3 = G'(r) / r^2; the initial field of the absorber is zero. The field solver runs with and
without the layer (r_absorb = 22, coefficient 1):
  * until the pulse reaches the layer both runs agree to the bit inside r < 18 (the layer
    acts only where the field differs from F_init, and only beyond r_absorb);
  * without the layer the energy is conserved and the pulse, reflected off the outer
    boundary, is back inside r in [5, 21] at t = 34; with it, the energy left anywhere at
    t = 24 and inside at t = 34 is a trace (the reflection off the layer's ramp);
  * the layer never adds energy.
The energy is 1/2 of the sum over the staggered points of sqrt(h) h_ii (F^i)^2 (the flat
metric is diagonal), with the flat-space metric of the grid computed here.
"""
import math

import numpy as np
import pytest

from oracle import oracle as O

G_ = O.G
CFG = dict(metric="ks0", a=0.0, n_r=120, n_theta=24, r_min=3.0, r_max=30.0, cfl=0.5)


def flat_metric(cfg, x1, x2):
    """sqrt(h), h_11, h_22, h_33 of flat space in the grid's code coordinates."""
    dxi = math.log(cfg["r_max"] / cfg["r_min"]) / cfg["n_r"]
    dth = math.pi / cfg["n_theta"]
    r = cfg["r_min"] * np.exp(x1 * dxi)
    th = x2 * dth
    f, s = dxi * r, np.sin(th)
    return f * dth * r * r * s, f * f, dth * dth * r * r, r * r * s * s, r


def pulse_state(cfg):
    """em planes of the outgoing pulse (B and D; the previous time level equal to them)."""
    NX, NY = cfg["n_r"] + 2 * G_ + 1, cfg["n_theta"] + 2 * G_ + 1
    i = np.arange(NX)[None, :] - G_
    j = np.arange(NY)[:, None] - G_
    dxi = math.log(cfg["r_max"] / cfg["r_min"]) / cfg["n_r"]
    dth = math.pi / cfg["n_theta"]

    def A3(x1, x2):
        r = cfg["r_min"] * np.exp(x1 * dxi)
        return np.sin(x2 * dth) ** 2 * np.exp(-(r - 9.0) ** 2)

    F = np.zeros((O.NPLANES, NY, NX))
    sq, *_ = flat_metric(cfg, i + 0.0, j + 0.5)
    F[O.B1] = (A3(i, j + 1.0) - A3(i, j + 0.0)) / np.where(sq != 0.0, sq, np.inf)
    sq, *_ = flat_metric(cfg, i + 0.5, j + 0.0)
    F[O.B2] = -(A3(i + 1.0, j + 0.0) - A3(i, j + 0.0)) / np.where(sq != 0.0, sq, np.inf)
    r = cfg["r_min"] * np.exp(i * dxi) + 0.0 * j
    F[O.D3] = -2.0 * (r - 9.0) * np.exp(-(r - 9.0) ** 2) / (r * r)
    # only stored points inside the domain carry the pulse; the axis rows of D^3 hold 0
    inside_j = (j >= 0) & (j <= cfg["n_theta"])
    for k in (O.B1, O.B2, O.D3):
        F[k] = np.where(inside_j & (i >= 0) & (i <= cfg["n_r"]), F[k], 0.0)
    F[O.D3][((j == 0) | (j == cfg["n_theta"])).ravel(), :] = 0.0
    for k in range(6):
        F[O.B01 + k] = F[O.B1 + k]
    return F


# points of each em component: (plane, x1 offset, x2 offset)
POINTS = [(O.B1, 0.0, 0.5), (O.B2, 0.5, 0.0), (O.B3, 0.5, 0.5),
          (O.D1, 0.5, 0.0), (O.D2, 0.0, 0.5), (O.D3, 0.0, 0.0)]


def energy(cfg, F, r_lo, r_hi):
    NX, NY = F.shape[2], F.shape[1]
    i = np.arange(NX)[None, :] - G_
    j = np.arange(NY)[:, None] - G_
    e = 0.0
    for k, o1, o2 in POINTS:
        sq, h11, h22, h33, r = flat_metric(cfg, i + o1, j + o2)
        hii = (h11, h22, h33)[k % 3]
        keep = (r >= r_lo) & (r <= r_hi) & (j + o2 >= 0) & (j + o2 <= cfg["n_theta"])
        e += 0.5 * np.sum(np.where(keep, sq * hii * F[k] ** 2, 0.0))
    return e


def run(cfg, t_marks):
    osim = O.OracleSim(cfg)
    osim.F[:] = pulse_state(osim.cfg)
    out, t, dt = [], 0.0, osim.dt
    for tm in t_marks:
        n = int(round((tm - t) / dt))
        osim.step(n)
        t += n * dt
        out.append(osim.F.copy())
    return osim, out


@pytest.fixture(scope="module")
def runs():
    t_marks = [4.0, 8.0, 16.0, 24.0, 34.0]
    absorb = dict(CFG, r_absorb=22.0, absorb_coef=1.0)
    plain = dict(CFG, r_absorb=1e300, absorb_coef=0.0)
    return t_marks, run(absorb, t_marks), run(plain, t_marks)


def test_the_initial_pulse_is_divergence_free():
    osim = O.OracleSim(CFG)
    F = pulse_state(osim.cfg)
    i = np.arange(F.shape[2])[None, :] - G_
    j = np.arange(F.shape[1])[:, None] - G_
    sq1, *_ = flat_metric(CFG, i + 0.0, j + 0.5)
    sq2, *_ = flat_metric(CFG, i + 0.5, j + 0.0)
    f1, f2 = sq1 * F[O.B1], sq2 * F[O.B2]
    # d1 (sqrt(h) B^1) + d2 (sqrt(h) B^2) at the centres of cells (i, j) of the domain
    nr, nt = CFG["n_r"], CFG["n_theta"]
    J, I = slice(G_, G_ + nt), slice(G_, G_ + nr)
    div = (f1[J, G_ + 1:G_ + nr + 1] - f1[J, I]) + (f2[G_ + 1:G_ + nt + 1, I] - f2[J, I])
    scale = np.abs(f1).max() + np.abs(f2).max()
    assert np.abs(div).max() <= 1e-14 * scale


def test_layer_acts_only_beyond_r_absorb(runs):
    """Until t = 8 the pulse (e^-1 half width 1 around r = 9 + t) has not reached r = 22: the
    layer has only damped the pulse's far tail (~e^-169) beyond r_absorb, and inside r < 18
    the fields of both runs are the same to the bit (the discrete solver carries a signal one
    cell per step, faster than light on the outer cells, but at t = 8 nothing of the layer's
    effect has reached r = 18)."""
    t_marks, (osim, with_layer), (_, without) = runs
    cfg = osim.cfg
    i = np.arange(with_layer[0].shape[2]) - G_
    r = cfg["r_min"] * np.exp(i * math.log(cfg["r_max"] / cfg["r_min"]) / cfg["n_r"])
    for k in (0, 1):
        assert np.array_equal(with_layer[k][:6][:, :, r < 18.0], without[k][:6][:, :, r < 18.0])


def test_outgoing_pulse_leaves_through_the_layer(runs):
    t_marks, (osim_a, with_layer), (osim_p, without) = runs
    e0 = energy(osim_a.cfg, pulse_state(osim_a.cfg), 5.0, 21.0)
    e_total0 = energy(osim_a.cfg, pulse_state(osim_a.cfg), 0.0, 1e9)
    e_with = [energy(osim_a.cfg, F, 5.0, 21.0) for F in with_layer]
    e_without = [energy(osim_p.cfg, F, 5.0, 21.0) for F in without]
    # without the layer the vacuum solver conserves the pulse's energy (the outer ghosts hold
    # the initial, zero, field: a conducting wall), and at t = 34 the reflection off the
    # outer boundary is back inside
    # (the sum over staggered points and time levels is conserved to ~1%)
    for F in without:
        assert abs(energy(osim_p.cfg, F, 0.0, 1e9) / e_total0 - 1.0) < 0.02
    assert e_without[-1] > 0.5 * e0, e_without
    # with it the pulse has left: by t = 24 almost nothing is left anywhere, and what comes
    # back inside by t = 34 is a trace
    assert energy(osim_a.cfg, with_layer[3], 0.0, 1e9) < 0.01 * e_total0
    assert e_with[-1] < 1e-3 * e0, (e_with, e0)
    # and the layer never adds energy
    for F in with_layer:
        assert energy(osim_a.cfg, F, 0.0, 1e9) <= 1.02 * e_total0
