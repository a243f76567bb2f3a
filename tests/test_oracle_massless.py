"""Pins of the oracle's massless particles (Sec. 2.3: gamma = sqrt(h^ij u_i u_j); Sec. 3.1:
no EM push for them). Massless particles are taken to be neutral (photons): they deposit
no current and carry no charge.

Checked against what geometry fixes, not against the oracle's own formulas:
* homogeneity: a null geodesic does not depend on the photon's energy, so momenta scaled by
  a power of two give the same positions and phases to the last bit and the momenta scaled
  exactly (a massive particle's orbit depends on the scale);
* a flat-space radial photon moves at dr/dt = 1, reached at second order in dt;
* the equatorial circular photon orbit of Kerr (Bardeen, Press & Teukolsky 1972) is a fixed
  point of the implicit midpoint scheme, and its angular frequency is 1 / (r^{3/2} + a);
* E = -u_0 and L = u_3 (Sec. 2.3) on a scattering orbit: L exactly, E at second order;
* fields of any strength leave a massless particle's orbit unchanged; deposit and charge
  skip it.
"""
import math

import numpy as np
import pytest

from oracle import oracle as O
from test_oracle_pusher import bl_inverse_metric, code_state, grid


def photon_sim(cfg, dt, x1, x2, u, massless=True, n_iter=10, qm=0.0, qc=0.0):
    c = dict(cfg, dt=dt, n_iter=n_iter, small_angle=1e-5)
    sim = O.OracleSim(c)
    u = np.atleast_2d(np.asarray(u, dtype=np.float64))
    n = u.shape[0]
    x1 = np.broadcast_to(np.asarray(x1, dtype=np.float64), (n,))
    x2 = np.broadcast_to(np.asarray(x2, dtype=np.float64), (n,))
    i1, i2 = np.floor(x1).astype(np.int32), np.floor(x2).astype(np.int32)
    arr = {k: np.zeros(n, dtype=t) for k, t in O.PARTICLE_FIELDS.items()}
    arr.update(i1=i1, i2=i2, dx1=x1 - i1, dx2=x2 - i2, u1=u[:, 0], u2=u[:, 1], u3=u[:, 2],
               tag=np.ones(n, np.uint8), w=np.ones(n))
    for k in ("i1", "i2", "dx1", "dx2"):
        arr[k + "p"] = arr[k]
    sim.add_raw_species(arr, qm, qc, massless=massless)
    return sim


def pos(sim, prev=False):
    s = sim.species[0].view()
    p = "p" if prev else ""
    return s["i1" + p] + s["dx1" + p], s["i2" + p] + s["dx2" + p]


def mom(sim):
    s = sim.species[0].view()
    return np.stack([s["u1"], s["u2"], s["u3"]], axis=1)


def test_photon_orbit_is_independent_of_its_energy():
    cfg = grid(0.9, 30.0, 128)
    rng = np.random.default_rng(7)
    n = 64
    x1 = rng.uniform(20.0, 110.0, n)
    x2 = rng.uniform(5.0, 123.0, n)
    u = rng.normal(size=(n, 3)) * np.array([8.0, 10.0, 3.0])
    a = photon_sim(cfg, 0.05, x1, x2, u)
    b = photon_sim(cfg, 0.05, x1, x2, u * 1024.0)
    for _ in range(40):
        a.push(0, field_mode=1, fkind=0)
        b.push(0, field_mode=1, fkind=0)
    sa, sb = a.species[0].view(), b.species[0].view()
    alive = sa["tag"] == 1
    assert alive.sum() > n // 2
    for k in ("i1", "i2", "dx1", "dx2", "phi", "tag"):
        assert np.array_equal(sa[k], sb[k]), k
    for k in ("u1", "u2", "u3"):
        assert np.array_equal(sa[k][alive] * 1024.0, sb[k][alive]), k
    # a massive particle's orbit does depend on the scale of its momentum
    c = photon_sim(cfg, 0.05, x1, x2, u, massless=False)
    d = photon_sim(cfg, 0.05, x1, x2, u * 1024.0, massless=False)
    for _ in range(40):
        c.push(0, field_mode=1, fkind=0)
        d.push(0, field_mode=1, fkind=0)
    assert not np.array_equal(c.species[0].view()["dx1"], d.species[0].view()["dx1"])


def test_flat_radial_photon_moves_at_light_speed():
    cfg = grid(0.0, 100.0, 256, metric="ks0", r_min=1.0)
    dxi = math.log(cfg["r_max"] / cfg["r_min"]) / cfg["n_r"]
    r0, T = 5.0, 20.0
    errs = []
    for dt in (0.1, 0.05, 0.025):
        x1, x2, u = code_state(cfg, r0, math.pi / 2, 1.0, 0.0, 0.0)
        sim = photon_sim(cfg, dt, x1, x2, u)
        for _ in range(int(round(T / dt))):
            sim.push(0, field_mode=1, fkind=0)
        r = cfg["r_min"] * math.exp(pos(sim)[0][0] * dxi)
        errs.append(abs(r - (r0 + T)))
        # the photon stays in the equatorial plane and keeps u_2 = u_3 = 0
        assert pos(sim)[1][0] == x2 and mom(sim)[0, 1] == 0.0 and mom(sim)[0, 2] == 0.0
    assert errs[-1] < 1e-4
    for e0, e1 in zip(errs, errs[1:]):
        assert 3.5 < e0 / e1 < 4.5, errs


def kerr_photon_ring(a, prograde):
    """Equatorial circular photon orbit: radius 2 (1 + cos(2/3 arccos(-+a))) and impact
    parameter b = L / E (Bardeen, Press & Teukolsky 1972)."""
    sg = 1.0 if prograde else -1.0
    r = 2.0 * (1.0 + math.cos(2.0 / 3.0 * math.acos(-sg * a)))
    b = -(r ** 3 - 3 * r * r + a * a * r + a * a) / (a * (r - 1.0)) if a else sg * 3 * math.sqrt(3)
    return r, b


def null_state(a, r, th, u_phi):
    """Covariant KS momentum of a photon with u_r,BL = u_theta,BL = 0 and u_phi given: u_t from
    g^{mu nu} u_mu u_nu = 0 in BL, then Eq. (BL-KS)."""
    gb, gk, Del = bl_inverse_metric(a, r, th)
    roots = np.roots([gb[0, 0], 2 * gb[0, 3] * u_phi, gb[3, 3] * u_phi ** 2])
    u_t = float(np.min(roots.real))
    u_r = -(2 * r * u_t + a * u_phi) / Del
    return u_t, u_r


@pytest.mark.parametrize("a,pro", [(0.0, True), (0.9, True), (0.9, False), (0.5, True)])
def test_kerr_circular_photon_orbit_is_a_fixed_point(a, pro):
    r, b = kerr_photon_ring(a, pro)
    # the orbit's own conditions: the radial potential of a Q = 0 photon with E = 1,
    # R(r) = (r^2 + a^2 - a b)^2 - Delta (b - a)^2, and its derivative vanish there
    R = lambda x: (x * x + a * a - a * b) ** 2 - (x * x - 2 * x + a * a) * (b - a) ** 2
    h = 1e-5
    assert abs(R(r)) < 1e-10 * r ** 4
    assert abs((R(r + h) - R(r - h)) / (2 * h)) < 1e-7 * r ** 3
    u_t, u_r = null_state(a, r, math.pi / 2, b)
    assert u_t == pytest.approx(-1.0, rel=1e-12)
    cfg = grid(a, 30.0, 256)
    x1, x2, u = code_state(cfg, r, math.pi / 2, u_r, 0.0, b)
    sim = photon_sim(cfg, 0.02, x1, x2, u)
    n = 250  # t = 5: perturbations grow by e^{t / (3 sqrt 3)} or less
    for _ in range(n):
        sim.push(0, field_mode=1, fkind=0)
    x = pos(sim)
    assert abs(x[0][0] - x1) < 1e-10 * x1 and x[1][0] == x2
    assert np.allclose(mom(sim)[0], u, rtol=1e-10, atol=1e-12)
    Om = (1.0 if pro else -1.0) / (r ** 1.5 + (a if pro else -a))
    assert sim.species[0].view()["phi"][0] == pytest.approx(n * 0.02 * Om, rel=1e-9)
    # with the massive gamma the same momentum is not a circular orbit
    m = photon_sim(cfg, 0.02, x1, x2, u, massless=False)
    for _ in range(n):
        m.push(0, field_mode=1, fkind=0)
    assert abs(pos(m)[0][0] - x1) > 1e-4


def invariants(cfg, x1, x2, u):
    return -O.u_lower0(cfg, x1, x2, u, massless=True), u[2]


def test_photon_scattering_invariants_converge():
    """A photon from r = 20 with impact parameter 1.3 times the prograde photon ring's,
    a = 0.9, slightly off the equator: passes periapsis and leaves. L = u_3 exactly, E at
    second order in dt."""
    a = 0.9
    cfg = grid(a, 60.0, 256)
    r_ring, b_ring = kerr_photon_ring(a, True)
    th0 = math.pi / 2 - 0.1
    errs = []
    for dt in (0.04, 0.02):
        _, gk, _ = bl_inverse_metric(a, 20.0, th0)
        b = 1.3 * b_ring
        # E = 1 (u_t = -1), u_th = 0: the null condition in KS is a quadratic in u_r; take the
        # ingoing root, u^r = g^{rt} u_t + g^{rr} u_r + g^{r phi} u_phi < 0
        roots = np.roots([gk[1, 1], 2 * (-gk[0, 1] + gk[1, 3] * b),
                          gk[0, 0] + gk[3, 3] * b * b - 2 * gk[0, 3] * b]).real
        u_r = [x for x in roots if -gk[1, 0] + gk[1, 1] * x + gk[1, 3] * b < 0][0]
        x1, x2, u = code_state(cfg, 20.0, th0, u_r, 0.0, b)
        E0, L0 = invariants(cfg, x1, x2, u)
        assert E0 == pytest.approx(1.0, rel=1e-12)
        sim = photon_sim(cfg, dt, x1, x2, u)
        e, rmin = [], 1e9
        dxi = math.log(cfg["r_max"] / cfg["r_min"]) / cfg["n_r"]
        for _ in range(int(round(40.0 / dt))):
            sim.push(0, field_mode=1, fkind=0)
            xa, xb = pos(sim), pos(sim, prev=True)
            xm = (0.5 * (xa[0][0] + xb[0][0]), 0.5 * (xa[1][0] + xb[1][0]))
            E, L = invariants(cfg, *xm, mom(sim)[0])
            if not e:
                # the start momentum stands for t = -dt/2 (leapfrog): the discrete orbit's
                # energy is fixed after the first step, within O(dt) of E0
                assert abs(E / E0 - 1) < 2 * dt
                E0 = E
            e.append((abs(E / E0 - 1), abs(L / L0 - 1)))
            rmin = min(rmin, cfg["r_min"] * math.exp(xa[0][0] * dxi))
        assert sim.species[0].view()["tag"][0] == 1
        assert rmin < 6.0  # it came close and went back out
        errs.append(np.max(np.array(e), axis=0))
    assert errs[0][1] == 0.0 and errs[1][1] == 0.0
    assert errs[1][0] < 1e-3
    assert 3.0 < errs[0][0] / errs[1][0] < 5.5, errs


def test_fields_leave_photons_alone_and_photons_deposit_nothing():
    cfg = grid(0.9, 30.0, 64)
    rng = np.random.default_rng(3)
    x1, x2 = rng.uniform(8.0, 56.0, 32), rng.uniform(4.0, 60.0, 32)
    u = rng.normal(size=(32, 3))
    a = photon_sim(cfg, 0.05, x1, x2, u, qm=-50.0, qc=-1.0)
    b = photon_sim(cfg, 0.05, x1, x2, u, qm=-50.0, qc=-1.0)
    b.init_fields(O.FIELD_WALD, 3.0)
    b.predict()
    for _ in range(5):
        a.push(0)
        b.push(0, field_mode=0)  # interpolated Wald field
    for k in ("i1", "i2", "dx1", "dx2", "u1", "u2", "u3", "phi"):
        assert np.array_equal(a.species[0].view()[k], b.species[0].view()[k]), k
    b.deposit()
    assert not b.F[12:15].any()
    assert not b.charge(prev=False).any() and not b.charge(prev=True).any()
    # the same particles, massive: they do deposit
    c = photon_sim(cfg, 0.05, x1, x2, u, massless=False, qm=-50.0, qc=-1.0)
    c.init_fields(O.FIELD_WALD, 3.0)
    c.predict()
    c.push(0)
    c.deposit()
    assert c.F[12:15].any()
