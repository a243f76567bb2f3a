"""Pins of the oracle's particle pusher (Sec. 3.1 of arXiv:2511.17701).

Checked against what the paper and textbook mechanics fix:
* Table 1 initial conditions (energy, angular momentum, KS radial velocity) from
  the 4-metric of Appendix A, the BL -> KS map (Eq. BL-KS) and Eq. (Wald);
* circular equatorial Kerr geodesics (Bardeen, Press & Teukolsky 1972) are exact
  fixed points of the implicit midpoint scheme, so their radius must stay fixed;
* conservation of E and L (Sec. 2.3) with second-order convergence in dt;
* the SR-EM gyration radius rho0 u_perp of Sec. 4.1.2;
* closed forms of the Boris step; axis reflection and horizon removal rules.
"""
import math
import os

import numpy as np
import pytest

from oracle import oracle as O

GOLD = os.path.join(os.path.dirname(__file__), "golden", "table1.txt")


def table1():
    rows = {}
    for line in open(GOLD):
        if line.startswith("#") or not line.strip():
            continue
        t = line.split()
        th = math.pi / 2 if t[9] == "pi/2" else math.pi / 2 - 0.2
        rows[t[0]] = dict(field=t[1], a=float(t[2]), r_max=float(t[3]), N=int(t[4]),
                          dt=float(t[5]), E=float(t[6]), L=float(t[7]), r=float(t[8]),
                          th=th, u1=float(t[10]), u3=float(t[11]))
    return rows


def bl_inverse_metric(a, r, th):
    """g^{mu nu} in Boyer-Lindquist coordinates from the KS one of Appendix A and the
    Jacobian J^{mu~}_{nu} of Appendix A.4: g_BL^{-1} = J g_KS^{-1} J^T."""
    s, c = math.sin(th), math.cos(th)
    Sig = r * r + a * a * c * c
    Del = r * r - 2 * r + a * a
    z = 2 * r / Sig
    gi = np.array([[-(1 + z), z, 0, 0], [z, Del / Sig, 0, a / Sig], [0, 0, 1 / Sig, 0],
                   [0, a / Sig, 0, 1 / (Sig * s * s)]])
    J = np.eye(4)
    J[0, 1] = -2 * r / Del
    J[3, 1] = -a / Del
    return J @ gi @ J.T, gi, Del


def bl_state(a, r, th, u_phi):
    """Covariant KS four-velocity of a particle with u_r,BL = u_theta,BL = 0 (Sec. 4.1):
    u_t from u.u = -1 in BL, then Eq. (BL-KS)."""
    gb, gk, Del = bl_inverse_metric(a, r, th)
    A, B, Cc = gb[0, 0], 2 * gb[0, 3] * u_phi, gb[3, 3] * u_phi ** 2 + 1.0
    roots = np.roots([A, B, Cc])
    u_t = float(np.min(roots.real))  # future directed: u_t < 0
    u_r = -(2 * r * u_t + a * u_phi) / Del
    return u_t, u_r, gk


def grid(a, r_max, N, metric="ks", r_min=None):
    if r_min is None:
        r_min = 0.95 * (1 + math.sqrt(1 - a * a)) if metric == "ks" else 1.0
    return dict(metric=metric, a=a, n_r=N, n_theta=N, r_min=r_min, r_max=r_max)


def code_state(cfg, r, th, u_r, u_th, u_phi):
    dxi = math.log(cfg["r_max"] / cfg["r_min"]) / cfg["n_r"]
    x1 = math.log(r / cfg["r_min"]) / dxi
    x2 = th / (math.pi / cfg["n_theta"])
    return x1, x2, np.array([dxi * r * u_r, (math.pi / cfg["n_theta"]) * u_th, u_phi])


def test_table1_geodesic_row():
    row = table1()["GR"]
    u_t, u_r, gk = bl_state(row["a"], row["r"], row["th"], row["L"])
    assert math.isclose(-u_t, row["E"], rel_tol=2e-5)
    assert abs(u_r - row["u1"]) < 1e-4
    # the paper's KS quadratic (Sec. 4.1) gives the same energy
    A, B = gk[0, 0], -2 * gk[0, 1] * u_r
    Cc = gk[1, 1] * u_r ** 2 + gk[3, 3] * row["u3"] ** 2 + 2 * gk[1, 3] * u_r * row["u3"] + 1
    E = (-B - math.sqrt(B * B - 4 * A * Cc)) / (2 * A)
    assert math.isclose(E, -u_t, rel_tol=1e-12)
    # the oracle's 3+1 u_0 = -alpha gamma + beta^1 u_1 at the same state
    cfg = grid(row["a"], row["r_max"], row["N"])
    x1, x2, u = code_state(cfg, row["r"], row["th"], u_r, 0.0, row["u3"])
    assert math.isclose(O.u_lower0(cfg, x1, x2, u), u_t, rel_tol=1e-12)


def test_table1_sr_em_row():
    row = table1()["SR-EM"]
    cfg = grid(0.0, row["r_max"], row["N"], metric="ks0")
    x1, x2, u = code_state(cfg, row["r"], row["th"], 0.0, 0.0, row["u3"])
    E, _ = O.invariants(cfg, O.FIELD_WALD, 1.0, 0.5, x1, x2, u)
    assert math.isclose(E, row["E"], rel_tol=1e-5)


@pytest.mark.parametrize("name,qm", [("GR-EM-2D", 0.2), ("GR-EM-3D", 2.0)])
def test_table1_charged_rows(name, qm):
    """E = -u_0 - qA_0 and L = u_3 + qA_3 (Sec. 2.3) with the Wald potential (Eq. Wald)."""
    row = table1()[name]
    u_t, u_r, _ = bl_state(row["a"], row["r"], row["th"], row["u3"])
    cfg = grid(row["a"], row["r_max"], row["N"])
    x1, x2, u = code_state(cfg, row["r"], row["th"], u_r, 0.0, row["u3"])
    assert math.isclose(O.u_lower0(cfg, x1, x2, u), u_t, rel_tol=1e-12)
    E, L = O.invariants(cfg, O.FIELD_WALD, 1.0, qm, x1, x2, u)
    tolE = 5e-4 if name == "GR-EM-2D" else 1e-4
    assert abs(E / row["E"] - 1) < tolE
    assert abs(L / row["L"] - 1) < 3e-6
    assert abs(u_r - row["u1"]) < (5e-4 if name == "GR-EM-2D" else 5e-5)


def new_sim(cfg, dt, x1, x2, u, qm=0.0, n_iter=10):
    c = dict(cfg, dt=dt, n_iter=n_iter, small_angle=1e-5)
    sim = O.OracleSim(c)
    i1, i2 = int(math.floor(x1)), int(math.floor(x2))
    arr = {k: np.zeros(1, dtype=t) for k, t in O.PARTICLE_FIELDS.items()}
    arr.update(i1=[i1], i2=[i2], dx1=[x1 - i1], dx2=[x2 - i2], u1=[u[0]], u2=[u[1]],
               u3=[u[2]], tag=[1], w=[1.0])
    for k in ("i1", "i2", "dx1", "dx2"):
        arr[k + "p"] = arr[k]
    sim.add_raw_species(arr, qm, 0.0)
    return sim


def state(sim):
    s = sim.species[0].view()
    x = np.array([s["i1"][0] + s["dx1"][0], s["i2"][0] + s["dx2"][0]])
    xp = np.array([s["i1p"][0] + s["dx1p"][0], s["i2p"][0] + s["dx2p"][0]])
    u = np.array([s["u1"][0], s["u2"][0], s["u3"][0]])
    return x, xp, u, s["phi"][0]


def bpt_circular(a, r, prograde=True):
    sg = 1.0 if prograde else -1.0
    den = r ** 0.75 * math.sqrt(r ** 1.5 - 3 * r ** 0.5 + sg * 2 * a)
    E = (r ** 1.5 - 2 * r ** 0.5 + sg * a) / den
    L = sg * (r * r - sg * 2 * a * r ** 0.5 + a * a) / den
    return E, L


@pytest.mark.parametrize("a,r,pro", [(0.9, 8.0, True), (0.0, 10.0, True), (0.5, 6.5, True),
                                     (0.9, 12.0, False)])
def test_circular_geodesic_is_a_fixed_point(a, r, pro):
    E, L = bpt_circular(a, r, pro)
    u_t, u_r, _ = bl_state(a, r, math.pi / 2, L)
    assert math.isclose(-u_t, E, rel_tol=1e-12)  # BPT energy satisfies the normalisation
    cfg = grid(a, 30.0, 256)
    x1, x2, u = code_state(cfg, r, math.pi / 2, u_r, 0.0, L)
    sim = new_sim(cfg, 0.05, x1, x2, u)
    for _ in range(600):
        sim.push(0, field_mode=1, fkind=0)
    x, xp, u1, phi = state(sim)
    assert abs(x[0] - x1) < 1e-9 * x1 and abs(x[1] - x2) < 1e-9
    assert np.allclose(u1, u, rtol=1e-10, atol=1e-12)
    assert u1[2] == pytest.approx(L, rel=1e-14)  # u_3 untouched without a field
    # azimuthal advance: dphi/dt = Omega = +-1/(r^{3/2} +- a) in BL; KS phi differs from BL
    # phi only by a function of r, so the rates agree on a circular orbit
    Om = (1.0 if pro else -1.0) / (r ** 1.5 + (a if pro else -a))
    assert phi == pytest.approx(600 * 0.05 * Om, rel=1e-9)


def energy_errors(sim, n, kind, B0, qm, E0=None):
    errs = []
    for _ in range(n):
        sim.push(0, field_mode=1, fkind=kind, B0=B0)
        x, xp, u, _ = state(sim)
        xm = 0.5 * (x + xp)
        E, L = O.invariants(sim.cfg, kind, B0, qm, xm[0], xm[1], u)
        errs.append((E, L))
    e = np.array(errs)
    if E0 is None:
        E0 = e[0]
    return np.max(np.abs(e / E0 - 1), axis=0)


def test_three_leaf_orbit_energy_converges_second_order():
    row = table1()["GR"]
    u_t, u_r, _ = bl_state(row["a"], row["r"], row["th"], row["L"])
    cfg = grid(row["a"], row["r_max"], row["N"])
    x1, x2, u = code_state(cfg, row["r"], row["th"], u_r, 0.0, row["u3"])
    errs = []
    for dt in (0.04, 0.02):
        sim = new_sim(cfg, dt, x1, x2, u)
        errs.append(energy_errors(sim, int(round(300 / dt)), 0, 0.0, 0.0,
                                  E0=np.array([-u_t, row["L"]])))
    ratio = errs[0][0] / errs[1][0]
    assert 3.0 < ratio < 5.5, errs
    assert errs[1][0] < 1e-3
    assert errs[1][1] < 1e-13  # L = u_3 exactly conserved by the geodesic substep


def test_sr_em_gyration_radius():
    """Flat spacetime, uniform vertical field, u_phi^ = 1, rho0 = 2: a circle of radius
    rho0 u_perp = 2 in the equatorial plane (Sec. 4.1.2)."""
    row = table1()["SR-EM"]
    cfg = grid(0.0, row["r_max"], row["N"], metric="ks0")
    x1, x2, u = code_state(cfg, row["r"], row["th"], 0.0, 0.0, row["u3"])
    sim = new_sim(cfg, row["dt"], x1, x2, u, qm=0.5)
    dxi = math.log(cfg["r_max"] / cfg["r_min"]) / cfg["n_r"]
    T = 2 * math.pi * math.sqrt(2.0) / 0.5  # gyration period gamma / ((q/m) B)
    n = int(round(2 * T / row["dt"]))
    xy, gam = [], []
    for _ in range(n):
        sim.push(0, field_mode=1, fkind=O.FIELD_VERTICAL, B0=1.0)
        x, xp, uu, phi = state(sim)
        r = cfg["r_min"] * math.exp(x[0] * dxi)
        xy.append((r * math.cos(phi), r * math.sin(phi)))
        E, _ = O.invariants(sim.cfg, O.FIELD_VERTICAL, 1.0, 0.5, *(0.5 * (x + xp)), uu)
        gam.append(E)
    xy = np.array(xy)
    # least-squares circle
    A = np.c_[2 * xy[:, 0], 2 * xy[:, 1], np.ones(len(xy))]
    b = (xy ** 2).sum(1)
    cx, cy, c0 = np.linalg.lstsq(A, b, rcond=None)[0]
    R = math.sqrt(c0 + cx * cx + cy * cy)
    assert abs(R - 2.0) < 2e-3
    assert np.max(np.abs(np.hypot(xy[:, 0] - cx, xy[:, 1] - cy) - R)) < 2e-3
    # q > 0: the force v x B points outward, centre at r = 12; the start velocity belongs
    # to t = -dt/2 (leapfrog), which turns the centre by at most omega dt / 2
    omega = 0.5 / math.sqrt(2.0)
    assert abs(cx - 12.0) < 2e-3 and abs(cy) < 2.0 * omega * row["dt"]
    assert np.max(np.abs(np.array(gam) / math.sqrt(2.0) - 1)) < 1e-5


@pytest.mark.parametrize("name,qm,T", [("GR-EM-2D", 0.2, 60.0), ("GR-EM-3D", 2.0, 8.0)])
def test_charged_orbit_invariants_converge(name, qm, T):
    row = table1()[name]
    u_t, u_r, _ = bl_state(row["a"], row["r"], row["th"], row["u3"])
    cfg = grid(row["a"], row["r_max"], row["N"])
    x1, x2, u = code_state(cfg, row["r"], row["th"], u_r, 0.0, row["u3"])
    E0, L0 = O.invariants(cfg, O.FIELD_WALD, 1.0, qm, x1, x2, u)
    errs = []
    for dt in (4 * row["dt"], 2 * row["dt"]):
        sim = new_sim(cfg, dt, x1, x2, u, qm=qm)
        errs.append(energy_errors(sim, int(round(T / dt)), O.FIELD_WALD, 1.0, qm,
                                  E0=np.array([E0, L0])))
    for k in (0, 1):
        ratio = errs[0][k] / errs[1][k]
        assert 2.8 < ratio < 6.0, (k, errs)
    assert errs[1][0] < 2e-4 and errs[1][1] < 2e-4


def test_boris_closed_forms():
    # pure magnetic field: rotation by 2 atan(|t|), |u| unchanged
    u = O.boris([1.0, 0.0, 0.0], [0, 0, 0], [0, 0, 0.8], 0.3)
    t = 0.5 * 0.3 * 0.8 / math.sqrt(2.0)
    ang = 2 * math.atan(t)
    assert np.allclose(u, [math.cos(ang), -math.sin(ang), 0.0], atol=1e-15)
    rng = np.random.default_rng(1)
    for _ in range(20):
        u0, B = rng.normal(size=3) * 3, rng.normal(size=3)
        u1 = O.boris(u0, [0, 0, 0], B, 0.7)
        assert math.isclose(np.linalg.norm(u1), np.linalg.norm(u0), rel_tol=1e-14)
    # pure electric field: two half kicks
    u = O.boris([0.1, 0.2, 0.3], [1.0, -2.0, 0.5], [0, 0, 0], 0.25)
    assert np.allclose(u, [0.35, -0.3, 0.425], atol=1e-15)


def test_axis_reflection_and_horizon_removal():
    cfg = grid(0.9, 10.0, 64)
    # moving fast towards theta = 0 from the first cell: reflected, u_2 flips sign
    x1, x2 = 30.5, 0.05
    m = O.metric_point(cfg, x1, x2, clamp=True)
    u = np.array([0.0, -3.0 * math.sqrt(m["h22"]), 0.0])
    sim = new_sim(cfg, 0.03, x1, x2, u)
    sim.push(0, field_mode=1, fkind=0)
    s = sim.species[0].view()
    assert s["i2"][0] == 0 and 0.0 <= s["dx2"][0] < 1.0 and s["u2"][0] > 0
    assert sim.counters[2] == 1 and s["tag"][0] == 1
    # same at theta = pi
    sim = new_sim(cfg, 0.03, x1, 64 - 0.05, -u)
    sim.push(0, field_mode=1, fkind=0)
    s = sim.species[0].view()
    assert s["i2"][0] == 63 and s["u2"][0] < 0 and sim.counters[2] == 1
    # falling in through the horizon layer: tagged when it enters the ghost zone
    x1 = 0.3
    m = O.metric_point(cfg, x1, 20.0, clamp=True)
    sim = new_sim(cfg, 0.05, x1, 20.0, np.array([-5.0 * math.sqrt(m["h11"]), 0.0, 0.0]))
    sim.push(0, field_mode=1, fkind=0)
    s = sim.species[0].view()
    assert s["i1"][0] < 0 and s["tag"][0] == 2 and sim.counters[0] == 1
    sim.push(0, field_mode=1, fkind=0)
    assert sim.species[0].view()["tag"][0] == 0
