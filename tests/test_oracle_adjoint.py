"""Pins of the oracle's frozen-field test-particle push and of its FP64 reference Jacobian
(complex step), which the GPU adjoint is checked against.

The Jacobian is pinned to the derivative of the actual double map by central finite
differences (brute force), to an exact identity (the phi column), to a different
parameter (scaling the fields equals scaling q/m, Sec. 3.1's Boris coefficient), and to the
chain rule across segments; the frozen push itself is pinned to the oracle's main pusher.
"""
import numpy as np
import pytest

import workloads as W
from oracle import oracle as O

N_ITER = 60  # both implicit pushes iterated to convergence (contraction well below 0.5)


@pytest.fixture(scope="module")
def setup():
    cfg = W.grid_config("wald64", r_absorb=1e300)
    osim = O.OracleSim(cfg)
    osim.init_fields(O.FIELD_WALD, 1.0)
    tp = W.probe_particles(cfg, 16, 3, (15.0, 50.0), (12.0, 52.0), 0.5)
    qm, qc = W.species_coefficients(1.0)
    sp = osim.add_species(tp["pos"], tp["uhat"], tp["w0"], qm, qc)
    v = sp.view()
    st0 = np.stack([v["i1"] + v["dx1"], v["i2"] + v["dx2"], v["phi"], v["u1"], v["u2"], v["u3"]])
    return osim, st0, qm


def central_fd(osim, st0, qm, n_steps, name, h=1e-6):
    sp, sm = st0.copy(), st0.copy()
    s_p = s_m = 1.0
    if name == "scale":
        s_p, s_m = 1.0 + h, 1.0 - h
    else:
        k = O.FROZEN_STATE.index(name)
        sp[k] += h
        sm[k] -= h
    fp = O.frozen_push(osim, sp, s_p, qm, n_steps, N_ITER)
    fm = O.frozen_push(osim, sm, s_m, qm, n_steps, N_ITER)
    return ((fp - fm) / (2 * h)).T


def test_frozen_push_equals_main_pusher(setup):
    """Frozen push (absolute coordinates) against ora_push (cell + offset storage) with the
    predicted-field planes set to the em planes: same steps of Sec. 3.1."""
    osim, st0, qm = setup
    o2 = O.OracleSim(osim.cfg)
    o2.F[:] = osim.F
    o2.F[O.BN1:O.BN1 + 3] = o2.F[O.B1:O.B1 + 3]
    n = st0.shape[1]
    arrays = {k: np.zeros(n, dtype=t) for k, t in O.PARTICLE_FIELDS.items()}
    for q, (ik, dk) in enumerate((("i1", "dx1"), ("i2", "dx2"))):
        arrays[ik] = np.floor(st0[q]).astype(np.int32)
        arrays[dk] = st0[q] - arrays[ik]
    arrays["u1"], arrays["u2"], arrays["u3"] = st0[3], st0[4], st0[5]
    arrays["tag"][:] = 1
    o2.add_raw_species(arrays, qm, 1.0)
    for _ in range(20):
        o2.push(0)
    v = o2.species[0].view()
    fin = O.frozen_push(osim, st0, 1.0, qm, 20)  # the configuration's n_iter, as ora_push
    ok = ~np.isnan(fin[0])
    assert ok.sum() >= 12
    got = np.stack([v["i1"] + v["dx1"], v["i2"] + v["dx2"], v["phi"], v["u1"], v["u2"], v["u3"]])
    scale = np.maximum(1.0, np.abs(fin[:, ok]))
    assert np.max(np.abs(got[:, ok] - fin[:, ok]) / scale) < 1e-11


def test_complex_step_jacobian_matches_central_differences(setup):
    osim, st0, qm = setup
    fin, J = O.frozen_jacobian(osim, st0, 1.0, qm, 100, N_ITER)
    ok = ~np.isnan(fin[0])
    assert ok.sum() >= 12
    for c, name in enumerate(list(O.FROZEN_STATE) + ["scale"]):
        fd = central_fd(osim, st0, qm, 100, name)
        cs = J[ok, :, c]
        scale = np.abs(cs).max(axis=1, keepdims=True) + 1e-300
        err = np.abs(fd[ok] - cs) / scale
        assert err.max() < 1e-6, (name, err.max())


def test_phi_column_is_exact(setup):
    """phi never feeds back: d(final)/d(phi0) is the unit vector of phi, to the bit."""
    osim, st0, qm = setup
    fin, J = O.frozen_jacobian(osim, st0, 1.0, qm, 50, N_ITER, inputs=["phi"])
    ok = ~np.isnan(fin[0])
    e = np.zeros(6)
    e[2] = 1.0
    assert np.array_equal(J[ok, :, 0], np.broadcast_to(e, (ok.sum(), 6)))


def test_scale_column_equals_charge_to_mass_derivative(setup):
    """Fields enter only through (q/m) * field in the Boris step, so
    d/d(scale) at scale 1 = qm * d/d(qm): complex step in one, central differences in the
    other."""
    osim, st0, qm = setup
    fin, J = O.frozen_jacobian(osim, st0, 1.0, qm, 60, N_ITER, inputs=["scale"])
    h = 1e-6 * abs(qm)
    fp = O.frozen_push(osim, st0, 1.0, qm + h, 60, N_ITER)
    fm = O.frozen_push(osim, st0, 1.0, qm - h, 60, N_ITER)
    dq = ((fp - fm) / (2 * h)).T * qm
    ok = ~np.isnan(fin[0])
    scale = np.abs(J[ok, :, 0]).max(axis=1, keepdims=True)
    assert np.max(np.abs(dq[ok] - J[ok, :, 0]) / scale) < 1e-6


def test_jacobian_obeys_the_chain_rule(setup):
    """J over 2N steps = J(second N steps at the intermediate state) J(first N steps)."""
    osim, st0, qm = setup
    mid, J1 = O.frozen_jacobian(osim, st0, 1.0, qm, 40, N_ITER)
    fin, J2 = O.frozen_jacobian(osim, mid, 1.0, qm, 40, N_ITER)
    fin2, J = O.frozen_jacobian(osim, st0, 1.0, qm, 80, N_ITER)
    ok = ~np.isnan(fin2[0]) & ~np.isnan(fin[0])
    assert ok.sum() >= 12
    # extend to 7 x 7 with the scale as a constant input
    for k in np.flatnonzero(ok):
        A = np.vstack([J1[k], np.eye(7)[6]])
        B = np.vstack([J2[k], np.eye(7)[6]])
        C = (B @ A)[:6]
        sc = np.abs(J[k]).max() + 1e-300
        assert np.max(np.abs(C - J[k])) / sc < 1e-11, k
    assert np.allclose(fin[:, ok], fin2[:, ok], rtol=1e-13, atol=1e-13)
