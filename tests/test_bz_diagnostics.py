"""The BZ monopole diagnostics of bench.py --bz-physics (Sec. 4.5) on the exact force-free
monopole turning at Omega (no GPU: the planes are written here).

For A_phi = -B0 cos(theta) the flux density is sqrt(h) B^r = B0 sin(theta), so in the code
coordinates sqrt(h) B^1 = B0 sin(theta) dtheta/dx2; a field line turning at Omega has
E_theta = -Omega sqrt(h) B^r, i.e. E_2 = -Omega sqrt(h) B^1, and the outgoing solution has
H_phi = -B0 Omega sin^2(theta), E_phi = H_theta = 0. The diagnostics must return Omega at
every radius, the H_phi amplitude -B0 Omega, and L = (2/3) Omega^2 B0^2 (the integral of
sin^3 is 4/3), which for Omega = omega_h / 2 is L_BZ = B0^2 omega_h^2 / 6: the BZ values, with
omega_h = a / (2 r_h), make H_phi = -B0 a sin^2(theta) / 8 up to O(a^2) as the paper has it.
"""
import math

import numpy as np

import bench
import workloads as W

G = 2


class ForceFreeMonopole:
    """Stands for the library context: em planes and auxiliary fields of the BZ solution."""

    def __init__(self, cfg, omega, B0=1.0):
        nr, nt = cfg["n_r"], cfg["n_theta"]
        NX, NY = nr + 2 * G + 1, nt + 2 * G + 1
        a = cfg["a"]
        dxi = math.log(cfg["r_max"] / cfg["r_min"]) / nr
        dth = math.pi / nt
        i = np.arange(NX)[None, :] - G
        j = np.arange(NY)[:, None] - G
        r = cfg["r_min"] * np.exp(i * dxi) + 0.0 * j
        th_half = (j + 0.5) * dth + 0.0 * i          # rows j + 1/2
        sig = r * r + a * a * np.cos(th_half) ** 2
        sqrt_h = dxi * r * dth * sig * np.sin(th_half) * np.sqrt(1.0 + 2.0 * r / sig)
        flux = B0 * np.sin(th_half) * dth                # sqrt(h) B^1 at (i, j + 1/2)
        self.F = np.zeros((28, NY, NX))
        self.F[0] = flux / sqrt_h
        self.E = np.zeros((3, NY, NX))
        self.H = np.zeros((3, NY, NX))
        self.E[1] = -omega * flux
        self.H[2] = -B0 * omega * np.sin(th_half) ** 2  # at (i + 1/2, j + 1/2)

    def planes(self):
        return self.F

    def aux_fields(self):
        return self.E, self.H


def test_diagnostics_return_the_bz_values():
    cfg = W.grid_config("bz1024", n_r=256, n_theta=256)
    a, B0 = cfg["a"], cfg["B0"]
    r_h = 1.0 + math.sqrt(1.0 - a * a)
    omega_h = a / (2.0 * r_h)
    L_BZ = B0 * B0 * omega_h * omega_h / 6.0
    sim = ForceFreeMonopole(cfg, 0.5 * omega_h, B0)
    out = bench.bz_diagnostics(sim, cfg, (2.0, 3.0, 5.0, 8.0))
    for rr, d in out.items():
        assert abs(d["omega"] / omega_h - 0.5) < 1e-12, rr
        assert abs(d["hphi_amp"] / (-B0 * 0.5 * omega_h) - 1.0) < 1e-12, rr
        # the midpoint rule of the sin^3 integral on 256 rows
        assert abs(d["L"] / L_BZ - 1.0) < 1e-4, rr
        # and the paper's H_phi = -B0 a sin^2 / 8 agrees with Omega = omega_h / 2 to O(a^2)
        assert abs(d["hphi_amp"] / (-B0 * a / 8.0) - 1.0) < a * a


def test_diagnostics_follow_omega():
    """Omega enters linearly, L quadratically: a monopole turning at a third of omega_h."""
    cfg = W.grid_config("bz1024", n_r=128, n_theta=96)
    a = cfg["a"]
    omega_h = a / (2.0 * (1.0 + math.sqrt(1.0 - a * a)))
    L_BZ = omega_h * omega_h / 6.0
    out = bench.bz_diagnostics(ForceFreeMonopole(cfg, omega_h / 3.0), cfg, (2.0, 6.0))
    for d in out.values():
        assert abs(d["omega"] / omega_h - 1.0 / 3.0) < 1e-12
        assert abs(d["L"] / L_BZ - 4.0 / 9.0) < 1e-3
