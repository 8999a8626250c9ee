"""Pins of the oracle's diagnostics (Secs. 3-6) against closed forms."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1610_10053_gb300 import inputs as I


@pytest.mark.parametrize("n", [4, 8, 16])
def test_tgv_initial_kinetic_energy(n):
    """Sec. 5: the volume-averaged kinetic energy of the Taylor-Green
    initial field is rho0 u0^2 / 8; sampled on the staggered grid the face
    sums are exact by discrete orthogonality for n >= 3."""
    p = I.taylor_green(n=n)
    d = O.diagnostics(p, p.U)
    assert abs(d["mean_kinetic_energy"] - 0.125) <= 1e-14


def test_rt_initial_mixing_height_is_zero():
    """Sec. 3 (Cabot & Cook): unmixed layers have X_H in {0, 1}, so X_M = 0."""
    p = I.rayleigh_taylor(perturbation="none")
    assert O.diagnostics(p, p.U)["mixing_height"] == 0.0


def test_mixing_height_of_linear_ramp():
    """A density rising linearly from rho_L to rho_H across the box gives a
    tent-shaped X_M whose integral is half the box height."""
    p = I.rayleigh_taylor(nx=8, ny=32, perturbation="none")
    N = p.ncells
    U = p.U.copy()
    y = (np.arange(32) + 0.5) / 32
    U[:N] = np.repeat(1.0 + y, 8)
    assert abs(O.diagnostics(p, U)["mixing_height"] - 0.75) <= 1e-13


def test_mode_amplitude_and_vertical_energy():
    """Sec. 4: for v_y = A sin(4 pi x) + B cos(4 pi x) at uniform density the
    projection on the two-wavelength mode returns sqrt(A^2 + B^2), and the
    vertical kinetic energy is the integral of rho v^2 / 2 = rho (A^2 + B^2)/4."""
    A, B, rho = 0.03, -0.02, 1.5
    p = I.uniform_flow(2, (16, 12), rho=rho, p=1.0, u=(0.0, 0.0, 0.0))
    N = p.ncells
    x = (np.arange(16) + 0.5) / 16
    v = A * np.sin(4 * np.pi * x) + B * np.cos(4 * np.pi * x)
    U = p.U.copy()
    U[3 * N:] = np.tile(rho * v, 12)
    d = O.diagnostics(p, U)
    assert abs(d["kh_mode_amplitude"] - np.hypot(A, B)) <= 1e-15
    assert abs(d["vertical_kinetic_energy"] - rho * (A * A + B * B) / 4) <= 1e-15


def test_mach_and_speed_of_uniform_flow():
    gamma, rho, pr = 1.4, 1.3, 2.0
    u = (0.3, -0.2)
    p = I.uniform_flow(2, (6, 6), rho=rho, p=pr, u=u, gamma=gamma)
    d = O.diagnostics(p, p.U)
    speed = np.hypot(*u)
    assert abs(d["max_speed"] - speed) <= 1e-15
    assert abs(d["max_mach"] - speed / np.sqrt(gamma * pr / rho)) <= 1e-15
