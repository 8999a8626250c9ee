"""Pins of the velocity-error measure of the grid-convergence study (Sec. 4):
face-average coarsening of the staggered vertical velocity and the relative
L1 error against the coarsened finest solution."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1610_10053_gb300 import inputs as I


def state_with_vy(prob, vy_of_face):
    """Density 1 + x-only variation (so the face mean density is exact) and
    m_y = rho_bar * v on every y-face."""
    nx, ny = prob.n[0], prob.n[1]
    N = nx * ny
    U = prob.U.copy()
    x = (np.arange(nx) + 0.5) / nx
    rho = np.tile(1.0 + 0.2 * np.sin(2 * np.pi * x), (ny, 1))
    U[:N] = rho.ravel()
    yf = np.arange(ny)[:, None] / ny
    xc = np.tile(x, (ny, 1))
    U[3 * N:4 * N] = (rho * vy_of_face(xc, yf)).ravel()
    return U


def test_coarsening_of_a_field_linear_in_x_is_its_face_centre_value():
    pf, pc = I.kelvin_helmholtz(n=32, nsteps=1), I.kelvin_helmholtz(n=8, nsteps=1)
    vf = O.face_vy(pf, state_with_vy(pf, lambda x, y: 0.3 + 0.5 * x + 0.0 * y))
    vc = O.coarsen_faces(vf, 4)
    xc = (np.arange(8) + 0.5) / 8
    assert np.allclose(vc, np.tile(0.3 + 0.5 * xc, (8, 1)), rtol=0, atol=1e-15)


def test_identical_fields_have_no_error_and_constants_a_closed_form():
    pf, pc = I.kelvin_helmholtz(n=32, nsteps=1), I.kelvin_helmholtz(n=16, nsteps=1)
    f = lambda x, y: np.sin(2 * np.pi * y) * (1 + 0 * x)  # constant along x: coarsening exact
    assert O.velocity_error(pf, state_with_vy(pf, f), pc, state_with_vy(pc, f)) == pytest.approx(0.0, abs=1e-14)
    a, b = 0.7, 0.65
    e = O.velocity_error(pf, state_with_vy(pf, lambda x, y: a + 0 * x), pc, state_with_vy(pc, lambda x, y: b + 0 * x))
    assert e == pytest.approx(abs(b - a) / abs(a), rel=1e-13)


def test_error_of_a_smooth_field_sampled_on_two_grids_is_second_order():
    """The coarse grid's face samples of a smooth field differ from the face
    averages of the fine samples by the midpoint-rule error, O(h^2)."""
    f = lambda x, y: np.sin(2 * np.pi * x) * np.cos(2 * np.pi * y)
    pf = I.kelvin_helmholtz(n=256, nsteps=1)
    Uf = state_with_vy(pf, f)
    errs = []
    for n in (16, 32, 64):
        pc = I.kelvin_helmholtz(n=n, nsteps=1)
        errs.append(O.velocity_error(pf, Uf, pc, state_with_vy(pc, f)))
    order = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert np.all(order > 1.8), (errs, order)
