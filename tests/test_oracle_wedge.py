"""Pins of the oracle's spherical geometry and radiative diffusion (Sec. 2,
Eqs. 1-3 with div(chi grad T) and the photon conductivity; Sec. 6 setup).

As for the Cartesian operator, the discrete R is checked against the
continuous right-hand sides, here written in axisymmetric spherical
coordinates by sympy, plus exact discrete invariants and closed forms.
"""
import json
import os

import numpy as np
import pytest
import sympy as sp

from oracle import oracle as O
from paper_1610_10053_gb300 import inputs as I

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def test_lane_emden_n3_constants():
    """Textbook constants of the n = 3 polytrope (first zero and the mass
    integral) that the wedge background is built from."""
    with open(os.path.join(GOLD, "lane_emden_n3.json")) as fh:
        gold = json.load(fh)
    xs, ts, ds, xi1 = I.lane_emden(3.0)
    assert abs(xi1 - gold["xi1"]) <= 2e-5
    assert abs(-xi1 ** 2 * ds[-1] - gold["mass"]) <= 2e-5


def wedge_problem(nr, nth, chi0=0.0, gface=None, length=(1.0, np.pi / 2)):
    r0, th0 = 0.5, np.pi / 4
    n = (nr, nth, 1)
    U = np.zeros(4 * nr * nth)
    p = I.Problem("sph", 2, n, (r0, th0, 0.0), (length[0], length[1], 1.0), (I.BC_WALL, I.BC_PERIODIC, 0),
                  (I.WALL_MIRROR, 0, 0), 5.0 / 3.0, (0.0, 0.0, 0.0), U, geometry=I.GEOM_SPHERICAL,
                  gface=gface, conduct=1 if chi0 else 0, chi0=chi0)
    return p


def symbolic_sph(gamma, chi0, L, th0, dth):
    r, t = sp.symbols("r t", positive=True)
    r0 = sp.Rational(1, 2)
    a = sp.pi * (r - r0) / L           # 0 .. pi across the radial range
    b = 2 * sp.pi * (t - th0) / dth    # one period across the wedge
    # scalars: zero radial slope at the walls; radial velocity zero there,
    # polar velocity with zero radial slope (stress free)
    rho = 1 + sp.Rational(1, 5) * sp.cos(a) + sp.Rational(1, 10) * sp.sin(b)
    p = 1 + sp.Rational(1, 5) * sp.cos(2 * a) * sp.cos(b + sp.Rational(1, 3))
    ur = sp.Rational(3, 10) * sp.sin(a) * sp.cos(b)
    ut = sp.Rational(1, 4) * sp.cos(a) * sp.sin(b) + sp.Rational(1, 10)
    gr = -1 / r ** 2
    E = p / (gamma - 1)
    T = p / rho
    chi = chi0 * T ** sp.Rational(13, 2) / rho ** 2

    def div(Fr, Ft):
        return sp.diff(r ** 2 * Fr, r) / r ** 2 + sp.diff(sp.sin(t) * Ft, t) / (r * sp.sin(t))

    divu = div(ur, ut)
    drho = -div(rho * ur, rho * ut)
    dE = -div(E * ur, E * ut) - p * divu + div(chi * sp.diff(T, r), chi * sp.diff(T, t) / r)
    dmr = -div(rho * ur * ur, rho * ur * ut) + rho * ut ** 2 / r - sp.diff(p, r) + rho * gr
    dmt = -div(rho * ut * ur, rho * ut * ut) - rho * ur * ut / r - sp.diff(p, t) / r
    f = lambda e: sp.lambdify((r, t), e, "numpy")
    return [f(q) for q in (rho, E, ur, ut, drho, dE, dmr, dmt, gr)]


@pytest.mark.parametrize("chi0", [0.0, 0.02])
def test_spherical_truncation_error_is_second_order(chi0):
    """Axisymmetric spherical form of Eqs. 1-3 (area-weighted divergences,
    the geometric terms +rho u_t^2/r and -rho u_r u_t/r, radial gravity g(r)
    on the r-faces, and div(chi grad T)): the discrete operator converges to
    the symbolic right-hand side at second order in L1."""
    gamma, L, th0, dth = 5.0 / 3.0, 1.0, np.pi / 4, np.pi / 2
    fns = symbolic_sph(gamma, chi0, L, th0, dth)
    rho_f, E_f, ur_f, ut_f, drho_f, dE_f, dmr_f, dmt_f, g_f = fns
    errs = []
    for m in (32, 64, 128):
        nr, nth = m, m // 2
        rf = 0.5 + np.arange(nr + 1) * (L / nr)
        p = wedge_problem(nr, nth, chi0=chi0, gface=g_f(rf, 0.0) * np.ones(nr + 1))
        rc = 0.5 + (np.arange(nr) + 0.5) * (L / nr)
        tc = th0 + (np.arange(nth) + 0.5) * (dth / nth)
        rfa = 0.5 + np.arange(nr) * (L / nr)
        tfa = th0 + np.arange(nth) * (dth / nth)
        Rc, Tc = np.meshgrid(rc, tc)
        Rr, Tr = np.meshgrid(rfa, tc)   # r-faces
        Rt, Tt = np.meshgrid(rc, tfa)   # theta-faces
        U = np.concatenate([rho_f(Rc, Tc).ravel(), E_f(Rc, Tc).ravel(),
                            (rho_f(Rr, Tr) * ur_f(Rr, Tr)).ravel(), (rho_f(Rt, Tt) * ut_f(Rt, Tt)).ravel()])
        ex = [drho_f(Rc, Tc), dE_f(Rc, Tc), dmr_f(Rr, Tr), dmt_f(Rt, Tt)]
        ex[2] = np.where(Rr == 0.5, 0.0, ex[2])  # the stored wall face carries R = 0
        R = O.spatial_operator(p, U)
        N = nr * nth
        errs.append([np.abs(R[v * N:(v + 1) * N] - np.ravel(ex[v])).mean() for v in range(4)])
    errs = np.array(errs)
    order = np.log2(errs[:-1] / errs[1:])
    assert np.all(order[-1] >= 1.6), (errs, order)


def test_wedge_background_is_a_discrete_equilibrium():
    """Sec. 6: the polytrope-seeded background balances pressure, gravity and
    the radiative flux on the staggered spherical grid to rounding, and an
    implicit step at 100x the acoustic CFL limit keeps it at rest."""
    p = I.spherical_wedge(nr=32, nth=16, noise=0.0)
    N = p.ncells
    R = O.spatial_operator(p, p.U)
    E = p.U[N:2 * N]
    assert np.abs(R[:N]).max() == 0.0
    assert np.abs(R[N:2 * N]).max() <= 1e-11 * np.abs(E).max()
    assert np.abs(R[2 * N:]).max() <= 1e-12
    dt = O.cfl_dt(p, p.U, 100.0)
    U1, st, rc = O.newton_step(p, p.U, dt)
    assert rc == 0
    assert np.abs(U1[2 * N:]).max() <= 1e-15


def test_spherical_mass_conservation():
    """Volume-weighted sum of R_rho vanishes: walls carry no mass flux and
    every interior face flux enters two cells with the same area."""
    p = I.spherical_wedge(nr=24, nth=12, noise=1e-3)
    N = p.ncells
    rng = np.random.default_rng(2)
    U = p.U.copy()
    U[2 * N:] = 1e-3 * rng.standard_normal(2 * N)
    U[2 * N:3 * N].reshape(12, 24)[:, 0] = 0.0
    R = O.spatial_operator(p, U)
    g = O.grid(p)
    r = p.x0[0] + np.arange(25) * p.dx[0]
    th = p.x0[1] + np.arange(13) * p.dx[1]
    V = np.outer(np.cos(th[:-1]) - np.cos(th[1:]), (r[1:] ** 3 - r[:-1] ** 3) / 3.0).ravel()
    assert abs((V * R[:N]).sum()) <= 1e-13 * (V * np.abs(R[:N])).sum()


def test_fd_jv_with_conduction_matches_exact_derivative():
    """Cartesian, with conduction: Knoll & Keyes' product against the exact
    complex-step derivative."""
    p = I.random_smooth(2, (8, 8), seed=31, amp=0.3).with_options(conduct=1, chi0=0.05)
    dt = 1e-2
    rng = np.random.default_rng(3)
    v = rng.standard_normal(p.U.size)
    ref = v - 0.5 * dt * O.spatial_operator_dir(p, p.U, v)
    got = O.jv(p, p.U, v, dt)
    assert np.linalg.norm(got - ref) <= 1e-6 * np.linalg.norm(ref)


def test_spherical_fd_derivative_converges_to_exact():
    """Spherical wedge with conduction (strong stratification, chi ~ T^6.5 /
    rho^2): the finite-difference quotient of R converges at first order to
    the exact complex-step derivative (error / eps constant as eps -> 0)."""
    p = I.spherical_wedge(nr=10, nth=8, noise=0.0)
    N = p.ncells
    U = p.U.copy()
    i = np.arange(10)[None, :] + 0.5
    j = np.arange(8)[:, None] + 0.5
    # a smooth flow and a smooth polar density mode, off the limiter's switches
    U[2 * N:3 * N] = (1e-2 * np.sin(np.pi * (i - 0.5) / 10) * np.cos(2 * np.pi * j / 8)).ravel()
    U[3 * N:] = (1e-2 * np.cos(np.pi * i / 10) * np.sin(2 * np.pi * j / 8 + 0.3)).ravel()
    U[:N] *= (1.0 + 1e-2 * np.cos(2 * np.pi * j / 8 + 0.5) * np.ones_like(i)).ravel()
    p = p.with_state(U)
    v = np.random.default_rng(3).standard_normal(p.U.size)
    exact = O.spatial_operator_dir(p, p.U, v)
    R0 = O.spatial_operator(p, p.U)
    err = [np.linalg.norm((O.spatial_operator(p, p.U + e * v) - R0) / e - exact) for e in (1e-6, 1e-7, 1e-8)]
    assert 7.0 <= err[0] / err[1] <= 14.0 and 7.0 <= err[1] / err[2] <= 14.0, err
    assert err[2] <= 1e-3 * np.linalg.norm(exact), (err, np.linalg.norm(exact))


@pytest.mark.parametrize("sph", [False, True])
def test_thermal_preconditioner_inverts_jacobian_at_rest(sph):
    """At a uniform state at rest the temperature gradient vanishes, so the
    linearised operator is the acoustic system plus conduction of the energy
    perturbation; for directions without a density part the preconditioner
    with converged relaxation inverts it exactly."""
    if sph:
        p = wedge_problem(8, 6, chi0=0.3)
        N = p.ncells
        U = np.concatenate([np.full(N, 1.3), np.full(N, 3.0), np.zeros(2 * N)])
        p = p.with_state(U)
    else:
        p = I.uniform_flow(2, (8, 6), rho=1.3, p=2.0, u=(0.0, 0.0, 0.0)).with_options(conduct=1, chi0=0.3)
    p = p.with_options(sweeps=4000)
    N = p.ncells
    dt = 0.05
    rng = np.random.default_rng(4)
    v = rng.standard_normal(p.U.size)
    v[:N] = 0.0
    if sph:
        v[2 * N:3 * N].reshape(6, 8)[:, 0] = 0.0
    Jv = v - 0.5 * dt * O.spatial_operator_dir(p, p.U, v)
    z = O.precond(p, p.U, dt, Jv)
    assert np.linalg.norm(z - v) <= 1e-9 * np.linalg.norm(v)


def test_cartesian_conduction_truncation_error():
    """div(chi grad T) with chi = chi0 T^6.5/rho^2 added to Eq. 2 converges at
    second order against the symbolic right-hand side (periodic box)."""
    x, y = sp.symbols("x y", real=True)
    tp = 2 * sp.pi
    gamma, chi0 = 1.4, 0.05
    rho = 1 + sp.Rational(1, 5) * sp.sin(tp * x + 0.3) * sp.cos(tp * y)
    p = 1 + sp.Rational(1, 5) * sp.cos(tp * x) * sp.sin(tp * y + 0.4)
    T = p / rho
    chi = chi0 * T ** sp.Rational(13, 2) / rho ** 2
    dE = sp.diff(chi * sp.diff(T, x), x) + sp.diff(chi * sp.diff(T, y), y)
    f_rho, f_E, f_dE = [sp.lambdify((x, y), e, "numpy") for e in (rho, p / (gamma - 1), dE)]
    errs = []
    for n in (32, 64, 128):
        c = (np.arange(n) + 0.5) / n
        X, Y = np.meshgrid(c, c)
        prob = I.uniform_flow(2, (n, n), gamma=gamma, u=(0.0, 0.0, 0.0))
        U = np.concatenate([f_rho(X, Y).ravel(), f_E(X, Y).ravel(), np.zeros(2 * n * n)])
        R1 = O.spatial_operator(prob.with_options(conduct=1, chi0=chi0), U)
        R0 = O.spatial_operator(prob, U)
        N = n * n
        errs.append(np.abs((R1 - R0)[N:2 * N] - f_dE(X, Y).ravel()).mean())
    order = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert order[-1] >= 1.8, (errs, order)
