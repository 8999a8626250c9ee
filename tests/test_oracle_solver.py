"""Pins of the oracle's JFNK solver (Sec. 2): the finite-difference Jv, GMRES,
the physics-based preconditioner, Newton and the CFL time step.

The exact Jacobian comes from complex-step differentiation of R (an exact
derivative, independent of the finite-difference formula) and dense linear
algebra from numpy.
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1610_10053_gb300 import inputs as I


def exact_jv(prob, U, v, dt):
    """J v = v - dt/2 (dR/dU) v with the exact derivative."""
    return v - 0.5 * dt * O.spatial_operator_dir(prob, U, v)


def dense_jacobian(prob, U, dt):
    n = U.size
    J = np.empty((n, n))
    e = np.zeros(n)
    for j in range(n):
        e[j] = 1.0
        J[:, j] = exact_jv(prob, U, e, dt)
        e[j] = 0.0
    return J


@pytest.mark.parametrize("make", [
    lambda: I.random_smooth(2, (8, 8), seed=11, amp=0.3),
    lambda: I.random_smooth(2, (8, 10), seed=16, amp=0.3, bc=(I.BC_PERIODIC, I.BC_WALL, I.BC_PERIODIC),
                            wall_scalar=(0, I.WALL_HSE, 0), g=(0.0, -0.3, 0.0)),
    lambda: I.random_smooth(3, (5, 4, 6), seed=12, amp=0.3),
])
def test_fd_jv_matches_exact_derivative(make):
    """Knoll & Keyes' finite-difference product approximates the exact
    directional derivative to O(sqrt(machine eps)) away from limiter switches."""
    p = make()
    rng = np.random.default_rng(0)
    v = rng.standard_normal(p.U.size)
    dt = 0.01
    ref = exact_jv(p, p.U, v, dt)
    got = O.jv(p, p.U, v, dt)
    assert np.linalg.norm(got - ref) <= 1e-6 * np.linalg.norm(ref)


def test_complex_step_jacobian_matches_central_differences():
    """The complex-step derivative itself agrees with central differences."""
    p = I.random_smooth(2, (6, 6), seed=13, amp=0.3)
    rng = np.random.default_rng(1)
    v = rng.standard_normal(p.U.size)
    h = 1e-6
    cd = (O.spatial_operator(p, p.U + h * v) - O.spatial_operator(p, p.U - h * v)) / (2 * h)
    cs = O.spatial_operator_dir(p, p.U, v)
    assert np.linalg.norm(cs - cd) <= 1e-7 * np.linalg.norm(cs)


@pytest.mark.parametrize("m,restarts", [(30, 0), (5, 40)])
def test_gmres_dense_solves(m, restarts):
    """GMRES (Saad & Schultz) on a nonsymmetric well-conditioned matrix, with
    and without restarts, against a direct solve."""
    rng = np.random.default_rng(2)
    n = 24
    A = np.eye(n) * 4 + rng.standard_normal((n, n)) * 0.5
    b = rng.standard_normal(n)
    x, rc, its = O.gmres_dense(A, b, m=m, max_restarts=restarts, rtol=1e-12)
    assert rc == 0
    xr = np.linalg.solve(A, b)
    assert np.linalg.norm(x - xr) <= 1e-10 * np.linalg.norm(xr)
    if restarts == 0:
        assert its <= n


def test_gmres_zero_rhs():
    A = np.eye(4)
    x, rc, its = O.gmres_dense(A, np.zeros(4))
    assert rc == 0 and its == 0 and np.all(x == 0)


def _rest_state(nd, n, walls=False):
    p = I.uniform_flow(nd, n, rho=1.3, p=2.0, u=(0.0, 0.0, 0.0))
    if walls:
        p = p.with_options(bc=(I.BC_PERIODIC, I.BC_WALL, I.BC_PERIODIC))
    return p


@pytest.mark.parametrize("nd,n,walls", [(2, (8, 6), False), (2, (6, 8), True), (3, (4, 6, 4), False)])
def test_preconditioner_inverts_acoustic_jacobian(nd, n, walls):
    """At a uniform state at rest the linearised operator is exactly the
    acoustic system the preconditioner eliminates (advection and gravity
    vanish), so with converged relaxation M^-1 J v = v for every v."""
    p = _rest_state(nd, n, walls).with_options(sweeps=3000)
    dt = 0.05
    rng = np.random.default_rng(3)
    v = rng.standard_normal(p.U.size)
    if walls:
        N = p.ncells
        my = v[3 * N:4 * N].reshape(p.n[2], p.n[1], p.n[0])
        my[:, 0, :] = 0.0  # stored wall faces carry no unknown
    Jv = exact_jv(p, p.U, v, dt)
    z = O.precond(p, p.U, dt, Jv)
    assert np.linalg.norm(z - v) <= 1e-10 * np.linalg.norm(v)


def test_preconditioner_linear_conservative_and_consistent():
    p = I.random_smooth(2, (8, 10), seed=14, amp=0.3)
    N = p.ncells
    rng = np.random.default_rng(4)
    r1, r2 = rng.standard_normal((2, p.U.size))
    dt = 0.02
    z1, z2 = O.precond(p, p.U, dt, r1), O.precond(p, p.U, dt, r2)
    z12 = O.precond(p, p.U, dt, 2.0 * r1 - 3.0 * r2)
    assert np.linalg.norm(z12 - (2 * z1 - 3 * z2)) <= 1e-12 * np.linalg.norm(z12)
    # flux form: mass and momentum sums are unchanged (periodic)
    for v in (0, 2, 3):
        s = slice(v * N, (v + 1) * N)
        assert abs(z1[s].sum() - r1[s].sum()) <= 1e-12 * np.abs(r1[s]).sum()
    # dt -> 0: M -> I
    z0 = O.precond(p, p.U, 1e-12, r1)
    assert np.linalg.norm(z0 - r1) <= 1e-9 * np.linalg.norm(r1)
    # NONE is the identity
    assert np.array_equal(O.precond(p.with_options(precond=I.PC_NONE), p.U, dt, r1), r1)


@pytest.mark.parametrize("pc", [I.PC_NONE, I.PC_ACOUSTIC])
def test_newton_matches_dense_lu_newton(pc):
    """Sec. 2: the JFNK step reaches the same Crank-Nicolson solution as a
    Newton iteration with the exact dense Jacobian and an LU solve."""
    p = I.random_smooth(2, (8, 8), seed=15, amp=0.3).with_options(
        precond=pc, newton_tol=1e-12, gmres_rtol=1e-8, newton_max=20)
    dt = 0.5 * O.cfl_dt(p, p.U, 2.0)
    Un = p.U
    U = Un.copy()
    for _ in range(30):
        F = O.cn_residual(p, U, Un, dt)
        J = dense_jacobian(p, U, dt)
        dU = np.linalg.solve(J, -F)
        U = U + dU
        if np.abs(dU).max() <= 1e-14 * np.abs(U).max():
            break
    assert np.abs(O.cn_residual(p, U, Un, dt)).max() <= 1e-12
    Uj, st, rc = O.newton_step(p, Un, dt)
    assert rc == 0
    assert np.abs(Uj - U).max() <= 1e-9 * np.abs(U).max()


def test_cfl_time_step_closed_form():
    """Eq. 4: CFL_hydro = max((|u| + c_s)/dx) dt."""
    gamma, rho, pr = 1.4, 1.3, 2.0
    u = (0.3, -0.2, 0.1)
    p = I.uniform_flow(3, (4, 5, 6), rho=rho, p=pr, u=u, gamma=gamma, length=(1.0, 2.0, 0.5))
    cs = np.sqrt(gamma * pr / rho)
    rate = max((abs(u[d]) + cs) / (p.length[d] / p.n[d]) for d in range(3))
    assert abs(O.cfl_dt(p, p.U, 3.0) - 3.0 / rate) <= 1e-14 * 3.0 / rate


def test_step_conserves_mass_and_momentum():
    """Periodic, g = 0: every Newton correction is a sum of flux differences
    and conservative preconditioned Krylov vectors, so sum rho and sum m are
    constant to rounding whatever the Newton tolerance."""
    p = I.kelvin_helmholtz(n=16).with_options(newton_tol=1e-4)
    N = p.ncells
    U, st = O.run(p, nsteps=2)
    for v in (0, 2, 3):
        s = slice(v * N, (v + 1) * N)
        assert abs(U[s].sum() - p.U[s].sum()) <= 1e-13 * np.abs(p.U[s]).sum()


def test_newton_converged_state_solves_cn_system():
    p = I.rayleigh_taylor(nx=16, ny=48)
    dt = O.cfl_dt(p, p.U, 5.0)
    U1, st, rc = O.newton_step(p, p.U, dt)
    assert rc == 0 and st["max_drho"] <= 1e-8 and st["newton_its"] >= 2
    F = O.cn_residual(p, U1, p.U, dt)
    assert np.linalg.norm(F) <= 1e-6 * np.linalg.norm(O.cn_residual(p, p.U, p.U, dt))


def test_rt_linear_growth_rate():
    """Sec. 3: Atwood number 1/3, g = 0.1 and the k = 4 pi mode give the
    linear Rayleigh-Taylor growth rate sqrt(A g k) = 0.647; a small-amplitude
    run of the oracle reaches it within 15 % once the seeding transient has
    passed (finite depth, compressibility and numerical diffusion lower it
    slightly)."""
    p = I.rayleigh_taylor(nx=32, ny=96)
    N = p.ncells
    U = p.U.copy()
    U[3 * N:] *= 1e-3
    t, ts, vs = 0.0, [], []
    while t < 7.0:
        U, st = O.run(p, U=U, nsteps=1, cfl=2.0)
        t += st[0]["dt"]
        ts.append(t)
        vs.append(np.abs(U[3 * N:]).max())
    ts, vs = np.array(ts), np.array(vs)
    m = (ts >= 5.0) & (ts <= 7.0)
    sigma = np.polyfit(ts[m], np.log(vs[m]), 1)[0]
    expect = np.sqrt((1.0 / 3.0) * 0.1 * 4 * np.pi)
    assert abs(sigma - expect) <= 0.15 * expect, sigma
