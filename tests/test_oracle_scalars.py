"""Pins of the oracle's passive scalars (Sec. 2.2, Sec. 3).

The scalar operator S_i(q) = -div(c_i rho u) takes the fluid's face mass
fluxes and reconstructs c_i upwind with the van Leer limiter.  Pinned by: a
uniform concentration is carried exactly like the density; the flux form
conserves sum(q_i); second-order truncation against the exact advection of a
smooth profile; the finite-difference product against the exact complex-step
derivative; passivity (the fluid is bitwise the same with and without
scalars); the renormalisation; closed forms of the mixing width.
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1610_10053_gb300 import inputs as I


def _with_scalars(p, c_list):
    N = p.ncells
    rho = p.U[:N]
    return p.with_options(q=np.concatenate([np.asarray(c, dtype=np.float64).ravel() * rho for c in c_list]))


def _smooth_c(p, seed):
    rng = np.random.default_rng(seed)
    N = p.ncells
    i = np.arange(N) % p.n[0]
    j = (np.arange(N) // p.n[0]) % p.n[1]
    k = np.arange(N) // (p.n[0] * p.n[1])
    a = rng.uniform(0, 2 * np.pi, 3)
    return 0.5 + 0.3 * np.sin(2 * np.pi * i / p.n[0] + a[0]) * np.cos(2 * np.pi * j / p.n[1] + a[1]) * \
        np.cos(2 * np.pi * k / p.n[2] + a[2])


CASES = {
    "periodic_2d": lambda: I.random_smooth(2, (20, 14), seed=61, amp=0.3),
    "periodic_3d": lambda: I.random_smooth(3, (9, 8, 7), seed=62, amp=0.3),
    "walls_2d": lambda: I.random_smooth(2, (12, 18), seed=63, amp=0.3, bc=(I.BC_PERIODIC, I.BC_WALL, I.BC_PERIODIC),
                                        wall_scalar=(0, I.WALL_HSE, 0), g=(0.0, -0.4, 0.0)),
}


@pytest.mark.parametrize("case", sorted(CASES))
def test_uniform_concentration_is_carried_like_density(case):
    """c_i uniform: every reconstructed face value is c_i, so S_i = c_i R_rho."""
    p = CASES[case]()
    N = p.ncells
    q = _with_scalars(p, [np.full(N, 0.3), np.full(N, 0.7)])
    S = O.scalar_operator(q, q.U, q.q)
    Rr = O.spatial_operator(p, p.U)[:N]
    scale = np.abs(Rr).max()
    assert np.abs(S[:N] - 0.3 * Rr).max() <= 1e-14 * scale
    assert np.abs(S[N:] - 0.7 * Rr).max() <= 1e-14 * scale


@pytest.mark.parametrize("case", sorted(CASES))
def test_flux_form_conserves_each_scalar(case):
    p = CASES[case]()
    q = _with_scalars(p, [_smooth_c(p, 3), 1.0 - _smooth_c(p, 3)])
    S = O.scalar_operator(q, q.U, q.q)
    N = p.ncells
    for i in range(2):
        Si = S[i * N:(i + 1) * N]
        assert abs(Si.sum()) <= 1e-12 * np.abs(Si).sum()


def _advection_state(n1):
    """rho = 1, uniform velocity (u0, v0), c = smooth periodic profile."""
    u0, v0 = 0.3, -0.2
    p = I.uniform_flow(2, (n1, n1), u=(u0, v0, 0.0))
    N = p.ncells
    x = (np.arange(N) % n1 + 0.5) / n1
    y = (np.arange(N) // n1 + 0.5) / n1
    c = 0.5 + 0.25 * np.sin(2 * np.pi * x) * np.cos(2 * np.pi * y)
    dcdx = 0.25 * 2 * np.pi * np.cos(2 * np.pi * x) * np.cos(2 * np.pi * y)
    dcdy = -0.25 * 2 * np.pi * np.sin(2 * np.pi * x) * np.sin(2 * np.pi * y)
    rho = p.U[:N]
    exact = -rho * (u0 * dcdx + v0 * dcdy)
    return _with_scalars(p, [c]), exact


def test_truncation_error_is_second_order():
    """Uniform rho and u: S = -rho u . grad c exactly for the PDE.  The
    discrete operator converges at second order (L1; limiter clipping at the
    extrema costs a little), which pins the upwinding, the reconstruction and
    the flux difference."""
    errs = []
    for n1 in (16, 32, 64, 128):
        p, exact = _advection_state(n1)
        S = O.scalar_operator(p, p.U, p.q)
        errs.append(np.abs(S - exact).mean())
    errs = np.array(errs)
    order = np.log2(errs[:-1] / errs[1:])
    assert np.all(order > 1.0), (errs, order)
    assert order[-1] >= 1.6, (errs, order)


@pytest.mark.parametrize("case", ["periodic_2d", "walls_2d"])
def test_fd_product_matches_exact_derivative(case):
    p = CASES[case]()
    q = _with_scalars(p, [_smooth_c(p, 5), 1.0 - _smooth_c(p, 5)])
    rng = np.random.default_rng(7)
    v = rng.standard_normal(q.q.size) * 1e-2
    dS = O.scalar_operator_dir(q, q.U, q.q, v)
    eps = 1e-7
    fd = (O.scalar_operator(q, q.U, q.q + eps * v) - O.scalar_operator(q, q.U, q.q)) / eps
    assert np.linalg.norm(fd - dS) <= 1e-5 * np.linalg.norm(dS)


def test_scalars_are_passive():
    """Sec. 2.2: the fluid is advanced exactly as without scalars."""
    p = I.rayleigh_taylor(nx=16, ny=48, nsteps=3, scalars=True)
    U, q, st, sg = O.run_s(p)
    U0, st0 = O.run(p)
    assert np.array_equal(U, U0)
    assert [s["newton_its"] for s in st] == [s["newton_its"] for s in st0]


def test_concentrations_sum_to_one_after_each_step():
    p = I.rayleigh_taylor(nx=16, ny=48, nsteps=3, scalars=True)
    U, q, st, sg = O.run_s(p)
    N = p.ncells
    c = q.reshape(2, N) / U[:N]
    assert np.abs(c.sum(axis=0) - 1.0).max() <= 4e-16
    assert c.min() >= -1e-6 and c.max() <= 1.0 + 1e-6
    assert all(n >= 1 for n in sg)


def test_uniform_concentration_stays_uniform_over_steps():
    """q = c rho solves the same Crank-Nicolson system as rho, to the Newton
    and GMRES tolerances."""
    p = I.kelvin_helmholtz(n=32, seed=9, nsteps=2)
    N = p.ncells
    q = _with_scalars(p, [np.full(N, 0.4), np.full(N, 0.6)])
    U, qq, st, sg = O.run_s(q)
    c = qq.reshape(2, N) / U[:N]
    assert np.abs(c[0] - 0.4).max() <= 1e-6
    assert np.abs(c[1] - 0.6).max() <= 1e-6


def test_enforcing_scalar_convergence():
    """Sec. 3: requiring the scalar corrections to converge as well takes at
    least as many Newton iterations and changes the scalars only at the
    Newton tolerance."""
    p = I.rayleigh_taylor(nx=16, ny=48, nsteps=2, scalars=True)
    U, q, st, sg = O.run_s(p, enforce=0)
    U2, q2, st2, sg2 = O.run_s(p, enforce=1)
    assert all(b["newton_its"] >= a["newton_its"] for a, b in zip(st, st2))
    assert np.abs(q2 - q).max() <= 1e-6


def test_mixing_width_closed_forms():
    p = I.rayleigh_taylor(nx=8, ny=40, nsteps=1, scalars=True)
    N, nx, ny = p.ncells, p.n[0], p.n[1]
    L = p.length[1]
    # the initial sharp interface: no mixed row
    assert O.scalar_mixing_width(p, p.U, p.q) == 0.0
    # a linear ramp of <c_1> from 1 to 0 over the box: 2 min(c, 1 - c) is a
    # tent whose midpoint sum on an even number of rows is exact: L / 2
    j = np.arange(N) // nx
    c1 = 1.0 - (j + 0.5) / ny
    q = _with_scalars(p, [c1, 1.0 - c1])
    assert O.scalar_mixing_width(q, q.U, q.q) == pytest.approx(L / 2, rel=1e-13)
    # rows are averaged before the minimum: half a row pure c_1, half pure
    # c_2 gives <c> = (1/2, 1/2), a fully mixed row of width dy
    i = np.arange(N) % nx
    c1 = np.where((i < nx // 2) & (j == 7), 1.0, np.where(j < 7, 1.0, 0.0))
    q = _with_scalars(p, [c1, 1.0 - c1])
    assert O.scalar_mixing_width(q, q.U, q.q) == pytest.approx(L / ny, rel=1e-13)
