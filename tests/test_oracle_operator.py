"""Pins of the oracle's spatial operator R(U) (Eqs. 1-3, Sec. 2).

None of these compare the oracle with itself: they check it against the
continuous equations (symbolic right-hand sides), exact invariants of the
discretisation the paper describes (conservation form, hydrostatic balance on
the staggered grid, mirror symmetry of Sec. 3) and closed forms.
"""
import numpy as np
import pytest
import sympy as sp

from oracle import oracle as O
from paper_1610_10053_gb300 import inputs as I


def split(prob, U):
    N = prob.ncells
    nz, ny, nx = prob.n[2], prob.n[1], prob.n[0]
    return [U[v * N:(v + 1) * N].reshape(nz, ny, nx) for v in range(prob.nvars)]


# ---------------------------------------------------------------- closed forms
@pytest.mark.parametrize("nd,n", [(2, (8, 6)), (3, (5, 4, 6))])
def test_uniform_flow_is_steady(nd, n):
    """Constant rho, p, u in a periodic box: every flux difference vanishes."""
    p = I.uniform_flow(nd, n)
    R = O.spatial_operator(p, p.U)
    assert np.abs(R).max() <= 1e-13


def test_term_magnitudes_of_uniform_flow():
    """Per-cell sum of the magnitudes of R's terms (the scale the GPU parity
    tests hold R's rounding to), on a uniform flow along x and y, where every
    term is a known flux: mass rho u_d and energy u_d E through both faces of
    each direction, p |u_d| of the velocity divergence, centre momentum flux
    rho u_d^2, edge flux rho u_q u_d, and the pressure on both faces.  R
    itself vanishes, so this also shows the sum is not |R|."""
    nx, ny, rho, pr, ux, uy, gam = 8, 6, 1.3, 2.0, 0.3, -0.2, 1.4
    p = I.uniform_flow(2, (nx, ny), rho=rho, p=pr, u=(ux, uy, 0.0), gamma=gam)
    R, A = O.spatial_operator_terms(p, p.U)
    assert np.array_equal(R, O.spatial_operator(p, p.U))
    E = pr / (gam - 1.0)
    ix, iy = nx, ny  # 1 / dx, 1 / dy on the unit box
    want = [2 * rho * (abs(ux) * ix + abs(uy) * iy),
            2 * (abs(ux) * E * ix + abs(uy) * E * iy) + pr * 2 * (abs(ux) * ix + abs(uy) * iy),
            2 * rho * ux * ux * ix + 2 * abs(rho * uy * ux) * iy + 2 * pr * ix,
            2 * rho * uy * uy * iy + 2 * abs(rho * ux * uy) * ix + 2 * pr * iy]
    N = p.ncells
    for v, w in enumerate(want):
        np.testing.assert_allclose(A[v * N:(v + 1) * N], w, rtol=1e-12)


@pytest.mark.parametrize("case", ["periodic3d", "walls_gravity2d", "wedge", "conduct2d"])
def test_term_magnitudes_bound_the_residual(case):
    """|R| <= sum of |terms| per cell and variable (the triangle inequality,
    up to rounding), with equality to zero where R is zero by construction
    (lower wall faces); R as the plain operator gives it."""
    if case == "periodic3d":
        p = I.random_smooth(3, (7, 6, 5), seed=41, amp=0.4)
    elif case == "walls_gravity2d":
        p = I.random_smooth(2, (12, 10), seed=42, amp=0.3, bc=(I.BC_WALL, I.BC_WALL, I.BC_PERIODIC), g=(0.0, -0.5, 0.0))
    elif case == "wedge":
        p = I.spherical_wedge(nr=16, nth=12)
    else:
        p = I.random_smooth(2, (12, 10), seed=43, amp=0.3).with_options(conduct=1, chi0=0.01)
    R, A = O.spatial_operator_terms(p, p.U)
    assert np.array_equal(R, O.spatial_operator(p, p.U))
    assert (A >= 0).all()
    assert (np.abs(R) <= A * (1 + 1e-12)).all()
    N = p.ncells
    for d in range(p.nd):
        if p.bc[d] == I.BC_WALL:
            a = A[(2 + d) * N:(3 + d) * N].reshape(p.n[2], p.n[1], p.n[0])
            sl = [slice(None)] * 3
            sl[2 - d] = 0
            assert (a[tuple(sl)] == 0).all()
    # terms cancel: |R| is well below their magnitudes in most cells
    assert np.median(np.abs(R) / np.where(A > 0, A, 1.0)) < 0.5


def test_rt_hydrostatic_state_is_discrete_equilibrium():
    """Sec. 3 / Sec. 6: the unperturbed Rayleigh-Taylor state P = P0 - rho g y
    is balanced exactly by the staggered pressure gradient and the face
    gravity rho_bar g, including across the density jump (the mean of the two
    densities multiplies g)."""
    p = I.rayleigh_taylor(perturbation="none")
    R = O.spatial_operator(p, p.U)
    N = p.ncells
    assert np.abs(R[:N]).max() == 0.0
    # momentum: the balance -dp/dy + rho_bar g holds to rounding of O(1) terms
    scale = 0.1 * 2.0
    assert np.abs(R[3 * N:]).max() <= 1e-12 * scale
    # one implicit step keeps it at rest
    dt = O.cfl_dt(p, p.U, 5.0)
    U1, st, rc = O.newton_step(p, p.U, dt)
    assert rc == 0
    assert np.abs(U1 - p.U).max() <= 1e-12


# ------------------------------------------------------- consistency with PDE
def _symbolic_rhs(nd, gamma, gvec):
    """Continuous right-hand sides of Eqs. 1-3 for analytic smooth fields,
    differentiated symbolically."""
    x, y, z = sp.symbols("x y z", real=True)
    X = (x, y, z)[:nd]
    tp = 2 * sp.pi
    rho = 1 + sp.Rational(1, 5) * sp.sin(tp * x + 0.3) * sp.cos(tp * y - 0.7)
    p = 1 + sp.Rational(1, 5) * sp.cos(tp * x - 0.2) * sp.sin(2 * tp * y + 0.4)
    u = [sp.Rational(3, 10) * sp.sin(tp * y + 0.1) + sp.Rational(1, 5) * sp.cos(tp * x),
         sp.Rational(1, 4) * sp.cos(tp * x + 0.5) * sp.sin(tp * y) - sp.Rational(1, 10)]
    if nd == 3:
        rho = rho + sp.Rational(1, 10) * sp.cos(tp * z + 0.2)
        p = p + sp.Rational(1, 10) * sp.sin(tp * z - 0.6) * sp.cos(tp * x)
        u[0] = u[0] + sp.Rational(1, 10) * sp.sin(tp * z)
        u[1] = u[1] + sp.Rational(1, 10) * sp.cos(tp * z + tp * x)
        u.append(sp.Rational(1, 5) * sp.sin(tp * x + tp * y) * sp.cos(tp * z + 0.3) + sp.Rational(1, 20))
    E = p / (gamma - 1)
    drho = -sum(sp.diff(rho * u[d], X[d]) for d in range(nd))
    divu = sum(sp.diff(u[d], X[d]) for d in range(nd))
    dE = -sum(sp.diff(E * u[d], X[d]) for d in range(nd)) - p * divu
    dm = [-sum(sp.diff(rho * u[d] * u[q], X[q]) for q in range(nd)) - sp.diff(p, X[d]) + rho * gvec[d]
          for d in range(nd)]
    f = lambda e: sp.lambdify((x, y, z), e, "numpy")
    return (f(rho), f(p), [f(ui) for ui in u], f(E), f(drho), f(dE), [f(m) for m in dm])


def _sample(nd, n, fns, gamma, gvec):
    rho_f, p_f, u_f, E_f, drho_f, dE_f, dm_f = fns
    prob = I.uniform_flow(nd, n, gamma=gamma)
    prob = prob.with_options(g=tuple(gvec))
    n = prob.n
    h = [1.0 / n[d] for d in range(3)]
    cen = [(np.arange(n[d]) + 0.5) * h[d] for d in range(3)]
    face = [np.arange(n[d]) * h[d] for d in range(3)]
    if nd == 2:
        cen[2] = face[2] = np.array([0.0])

    def mesh(ax):
        Z, Y, Xx = np.meshgrid(ax[2], ax[1], ax[0], indexing="ij")
        return Xx, Y, Z

    def ev(fn, ax):
        Xx, Y, Z = mesh(ax)
        return np.broadcast_to(np.asarray(fn(Xx, Y, Z), dtype=float), Xx.shape)

    planes = [ev(rho_f, cen), ev(E_f, cen)]
    exact = [ev(drho_f, cen), ev(dE_f, cen)]
    for d in range(nd):
        ax = list(cen)
        ax[d] = face[d]
        planes.append(ev(rho_f, ax) * ev(u_f[d], ax))
        exact.append(ev(dm_f[d], ax))
    U = np.concatenate([q.reshape(-1) for q in planes])
    return prob.with_state(U), np.concatenate([q.reshape(-1) for q in exact])


@pytest.mark.parametrize("nd,sizes", [(2, (32, 64, 128)), (3, (24, 48))])
def test_truncation_error_is_second_order(nd, sizes):
    """R(U_exact) - dU/dt|_PDE -> 0 at second order (L1) for smooth fields:
    this pins every term of Eqs. 1-3 (a dropped term, a wrong sign or a
    transposed operand leaves an O(1) error), the staggering and the
    second-order upstream reconstruction of Sec. 2 (limiter clipping at
    extrema costs a little order)."""
    gamma = 1.4
    gvec = (0.3, -0.7, 0.2)
    fns = _symbolic_rhs(nd, gamma, gvec)
    errs = []
    for n1 in sizes:
        n = (n1,) * nd
        prob, exact = _sample(nd, n, fns, gamma, gvec)
        R = O.spatial_operator(prob, prob.U)
        N = prob.ncells
        errs.append([np.abs(R[v * N:(v + 1) * N] - exact[v * N:(v + 1) * N]).mean()
                     for v in range(prob.nvars)])
    errs = np.array(errs)
    order = np.log2(errs[:-1] / errs[1:])
    assert np.all(errs[-1] < 0.05), errs
    assert np.all(order > 1.0), (errs, order)      # every error shrinks fast
    assert np.all(order[-1] >= 1.6), (errs, order)   # second order (first order gives <= 1)


# ----------------------------------------------------------------- invariants
def test_conservation_form_periodic():
    """Flux form: sum R_rho = 0 and sum R_m = 0 (g = 0), and the internal
    energy changes only through the p div(u) work term."""
    p = I.random_smooth(2, (12, 10), seed=3, amp=0.3)
    R = O.spatial_operator(p, p.U)
    N = p.ncells
    rho, E, mx, my = split(p, p.U)
    assert abs(R[:N].sum()) <= 1e-13 * np.abs(R[:N]).sum()
    assert abs(R[2 * N:3 * N].sum()) <= 1e-13 * np.abs(R[2 * N:3 * N]).sum()
    assert abs(R[3 * N:].sum()) <= 1e-13 * np.abs(R[3 * N:]).sum()
    # p div(u) from face velocities u = m / rho_bar
    dx, dy = p.dx[0], p.dx[1]
    u = mx / (0.5 * (rho + np.roll(rho, 1, axis=2)))
    v = my / (0.5 * (rho + np.roll(rho, 1, axis=1)))
    div = (np.roll(u, -1, axis=2) - u) / dx + (np.roll(v, -1, axis=1) - v) / dy
    work = -((0.4 * E) * div).sum()
    assert abs(R[N:2 * N].sum() - work) <= 1e-12 * np.abs(R[N:2 * N]).sum()


def test_translation_and_axis_permutation():
    """A periodic shift of the state shifts R; swapping x and y (with m_x and
    m_y) on a square grid swaps R the same way (both code paths agree)."""
    p = I.random_smooth(2, (10, 10), seed=5, amp=0.3)
    N = p.ncells
    R = split(p, O.spatial_operator(p, p.U))
    rho, E, mx, my = split(p, p.U)
    sh = [np.roll(a, (2, -3), axis=(1, 2)) for a in (rho, E, mx, my)]
    Rs = split(p, O.spatial_operator(p, np.concatenate([a.reshape(-1) for a in sh])))
    for a, b in zip(Rs, R):
        assert np.abs(a - np.roll(b, (2, -3), axis=(1, 2))).max() <= 1e-14 * np.abs(b).max()
    tr = [np.swapaxes(a, 1, 2) for a in (rho, E, my, mx)]
    Rt = split(p, O.spatial_operator(p, np.concatenate([a.reshape(-1) for a in tr])))
    expect = [np.swapaxes(a, 1, 2) for a in (R[0], R[1], R[3], R[2])]
    for a, b in zip(Rt, expect):
        assert np.abs(a - b).max() <= 1e-14 * np.abs(b).max()


def test_3d_axis_permutation():
    p = I.random_smooth(3, (6, 6, 6), seed=6, amp=0.3)
    R = split(p, O.spatial_operator(p, p.U))
    rho, E, mx, my, mz = split(p, p.U)
    # relabel axes x' = y, y' = z, z' = x: A'[k', j', i'] = A[j', i', k']
    perm = (2, 0, 1)  # array axes are (z, y, x)
    f = lambda a: np.transpose(a, perm)
    Up = np.concatenate([f(a).reshape(-1) for a in (rho, E, my, mz, mx)])
    Rp = split(p, O.spatial_operator(p, Up))
    expect = [f(R[0]), f(R[1]), f(R[3]), f(R[4]), f(R[2])]
    for a, b in zip(Rp, expect):
        assert np.abs(a - b).max() <= 1e-14 * np.abs(b).max()


def _mirror_error(prob, U):
    N = prob.ncells
    nx = prob.n[0]
    rho, E, mx, my = split(prob, U)
    idx = (nx - np.arange(nx)) % nx
    return max(np.abs(rho - rho[:, :, ::-1]).max(), np.abs(E - E[:, :, ::-1]).max(),
               np.abs(my - my[:, :, ::-1]).max(), np.abs(mx + mx[:, :, idx]).max())


def test_rt_mirror_symmetry_is_exact():
    """Sec. 3: with mirror-consistent arithmetic the residual, the
    preconditioner and hence GMRES keep the x -> -x symmetry exactly."""
    p = I.rayleigh_taylor(nx=16, ny=48, nsteps=2)
    assert _mirror_error(p, p.U) == 0.0
    assert _mirror_error(p, O.spatial_operator(p, p.U)) == 0.0
    U, st = O.run(p)
    assert _mirror_error(p, U) == 0.0
    assert np.abs(U - p.U).max() > 1e-6


def test_rt_initial_state_scale_heights():
    """Sec. 3 quotes pressure scale heights of about 25.752 (bottom) and
    11.752 (top) for P = P0 - rho g y; the sampled cell-centre state gives
    them to within half a cell."""
    import json, os
    with open(os.path.join(os.path.dirname(__file__), "golden", "rt_scale_heights.json")) as fh:
        gold = json.load(fh)
    p = I.rayleigh_taylor()
    rho, E, _, _ = split(p, p.U)
    P = 0.4 * E
    Hb = P[0, 0, 0] / (rho[0, 0, 0] * 0.1)
    Ht = P[0, -1, 0] / (rho[0, -1, 0] * 0.1)
    h = p.dx[1]
    # d(P / rho g)/dy = -1 inside each layer: half a cell moves H by h/2
    assert abs(Hb - gold["bottom"]) <= h
    assert abs(Ht - gold["top"]) <= h
