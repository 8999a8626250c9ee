"""Closed-form pins of the reconstruction in the oracle's R(U) (Sec. 2:
upstream linear extrapolation with the van Leer limiter).

The truncation-order pins elsewhere pass for any second-order TVD limiter and
do not see which side is upstream.  Here R is evaluated on piecewise-linear,
kinked profiles where the van Leer slope vL(a, b) = 2ab/(a+b) (ab > 0, else
0), minmod, MC and superbee all give different face values, and where the
upstream and downstream cells give different fluxes.  Every expected number
below is worked out by hand from the definitions, with the arithmetic in the
comments; `test_profiles_discriminate` shows that each plausible mistake
(another limiter, a halved slope, the downstream cell) moves at least one
value far outside the tolerance.

Profile w (cell index 0..7, periodic): 1, 1, 2, 4, 4, 4, 3, 1.
One-sided differences a_j = w_j - w_{j-1}, b_j = w_{j+1} - w_j:
  j : 0   1   2   3   4   5   6    7
  a : 0   0   1   2   0   0  -1   -2
  b : 0   1   2   0   0  -1  -2    0
van Leer slopes s_j (nonzero only where a b > 0):
  s_2 = 2*1*2/(1+2) = 4/3,  s_6 = 2*(-1)*(-2)/(-3) = -4/3, all others 0.
"""
from fractions import Fraction as Fr

import numpy as np

from oracle import oracle as O
from paper_1610_10053_gb300 import inputs as I

W = [1, 1, 2, 4, 4, 4, 3, 1]
TOL = 1e-13


def _problem(n, U):
    return I.Problem("limiter_pin", 2, n, (0.0, 0.0, 0.0), (1.0, 1.0, 1.0), (I.BC_PERIODIC,) * 3,
                     (I.WALL_MIRROR,) * 3, 1.4, (0.0, 0.0, 0.0), np.ascontiguousarray(U, dtype=np.float64))


def _planes(ny, nx, rho, E, mx, my):
    return np.concatenate([np.asarray(a, dtype=np.float64).reshape(ny, nx).ravel() for a in (rho, E, mx, my)])


def _mass_case(u0):
    """rho = w along x (8 cells, dx = 1/8), uniform along y (4 cells);
    p = 1; face velocity u0 everywhere (m_x = u0 times the mean density of
    the face's two cells, so m / rho_bar = u0 exactly); m_y = 0."""
    nx, ny = 8, 4
    rho = np.tile(np.array(W, dtype=np.float64), (ny, 1))
    rbar = 0.5 * (np.roll(rho, 1, axis=1) + rho)
    E = np.full_like(rho, 1.0 / 0.4)
    return _problem((nx, ny, 1), _planes(ny, nx, rho, E, u0 * rbar, np.zeros_like(rho)))


def test_mass_flux_upstream_van_leer_positive_velocity():
    """u0 = +1/2: the face value on face i (lower face of cell i) comes from
    cell i-1, rho*_i = w_{i-1} + s_{i-1}/2:
      faces 0..7: 1, 1, 1, 2 + 2/3 = 8/3, 4, 4, 4, 3 - 2/3 = 7/3.
    R_rho[i] = -u0 (rho*_{i+1} - rho*_i)/dx = -4 (rho*_{i+1} - rho*_i):
      0, 0, -4(5/3), -4(4/3), 0, 0, -4(-5/3), -4(-4/3)."""
    p = _mass_case(0.5)
    R = O.spatial_operator(p, p.U)
    N = p.ncells
    exp = [0, 0, Fr(-20, 3), Fr(-16, 3), 0, 0, Fr(20, 3), Fr(16, 3)]
    got = R[:N].reshape(4, 8)
    for row in got:
        assert np.abs(row - np.array([float(x) for x in exp])).max() <= TOL * 8


def test_mass_flux_upstream_van_leer_negative_velocity():
    """u0 = -1/2: face i takes cell i, rho*_i = w_i - s_i/2:
      faces 0..7: 1, 1, 2 - 2/3 = 4/3, 4, 4, 4, 3 + 2/3 = 11/3, 1.
    R_rho[i] = +4 (rho*_{i+1} - rho*_i):
      0, 4(1/3), 4(8/3), 0, 0, 4(-1/3), 4(-8/3), 0."""
    p = _mass_case(-0.5)
    R = O.spatial_operator(p, p.U)
    N = p.ncells
    exp = [0, Fr(4, 3), Fr(32, 3), 0, 0, Fr(-4, 3), Fr(-32, 3), 0]
    got = R[:N].reshape(4, 8)
    for row in got:
        assert np.abs(row - np.array([float(x) for x in exp])).max() <= TOL * 11


def _momentum_case(sign):
    """rho = 1, p = 1 everywhere; x-face velocity u_i = sign * w_i / 10 on
    face i (uniform along y); m_y = 0.  The mass flux on x-faces is u_i
    exactly (every density slope is 0), the pressure gradient and every
    y-flux vanish, so R_mx is the centre-flux difference alone."""
    nx, ny = 8, 4
    u = sign * np.tile(np.array(W, dtype=np.float64), (ny, 1)) / 10.0
    one = np.ones((ny, nx))
    return _problem((nx, ny, 1), _planes(ny, nx, one, one / 0.4, u, np.zeros_like(one)))


def test_momentum_centre_flux_positive_velocity():
    """Centre c lies between faces c and c+1.  Mass flux there
    fm_c = (u_c + u_{c+1})/2 = 0.1 (1, 1.5, 3, 4, 4, 3.5, 2, 1) > 0, so u_x
    is extrapolated from face c: us_c = u_c + su_c/2 with su the van Leer
    slope of u along x, = 0.1 (1, 1, 8/3, 4, 4, 4, 7/3, 1).
    Phi_c = fm_c us_c = 0.01 (1, 1.5, 8, 16, 16, 14, 14/3, 1) and
    R_mx[c] = -(Phi_c - Phi_{c-1})/dx = -8 (Phi_c - Phi_{c-1}):
      0, -0.04, -0.52, -0.64, 0, 0.16, 0.08 (28/3), 0.08 (11/3)."""
    p = _momentum_case(1.0)
    R = O.spatial_operator(p, p.U)
    N = p.ncells
    exp = [0.0, -0.04, -0.52, -0.64, 0.0, 0.16, 0.08 * 28 / 3, 0.08 * 11 / 3]
    got = R[2 * N:3 * N].reshape(4, 8)
    for row in got:
        assert np.abs(row - np.array(exp)).max() <= TOL
    assert np.abs(R[3 * N:]).max() <= TOL  # R_my: nothing moves along y


def test_momentum_centre_flux_negative_velocity():
    """u_i = -w_i/10: fm_c = -0.1 (1, 1.5, 3, 4, 4, 3.5, 2, 1) < 0, so u_x
    comes from face c+1: us_c = u_{c+1} - su_{c+1}/2
      = -0.1 (1, 2 - 2/3, 4, 4, 4, 3 + 2/3, 1, 1) = -0.1 (1, 4/3, 4, 4, 4, 11/3, 1, 1).
    Phi_c = 0.01 (1, 2, 12, 16, 16, 77/6, 2, 1) and R_mx[c] = -8 (Phi_c - Phi_{c-1}):
      0, -0.08, -0.8, -0.32, 0, 0.08 (19/6), 0.08 (65/6), 0.08."""
    p = _momentum_case(-1.0)
    R = O.spatial_operator(p, p.U)
    N = p.ncells
    exp = [0.0, -0.08, -0.8, -0.32, 0.0, 0.08 * 19 / 6, 0.08 * 65 / 6, 0.08]
    got = R[2 * N:3 * N].reshape(4, 8)
    for row in got:
        assert np.abs(row - np.array(exp)).max() <= TOL


def _edge_case(v0):
    """rho = 1, p = 1; x-face velocity u_j = w_j / 10 on every x-face of row j
    (8 rows, dy = 1/8; 4 columns); y-face velocity v0 everywhere.  Along x
    nothing varies, so R_mx is the difference of the edge fluxes
    Psi_j = v0 us_j (m_x carried across the lower y-face of row j)."""
    nx, ny = 4, 8
    u = np.repeat(np.array(W, dtype=np.float64)[:, None], nx, axis=1) / 10.0
    one = np.ones((ny, nx))
    return _problem((nx, ny, 1), _planes(ny, nx, one, one / 0.4, u, v0 * one))


def test_momentum_edge_flux_upstream():
    """v0 = +1/2: the edge value of u_x comes from row j-1,
    us_j = u_{j-1} + su_{j-1}/2 = 0.1 (1, 1, 1, 8/3, 4, 4, 4, 7/3), and
    R_mx[j] = -(Psi_{j+1} - Psi_j)/dy = -8 v0 (us_{j+1} - us_j)
            = -0.4 (0, 0, 5/3, 4/3, 0, 0, -5/3, -4/3).
    v0 = -1/2: from row j, us_j = u_j - su_j/2 = 0.1 (1, 1, 4/3, 4, 4, 4, 11/3, 1),
    R_mx[j] = +0.4 (0, 1/3, 8/3, 0, 0, -1/3, -8/3, 0)."""
    for v0, exp in ((0.5, [0.0, 0.0, -0.4 * 5 / 3, -0.4 * 4 / 3, 0.0, 0.0, 0.4 * 5 / 3, 0.4 * 4 / 3]),
                    (-0.5, [0.0, 0.4 / 3, 0.4 * 8 / 3, 0.0, 0.0, -0.4 / 3, -0.4 * 8 / 3, 0.0])):
        p = _edge_case(v0)
        R = O.spatial_operator(p, p.U)
        N = p.ncells
        got = R[2 * N:3 * N].reshape(8, 4)
        for col in got.T:
            assert np.abs(col - np.array(exp)).max() <= TOL, v0
        assert np.abs(R[3 * N:]).max() <= TOL


def test_profiles_discriminate():
    """The hand-computed mass-flux values above differ by far more than the
    tolerance from what minmod, MC, superbee, a halved slope or the
    downstream cell would give on the same profile, so a wrong limiter or a
    wrong upwind side in the oracle cannot pass these pins."""
    def minmod(a, b):
        return 0 if a * b <= 0 else (min(abs(a), abs(b)) * (1 if a > 0 else -1))

    limiters = {
        "van_leer": lambda a, b: Fr(2 * a * b, a + b) if a * b > 0 else Fr(0),
        "minmod": lambda a, b: Fr(minmod(a, b)),
        "mc": lambda a, b: Fr(0) if a * b <= 0 else (1 if a > 0 else -1) * min(2 * abs(Fr(a)), 2 * abs(Fr(b)),
                                                                         abs(Fr(a + b, 2))),
        "superbee": lambda a, b: Fr(0) if a * b <= 0 else (1 if a > 0 else -1) * max(
            min(2 * abs(Fr(a)), abs(Fr(b))), min(abs(Fr(a)), 2 * abs(Fr(b)))),
    }

    def r_rho(limiter, upstream=True, half=Fr(1, 2)):
        n = len(W)
        s = [limiter(W[j] - W[j - 1], W[(j + 1) % n] - W[j]) for j in range(n)]
        face = []
        for i in range(n):  # u0 = +1/2
            j = i - 1 if upstream else i
            face.append(W[j] + (half if upstream else -half) * s[j])
        return [-4 * (face[(i + 1) % n] - face[i]) for i in range(n)]

    ref = r_rho(limiters["van_leer"])
    assert ref == [0, 0, Fr(-20, 3), Fr(-16, 3), 0, 0, Fr(20, 3), Fr(16, 3)]  # the pinned values
    wrong = [r_rho(limiters[k]) for k in ("minmod", "mc", "superbee")]
    wrong.append(r_rho(limiters["van_leer"], half=Fr(1, 4)))
    wrong.append(r_rho(limiters["van_leer"], upstream=False))
    for w in wrong:
        assert max(abs(float(x - y)) for x, y in zip(w, ref)) >= 0.1
