"""Seeded synthetic problem setups (initial conditions and grid descriptions).

This module only samples the initial-condition formulas of the test problems
on the staggered grid; it holds none of the solver's arithmetic, so both the
CUDA library's tests and the CPU oracle take their inputs from here.

State layout (shared by every consumer): ``nv`` planes of ``N = nx*ny*nz``
float64 values, x fastest, in the order rho, E = rho*e (internal energy per
volume), m_x, m_y[, m_z].  ``m_d[c]`` sits on the lower d-face of cell ``c``.
On a wall direction the lower wall face of the first cell layer is stored
(always zero); the upper wall face is implicit.  Momenta are the analytic
density at the face position times the analytic velocity there.

Problems (paper sections):
  * Rayleigh-Taylor, Sec. 3: box [-0.25,0.25]x[-0.75,0.75], rho = 2 above
    y = 0 and 1 below, g = 0.1 downwards, P = P0 - rho g y with P0 = 2.5,
    gamma = 1.4, periodic in x, reflecting walls in y with hydrostatic ghost
    cells.  Velocity seed either the 64x192 benchmark form
    v_y = 0.01 (1 + cos 4 pi x)(1 + cos 3 pi y)/4 or the paper's Eq. 7 form
    v_y = 0.0025 (1 + cos 4 pi x)(1 + cos 4 pi y / 3).
  * Kelvin-Helmholtz, Sec. 4 (smooth shear layers): periodic unit box,
    gamma = 5/3, u_x = tanh((y-0.25)/0.05) - tanh((y-0.75)/0.05) - 1 (zero
    net momentum), rho = 1 + (1/2)(tanh((y-0.25)/0.05) - tanh((y-0.75)/0.05)),
    P0 = 120 so that the flow Mach number is 0.1, seeded mode
    u_y = 0.01 sin(4 pi x) exp(-(y-0.25)^2/0.01) and uniform noise of
    amplitude 1e-4 on both components (Philox counter-based generator).
  * Taylor-Green vortex, Sec. 5: periodic [0, 2 pi]^3, gamma = 5/3, rho0 = 1,
    u0 = 1, u = sin x cos y cos z, v = -cos x sin y cos z, w = 0,
    p = p0 + rho0 u0^2 (cos 2x + cos 2y)(cos 2z + 2)/16 with p0 chosen for a
    Mach number of 0.1 (p0 = rho0 u0^2 / (gamma M^2) = 60).
"""
from __future__ import annotations

import dataclasses
import math
from typing import Optional

import numpy as np

BC_PERIODIC = 0
BC_WALL = 1
WALL_MIRROR = 0
WALL_HSE = 1
PC_NONE = 0
PC_ACOUSTIC = 1
GEOM_CARTESIAN = 0
GEOM_SPHERICAL = 1


@dataclasses.dataclass
class Problem:
    """Grid, physics, solver options and an initial state."""

    name: str
    nd: int
    n: tuple            # (nx, ny, nz); nz = 1 in 2-D
    x0: tuple           # lower corner
    length: tuple       # box edge lengths
    bc: tuple           # BC_* per direction
    wall_scalar: tuple  # WALL_* per direction (only read on walls)
    gamma: float
    g: tuple            # constant gravity vector
    U: np.ndarray       # initial state, shape (nv * N,)
    cfl: float = 1.0                   # CFL_hydro limit of the time step
    nsteps: int = 1
    dt_max: float = 0.0
    cfl_adv: float = 0.0               # advective CFL limit (0: none)
    cfl_rad: float = 0.0               # radiative CFL limit (0: none)
    restart: int = 30
    max_restarts: int = 10
    gmres_rtol: float = 1e-1
    newton_max: int = 12
    newton_tol: float = 1e-8
    precond: int = PC_ACOUSTIC
    sweeps: int = 16
    max_halvings: int = 4
    rho_L: float = 1.0   # light / heavy densities for the mixing height
    rho_H: float = 2.0
    # geometry and radiative diffusion
    geometry: int = GEOM_CARTESIAN      # GEOM_SPHERICAL: 2-D (r, theta), direction 0 = r
    gface: Optional[np.ndarray] = None  # radial gravity on the n[0]+1 r-faces (spherical)
    conduct: int = 0                    # div(chi grad T) with chi = chi0 T^6.5 / rho^2
    chi0: float = 0.0
    flux_wall: tuple = (0, 0, 0)        # walls with the prescribed flux chi dT/dn = lum (/ r^2)
    lum: float = 0.0
    # passive scalars (Sec. 2.2): partial densities q_i = c_i rho, ns planes of N
    q: Optional[np.ndarray] = None
    scalar_enforce: int = 0             # 1: the Newton test also checks the scalar corrections

    @property
    def nscalars(self) -> int:
        return 0 if self.q is None else int(self.q.size // self.ncells)

    @property
    def ncells(self) -> int:
        return int(self.n[0] * self.n[1] * self.n[2])

    @property
    def nvars(self) -> int:
        return 2 + self.nd

    @property
    def dx(self) -> tuple:
        return tuple(self.length[d] / self.n[d] for d in range(3))

    def with_state(self, U: np.ndarray) -> "Problem":
        return dataclasses.replace(self, U=np.ascontiguousarray(U, dtype=np.float64))

    def with_options(self, **kw) -> "Problem":
        return dataclasses.replace(self, **kw)


def _axes(n, x0, length):
    """Cell-centre and lower-face coordinates per direction."""
    cen, face = [], []
    for d in range(3):
        h = length[d] / n[d]
        cen.append(x0[d] + (np.arange(n[d]) + 0.5) * h)
        face.append(x0[d] + np.arange(n[d]) * h)
    return cen, face


def _mesh(ax, ay, az):
    """Arrays indexed [k, j, i] (x fastest when flattened)."""
    Z, Y, X = np.meshgrid(az, ay, ax, indexing="ij")
    return X, Y, Z


def _pack(nd, rho, E, moms):
    planes = [rho, E] + list(moms[:nd])
    return np.ascontiguousarray(np.concatenate([p.reshape(-1) for p in planes]), dtype=np.float64)


def rayleigh_taylor(nx: int = 64, ny: int = 192, perturbation: str = "benchmark",
                    cfl: float = 5.0, nsteps: int = 10, scalars: bool = False) -> Problem:
    """Single-mode Rayleigh-Taylor instability (Sec. 3); with `scalars`, the
    two marker scalars of Sec. 3: (c_1, c_2) = (1, 0) where the cell centre
    has y <= 0 and (0, 1) above, as partial densities c_i rho."""
    gamma, gmag, P0 = 1.4, 0.1, 2.5
    n = (nx, ny, 1)
    x0, length = (-0.25, -0.75, 0.0), (0.5, 1.5, 1.0)
    cen, face = _axes(n, x0, length)

    def dens(y):
        return np.where(y > 0.0, 2.0, 1.0)

    Xc, Yc, _ = _mesh(cen[0], cen[1], cen[2])
    rho = dens(Yc)
    p = P0 - rho * gmag * Yc
    E = p / (gamma - 1.0)
    mx = np.zeros_like(rho)
    Xf, Yf, _ = _mesh(cen[0], face[1], cen[2])
    if perturbation == "benchmark":
        vy = 0.01 * (1.0 + np.cos(4 * np.pi * Xf)) * (1.0 + np.cos(3 * np.pi * Yf)) / 4.0
    elif perturbation == "paper":
        vy = 0.0025 * (1.0 + np.cos(4 * np.pi * Xf)) * (1.0 + np.cos(4 * np.pi * Yf / 3.0))
    elif perturbation == "none":
        vy = np.zeros_like(Yf)
    else:
        raise ValueError(perturbation)
    my = dens(Yf) * vy
    my[:, 0, :] = 0.0  # lower wall face
    U = _pack(2, rho, E, [mx, my])
    q = None
    if scalars:
        c1 = np.where(Yc <= 0.0, 1.0, 0.0)
        q = np.concatenate([(c1 * rho).ravel(), ((1.0 - c1) * rho).ravel()])
    return Problem("rayleigh_taylor", 2, n, x0, length, (BC_PERIODIC, BC_WALL, BC_PERIODIC),
                   (WALL_MIRROR, WALL_HSE, WALL_MIRROR), gamma, (0.0, -gmag, 0.0), U,
                   cfl=cfl, nsteps=nsteps, rho_L=1.0, rho_H=2.0, q=q)


def rt_paper(nx: int = 100, ny: int = 300, nsteps: int = 100, scalars: bool = True) -> Problem:
    """The paper's own Rayleigh-Taylor runs (Sec. 3): the perturbation of its
    Eq. for the initial vertical velocity, grids of aspect ratio one (100x300,
    300x900), CFL_hydro fixed at 0.8, the unpreconditioned JFNK solver, and
    the two marker scalars."""
    p = rayleigh_taylor(nx=nx, ny=ny, perturbation="paper", cfl=0.8, nsteps=nsteps, scalars=scalars)
    return dataclasses.replace(p, name="rt_paper", precond=PC_NONE)


def kelvin_helmholtz(n: int = 512, seed: int = 2, noise: float = 1e-4, cfl: float = 10.0,
                     nsteps: int = 200, ny: Optional[int] = None) -> Problem:
    """Smooth two-shear-layer Kelvin-Helmholtz setup (Sec. 4)."""
    gamma, P0, a = 5.0 / 3.0, 120.0, 0.05
    nyy = n if ny is None else ny
    shape = (n, nyy, 1)
    x0, length = (0.0, 0.0, 0.0), (1.0, 1.0, 1.0)
    cen, face = _axes(shape, x0, length)

    def prof(y):
        return np.tanh((y - 0.25) / a) - np.tanh((y - 0.75) / a)

    def dens(y):
        return 1.0 + 0.5 * prof(y)

    Xc, Yc, _ = _mesh(cen[0], cen[1], cen[2])
    rho = dens(Yc)
    E = np.full_like(rho, P0 / (gamma - 1.0))
    rng = np.random.Generator(np.random.Philox(seed))
    nz = rng.uniform(-noise, noise, size=(2,) + rho.shape)
    Xu, Yu, _ = _mesh(face[0], cen[1], cen[2])
    ux = prof(Yu) - 1.0 + nz[0]
    Xv, Yv, _ = _mesh(cen[0], face[1], cen[2])
    uy = 0.01 * np.sin(4 * np.pi * Xv) * np.exp(-((Yv - 0.25) ** 2) / 0.01) + nz[1]
    U = _pack(2, rho, E, [dens(Yu) * ux, dens(Yv) * uy])
    # solver settings of this setup (measured on the GPU: fewest ms per step)
    return Problem("kelvin_helmholtz", 2, shape, x0, length, (BC_PERIODIC,) * 3, (WALL_MIRROR,) * 3,
                   gamma, (0.0, 0.0, 0.0), U, cfl=cfl, nsteps=nsteps, rho_L=1.0, rho_H=2.0,
                   gmres_rtol=0.2, sweeps=24)


def taylor_green(n: int = 128, mach: float = 0.1, cfl: float = 20.0, nsteps: int = 100) -> Problem:
    """Taylor-Green vortex (Sec. 5)."""
    gamma, rho0, u0 = 5.0 / 3.0, 1.0, 1.0
    p0 = rho0 * u0 * u0 / (gamma * mach * mach)
    shape = (n, n, n)
    x0, length = (0.0, 0.0, 0.0), (2 * np.pi,) * 3
    cen, face = _axes(shape, x0, length)
    X, Y, Z = _mesh(cen[0], cen[1], cen[2])
    rho = np.full(X.shape, rho0)
    p = p0 + rho0 * u0 * u0 * (np.cos(2 * X) + np.cos(2 * Y)) * (np.cos(2 * Z) + 2.0) / 16.0
    E = p / (gamma - 1.0)
    Xu, Yu, Zu = _mesh(face[0], cen[1], cen[2])
    Xv, Yv, Zv = _mesh(cen[0], face[1], cen[2])
    mx = rho0 * u0 * np.sin(Xu) * np.cos(Yu) * np.cos(Zu)
    my = -rho0 * u0 * np.cos(Xv) * np.sin(Yv) * np.cos(Zv)
    mz = np.zeros_like(rho)
    U = _pack(3, rho, E, [mx, my, mz])
    # solver settings of this setup (measured on the GPU: fewest ms per step)
    return Problem("taylor_green", 3, shape, x0, length, (BC_PERIODIC,) * 3, (WALL_MIRROR,) * 3,
                   gamma, (0.0, 0.0, 0.0), U, cfl=cfl, nsteps=nsteps, sweeps=24)


def random_smooth(nd: int, n: tuple, seed: int, amp: float = 0.05, bc=None, wall_scalar=None,
                  gamma: float = 1.4, g=(0.0, 0.0, 0.0), length=None) -> Problem:
    """A smooth random state (a few low Fourier modes per field) for parity tests.

    rho and p are positive and O(1); velocities are O(amp * c_s).  Wall faces
    are zeroed."""
    rng = np.random.Generator(np.random.Philox(seed))
    n = tuple(n) + (1,) * (3 - len(n))
    length = tuple(length) if length is not None else (1.0, 1.0, 1.0)
    x0 = (0.0, 0.0, 0.0)
    bc = tuple(bc) if bc is not None else (BC_PERIODIC,) * 3
    wall_scalar = tuple(wall_scalar) if wall_scalar is not None else (WALL_MIRROR,) * 3
    cen, face = _axes(n, x0, length)

    def field(ax, ay, az, base, scale):
        X, Y, Z = _mesh(ax, ay, az)
        f = np.full(X.shape, base, dtype=np.float64)
        for _ in range(4):
            k = rng.integers(1, 4, size=3)
            if nd == 2:
                k[2] = 0
            ph = rng.uniform(0, 2 * np.pi, size=3)
            a = rng.uniform(-1, 1)
            f = f + scale * a * (np.sin(2 * np.pi * k[0] * X / length[0] + ph[0])
                                 * np.cos(2 * np.pi * k[1] * Y / length[1] + ph[1])
                                 * np.cos(2 * np.pi * k[2] * Z / length[2] + ph[2]))
        return f

    rho = field(cen[0], cen[1], cen[2], 1.0, 0.15)
    p = field(cen[0], cen[1], cen[2], 1.0, 0.15)
    E = p / (gamma - 1.0)
    cs = math.sqrt(gamma)
    moms = []
    for d in range(nd):
        ax = [cen[0], cen[1], cen[2]]
        ax[d] = face[d]
        u = field(ax[0], ax[1], ax[2], 0.0, amp * cs)
        m = 1.0 * u
        if bc[d] == BC_WALL:
            sl = [slice(None)] * 3
            sl[2 - d] = 0
            m[tuple(sl)] = 0.0
        moms.append(m)
    U = _pack(nd, rho, E, moms)
    return Problem("random_smooth", nd, n, x0, length, bc, wall_scalar, gamma, tuple(g), U)


def uniform_flow(nd: int, n: tuple, rho: float = 1.3, p: float = 2.0, u=(0.3, -0.2, 0.1),
                 gamma: float = 1.4, length=None) -> Problem:
    """Constant density, pressure and velocity in a periodic box."""
    n = tuple(n) + (1,) * (3 - len(n))
    length = tuple(length) if length is not None else (1.0, 1.0, 1.0)
    shape = (n[2], n[1], n[0])
    planes = [np.full(shape, rho), np.full(shape, p / (gamma - 1.0))]
    for d in range(nd):
        planes.append(np.full(shape, rho * u[d]))
    U = _pack(nd, planes[0], planes[1], planes[2:])
    return Problem("uniform_flow", nd, n, (0.0, 0.0, 0.0), length, (BC_PERIODIC,) * 3,
                   (WALL_MIRROR,) * 3, gamma, (0.0, 0.0, 0.0), U)


def config_problem(index: int, **kw) -> Problem:
    """The benchmark workloads by number: 0 RT 64x192 (10 steps, CFL 5),
    1 KH 512^2 (200 steps, CFL 10), 2 TGV 128^3 (100 steps, CFL 20)."""
    if index == 0:
        return rayleigh_taylor(**kw)
    if index == 1:
        return kelvin_helmholtz(**kw)
    if index == 2:
        return taylor_green(**kw)
    raise ValueError(index)


# ------------------------------------------------------------ spherical wedge
def lane_emden(n: float = 3.0, h: float = 1e-4):
    """Lane-Emden solution theta(xi) of index n by classical RK4 (series start
    at small xi).  Returns (xi, theta, dtheta) arrays up to the first zero and
    the zero xi_1 (interpolated)."""
    def f(x, y):
        return np.array([y[1], -y[0] ** n - 2.0 * y[1] / x]) if y[0] > 0 else np.array([y[1], -2.0 * y[1] / x])
    x = 1e-6
    y = np.array([1.0 - x * x / 6.0, -x / 3.0])
    xs, ts, ds = [0.0], [1.0], [0.0]
    while y[0] > 0:
        k1 = f(x, y)
        k2 = f(x + h / 2, y + h / 2 * k1)
        k3 = f(x + h / 2, y + h / 2 * k2)
        k4 = f(x + h, y + h * k3)
        yn = y + h / 6 * (k1 + 2 * k2 + 2 * k3 + k4)
        if yn[0] <= 0:
            frac = y[0] / (y[0] - yn[0])
            xi1 = x + frac * h
            xs.append(xi1)
            ts.append(0.0)
            ds.append(y[1] + frac * (yn[1] - y[1]))
            return np.array(xs), np.array(ts), np.array(ds), xi1
        x += h
        y = yn
        xs.append(x)
        ts.append(y[0])
        ds.append(y[1])


def spherical_wedge(nr: int = 256, nth: int = 128, seed: int = 5, noise: float = 1e-6, cfl: float = 100.0,
                    nsteps: int = 500, cfl_rad: float = 500.0, gamma: float = 5.0 / 3.0) -> Problem:
    """2-D spherical-wedge radiative hydrostatic test (Sec. 6 setup, polytrope
    background in code units).

    A Lane-Emden n = 3 polytrope with central density and temperature 1
    (p = rho T, G = 1, so K = 1 and the length unit alpha = 1/sqrt(pi))
    gives the radial gravity g(r) = -M(r)/r^2 on the r-faces and seeds the
    first cell.  Outward from there each cell is set so that the discrete
    balance across the face between it and the previous cell holds exactly:
    p_j - p_{j-1} = dr g_f (rho_j + rho_{j-1})/2 (hydrostatic) and
    r_f^2 chi_f (T_j - T_{j-1})/dr = Lambda (constant luminosity), chi_f the
    mean of the two cells' chi = chi0 T^6.5/rho^2, Lambda from the
    polytrope's temperature gradient at the first face.  chi0 makes the
    radiative CFL number max(D dt / dx^2), D = chi/(rho c_v), equal cfl_rad
    at dt = cfl x the acoustic limit on the polytrope.  Domain r in
    [0.1, 0.9] R, theta in [pi/4, 3 pi/4] (periodic); radial walls with
    hydrostatic ghosts and the prescribed flux Lambda/r^2; relative density
    noise of 1e-6 (Philox, seed 5); fluid at rest.
    """
    xs, ts, ds, xi1 = lane_emden(3.0)
    alpha = 1.0 / math.sqrt(math.pi)
    R = xi1 * alpha
    r0, r1 = 0.1 * R, 0.9 * R
    th0, th1 = math.pi / 4, 3 * math.pi / 4
    dr, dth = (r1 - r0) / nr, (th1 - th0) / nth

    def poly(r):
        xi = r / alpha
        t = np.interp(xi, xs, ts)
        dt_ = np.interp(xi, xs, ds)
        return t, dt_

    rf = r0 + np.arange(nr + 1) * dr
    tf, dtf = poly(rf)
    xi_f = rf / alpha
    mass = 4 * math.pi * alpha ** 3 * (-(xi_f ** 2) * dtf)
    gface = -mass / rf ** 2
    rc = r0 + (np.arange(nr) + 0.5) * dr
    tc, _ = poly(rc)
    rho_p, T_p = tc ** 3, tc
    cv = 1.0 / (gamma - 1.0)
    cs = np.sqrt(gamma * T_p)
    h_min = np.minimum(dr, rc * dth)
    dt_ac = cfl / np.max(cs / h_min)
    D_over = T_p ** 6.5 / rho_p ** 2 / (rho_p * cv) / h_min ** 2
    chi0 = cfl_rad / (dt_ac * np.max(D_over))

    def chi(rho, T):
        return chi0 * T ** 6.5 / rho ** 2

    # Lambda from the polytrope's temperature gradient at the first interior face
    t1, dt1 = poly(rf[1])
    Lam = rf[1] ** 2 * chi(t1 ** 3, t1) * dt1 / alpha
    rho = np.empty(nr)
    T = np.empty(nr)
    rho[0], T[0] = rho_p[0], T_p[0]
    for j in range(1, nr):
        gf, r_ = gface[j], rf[j]
        x = np.array([rho_p[j] / rho_p[j - 1] * rho[j - 1], T[j - 1] + Lam * dr / (r_ ** 2 * chi(rho[j - 1], T[j - 1]))])
        for _ in range(60):
            ro, Tn = x
            f1 = ro * Tn - rho[j - 1] * T[j - 1] - dr * gf * (ro + rho[j - 1]) / 2
            cf = 0.5 * (chi(ro, Tn) + chi(rho[j - 1], T[j - 1]))
            f2 = r_ ** 2 * cf * (Tn - T[j - 1]) / dr - Lam
            dcr = 0.5 * chi(ro, Tn) * (-2.0 / ro)
            dct = 0.5 * chi(ro, Tn) * (6.5 / Tn)
            J = np.array([[Tn - dr * gf / 2, ro],
                          [r_ ** 2 * dcr * (Tn - T[j - 1]) / dr, r_ ** 2 * (dct * (Tn - T[j - 1]) + cf) / dr]])
            step = np.linalg.solve(J, -np.array([f1, f2]))
            x = x + step
            if np.all(np.abs(step) <= 1e-15 * np.abs(x)):
                break
        rho[j], T[j] = x
    if np.any(rho <= 0) or np.any(T <= 0):
        raise RuntimeError("radiative-equilibrium march left the physical range")
    shape = (nr, nth, 1)
    rho2 = np.repeat(rho[None, :], nth, axis=0)
    T2 = np.repeat(T[None, :], nth, axis=0)
    rng = np.random.Generator(np.random.Philox(seed))
    rho2 = rho2 * (1.0 + noise * rng.uniform(-1.0, 1.0, size=rho2.shape))
    # the noise perturbs density at fixed pressure (temperature compensates)
    E = (rho[None, :] * T[None, :]).repeat(nth, axis=0) / (gamma - 1.0)
    z = np.zeros_like(rho2)
    U = _pack(2, rho2.reshape(1, nth, nr), E.reshape(1, nth, nr), [z.reshape(1, nth, nr), z.reshape(1, nth, nr)])
    return Problem("spherical_wedge", 2, shape, (r0, th0, 0.0), (r1 - r0, th1 - th0, 1.0),
                   (BC_WALL, BC_PERIODIC, BC_PERIODIC), (WALL_HSE, WALL_MIRROR, WALL_MIRROR), gamma,
                   (0.0, 0.0, 0.0), U, cfl=cfl, nsteps=nsteps, geometry=GEOM_SPHERICAL, gface=gface,
                   conduct=1, chi0=float(chi0), flux_wall=(1, 0, 0), lum=float(Lam))
