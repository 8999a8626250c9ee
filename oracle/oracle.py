"""ORACLE - TEST INFRASTRUCTURE ONLY.

ctypes front end of ``music_oracle.c``, the plain FP64 CPU restatement of the
paper's implicit step (Sec. 2).  Only the tests, ``__graft_entry__.smoke`` and
the benchmark's CPU baseline may import this module.  It never imports the
CUDA package and the CUDA package never imports it; both take their inputs
from ``paper_1610_10053_gb300.inputs`` only.
"""
from __future__ import annotations

import contextlib
import ctypes
import os
import subprocess

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(BUILD, "liboracle.so")
# the same source built with -fopenmp: its independent per-cell loops run on
# all host cores (the multi-core CPU baseline); every reduction stays serial
LIB_OMP = os.path.join(BUILD, "liboracle_omp.so")
SRC = [os.path.join(HERE, "music_oracle.c"), os.path.join(HERE, "residual_body.h")]

_dbl_p = ctypes.POINTER(ctypes.c_double)


class OrGrid(ctypes.Structure):
    _fields_ = [
        ("nd", ctypes.c_int), ("n", ctypes.c_int * 3), ("dx", ctypes.c_double * 3),
        ("x0", ctypes.c_double * 3), ("bc", ctypes.c_int * 3), ("wall_scalar", ctypes.c_int * 3),
        ("gamma", ctypes.c_double), ("g", ctypes.c_double * 3),
        ("restart", ctypes.c_int), ("max_restarts", ctypes.c_int), ("gmres_rtol", ctypes.c_double),
        ("newton_max", ctypes.c_int), ("newton_tol", ctypes.c_double), ("precond", ctypes.c_int),
        ("sweeps", ctypes.c_int), ("max_halvings", ctypes.c_int),
        ("geom", ctypes.c_int), ("gface", ctypes.POINTER(ctypes.c_double)), ("conduct", ctypes.c_int),
        ("chi0", ctypes.c_double), ("flux_wall", ctypes.c_int * 3), ("lum", ctypes.c_double),
    ]


class OrStepStats(ctypes.Structure):
    _fields_ = [
        ("dt", ctypes.c_double), ("newton_its", ctypes.c_int), ("gmres_its", ctypes.c_int),
        ("halvings", ctypes.c_int), ("gmres_failures", ctypes.c_int), ("fnorm0", ctypes.c_double),
        ("fnorm", ctypes.c_double), ("max_drho", ctypes.c_double),
    ]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


def _compile(out, extra):
    if os.path.exists(out) and os.path.getmtime(out) >= max(os.path.getmtime(s) for s in SRC):
        return
    tmp = out + ".tmp%d" % os.getpid()
    cmd = ["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared", "-std=gnu11"] + extra + [
        "-o", tmp, SRC[0], "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, out)


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (-O2, no FMA contraction, no fast-math),
    and its OpenMP build where the compiler supports -fopenmp."""
    os.makedirs(BUILD, exist_ok=True)
    if force:
        for f in (LIB, LIB_OMP):
            if os.path.exists(f):
                os.remove(f)
    _compile(LIB, [])
    try:
        _compile(LIB_OMP, ["-fopenmp"])
    except (subprocess.CalledProcessError, OSError):
        pass  # no OpenMP runtime: only the serial baseline is available
    return LIB


_libs = {}
_active = "serial"


def openmp_available() -> bool:
    build()
    return os.path.exists(LIB_OMP)


@contextlib.contextmanager
def threaded(threads: int = 0):
    """Run the oracle calls inside the block with the OpenMP build on
    `threads` host threads (0: all).  Results are bitwise those of the serial
    build."""
    global _active
    if not openmp_available():
        raise RuntimeError("the oracle's OpenMP build is not available")
    prev = _active
    _active = "omp"
    try:
        lib().or_set_threads(int(threads) if threads > 0 else (os.cpu_count() or 1))
        yield lib().or_threads()
    finally:
        _active = prev


def lib():
    key = _active
    if key not in _libs:
        _libs[key] = ctypes.CDLL(LIB_OMP if key == "omp" else build())
        L = _libs[key]
        L.or_threads.restype = ctypes.c_int
        L.or_set_threads.argtypes = [ctypes.c_int]
        G = ctypes.POINTER(OrGrid)
        L.or_spatial_operator.argtypes = [G, _dbl_p, _dbl_p]
        L.or_spatial_operator_terms.argtypes = [G, _dbl_p, _dbl_p, _dbl_p]
        L.or_spatial_operator_dir.argtypes = [G, _dbl_p, _dbl_p, _dbl_p]
        L.or_cn_residual.argtypes = [G, _dbl_p, _dbl_p, ctypes.c_double, _dbl_p]
        L.or_step_constant.argtypes = [G, _dbl_p, ctypes.c_double, _dbl_p]
        L.or_fd_eps.argtypes = [ctypes.c_long, ctypes.c_double, _dbl_p]
        L.or_fd_eps.restype = ctypes.c_double
        L.or_norm2.argtypes = [ctypes.c_long, _dbl_p]
        L.or_norm2.restype = ctypes.c_double
        L.or_jv.argtypes = [G, _dbl_p, _dbl_p, _dbl_p, ctypes.c_double, ctypes.c_double, _dbl_p]
        L.or_precond.argtypes = [G, _dbl_p, ctypes.c_double, _dbl_p, _dbl_p]
        L.or_gmres_dense.argtypes = [ctypes.c_long, _dbl_p, _dbl_p, _dbl_p, ctypes.c_int,
                                     ctypes.c_int, ctypes.c_double, ctypes.POINTER(ctypes.c_int)]
        L.or_newton_step.argtypes = [G, _dbl_p, ctypes.c_double, ctypes.POINTER(OrStepStats)]
        L.or_cfl_rate.argtypes = [G, _dbl_p]
        L.or_cfl_rate.restype = ctypes.c_double
        L.or_run.argtypes = [G, _dbl_p, ctypes.c_int, ctypes.c_double, ctypes.c_double,
                             ctypes.POINTER(OrStepStats)]
        L.or_diagnostics.argtypes = [G, _dbl_p, ctypes.c_double, ctypes.c_double, _dbl_p]
        L.or_scalar_operator.argtypes = [G, _dbl_p, _dbl_p, ctypes.c_int, _dbl_p]
        L.or_scalar_operator_dir.argtypes = [G, _dbl_p, _dbl_p, _dbl_p, ctypes.c_int, _dbl_p]
        L.or_newton_step_s.argtypes = [G, _dbl_p, _dbl_p, ctypes.c_int, ctypes.c_double, ctypes.c_int,
                                       ctypes.POINTER(OrStepStats), ctypes.POINTER(ctypes.c_int)]
        L.or_run_s.argtypes = [G, _dbl_p, _dbl_p, ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_double,
                               ctypes.c_double, ctypes.c_double, ctypes.c_int, ctypes.POINTER(OrStepStats),
                               ctypes.POINTER(ctypes.c_int)]
        L.or_run_dt.argtypes = [G, _dbl_p, ctypes.c_int, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                ctypes.c_double, ctypes.POINTER(OrStepStats)]
        L.or_scalar_mixing_width.argtypes = [G, _dbl_p, _dbl_p]
        L.or_scalar_mixing_width.restype = ctypes.c_double
        L.or_dt_rates.argtypes = [G, _dbl_p, _dbl_p]
        L.or_select_dt.argtypes = [G, _dbl_p, ctypes.c_double, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                   ctypes.POINTER(ctypes.c_int)]
        L.or_select_dt.restype = ctypes.c_double
    return _libs[key]


def _p(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(_dbl_p)


def _vec(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


def grid(prob) -> OrGrid:
    g = OrGrid()
    g.nd = prob.nd
    for d in range(3):
        g.n[d] = int(prob.n[d])
        g.dx[d] = float(prob.length[d] / prob.n[d])
        g.x0[d] = float(prob.x0[d])
        g.bc[d] = int(prob.bc[d])
        g.wall_scalar[d] = int(prob.wall_scalar[d])
        g.g[d] = float(prob.g[d])
    g.gamma = float(prob.gamma)
    g.restart = int(prob.restart)
    g.max_restarts = int(prob.max_restarts)
    g.gmres_rtol = float(prob.gmres_rtol)
    g.newton_max = int(prob.newton_max)
    g.newton_tol = float(prob.newton_tol)
    g.precond = int(prob.precond)
    g.sweeps = int(prob.sweeps)
    g.max_halvings = int(prob.max_halvings)
    g.geom = int(prob.geometry)
    if prob.gface is not None:
        gf = np.ascontiguousarray(prob.gface, dtype=np.float64)
        g._keep = gf  # keep the table alive as long as the struct
        g.gface = gf.ctypes.data_as(_dbl_p)
    g.conduct = int(prob.conduct)
    g.chi0 = float(prob.chi0)
    for d in range(3):
        g.flux_wall[d] = int(prob.flux_wall[d])
    g.lum = float(prob.lum)
    return g


def spatial_operator(prob, U) -> np.ndarray:
    """R(U), Eqs. 1-3."""
    U = _vec(U)
    R = np.empty_like(U)
    g = grid(prob)
    lib().or_spatial_operator(ctypes.byref(g), _p(U), _p(R))
    return R


def spatial_operator_terms(prob, U):
    """(R(U), A): A per cell and variable is the sum of the magnitudes of the
    terms R adds there, the scale of R's rounding (per-cell tolerances)."""
    U = _vec(U)
    R = np.empty_like(U)
    A = np.empty_like(U)
    g = grid(prob)
    lib().or_spatial_operator_terms(ctypes.byref(g), _p(U), _p(R), _p(A))
    return R, A


def spatial_operator_dir(prob, U, V) -> np.ndarray:
    """Exact (dR/dU) V by complex-step differentiation."""
    U, V = _vec(U), _vec(V)
    dR = np.empty_like(U)
    g = grid(prob)
    lib().or_spatial_operator_dir(ctypes.byref(g), _p(U), _p(V), _p(dR))
    return dR


def cn_residual(prob, U, Un, dt) -> np.ndarray:
    """F(U) = U - U^n - dt/2 (R(U) + R(U^n)) (Crank-Nicolson)."""
    U, Un = _vec(U), _vec(Un)
    F = np.empty_like(U)
    g = grid(prob)
    lib().or_cn_residual(ctypes.byref(g), _p(U), _p(Un), float(dt), _p(F))
    return F


def fd_eps(U, v) -> float:
    U, v = _vec(U), _vec(v)
    un = lib().or_norm2(U.size, _p(U))
    return lib().or_fd_eps(U.size, un, _p(v))


def jv(prob, U, v, dt, eps: float = 0.0) -> np.ndarray:
    """Jacobian-free J v (Knoll & Keyes 2004); eps <= 0 selects the default."""
    U, v = _vec(U), _vec(v)
    RU = spatial_operator(prob, U)
    out = np.empty_like(U)
    g = grid(prob)
    lib().or_jv(ctypes.byref(g), _p(U), _p(RU), _p(v), float(dt), float(eps), _p(out))
    return out


def precond(prob, U, dt, r) -> np.ndarray:
    """z = M^-1 r, the physics-based preconditioner with coefficients at U."""
    U, r = _vec(U), _vec(r)
    z = np.empty_like(U)
    g = grid(prob)
    lib().or_precond(ctypes.byref(g), _p(U), float(dt), _p(r), _p(z))
    return z


def gmres_dense(A, b, m=30, max_restarts=10, rtol=1e-10):
    """The oracle's GMRES on a dense matrix with no preconditioner."""
    A = _vec(A)
    b = _vec(b)
    x = np.empty_like(b)
    its = ctypes.c_int(0)
    rc = lib().or_gmres_dense(b.size, _p(A), _p(b), _p(x), int(m), int(max_restarts), float(rtol),
                              ctypes.byref(its))
    return x, rc, its.value


def newton_step(prob, U, dt):
    """One implicit step of size dt.  Returns (U_new, stats, rc)."""
    U = _vec(U).copy()
    st = OrStepStats()
    g = grid(prob)
    rc = lib().or_newton_step(ctypes.byref(g), _p(U), float(dt), ctypes.byref(st))
    return U, st.as_dict(), rc


def cfl_dt(prob, U, cfl) -> float:
    U = _vec(U)
    g = grid(prob)
    return float(cfl) / lib().or_cfl_rate(ctypes.byref(g), _p(U))


def run(prob, U=None, nsteps=None, cfl=None, dt_max=None):
    """Advance nsteps CFL-limited implicit steps.  Returns (U, [stats])."""
    U = _vec(prob.U if U is None else U).copy()
    nsteps = prob.nsteps if nsteps is None else nsteps
    cfl = prob.cfl if cfl is None else cfl
    dt_max = prob.dt_max if dt_max is None else dt_max
    st = (OrStepStats * max(nsteps, 1))()
    g = grid(prob)
    if prob.cfl_adv > 0.0 or prob.cfl_rad > 0.0:
        done = lib().or_run_dt(ctypes.byref(g), _p(U), int(nsteps), float(cfl), float(prob.cfl_adv),
                               float(prob.cfl_rad), float(dt_max), st)
    else:
        done = lib().or_run(ctypes.byref(g), _p(U), int(nsteps), float(cfl), float(dt_max), st)
    if done != nsteps:
        raise RuntimeError("oracle: Newton failed at step %d" % done)
    return U, [st[i].as_dict() for i in range(nsteps)]


DIAG_NAMES = ("mixing_height", "max_mach", "kh_mode_amplitude", "vertical_kinetic_energy",
              "mean_kinetic_energy", "max_speed")


def diagnostics(prob, U) -> dict:
    U = _vec(U)
    out = np.zeros(6)
    g = grid(prob)
    lib().or_diagnostics(ctypes.byref(g), _p(U), float(prob.rho_L), float(prob.rho_H), _p(out))
    return dict(zip(DIAG_NAMES, out.tolist()))


# ---------------- passive scalars (Sec. 2.2) ----------------
def scalar_operator(prob, U, q) -> np.ndarray:
    """S_i = -div(c_i rho u) of the partial densities q with the fluid frozen at U."""
    U, q = _vec(U), _vec(q)
    ns = q.size // prob.ncells
    S = np.empty_like(q)
    g = grid(prob)
    lib().or_scalar_operator(ctypes.byref(g), _p(U), _p(q), ns, _p(S))
    return S


def scalar_operator_dir(prob, U, q, v) -> np.ndarray:
    """Exact (dS/dq) v by complex-step differentiation."""
    U, q, v = _vec(U), _vec(q), _vec(v)
    ns = q.size // prob.ncells
    dS = np.empty_like(q)
    g = grid(prob)
    lib().or_scalar_operator_dir(ctypes.byref(g), _p(U), _p(q), _p(v), ns, _p(dS))
    return dS


def newton_step_s(prob, U, q, dt, enforce=None):
    """One implicit step of the fluid and its scalars.  Returns (U, q, stats, scalar GMRES steps, rc)."""
    U, q = _vec(U).copy(), _vec(q).copy()
    ns = q.size // prob.ncells
    st = OrStepStats()
    its = ctypes.c_int(0)
    enforce = prob.scalar_enforce if enforce is None else enforce
    g = grid(prob)
    rc = lib().or_newton_step_s(ctypes.byref(g), _p(U), _p(q), ns, float(dt), int(enforce), ctypes.byref(st),
                                ctypes.byref(its))
    return U, q, st.as_dict(), its.value, rc


def run_s(prob, U=None, q=None, nsteps=None, cfl=None, dt_max=None, enforce=None):
    """nsteps CFL-limited steps of the fluid and its scalars.  Returns (U, q, [stats], [scalar GMRES steps])."""
    U = _vec(prob.U if U is None else U).copy()
    q = _vec(prob.q if q is None else q).copy()
    ns = q.size // prob.ncells
    nsteps = prob.nsteps if nsteps is None else nsteps
    cfl = prob.cfl if cfl is None else cfl
    dt_max = prob.dt_max if dt_max is None else dt_max
    enforce = prob.scalar_enforce if enforce is None else enforce
    st = (OrStepStats * max(nsteps, 1))()
    its = (ctypes.c_int * max(nsteps, 1))()
    g = grid(prob)
    done = lib().or_run_s(ctypes.byref(g), _p(U), _p(q), ns, int(nsteps), float(cfl), float(prob.cfl_adv),
                          float(prob.cfl_rad), float(dt_max), int(enforce), st, its)
    if done != nsteps:
        raise RuntimeError("oracle: Newton failed at step %d" % done)
    return U, q, [st[i].as_dict() for i in range(nsteps)], [its[i] for i in range(nsteps)]


def scalar_mixing_width(prob, U, q) -> float:
    """h = sum_rows 2 min(<c_1>, <c_2>) dy (Sec. 3, passive-scalar form)."""
    U, q = _vec(U), _vec(q)
    g = grid(prob)
    return float(lib().or_scalar_mixing_width(ctypes.byref(g), _p(U), _p(q)))


# ---------------- time-step limits ----------------
def dt_rates(prob, U) -> tuple:
    """(max (|u|+c_s)/h, max |u|/h, max D/h^2) over cells and directions."""
    U = _vec(U)
    r = np.zeros(3)
    g = grid(prob)
    lib().or_dt_rates(ctypes.byref(g), _p(U), _p(r))
    return tuple(r.tolist())


def select_dt(prob, U, cfl_hydro=0.0, cfl_adv=0.0, cfl_rad=0.0, dt_max=0.0):
    """The most restrictive limit; returns (dt, which) with which = 0 hydro,
    1 advective, 2 radiative, 3 dt_max."""
    U = _vec(U)
    w = ctypes.c_int(-1)
    g = grid(prob)
    dt = lib().or_select_dt(ctypes.byref(g), _p(U), float(cfl_hydro), float(cfl_adv), float(cfl_rad),
                            float(dt_max), ctypes.byref(w))
    return float(dt), w.value


# ---------------- grid convergence of the velocity field (Sec. 4) ----------------
def face_vy(prob, U) -> np.ndarray:
    """Vertical velocity on the lower y-faces of a 2-D grid, (ny, nx): m_y over
    the mean density of the two cells sharing the face (the staggered
    velocity of Sec. 2); a walled lower face carries zero."""
    U = _vec(U)
    nx, ny = prob.n[0], prob.n[1]
    N = nx * ny
    rho = U[:N].reshape(ny, nx)
    my = U[3 * N:4 * N].reshape(ny, nx)
    below = np.roll(rho, 1, axis=0)
    v = my / (0.5 * (below + rho))
    if prob.bc[1] == 1:  # wall: the lower boundary face
        v[0, :] = 0.0
    return v


def coarsen_faces(v, r) -> np.ndarray:
    """Face-average coarsening by r of y-face values (ny, nx): a coarse y-face
    coincides with every r-th fine y-face row and is the mean of the r fine
    faces that tile it."""
    ny, nx = v.shape
    rows = v[::r, :]
    return rows.reshape(ny // r, nx // r, r).mean(axis=2)


def velocity_error(prob_fine, U_fine, prob_coarse, U_coarse) -> float:
    """Relative L1 error of the coarse vertical velocity against the coarsened
    fine one: sum |v_low - coarse(v_high)| / sum |coarse(v_high)|."""
    r = prob_fine.n[0] // prob_coarse.n[0]
    assert prob_fine.n[0] == r * prob_coarse.n[0] and prob_fine.n[1] == r * prob_coarse.n[1]
    vh = coarsen_faces(face_vy(prob_fine, U_fine), r)
    vl = face_vy(prob_coarse, U_coarse)
    return float(np.abs(vl - vh).sum() / np.abs(vh).sum())
