"""Thin ctypes binding of libmusic (include/music.h).

Argument marshalling only: every computation happens inside the CUDA
library.  Device arrays are torch CUDA tensors (PyTorch supplies device
memory and streams); their raw pointers and the current stream's handle are
passed through the C ABI.  There is no CPU fallback: if the library cannot be
loaded, every call raises.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional

import numpy as np

from . import build as _build

_dbl_p = ctypes.POINTER(ctypes.c_double)

MUSIC_OK = 0
STATUS = {0: "OK", 1: "E_INVAL", 2: "E_OOM", 3: "E_CUDA", 4: "E_NEWTON_FAIL", 5: "E_GMRES_FAIL",
          6: "E_NONFINITE", 7: "E_TIMEOUT", 8: "E_BUSY", 9: "E_NOTFOUND"}
FP64, MIXED = 0, 1
JV_FD64, JV_DIFF32 = 0, 1  # forms of the Jacobian-free product (music_set_jv_form)
PROF_JV, PROF_PRECOND, PROF_RESIDUAL, PROF_VECTOR = 0, 1, 2, 3  # profiled kernel classes (music_profile_read_class)


class MusicError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("%s (%d): %s" % (STATUS.get(code, "?"), code, msg))
        self.code = code


class GridDesc(ctypes.Structure):
    _fields_ = [
        ("ndim", ctypes.c_int), ("n", ctypes.c_int * 3), ("origin", ctypes.c_double * 3),
        ("length", ctypes.c_double * 3), ("bc", ctypes.c_int * 3), ("wall_scalar", ctypes.c_int * 3),
        ("gamma", ctypes.c_double), ("g", ctypes.c_double * 3), ("precision", ctypes.c_int),
        ("gmres_restart", ctypes.c_int), ("gmres_max_restarts", ctypes.c_int),
        ("gmres_rtol", ctypes.c_double), ("newton_max_its", ctypes.c_int), ("newton_tol", ctypes.c_double),
        ("precond", ctypes.c_int), ("precond_sweeps", ctypes.c_int), ("max_dt_halvings", ctypes.c_int),
        ("geometry", ctypes.c_int), ("g_radial", ctypes.POINTER(ctypes.c_double)), ("conduct", ctypes.c_int),
        ("chi0", ctypes.c_double), ("flux_wall", ctypes.c_int * 3), ("lum", ctypes.c_double),
        ("nscalars", ctypes.c_int), ("scalar_enforce", ctypes.c_int),
        ("cfl_hydro", ctypes.c_double), ("cfl_adv", ctypes.c_double), ("cfl_rad", ctypes.c_double),
    ]


class StepStats(ctypes.Structure):
    _fields_ = [
        ("dt", ctypes.c_double), ("newton_its", ctypes.c_int), ("gmres_its", ctypes.c_int),
        ("dt_halvings", ctypes.c_int), ("gmres_unconverged", ctypes.c_int), ("fnorm0", ctypes.c_double),
        ("fnorm", ctypes.c_double), ("max_drho", ctypes.c_double), ("wall_ms", ctypes.c_double),
        ("scalar_gmres_its", ctypes.c_int), ("pad", ctypes.c_int),
    ]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_ if k != "pad"}


# every exported symbol of include/music.h with its ctypes signature
class DtLimits(ctypes.Structure):
    _fields_ = [("cfl_hydro", ctypes.c_double), ("cfl_adv", ctypes.c_double), ("cfl_rad", ctypes.c_double),
                ("dt_max", ctypes.c_double)]


class TuneReport(ctypes.Structure):
    _fields_ = [("tunable", ctypes.c_int), ("from_cache", ctypes.c_int), ("stencil_tile", ctypes.c_int * 2),
                ("precond_tile", ctypes.c_int * 2), ("precond_stages", ctypes.c_int), ("n_stencil", ctypes.c_int),
                ("n_precond", ctypes.c_int), ("stencil_cand", (ctypes.c_int * 2) * 8),
                ("precond_cand", (ctypes.c_int * 3) * 24), ("stencil_us", ctypes.c_double * 8),
                ("precond_us", ctypes.c_double * 24), ("residual_tile", ctypes.c_int * 2),
                ("residual_us", ctypes.c_double * 8), ("batch_tile", ctypes.c_int * 2), ("n_batch", ctypes.c_int),
                ("pad", ctypes.c_int), ("batch_cand", (ctypes.c_int * 2) * 4), ("batch_us", ctypes.c_double * 4)]

    def as_dict(self):
        """stencil_us and residual_us keys: (TX, TY); precond_us keys: (TX, TY, stages)."""
        return {"tunable": self.tunable, "from_cache": self.from_cache,
                "stencil_tile": tuple(self.stencil_tile), "precond_tile": tuple(self.precond_tile),
                "precond_stages": self.precond_stages, "residual_tile": tuple(self.residual_tile),
                "stencil_us": {tuple(self.stencil_cand[i]): self.stencil_us[i] for i in range(self.n_stencil)},
                "residual_us": {tuple(self.stencil_cand[i]): self.residual_us[i] for i in range(self.n_stencil)},
                "precond_us": {tuple(self.precond_cand[i]): self.precond_us[i] for i in range(self.n_precond)},
                "batch_tile": tuple(self.batch_tile),
                "batch_us": {tuple(self.batch_cand[i]): self.batch_us[i] for i in range(self.n_batch)}}


MUSIC_TUNE_FORCE = 1
MUSIC_TUNE_BATCH = 2


class Peaks(ctypes.Structure):
    _fields_ = [("fp64_fma_tflops", ctypes.c_double), ("fp32_fma_tflops", ctypes.c_double),
                ("fp64_div_gops", ctypes.c_double), ("sms", ctypes.c_int), ("pad", ctypes.c_int)]

SIGNATURES = {
    "music_last_error": (ctypes.c_size_t, [ctypes.c_char_p, ctypes.c_size_t]),
    "music_version": (ctypes.c_char_p, []),
    "music_kernel_launches": (ctypes.c_uint64, []),
    "music_create_grid": (ctypes.c_int, [ctypes.POINTER(GridDesc), ctypes.POINTER(ctypes.c_void_p)]),
    "music_destroy_grid": (ctypes.c_int, [ctypes.c_void_p]),
    "music_state_size": (ctypes.c_size_t, [ctypes.c_void_p]),
    "music_grid_footprint": (ctypes.c_int, [ctypes.POINTER(GridDesc), ctypes.POINTER(ctypes.c_size_t)]),
    "music_grid_bytes": (ctypes.c_size_t, [ctypes.c_void_p]),
    "music_set_state": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int]),
    "music_get_state": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int]),
    "music_spatial_operator": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    "music_residual": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_double,
                                      ctypes.c_void_p, ctypes.c_void_p]),
    "music_jv": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                ctypes.c_double, ctypes.c_double, ctypes.c_void_p]),
    "music_precond_apply": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_double, ctypes.c_void_p,
                                           ctypes.c_void_p, ctypes.c_void_p]),
    "music_newton_step": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_double, ctypes.POINTER(StepStats),
                                         ctypes.c_void_p]),
    "music_cfl_dt": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_double, _dbl_p, ctypes.c_void_p]),
    "music_diagnostics": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_double, ctypes.c_double, _dbl_p,
                                         ctypes.c_void_p]),
    "music_cfl_rate_noalloc": (ctypes.c_int, [ctypes.POINTER(GridDesc), ctypes.c_void_p, ctypes.c_void_p,
                                              ctypes.c_void_p]),
    "music_batch_step": (ctypes.c_int, [ctypes.POINTER(ctypes.c_void_p), ctypes.c_int, _dbl_p, _dbl_p,
                                        ctypes.POINTER(StepStats), ctypes.c_void_p]),
    "music_profile_enable": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int]),
    "music_set_scalars": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p]),
    "music_velocity_error": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, _dbl_p, ctypes.c_void_p]),
    "music_select_dt": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(DtLimits), _dbl_p,
                                       ctypes.POINTER(ctypes.c_int), ctypes.c_void_p]),
    "music_get_scalars": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p]),
    "music_scalar_operator": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                             ctypes.c_void_p]),
    "music_scalar_mixing_width": (ctypes.c_int, [ctypes.c_void_p, _dbl_p, ctypes.c_void_p]),
    "music_autotune": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_double, ctypes.c_uint, ctypes.POINTER(TuneReport),
                                      ctypes.c_void_p]),
    "music_set_tiles": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int),
                                       ctypes.c_int]),
    "music_get_tiles": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int),
                                       ctypes.POINTER(ctypes.c_int)]),
    "music_profile_read": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_uint64), _dbl_p]),
    "music_set_jv_form": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int]),
    "music_profile_read_class": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.POINTER(ctypes.c_uint64),
                                                _dbl_p]),
    "music_get_jv_form": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_int)]),
    "music_measure_peaks": (ctypes.c_int, [ctypes.POINTER(Peaks), ctypes.c_void_p]),
    "music_vanleer_slopes": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_longlong,
                                            ctypes.c_void_p]),
    "music_stencil_quotients": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                               ctypes.c_longlong, ctypes.c_void_p]),
    "music_set_batch_tile": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_int)]),
    "music_get_batch_tile": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_int)]),
}

_lib = None


def lib_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True):
    """Load libmusic.so (building it first if needed and nvcc exists)."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.LIB
    if build_if_missing and not _build.up_to_date():
        _build.build()
    if not os.path.exists(path):
        raise RuntimeError("libmusic.so is not built (%s); run paper_1610_10053_gb300.build.build()" % path)
    L = ctypes.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args
    _lib = L
    return L


def kernel_launches() -> int:
    return int(load().music_kernel_launches())


def last_error() -> str:
    buf = ctypes.create_string_buffer(1024)
    load().music_last_error(buf, 1024)
    return buf.value.decode(errors="replace")


def check(code: int):
    if code != MUSIC_OK:
        raise MusicError(code, last_error())


def _require(cond, msg: str):
    """Argument checks that stay on under python -O: a wrong size would have
    the library read or write past the caller's buffer."""
    if not cond:
        raise ValueError(msg)


def _check_vecs(*args):
    """Device vector arguments, each (tensor, entries, dtype, name): type,
    dtype and size of all of them, then their placement, checked before the
    library reads or writes that many entries through their pointers."""
    import torch
    for t, n, dtype, what in args:
        _require(isinstance(t, torch.Tensor), "%s must be a torch tensor" % what)
        _require(t.dtype == dtype, "%s must be %s, not %s" % (what, dtype, t.dtype))
        _require(t.numel() == n, "%s has %d entries, the grid needs %d" % (what, t.numel(), n))
    for t, _, _, what in args:
        _require(t.is_cuda and t.is_contiguous(), "%s must be a contiguous CUDA tensor" % what)


def _stream():
    import torch
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def _ptr(t) -> ctypes.c_void_p:
    import torch
    _require(isinstance(t, torch.Tensor) and t.is_cuda and t.is_contiguous(), "expected a contiguous CUDA tensor")
    return ctypes.c_void_p(t.data_ptr())


def desc_from_problem(prob, precision: int = FP64, **over) -> GridDesc:
    d = GridDesc()
    d.ndim = prob.nd
    for k in range(3):
        d.n[k] = int(prob.n[k])
        d.origin[k] = float(prob.x0[k])
        d.length[k] = float(prob.length[k])
        d.bc[k] = int(prob.bc[k])
        d.wall_scalar[k] = int(prob.wall_scalar[k])
        d.g[k] = float(prob.g[k])
    d.gamma = float(prob.gamma)
    d.precision = int(precision)
    d.gmres_restart = int(prob.restart)
    d.gmres_max_restarts = int(prob.max_restarts)
    d.gmres_rtol = float(prob.gmres_rtol)
    d.newton_max_its = int(prob.newton_max)
    d.newton_tol = float(prob.newton_tol)
    d.precond = 1 if int(prob.precond) == 1 else -1
    d.precond_sweeps = int(prob.sweeps)
    d.max_dt_halvings = int(prob.max_halvings)
    d.geometry = int(getattr(prob, "geometry", 0))
    gf = getattr(prob, "gface", None)
    if gf is not None:
        gf = np.ascontiguousarray(gf, dtype=np.float64)
        d._keep = gf  # the library copies the table at creation
        d.g_radial = gf.ctypes.data_as(_dbl_p)
    d.conduct = int(getattr(prob, "conduct", 0))
    d.chi0 = float(getattr(prob, "chi0", 0.0))
    for k in range(3):
        d.flux_wall[k] = int(getattr(prob, "flux_wall", (0, 0, 0))[k])
    d.lum = float(getattr(prob, "lum", 0.0))
    d.nscalars = int(getattr(prob, "nscalars", 0))
    d.scalar_enforce = int(getattr(prob, "scalar_enforce", 0))
    # the problem's time-step limits: music_newton_step applies them
    d.cfl_hydro = float(getattr(prob, "cfl", 0.0))
    d.cfl_adv = float(getattr(prob, "cfl_adv", 0.0))
    d.cfl_rad = float(getattr(prob, "cfl_rad", 0.0))
    for k, v in over.items():
        setattr(d, k, v)
    return d


def cfl_rate_noalloc(prob, U, rate, precision: int = FP64):
    """max (|u|+c)/dx of the device state U into the one-element device tensor
    `rate`, without any device allocation (music_cfl_rate_noalloc)."""
    import torch
    _check_vecs((U, prob.nvars * prob.ncells, torch.float64, "U"), (rate, 1, torch.float64, "rate"))
    d = desc_from_problem(prob, precision)
    check(load().music_cfl_rate_noalloc(ctypes.byref(d), _ptr(U), _ptr(rate), _stream()))


def batch_step(grids, cfl=None, dt_max=None):
    """One implicit step of every grid in one launch (music_batch_step), each
    with its problem's cfl (or the given per-grid values).
    Returns (status, [stats dict per grid])."""
    n = len(grids)
    arr = (ctypes.c_void_p * n)(*[g.h.value for g in grids])
    cf = (ctypes.c_double * n)(*[float(g.prob.cfl if cfl is None else cfl[i]) for i, g in enumerate(grids)])
    dm = (ctypes.c_double * n)(*[float(g.prob.dt_max if dt_max is None else dt_max[i]) for i, g in enumerate(grids)])
    st = (StepStats * n)()
    code = load().music_batch_step(arr, n, cf, dm, st, _stream())
    if code == 1:
        check(code)
    return code, [st[i].as_dict() for i in range(n)]


def measure_peaks() -> dict:
    """Measured FP64 / FP32 FMA and FP64 division throughput of the current
    device (music_measure_peaks)."""
    pk = Peaks()
    check(load().music_measure_peaks(ctypes.byref(pk), _stream()))
    return {"fp64_fma_tflops": pk.fp64_fma_tflops, "fp32_fma_tflops": pk.fp32_fma_tflops,
            "fp64_div_gops": pk.fp64_div_gops, "sms": pk.sms}


def vanleer_slopes(a, b):
    """The van Leer slopes of the one-sided differences a and b as the FP64
    stencils compute them (music_vanleer_slopes); a and b contiguous float64
    CUDA tensors of one size."""
    import torch
    _require(a.dtype == torch.float64 and b.dtype == torch.float64 and a.numel() == b.numel(),
             "a and b must be float64 tensors of one size")
    s = torch.empty_like(a)
    check(load().music_vanleer_slopes(_ptr(a), _ptr(b), _ptr(s), a.numel(), _stream()))
    return s


def stencil_quotients(n, d):
    """n / d as the FP64 stencils form E / rho and m / rbar
    (music_stencil_quotients); n and d contiguous float64 CUDA tensors of one
    size."""
    import torch
    _require(n.dtype == torch.float64 and d.dtype == torch.float64 and n.numel() == d.numel(),
             "n and d must be float64 tensors of one size")
    q = torch.empty_like(n)
    check(load().music_stencil_quotients(_ptr(n), _ptr(d), _ptr(q), n.numel(), _stream()))
    return q


def velocity_error(fine, coarse) -> float:
    """Relative L1 error of the coarse grid's vertical velocity against the
    fine grid's, coarsened by face averaging (music_velocity_error)."""
    e = ctypes.c_double()
    check(load().music_velocity_error(fine.h, coarse.h, ctypes.byref(e), _stream()))
    return e.value


def footprint(prob, precision: int = FP64, **over) -> int:
    """Device bytes a grid for `prob` would own."""
    d = desc_from_problem(prob, precision, **over)
    b = ctypes.c_size_t()
    check(load().music_grid_footprint(ctypes.byref(d), ctypes.byref(b)))
    return int(b.value)


class Grid:
    """Owns one music_grid (device state + solver workspace)."""

    def __init__(self, prob, precision: int = FP64, **over):
        L = load()
        self.prob = prob
        self.precision = precision
        self.desc = desc_from_problem(prob, precision, **over)
        h = ctypes.c_void_p()
        check(L.music_create_grid(ctypes.byref(self.desc), ctypes.byref(h)))
        self.h = h
        self.n = int(L.music_state_size(h))

    def close(self):
        if getattr(self, "h", None):
            load().music_destroy_grid(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    @property
    def device_bytes(self) -> int:
        return int(load().music_grid_bytes(self.h))

    @property
    def kdtype(self):
        import torch
        return torch.float32 if self.precision == MIXED else torch.float64

    # ---- state
    def set_state(self, U):
        import torch
        if isinstance(U, torch.Tensor) and U.is_cuda:
            _require(U.numel() == self.n, "state has %d entries, the grid %d" % (U.numel(), self.n))
            U = U.contiguous().to(torch.float64)
            check(load().music_set_state(self.h, _ptr(U), 1))
        elif isinstance(U, torch.Tensor):
            _require(U.dtype == torch.float64 and U.is_contiguous() and U.numel() == self.n,
                     "host state must be a contiguous float64 tensor of %d entries" % self.n)
            check(load().music_set_state(self.h, ctypes.c_void_p(U.data_ptr()), 0))
        else:
            a = np.ascontiguousarray(U, dtype=np.float64)
            _require(a.size == self.n, "state has %d entries, the grid %d" % (a.size, self.n))
            check(load().music_set_state(self.h, a.ctypes.data_as(ctypes.c_void_p), 0))

    def get_state_into(self, out):
        """Copy the state into a contiguous float64 host (e.g. pinned) tensor."""
        import torch
        _require(isinstance(out, torch.Tensor) and not out.is_cuda and out.dtype == torch.float64
                 and out.is_contiguous() and out.numel() == self.n,
                 "out must be a contiguous float64 host tensor of %d entries" % self.n)
        check(load().music_get_state(self.h, ctypes.c_void_p(out.data_ptr()), 0))
        return out

    def get_state(self) -> np.ndarray:
        a = np.empty(self.n, dtype=np.float64)
        check(load().music_get_state(self.h, a.ctypes.data_as(ctypes.c_void_p), 0))
        return a

    # ---- passive scalars (partial densities, nscalars planes)
    def set_scalars(self, q):
        a = np.ascontiguousarray(q, dtype=np.float64)
        check(load().music_set_scalars(self.h, a.ctypes.data_as(ctypes.c_void_p), 0, _stream()))

    def get_scalars(self) -> np.ndarray:
        a = np.empty(self.desc.nscalars * self.prob.ncells, dtype=np.float64)
        check(load().music_get_scalars(self.h, a.ctypes.data_as(ctypes.c_void_p), 0, _stream()))
        return a

    def scalar_operator(self, U, q):
        import torch
        _check_vecs((U, self.n, torch.float64, "U"),
                    (q, self.desc.nscalars * self.prob.ncells, torch.float64, "q"))
        S = torch.empty_like(q)
        check(load().music_scalar_operator(self.h, _ptr(U), _ptr(q), _ptr(S), _stream()))
        return S

    def scalar_mixing_width(self) -> float:
        h = ctypes.c_double()
        check(load().music_scalar_mixing_width(self.h, ctypes.byref(h), _stream()))
        return h.value

    # ---- single-call operators (device tensors in, device tensors out)
    def spatial_operator(self, U):
        import torch
        _check_vecs((U, self.n, torch.float64, "U"))
        R = torch.empty_like(U)
        check(load().music_spatial_operator(self.h, _ptr(U), _ptr(R), _stream()))
        return R

    def residual(self, U, Un, dt: float):
        import torch
        _check_vecs((U, self.n, torch.float64, "U"), (Un, self.n, torch.float64, "Un"))
        F = torch.empty_like(U)
        check(load().music_residual(self.h, _ptr(U), _ptr(Un), float(dt), _ptr(F), _stream()))
        return F

    def jv(self, U, v, dt: float, eps: float = 0.0):
        import torch
        _check_vecs((U, self.n, torch.float64, "U"), (v, self.n, self.kdtype, "v"))
        out = torch.empty_like(v)
        check(load().music_jv(self.h, _ptr(U), _ptr(v), _ptr(out), float(dt), float(eps), _stream()))
        return out

    def precond(self, U, dt: float, r):
        import torch
        _check_vecs((U, self.n, torch.float64, "U"), (r, self.n, self.kdtype, "r"))
        z = torch.empty_like(r)
        check(load().music_precond_apply(self.h, _ptr(U), float(dt), _ptr(r), _ptr(z), _stream()))
        return z

    # ---- stepping
    def cfl_dt(self, cfl: float) -> float:
        out = ctypes.c_double()
        check(load().music_cfl_dt(self.h, float(cfl), ctypes.byref(out), _stream()))
        return out.value

    def newton_step(self, dt_max: float = 0.0) -> dict:
        """One implicit step (music_newton_step): the most restrictive of the
        grid's time-step limits and dt_max (> 0), or dt_max itself on a grid
        created without limits (cfl_hydro = cfl_adv = cfl_rad = 0)."""
        st = StepStats()
        check(load().music_newton_step(self.h, float(dt_max), ctypes.byref(st), _stream()))
        return st.as_dict()

    def select_dt(self, cfl_hydro: float = 0.0, cfl_adv: float = 0.0, cfl_rad: float = 0.0,
                  dt_max: float = 0.0):
        """(dt, which) of music_select_dt: the most restrictive limit."""
        lim = DtLimits(float(cfl_hydro), float(cfl_adv), float(cfl_rad), float(dt_max))
        dt, w = ctypes.c_double(), ctypes.c_int()
        check(load().music_select_dt(self.h, ctypes.byref(lim), ctypes.byref(dt), ctypes.byref(w), _stream()))
        return dt.value, w.value

    def step(self, dt_max: Optional[float] = None) -> dict:
        """One implicit step with the grid's time-step limits (the problem's
        cfl, cfl_adv and cfl_rad), capped by dt_max (default: the problem's)."""
        return self.newton_step(self.prob.dt_max if dt_max is None else dt_max)

    def autotune(self, dt: Optional[float] = None, force: bool = False, batch: bool = False) -> dict:
        """Pick the fused kernels' tile shapes by timing (music_autotune), with
        `batch` also the batched kernel's; dt defaults to the CFL step of the
        problem."""
        if dt is None:
            dt = self.cfl_dt(self.prob.cfl)
            if self.prob.dt_max and 0 < self.prob.dt_max < dt:
                dt = self.prob.dt_max
        rep = TuneReport()
        flags = (MUSIC_TUNE_FORCE if force else 0) | (MUSIC_TUNE_BATCH if batch else 0)
        check(load().music_autotune(self.h, float(dt), flags, ctypes.byref(rep), _stream()))
        return rep.as_dict()

    def set_tiles(self, stencil=None, precond=None, stages: int = 0):
        st = (ctypes.c_int * 2)(*stencil) if stencil is not None else None
        pt = (ctypes.c_int * 2)(*precond) if precond is not None else None
        check(load().music_set_tiles(self.h, st, pt, int(stages)))

    def set_batch_tile(self, tile):
        """Tile shape of the persistent batched kernel (music_set_batch_tile)."""
        check(load().music_set_batch_tile(self.h, (ctypes.c_int * 2)(*tile)))

    def batch_tile(self):
        t = (ctypes.c_int * 2)()
        check(load().music_get_batch_tile(self.h, t))
        return tuple(t)

    def set_jv_form(self, form: int):
        """JV_FD64 or JV_DIFF32 (mixed grids): the form of the Jacobian-free
        product (music_set_jv_form)."""
        check(load().music_set_jv_form(self.h, int(form)))

    def jv_form(self) -> int:
        f = ctypes.c_int()
        check(load().music_get_jv_form(self.h, ctypes.byref(f)))
        return f.value

    def tiles(self):
        """((stencil TX, TY), (preconditioner TX, TY), preconditioner stages)"""
        st, pt, q = (ctypes.c_int * 2)(), (ctypes.c_int * 2)(), ctypes.c_int()
        check(load().music_get_tiles(self.h, st, pt, ctypes.byref(q)))
        return tuple(st), tuple(pt), q.value

    def run(self, nsteps: Optional[int] = None, dt_max: Optional[float] = None):
        nsteps = self.prob.nsteps if nsteps is None else nsteps
        return [self.step(dt_max) for _ in range(nsteps)]

    def profile(self, on: bool = True):
        """Time every Jv-mode stencil launch with CUDA events (see music.h)."""
        check(load().music_profile_enable(self.h, 1 if on else 0))

    def profile_read(self, cls: int = 0):
        """(launches, summed ms) of a profiled kernel class: PROF_JV,
        PROF_PRECOND, PROF_RESIDUAL or PROF_VECTOR (music_profile_read_class)."""
        n = ctypes.c_uint64()
        ms = ctypes.c_double()
        check(load().music_profile_read_class(self.h, int(cls), ctypes.byref(n), ctypes.byref(ms)))
        return int(n.value), float(ms.value)

    def diagnostics(self, rho_L: Optional[float] = None, rho_H: Optional[float] = None) -> dict:
        out = (ctypes.c_double * 6)()
        rl = self.prob.rho_L if rho_L is None else rho_L
        rh = self.prob.rho_H if rho_H is None else rho_H
        check(load().music_diagnostics(self.h, float(rl), float(rh), out, _stream()))
        names = ("mixing_height", "max_mach", "kh_mode_amplitude", "vertical_kinetic_energy",
                 "mean_kinetic_energy", "max_speed")
        return dict(zip(names, list(out)))


# ------------------------------------------------------------------ server
class ServerOpts(ctypes.Structure):
    _fields_ = [("mem_budget_bytes", ctypes.c_size_t), ("max_active", ctypes.c_int),
                ("batch_max_cells", ctypes.c_int), ("batch_size", ctypes.c_int), ("autotune", ctypes.c_int),
                ("graph", ctypes.c_int)]


class SolveReq(ctypes.Structure):
    _fields_ = [("desc", GridDesc), ("U0", ctypes.POINTER(ctypes.c_double)), ("n_steps", ctypes.c_int),
                ("cfl", ctypes.c_double), ("dt_max", ctypes.c_double), ("rho_L", ctypes.c_double),
                ("rho_H", ctypes.c_double), ("cfl_adv", ctypes.c_double), ("cfl_rad", ctypes.c_double)]


class SolveResult(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int), ("steps_done", ctypes.c_int), ("sim_time", ctypes.c_double),
                ("diag", ctypes.c_double * 6), ("step_ms_p50", ctypes.c_double), ("step_ms_p99", ctypes.c_double),
                ("queue_ms", ctypes.c_double), ("total_ms", ctypes.c_double), ("newton_its", ctypes.c_int),
                ("gmres_its", ctypes.c_int)]

    def as_dict(self):
        d = {k: getattr(self, k) for k, _ in self._fields_ if k != "diag"}
        d["diag"] = list(self.diag)
        return d


SIGNATURES.update({
    "music_server_create": (ctypes.c_int, [ctypes.POINTER(ServerOpts), ctypes.POINTER(ctypes.c_void_p)]),
    "music_submit_solve": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(SolveReq),
                                          ctypes.POINTER(ctypes.c_uint64)]),
    "music_poll": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_uint64, ctypes.POINTER(SolveResult)]),
    "music_wait": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_uint64, ctypes.c_int, ctypes.POINTER(SolveResult)]),
    "music_result_state": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_uint64, _dbl_p]),
    "music_release": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_uint64]),
    "music_server_stats": (ctypes.c_int, [ctypes.c_void_p, _dbl_p, _dbl_p, ctypes.POINTER(ctypes.c_int),
                                          ctypes.POINTER(ctypes.c_int)]),
    "music_server_step_times": (ctypes.c_int, [ctypes.c_void_p, _dbl_p, ctypes.c_size_t,
                                               ctypes.POINTER(ctypes.c_size_t)]),
    "music_server_destroy": (ctypes.c_int, [ctypes.c_void_p]),
})


class Server:
    """Continuous-batching solve server (include/music_server.h)."""

    def __init__(self, mem_budget_bytes: int = 0, max_active: int = 16, batch_max_cells: int = 0,
                 batch_size: int = 0, autotune: bool = False, graph: bool = False):
        L = load()
        o = ServerOpts(mem_budget_bytes, max_active, batch_max_cells, batch_size, 1 if autotune else 0,
                       1 if graph else 0)
        h = ctypes.c_void_p()
        check(L.music_server_create(ctypes.byref(o), ctypes.byref(h)))
        self.h = h
        self._n = {}

    def submit(self, prob, precision: int = FP64, n_steps=None, cfl=None, dt_max=None, **over) -> int:
        """The initial state is the fluid's planes, then the scalars' when the
        problem carries passive scalars (so is result_state)."""
        U0 = np.ascontiguousarray(prob.U if prob.q is None else np.concatenate([prob.U, prob.q]),
                                  dtype=np.float64)
        req = SolveReq()
        req.desc = desc_from_problem(prob, precision, **over)
        req.U0 = U0.ctypes.data_as(_dbl_p)
        req.n_steps = int(prob.nsteps if n_steps is None else n_steps)
        req.cfl = float(prob.cfl if cfl is None else cfl)
        req.dt_max = float(prob.dt_max if dt_max is None else dt_max)
        req.rho_L, req.rho_H = float(prob.rho_L), float(prob.rho_H)
        req.cfl_adv, req.cfl_rad = float(prob.cfl_adv), float(prob.cfl_rad)
        t = ctypes.c_uint64()
        check(load().music_submit_solve(self.h, ctypes.byref(req), ctypes.byref(t)))
        self._n[t.value] = U0.size
        return int(t.value)

    def poll(self, ticket: int):
        r = SolveResult()
        code = load().music_poll(self.h, ticket, ctypes.byref(r))
        if code == 8:
            return None
        check(code)
        return r.as_dict()

    def wait(self, ticket: int, timeout_ms: int = -1) -> dict:
        r = SolveResult()
        check(load().music_wait(self.h, ticket, int(timeout_ms), ctypes.byref(r)))
        return r.as_dict()

    def result_state(self, ticket: int) -> np.ndarray:
        a = np.empty(self._n[ticket], dtype=np.float64)
        check(load().music_result_state(self.h, ticket, a.ctypes.data_as(_dbl_p)))
        return a

    def release(self, ticket: int):
        check(load().music_release(self.h, ticket))
        self._n.pop(ticket, None)

    def stats(self) -> dict:
        cs, busy = ctypes.c_double(), ctypes.c_double()
        act, q = ctypes.c_int(), ctypes.c_int()
        check(load().music_server_stats(self.h, ctypes.byref(cs), ctypes.byref(busy), ctypes.byref(act),
                                        ctypes.byref(q)))
        return {"cell_steps": cs.value, "busy_ms": busy.value, "active": act.value, "queued": q.value}

    def step_times(self) -> np.ndarray:
        n = ctypes.c_size_t()
        check(load().music_server_step_times(self.h, None, 0, ctypes.byref(n)))
        a = np.empty(n.value, dtype=np.float64)
        check(load().music_server_step_times(self.h, a.ctypes.data_as(_dbl_p), n.value, ctypes.byref(n)))
        return a

    def close(self):
        if getattr(self, "h", None):
            load().music_server_destroy(self.h)
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
