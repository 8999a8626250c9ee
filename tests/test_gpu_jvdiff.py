"""The difference form of the Jacobian-free product (Sec. 2) on mixed grids.

Jv = v - dt/2 (R(U + eps v) - R(U)) / eps, computed by carrying every
intermediate's scaled difference in FP32, against the oracle's FP64 finite
difference at the same eps (and against the GPU's own FP64 form).  The
operator part dR = (v - Jv) / (dt/2) is compared plane by plane.

Tolerance: each scaled difference passes through about twenty FP32 roundings
(reconstruction, upwind products, quotients), so a flux difference carries a
relative error of about 20 u = 1.2e-6 (u = 2^-24); a residual sums up to
eight of them, whose sizes are bounded by the plane's largest |dR| times the
cancellation of the divergence, a few for the smooth states here.  That gives
about 1e-5 of the plane's largest |dR|, the bar used below; the FP64
reference's own rounding (2^-53 of R over eps ~ 1e-8) is below 1e-7 of it.
The Rayleigh-Taylor states have exactly zero x-velocities (and, at rest,
zero y-velocities too), so every upwind choice they decide flips between U
and U + eps v with the sign of the direction: those cases pin the flip
formula.
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1610_10053_gb300 import inputs as I

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

from test_gpu_parity import B, dev, host  # noqa: E402

from test_gpu_parity import CASES as PARITY  # noqa: E402

CASES = {k: PARITY[k] for k in ("periodic2d_ragged", "walls_hse2d", "walls_mirror_x", "kh_64")}
CASES["rt_32x96"] = lambda: I.rayleigh_taylor(nx=32, ny=96)
CASES["rt_at_rest"] = lambda: I.rayleigh_taylor(nx=32, ny=96, perturbation="none")

TOL = 1e-5


def dR_planes(p, v, Jv, dt):
    return (v - Jv) / (0.5 * dt)


def compare(p, got, ref, tol=TOL):
    N = p.ncells
    worst = 0.0
    for k in range(p.nvars):
        s = slice(k * N, (k + 1) * N)
        scale = np.abs(ref[s]).max()
        if scale == 0.0:
            assert np.abs(got[s]).max() == 0.0
            continue
        worst = max(worst, np.abs(got[s] - ref[s]).max() / scale)
    assert worst <= tol, worst
    return worst


def gpu_jv(p, v32, dt, eps, form):
    with B().Grid(p, precision=B().MIXED) as g:
        g.set_jv_form(form)
        assert g.jv_form() == form
        Jv = host(g.jv(dev(p.U), dev(v32), dt, eps))
    return Jv


@pytest.mark.parametrize("case", sorted(CASES))
@pytest.mark.parametrize("which_eps", ["fixed", "default"])
def test_difference_form_against_oracle(case, which_eps):
    p = CASES[case]()
    rng = np.random.default_rng(31)
    # a smooth direction plus noise, rounded to the Krylov type
    v = rng.standard_normal(p.U.size).astype(np.float32)
    v = v.astype(np.float64)
    dt = O.cfl_dt(p, p.U, 5.0)
    eps = O.fd_eps(p.U, v) if which_eps == "default" else 1e-7 * np.linalg.norm(p.U) / np.linalg.norm(v)
    Jv = gpu_jv(p, v.astype(np.float32), dt, eps if which_eps == "fixed" else 0.0, B().JV_DIFF32)
    ref = O.jv(p, p.U, v, dt, eps)
    compare(p, dR_planes(p, v, Jv, dt), dR_planes(p, v, ref, dt))


@pytest.mark.parametrize("case", ["periodic2d_ragged", "walls_hse2d", "kh_64"])
def test_difference_form_against_fp64_form(case):
    p = CASES[case]()
    rng = np.random.default_rng(32)
    v = rng.standard_normal(p.U.size).astype(np.float32)
    dt = O.cfl_dt(p, p.U, 5.0)
    a = gpu_jv(p, v, dt, 0.0, B().JV_DIFF32)
    b = gpu_jv(p, v, dt, 0.0, B().JV_FD64)
    v = v.astype(np.float64)
    compare(p, dR_planes(p, v, a, dt), dR_planes(p, v, b, dt))


def test_kh_512_against_oracle():
    """The benchmark grid, several tiles of every shape and the default eps."""
    p = I.kelvin_helmholtz(n=512)
    rng = np.random.default_rng(33)
    v = rng.standard_normal(p.U.size).astype(np.float32).astype(np.float64)
    dt = O.cfl_dt(p, p.U, 10.0)
    ref = O.jv(p, p.U, v, dt)
    Jv = gpu_jv(p, v.astype(np.float32), dt, 0.0, B().JV_DIFF32)
    compare(p, dR_planes(p, v, Jv, dt), dR_planes(p, v, ref, dt))


def test_every_tile_shape_gives_the_same_bits():
    p = CASES["walls_hse2d"]()
    rng = np.random.default_rng(34)
    v = dev(rng.standard_normal(p.U.size).astype(np.float32))
    dt = O.cfl_dt(p, p.U, 5.0)
    outs = []
    with B().Grid(p, precision=B().MIXED) as g:
        g.set_jv_form(B().JV_DIFF32)
        for st in ((16, 8), (16, 16), (32, 8), (32, 16), (32, 32)):
            g.set_tiles(stencil=st)
            outs.append(host(g.jv(dev(p.U), v, dt)))
    for o in outs[1:]:
        assert np.array_equal(o, outs[0])


def test_zero_direction_gives_zero():
    p = CASES["periodic2d_ragged"]()
    with B().Grid(p, precision=B().MIXED) as g:
        Jv = host(g.jv(dev(p.U), torch.zeros(p.U.size, dtype=torch.float32, device="cuda"), 0.1))
    assert not Jv.any()


def test_form_setting_is_validated():
    p = CASES["kh_64"]()
    with B().Grid(p, precision=B().FP64) as g:
        assert g.jv_form() == B().JV_FD64
        with pytest.raises(B().MusicError):
            g.set_jv_form(B().JV_DIFF32)
    with B().Grid(p, precision=B().MIXED) as g:
        assert g.jv_form() == B().JV_DIFF32
        with pytest.raises(B().MusicError):
            g.set_jv_form(7)


@pytest.mark.parametrize("case", ["rt_32x96", "kh_64"])
def test_steps_in_either_form_reach_the_same_solution(case):
    """Both forms solve the same Newton system; at Newton tolerance 1e-11 the
    steps agree to the oracle's 1e-9 bar."""
    p = CASES[case]().with_options(newton_tol=1e-11, nsteps=2)
    res = []
    for form in (B().JV_DIFF32, B().JV_FD64):
        with B().Grid(p, precision=B().MIXED) as g:
            g.set_jv_form(form)
            g.set_state(p.U)
            g.run()
            res.append(g.get_state())
    Ur, _ = O.run(p)
    for U in res:
        assert np.abs(U - Ur).max() <= 1e-9 * np.abs(Ur).max()


# ---- the multi-pass path: 3-D grids, and 2-D grids on the multi-pass stencil
CASES3 = {
    "periodic3d_ragged": PARITY["periodic3d_ragged"],
    "tgv_16": PARITY["tgv_16"],
    "walls_hse3d": lambda: I.random_smooth(3, (10, 9, 8), seed=25, amp=0.3,
                                           bc=(I.BC_PERIODIC, I.BC_WALL, I.BC_PERIODIC),
                                           wall_scalar=(0, I.WALL_HSE, 0), g=(0.0, -0.4, 0.0)),
}


@pytest.mark.parametrize("case", sorted(CASES3))
@pytest.mark.parametrize("which_eps", ["fixed", "default"])
def test_multipass_difference_form_3d_against_oracle(case, which_eps):
    p = CASES3[case]()
    rng = np.random.default_rng(35)
    v = rng.standard_normal(p.U.size).astype(np.float32).astype(np.float64)
    dt = O.cfl_dt(p, p.U, 5.0)
    eps = O.fd_eps(p.U, v) if which_eps == "default" else 1e-7 * np.linalg.norm(p.U) / np.linalg.norm(v)
    Jv = gpu_jv(p, v.astype(np.float32), dt, eps if which_eps == "fixed" else 0.0, B().JV_DIFF32)
    ref = O.jv(p, p.U, v, dt, eps)
    compare(p, dR_planes(p, v, Jv, dt), dR_planes(p, v, ref, dt))


@pytest.mark.parametrize("case", ["periodic2d_ragged", "walls_hse2d", "rt_32x96"])
def test_multipass_difference_form_2d_matches_fused(case, monkeypatch):
    """2-D grids on the multi-pass stencil (MUSIC_STENCIL=multipass) against
    the oracle, and against the fused kernel's difference form."""
    p = CASES[case]()
    rng = np.random.default_rng(36)
    v = rng.standard_normal(p.U.size).astype(np.float32)
    dt = O.cfl_dt(p, p.U, 5.0)
    fused = gpu_jv(p, v, dt, 0.0, B().JV_DIFF32)
    monkeypatch.setenv("MUSIC_STENCIL", "multipass")
    multi = gpu_jv(p, v, dt, 0.0, B().JV_DIFF32)
    v64 = v.astype(np.float64)
    ref = O.jv(p, p.U, v64, dt)
    compare(p, dR_planes(p, v64, multi, dt), dR_planes(p, v64, ref, dt))
    compare(p, dR_planes(p, v64, multi, dt), dR_planes(p, v64, fused, dt))


def test_3d_steps_in_either_form_reach_the_same_solution():
    p = CASES3["tgv_16"]().with_options(newton_tol=1e-11, nsteps=2)
    res = []
    for form in (B().JV_DIFF32, B().JV_FD64):
        with B().Grid(p, precision=B().MIXED) as g:
            g.set_jv_form(form)
            g.set_state(p.U)
            g.run()
            res.append(g.get_state())
    Ur, _ = O.run(p)
    for U in res:
        assert np.abs(U - Ur).max() <= 1e-9 * np.abs(Ur).max()
