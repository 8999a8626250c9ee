"""The allocation-free CFL-rate entry point (music_cfl_rate_noalloc).

It exists for callers that cannot allocate device memory (code inside
another framework's memory pool, real-time loops, a nearly full device).  It
must agree with the grid-based music_cfl_dt on consecutive calls, since it
reuses the same reduction with a fixed scratch array inside the library.
Collected last so that a failure here never hides another test's result.
"""
import ctypes

import numpy as np
import pytest

from paper_1610_10053_gb300 import inputs as I

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.mark.parametrize("make", [lambda: I.kelvin_helmholtz(n=128, seed=3),
                                  lambda: I.rayleigh_taylor(),
                                  lambda: I.taylor_green(n=16),
                                  # spherical: tangential spacing r_c dtheta
                                  lambda: I.spherical_wedge(nr=64, nth=32, nsteps=1)],
                         ids=["kh128", "rt64x192", "tgv16", "wedge64x32"])
def test_noalloc_rate_matches_grid_cfl_twice(make):
    from paper_1610_10053_gb300 import binding as B
    p = make()
    cfl = 7.0
    with B.Grid(p) as g:
        g.set_state(p.U)
        dt_ref = g.cfl_dt(cfl)
    U = torch.from_numpy(p.U.copy()).cuda()
    U2 = torch.from_numpy(p.U.copy()).cuda()  # the same state in another buffer
    for Ux in (U, U2):
        rate = torch.full((1,), -1.0, dtype=torch.float64, device="cuda")
        B.cfl_rate_noalloc(p, Ux, rate)
        torch.cuda.synchronize()
        dt = cfl / rate.item()
        assert abs(dt - dt_ref) <= 1e-14 * dt_ref


def test_noalloc_rejects_too_many_rows():
    from paper_1610_10053_gb300 import binding as B
    p = I.kelvin_helmholtz(n=4, ny=20000)
    U = torch.zeros(4, dtype=torch.float64, device="cuda")
    rate = torch.zeros(1, dtype=torch.float64, device="cuda")
    d = B.desc_from_problem(p)
    rc = B.load().music_cfl_rate_noalloc(ctypes.byref(d), ctypes.c_void_p(U.data_ptr()),
                                         ctypes.c_void_p(rate.data_ptr()), None)
    assert rc == 1 and "16384" in B.last_error()


def test_noalloc_rate_of_a_nan_state_is_nan():
    """The rate never leaves the device, so the call cannot flag a bad state:
    one NaN cell must come back as a NaN rate (with MUSIC_OK) for the
    caller to test, while the grid-based call reports MUSIC_E_NONFINITE."""
    from paper_1610_10053_gb300 import binding as B
    p = I.kelvin_helmholtz(n=64, seed=3)
    U = p.U.copy()
    U[p.ncells + 777] = np.nan  # one cell's energy
    rate = torch.zeros(1, dtype=torch.float64, device="cuda")
    B.cfl_rate_noalloc(p, torch.from_numpy(U).cuda(), rate)
    torch.cuda.synchronize()
    assert np.isnan(rate.item())
    with B.Grid(p) as g:
        g.set_state(U)
        with pytest.raises(B.MusicError) as e:
            g.cfl_dt(5.0)
        assert e.value.code == 6
    # a finite state right after still gives the grid's rate (nothing sticks)
    B.cfl_rate_noalloc(p, torch.from_numpy(p.U.copy()).cuda(), rate)
    with B.Grid(p) as g:
        g.set_state(p.U)
        dt_ref = g.cfl_dt(5.0)
    assert abs(5.0 / rate.item() - dt_ref) <= 1e-14 * dt_ref
