"""GPU time-step limits (Sec. 2, choice of the time step) against the oracle."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1610_10053_gb300 import inputs as I

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

from test_gpu_parity import B  # noqa: E402

CASES = {
    "kh": lambda: I.kelvin_helmholtz(n=40, ny=24, seed=5, nsteps=1),
    "rt": lambda: I.rayleigh_taylor(nx=16, ny=48, nsteps=1),
    "tgv": lambda: I.taylor_green(n=10, nsteps=1),
    "wedge": lambda: I.spherical_wedge(nr=24, nth=12, nsteps=1),
    "conduct": lambda: I.random_smooth(2, (18, 14), seed=81, amp=0.3).with_options(conduct=1, chi0=0.05),
}


@pytest.mark.parametrize("case", sorted(CASES))
@pytest.mark.parametrize("limit", [0, 1, 2])
def test_each_limit_against_oracle(case, limit):
    p = CASES[case]()
    cfl = [0.0, 0.0, 0.0]
    cfl[limit] = (5.0, 0.5, 100.0)[limit]
    ref, wref = O.select_dt(p, p.U, *cfl)
    with B().Grid(p, precision=B().MIXED) as g:
        g.set_state(p.U)
        if wref < 0:
            with pytest.raises(B().MusicError):
                g.select_dt(*cfl)
            return
        dt, w = g.select_dt(*cfl)
    assert w == wref == limit
    assert dt == pytest.approx(ref, rel=1e-14)


@pytest.mark.parametrize("case", sorted(CASES))
def test_hydro_limit_is_the_cfl_rule(case):
    p = CASES[case]()
    with B().Grid(p, precision=B().FP64) as g:
        g.set_state(p.U)
        dt, w = g.select_dt(7.0, 0.0, 0.0, 0.0)
        assert w == 0 and dt == g.cfl_dt(7.0)
        dt2, w2 = g.select_dt(7.0, 0.0, 0.0, 1e-6)
        assert w2 == 3 and dt2 == 1e-6


def test_capped_run_against_oracle():
    p = I.kelvin_helmholtz(n=32, seed=12, nsteps=3).with_options(cfl=10.0, cfl_adv=0.05)
    with B().Grid(p, precision=B().FP64) as g:
        g.set_state(p.U)
        st = g.run()
        U = g.get_state()
    Ur, str_ = O.run(p)
    assert [s["dt"] for s in st] == pytest.approx([s["dt"] for s in str_], rel=1e-12)
    assert np.abs(U - Ur).max() <= 1e-9 * np.abs(Ur).max()


def test_server_applies_the_caps():
    p = I.kelvin_helmholtz(n=32, seed=13, nsteps=2).with_options(cfl=10.0, cfl_adv=0.05)
    with B().Grid(p, precision=B().MIXED) as g:
        g.set_state(p.U)
        g.run()
        U = g.get_state()
    with B().Server(max_active=1) as s:
        t = s.submit(p, B().MIXED)
        assert s.wait(t, timeout_ms=300000)["status"] == 0
        assert np.array_equal(s.result_state(t), U)


def test_newton_step_takes_the_most_restrictive_limit():
    """music_newton_step chooses the step on the device from the grid's limits
    (here CFL_hydro 10 and CFL_adv 0.05), capped by dt_max; a grid without
    limits takes dt_max as given and refuses dt_max <= 0."""
    p = I.kelvin_helmholtz(n=32, seed=12, nsteps=1).with_options(cfl=10.0, cfl_adv=0.05)
    ref, w = O.select_dt(p, p.U, 10.0, 0.05, 0.0, 0.0)
    assert w == 1
    with B().Grid(p, precision=B().FP64) as g:
        g.set_state(p.U)
        st = g.newton_step(0.0)
    assert st["dt_halvings"] == 0 and st["dt"] == pytest.approx(ref, rel=1e-14)
    with B().Grid(p, precision=B().FP64) as g:
        g.set_state(p.U)
        st = g.newton_step(0.25 * ref)
    assert st["dt"] == 0.25 * ref
    with B().Grid(p, precision=B().FP64, cfl_hydro=0.0, cfl_adv=0.0) as g:
        g.set_state(p.U)
        with pytest.raises(B().MusicError) as e:
            g.newton_step(0.0)
        assert e.value.code == 1
        st = g.newton_step(0.5 * ref)
    assert st["dt"] == 0.5 * ref
