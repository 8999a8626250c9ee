"""The recorded solver graph (device-driven Newton / GMRES loops) against the
host-sequenced driver.

Both drivers launch the same vector kernels with the same arguments, and the
graph's control kernels round every Givens and back-substitution operation
exactly as the host does, so the states, the iteration counts and the norms
must agree bitwise, on every code path (fused 2-D, 3-D multi-pass, spherical
with radiative diffusion), through GMRES restarts, dt halvings and
non-finite input.
"""
import numpy as np
import pytest

from paper_1610_10053_gb300 import inputs as I

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

from test_gpu_wedge import wedge  # noqa: E402


def B():
    from paper_1610_10053_gb300 import binding
    return binding


STAT_KEYS = ("dt", "newton_its", "gmres_its", "dt_halvings", "gmres_unconverged", "fnorm0", "fnorm", "max_drho")

CASES = {
    "rt_fp64": (lambda: I.rayleigh_taylor(nx=32, ny=96, nsteps=3), "FP64"),
    "kh_mixed": (lambda: I.kelvin_helmholtz(n=64, seed=3, nsteps=3), "MIXED"),
    "kh_fp64_restarts": (lambda: I.kelvin_helmholtz(n=64, seed=4, nsteps=2).with_options(restart=3, gmres_rtol=1e-6),
                         "FP64"),
    "kh_mixed_restarts": (lambda: I.kelvin_helmholtz(n=48, seed=5, nsteps=2).with_options(restart=4,
                                                                                         gmres_rtol=1e-5),
                          "MIXED"),
    "tgv_mixed_3d": (lambda: I.taylor_green(n=16, nsteps=2), "MIXED"),
    "wedge_mixed": (lambda: wedge(nr=24, nth=16)[1].with_options(nsteps=2, cfl=20.0), "MIXED"),
    "no_precond_fp64": (lambda: I.kelvin_helmholtz(n=32, seed=6, nsteps=2).with_options(precond=0), "FP64"),
}


def run(prob, prec, solver, monkeypatch, nsteps=None):
    if solver == "host":
        monkeypatch.setenv("MUSIC_SOLVER", "host")
    else:
        monkeypatch.delenv("MUSIC_SOLVER", raising=False)
    with B().Grid(prob, precision=getattr(B(), prec)) as g:
        g.set_state(prob.U)
        stats = g.run(nsteps)
        return g.get_state(), stats


@pytest.mark.parametrize("case", sorted(CASES))
def test_graph_equals_host_driver(case, monkeypatch):
    make, prec = CASES[case]
    p = make()
    Ug, sg = run(p, prec, "graph", monkeypatch)
    Uh, sh = run(p, prec, "host", monkeypatch)
    assert np.array_equal(Ug, Uh), case
    for a, b in zip(sg, sh):
        for k in STAT_KEYS:
            assert a[k] == b[k], (case, k, a[k], b[k])
    if "restarts" in case:
        # the case exists to take the restart branch
        assert max(s["gmres_its"] for s in sg) > p.restart


def test_newton_failure_restores_state_in_both_drivers(monkeypatch):
    # one Newton iteration cannot meet a 1e-14 density-correction test
    p = I.kelvin_helmholtz(n=32, seed=8, nsteps=1).with_options(newton_max=1, newton_tol=1e-14, max_halvings=2)
    out = {}
    for solver in ("graph", "host"):
        if solver == "host":
            monkeypatch.setenv("MUSIC_SOLVER", "host")
        else:
            monkeypatch.delenv("MUSIC_SOLVER", raising=False)
        with B().Grid(p, precision=B().MIXED) as g:
            g.set_state(p.U)
            with pytest.raises(B().MusicError) as e:
                g.step()
            out[solver] = (e.value.code, g.get_state())
    assert out["graph"][0] == out["host"][0] == 4  # MUSIC_E_NEWTON_FAIL
    assert np.array_equal(out["graph"][1], p.U)
    assert np.array_equal(out["host"][1], p.U)


def test_nonfinite_state_reports_the_same_error(monkeypatch):
    p = I.kelvin_helmholtz(n=32, seed=9, nsteps=1)
    bad = p.with_state(np.where(np.arange(p.U.size) == 77, np.nan, p.U))
    codes = {}
    for solver in ("graph", "host"):
        if solver == "host":
            monkeypatch.setenv("MUSIC_SOLVER", "host")
        else:
            monkeypatch.delenv("MUSIC_SOLVER", raising=False)
        # no time-step limits: the step is the given dt, so the solver itself
        # meets the NaN (the limits' reduction would report it first)
        with B().Grid(bad, precision=B().FP64, cfl_hydro=0.0) as g:
            g.set_state(bad.U)
            with pytest.raises(B().MusicError) as e:
                g.newton_step(1e-3)
            codes[solver] = e.value.code
    assert codes["graph"] == codes["host"] == 6  # MUSIC_E_NONFINITE


def test_graph_replays_count_their_kernels(monkeypatch):
    """The launch counter includes the kernels each replay ran: about as many as
    the host driver launches, plus the single-thread control kernels."""
    p = I.kelvin_helmholtz(n=64, seed=10, nsteps=2)
    counts = {}
    for solver in ("graph", "host"):
        if solver == "host":
            monkeypatch.setenv("MUSIC_SOLVER", "host")
        else:
            monkeypatch.delenv("MUSIC_SOLVER", raising=False)
        with B().Grid(p, precision=B().MIXED) as g:
            g.set_state(p.U)
            g.step()  # the first graph step also records the graph
            k0 = B().kernel_launches()
            st = g.step()
            counts[solver] = (B().kernel_launches() - k0, st)
    (ng, sg), (nh, sh) = counts["graph"], counts["host"]
    assert sg["gmres_its"] == sh["gmres_its"]
    # host: the CFL rate kernels are counted in both; the graph adds its
    # control kernels (a few per Newton iteration and per Arnoldi step)
    assert nh < ng < nh + 3 * (sg["newton_its"] + sg["gmres_its"]) + 16


@pytest.mark.parametrize("case", ["kh_mixed", "rt_fp64", "tgv_mixed_3d", "wedge_mixed"])
def test_programmatic_launches_change_no_bit(case, monkeypatch):
    """The recorded graph with programmatic kernel-to-kernel edges (the
    default) and with plain edges (MUSIC_PDL=0) runs the same kernels on the
    same data in the same order: every kernel waits for its predecessor's
    completion before it reads anything."""
    make, prec = CASES[case]
    p = make()
    monkeypatch.delenv("MUSIC_PDL", raising=False)
    Ua, sa = run(p, prec, "graph", monkeypatch)
    monkeypatch.setenv("MUSIC_PDL", "0")
    Ub, sb = run(p, prec, "graph", monkeypatch)
    assert np.array_equal(Ua, Ub), case
    for a, b in zip(sa, sb):
        for k in STAT_KEYS:
            assert a[k] == b[k], (case, k, a[k], b[k])


@pytest.mark.parametrize("solver", ["graph", "host"])
def test_loop_body_bound_expires_with_timeout(solver, monkeypatch):
    """The bound on loop bodies of a Newton attempt (every Arnoldi step, GMRES
    cycle and Newton iteration counts one) lowered to 5: the attempt stops
    with MUSIC_E_TIMEOUT, through either driver, and the state is restored
    to U^n.  The bound is a counter in the control code, so its expiry is an
    ordinary status; the grid and the context stay usable."""
    p = I.kelvin_helmholtz(n=32, seed=9, nsteps=1)
    monkeypatch.setenv("MUSIC_LOOP_CAP", "5")
    if solver == "host":
        monkeypatch.setenv("MUSIC_SOLVER", "host")
    else:
        monkeypatch.delenv("MUSIC_SOLVER", raising=False)
    with B().Grid(p, precision=B().MIXED) as g:
        g.set_state(p.U)
        with pytest.raises(B().MusicError) as e:
            g.step()
        assert e.value.code == 7  # MUSIC_E_TIMEOUT
        assert np.array_equal(g.get_state(), p.U)
    monkeypatch.delenv("MUSIC_LOOP_CAP")
    with B().Grid(p, precision=B().MIXED) as g:
        g.set_state(p.U)
        st = g.step()
        assert st["newton_its"] >= 1 and st["gmres_its"] > 5

