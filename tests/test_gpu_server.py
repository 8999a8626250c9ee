"""Solve server (include/music_server.h): continuous batching on one GPU.

Each solve must give the same result alone and in a mix (every reduction is
deterministic, so equality is bitwise), admission must respect the memory
budget, and one failing solve must not disturb the others.  A solve the batch
lane takes is compared with the same solve stepped alone as a batch of one
(music_batch_step); every other solve with the per-grid path (music_newton_step).
"""
import numpy as np
import pytest

from paper_1610_10053_gb300 import inputs as I

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def B():
    from paper_1610_10053_gb300 import binding
    return binding


def mix():
    return [
        (I.rayleigh_taylor(nx=32, ny=96, nsteps=3), 0),
        (I.kelvin_helmholtz(n=64, seed=3, nsteps=2), 1),
        (I.kelvin_helmholtz(n=128, seed=4, nsteps=2), 1),
        (I.rayleigh_taylor(nsteps=2), 1),
        (I.kelvin_helmholtz(n=64, seed=5, nsteps=3), 0),
        (I.taylor_green(n=16, nsteps=1), 1),
    ]


LANE_CELLS = 16384  # batch_max_cells of the lane tests


def lane_route(prob, prec, lane_cells=LANE_CELLS):
    """The server's lane rule: small 2-D Cartesian solves without diffusion,
    of at most 24 preconditioner sweeps in mixed precision (16 in FP64)."""
    kmax = 24 if prec == B().MIXED else 16
    return (lane_cells > 0 and prob.nd == 2 and prob.geometry == I.GEOM_CARTESIAN and not prob.conduct
            and prob.sweeps <= kmax and prob.ncells <= lane_cells)


def alone(prob, prec, lane_cells=LANE_CELLS):
    with B().Grid(prob, precision=prec) as g:
        g.set_state(prob.U)
        if lane_route(prob, prec, lane_cells):
            for _ in range(prob.nsteps):
                code, _st = B().batch_step([g])
                assert code == 0
        else:
            g.run()
        return g.get_state(), g.diagnostics()


@pytest.mark.parametrize("lane_cells", [LANE_CELLS, 0], ids=["batch-lane", "workers-only"])
def test_same_result_alone_and_in_the_mix(lane_cells):
    reqs = mix()
    with B().Server(max_active=4, batch_max_cells=lane_cells) as s:
        tickets = [s.submit(p, prec) for p, prec in reqs]
        results = [s.wait(t, timeout_ms=300000) for t in tickets]
        states = [s.result_state(t) for t in tickets]
        st = s.stats()
        lat = s.step_times()
    for (p, prec), r, U in zip(reqs, results, states):
        assert r["status"] == 0 and r["steps_done"] == p.nsteps
        U1, d1 = alone(p, prec, lane_cells)
        assert np.array_equal(U, U1), p.name
        assert r["diag"] == [d1[k] for k in ("mixing_height", "max_mach", "kh_mode_amplitude",
                                             "vertical_kinetic_energy", "mean_kinetic_energy", "max_speed")]
        assert r["step_ms_p99"] >= r["step_ms_p50"] > 0.0
    assert st["cell_steps"] == sum(p.ncells * p.nsteps for p, _ in reqs)
    assert len(lat) == sum(p.nsteps for p, _ in reqs)
    assert st["active"] == 0 and st["queued"] == 0


def test_admission_by_device_footprint():
    big = I.kelvin_helmholtz(n=256, seed=6, nsteps=2)
    fp = B().footprint(big, B().MIXED)
    # room for one such solve at a time
    with B().Server(mem_budget_bytes=int(1.5 * fp), max_active=8) as s:
        t = [s.submit(big, B().MIXED) for _ in range(3)]
        r = [s.wait(x, timeout_ms=300000) for x in t]
        assert all(x["status"] == 0 for x in r)
        # the second and third waited for memory, not for a worker
        waited = sorted(x["queue_ms"] for x in r)
        assert waited[1] > 0.5 * r[0]["total_ms"] or waited[1] > 1.0
        huge = I.kelvin_helmholtz(n=1024, nsteps=1)
        with pytest.raises(B().MusicError) as e:
            s.submit(huge, B().MIXED)
        assert e.value.code == 8  # MUSIC_E_BUSY: can never fit


def test_wait_timeout_and_poll():
    p = I.kelvin_helmholtz(n=256, nsteps=4)
    with B().Server(max_active=1) as s:
        t1 = s.submit(p, B().FP64)
        t2 = s.submit(p, B().FP64)
        with pytest.raises(B().MusicError) as e:
            s.wait(t2, timeout_ms=0)
        assert e.value.code == 7  # MUSIC_E_TIMEOUT
        assert s.poll(t2) is None or s.poll(t2)["status"] == 0
        assert s.wait(t1)["status"] == 0 and s.wait(t2)["status"] == 0
        s.release(t1)
        with pytest.raises(B().MusicError):
            s.poll(t1)


def test_failing_solve_does_not_disturb_the_mix():
    good = I.kelvin_helmholtz(n=64, seed=7, nsteps=2)
    bad = good.with_state(np.where(np.arange(good.U.size) == 5, np.nan, good.U))
    with B().Server(max_active=2) as s:
        tb = s.submit(bad, B().MIXED)
        tg = s.submit(good, B().MIXED)
        rb, rg = s.wait(tb), s.wait(tg)
        Ug = s.result_state(tg)
    assert rb["status"] != 0
    assert rg["status"] == 0
    U1, _ = alone(good, B().MIXED, lane_cells=0)  # this server has no batch lane
    assert np.array_equal(Ug, U1)


def test_continuous_batching_in_the_lane():
    """More small solves than lane slots, of mixed lengths and precisions: they
    join and leave the batch at step boundaries and each matches its batch of one."""
    reqs = []
    for k in range(20):
        if k % 3 == 0:
            p = I.rayleigh_taylor(nx=16, ny=48, nsteps=1 + k % 4)
        else:
            p = I.kelvin_helmholtz(n=32 + 16 * (k % 3), seed=20 + k, nsteps=1 + k % 5)
            if k % 2 == B().FP64:
                p = p.with_options(sweeps=16)  # the lane's FP64 limit
        reqs.append((p, k % 2))
    with B().Server(max_active=2, batch_max_cells=LANE_CELLS, batch_size=6) as s:
        tickets = [s.submit(p, prec) for p, prec in reqs]
        results = [s.wait(t, timeout_ms=300000) for t in tickets]
        states = [s.result_state(t) for t in tickets]
        st = s.stats()
    for (p, prec), r, U in zip(reqs, results, states):
        assert lane_route(p, prec)
        assert r["status"] == 0 and r["steps_done"] == p.nsteps
        U1, _ = alone(p, prec)
        assert np.array_equal(U, U1), p.name
    assert st["cell_steps"] == sum(p.ncells * p.nsteps for p, _ in reqs)


def test_autotuning_server_gives_the_same_results():
    """With autotune each new configuration is tuned before its first step;
    every tile shape computes the same result, so the solves match the
    untuned ones bitwise."""
    reqs = [(I.kelvin_helmholtz(n=96, seed=31, nsteps=2), 1), (I.rayleigh_taylor(nx=24, ny=72, nsteps=2), 0),
            (I.kelvin_helmholtz(n=96, seed=32, nsteps=2), 1)]
    out = {}
    for tune in (False, True):
        with B().Server(max_active=2, autotune=tune) as s:
            t = [s.submit(p, prec) for p, prec in reqs]
            r = [s.wait(x, timeout_ms=300000) for x in t]
            out[tune] = [s.result_state(x) for x in t]
            assert all(x["status"] == 0 for x in r)
    for a, b in zip(out[False], out[True]):
        assert np.array_equal(a, b)


def test_graph_workers_give_the_same_results():
    """Workers stepping with the recorded solver graph and with host-sequenced
    kernels compute identical solves."""
    reqs = [(I.kelvin_helmholtz(n=64, seed=41, nsteps=2), 1), (I.rayleigh_taylor(nx=16, ny=48, nsteps=2), 0)]
    out = {}
    for graph in (False, True):
        with B().Server(max_active=2, graph=graph) as s:
            t = [s.submit(p, prec) for p, prec in reqs]
            assert all(s.wait(x, timeout_ms=300000)["status"] == 0 for x in t)
            out[graph] = [s.result_state(x) for x in t]
    for a, b in zip(out[False], out[True]):
        assert np.array_equal(a, b)
