"""Pins of the oracle's time-step limits (Sec. 2, choice of the time step).

Closed forms on uniform states: the hydrodynamic rate max (|u_d| + c_s)/h_d,
the advective rate max |u_d|/h_d, the radiative rate max D/h_d^2 with
D = chi/(rho c_v); spherical grids measure theta by the arc r_c dtheta; the
step takes the most restrictive limit.
"""
import math

import numpy as np
import pytest

from oracle import oracle as O
from paper_1610_10053_gb300 import inputs as I


@pytest.mark.parametrize("nd,u", [(2, (0.3, -0.2, 0.0)), (3, (0.1, -0.25, 0.4))])
def test_uniform_flow_rates(nd, u):
    n = (8, 6, 5)[:nd]
    rho, p, gamma = 1.3, 2.0, 1.4
    prob = I.uniform_flow(nd, n, rho=rho, p=p, u=u, gamma=gamma, length=(1.0, 0.75, 0.5))
    cs = math.sqrt(gamma * p / rho)
    dx = [prob.length[d] / prob.n[d] for d in range(nd)]
    hydro, adv, rad = O.dt_rates(prob, prob.U)
    assert hydro == pytest.approx(max((abs(u[d]) + cs) / dx[d] for d in range(nd)), rel=1e-14)
    assert adv == pytest.approx(max(abs(u[d]) / dx[d] for d in range(nd)), rel=1e-14)
    assert rad == 0.0


def test_radiative_rate_of_a_uniform_conducting_state():
    gamma, rho, p, chi0 = 5.0 / 3.0, 0.8, 1.2, 0.03
    prob = I.uniform_flow(2, (10, 7), rho=rho, p=p, u=(0.0, 0.0, 0.0), gamma=gamma,
                          length=(1.0, 0.5, 1.0)).with_options(conduct=1, chi0=chi0)
    T = p / rho
    D = chi0 * T ** 6.5 / rho ** 2 * (gamma - 1.0) / rho   # chi / (rho c_v), c_v = 1/(gamma - 1)
    hmin = min(1.0 / 10, 0.5 / 7)
    assert O.dt_rates(prob, prob.U)[2] == pytest.approx(D / hmin ** 2, rel=1e-13)


def test_spherical_rates_use_the_arc_length():
    """A uniform state at rest on an (r, theta) wedge: the fastest cell is the
    innermost, where r_c dtheta is shortest."""
    w = I.spherical_wedge(nr=12, nth=10)
    N = w.ncells
    U = np.zeros_like(w.U)
    U[:N] = 1.0
    U[N:2 * N] = 1.5
    w2 = w.with_state(U).with_options(conduct=0)
    gamma = w.gamma
    cs = math.sqrt(gamma * (gamma - 1.0) * 1.5 / 1.0)
    dr = w.length[0] / w.n[0]
    dth = w.length[1] / w.n[1]
    rc0 = w.x0[0] + 0.5 * dr
    hydro, adv, rad = O.dt_rates(w2, U)
    assert adv == 0.0
    assert hydro == pytest.approx(cs / min(dr, rc0 * dth), rel=1e-13)


def test_the_most_restrictive_limit_applies():
    prob = I.uniform_flow(2, (8, 8), u=(0.3, -0.2, 0.0))
    hydro, adv, _ = O.dt_rates(prob, prob.U)
    dt, which = O.select_dt(prob, prob.U, cfl_hydro=10.0, cfl_adv=0.5)
    assert which == 1 and dt == pytest.approx(0.5 / adv, rel=1e-15)
    dt, which = O.select_dt(prob, prob.U, cfl_hydro=1.0, cfl_adv=0.5)
    assert which == 0 and dt == pytest.approx(1.0 / hydro, rel=1e-15)
    dt, which = O.select_dt(prob, prob.U, cfl_hydro=10.0, cfl_adv=0.5, dt_max=1e-3)
    assert which == 3 and dt == 1e-3
    dt, which = O.select_dt(prob, prob.U)
    assert which == -1 and math.isinf(dt)


def test_run_honours_the_advective_cap():
    """Each step of a capped run has CFL_adv <= 0.5 on its starting state."""
    p = I.kelvin_helmholtz(n=16, seed=4, nsteps=3).with_options(cfl=10.0, cfl_adv=0.05)
    U = p.U.copy()
    U1, st = O.run(p, U=U)
    for s in st:
        _, adv, _ = O.dt_rates(p, U)
        assert s["dt"] * adv <= 0.05 * (1 + 1e-14)
        U, _ = O.run(p.with_options(cfl_adv=0.05), U=U, nsteps=1)
