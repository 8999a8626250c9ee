"""The grid-convergence measure of Sec. 4 on the GPU against the oracle's
definition, and a small convergence run."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1610_10053_gb300 import inputs as I

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

from test_gpu_parity import B  # noqa: E402


@pytest.mark.parametrize("pair", [("kh", 64, 16), ("rt", 32, 16)])
def test_velocity_error_against_oracle(pair):
    kind, nf, nc = pair
    if kind == "kh":
        pf, pc = I.kelvin_helmholtz(n=nf, seed=3, nsteps=1), I.kelvin_helmholtz(n=nc, seed=4, nsteps=1)
    else:
        pf, pc = I.rayleigh_taylor(nx=nf, ny=3 * nf, nsteps=1), I.rayleigh_taylor(nx=nc, ny=3 * nc, nsteps=1)
    with B().Grid(pf, precision=B().MIXED) as gf, B().Grid(pc, precision=B().MIXED) as gc:
        gf.set_state(pf.U)
        gc.set_state(pc.U)
        e = B().velocity_error(gf, gc)
    ref = O.velocity_error(pf, pf.U, pc, pc.U)
    assert e == pytest.approx(ref, rel=1e-12)


def run_to(prob, t_end, prec):
    g = B().Grid(prob, precision=prec)
    g.set_state(prob.U)
    t = 0.0
    while t < t_end * (1 - 1e-12):
        dt = min(g.cfl_dt(prob.cfl), t_end - t)
        t += g.newton_step(dt)["dt"]
    return g


def test_error_falls_with_resolution():
    """Once the shear layers (width 0.05) are resolved the error against a
    much finer solution falls with every doubling."""
    t_end = 0.02
    ref = run_to(I.kelvin_helmholtz(n=1024, seed=2, noise=0.0), t_end, B().MIXED)
    errs = []
    for n in (64, 128, 256):
        g = run_to(I.kelvin_helmholtz(n=n, seed=2, noise=0.0), t_end, B().MIXED)
        errs.append(B().velocity_error(ref, g))
        g.close()
    ref.close()
    assert errs[0] > errs[1] > errs[2], errs
