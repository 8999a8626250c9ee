"""The oracle's OpenMP build (the multi-core CPU baseline) gives bitwise the
results of the serial oracle: only loops over independent cells and vector
entries are split over threads, every reduction stays one fixed-order loop."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1610_10053_gb300 import inputs as I

pytestmark = pytest.mark.skipif(not O.openmp_available(), reason="no OpenMP runtime for the oracle")


@pytest.mark.parametrize("make", [lambda: I.kelvin_helmholtz(n=48, seed=3, nsteps=2),
                                  lambda: I.rayleigh_taylor(nx=16, ny=48, nsteps=2),
                                  lambda: I.taylor_green(n=8, nsteps=1),
                                  lambda: I.spherical_wedge(nr=16, nth=8, nsteps=1, noise=1e-3),
                                  lambda: I.rayleigh_taylor(nx=8, ny=24, nsteps=1, scalars=True)],
                         ids=["kh48", "rt16x48", "tgv8", "wedge16x8", "rt_scalars"])
def test_threaded_oracle_is_bitwise_serial(make):
    p = make()
    if p.q is not None:
        U1, q1, s1, _ = O.run_s(p)
        with O.threaded(4) as nt:
            assert nt == 4
            U4, q4, s4, _ = O.run_s(p)
        assert np.array_equal(q1, q4)
    else:
        U1, s1 = O.run(p)
        with O.threaded(4) as nt:
            assert nt == 4
            U4, s4 = O.run(p)
    assert np.array_equal(U1, U4)
    assert [(a["newton_its"], a["gmres_its"]) for a in s1] == [(a["newton_its"], a["gmres_its"]) for a in s4]
