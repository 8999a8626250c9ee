"""Whole-run parity at the benchmark tolerance, on the benchmark grids.

Every run here takes the Newton tolerance the benchmarks use (1e-8 on the
density corrections, Sec. 2.2) in BOTH precisions; nothing is re-run at a
tighter tolerance.  The GPU's post-run diagnostics are compared with the
FP64 oracle's after the same steps:

  * FP64 path: 1e-9 relative;
  * mixed path (FP32 Krylov basis and preconditioner): 1e-7 relative.

Grids: Kelvin-Helmholtz 512^2 (the benchmark workload, 3 steps), the
spherical wedge 256 x 128 (2 steps at 100x the acoustic CFL limit, Sec. 6),
the Taylor-Green vortex at 64^3 (2 steps, Sec. 5) and Rayleigh-Taylor
64 x 192 (all 10 steps, Sec. 3).  The diagnostic each workload is judged by
(the KH mode amplitude, the TGV kinetic energy, the wedge's velocity
residual max |u|, the RT mixing-layer height) is compared strictly
relative; the others are compared as in the other parity tests, relative
with a floor of 1e-3 absolute times the tolerance (a diagnostic that
vanishes by symmetry is rounding noise on both sides).

The wedge is the one exception, and only for its velocity diagnostics
(max |u| and the Mach number).  Its velocities are the residue of 1e-6
density noise on a hydrostatic background, max |u| = 6e-7 of the sound
speed, and a Newton test on density corrections at 1e-8 does not determine
them to 1e-7: the oracle itself stops 2.5e-3 (relative) away from its own
converged root there (its run at Newton tolerance 1e-11).  So for those two
diagnostics the FP64 path must agree with the oracle to 1e-9 relative or
to 1e-14 absolute (the rounding floor of the O(1) pressure and gravity terms
whose balance leaves that velocity; measured 1.5e-15), and the mixed path
must be ten times closer to the oracle than the oracle is to its converged
root (measured: fifteen times).  The GPU runs stay at tolerance 1e-8; the
tighter oracle run only measures how far that tolerance determines them.

With MUSIC_PARITY_REPORT=<file> every measured error is also written there
as JSON lines (one per config and precision).
"""
import functools
import json
import os

import numpy as np
import pytest

from oracle import oracle as O
from paper_1610_10053_gb300 import inputs as I

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

from test_gpu_parity import B  # noqa: E402

CONFIGS = {
    # name: (problem, the diagnostic the workload is judged by)
    "kh512": (lambda: I.kelvin_helmholtz(n=512, seed=2, nsteps=3), "kh_mode_amplitude"),
    "wedge256x128": (lambda: I.spherical_wedge(seed=5, nsteps=2), "max_speed"),
    "tgv64": (lambda: I.taylor_green(n=64, nsteps=2), "mean_kinetic_energy"),
    "rt64x192": (lambda: I.rayleigh_taylor(nsteps=10), "mixing_height"),
}
RTOL = {"fp64": 1e-9, "mixed": 1e-7}


# diagnostics of the wedge that its density-only Newton test leaves open
WEDGE_VELOCITY = ("max_speed", "max_mach")


@functools.lru_cache(maxsize=None)
def oracle_run(name, newton_tol=1e-8):
    p = CONFIGS[name][0]()
    if newton_tol != p.newton_tol:
        p = p.with_options(newton_tol=newton_tol, newton_max=20)
    U, st = O.run(p)
    return U, st, O.diagnostics(p, U)


def gpu_run(name, prec):
    p = CONFIGS[name][0]()
    pr = B().FP64 if prec == "fp64" else B().MIXED
    with B().Grid(p, precision=pr) as g:
        g.set_state(p.U)
        st = g.run()
        U = g.get_state()
        d = g.diagnostics()
    return p, U, st, d


def report(rec):
    path = os.environ.get("MUSIC_PARITY_REPORT")
    if path:
        with open(path, "a") as f:
            f.write(json.dumps(rec) + "\n")


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("name", list(CONFIGS))
def test_diagnostics_at_newton_tol_1e8(name, prec):
    p, U, st, d = gpu_run(name, prec)
    Uref, sref, dref = oracle_run(name)
    assert p.newton_tol == 1e-8
    key = CONFIGS[name][1]
    rtol = RTOL[prec]
    rel = {k: abs(d[k] - dref[k]) / max(abs(dref[k]), 1e-300) for k in dref}
    N = p.ncells
    planes = [float(np.abs(U[v * N:(v + 1) * N] - Uref[v * N:(v + 1) * N]).max()
                    / (np.abs(Uref[v * N:(v + 1) * N]).max() + 1e-300)) for v in range(p.nvars)]
    report({"config": name, "precision": prec, "newton_tol": p.newton_tol, "key": key,
            "diag_rel_err": rel, "diag": d, "diag_oracle": dref, "state_rel_err_per_plane": planes,
            "newton_its": [s["newton_its"] for s in st], "oracle_newton_its": [s["newton_its"] for s in sref],
            "gmres_its": [s["gmres_its"] for s in st], "oracle_gmres_its": [s["gmres_its"] for s in sref]})
    # the same steps were taken
    for a, b in zip(st, sref):
        assert abs(a["dt"] - b["dt"]) <= 1e-7 * b["dt"]
    open_keys = WEDGE_VELOCITY if name.startswith("wedge") else ()
    if open_keys:
        _, _, dconv = oracle_run(name, 1e-11)
        for k in open_keys:
            own = abs(dref[k] - dconv[k])  # the oracle's distance to its converged root
            err = abs(d[k] - dref[k])
            report({"config": name, "precision": prec, "diag": k, "abs_err": err, "oracle_own_abs_err": own,
                    "oracle_own_rel_err": own / abs(dconv[k])})
            if prec == "fp64":
                assert err <= max(rtol * abs(dref[k]), 1e-14), (k, err)
            else:
                assert err <= 0.1 * own, (k, err, own)
    else:
        assert rel[key] <= rtol, (key, rel[key])
    for k in dref:
        if k in open_keys:
            continue
        assert abs(d[k] - dref[k]) <= rtol * (abs(dref[k]) + 1e-3), (k, d[k], dref[k])
