"""Tile shapes of the fused 2-D kernels, the halo depth of the fused
preconditioner (its sweeps in 1, 2 or 4 launches), and the autotuner that
picks them.

Every candidate must give bitwise identical results: the stencil's
arithmetic is per cell, every Jacobi sweep computes the same values however
the sweeps are split, and the preconditioner reduces |z|^2 on a fixed 16 x 8
block decomposition of the grid whatever its tile, so the Jacobian-free step
eps, and with it every later iterate, cannot depend on the choice.  The tests
use ragged grids (extents that no tile divides) with periodic and wall
boundaries.
"""
import itertools

import numpy as np
import pytest

from paper_1610_10053_gb300 import inputs as I

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

STENCIL = [(16, 8), (16, 16), (32, 8), (32, 16), (32, 32)]
PRECOND = [(16, 8), (16, 16), (32, 8), (32, 16), (64, 16), (32, 32)]
STAGES = [1, 2, 3, 4]


def split_ok(sweeps, q):
    """One launch takes at most 16 sweeps; a split at most 8 a stage, and at
    least one."""
    return sweeps <= 16 if q == 1 else (sweeps >= q and -(-sweeps // q) <= 8)


def fits(pt, q, prec, sweeps=16):
    """The fused preconditioner's stage fits a CTA's 227 KB of shared memory:
    6 planes of the tile plus a halo of (sweeps per stage bound) + 1, and the
    |z|^2 buffer (FP64 on 64 x 16 tiles needs two stages)."""
    km = (4 if sweeps <= 4 else 8 if sweeps <= 8 else 12 if sweeps <= 12 else 16) if q == 1 else \
        (4 if -(-sweeps // q) <= 4 else 8)
    h = km + 1
    es = 4 if prec == "MIXED" else 8
    return 6 * (pt[0] + 2 * h) * (pt[1] + 2 * h) * es + pt[0] * pt[1] * 8 + 256 <= 227 * 1024


def valid(pt, q, prec, sweeps):
    """A preconditioner tile and split the library accepts for the grid."""
    return split_ok(sweeps, q) and fits(pt, q, prec, sweeps)


def default_split(sweeps):
    return 1 if sweeps <= 16 else 3 if sweeps <= 24 else 4


def B():
    from paper_1610_10053_gb300 import binding
    return binding


def problems():
    return {
        "kh_ragged": I.kelvin_helmholtz(n=45, ny=37, seed=11, nsteps=2),
        "rt_ragged_walls": I.rayleigh_taylor(nx=21, ny=70, nsteps=2),
    }


@pytest.mark.parametrize("name", ["kh_ragged", "rt_ragged_walls"])
@pytest.mark.parametrize("prec", ["FP64", "MIXED"])
def test_operators_identical_for_every_tile(name, prec):
    p = problems()[name]
    rng = np.random.default_rng(5)
    kt = torch.float32 if prec == "MIXED" else torch.float64
    U = torch.from_numpy(p.U).cuda()
    Un = U * 0.999
    v = torch.from_numpy(rng.standard_normal(p.U.size)).cuda().to(kt)
    dt = 2e-3
    ref = None
    for st in STENCIL:
        with B().Grid(p, precision=getattr(B(), prec)) as g:
            g.set_tiles(stencil=st)
            assert g.tiles()[0] == st
            out = [g.spatial_operator(U), g.residual(U, Un, dt), g.jv(U, v, dt)]
            torch.cuda.synchronize()
            out = [t.cpu().numpy() for t in out]
        if ref is None:
            ref = out
        for a, b in zip(out, ref):
            assert np.array_equal(a, b), (name, prec, st)
    ref = None
    for pt, q in itertools.product(PRECOND, STAGES):
        with B().Grid(p, precision=getattr(B(), prec)) as g:
            if not valid(pt, q, prec, p.sweeps):
                with pytest.raises(B().MusicError):
                    g.set_tiles(precond=pt, stages=q)
                continue
            g.set_tiles(precond=pt, stages=q)
            assert g.tiles()[1:] == (pt, q)
            z = g.precond(U, dt, v)
            torch.cuda.synchronize()
            z = z.cpu().numpy()
        if ref is None:
            ref = z
        assert np.array_equal(z, ref), (name, prec, pt, q)


@pytest.mark.parametrize("name,prec", [("kh_ragged", "MIXED"), ("rt_ragged_walls", "FP64")])
def test_steps_identical_for_every_tile_pair(name, prec):
    """Whole implicit steps: eps comes from the preconditioner's |z|, so this
    also checks that the fused reduction does not depend on the tile."""
    p = problems()[name]
    ref = None
    first = {t: min(q for q in STAGES if valid(t, q, prec, p.sweeps)) for t in PRECOND}
    extra = [c for c in (((16, 8), (16, 8), 2), ((32, 16), (32, 8), 4), ((16, 16), (32, 16), 2),
                         ((32, 8), (16, 16), 3), ((32, 32), (32, 16), 4)) if valid(c[1], c[2], prec, p.sweeps)]
    assert len({q for _, _, q in extra} | set(first.values())) >= 2  # at least two splits compared
    for st, pt, q in [(s, t, first[t]) for s, t in itertools.product(STENCIL, PRECOND)] + extra:
        with B().Grid(p, precision=getattr(B(), prec)) as g:
            g.set_tiles(stencil=st, precond=pt, stages=q)
            g.set_state(p.U)
            stats = g.run()
            U = g.get_state()
        key = (U, [(s["newton_its"], s["gmres_its"], s["fnorm"]) for s in stats])
        if ref is None:
            ref = key
        assert np.array_equal(key[0], ref[0]), (name, st, pt, q)
        assert key[1] == ref[1], (name, st, pt, q)


def test_autotune_picks_a_candidate_and_caches_it():
    p = I.kelvin_helmholtz(n=96, ny=80, seed=12, nsteps=1)
    with B().Grid(p, precision=B().MIXED) as g:
        g.set_state(p.U)
        U0 = g.get_state()
        rep = g.autotune(force=True)
        assert rep["tunable"] == 1 and rep["from_cache"] == 0
        assert set(rep["stencil_us"]) == set(STENCIL)
        assert set(rep["precond_us"]) == {pt + (q,) for pt, q in itertools.product(PRECOND, STAGES)
                                          if valid(pt, q, "MIXED", p.sweeps)}
        assert all(t > 0.0 for t in rep["stencil_us"].values())
        assert all(t > 0.0 for t in rep["precond_us"].values())
        assert rep["stencil_tile"] == min(rep["stencil_us"], key=rep["stencil_us"].get)
        assert set(rep["residual_us"]) == set(STENCIL) and all(t > 0.0 for t in rep["residual_us"].values())
        assert rep["residual_tile"] == min(rep["residual_us"], key=rep["residual_us"].get)
        best = min(rep["precond_us"], key=rep["precond_us"].get)
        assert rep["precond_tile"] + (rep["precond_stages"],) == best
        assert g.tiles() == (rep["stencil_tile"], rep["precond_tile"], rep["precond_stages"])
        assert np.array_equal(g.get_state(), U0)  # tuning leaves the state alone
        g.step()
    # a new grid of the same configuration starts with the tuned shapes
    with B().Grid(p, precision=B().MIXED) as g2:
        assert g2.tiles() == (rep["stencil_tile"], rep["precond_tile"], rep["precond_stages"])
        g2.set_state(p.U)
        rep2 = g2.autotune()
        assert rep2["from_cache"] == 1 and rep2["stencil_tile"] == rep["stencil_tile"]
    # another precision is another configuration
    with B().Grid(p, precision=B().FP64) as g3:
        assert g3.tiles() == ((32, 16), (32, 16), default_split(p.sweeps))


def test_autotune_pinned_by_the_environment(monkeypatch):
    """MUSIC_TILES pins the tuner's choice (no timing); an invalid value is
    ignored and the candidates are timed."""
    p = I.kelvin_helmholtz(n=64, ny=48, seed=13, nsteps=1).with_options(sweeps=16)  # one launch allowed
    monkeypatch.setenv("MUSIC_TILES", "16x8,32x16,32x8,1")
    with B().Grid(p, precision=B().MIXED) as g:
        g.set_state(p.U)
        rep = g.autotune(force=True)
        assert rep["stencil_tile"] == (16, 8) and rep["residual_tile"] == (32, 16)
        assert rep["precond_tile"] == (32, 8) and rep["precond_stages"] == 1
        assert all(t == 0.0 for t in rep["stencil_us"].values())
        g.step()
    monkeypatch.setenv("MUSIC_TILES", "24x8,32x16,32x8,1")  # not a candidate
    with B().Grid(p, precision=B().MIXED) as g:
        g.set_state(p.U)
        rep = g.autotune(force=True)
        assert all(t > 0.0 for t in rep["stencil_us"].values())


def test_autotune_has_nothing_to_do_on_general_grids():
    p = I.taylor_green(n=12, nsteps=1)
    with B().Grid(p, precision=B().MIXED) as g:
        g.set_state(p.U)
        assert g.autotune()["tunable"] == 0


def test_set_tiles_rejects_other_shapes():
    p = I.kelvin_helmholtz(n=32, nsteps=1)
    with B().Grid(p, precision=B().MIXED) as g:
        with pytest.raises(B().MusicError) as e:
            g.set_tiles(stencil=(24, 8))
        assert e.value.code == 1
        with pytest.raises(B().MusicError):
            g.set_tiles(precond=(64, 32))
        with pytest.raises(B().MusicError):
            g.set_tiles(stages=5)


def test_stage_split_must_fit_the_staged_halo():
    """A split must give every stage at least one sweep and at most eight."""
    p = I.kelvin_helmholtz(n=32, nsteps=1).with_options(sweeps=3)
    with B().Grid(p, precision=B().MIXED) as g:
        g.set_tiles(stages=2)
        with pytest.raises(B().MusicError):
            g.set_tiles(stages=4)  # more stages than sweeps
    with B().Grid(p.with_options(sweeps=20), precision=B().MIXED) as g:
        with pytest.raises(B().MusicError):
            g.set_tiles(stages=2)  # 10 sweeps per stage
        g.set_tiles(stages=4)


def test_fp64_autotune_skips_what_does_not_fit_and_leaves_no_error():
    """An FP64 grid is never tuned onto a preconditioner stage larger than a
    CTA's shared memory, and a rejected setting leaves no CUDA error behind
    for the next call on the thread."""
    p = I.rayleigh_taylor(nx=24, ny=72, nsteps=1)
    with B().Grid(p, precision=B().FP64) as g:
        g.set_state(p.U)
        rep = g.autotune(force=True)
        assert (64, 16, 1) not in rep["precond_us"] and (64, 16, 2) in rep["precond_us"]
        with pytest.raises(B().MusicError):
            g.set_tiles(precond=(64, 16), stages=1)
        st = g.step()
        assert st["newton_its"] >= 1
