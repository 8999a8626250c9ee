"""Persistent batched step (music_batch_step): many grids, one launch."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1610_10053_gb300 import inputs as I

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

from test_gpu_parity import B, diag_close  # noqa: E402


def problems(fp64=False):
    """Small RT and KH setups; in FP64 the KH ones at 16 sweeps (the batched
    kernel's FP64 limit; mixed takes their default 24)."""
    kh = (lambda p: p.with_options(sweeps=16)) if fp64 else (lambda p: p)
    return [I.rayleigh_taylor(nx=32, ny=96, nsteps=3), kh(I.kelvin_helmholtz(n=64, seed=3, nsteps=3)),
            kh(I.kelvin_helmholtz(n=40, ny=72, seed=4, nsteps=3)), I.rayleigh_taylor(nx=20, ny=60, nsteps=3)]


def run_batched(probs, prec, nsteps):
    grids = [B().Grid(p, precision=prec) for p in probs]
    for g, p in zip(grids, probs):
        g.set_state(p.U)
    stats = []
    for _ in range(nsteps):
        code, st = B().batch_step(grids)
        assert code == 0, B().last_error()
        stats.append(st)
    out = [(g.get_state(), g.diagnostics()) for g in grids]
    for g in grids:
        g.close()
    return out, stats


def test_batched_fp64_matches_oracle():
    probs = problems(fp64=True)
    out, stats = run_batched(probs, B().FP64, 3)
    for k, p in enumerate(probs):
        Uref, sref = O.run(p)
        dref = O.diagnostics(p, Uref)
        same = all(stats[s][k]["gmres_its"] == sref[s]["gmres_its"] for s in range(3))
        for s in range(3):
            assert stats[s][k]["newton_its"] == sref[s]["newton_its"]
        U, d = out[k]
        if not same:
            # a GMRES stopping test flipped by rounding: compare the two roots
            # at Newton tolerance 1e-11, where they no longer depend on the path
            p = p.with_options(newton_tol=1e-11, newton_max=20)
            Uref, _ = O.run(p)
            dref = O.diagnostics(p, Uref)
            (U, d), = run_batched([p], B().FP64, 3)[0]
        N = p.ncells
        for v in range(p.nvars):
            sl = slice(v * N, (v + 1) * N)
            assert np.abs(U[sl] - Uref[sl]).max() <= 1e-9 * (np.abs(Uref[sl]).max() + 1e-300), (k, v, same)
        diag_close(d, dref, 1e-9)


def test_batched_mixed_matches_oracle_diagnostics():
    probs = problems()
    out, _ = run_batched(probs, B().MIXED, 3)
    for k, p in enumerate(probs):
        Uref, _ = O.run(p)
        diag_close(out[k][1], O.diagnostics(p, Uref), 1e-6)


def test_batch_member_is_independent_of_the_batch():
    """A grid's step in a batch of one and in a batch of many is bitwise the
    same: every CTA works on its own grid only."""
    probs = problems()
    alone, _ = run_batched([probs[1]], B().MIXED, 2)
    mixed, _ = run_batched(probs, B().MIXED, 2)
    assert np.array_equal(alone[0][0], mixed[1][0])


def test_batch_rejects_unsupported_grids():
    p3 = I.taylor_green(n=8)
    with B().Grid(p3) as g3, B().Grid(problems()[0]) as g2:
        with pytest.raises(B().MusicError):
            B().batch_step([g2, g3])
    pc = I.random_smooth(2, (16, 16), seed=1).with_options(conduct=1, chi0=0.01)
    with B().Grid(pc) as gc:
        with pytest.raises(B().MusicError):
            B().batch_step([gc], cfl=[1.0])
    # more sweeps than the kernel's halo takes: 16 in FP64, 24 in mixed precision
    kh = I.kelvin_helmholtz(n=32, seed=1)
    with B().Grid(kh.with_options(sweeps=24), precision=B().FP64) as g64, \
            B().Grid(kh.with_options(sweeps=32), precision=B().MIXED) as g32:
        for g in (g64, g32):
            with pytest.raises(B().MusicError):
                B().batch_step([g])
    with B().Grid(kh.with_options(sweeps=24), precision=B().MIXED) as g24:
        g24.set_state(kh.U)
        code, _ = B().batch_step([g24])
        assert code == 0, B().last_error()


@pytest.mark.parametrize("prec", ["FP64", "MIXED"])
def test_batched_tile_shapes_give_the_same_bits(prec):
    """Every tile shape of the persistent batched kernel (a CTA of 512 threads
    whatever the shape) gives bitwise the same step."""
    probs = problems(fp64=(prec == "FP64"))
    out = {}
    for tile in ((32, 16), (16, 32), (64, 8)):
        grids = [B().Grid(p, precision=getattr(B(), prec)) for p in probs]
        for g, p in zip(grids, probs):
            g.set_state(p.U)
            g.set_batch_tile(tile)
            assert g.batch_tile() == tile
        for _ in range(2):
            code, st = B().batch_step(grids)
            assert code == 0, B().last_error()
        out[tile] = [g.get_state() for g in grids]
        for g in grids:
            g.close()
    ref = out[(32, 16)]
    for tile, states in out.items():
        for a, b in zip(states, ref):
            assert np.array_equal(a, b), tile


def test_autotune_picks_a_batched_tile_for_small_grids():
    """music_autotune with MUSIC_TUNE_BATCH times the batched kernel's shapes
    on a small grid (one batched step of it alone each, the state restored);
    without the flag, or on a grid too large for one SM, it leaves them."""
    p = I.kelvin_helmholtz(n=64, seed=31, nsteps=1)
    with B().Grid(p, precision=B().MIXED) as g:
        g.set_state(p.U)
        rep = g.autotune(force=True)
        assert rep["batch_us"] == {}
        rep = g.autotune(force=True, batch=True)
        assert set(rep["batch_us"]) == {(32, 16), (16, 32), (64, 8)}
        assert all(t > 0 for t in rep["batch_us"].values())
        assert rep["batch_tile"] == min(rep["batch_us"], key=rep["batch_us"].get)
        assert g.batch_tile() == rep["batch_tile"]
        assert np.array_equal(g.get_state(), p.U)  # tuning leaves the state alone
    big = I.kelvin_helmholtz(n=512, seed=31, nsteps=1)
    with B().Grid(big, precision=B().MIXED) as g:
        g.set_state(big.U)
        rep = g.autotune(force=True, batch=True)
        assert rep["batch_us"] == {} and rep["batch_tile"] == (32, 16)
    with B().Grid(p, precision=B().MIXED) as g:
        with pytest.raises(B().MusicError):
            g.set_batch_tile((8, 8))
