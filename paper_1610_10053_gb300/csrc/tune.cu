// Autotuner of the fused 2-D kernels' tile shapes (the stencil's Jv mode and
// its R / C^n / F modes separately, the preconditioner), of the halo depth
// of the fused preconditioner (its sweeps in 1, 2 or 4 launches) and of the
// persistent batched kernel's tile shape (small grids).  The paper's
// code ran on CPUs; this has no counterpart there.  Every candidate computes
// the same result bitwise (tiles.h), so the choice is by speed alone: each is
// timed with CUDA events on the grid's own state, the median of a few
// launches taken, and the fastest kept for the grid and for every later grid
// of the same configuration (extent, boundaries, precision, Jv form, sweeps) in this
// process.
#include <algorithm>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <tuple>

#include "internal.h"
#include "tile_precond.cuh"
#include "tiles.h"

namespace {

using Key = std::tuple<int, int, int, int, int, int, int>;

std::mutex g_tune_mu;
struct Choice {
    int stile, rtile, ptile, psplit, btile, btimed;  // btimed: the batched shapes were timed
};
std::map<Key, Choice> g_tune_cache;  // -> stencil tiles (Jv, residual), preconditioner tile and stages

bool fused_grid(const music_grid *g)
{
    return g->P.nd == 2 && g->stencil_variant != STENCIL_MULTIPASS && !general_grid(g->P);
}

bool fused_precond(const music_grid *g)
{
    return fused_grid(g) && g->desc.precond != MUSIC_PC_NONE && g->desc.precond_sweeps <= tile::PC_STAGED_MAXK &&
           g->pc_variant != PC_MULTIKERNEL;
}

Key key_of(const music_grid *g)
{
    return Key(g->P.n[0], g->P.n[1], g->P.bc[0], g->P.bc[1], g->mixed + 2 * g->jv_form, g->desc.precond_sweeps,
               g->desc.precond);
}

constexpr int WARM = 2, REPS = 5;

// median launch time in microseconds of `launch` on stream s
template <typename F>
int time_median(cudaStream_t s, cudaEvent_t *ev, F &&launch, double *us)
{
    for (int i = 0; i < WARM; i++) TRY(launch());
    float t[REPS];
    for (int i = 0; i < REPS; i++) {
        CUDA_TRY(cudaEventRecord(ev[2 * i], s));
        TRY(launch());
        CUDA_TRY(cudaEventRecord(ev[2 * i + 1], s));
    }
    CUDA_TRY(cudaEventSynchronize(ev[2 * REPS - 1]));
    for (int i = 0; i < REPS; i++) CUDA_TRY(cudaEventElapsedTime(&t[i], ev[2 * i], ev[2 * i + 1]));
    std::sort(t, t + REPS);
    *us = 1e3 * (double)t[REPS / 2];
    return MUSIC_OK;
}

struct Events {
    cudaEvent_t ev[2 * REPS] = {};
    ~Events()
    {
        for (cudaEvent_t e : ev)
            if (e) cudaEventDestroy(e);
    }
    int make()
    {
        for (cudaEvent_t &e : ev) CUDA_TRY(cudaEventCreate(&e));
        return MUSIC_OK;
    }
};

int tune(music_grid *g, double dt, music_tune_report *rep, cudaStream_t s)
{
    Events E;
    TRY(E.make());
    const int kd = !g->mixed;
    // R(U) for the products, coefficients at U, |U| for eps, and a Krylov-type
    // right-hand side (R(U) cast) for the preconditioner
    TRY(stencil_apply(g, SM_R, g->U, nullptr, nullptr, 1, g->RU, 1, nullptr, dt, 1.0, s));
    TRY(dev_norm2(g, g->U, 1, g->n, &g->ds->unorm2, s));
    TRY(vec_cast_copy(g->RU, 1, g->w, kd, g->n, s));
    int best_p = g->ptile, best_q = g->psplit;
    if (fused_precond(g)) {
        TRY(precond_setup(g, g->U, dt, s));
        double best = 1e300;
        int nc = 0;
        for (int p = 0; p < N_PRECOND_TILES; p++) {
            for (int q = 0; q < N_PRECOND_SPLITS; q++) {
                if (!split_ok(g->desc.precond_sweeps, PRECOND_SPLITS[q])) continue;
                if (!pc_fits(PRECOND_TILES[p], g->desc.precond_sweeps, PRECOND_SPLITS[q], g->mixed ? 4 : 8)) continue;
                g->ptile = p;
                g->psplit = PRECOND_SPLITS[q];
                double us = 0.0;
                TRY(time_median(s, E.ev, [&] { return precond_apply(g, dt, g->w, g->z, 1, s); }, &us));
                rep->precond_cand[nc][0] = PRECOND_TILES[p].x;
                rep->precond_cand[nc][1] = PRECOND_TILES[p].y;
                rep->precond_cand[nc][2] = PRECOND_SPLITS[q];
                rep->precond_us[nc] = us;
                nc++;
                if (us < best) {
                    best = us;
                    best_p = p;
                    best_q = PRECOND_SPLITS[q];
                }
            }
        }
        rep->n_precond = nc;
        g->ptile = best_p;
        g->psplit = best_q;
    } else {
        TRY(vec_cast_copy(g->RU, 1, g->z, kd, g->n, s));
    }
    // the input of the timed products: z (M^-1 R(U), or R(U)) with its eps
    TRY(dev_norm2(g, g->z, kd, g->n, &g->ds->vnorm2, s));
    TRY(dev_set_eps(g, 0.0, s));
    double best = 1e300;
    int best_s = g->stile;
    for (int t = 0; t < N_STENCIL_TILES; t++) {
        g->stile = t;
        double us = 0.0;
        TRY(time_median(s, E.ev, [&] {
            return stencil_apply(g, SM_JV, g->U, g->RU, g->z, kd, g->u, kd, nullptr, dt, 1.0, s);
        }, &us));
        rep->stencil_cand[t][0] = STENCIL_TILES[t].x;
        rep->stencil_cand[t][1] = STENCIL_TILES[t].y;
        rep->stencil_us[t] = us;
        if (us < best) {
            best = us;
            best_s = t;
        }
    }
    rep->n_stencil = N_STENCIL_TILES;
    g->stile = best_s;
    // the R / C^n / F modes (FP64) on their own: F at U with R(U) standing
    // in for C^n, into scratch (R(U) and the linearisation planes are
    // rewritten with the same values)
    best = 1e300;
    int best_r = g->rtile;
    for (int t = 0; t < N_STENCIL_TILES; t++) {
        g->rtile = t;
        double us = 0.0;
        TRY(time_median(s, E.ev, [&] {
            return stencil_apply(g, SM_F, g->U, g->RU, nullptr, 1, g->t64, 1, g->RU, dt, -1.0, s);
        }, &us));
        rep->residual_us[t] = us;
        if (us < best) {
            best = us;
            best_r = t;
        }
    }
    g->rtile = best_r;
    return MUSIC_OK;
}

// The batched kernel's tile: one batched step of this grid alone per
// candidate (a batched step runs the whole grid on one SM, so the grid's
// latency on one SM is what the shape changes), from the same state each
// time; the step size is dt (cfl left unbounded, dt_max = dt).
int tune_batch(music_grid *g, double dt, music_tune_report *rep, cudaStream_t s)
{
    Events E;
    TRY(E.make());
    double best = 1e300;
    if (batchable(g) && g->P.N <= BATCH_TUNE_MAX_CELLS) {
        const size_t bytes = g->n * sizeof(double);
        double *U0 = nullptr;
        CUDA_TRY(cudaMallocAsync((void **)&U0, bytes, s));
        int rc = MUSIC_OK;
        if (cudaMemcpyAsync(U0, g->U, bytes, cudaMemcpyDeviceToDevice, s) != cudaSuccess) {
            cudaGetLastError();
            set_error("music_autotune: state copy failed");
            rc = MUSIC_E_CUDA;
        }
        const double cfl = 1e300, dtm = dt;
        music_grid *one[1] = {g};
        best = 1e300;
        int best_b = g->btile;
        for (int t = 0; t < N_BATCH_TILES && rc == MUSIC_OK; t++) {
            double us = 0.0;
            rc = time_median(s, E.ev, [&]() -> int {
                CUDA_TRY(cudaMemcpyAsync(g->U, U0, bytes, cudaMemcpyDeviceToDevice, s));
                return batch_launch(one, 1, &cfl, &dtm, t, s);
            }, &us);
            rep->batch_cand[t][0] = BATCH_TILES[t].x;
            rep->batch_cand[t][1] = BATCH_TILES[t].y;
            rep->batch_us[t] = us;
            if (us < best) {
                best = us;
                best_b = t;
            }
        }
        if (rc == MUSIC_OK) {
            rep->n_batch = N_BATCH_TILES;
            g->btile = best_b;
        }
        if (cudaMemcpyAsync(g->U, U0, bytes, cudaMemcpyDeviceToDevice, s) != cudaSuccess && rc == MUSIC_OK) {
            cudaGetLastError();
            set_error("music_autotune: state restore failed");
            rc = MUSIC_E_CUDA;
        }
        cudaFreeAsync(U0, s);
        if (cudaStreamSynchronize(s) != cudaSuccess && rc == MUSIC_OK) {
            cudaGetLastError();
            set_error("music_autotune: batched timing failed");
            rc = MUSIC_E_CUDA;
        }
        TRY(rc);
    }
    return MUSIC_OK;
}

int tile_index(const TileShape *tab, int n, const int *xy)
{
    for (int i = 0; i < n; i++)
        if (tab[i].x == xy[0] && tab[i].y == xy[1]) return i;
    return -1;
}

// MUSIC_TILES=<Jv>,<residual>,<preconditioner>,<stages>, e.g.
// 32x16,16x16,64x16,1, pins the choice instead of timing the candidates (a
// profiler slows every launch, so a tuner run under it picks at random):
// true when the variable names valid candidates for this grid
bool pinned_tiles(music_grid *g)
{
    const char *e = getenv("MUSIC_TILES");
    if (!e) return false;
    int a[2], b[2], c[2], q;
    if (sscanf(e, "%dx%d,%dx%d,%dx%d,%d", &a[0], &a[1], &b[0], &b[1], &c[0], &c[1], &q) != 7) return false;
    const int st = tile_index(STENCIL_TILES, N_STENCIL_TILES, a), rt = tile_index(STENCIL_TILES, N_STENCIL_TILES, b);
    const int pt = tile_index(PRECOND_TILES, N_PRECOND_TILES, c);
    bool q_ok = false;
    for (int i = 0; i < N_PRECOND_SPLITS; i++) q_ok |= (PRECOND_SPLITS[i] == q);
    if (st < 0 || rt < 0 || pt < 0 || !q_ok || !split_ok(g->desc.precond_sweeps, q) ||
        !pc_fits(PRECOND_TILES[pt], g->desc.precond_sweeps, q, g->mixed ? 4 : 8))
        return false;
    g->stile = st;
    g->rtile = rt;
    g->ptile = pt;
    g->psplit = q;
    return true;
}

}  // namespace

void tune_lookup(music_grid *g)
{
    if (!fused_grid(g)) return;
    std::lock_guard<std::mutex> lk(g_tune_mu);
    auto it = g_tune_cache.find(key_of(g));
    if (it == g_tune_cache.end()) return;
    g->stile = it->second.stile;
    g->rtile = it->second.rtile;
    g->ptile = it->second.ptile;
    g->psplit = it->second.psplit;
    g->btile = it->second.btile;
}

bool batch_tunable(const music_grid *g) { return batchable(g) && g->P.N <= BATCH_TUNE_MAX_CELLS; }

extern "C" int music_autotune(music_grid *g, double dt, unsigned flags, music_tune_report *rep, void *stream)
{
    if (!g || !rep || !(dt > 0.0)) {
        set_error("music_autotune: need a grid, a report and dt > 0");
        return MUSIC_E_INVAL;
    }
    memset(rep, 0, sizeof(*rep));
    if (!fused_grid(g)) return MUSIC_OK;  // nothing to tune
    rep->tunable = 1;
    const int s0 = g->stile, r0 = g->rtile, p0 = g->ptile, q0 = g->psplit, b0 = g->btile;
    bool cached = false, btimed = false;
    if (!(flags & MUSIC_TUNE_FORCE)) {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        auto it = g_tune_cache.find(key_of(g));
        if (it != g_tune_cache.end()) {
            g->stile = it->second.stile;
            g->rtile = it->second.rtile;
            g->ptile = it->second.ptile;
            g->psplit = it->second.psplit;
            g->btile = it->second.btile;
            btimed = it->second.btimed;
            cached = true;
        }
    }
    const bool want_batch = (flags & MUSIC_TUNE_BATCH) && batch_tunable(g) && !btimed;
    int rc = MUSIC_OK;
    if (!cached) rc = pinned_tiles(g) ? MUSIC_OK : tune(g, dt, rep, (cudaStream_t)stream);
    if (rc == MUSIC_OK && want_batch) {
        rc = tune_batch(g, dt, rep, (cudaStream_t)stream);
        btimed = (rc == MUSIC_OK);
    }
    if (rc != MUSIC_OK) {
        g->stile = s0;
        g->rtile = r0;
        g->ptile = p0;
        g->psplit = q0;
        g->btile = b0;
        return rc;
    }
    if (!cached || want_batch) {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        g_tune_cache[key_of(g)] = Choice{g->stile, g->rtile, g->ptile, g->psplit, g->btile, btimed ? 1 : 0};
    }
    rep->from_cache = cached ? 1 : 0;
    rep->stencil_tile[0] = STENCIL_TILES[g->stile].x;
    rep->stencil_tile[1] = STENCIL_TILES[g->stile].y;
    rep->precond_tile[0] = PRECOND_TILES[g->ptile].x;
    rep->precond_tile[1] = PRECOND_TILES[g->ptile].y;
    rep->precond_stages = g->psplit;
    rep->residual_tile[0] = STENCIL_TILES[g->rtile].x;
    rep->residual_tile[1] = STENCIL_TILES[g->rtile].y;
    rep->batch_tile[0] = BATCH_TILES[g->btile].x;
    rep->batch_tile[1] = BATCH_TILES[g->btile].y;
    if (g->stile != s0 || g->rtile != r0 || g->ptile != p0 || g->psplit != q0)
        graph_release(g);  // recorded with the old ones
    return MUSIC_OK;
}

extern "C" int music_set_tiles(music_grid *g, const int *stencil_tile, const int *precond_tile, int precond_stages)
{
    if (!g) {
        set_error("music_set_tiles: grid is NULL");
        return MUSIC_E_INVAL;
    }
    int st = g->stile, pt = g->ptile, q = g->psplit;
    if (stencil_tile) st = tile_index(STENCIL_TILES, N_STENCIL_TILES, stencil_tile);
    if (precond_tile) pt = tile_index(PRECOND_TILES, N_PRECOND_TILES, precond_tile);
    if (precond_stages > 0) q = precond_stages;
    bool q_ok = false;
    for (int i = 0; i < N_PRECOND_SPLITS; i++) q_ok |= (PRECOND_SPLITS[i] == q);
    if (st < 0 || pt < 0 || !q_ok || !split_ok(g->desc.precond_sweeps, q) ||
        !pc_fits(PRECOND_TILES[pt], g->desc.precond_sweeps, q, g->mixed ? 4 : 8)) {
        set_error("music_set_tiles: not a candidate tile shape or stage count (or too large for shared memory)");
        return MUSIC_E_INVAL;
    }
    if (st != g->stile || (stencil_tile && st != g->rtile) || pt != g->ptile || q != g->psplit) graph_release(g);
    if (stencil_tile) g->rtile = st;
    g->stile = st;
    g->ptile = pt;
    g->psplit = q;
    return MUSIC_OK;
}

extern "C" int music_get_tiles(const music_grid *g, int *stencil_tile, int *precond_tile, int *precond_stages)
{
    if (!g || !stencil_tile || !precond_tile || !precond_stages) {
        set_error("music_get_tiles: NULL argument");
        return MUSIC_E_INVAL;
    }
    *precond_stages = g->psplit;
    stencil_tile[0] = STENCIL_TILES[g->stile].x;
    stencil_tile[1] = STENCIL_TILES[g->stile].y;
    precond_tile[0] = PRECOND_TILES[g->ptile].x;
    precond_tile[1] = PRECOND_TILES[g->ptile].y;
    return MUSIC_OK;
}
