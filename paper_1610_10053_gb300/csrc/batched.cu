// music_batch_step: many small grids advance one implicit step each in one
// launch of the persistent batched kernel (batched_impl.cuh), with the tile
// shape the first grid was tuned to (every shape gives the same bits).
#include "internal.h"
#include "tile_precond.cuh"
#include "tiles.h"

namespace batch {
template <typename KT, int KM, int TX, int TY>
int launch_batched(music_grid **grids, int count, const double *cfl, const double *dt_max, cudaStream_t s);
}

#define MUSIC_BATCHED_DECLARE(TX, TY)                                                                                    \
    extern template int batch::launch_batched<float, 16, TX, TY>(music_grid **, int, const double *, const double *,   \
                                                                 cudaStream_t);                                       \
    extern template int batch::launch_batched<float, 24, TX, TY>(music_grid **, int, const double *, const double *,   \
                                                                 cudaStream_t);                                       \
    extern template int batch::launch_batched<double, 16, TX, TY>(music_grid **, int, const double *, const double *,  \
                                                                  cudaStream_t);
MUSIC_BATCHED_DECLARE(32, 16)
MUSIC_BATCHED_DECLARE(16, 32)
MUSIC_BATCHED_DECLARE(64, 8)

namespace {

template <int TX, int TY>
int launch_shape(music_grid **grids, int count, const double *cfl, const double *dt_max, bool mixed, int km,
                 cudaStream_t s)
{
    if (km <= 16)
        return mixed ? batch::launch_batched<float, 16, TX, TY>(grids, count, cfl, dt_max, s)
                     : batch::launch_batched<double, 16, TX, TY>(grids, count, cfl, dt_max, s);
    // deeper halos in FP32 only (FP64 planes of that halo exceed shared memory; batchable)
    return batch::launch_batched<float, 24, TX, TY>(grids, count, cfl, dt_max, s);
}

}  // namespace

bool batchable(const music_grid *g)
{
    if (!g) return false;
    const int kmax = g->mixed ? tile::PC_BATCH_MAXK_F32 : tile::PC_FUSED_MAXK;
    return g->P.nd == 2 && !general_grid(g->P) && g->desc.precond_sweeps <= kmax && g->ns == 0;
}

int batch_launch(music_grid **grids, int count, const double *cfl, const double *dt_max, int tile, cudaStream_t s)
{
    int kmax = 0;
    for (int i = 0; i < count; i++)
        if (grids[i]->desc.precond_sweeps > kmax) kmax = grids[i]->desc.precond_sweeps;
    const bool mixed = grids[0]->mixed;
    switch (tile) {
    case 0:
        return launch_shape<32, 16>(grids, count, cfl, dt_max, mixed, kmax, s);
    case 1:
        return launch_shape<16, 32>(grids, count, cfl, dt_max, mixed, kmax, s);
    case 2:
        return launch_shape<64, 8>(grids, count, cfl, dt_max, mixed, kmax, s);
    }
    set_error("music_batch_step: bad batched tile index %d", tile);
    return MUSIC_E_INVAL;
}

extern "C" int music_batch_step(music_grid **grids, int count, const double *cfl, const double *dt_max,
                                music_step_stats *stats, void *stream)
{
    if (!grids || !cfl || count < 1 || count > MUSIC_BATCH_MAX) {
        set_error("music_batch_step: need 1..%d grids and their cfl values", MUSIC_BATCH_MAX);
        return MUSIC_E_INVAL;
    }
    for (int i = 0; i < count; i++)
        if (!(cfl[i] > 0.0)) {
            set_error("music_batch_step: cfl[%d] must be > 0", i);
            return MUSIC_E_INVAL;
        }
    for (int i = 0; i < count; i++) {
        music_grid *g = grids[i];
        if (!g) {
            set_error("music_batch_step: grid %d is NULL", i);
            return MUSIC_E_INVAL;
        }
        if (!batchable(g) || g->mixed != grids[0]->mixed) {
            set_error("music_batch_step: grid %d is not a batchable 2-D Cartesian grid of the batch's precision "
                      "(at most %d preconditioner sweeps)", i, tile::PC_FUSED_MAXK);
            return MUSIC_E_INVAL;
        }
        for (int k = 0; k < i; k++)
            if (grids[k] == g) {
                set_error("music_batch_step: grid %d appears twice", i);
                return MUSIC_E_INVAL;
            }
    }
    cudaStream_t s = (cudaStream_t)stream;
    TRY(batch_launch(grids, count, cfl, dt_max, grids[0]->btile, s));
    int worst = MUSIC_OK;
    for (int i = 0; i < count; i++) {
        music_grid *g = grids[i];
        CUDA_TRY(cudaMemcpyAsync(g->hs, g->ds, sizeof(DevScalars), cudaMemcpyDeviceToHost, s));
    }
    CUDA_TRY(cudaStreamSynchronize(s));
    for (int i = 0; i < count; i++) {
        const DevScalars *h = grids[i]->hs;
        if (stats) {
            music_step_stats &st = stats[i];
            memset(&st, 0, sizeof(st));
            st.dt = h->step_dt;
            st.newton_its = h->step_newton;
            st.gmres_its = h->step_gmres;
            st.dt_halvings = h->step_halvings;
            st.gmres_unconverged = h->step_unconverged;
            st.fnorm0 = h->step_fnorm0;
            st.fnorm = h->step_fnorm;
            st.max_drho = h->step_maxdrho;
        }
        if (h->step_status != MUSIC_OK && worst == MUSIC_OK) worst = h->step_status;
    }
    if (worst != MUSIC_OK) set_error("music_batch_step: at least one grid failed its step (see its stats)");
    return worst;
}

extern "C" int music_set_batch_tile(music_grid *g, const int *tile)
{
    if (!g || !tile) {
        set_error("music_set_batch_tile: NULL argument");
        return MUSIC_E_INVAL;
    }
    for (int i = 0; i < N_BATCH_TILES; i++)
        if (BATCH_TILES[i].x == tile[0] && BATCH_TILES[i].y == tile[1]) {
            g->btile = i;
            return MUSIC_OK;
        }
    set_error("music_set_batch_tile: %d x %d is not a batched tile shape", tile[0], tile[1]);
    return MUSIC_E_INVAL;
}

extern "C" int music_get_batch_tile(const music_grid *g, int *tile)
{
    if (!g || !tile) {
        set_error("music_get_batch_tile: NULL argument");
        return MUSIC_E_INVAL;
    }
    tile[0] = BATCH_TILES[g->btile].x;
    tile[1] = BATCH_TILES[g->btile].y;
    return MUSIC_OK;
}
