// Tile shapes of the fused 2-D kernels (residual / Jacobian-free product
// stencil and physics-based preconditioner) and their per-shape entry
// points.  Every shape computes the same arithmetic per cell, and the
// preconditioner's |z|^2 is reduced on a tile-independent decomposition, so
// all shapes give bitwise identical results; the autotuner (tune.cu) picks
// the fastest by timing.  Each shape is instantiated in its own translation
// unit (tiles_<TX>x<TY>.cu) so the library builds in parallel.
#pragma once
#include "internal.h"

struct TileShape {
    int x, y;
};

constexpr int N_STENCIL_TILES = 5, N_PRECOND_TILES = 6;
constexpr TileShape STENCIL_TILES[N_STENCIL_TILES] = {{16, 8}, {16, 16}, {32, 8}, {32, 16}, {32, 32}};
constexpr TileShape PRECOND_TILES[N_PRECOND_TILES] = {{16, 8}, {16, 16}, {32, 8}, {32, 16}, {64, 16}, {32, 32}};
constexpr int STENCIL_TILE_DEFAULT = 3, PRECOND_TILE_DEFAULT = 3;  // 32 x 16 both
// the preconditioner's K sweeps run in 1, 2 or 4 launches (halo depth K + 1,
// K/2 + 1 or K/4 + 1): one launch takes up to 16 sweeps, a split up to 8 per
// stage (so 17..32 sweeps need 4 stages)
constexpr int N_PRECOND_SPLITS = 4;
constexpr int PRECOND_SPLITS[N_PRECOND_SPLITS] = {1, 2, 3, 4};
inline bool split_ok(int sweeps, int stages)
{
    if (stages == 1) return sweeps <= 16;
    return sweeps >= stages && (sweeps + stages - 1) / stages <= 8;
}
// the split a grid starts with: the fewest launches the sweeps allow
inline int default_split(int sweeps) { return sweeps <= 16 ? 1 : sweeps <= 24 ? 3 : 4; }
// Shared memory of the widest stage of a fused preconditioner application
// (6 planes of the tile and its halo of KM + 1 cells, KM the stage's sweep
// bound, plus the |z|^2 buffer of TX*TY doubles) against the 227 KB a CTA
// may have: an FP64 single-stage application on 64 x 16 tiles does not fit.
constexpr size_t PC_SMEM_LIMIT = 227 * 1024;
inline bool pc_fits(TileShape t, int sweeps, int stages, size_t elem)
{
    int km;
    if (stages <= 1 || sweeps < 2)
        km = sweeps <= 4 ? 4 : sweeps <= 8 ? 8 : sweeps <= 12 ? 12 : 16;
    else
        km = (sweeps + stages - 1) / stages <= 4 ? 4 : 8;
    const size_t h = (size_t)km + 1;
    return 6 * (t.x + 2 * h) * (t.y + 2 * h) * elem + (size_t)t.x * t.y * sizeof(double) + 256 <= PC_SMEM_LIMIT;
}

// Tile shapes of the persistent batched kernel (music_batch_step).  Its CTA
// is one tile of 512 threads whatever the shape, so every CTA-wide sum runs
// in the same order and all shapes give bitwise identical results.
constexpr int N_BATCH_TILES = 3;
constexpr TileShape BATCH_TILES[N_BATCH_TILES] = {{32, 16}, {16, 32}, {64, 8}};
constexpr int BATCH_TILE_DEFAULT = 0;
// grids small enough for the autotuner to time a batched step of (a batched
// step runs a whole grid on one SM)
constexpr long long BATCH_TUNE_MAX_CELLS = 65536;
// a grid the batched kernel accepts: 2-D Cartesian, no radiative diffusion,
// at most 16 preconditioner sweeps, no passive scalars (batched.cu)
bool batchable(const music_grid *g);
// one batched step of `count` grids with batched tile `tile` (no read-back;
// grids must be batchable and share a precision; batched.cu)
int batch_launch(music_grid **grids, int count, const double *cfl, const double *dt_max, int tile, cudaStream_t s);

// fused 2-D stencil of one tile shape (same contract as stencil_apply's
// fused branch; hdt = dt / 2)
template <int TX, int TY>
int fused2d_apply_t(music_grid *g, int mode, const double *U, const double *aux, const void *v, int vin_double,
                    void *out, int out_double, double *RU_out, double hdt, double sign, cudaStream_t s);

// fused 2-D preconditioner of one tile shape: z = M^-1 r (Krylov type of the
// grid), with want_norm also |z|^2 -> ds->vnorm2 and the Jv step -> ds->eps
template <int TX, int TY>
int precond2d_apply_t(music_grid *g, double dt, const void *r, void *z, int want_norm, cudaStream_t s);

// the grid's shapes, by index into the tables above
int fused2d_dispatch(music_grid *g, int mode, const double *U, const double *aux, const void *v, int vin_double,
                     void *out, int out_double, double *RU_out, double hdt, double sign, cudaStream_t s);
int precond2d_dispatch(music_grid *g, double dt, const void *r, void *z, int want_norm, cudaStream_t s);
