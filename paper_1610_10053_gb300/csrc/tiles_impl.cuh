// Definitions behind tiles.h; included once per tile shape by tiles_*.cu,
// which instantiate fused2d_apply_t / precond2d_apply_t for that shape.
#pragma once
#include "tile_jvdiff.cuh"
#include "tile_precond.cuh"
#include "tile_stencil.cuh"
#include "tiles.h"

namespace {

using namespace tile;

template <int MODE, typename VIN, typename VOUT, int TX, int TY>
__global__ void __launch_bounds__(TX *TY) k_fused2d(GridParams P, const double *U, const double *aux,
                                                    const VIN *v, VOUT *out, double *RU_out, double hdt,
                                                    double sign, const double *eps, double *Fr_out, float *lin,
                                                    double *Cn_out)
{
    pdl_entry();
    extern __shared__ double sm[];
    const double epsv = (MODE == SM_JV) ? *eps : 0.0;
    fused2d_tile<MODE, VIN, VOUT, TX, TY>(P, U, aux, v, out, RU_out, call_hdt(P, hdt), sign, epsv, blockIdx.x,
                                          blockIdx.y, sm, Fr_out, lin, Cn_out);
}

template <int MODE, typename VIN, typename VOUT, int TX, int TY>
int launch_fused2d(music_grid *g, const double *U, const double *aux, const VIN *v, VOUT *out, double *RU_out,
                   double hdt, double sign, cudaStream_t s)
{
    using TL = Tile2D<TX, TY>;
    static std::atomic<uint64_t> attr{0};
    auto kern = k_fused2d<MODE, VIN, VOUT, TX, TY>;
    TRY(allow_dynamic_smem(kern, TL::SMEM, attr));
    const GridParams &P = g->P;
    dim3 grid((P.n[0] + TX - 1) / TX, (P.n[1] + TY - 1) / TY);
    // R and F evaluations refresh the difference-form Jv's linearisation planes
    float *lin = (MODE != SM_JV && MODE != SM_CN && g->jv_form == JV_DIFF) ? g->lin : nullptr;
    // SM_CNF writes the step constant into aux
    double *cn = (MODE == SM_CNF) ? const_cast<double *>(aux) : nullptr;
    kern<<<grid, TX * TY, TL::SMEM, s>>>(P, U, MODE == SM_CNF ? nullptr : aux, v, out, RU_out, hdt, sign,
                                         &g->ds->eps, MODE == SM_JV ? nullptr : g->fr_capture, lin, cn);
    CHECK_LAUNCH();
    return MUSIC_OK;
}

// Jv in difference form (tile_jvdiff.cuh): FP32 Krylov vectors in and out.
// At least 1024 resident threads per SM (64 registers a thread).
template <int TX, int TY>
__global__ void __launch_bounds__(TX *TY, (TX * TY >= 1024) ? 1 : 1024 / (TX * TY)) k_jvdiff2d(GridParams P, JvConst K, const double *U, const float *lin,
                                                     const float *v, float *out, double hdt, const double *eps)
{
    pdl_entry();
    extern __shared__ double sm[];
    jvdiff2d_tile<float, float, TX, TY>(P, K, U, lin, v, out, hdt, eps, blockIdx.x, blockIdx.y, sm);
}

template <int TX, int TY>
int launch_jvdiff2d(music_grid *g, const double *U, const float *v, float *out, double hdt, cudaStream_t s)
{
    using TL = JvTile<TX, TY>;
    static std::atomic<uint64_t> attr{0};
    auto kern = k_jvdiff2d<TX, TY>;
    TRY(allow_dynamic_smem(kern, TL::SMEM, attr));
    const GridParams &P = g->P;
    dim3 grid((P.n[0] + TX - 1) / TX, (P.n[1] + TY - 1) / TY);
    const JvConst K{(float)P.idx[0], (float)P.idx[1], (float)P.gm1, (float)P.g[0], (float)P.g[1]};
    kern<<<grid, TX * TY, TL::SMEM, s>>>(P, K, U, g->lin, v, out, hdt, &g->ds->eps);
    CHECK_LAUNCH();
    return MUSIC_OK;
}

// Two 1024-thread CTAs of a single-precision stage whose shared memory is
// under half an SM's fit one SM once a thread holds at most 32 registers:
// the 16 x 16 launches of a 512^2 grid then run in one wave.
template <typename PT, int KM, int TX, int TY>
constexpr int pc_min_blocks()
{
    constexpr size_t smem = (size_t)pc_planes<PT, KM, TX, TY>() * (TX + 2 * (KM + 1)) * (TY + 2 * (KM + 1)) *
                                sizeof(PT) + TX * TY * sizeof(double);
    return sizeof(PT) == 4 && TX * TY == 1024 && smem <= 100 * 1024 ? 2 : 1;
}

// The application z = M^-1 r in one kernel, or in a few (stages) with a
// shallower halo each: a CTA owns a TX x TY tile and stages the frozen
// coefficients and r (or, after the first stage, the right-hand side and dp)
// on the tile plus a halo of H = KM + 1 cells (KM >= the stage's sweeps, a
// compile-time size so that all tile index arithmetic is by constants).  The
// right-hand side, the stage's Jacobi sweeps (sweep k is computed on the
// staged region shrunk by k cells, which is exactly where it equals the
// global iterate) and, in the last stage, the back substitution all run in
// shared memory.  One stage reads r and writes z once; more stages trade a
// global write and read of the right-hand side and dp per stage for less
// redundant halo work.  |z|^2 is reduced on the tile-independent
// decomposition, and the last block finishes it and the finite-difference
// step of the Jv that follows.
// With sc (the solver graph's control), the input is r * sc->inv and the
// first stage writes it to basis vector sc->scale_idx of Vb (nV entries each).
template <typename PT, int KM, int TX, int TY, bool FIRST, bool LAST>
__global__ void __launch_bounds__(TX *TY, pc_min_blocks<PT, KM, TX, TY>()) k_precond_fused2d(GridParams P, PC<PT> C, const PT *r, PT *z, PT tau,
                                                             PT tau2, int K, double *partial, DevScalars *ds,
                                                             PT *bg, const PT *dpin, PT *dpout, const SolveCtl *sc,
                                                             PT *Vb, long long nV)
{
    pdl_entry();
    extern __shared__ unsigned char smraw[];
    __shared__ double buf[TX * TY];
    PT rs = (PT)1;
    PT *vout = nullptr;
    if (sc) {
        rs = (PT)sc->inv;
        if (FIRST) vout = Vb + (long long)sc->scale_idx * nV;
    }
    const double nrm = precond2d_tile<PT, KM, TX, TY, FIRST, LAST>(P, C, r, z, tau, tau2, K, blockIdx.x,
                                                                   blockIdx.y, smraw, bg, dpin, dpout, rs, vout);
    if (LAST && partial) {
        norm_partials<TX, TY>(P, nrm, blockIdx.x, blockIdx.y, partial, buf);
        if (last_block_done(&ds->counters[CNT_PRECOND])) {
            sum_partials_fixed(partial, norm_partial_count(P), &ds->vnorm2, buf);
            if (threadIdx.x == 0) ds->eps = fd_eps(ds->unorm2, ds->vnorm2);
        }
    }
}

template <typename PT, int KM, int TX, int TY, bool FIRST, bool LAST>
int launch_pc_stage(music_grid *g, double dt, const PT *r, PT *z, int K, int want_norm, PT *dpin, PT *dpout,
                    cudaStream_t s)
{
    constexpr int H = KM + 1;
    constexpr size_t smem = (size_t)pc_planes<PT, KM, TX, TY>() * (TX + 2 * H) * (TY + 2 * H) * sizeof(PT);
    auto kern = k_precond_fused2d<PT, KM, TX, TY, FIRST, LAST>;
    static std::atomic<uint64_t> attr{0};
    TRY(allow_dynamic_smem(kern, smem, attr));
    const GridParams &P = g->P;
    const double tau = 0.5 * dt;
    dim3 grid((P.n[0] + TX - 1) / TX, (P.n[1] + TY - 1) / TY);
    PC<PT> C;
    for (int d = 0; d < 3; d++) C.a[d] = (PT *)g->pa[d];
    C.gp = (PT *)g->pgp;
    C.hp = (PT *)g->php;
    C.D = (PT *)g->pD;
    kern<<<grid, TX * TY, smem, s>>>(P, C, r, z, (PT)tau, (PT)(tau * tau), K, want_norm ? g->partials : nullptr,
                                     g->ds, (PT *)g->pb, dpin, dpout, g->pc_scale, (PT *)g->V, (long long)g->n);
    CHECK_LAUNCH();
    return MUSIC_OK;
}

// the K sweeps in `stages` launches of ceil(K / stages) sweeps (the last may
// have fewer); one stage takes KM = the smallest of 4, 8, 12, 16 covering K,
// split stages 4 or 8
template <typename PT, int TX, int TY>
int apply_fused2d(music_grid *g, double dt, const PT *r, PT *z, int want_norm, int stages, cudaStream_t s)
{
    const int K = g->desc.precond_sweeps;
    if ((stages <= 1 || K < 2) && K <= 16) {
        if (K <= 4) return launch_pc_stage<PT, 4, TX, TY, true, true>(g, dt, r, z, K, want_norm, 0, 0, s);
        if (K <= 8) return launch_pc_stage<PT, 8, TX, TY, true, true>(g, dt, r, z, K, want_norm, 0, 0, s);
        if (K <= 12) return launch_pc_stage<PT, 12, TX, TY, true, true>(g, dt, r, z, K, want_norm, 0, 0, s);
        return launch_pc_stage<PT, 16, TX, TY, true, true>(g, dt, r, z, K, want_norm, 0, 0, s);
    }
    const int d = (K + stages - 1) / stages;
    if (d > 8) {
        set_error("preconditioner: %d stages of %d sweeps exceed the staged halo", stages, d);
        return MUSIC_E_INVAL;
    }
    PT *buf[2] = {(PT *)g->pdp, (PT *)g->pdq};
    int done = 0, st = 0;
    while (done < K) {
        const int k = (K - done < d) ? K - done : d;
        const bool first = (done == 0), last = (done + k == K);
        PT *in = buf[(st + 1) & 1], *out = buf[st & 1];
        if (d <= 4) {
            if (first)
                TRY((launch_pc_stage<PT, 4, TX, TY, true, false>(g, dt, r, z, k, 0, nullptr, out, s)));
            else if (last)
                TRY((launch_pc_stage<PT, 4, TX, TY, false, true>(g, dt, r, z, k, want_norm, in, nullptr, s)));
            else
                TRY((launch_pc_stage<PT, 4, TX, TY, false, false>(g, dt, r, z, k, 0, in, out, s)));
        } else {
            if (first)
                TRY((launch_pc_stage<PT, 8, TX, TY, true, false>(g, dt, r, z, k, 0, nullptr, out, s)));
            else if (last)
                TRY((launch_pc_stage<PT, 8, TX, TY, false, true>(g, dt, r, z, k, want_norm, in, nullptr, s)));
            else
                TRY((launch_pc_stage<PT, 8, TX, TY, false, false>(g, dt, r, z, k, 0, in, out, s)));
        }
        done += k;
        st++;
    }
    return MUSIC_OK;
}

}  // namespace

template <int TX, int TY>
int fused2d_apply_t(music_grid *g, int mode, const double *U, const double *aux, const void *v, int vin_double,
                    void *out, int out_double, double *RU_out, double hdt, double sign, cudaStream_t s)
{
    switch (mode) {
    case SM_R:
        return launch_fused2d<SM_R, double, double, TX, TY>(g, U, aux, nullptr, (double *)out, nullptr, hdt, sign,
                                                            s);
    case SM_CN:
        return launch_fused2d<SM_CN, double, double, TX, TY>(g, U, aux, nullptr, (double *)out, nullptr, hdt,
                                                             sign, s);
    case SM_F:
        return launch_fused2d<SM_F, double, double, TX, TY>(g, U, aux, nullptr, (double *)out, RU_out, hdt, sign,
                                                            s);
    case SM_CNF:
        return launch_fused2d<SM_CNF, double, double, TX, TY>(g, U, aux, nullptr, (double *)out, RU_out, hdt,
                                                              sign, s);
    case SM_JV:
        if (vin_double && out_double)
            return launch_fused2d<SM_JV, double, double, TX, TY>(g, U, aux, (const double *)v, (double *)out,
                                                                 nullptr, hdt, sign, s);
        if (!vin_double && !out_double && g->jv_form == JV_DIFF)
            return launch_jvdiff2d<TX, TY>(g, U, (const float *)v, (float *)out, hdt, s);
        if (!vin_double && !out_double)
            return launch_fused2d<SM_JV, float, float, TX, TY>(g, U, aux, (const float *)v, (float *)out, nullptr,
                                                               hdt, sign, s);
        if (vin_double)
            return launch_fused2d<SM_JV, double, float, TX, TY>(g, U, aux, (const double *)v, (float *)out,
                                                                nullptr, hdt, sign, s);
        return launch_fused2d<SM_JV, float, double, TX, TY>(g, U, aux, (const float *)v, (double *)out, nullptr,
                                                            hdt, sign, s);
    }
    set_error("stencil: bad mode %d", mode);
    return MUSIC_E_INVAL;
}

template <int TX, int TY>
int precond2d_apply_t(music_grid *g, double dt, const void *r, void *z, int want_norm, cudaStream_t s)
{
    if (!pc_fits(TileShape{TX, TY}, g->desc.precond_sweeps, g->psplit, g->mixed ? 4 : 8)) {
        set_error("preconditioner: %dx%d tiles in %d stage(s) exceed the shared memory of a CTA", TX, TY, g->psplit);
        return MUSIC_E_INVAL;
    }
    if (g->mixed)
        return apply_fused2d<float, TX, TY>(g, dt, (const float *)r, (float *)z, want_norm, g->psplit, s);
    return apply_fused2d<double, TX, TY>(g, dt, (const double *)r, (double *)z, want_norm, g->psplit, s);
}
