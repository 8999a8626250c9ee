// Persistent batched implicit step: many small grids advance one Crank-
// Nicolson step (Sec. 2: CFL time step, Newton, restarted right-preconditioned
// GMRES with Jacobian-free products) in a single launch.  The kernel is a
// template over its tile shape; each shape is instantiated in its own
// translation unit (batched_<TX>x<TY>.cu) and chosen by the autotuner.
//
// One CTA owns one grid for the whole step.  It walks the grid's tiles with
// the same per-tile stencil and preconditioner code as the one-kernel-per-
// operation path (tile_stencil.cuh, tile_precond.cuh); every reduction is a
// CTA-wide tree in a fixed order and the Hessenberg least-squares update runs
// in thread 0, so the step needs no host synchronisation and no grid-wide
// barrier.  Small grids (the 64^2 .. 128^2 solves of a serving mix) cannot
// fill the GPU alone; a batch of them fills it with one CTA per SM.
#pragma once
#include <cmath>
#include <vector>

#include "internal.h"
#include "tile_jvdiff.cuh"
#include "tile_precond.cuh"
#include "tile_stencil.cuh"

namespace {

using namespace tile;
// CTA size, the same for every tile shape (TX x TY = NT), so every CTA-wide
// reduction (strided by NT, then a fixed tree) runs in the same order and
// all shapes give the same bits
constexpr int NT = 512;

template <typename KT>
struct BInst {
    GridParams P;
    double *U, *Un, *Cn, *RU, *b, *x, *t64;
    KT *V, *w, *z, *u;
    PC<KT> pc;
    double *H, *cs, *sn, *gv, *yv;  // (m+1) x m Hessenberg, rotations, rhs, solution
    DevScalars *ds;
    int restart, max_restarts, newton_max, sweeps, max_halvings, precond;
    double rtol, newton_tol;
    float *lin;   // linearisation planes: FP32 products in difference form (tile_jvdiff.cuh), or null
};
static_assert(sizeof(BInst<double>) <= 1024, "descriptor must fit the grid's 1 KiB slot");

__device__ double cta_sum(double v, double *red)
{
    __shared__ double bc;
    const double r = block_sum<NT>(v, red);
    if (threadIdx.x == 0) bc = r;
    __syncthreads();
    const double o = bc;
    __syncthreads();
    return o;
}

__device__ double cta_max(double v, double *red)
{
    __shared__ double bc;
    const double r = block_max<NT>(v, red);
    if (threadIdx.x == 0) bc = r;
    __syncthreads();
    const double o = bc;
    __syncthreads();
    return o;
}

// <a, b> over n elements: FP32 products of FP32 vectors summed in FP32 over
// runs of 16 elements, then in FP64; FP64 vectors in FP64
template <typename KT>
__device__ double cta_dot(const KT *a, const KT *b, long long n, double *red)
{
    double s = 0.0;
    KT run = 0;
    int k = 0;
    for (long long e = threadIdx.x; e < n; e += NT) {
        run += a[e] * b[e];
        if (++k == 16) {
            s += (double)run;
            run = 0;
            k = 0;
        }
    }
    s += (double)run;
    return cta_sum(s, red);
}

template <int MODE, typename VIN, typename VOUT, int TX, int TY>
__device__ void stencil_all(const GridParams &P, const double *U, const double *aux, const VIN *v, VOUT *out,
                            double *RU_out, double hdt, double sign, double epsv, double *sm, float *lin = nullptr)
{
    const int ntx = (P.n[0] + TX - 1) / TX, nty = (P.n[1] + TY - 1) / TY;
    for (int t = 0; t < ntx * nty; t++) {
        fused2d_tile<MODE, VIN, VOUT, TX, TY>(P, U, aux, v, out, RU_out, hdt, sign, epsv, t % ntx, t / ntx, sm,
                                                nullptr, lin);
        __syncthreads();
    }
}

// Jv of an FP32 direction in difference form over all tiles of the grid, from
// the linearisation planes of the last F evaluation; eps in shared memory
template <int TX, int TY>
__device__ void jvdiff_all(const GridParams &P, const double *U, const float *lin, const float *v, float *out,
                           double hdt, const double *eps_sh, double *sm)
{
    const JvConst K{(float)P.idx[0], (float)P.idx[1], (float)P.gm1, (float)P.g[0], (float)P.g[1]};
    const int ntx = (P.n[0] + TX - 1) / TX, nty = (P.n[1] + TY - 1) / TY;
    for (int t = 0; t < ntx * nty; t++) {
        jvdiff2d_tile<float, float, TX, TY>(P, K, U, lin, v, out, hdt, eps_sh, t % ntx, t / ntx, sm);
        __syncthreads();
    }
}

// z = M^-1 r (or a copy without preconditioner); returns this thread's share
// of |z|^2, summed over the entries e = threadIdx.x + k NT whatever the tile
// shape (so the CTA-wide sum is the same for every shape)
template <typename KT, int KM, int TX, int TY>
__device__ double precond_all(const BInst<KT> &I, double dt, const KT *r, KT *z, unsigned char *sm)
{
    const GridParams &P = I.P;
    const long long n = (long long)P.nv * P.N;
    double nrm = 0.0;
    if (I.precond == MUSIC_PC_NONE) {
        for (long long e = threadIdx.x; e < n; e += NT) {
            z[e] = r[e];
            nrm += (double)r[e] * (double)r[e];
        }
        __syncthreads();
        return nrm;
    }
    const int ntx = (P.n[0] + TX - 1) / TX, nty = (P.n[1] + TY - 1) / TY;
    const double tau = 0.5 * dt;
    for (int t = 0; t < ntx * nty; t++)
        precond2d_tile<KT, KM, TX, TY, true, true, 0>(P, I.pc, r, z, (KT)tau, (KT)(tau * tau), I.sweeps, t % ntx,
                                                      t / ntx, sm);
    __syncthreads();
    for (long long e = threadIdx.x; e < n; e += NT) nrm += (double)z[e] * (double)z[e];
    return nrm;
}

// frozen preconditioner coefficients at U (same formulas as the per-grid setup)
template <typename KT>
__device__ void precond_setup_cta(const BInst<KT> &I, double dt)
{
    const GridParams &P = I.P;
    if (I.precond == MUSIC_PC_NONE) return;
    const double tau = 0.5 * dt;
    for (long long c = threadIdx.x; c < P.N; c += NT) {
        int ix[3];
        cell_coords(P, c, ix);
        const double E = I.U[P.N + c];
        I.pc.gp[c] = (KT)(P.gamma * (P.gm1 * E));
        I.pc.hp[c] = (KT)(P.gamma * E);
        for (int d = 0; d < 2; d++)
            I.pc.a[d][c] = lower_wall(P, ix, d) ? (KT)0
                                                : (KT)(1.0 / (0.5 * (I.U[cell_nb(P, ix, d, -1)] + I.U[c])));
    }
    __syncthreads();
    const KT tau2 = (KT)(tau * tau);
    for (long long c = threadIdx.x; c < P.N; c += NT) {
        int ix[3];
        cell_coords(P, c, ix);
        KT diag = 0;
        for (int d = 0; d < 2; d++) {
            const KT ap = upper_wall(P, ix, d) ? (KT)0 : I.pc.a[d][cell_nb(P, ix, d, +1)];
            diag += (ap + I.pc.a[d][c]) * (KT)P.idx2[d];
        }
        I.pc.D[c] = (KT)1 / I.pc.gp[c] + tau2 * diag;
    }
    __syncthreads();
}

// max over cells and directions of (|u| + c_s) / dx (Eq. 4)
__device__ double cfl_rate_cta(const GridParams &P, const double *U, double *red)
{
    double m = 0.0;
    for (long long c = threadIdx.x; c < P.N; c += NT) {
        int ix[3];
        cell_coords(P, c, ix);
        const double rho = U[c];
        const double cs = sqrt(P.gamma * (P.gm1 * U[P.N + c]) / rho);
        for (int d = 0; d < P.nd; d++) {
            double um = 0.0, up = 0.0;
            if (!lower_wall(P, ix, d)) um = U[(2 + d) * P.N + c] / (0.5 * (U[cell_nb(P, ix, d, -1)] + rho));
            if (!upper_wall(P, ix, d)) {
                const long long r = cell_nb(P, ix, d, +1);
                up = U[(2 + d) * P.N + r] / (0.5 * (rho + U[r]));
            }
            m = nanmax(m, (fabs(0.5 * (um + up)) + cs) * P.idx[d]);
        }
    }
    return cta_max(m, red);
}

struct GmresRes {
    int its, converged;
    double bnorm;
};

// right-preconditioned restarted GMRES on J x = b inside one CTA
template <typename KT, int KM, int TX, int TY>
__device__ GmresRes gmres_cta(const BInst<KT> &I, double dt, double unorm2, double *red, unsigned char *sm)
{
    const GridParams &P = I.P;
    const long long n = (long long)P.nv * P.N;
    const int m = I.restart;
    const double hdt = 0.5 * dt;
    __shared__ double sh_resid, sh_hn;
    __shared__ double sh_h[MUSIC_MAXV];
    __shared__ int sh_stop;
    GmresRes o{0, 0, 0.0};
    for (long long e = threadIdx.x; e < n; e += NT) I.x[e] = 0.0;
    double bb = 0.0;
    for (long long e = threadIdx.x; e < n; e += NT) bb += I.b[e] * I.b[e];
    const double bnorm = sqrt(cta_sum(bb, red));
    o.bnorm = bnorm;
    if (!(bnorm > 0.0) || !isfinite(bnorm)) {
        o.converged = (bnorm == 0.0);
        return o;
    }
    const double target = I.rtol * bnorm;
    double resid = bnorm;
    for (int cycle = 0; cycle <= I.max_restarts; cycle++) {
        double beta = bnorm;
        const double *r = I.b;
        if (cycle > 0) {
            // r = b - J x with J x in FP64 (eps from |U| and |x|)
            double xx = 0.0;
            for (long long e = threadIdx.x; e < n; e += NT) xx += I.x[e] * I.x[e];
            const double eps = fd_eps(unorm2, cta_sum(xx, red));
            stencil_all<SM_JV, double, double, TX, TY>(P, I.U, I.RU, I.x, I.t64, nullptr, hdt, 1.0, eps,
                                                       (double *)sm);
            double rr = 0.0;
            for (long long e = threadIdx.x; e < n; e += NT) {
                const double t = I.b[e] - I.t64[e];
                I.t64[e] = t;
                rr += t * t;
            }
            beta = sqrt(cta_sum(rr, red));
            r = I.t64;
        }
        resid = beta;
        if (beta <= target) {
            o.converged = 1;
            break;
        }
        for (long long e = threadIdx.x; e < n; e += NT) I.V[e] = (KT)(r[e] / beta);
        if (threadIdx.x == 0) {
            for (int i = 0; i <= m; i++) I.gv[i] = 0.0;
            I.gv[0] = beta;
        }
        __syncthreads();
        int k = 0;
        for (int j = 0; j < m; j++) {
            const KT *Vj = I.V + (long long)j * n;
            const double zz = cta_sum(precond_all<KT, KM, TX, TY>(I, dt, Vj, I.z, sm), red);
            const double eps = fd_eps(unorm2, zz);
            if constexpr (sizeof(KT) == 4) {
                if (I.lin) {
                    __shared__ double sh_eps;
                    if (threadIdx.x == 0) sh_eps = eps;
                    __syncthreads();
                    jvdiff_all<TX, TY>(P, I.U, I.lin, I.z, I.w, hdt, &sh_eps, (double *)sm);
                } else {
                    stencil_all<SM_JV, KT, KT, TX, TY>(P, I.U, I.RU, I.z, I.w, nullptr, hdt, 1.0, eps, (double *)sm);
                }
            } else {
                stencil_all<SM_JV, KT, KT, TX, TY>(P, I.U, I.RU, I.z, I.w, nullptr, hdt, 1.0, eps, (double *)sm);
            }
            // classical Gram-Schmidt, twice: all dots against the same w,
            // then one update
            for (int pass = 0; pass < 2; pass++) {
                for (int i = 0; i <= j; i++) {
                    const double hi = cta_dot<KT>(I.V + (long long)i * n, I.w, n, red);
                    if (threadIdx.x == 0) {
                        sh_h[i] = hi;
                        I.H[i * m + j] = (pass == 0) ? hi : I.H[i * m + j] + hi;
                    }
                }
                __syncthreads();
                for (long long e = threadIdx.x; e < n; e += NT) {
                    KT we = I.w[e];
                    for (int i = 0; i <= j; i++) we -= (KT)sh_h[i] * I.V[(long long)i * n + e];
                    I.w[e] = we;
                }
                __syncthreads();
            }
            const double hn = sqrt(cta_dot<KT>(I.w, I.w, n, red));
            if (threadIdx.x == 0) {
                double *H = I.H;
                H[(j + 1) * m + j] = hn;
                for (int i = 0; i < j; i++) {
                    const double t0 = H[i * m + j], t1 = H[(i + 1) * m + j];
                    H[i * m + j] = I.cs[i] * t0 + I.sn[i] * t1;
                    H[(i + 1) * m + j] = -I.sn[i] * t0 + I.cs[i] * t1;
                }
                const double a0 = H[j * m + j], a1 = H[(j + 1) * m + j];
                if (a1 == 0.0) {
                    I.cs[j] = 1.0;
                    I.sn[j] = 0.0;
                } else {
                    const double t = sqrt(a0 * a0 + a1 * a1);
                    I.cs[j] = a0 / t;
                    I.sn[j] = a1 / t;
                }
                H[j * m + j] = I.cs[j] * a0 + I.sn[j] * a1;
                H[(j + 1) * m + j] = 0.0;
                I.gv[j + 1] = -I.sn[j] * I.gv[j];
                I.gv[j] = I.cs[j] * I.gv[j];
                sh_resid = fabs(I.gv[j + 1]);
                sh_hn = hn;
                sh_stop = (hn == 0.0 || !isfinite(hn) || fabs(I.gv[j + 1]) <= target);
            }
            __syncthreads();
            o.its++;
            k = j + 1;
            resid = sh_resid;
            if (sh_stop) break;
            const KT inv = (KT)(1.0 / sh_hn);
            for (long long e = threadIdx.x; e < n; e += NT) I.V[(long long)(j + 1) * n + e] = I.w[e] * inv;
            __syncthreads();
        }
        if (threadIdx.x == 0) {
            for (int i = k - 1; i >= 0; i--) {
                double t = I.gv[i];
                for (int l = i + 1; l < k; l++) t -= I.H[i * m + l] * I.yv[l];
                I.yv[i] = t / I.H[i * m + i];
            }
        }
        __syncthreads();
        for (long long e = threadIdx.x; e < n; e += NT) {
            KT s = 0;
            for (int i = 0; i < k; i++) s += (KT)I.yv[i] * I.V[(long long)i * n + e];
            I.u[e] = s;
        }
        __syncthreads();
        precond_all<KT, KM, TX, TY>(I, dt, I.u, I.z, sm);
        for (long long e = threadIdx.x; e < n; e += NT) I.x[e] += (double)I.z[e];
        __syncthreads();
        if (!isfinite(resid)) break;
        if (resid <= target) {
            o.converged = 1;
            break;
        }
    }
    return o;
}

struct BArgs {
    const void *p[MUSIC_BATCH_MAX];  // device descriptors, one per CTA
    double cfl[MUSIC_BATCH_MAX];
    double dt_max[MUSIC_BATCH_MAX];
};

template <typename KT, int KM, int TX, int TY>
__global__ void __launch_bounds__(NT, 1) k_batched_step(const __grid_constant__ BArgs args)
{
    pdl_entry();
    static_assert(TX * TY == NT, "the CTA is one tile");
    extern __shared__ __align__(16) unsigned char sm[];
    __shared__ double red[NT / 32];
    const BInst<KT> &I = *(const BInst<KT> *)args.p[blockIdx.x];
    const GridParams &P = I.P;
    const long long n = (long long)P.nv * P.N;
    double dt = args.cfl[blockIdx.x] / cfl_rate_cta(P, I.U, red);
    const double dt_max = args.dt_max[blockIdx.x];
    if (dt_max > 0.0 && dt > dt_max) dt = dt_max;
    int status = MUSIC_E_NONFINITE, newton = 0, gmres = 0, halvings = 0, unconv = 0;
    double fnorm0 = 0.0, fnorm = 0.0, maxdrho = 0.0;
    if (isfinite(dt) && dt > 0.0) {
        status = MUSIC_E_NEWTON_FAIL;
        for (;;) {
            for (long long e = threadIdx.x; e < n; e += NT) I.Un[e] = I.U[e];
            __syncthreads();
            stencil_all<SM_CN, double, double, TX, TY>(P, I.Un, nullptr, nullptr, I.Cn, nullptr, 0.5 * dt, 1.0, 0.0,
                                               (double *)sm);
            newton = gmres = unconv = 0;
            int ok = 0;
            for (int k = 0; k < I.newton_max; k++) {
                stencil_all<SM_F, double, double, TX, TY>(P, I.U, I.Cn, nullptr, I.b, I.RU, 0.5 * dt, -1.0, 0.0,
                                                  (double *)sm, I.lin);
                double uu = 0.0;
                for (long long e = threadIdx.x; e < n; e += NT) uu += I.U[e] * I.U[e];
                const double unorm2 = cta_sum(uu, red);
                precond_setup_cta<KT>(I, dt);
                const GmresRes gr = gmres_cta<KT, KM, TX, TY>(I, dt, unorm2, red, sm);
                gmres += gr.its;
                unconv += !gr.converged;
                fnorm = gr.bnorm;
                if (k == 0) fnorm0 = fnorm;
                double mx = 0.0;
                for (long long e = threadIdx.x; e < n; e += NT) {
                    const double u = I.U[e] + I.x[e];
                    I.U[e] = u;
                    if (e < P.N) mx = nanmax(mx, fabs(I.x[e]) / u);
                }
                maxdrho = cta_max(mx, red);
                newton = k + 1;
                if (maxdrho <= I.newton_tol) {
                    ok = 1;
                    break;
                }
                if (!isfinite(maxdrho)) break;
            }
            if (ok) {
                status = MUSIC_OK;
                break;
            }
            for (long long e = threadIdx.x; e < n; e += NT) I.U[e] = I.Un[e];
            __syncthreads();
            if (halvings >= I.max_halvings || !isfinite(maxdrho)) break;
            dt *= 0.5;
            halvings++;
        }
    }
    if (threadIdx.x == 0) {
        DevScalars *ds = I.ds;
        ds->step_dt = dt;
        ds->step_status = status;
        ds->step_newton = newton;
        ds->step_gmres = gmres;
        ds->step_halvings = halvings;
        ds->step_unconverged = unconv;
        ds->step_fnorm0 = fnorm0;
        ds->step_fnorm = fnorm;
        ds->step_maxdrho = maxdrho;
    }
}

template <typename KT>
BInst<KT> make_inst(music_grid *g)
{
    BInst<KT> I;
    memset(&I, 0, sizeof(I));
    I.P = g->P;
    I.U = g->U;
    I.Un = g->Un;
    I.Cn = g->Cn;
    I.RU = g->RU;
    I.b = g->b;
    I.x = g->x;
    I.t64 = g->t64;
    I.V = (KT *)g->V;
    I.w = (KT *)g->w;
    I.z = (KT *)g->z;
    I.u = (KT *)g->u;
    for (int d = 0; d < 3; d++) I.pc.a[d] = (KT *)g->pa[d];
    I.pc.gp = (KT *)g->pgp;
    I.pc.hp = (KT *)g->php;
    I.pc.D = (KT *)g->pD;
    const int M = MUSIC_MAXV;
    I.H = g->hg;
    I.cs = g->hg + M * M;
    I.sn = I.cs + M;
    I.gv = I.sn + M;
    I.yv = I.gv + M;
    I.ds = g->ds;
    I.restart = g->desc.gmres_restart;
    I.max_restarts = g->desc.gmres_max_restarts;
    I.newton_max = g->desc.newton_max_its;
    I.sweeps = g->desc.precond_sweeps;
    I.max_halvings = g->desc.max_dt_halvings;
    I.precond = g->desc.precond;
    I.rtol = g->desc.gmres_rtol;
    I.newton_tol = g->desc.newton_tol;
    I.lin = (g->mixed && g->jv_form == JV_DIFF) ? g->lin : nullptr;
    return I;
}

}  // namespace

namespace batch {

// One batched step of `count` grids with the TX x TY tile (instantiated in
// batched_<TX>x<TY>.cu).
template <typename KT, int KM, int TX, int TY>
int launch_batched(music_grid **grids, int count, const double *cfl, const double *dt_max, cudaStream_t s)
{
    // stencil tile (16 planes of (TX + 5) x (TY + 5) doubles), product tile or
    // preconditioner tile (6 planes with a halo of KM + 1)
    const size_t st = Tile2D<TX, TY>::SMEM > JvTile<TX, TY>::SMEM ? Tile2D<TX, TY>::SMEM : JvTile<TX, TY>::SMEM;
    const size_t pc = (size_t)6 * (TX + 2 * (KM + 1)) * (TY + 2 * (KM + 1)) * sizeof(KT);
    const size_t smem = st > pc ? st : pc;
    static std::atomic<uint64_t> attr{0};
    TRY(allow_dynamic_smem(k_batched_step<KT, KM, TX, TY>, smem, attr));
    BArgs args;
    for (int i = 0; i < count; i++) {
        music_grid *g = grids[i];
        args.cfl[i] = cfl[i];
        args.dt_max[i] = dt_max ? dt_max[i] : 0.0;
        if (!g->binst_ready) {
            // the descriptor never changes for a grid: upload it once
            const BInst<KT> I = make_inst<KT>(g);
            CUDA_TRY(cudaMemcpyAsync(g->binst, &I, sizeof(I), cudaMemcpyHostToDevice, s));
            CUDA_TRY(cudaStreamSynchronize(s));
            g->binst_ready = 1;
        }
        args.p[i] = g->binst;
    }
    k_batched_step<KT, KM, TX, TY><<<count, NT, smem, s>>>(args);
    CHECK_LAUNCH();
    return MUSIC_OK;
}

// the instantiations of one tile shape: FP32 with the halos of 16 and 24
// sweeps, FP64 with that of 16 (one translation unit each, so the library
// builds in parallel)
#define MUSIC_BATCHED_INSTANTIATE_F32(TX, TY)                                                                     \
    template int launch_batched<float, 16, TX, TY>(music_grid **, int, const double *, const double *, cudaStream_t); \
    template int launch_batched<float, 24, TX, TY>(music_grid **, int, const double *, const double *, cudaStream_t);
#define MUSIC_BATCHED_INSTANTIATE_F64(TX, TY)                                                                     \
    template int launch_batched<double, 16, TX, TY>(music_grid **, int, const double *, const double *, cudaStream_t);

}  // namespace batch
