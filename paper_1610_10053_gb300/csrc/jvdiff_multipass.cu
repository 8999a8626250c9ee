// The Jacobian-free product in difference form (tile_jvdiff.cuh) on the
// multi-pass path: Cartesian grids without radiative diffusion that do not
// run the fused 2-D kernels, that is 3-D grids (and 2-D grids on the
// multi-pass stencil).  Same identities, branch rules and accuracy as the
// fused 2-D kernel; the intermediates live on the ghosted grid, one kernel
// per stage:
//   lin   (after every R / F evaluation): FP32 copies of rho, e and the face
//         velocities at U, the face densities, and the FP64-formed backward
//         differences of rho, e and every u_q along every d
//   A     the direction's entries: d rho, d E, d e and every d u_q
//   C     upwind mass and energy fluxes at U and their differences
//   D     momentum flux differences at cell centres and on edges
//   E     dR of the interior cells and Jv = v - dt/2 dR.
// The limited slopes (and their differences) that C and D need are formed
// where they are used, by the same function on the same inputs as a slope
// stage would (twice the slope arithmetic, in FP32, instead of thirty planes
// written and read back).  Stages A-E keep their FP32 planes in the FP64
// planes of the multi-pass scratch, which are free once the evaluation that
// opens the Newton iteration has written the linearisation arrays.
#include "internal.h"
#include "tile_jvdiff.cuh"

namespace {

using namespace tile;
constexpr int BS = 256;

// linearisation arrays, (2 + 4 nd + nd^2) planes of M floats at g->linx
struct LinX {
    float *r, *e, *u[3], *rb[3], *Dr[3], *De[3], *Du[3][3];  // Du[q][d]: u_q along d
};

LinX linx_of(const music_grid *g)
{
    const GridParams &P = g->P;
    const long long M = P.M;
    float *p = g->linx;
    LinX L{};
    L.r = p;
    p += M;
    L.e = p;
    p += M;
    for (int d = 0; d < P.nd; d++) {
        L.u[d] = p;
        p += M;
        L.rb[d] = p;
        p += M;
        L.Dr[d] = p;
        p += M;
        L.De[d] = p;
        p += M;
    }
    for (int q = 0; q < P.nd; q++)
        for (int d = 0; d < P.nd; d++) {
            L.Du[q][d] = p;
            p += M;
        }
    return L;
}

// FP32 scratch of stages A-E, carved from the FP64 multi-pass planes
struct DiffX {
    float *dr, *dE, *de, *du[3];
    float *Fr[3], *dFr[3], *dFE[3];
    float *dPhi[3], *dPsi[3][3];
};

int diffx_of(music_grid *g, DiffX *D)
{
    const GridParams &P = g->P;
    const int nd = P.nd;
    ExtScratch &X = g->ext;
    // every FP64 plane of M doubles holds two FP32 planes of M floats
    double *pool[64];
    int np = 0;
    for (double *p : {X.rho, X.e, X.p}) pool[np++] = p;
    for (int d = 0; d < nd; d++)
        for (double *p : {X.uf[d], X.srho[d], X.se[d], X.Frho[d], X.FE[d], X.Phi[d]}) pool[np++] = p;
    for (int d = 0; d < nd; d++)
        for (int q = 0; q < nd; q++) {
            pool[np++] = X.su[d][q];
            if (q != d) pool[np++] = X.Psi[d][q];
        }
    int k = 0;
    auto take = [&]() -> float * {
        const int i = k++;
        if (i / 2 >= np) return nullptr;
        return (float *)pool[i / 2] + (i % 2) * P.M;
    };
    DiffX R{};
    R.dr = take();
    R.dE = take();
    R.de = take();
    for (int d = 0; d < nd; d++) R.du[d] = take();
    for (int d = 0; d < nd; d++) {
        R.Fr[d] = take();
        R.dFr[d] = take();
        R.dFE[d] = take();
        R.dPhi[d] = take();
    }
    for (int q = 0; q < nd; q++)
        for (int d = 0; d < nd; d++)
            if (q != d) R.dPsi[q][d] = take();
    if (k > 2 * np) {
        set_error("difference-form Jv: %d FP32 planes exceed the multi-pass scratch", k);
        return MUSIC_E_INVAL;
    }
    *D = R;
    return MUSIC_OK;
}

// FP32 grid constants, formed once per launch on the host
struct DConst {
    float idx[3], g[3], gm1;
};

// ---- lin: the values at U from the FP64 planes of the evaluation just run
__global__ void __launch_bounds__(BS) k_lin_ext(GridParams P, const double *U, ExtScratch X, LinX L)
{
    pdl_entry();
    for (long long x = blockIdx.x * (long long)BS + threadIdx.x; x < P.M; x += (long long)gridDim.x * BS) {
        int ix[3];
        ext_coords(P, x, ix);
        L.r[x] = (float)X.rho[x];
        L.e[x] = (float)X.e[x];
        for (int d = 0; d < P.nd; d++) {
            L.u[d][x] = (float)X.uf[d][x];
            // the face's mean density as its velocity divides by it (the two
            // cells the face joins, through the ghost mapping), in FP32
            long long c, cl;
            double sgn;
            L.rb[d][x] = face_map(P, ix, d, c, cl, sgn) ? 0.5f * ((float)U[cl] + (float)U[c]) : 1.0f;
            if (!ext_has(P, ix, d, -1)) continue;
            const long long s = P.es[d];
            L.Dr[d][x] = (float)(X.rho[x] - X.rho[x - s]);
            L.De[d][x] = (float)(X.e[x] - X.e[x - s]);
            for (int q = 0; q < P.nd; q++) L.Du[q][d][x] = (float)(X.uf[q][x] - X.uf[q][x - s]);
        }
    }
}

// eps, 1 / eps and dt/2 of the launch in FP32 (and eps in FP64), per CTA
struct Kc {
    double eps64;
    float eps, ieps, h;
};

__device__ __forceinline__ Kc launch_consts(const GridParams &P, const double *eps_dev, double hdt)
{
    __shared__ double s_e;
    __shared__ float s_h;
    if (threadIdx.x == 0) {
        s_e = *eps_dev;
        s_h = (float)call_hdt(P, hdt);
    }
    __syncthreads();
    Kc k;
    k.eps64 = s_e;
    k.eps = (float)s_e;
    k.ieps = (s_e != 0.0) ? 1.0f / k.eps : 0.0f;
    k.h = s_h;
    return k;
}

// ---- A: the direction's entries (cells through the ghost mapping; faces as
// d(m / rb) = (dm - u drb) / rb')
template <typename VT, int ND>
__global__ void __launch_bounds__(BS) k_dload(GridParams P, const double *U, const VT *v, const double *eps_dev,
                                              LinX L, DiffX D)
{
    pdl_entry();
    const Kc K = launch_consts(P, eps_dev, 0.0);
    if (K.eps64 == 0.0) return;
    const long long N = P.N;
    for (long long x = blockIdx.x * (long long)BS + threadIdx.x; x < P.M; x += (long long)gridDim.x * BS) {
        int ix[3];
        ext_coords(P, x, ix);
        int j[3] = {ix[0], ix[1], ix[2]};
        int lower;
        float d1, d2;
        if (cell_map(P, j, lower) < 0) {
            const long long c = cell_index(P, j);
            d1 = (float)v[c];
            d2 = (float)v[N + c];
        } else {
            double r, E;
            ghost_cell_d(P, U, v, K.eps64, ix, r, E, d1, d2);
        }
        const float r = L.r[x], e = L.e[x];
        D.dr[x] = d1;
        D.dE[x] = d2;
        D.de[x] = __fdividef(d2 - e * d1, fmaf(K.eps, d1, r));
        for (int d = 0; d < ND; d++) {
            long long c, cl;
            double sgn;
            float du = 0.0f;
            if (face_map(P, ix, d, c, cl, sgn)) {
                const float vm = (float)v[(long long)(2 + d) * N + c];
                const float dm = (sgn > 0.0) ? vm : -vm;
                const float drb = 0.5f * ((float)v[cl] + (float)v[c]);
                du = __fdividef(dm - L.u[d][x] * drb, fmaf(K.eps, drb, L.rb[d][x]));
            }
            D.du[d][x] = du;
        }
    }
}

// The limited slope of a quantity along d at point y, and its difference:
// backward differences at U (FP64-formed, Dq) at y and y + s, the
// direction's entries dq at y - s, y, y + s.  Valid where y has both
// neighbours along d.
__device__ __forceinline__ void slope_at(const float *Dq, const float *dq, long long y, long long s, const Kc &K,
                                         float &S, float &dS)
{
    vanleer_d(Dq[y], Dq[y + s], dq[y] - dq[y - s], dq[y + s] - dq[y], K.eps, K.ieps, S, dS);
}

// ---- C: upwind mass and energy fluxes on d-faces; the face velocity decides
__global__ void __launch_bounds__(BS) k_dfluxes(GridParams P, const double *eps_dev, LinX L, DiffX D)
{
    pdl_entry();
    const Kc K = launch_consts(P, eps_dev, 0.0);
    if (K.eps64 == 0.0) return;
    for (long long x = blockIdx.x * (long long)BS + threadIdx.x; x < P.M; x += (long long)gridDim.x * BS) {
        int ix[3];
        ext_coords(P, x, ix);
        for (int d = 0; d < P.nd; d++) {
            if (!ext_has(P, ix, d, -2) || !ext_has(P, ix, d, +1)) continue;
            const long long s = P.es[d];
            const float u = L.u[d][x], du = D.du[d][x], u2 = fmaf(K.eps, du, u);
            // slopes of rho and e of the two cells the face joins
            float Srm, dSrm, Sr0, dSr0, Sem, dSem, Se0, dSe0;
            slope_at(L.Dr[d], D.dr, x - s, s, K, Srm, dSrm);
            slope_at(L.Dr[d], D.dr, x, s, K, Sr0, dSr0);
            slope_at(L.De[d], D.de, x - s, s, K, Sem, dSem);
            slope_at(L.De[d], D.de, x, s, K, Se0, dSe0);
            float rs, drs, es, des;
            upwind_d(u, u2, L.r[x - s] + 0.5f * Srm, D.dr[x - s] + 0.5f * dSrm, L.r[x] - 0.5f * Sr0,
                     D.dr[x] - 0.5f * dSr0, K.ieps, rs, drs);
            upwind_d(u, u2, L.e[x - s] + 0.5f * Sem, D.de[x - s] + 0.5f * dSem, L.e[x] - 0.5f * Se0,
                     D.de[x] - 0.5f * dSe0, K.ieps, es, des);
            const float fr = u * rs, dfr = du * fmaf(K.eps, drs, rs) + u * drs;
            D.Fr[d][x] = fr;
            D.dFr[d][x] = dfr;
            D.dFE[d][x] = dfr * fmaf(K.eps, des, es) + fr * des;
        }
    }
}

// ---- D: momentum flux differences at cell centres (Phi, along d) and on
// edges (Psi, the flux of u_d across q)
template <int ND>
__global__ void __launch_bounds__(BS) k_dmomentum(GridParams P, const double *eps_dev, LinX L, DiffX D)
{
    pdl_entry();
    const Kc K = launch_consts(P, eps_dev, 0.0);
    if (K.eps64 == 0.0) return;
    for (long long x = blockIdx.x * (long long)BS + threadIdx.x; x < P.M; x += (long long)gridDim.x * BS) {
        int ix[3];
        ext_coords(P, x, ix);
        for (int d = 0; d < ND; d++) {
            const long long s = P.es[d];
            if (ext_has(P, ix, d, -2) && ext_has(P, ix, d, +2)) {
                // slopes of u_d along d at the centre's two faces
                float S0, dS0, S1, dS1;
                slope_at(L.Du[d][d], D.du[d], x, s, K, S0, dS0);
                slope_at(L.Du[d][d], D.du[d], x + s, s, K, S1, dS1);
                D.dPhi[d][x] = momflux_d(D.Fr[d][x], D.Fr[d][x + s], D.dFr[d][x], D.dFr[d][x + s], L.u[d][x], S0,
                                         D.du[d][x], dS0, L.u[d][x + s], S1, D.du[d][x + s], dS1, K.eps, K.ieps);
            }
            for (int q = 0; q < ND; q++) {
                if (q == d) continue;
                if (!ext_has(P, ix, d, -1) || !ext_has(P, ix, q, -2) || !ext_has(P, ix, q, +1)) continue;
                const long long t = P.es[q];
                // slopes of u_d along q at the edge's two faces
                float Sm, dSm, S0, dS0;
                slope_at(L.Du[d][q], D.du[d], x - t, t, K, Sm, dSm);
                slope_at(L.Du[d][q], D.du[d], x, t, K, S0, dS0);
                D.dPsi[d][q][x] = momflux_d(D.Fr[q][x - s], D.Fr[q][x], D.dFr[q][x - s], D.dFr[q][x], L.u[d][x - t],
                                            Sm, D.du[d][x - t], dSm, L.u[d][x], S0, D.du[d][x], dS0, K.eps, K.ieps);
            }
        }
    }
}

// ---- E: dR of the interior cells and Jv = v - dt/2 dR (zero for eps = 0)
template <typename VT>
__global__ void __launch_bounds__(BS) k_dassemble(GridParams P, DConst C, const double *eps_dev, double hdt,
                                                  LinX L, DiffX D, const VT *v, VT *out)
{
    pdl_entry();
    const Kc K = launch_consts(P, eps_dev, hdt);
    for (long long c = blockIdx.x * (long long)BS + threadIdx.x; c < P.N; c += (long long)gridDim.x * BS) {
        if (K.eps64 == 0.0) {
            for (int q = 0; q < P.nv; q++) out[(long long)q * P.N + c] = (VT)0;
            continue;
        }
        int ix[3];
        cell_coords(P, c, ix);
        const long long x = ext_index(P, ix[0], ix[1], ix[2]);
        float dR[5];
        float accr = 0.0f, acce = 0.0f, divu = 0.0f, ddivu = 0.0f;
        for (int d = 0; d < P.nd; d++) {
            const long long s = P.es[d];
            accr += (D.dFr[d][x + s] - D.dFr[d][x]) * C.idx[d];
            acce += (D.dFE[d][x + s] - D.dFE[d][x]) * C.idx[d];
            divu += L.Du[d][d][x + s] * C.idx[d];
            ddivu += (D.du[d][x + s] - D.du[d][x]) * C.idx[d];
        }
        // p div u at U and its difference (div u from the FP64-formed differences)
        const float p = C.gm1 * L.r[x] * L.e[x], dp = C.gm1 * D.dE[x];
        dR[0] = -accr;
        dR[1] = -acce - (dp * fmaf(K.eps, ddivu, divu) + p * ddivu);
        for (int d = 0; d < P.nd; d++) {
            if (P.bc[d] == MUSIC_BC_WALL && ix[d] == 0) {
                dR[2 + d] = 0.0f;
                continue;
            }
            const long long s = P.es[d];
            float acc = 0.0f;
            for (int q = 0; q < P.nd; q++) {
                if (q == d)
                    acc += (D.dPhi[d][x] - D.dPhi[d][x - s]) * C.idx[d];
                else
                    acc += (D.dPsi[d][q][x + P.es[q]] - D.dPsi[d][q][x]) * C.idx[q];
            }
            dR[2 + d] = (-acc - C.gm1 * (D.dE[x] - D.dE[x - s]) * C.idx[d]) + 0.5f * (D.dr[x - s] + D.dr[x]) * C.g[d];
        }
        for (int q = 0; q < P.nv; q++) {
            const long long i = (long long)q * P.N + c;
            out[i] = (VT)((float)v[i] - K.h * dR[q]);
        }
    }
}

int blocks_for(long long n)
{
    long long b = (n + BS - 1) / BS;
    if (b > 152 * 16) b = 152 * 16;
    if (b < 1) b = 1;
    return (int)b;
}

}  // namespace

bool jvdiff_multipass_grid(const music_grid *g) { return g->linx != nullptr; }

int lin_ext_write(music_grid *g, const double *U, cudaStream_t s)
{
    k_lin_ext<<<blocks_for(g->P.M), BS, 0, s>>>(g->P, U, g->ext, linx_of(g));
    CHECK_LAUNCH();
    return MUSIC_OK;
}

int jvdiff_multipass(music_grid *g, const double *U, const float *v, float *out, double hdt, cudaStream_t s)
{
    const GridParams &P = g->P;
    DiffX D;
    TRY(diffx_of(g, &D));
    const LinX L = linx_of(g);
    const double *eps = &g->ds->eps;
    const int nbm = blocks_for(P.M);
    // the direction entries and the momentum fluxes instantiated for the grid's
    // dimension count (their direction loops unroll: k_dmomentum 206 -> 161 us
    // a launch cold on TGV 128^3; the flux pass ran slower that way)
    if (P.nd == 3)
        k_dload<float, 3><<<nbm, BS, 0, s>>>(P, U, v, eps, L, D);
    else
        k_dload<float, 2><<<nbm, BS, 0, s>>>(P, U, v, eps, L, D);
    CHECK_LAUNCH();
    k_dfluxes<<<nbm, BS, 0, s>>>(P, eps, L, D);
    CHECK_LAUNCH();
    if (P.nd == 3)
        k_dmomentum<3><<<nbm, BS, 0, s>>>(P, eps, L, D);
    else
        k_dmomentum<2><<<nbm, BS, 0, s>>>(P, eps, L, D);
    CHECK_LAUNCH();
    DConst C{};
    for (int d = 0; d < 3; d++) {
        C.idx[d] = (float)P.idx[d];
        C.g[d] = (float)P.g[d];
    }
    C.gm1 = (float)P.gm1;
    k_dassemble<float><<<blocks_for(P.N), BS, 0, s>>>(P, C, eps, hdt, L, D, v, out);
    CHECK_LAUNCH();
    return MUSIC_OK;
}
