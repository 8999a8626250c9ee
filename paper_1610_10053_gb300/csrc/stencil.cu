// Spatial operator R(U) (paper Sec. 2, Eqs. 1-3) and the quantities built on
// it: the Crank-Nicolson residual and the Jacobian-free product.
//
// Generic multi-pass path for 2-D and 3-D grids: each pass is one kernel over
// the ghosted ("extended") grid, writing its per-point results to scratch
// planes, so no value is computed twice:
//   1 load   : ghost filling (periodic / mirror / hydrostatic walls), e, p,
//              face velocities u_d = m_d / rbar (W = U + eps v for Jv)
//   2 slopes : van Leer limited slopes of rho, e and every u_q along every d
//   3 fluxes : upwind mass and internal-energy fluxes on d-faces
//   4 momentum fluxes at cell centres (along d) and on edges (across d)
//   5 assemble the interior residuals and write R, C^n, F or Jv.
#include <cmath>

#include "internal.h"
#include "tiles.h"
#include "tile_stencil.cuh"

namespace {

using namespace tile;
constexpr int BS = 256;

template <typename VT>
__global__ void __launch_bounds__(BS) k_load(GridParams P, const double *U, const VT *v, const double *eps,
                                             ExtScratch X)
{
    pdl_entry();
    const WLoad<VT> W{U, v, v ? *eps : 0.0};
    for (long long x = blockIdx.x * (long long)BS + threadIdx.x; x < P.M; x += (long long)gridDim.x * BS) {
        int ix[3];
        ext_coords(P, x, ix);
        double rho, E;
        load_cell(P, W, ix, rho, E);
        X.rho[x] = rho;
        const double e = E / rho;
        X.e[x] = e;
        X.p[x] = P.gm1 * E;
        for (int d = 0; d < P.nd; d++) X.uf[d][x] = face_velocity<false>(P, W, ix, d);
        if (P.conduct) {
            // T = (gamma-1) e and the photon conductivity chi = chi0 T^6.5 / rho^2
            const double T = P.gm1 * e;
            const double t3 = T * T * T;
            X.Tt[x] = T;
            X.chi[x] = P.chi0 * (t3 * t3 * sqrt(T)) / (rho * rho);
        }
    }
}

// radiative diffusion: chi dT/dn on every d-face (mean of the two cells' chi);
// wall faces carry the prescribed flux (lum, or lum / r^2 on spherical
// r-walls) or none
__global__ void __launch_bounds__(BS) k_cond(GridParams P, ExtScratch X)
{
    pdl_entry();
    for (long long x = blockIdx.x * (long long)BS + threadIdx.x; x < P.M; x += (long long)gridDim.x * BS) {
        int ix[3];
        ext_coords(P, x, ix);
        for (int d = 0; d < P.nd; d++) {
            if (!ext_has(P, ix, d, -1)) continue;
            if (P.bc[d] == MUSIC_BC_WALL && (ix[d] == 0 || ix[d] == P.n[d])) {
                double G = 0.0;
                if (P.flux_wall[d]) {
                    G = P.lum;
                    if (P.geom == MUSIC_GEOM_SPHERICAL && d == 0) {
                        const double rf = sph_r(P, ix[0]);
                        G = G / (rf * rf);
                    }
                }
                X.Gc[d][x] = G;
                continue;
            }
            const long long s = P.es[d];
            const double h = (P.geom == MUSIC_GEOM_SPHERICAL) ? sph_h(P, d, ix[0]) : P.dx[d];
            X.Gc[d][x] = 0.5 * (X.chi[x - s] + X.chi[x]) * (X.Tt[x] - X.Tt[x - s]) / h;
        }
    }
}

__global__ void __launch_bounds__(BS) k_slopes(GridParams P, ExtScratch X)
{
    pdl_entry();
    for (long long x = blockIdx.x * (long long)BS + threadIdx.x; x < P.M; x += (long long)gridDim.x * BS) {
        int ix[3];
        ext_coords(P, x, ix);
        for (int d = 0; d < P.nd; d++) {
            if (!ext_has(P, ix, d, -1) || !ext_has(P, ix, d, +1)) continue;
            const long long s = P.es[d];
            X.srho[d][x] = vanleer(X.rho[x] - X.rho[x - s], X.rho[x + s] - X.rho[x]);
            X.se[d][x] = vanleer(X.e[x] - X.e[x - s], X.e[x + s] - X.e[x]);
            for (int q = 0; q < P.nd; q++)
                X.su[q][d][x] = vanleer(X.uf[q][x] - X.uf[q][x - s], X.uf[q][x + s] - X.uf[q][x]);
        }
    }
}

__global__ void __launch_bounds__(BS) k_fluxes(GridParams P, ExtScratch X)
{
    pdl_entry();
    for (long long x = blockIdx.x * (long long)BS + threadIdx.x; x < P.M; x += (long long)gridDim.x * BS) {
        int ix[3];
        ext_coords(P, x, ix);
        for (int d = 0; d < P.nd; d++) {
            if (!ext_has(P, ix, d, -2) || !ext_has(P, ix, d, +1)) continue;
            const long long s = P.es[d];
            const double u = X.uf[d][x];
            double rs, es;
            if (u >= 0.0) {
                rs = X.rho[x - s] + 0.5 * X.srho[d][x - s];
                es = X.e[x - s] + 0.5 * X.se[d][x - s];
            } else {
                rs = X.rho[x] - 0.5 * X.srho[d][x];
                es = X.e[x] - 0.5 * X.se[d][x];
            }
            const double fr = u * rs;
            X.Frho[d][x] = fr;
            X.FE[d][x] = fr * es;
        }
    }
}

__global__ void __launch_bounds__(BS) k_momentum(GridParams P, ExtScratch X)
{
    pdl_entry();
    for (long long x = blockIdx.x * (long long)BS + threadIdx.x; x < P.M; x += (long long)gridDim.x * BS) {
        int ix[3];
        ext_coords(P, x, ix);
        for (int d = 0; d < P.nd; d++) {
            const long long s = P.es[d];
            if (ext_has(P, ix, d, -2) && ext_has(P, ix, d, +2)) {
                const double fm = 0.5 * (X.Frho[d][x] + X.Frho[d][x + s]);
                const double us = (fm >= 0.0) ? X.uf[d][x] + 0.5 * X.su[d][d][x]
                                              : X.uf[d][x + s] - 0.5 * X.su[d][d][x + s];
                X.Phi[d][x] = fm * us;
            }
            for (int q = 0; q < P.nd; q++) {
                if (q == d) continue;
                if (!ext_has(P, ix, d, -1) || !ext_has(P, ix, q, -2) || !ext_has(P, ix, q, +1)) continue;
                const long long t = P.es[q];
                const double fm = 0.5 * (X.Frho[q][x - s] + X.Frho[q][x]);
                const double us = (fm >= 0.0) ? X.uf[d][x - t] + 0.5 * X.su[d][q][x - t]
                                              : X.uf[d][x] - 0.5 * X.su[d][q][x];
                X.Psi[d][q][x] = fm * us;
            }
        }
    }
}

// Spherical (r, theta) assembly of one cell and its lower faces: every
// divergence is (1/V) sum(A F) over the control volume, the momenta carry
// the geometric terms +rho u_t^2 / r (radial) and -rho u_r u_t / r (polar),
// pressure gradients divide by dr or r_c dtheta, gravity from the r-face table.
// The metric comes from the grid's table (SphGeo).
__device__ void sph_assemble(const GridParams &P, const ExtScratch &X, const int ix[3], long long x, long long c,
                             double *R)
{
    const int i = ix[0], j = ix[1];
    const long long s0 = P.es[0], s1 = P.es[1];
    const double V = sgeo(P, SG_V, c);
    const double Arm = sgeo(P, SG_ARM, c), Arp = sgeo(P, SG_ARP, c);
    const double Atm = sgeo(P, SG_ATM, c), Atp = sgeo(P, SG_ATP, c);
    const double fr = (Arp * X.Frho[0][x + s0] - Arm * X.Frho[0][x]) + (Atp * X.Frho[1][x + s1] - Atm * X.Frho[1][x]);
    const double fe = (Arp * X.FE[0][x + s0] - Arm * X.FE[0][x]) + (Atp * X.FE[1][x + s1] - Atm * X.FE[1][x]);
    const double du = (Arp * X.uf[0][x + s0] - Arm * X.uf[0][x]) + (Atp * X.uf[1][x + s1] - Atm * X.uf[1][x]);
    R[0] = -fr / V;
    R[1] = -fe / V - X.p[x] * (du / V);
    if (P.conduct) {
        const double cd = (Arp * X.Gc[0][x + s0] - Arm * X.Gc[0][x]) + (Atp * X.Gc[1][x + s1] - Atm * X.Gc[1][x]);
        R[1] = R[1] + cd / V;
    }
    if (P.bc[0] == MUSIC_BC_WALL && i == 0) {
        R[2] = 0.0;
    } else {
        const double Vr = sgeo(P, SG_VR, c), Acp = sgeo(P, SG_ACP, c), Acm = sgeo(P, SG_ACM, c);
        const double Em = sgeo(P, SG_EM, c), Ep = sgeo(P, SG_EP, c), rf = sgeo(P, SG_RF, c);
        const double acc = (Acp * X.Phi[0][x] - Acm * X.Phi[0][x - s0]) + (Ep * X.Psi[0][1][x + s1] - Em * X.Psi[0][1][x]);
        const double rbar = 0.5 * (X.rho[x - s0] + X.rho[x]);
        const double ut = 0.25 * ((X.uf[1][x - s0] + X.uf[1][x]) + (X.uf[1][x - s0 + s1] + X.uf[1][x + s1]));
        R[2] = ((-acc / Vr - (X.p[x] - X.p[x - s0]) / P.dx[0]) + rbar * ut * ut / rf) + rbar * face_g(P, 0, i);
    }
    if (P.bc[1] == MUSIC_BC_WALL && j == 0) {
        R[3] = 0.0;
    } else {
        const double Vt = sgeo(P, SG_VT, c), Bp = sgeo(P, SG_BP, c), Bm = sgeo(P, SG_BM, c);
        const double Fa = sgeo(P, SG_FA, c), Fb = sgeo(P, SG_FB, c), rc = sgeo(P, SG_RC, c);
        const double acc = (Fb * X.Psi[1][0][x + s0] - Fa * X.Psi[1][0][x]) + (Bp * X.Phi[1][x] - Bm * X.Phi[1][x - s1]);
        const double rbar = 0.5 * (X.rho[x - s1] + X.rho[x]);
        const double ur = 0.25 * ((X.uf[0][x - s1] + X.uf[0][x]) + (X.uf[0][x - s1 + s0] + X.uf[0][x + s0]));
        R[3] = ((-acc / Vt - (X.p[x] - X.p[x - s1]) / (rc * P.dx[1])) - rbar * ur * X.uf[1][x] / rc) + rbar * P.g[1];
    }
}

// the table of the metric, from the expressions of common.cuh
__global__ void __launch_bounds__(BS) k_sph_geo(GridParams P, double *T)
{
    pdl_entry();
    for (long long c = blockIdx.x * (long long)BS + threadIdx.x; c < P.N; c += (long long)gridDim.x * BS) {
        int ix[3];
        cell_coords(P, c, ix);
        const int i = ix[0], j = ix[1];
        const long long N = P.N;
        T[SG_V * N + c] = sph_vol(P, i, j);
        T[SG_ARM * N + c] = sph_area(P, 0, i, j);
        T[SG_ARP * N + c] = sph_area(P, 0, i + 1, j);
        T[SG_ATM * N + c] = sph_area(P, 1, i, j);
        T[SG_ATP * N + c] = sph_area(P, 1, i, j + 1);
        const double ctj = cos(sph_th(P, j)), ctj1 = cos(sph_th(P, j + 1));
        const double rm = sph_r(P, i - 0.5), rp = sph_r(P, i + 0.5), rf = sph_r(P, i);
        T[SG_VR * N + c] = (rp * rp * rp - rm * rm * rm) / 3.0 * (ctj - ctj1);
        T[SG_ACP * N + c] = rp * rp * (ctj - ctj1);
        T[SG_ACM * N + c] = rm * rm * (ctj - ctj1);
        T[SG_EM * N + c] = 0.5 * (rp * rp - rm * rm) * sin(sph_th(P, j));
        T[SG_EP * N + c] = 0.5 * (rp * rp - rm * rm) * sin(sph_th(P, j + 1));
        T[SG_RF * N + c] = rf;
        const double ra = sph_r(P, i), rb = sph_r(P, i + 1), rc = sph_r(P, i + 0.5);
        const double cm = cos(sph_th(P, j - 0.5)), cp = cos(sph_th(P, j + 0.5));
        T[SG_VT * N + c] = (rb * rb * rb - ra * ra * ra) / 3.0 * (cm - cp);
        T[SG_BP * N + c] = 0.5 * (rb * rb - ra * ra) * sin(sph_th(P, j + 0.5));
        T[SG_BM * N + c] = 0.5 * (rb * rb - ra * ra) * sin(sph_th(P, j - 0.5));
        T[SG_FA * N + c] = ra * ra * (cm - cp);
        T[SG_FB * N + c] = rb * rb * (cm - cp);
        T[SG_RC * N + c] = rc;
    }
}

template <int MODE, typename VIN, typename VOUT, int ND>
__global__ void __launch_bounds__(BS) k_assemble(GridParams P, ExtScratch X, const double *U,
                                                 const double *aux, const VIN *v, VOUT *out,
                                                 double *RU_out, double hdt, double sign,
                                                 const double *eps)
{
    pdl_entry();
    hdt = call_hdt(P, hdt);
    double c_jv = 0.0;
    bool zero = false;
    if (MODE == SM_JV) {
        const double e = *eps;
        zero = (e == 0.0);
        c_jv = zero ? 0.0 : hdt / e;
    }
    for (long long c = blockIdx.x * (long long)BS + threadIdx.x; c < P.N; c += (long long)gridDim.x * BS) {
        int ix[3];
        cell_coords(P, c, ix);
        const long long x = ext_index(P, ix[0], ix[1], ix[2]);
        double R[5];
        double accr = 0.0, acce = 0.0, divu = 0.0;
        for (int d = 0; d < ND; d++) {
            const long long s = P.es[d];
            accr += (X.Frho[d][x + s] - X.Frho[d][x]) * P.idx[d];
            acce += (X.FE[d][x + s] - X.FE[d][x]) * P.idx[d];
            divu += (X.uf[d][x + s] - X.uf[d][x]) * P.idx[d];
        }
        R[0] = -accr;
        R[1] = -acce - X.p[x] * divu;
        if (P.conduct) {
            double cond = 0.0;
            for (int d = 0; d < ND; d++) cond += (X.Gc[d][x + P.es[d]] - X.Gc[d][x]) * P.idx[d];
            R[1] = R[1] + cond;
        }
        if (P.geom == MUSIC_GEOM_SPHERICAL) sph_assemble(P, X, ix, x, c, R);
        for (int d = 0; d < ND && P.geom != MUSIC_GEOM_SPHERICAL; d++) {
            if (P.bc[d] == MUSIC_BC_WALL && ix[d] == 0) {
                R[2 + d] = 0.0;
                continue;
            }
            const long long s = P.es[d];
            double acc = 0.0;
            for (int q = 0; q < ND; q++) {
                if (q == d)
                    acc += (X.Phi[d][x] - X.Phi[d][x - s]) * P.idx[d];
                else
                    acc += (X.Psi[d][q][x + P.es[q]] - X.Psi[d][q][x]) * P.idx[q];
            }
            const double rbar = 0.5 * (X.rho[x - s] + X.rho[x]);
            R[2 + d] = (-acc - (X.p[x] - X.p[x - s]) * P.idx[d]) + rbar * P.g[d];
        }
        for (int q = 0; q < P.nv; q++) {
            const long long i = (long long)q * P.N + c;
            if (MODE == SM_R) {
                out[i] = (VOUT)R[q];
            } else if (MODE == SM_CN) {
                out[i] = (VOUT)(U[i] + hdt * R[q]);
            } else if (MODE == SM_F) {
                out[i] = (VOUT)(sign * ((U[i] - aux[i]) - hdt * R[q]));
                if (RU_out) RU_out[i] = R[q];
            } else if (MODE == SM_CNF) {
                // the step constant as SM_CN writes it (into aux), then the residual as SM_F forms it
                const double cn = U[i] + hdt * R[q];
                const_cast<double *>(aux)[i] = cn;
                out[i] = (VOUT)(sign * ((U[i] - cn) - hdt * R[q]));
                if (RU_out) RU_out[i] = R[q];
            } else {
                out[i] = zero ? (VOUT)0 : (VOUT)((double)v[i] - c_jv * (R[q] - aux[i]));
            }
        }
    }
}


// k_assemble instantiated for the grid's dimension count: its direction
// loops then unroll, so the loads of a cell are all in flight at once
// (measured on TGV 128^3: 392 -> 282 us a launch cold; the other passes of
// the multi-pass stencil ran slower that way, their registers doubling)
template <int MODE, typename VIN, typename VOUT>
void assemble(const GridParams &P, int nb, cudaStream_t s, const ExtScratch &X, const double *U, const double *aux,
              const VIN *v, VOUT *out, double *RU_out, double hdt, double sign, const double *eps)
{
    if (P.nd == 3)
        k_assemble<MODE, VIN, VOUT, 3><<<nb, BS, 0, s>>>(P, X, U, aux, v, out, RU_out, hdt, sign, eps);
    else
        k_assemble<MODE, VIN, VOUT, 2><<<nb, BS, 0, s>>>(P, X, U, aux, v, out, RU_out, hdt, sign, eps);
}

int blocks_for(long long n)
{
    long long b = (n + BS - 1) / BS;
    if (b > 152 * 16) b = 152 * 16;
    if (b < 1) b = 1;
    return (int)b;
}

template <typename VT>
int run_passes(music_grid *g, const double *U, const VT *v, cudaStream_t s)
{
    const GridParams &P = g->P;
    const int nbm = blocks_for(P.M);
    k_load<VT><<<nbm, BS, 0, s>>>(P, U, v, &g->ds->eps, g->ext);
    CHECK_LAUNCH();
    k_slopes<<<nbm, BS, 0, s>>>(P, g->ext);
    CHECK_LAUNCH();
    k_fluxes<<<nbm, BS, 0, s>>>(P, g->ext);
    CHECK_LAUNCH();
    k_momentum<<<nbm, BS, 0, s>>>(P, g->ext);
    CHECK_LAUNCH();
    if (P.conduct) {
        k_cond<<<nbm, BS, 0, s>>>(P, g->ext);
        CHECK_LAUNCH();
    }
    return MUSIC_OK;
}

}  // namespace

int stencil_apply(music_grid *g, int mode, const double *U, const double *aux, const void *v,
                  int vin_double, void *out, int out_double, double *RU_out, double dt, double sign,
                  cudaStream_t s)
{
    if (g->in_scalar) return scalar_apply(g, mode, U, aux, v, vin_double, out, out_double, RU_out, dt, sign, s);
    const GridParams &P = g->P;
    const double hdt = 0.5 * dt;
    if (P.nd == 2 && g->stencil_variant != STENCIL_MULTIPASS && !general_grid(P)) {
        ProfScope prof_(g, mode == SM_JV ? MUSIC_PROF_JV : MUSIC_PROF_RESIDUAL, s);
        return fused2d_dispatch(g, mode, U, aux, v, vin_double, out, out_double, RU_out, hdt, sign, s);
    }
    ProfScope prof_(g, mode == SM_JV ? MUSIC_PROF_JV : MUSIC_PROF_RESIDUAL, s);
    const bool diff = g->linx && g->jv_form == JV_DIFF;
    if (mode == SM_JV && diff && !vin_double && !out_double)
        return jvdiff_multipass(g, U, (const float *)v, (float *)out, hdt, s);
    const int nbn = blocks_for(P.N);
    const double *eps = &g->ds->eps;
    if (mode == SM_JV) {
        if (vin_double)
            TRY(run_passes<double>(g, U, (const double *)v, s));
        else
            TRY(run_passes<float>(g, U, (const float *)v, s));
    } else {
        TRY(run_passes<double>(g, U, nullptr, s));
        if (g->fr_capture) TRY(capture_ext_fluxes(g, s));  // face mass fluxes for passive scalars
        if (diff && (mode == SM_R || mode == SM_F || mode == SM_CNF)) TRY(lin_ext_write(g, U, s));
    }
    switch (mode) {
    case SM_R:
        assemble<SM_R, double, double>(P, nbn, s, g->ext, U, aux, nullptr, (double *)out,
                                                             nullptr, hdt, sign, eps);
        break;
    case SM_CN:
        assemble<SM_CN, double, double>(P, nbn, s, g->ext, U, aux, nullptr, (double *)out,
                                                              nullptr, hdt, sign, eps);
        break;
    case SM_F:
        assemble<SM_F, double, double>(P, nbn, s, g->ext, U, aux, nullptr, (double *)out,
                                                             RU_out, hdt, sign, eps);
        break;
    case SM_CNF:
        assemble<SM_CNF, double, double>(P, nbn, s, g->ext, U, aux, nullptr, (double *)out,
                                                               RU_out, hdt, sign, eps);
        break;
    case SM_JV:
        if (vin_double && out_double)
            assemble<SM_JV, double, double>(P, nbn, s, g->ext, U, aux, (const double *)v,
                                                                  (double *)out, nullptr, hdt, sign, eps);
        else if (!vin_double && !out_double)
            assemble<SM_JV, float, float>(P, nbn, s, g->ext, U, aux, (const float *)v,
                                                                (float *)out, nullptr, hdt, sign, eps);
        else if (vin_double && !out_double)
            assemble<SM_JV, double, float>(P, nbn, s, g->ext, U, aux, (const double *)v,
                                                                 (float *)out, nullptr, hdt, sign, eps);
        else
            assemble<SM_JV, float, double>(P, nbn, s, g->ext, U, aux, (const float *)v,
                                                                 (double *)out, nullptr, hdt, sign, eps);
        break;
    default:
        set_error("stencil_apply: bad mode %d", mode);
        return MUSIC_E_INVAL;
    }
    CHECK_LAUNCH();
    return MUSIC_OK;
}

int sph_geo_build(music_grid *g, cudaStream_t s)
{
    k_sph_geo<<<blocks_for(g->P.N), BS, 0, s>>>(g->P, g->sgeo);
    CHECK_LAUNCH();
    return MUSIC_OK;
}

int fused2d_dispatch(music_grid *g, int mode, const double *U, const double *aux, const void *v, int vin_double,
                     void *out, int out_double, double *RU_out, double hdt, double sign, cudaStream_t s)
{
    const int tile = (mode == SM_JV) ? g->stile : g->rtile;
    switch (tile) {
    case 0:
        return fused2d_apply_t<16, 8>(g, mode, U, aux, v, vin_double, out, out_double, RU_out, hdt, sign, s);
    case 1:
        return fused2d_apply_t<16, 16>(g, mode, U, aux, v, vin_double, out, out_double, RU_out, hdt, sign, s);
    case 2:
        return fused2d_apply_t<32, 8>(g, mode, U, aux, v, vin_double, out, out_double, RU_out, hdt, sign, s);
    case 3:
        return fused2d_apply_t<32, 16>(g, mode, U, aux, v, vin_double, out, out_double, RU_out, hdt, sign, s);
    case 4:
        return fused2d_apply_t<32, 32>(g, mode, U, aux, v, vin_double, out, out_double, RU_out, hdt, sign, s);
    }
    set_error("stencil: bad tile index %d", tile);
    return MUSIC_E_INVAL;
}

__global__ void __launch_bounds__(BS) k_vanleer(const double *a, const double *b, double *s, long long count)
{
    pdl_entry();
    for (long long i = blockIdx.x * (long long)BS + threadIdx.x; i < count; i += (long long)gridDim.x * BS)
        s[i] = vanleer(a[i], b[i]);
}

extern "C" int music_vanleer_slopes(const double *a, const double *b, double *s, long long count, void *stream)
{
    if (count < 0 || (count > 0 && (!a || !b || !s))) {
        set_error("music_vanleer_slopes: NULL array or negative count");
        return MUSIC_E_INVAL;
    }
    if (count == 0) return MUSIC_OK;
    k_vanleer<<<blocks_for(count), BS, 0, (cudaStream_t)stream>>>(a, b, s, count);
    CHECK_LAUNCH();
    return MUSIC_OK;
}

__global__ void __launch_bounds__(BS) k_quot(const double *n, const double *d, double *q, long long count)
{
    pdl_entry();
    for (long long i = blockIdx.x * (long long)BS + threadIdx.x; i < count; i += (long long)gridDim.x * BS)
        q[i] = quot(n[i], d[i]);
}

extern "C" int music_stencil_quotients(const double *n, const double *d, double *q, long long count, void *stream)
{
    if (count < 0 || (count > 0 && (!n || !d || !q))) {
        set_error("music_stencil_quotients: NULL array or negative count");
        return MUSIC_E_INVAL;
    }
    if (count == 0) return MUSIC_OK;
    k_quot<<<blocks_for(count), BS, 0, (cudaStream_t)stream>>>(n, d, q, count);
    CHECK_LAUNCH();
    return MUSIC_OK;
}
