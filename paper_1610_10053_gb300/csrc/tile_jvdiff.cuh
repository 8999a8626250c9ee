// The finite-difference Jacobian-vector product of the fused 2-D stencil in
// difference form (Sec. 2, the Jacobian-free product after Knoll & Keyes):
//
//   Jv = v - dt/2 (R(U + eps v) - R(U)) / eps
//
// computed without forming R(U + eps v) and R(U).  Every intermediate x of
// R (Eqs. 1-3 on the staggered grid with van Leer reconstruction) is carried
// as its value at U and its scaled difference dx = (x(U + eps v) - x(U)) /
// eps, propagated through the exact identities
//
//   sums        d(a + b)       = da + db
//   products    d(a b)         = da b' + a db                 (b' = b + eps db)
//   quotients   d(a / b)       = (da b - a db) / (b b')
//   van Leer    d(2ab / (a+b)) = 2 (a a' db + b b' da) / ((a + b)(a' + b'))
//
// and every upwind or limiter branch is taken twice, at U and at U + eps v,
// as the two evaluations of the finite difference take it; where the two
// branches differ the difference is (other side at U - chosen side at U) /
// eps + d(other side), which stays bounded because a branch flips only when
// the deciding quantity is within eps of zero.  The result is the same
// finite difference as the FP64 form (same eps, same branches, the same
// second-order terms), but no step subtracts two nearly equal residuals: the
// differences hold no cancellation and are carried in FP32.  What does need
// FP64 is the van Leer ratio's inputs, the differences of neighbouring
// values at U, which decide the limiter's branch and must resolve steps
// below FP32's resolution of the values themselves: they are formed in
// FP64 and only then rounded.  All values at U are fixed while GMRES solves
// one Newton iteration, so the R / F evaluation that opens the iteration
// writes them (rho, e, the face velocities and the eight neighbour
// differences, as FP32 planes) and the products only read them; tiles whose
// staged region reaches a wall ghost form them from U the same way.
// Hydrostatic ghost cells (Sec. 3) are extrapolated at U and at U + eps v in
// FP64 and differenced there.
#pragma once
#include "tile_stencil.cuh"

namespace tile {

// (rho, E) of a hydrostatic ghost cell (Sec. 3) at U and their scaled
// differences: the extrapolation evaluated at U and at U + eps v in FP64
template <typename VT>
__device__ void ghost_cell_d(const GridParams &P, const double *U, const VT *v, double eps, const int ix[3],
                             double &rho, double &E, float &drho, float &dE)
{
    const WLoad<VT> W0{U, nullptr, 0.0}, W1{U, v, eps};
    double r1, E1;
    load_cell(P, W0, ix, rho, E);
    load_cell(P, W1, ix, r1, E1);
    drho = (float)((r1 - rho) / eps);
    dE = (float)((E1 - E) / eps);
}

// van Leer slope s = phi(a, b) at U and its scaled difference, given the
// one-sided differences a, b at U and their scaled differences da, db
__device__ inline void vanleer_d(float a, float b, float da, float db, float eps, float ieps, float &s,
                                 float &ds)
{
    const float a2 = fmaf(eps, da, a), b2 = fmaf(eps, db, b);
    const bool on = a * b > 0.0f, on2 = a2 * b2 > 0.0f;
    s = on ? __fdividef((2.0f * a) * b, a + b) : 0.0f;
    if (on && on2)
        ds = __fdividef(2.0f * (a * a2 * db + b * b2 * da), (a + b) * (a2 + b2));
    else if (on)
        ds = -s * ieps;
    else if (on2)
        ds = __fdividef((2.0f * a2) * b2, a2 + b2) * ieps;
    else
        ds = 0.0f;
}

// Upwind choice between the reconstructions xL (from the left / lower cell)
// and xR by the sign of the deciding quantity, f at U and f2 at U + eps v:
// the chosen value at U and the scaled difference of the chosen values.
__device__ inline void upwind_d(float f, float f2, float xL, float dxL, float xR, float dxR, float ieps, float &x,
                                float &dx)
{
    const bool up = (f >= 0.0f), up2 = (f2 >= 0.0f);
    x = up ? xL : xR;
    if (up == up2)
        dx = up ? dxL : dxR;
    else
        dx = up2 ? fmaf(xL - xR, ieps, dxL) : fmaf(xR - xL, ieps, dxR);
}

// momentum flux fm us (fm the mean of two mass fluxes fa, fb; us upwinded
// by fm from xL + sL/2 or xR - sR/2): its scaled difference
__device__ inline float momflux_d(float fa, float fb, float dfa, float dfb, float xL, float sL, float dxL,
                                  float dsL, float xR, float sR, float dxR, float dsR, float eps, float ieps)
{
    const float fm = 0.5f * (fa + fb), dfm = 0.5f * (dfa + dfb);
    float us, dus;
    upwind_d(fm, fmaf(eps, dfm, fm), xL + 0.5f * sL, dxL + 0.5f * dsL, xR - 0.5f * sR, dxR - 0.5f * dsR, ieps, us,
             dus);
    return dfm * fmaf(eps, dus, us) + fm * dus;
}

// Shared-memory plan of one TX x TY tile (the staging region and local
// coordinates of Tile2D): 6 FP64 planes (of which wall tiles use 4 for rho,
// e, u and v at U), then 21 FP32 planes.  The FP64 planes are dead once the
// neighbour differences are formed and then hold 12 of the 16 slope planes;
// the fluxes reuse difference planes, the momentum fluxes the scalars' slope
// planes.
template <int TX, int TY>
struct JvTile {
    static constexpr int RX = TX + 5, RY = TY + 5, R = RX * RY;
    static constexpr int N64 = 6, N32 = 21;
    static constexpr size_t SMEM = (size_t)R * (N64 * sizeof(double) + N32 * sizeof(float));
};

#define JV_RECT(x0, x1, y0, y1)                                                     \
    for (int k_ = tid, w_ = (x1) - (x0), n_ = ((x1) - (x0)) * ((y1) - (y0)); k_ < n_; \
         k_ += NT)                                                                  \
        for (int lx = (x0) + k_ % w_, ly = (y0) + k_ / w_, q = ly * RX + lx, once_ = 1; once_; once_ = 0)

// One tile (bx, by) of Jv by a CTA of TX*TY threads with JvTile::SMEM bytes
// at sm.  eps == 0 (a zero direction) gives Jv = 0, as the FP64 form does.
// FP32 copies of grid constants, formed once per launch on the host
struct JvConst {
    float ix0, ix1, gm1, g0, g1;
};

template <typename VIN, typename VOUT, int TX, int TY>
__device__ void jvdiff2d_tile(const GridParams &P, const JvConst &K, const double *U, const float *lin, const VIN *v,
                              VOUT *out, double hdt, const double *eps_dev, int bx, int by, double *sm)
{
    using TL = JvTile<TX, TY>;
    constexpr int RX = TL::RX, RY = TL::RY, R = TL::R, NT = TX * TY;
    constexpr int X0 = 3, X1 = 3 + TX, Y0 = 3, Y1 = 3 + TY;
    const int tid = threadIdx.x;
    const int tx = tid % TX, ty = tid / TX;
    const int gx = bx * TX + tx, gy = by * TY + ty;
    // eps and dt/2 (device values) converted once per CTA
    __shared__ double s_eps;
    __shared__ float s_k[3];
    if (tid == 0) {
        const double e = *eps_dev;
        s_eps = e;
        s_k[0] = (float)e;
        s_k[1] = (e != 0.0) ? 1.0f / (float)e : 0.0f;
        s_k[2] = (float)call_hdt(P, hdt);
    }
    __syncthreads();
    const double eps64 = s_eps;
    if (eps64 == 0.0) {
        if (gx < P.n[0] && gy < P.n[1]) {
            const long long c = gx + (long long)P.n[0] * gy;
            for (int k = 0; k < 4; k++) out[(long long)k * P.N + c] = (VOUT)0;
        }
        return;
    }
    const float eps = s_k[0], ieps = s_k[1];
    double *r64 = sm, *e64 = sm + R, *u64 = sm + 2 * R, *v64 = sm + 3 * R;  // general tiles only
    float *lo = (float *)sm;            // the FP64 region as 12 FP32 planes (after phase 1)
    float *fp = (float *)(sm + 6 * R);  // the 21 FP32 planes
    float *rf = fp, *ef = fp + R, *uf = fp + 2 * R, *vf = fp + 3 * R;
    float *dr = fp + 4 * R, *de = fp + 5 * R, *dE = fp + 6 * R, *du = fp + 7 * R, *dv = fp + 8 * R;
    float *Drx = fp + 9 * R, *Dry = fp + 10 * R, *Dex = fp + 11 * R, *Dey = fp + 12 * R;
    float *Dux = fp + 13 * R, *Duy = fp + 14 * R, *Dvx = fp + 15 * R, *Dvy = fp + 16 * R;
    // slopes at U and their differences
    float *srx = lo, *dsrx = lo + R, *sry = lo + 2 * R, *dsry = lo + 3 * R;
    float *sex = lo + 4 * R, *dsex = lo + 5 * R, *sey = lo + 6 * R, *dsey = lo + 7 * R;
    float *sux = lo + 8 * R, *dsux = lo + 9 * R, *suy = lo + 10 * R, *dsuy = lo + 11 * R;
    float *svx = fp + 17 * R, *dsvx = fp + 18 * R, *svy = fp + 19 * R, *dsvy = fp + 20 * R;
    // mass fluxes at U and the flux differences (difference planes dead after phase 2)
    float *Frx = Drx, *Fry = Dry, *dFrx = Dex, *dFry = Dey, *dFEx = Duy, *dFEy = Dvx;
    // momentum flux differences (rho / e slope planes dead after phase 3)
    float *dPhx = srx, *dPhy = dsrx, *dPsxy = sry, *dPsyx = dsry;
    const int i0 = bx * TX - 3, j0 = by * TY - 3;
    const long long N = P.N;
    // cells whose energy slopes and fluxes the tile needs (a sub-region of
    // the staged cross, where rho is needed)
    auto ine = [&](int lx, int ly) { return (ly >= Y0 && ly < Y1 && lx >= 1) || (lx >= X0 && lx < X1 && ly >= 1); };
    // A tile whose staged region reaches no wall ghost reads the values at U
    // from the linearisation planes of the last R / F evaluation; one that
    // does forms them from U as that evaluation did (FP64 e = E / rho and
    // u = m / rb, differences in FP64).  Both give the same bits.
    bool planes = true;
    if (P.bc[0] == MUSIC_BC_WALL) planes &= (i0 >= 0 && i0 + RX <= P.n[0]);
    if (P.bc[1] == MUSIC_BC_WALL) planes &= (j0 >= 0 && j0 + RY <= P.n[1]);

    if (planes) {
        // ---- phase 1 (plane tiles): values at U, the direction's entries
        // periodic images by repeated shifts: the staged region overhangs
        // the grid by less than one tile on either side
        // (the wrapped column and row offset of every staged point, formed
        // once per CTA)
        const int n0 = P.n[0], n1 = P.n[1];
        __shared__ int s_col[RX];
        __shared__ long long s_row[RY];
        for (int t = tid; t < RX + RY; t += NT) {
            if (t < RX) {
                int gx = i0 + t;
                while (gx < 0) gx += n0;
                while (gx >= n0) gx -= n0;
                s_col[t] = gx;
            } else {
                int gy = j0 + (t - RX);
                while (gy < 0) gy += n1;
                while (gy >= n1) gy -= n1;
                s_row[t - RX] = (long long)n0 * gy;
            }
        }
        __syncthreads();
        auto cidx = [&](int lx, int ly) { return s_row[ly] + s_col[lx]; };
        auto cell_at = [&](int lx, int ly, int q) {
            const long long c = cidx(lx, ly);
            const float r = lin[LIN_R * N + c], d1 = (float)v[c];
            rf[q] = r;
            dr[q] = d1;
            if (ine(lx, ly)) {
                const float e = lin[LIN_E * N + c], d2 = (float)v[N + c];
                ef[q] = e;
                dE[q] = d2;
                de[q] = __fdividef(d2 - e * d1, fmaf(eps, d1, r));
            }
        };
        JV_RECT(0, RX, Y0 - 1, Y1) cell_at(lx, ly, q);
        JV_RECT(X0 - 1, X1, 0, Y0 - 1) cell_at(lx, ly, q);
        JV_RECT(X0 - 1, X1, Y1, RY) cell_at(lx, ly, q);
        // face velocities; du, dv hold the momentum entries until phase 1b
        auto uface = [&](int lx, int ly, int q) {
            const long long c = cidx(lx, ly);
            uf[q] = lin[LIN_U * N + c];
            du[q] = (float)v[2 * N + c];
        };
        auto vface = [&](int lx, int ly, int q) {
            const long long c = cidx(lx, ly);
            vf[q] = lin[LIN_V * N + c];
            dv[q] = (float)v[3 * N + c];
        };
        JV_RECT(1, RX, Y0, Y1) uface(lx, ly, q);
        JV_RECT(X0, X1, 1, Y0) uface(lx, ly, q);
        JV_RECT(X0, X1, Y1, RY) uface(lx, ly, q);
        if (tid == 0) uface(X0 - 1, Y0 - 1, (Y0 - 1) * RX + X0 - 1);
        if (tid == 1) uface(X1, Y0 - 1, (Y0 - 1) * RX + X1);
        JV_RECT(X0, X1, 1, RY) vface(lx, ly, q);
        JV_RECT(1, X0, Y0, Y1) vface(lx, ly, q);
        JV_RECT(X1, RX, Y0, Y1) vface(lx, ly, q);
        if (tid == 2) vface(X0 - 1, Y0 - 1, (Y0 - 1) * RX + X0 - 1);
        if (tid == 3) vface(X0 - 1, Y1, Y1 * RX + X0 - 1);
        // neighbour differences at U
        JV_RECT(X0 - 2, X1 + 2, Y0 - 1, Y1) Drx[q] = lin[LIN_DRX * N + cidx(lx, ly)];
        JV_RECT(X0 - 1, X1, Y0 - 2, Y1 + 2) Dry[q] = lin[LIN_DRY * N + cidx(lx, ly)];
        JV_RECT(X0 - 1, X1 + 2, Y0, Y1) {
            const long long c = cidx(lx, ly);
            Dex[q] = lin[LIN_DEX * N + c];
            Dux[q] = lin[LIN_DUX * N + c];
            Dvx[q] = lin[LIN_DVX * N + c];
        }
        JV_RECT(X0, X1, Y0 - 1, Y1 + 2) {
            const long long c = cidx(lx, ly);
            Dey[q] = lin[LIN_DEY * N + c];
            Duy[q] = lin[LIN_DUY * N + c];
            Dvy[q] = lin[LIN_DVY * N + c];
        }
        __syncthreads();
        // ---- phase 1b: face velocity differences d(m / rb) = (dm - u drb) / rb'
        auto uvel = [&](int q, int p, float *vel, float *dvel) {
            const float rb = 0.5f * (rf[p] + rf[q]), drb = 0.5f * (dr[p] + dr[q]);
            dvel[q] = __fdividef(dvel[q] - vel[q] * drb, fmaf(eps, drb, rb));
        };
        JV_RECT(1, RX, Y0, Y1) uvel(q, q - 1, uf, du);
        JV_RECT(X0, X1, 1, Y0) uvel(q, q - 1, uf, du);
        JV_RECT(X0, X1, Y1, RY) uvel(q, q - 1, uf, du);
        if (tid == 0) uvel((Y0 - 1) * RX + X0 - 1, (Y0 - 1) * RX + X0 - 2, uf, du);
        if (tid == 1) uvel((Y0 - 1) * RX + X1, (Y0 - 1) * RX + X1 - 1, uf, du);
        JV_RECT(X0, X1, 1, RY) uvel(q, q - RX, vf, dv);
        JV_RECT(1, X0, Y0, Y1) uvel(q, q - RX, vf, dv);
        JV_RECT(X1, RX, Y0, Y1) uvel(q, q - RX, vf, dv);
        if (tid == 2) uvel((Y0 - 1) * RX + X0 - 1, (Y0 - 2) * RX + X0 - 1, vf, dv);
        if (tid == 3) uvel(Y1 * RX + X0 - 1, (Y1 - 1) * RX + X0 - 1, vf, dv);
        __syncthreads();
    } else {
        // ---- phase 1 (wall tiles): values at U in FP64 through the ghost
        // mapping, and the direction's entries (hydrostatic ghosts: the
        // extrapolation differenced in FP64)
        auto cell_at = [&](int lx, int ly, int q) {
            int j[3] = {i0 + lx, j0 + ly, 0};
            int lower;
            double r, E = 0.0;
            float d1, d2 = 0.0f;
            const bool wantE = ine(lx, ly);
            if (cell_map(P, j, lower) < 0) {
                const long long c = cell_index(P, j);
                r = U[c];
                d1 = (float)v[c];
                if (wantE) {
                    E = U[N + c];
                    d2 = (float)v[N + c];
                }
            } else {
                const int ix[3] = {i0 + lx, j0 + ly, 0};
                ghost_cell_d(P, U, v, eps64, ix, r, E, d1, d2);
            }
            const float r32 = (float)r;
            r64[q] = r;
            rf[q] = r32;
            dr[q] = d1;
            if (wantE) {
                const double e = E / r;
                const float e32 = (float)e;
                e64[q] = e;
                ef[q] = e32;
                dE[q] = d2;
                de[q] = __fdividef(d2 - e32 * d1, fmaf(eps, d1, r32));
            }
        };
        JV_RECT(0, RX, Y0 - 1, Y1) cell_at(lx, ly, q);
        JV_RECT(X0 - 1, X1, 0, Y0 - 1) cell_at(lx, ly, q);
        JV_RECT(X0 - 1, X1, Y1, RY) cell_at(lx, ly, q);
        // face velocity u = m / rb at U (as the stencil forms it, by the IEEE
        // division where the fused stencil's quotient is within 2 ulp of it)
        // and its difference
        auto face_at = [&](int lx, int ly, int q, int d, double *vel64, float *vel, float *dvel) {
            const int ix[3] = {i0 + lx, j0 + ly, 0};
            long long c, cl;
            double sgn;
            if (!face_map(P, ix, d, c, cl, sgn)) {
                vel64[q] = 0.0;
                vel[q] = 0.0f;
                dvel[q] = 0.0f;
                return;
            }
            const long long im = (long long)(2 + d) * N + c;
            const double rbar = 0.5 * (U[cl] + U[c]);
            const double u = sgn * (U[im] / rbar);
            const float u32 = (float)u, vm = (float)v[im];
            const float dm = (sgn > 0.0) ? vm : -vm;
            const float rb = 0.5f * ((float)U[cl] + (float)U[c]), drb = 0.5f * ((float)v[cl] + (float)v[c]);
            vel64[q] = u;
            vel[q] = u32;
            dvel[q] = __fdividef(dm - u32 * drb, fmaf(eps, drb, rb));
        };
        JV_RECT(1, RX, Y0, Y1) face_at(lx, ly, q, 0, u64, uf, du);
        JV_RECT(X0, X1, 1, Y0) face_at(lx, ly, q, 0, u64, uf, du);
        JV_RECT(X0, X1, Y1, RY) face_at(lx, ly, q, 0, u64, uf, du);
        if (tid == 0) face_at(X0 - 1, Y0 - 1, (Y0 - 1) * RX + X0 - 1, 0, u64, uf, du);
        if (tid == 1) face_at(X1, Y0 - 1, (Y0 - 1) * RX + X1, 0, u64, uf, du);
        JV_RECT(X0, X1, 1, RY) face_at(lx, ly, q, 1, v64, vf, dv);
        JV_RECT(1, X0, Y0, Y1) face_at(lx, ly, q, 1, v64, vf, dv);
        JV_RECT(X1, RX, Y0, Y1) face_at(lx, ly, q, 1, v64, vf, dv);
        if (tid == 2) face_at(X0 - 1, Y0 - 1, (Y0 - 1) * RX + X0 - 1, 1, v64, vf, dv);
        if (tid == 3) face_at(X0 - 1, Y1, Y1 * RX + X0 - 1, 1, v64, vf, dv);
        __syncthreads();
        // ---- phase 1b: differences of neighbouring values at U, in FP64
        // (backward: D[q] = x_q - x_p, p the lower neighbour)
        JV_RECT(X0 - 2, X1 + 2, Y0 - 1, Y1) Drx[q] = (float)(r64[q] - r64[q - 1]);
        JV_RECT(X0 - 1, X1, Y0 - 2, Y1 + 2) Dry[q] = (float)(r64[q] - r64[q - RX]);
        JV_RECT(X0 - 1, X1 + 2, Y0, Y1) {
            Dex[q] = (float)(e64[q] - e64[q - 1]);
            Dux[q] = (float)(u64[q] - u64[q - 1]);
            Dvx[q] = (float)(v64[q] - v64[q - 1]);
        }
        JV_RECT(X0, X1, Y0 - 1, Y1 + 2) {
            Dey[q] = (float)(e64[q] - e64[q - RX]);
            Duy[q] = (float)(u64[q] - u64[q - RX]);
            Dvy[q] = (float)(v64[q] - v64[q - RX]);
        }
        __syncthreads();
    }

    // ---- phase 2: limited slopes and their differences (FP64 planes now free)
    JV_RECT(X0 - 2, X1 + 1, Y0 - 1, Y1)
    vanleer_d(Drx[q], Drx[q + 1], dr[q] - dr[q - 1], dr[q + 1] - dr[q], eps, ieps, srx[q], dsrx[q]);
    JV_RECT(X0 - 1, X1 + 1, Y0, Y1) {
        vanleer_d(Dex[q], Dex[q + 1], de[q] - de[q - 1], de[q + 1] - de[q], eps, ieps, sex[q], dsex[q]);
        vanleer_d(Dux[q], Dux[q + 1], du[q] - du[q - 1], du[q + 1] - du[q], eps, ieps, sux[q], dsux[q]);
        vanleer_d(Dvx[q], Dvx[q + 1], dv[q] - dv[q - 1], dv[q + 1] - dv[q], eps, ieps, svx[q], dsvx[q]);
    }
    JV_RECT(X0 - 1, X1, Y0 - 2, Y1 + 1)
    vanleer_d(Dry[q], Dry[q + RX], dr[q] - dr[q - RX], dr[q + RX] - dr[q], eps, ieps, sry[q], dsry[q]);
    JV_RECT(X0, X1, Y0 - 1, Y1 + 1) {
        vanleer_d(Dey[q], Dey[q + RX], de[q] - de[q - RX], de[q + RX] - de[q], eps, ieps, sey[q], dsey[q]);
        vanleer_d(Duy[q], Duy[q + RX], du[q] - du[q - RX], du[q + RX] - du[q], eps, ieps, suy[q], dsuy[q]);
        vanleer_d(Dvy[q], Dvy[q + RX], dv[q] - dv[q - RX], dv[q + RX] - dv[q], eps, ieps, svy[q], dsvy[q]);
    }
    __syncthreads();

    // ---- phase 3: upwind mass and energy fluxes; the face velocity decides
    JV_RECT(X0 - 1, X1 + 1, Y0 - 1, Y1) {
        const float u = uf[q], dU = du[q], u2 = fmaf(eps, dU, u);
        float rs, drs;
        upwind_d(u, u2, rf[q - 1] + 0.5f * srx[q - 1], dr[q - 1] + 0.5f * dsrx[q - 1], rf[q] - 0.5f * srx[q],
                 dr[q] - 0.5f * dsrx[q], ieps, rs, drs);
        const float fr = u * rs, dfr = dU * fmaf(eps, drs, rs) + u * drs;
        if (lx >= X0 && ly >= Y0) {
            float es, des;
            upwind_d(u, u2, ef[q - 1] + 0.5f * sex[q - 1], de[q - 1] + 0.5f * dsex[q - 1], ef[q] - 0.5f * sex[q],
                     de[q] - 0.5f * dsex[q], ieps, es, des);
            dFEx[q] = dfr * fmaf(eps, des, es) + fr * des;
        }
        Frx[q] = fr;
        dFrx[q] = dfr;
    }
    JV_RECT(X0 - 1, X1, Y0 - 1, Y1 + 1) {
        const float u = vf[q], dU = dv[q], u2 = fmaf(eps, dU, u);
        float rs, drs;
        upwind_d(u, u2, rf[q - RX] + 0.5f * sry[q - RX], dr[q - RX] + 0.5f * dsry[q - RX], rf[q] - 0.5f * sry[q],
                 dr[q] - 0.5f * dsry[q], ieps, rs, drs);
        const float fr = u * rs, dfr = dU * fmaf(eps, drs, rs) + u * drs;
        if (lx >= X0 && ly >= Y0) {
            float es, des;
            upwind_d(u, u2, ef[q - RX] + 0.5f * sey[q - RX], de[q - RX] + 0.5f * dsey[q - RX],
                     ef[q] - 0.5f * sey[q], de[q] - 0.5f * dsey[q], ieps, es, des);
            dFEy[q] = dfr * fmaf(eps, des, es) + fr * des;
        }
        Fry[q] = fr;
        dFry[q] = dfr;
    }
    __syncthreads();

    // ---- phase 4: momentum flux differences (centres Phi, corners Psi)
    JV_RECT(X0 - 1, X1, Y0, Y1)
    dPhx[q] = momflux_d(Frx[q], Frx[q + 1], dFrx[q], dFrx[q + 1], uf[q], sux[q], du[q], dsux[q], uf[q + 1],
                        sux[q + 1], du[q + 1], dsux[q + 1], eps, ieps);
    JV_RECT(X0, X1, Y0 - 1, Y1)
    dPhy[q] = momflux_d(Fry[q], Fry[q + RX], dFry[q], dFry[q + RX], vf[q], svy[q], dv[q], dsvy[q], vf[q + RX],
                        svy[q + RX], dv[q + RX], dsvy[q + RX], eps, ieps);
    JV_RECT(X0, X1, Y0, Y1 + 1)
    dPsxy[q] = momflux_d(Fry[q - 1], Fry[q], dFry[q - 1], dFry[q], uf[q - RX], suy[q - RX], du[q - RX],
                         dsuy[q - RX], uf[q], suy[q], du[q], dsuy[q], eps, ieps);
    JV_RECT(X0, X1 + 1, Y0, Y1)
    dPsyx[q] = momflux_d(Frx[q - RX], Frx[q], dFrx[q - RX], dFrx[q], vf[q - 1], svx[q - 1], dv[q - 1],
                         dsvx[q - 1], vf[q], svx[q], dv[q], dsvx[q], eps, ieps);
    __syncthreads();

    // ---- phase 5: dR of the tile's cells and Jv = v - dt/2 dR
    if (gx >= P.n[0] || gy >= P.n[1]) return;
    const int q = (ty + Y0) * RX + (tx + X0);
    const float ix0 = K.ix0, ix1 = K.ix1, gm1 = K.gm1;
    const long long c = gx + (long long)P.n[0] * gy;
    float dR[4];
    {
        dR[0] = -((dFrx[q + 1] - dFrx[q]) * ix0 + (dFry[q + RX] - dFry[q]) * ix1);
        // p div u at U and its difference (div u from the FP64-formed differences)
        const float p = gm1 * rf[q] * ef[q], dp = gm1 * dE[q];
        const float divu = Dux[q + 1] * ix0 + Dvy[q + RX] * ix1;
        const float ddivu = (du[q + 1] - du[q]) * ix0 + (dv[q + RX] - dv[q]) * ix1;
        const float dpdiv = dp * fmaf(eps, ddivu, divu) + p * ddivu;
        dR[1] = -((dFEx[q + 1] - dFEx[q]) * ix0 + (dFEy[q + RX] - dFEy[q]) * ix1) - dpdiv;
    }
    if (P.bc[0] == MUSIC_BC_WALL && gx == 0) {
        dR[2] = 0.0f;
    } else {
        const float acc = (dPhx[q] - dPhx[q - 1]) * ix0 + (dPsxy[q + RX] - dPsxy[q]) * ix1;
        dR[2] = (-acc - gm1 * (dE[q] - dE[q - 1]) * ix0) + 0.5f * (dr[q - 1] + dr[q]) * K.g0;
    }
    if (P.bc[1] == MUSIC_BC_WALL && gy == 0) {
        dR[3] = 0.0f;
    } else {
        const float acc = (dPsyx[q + 1] - dPsyx[q]) * ix0 + (dPhy[q] - dPhy[q - RX]) * ix1;
        dR[3] = (-acc - gm1 * (dE[q] - dE[q - RX]) * ix1) + 0.5f * (dr[q - RX] + dr[q]) * K.g1;
    }
    const float h = s_k[2];
#pragma unroll
    for (int k = 0; k < 4; k++) {
        const long long i = (long long)k * P.N + c;
        out[i] = (VOUT)((float)v[i] - h * dR[k]);
    }
}
#undef JV_RECT

}  // namespace tile
