// Per-tile device code of the fused 2-D stencil (Sec. 2, Eqs. 1-3): used by
// the one-launch-per-evaluation kernel and by the persistent batched kernel.
#pragma once
#include "internal.h"

namespace tile {

template <typename VT>
struct WLoad {
    const double *U;
    const VT *v;        // Jv direction or null
    double eps;         // finite-difference step (Jv only)
    __device__ inline double operator()(long long i) const
    {
        double u = U[i];
        if (v) u = u + eps * (double)v[i];
        return u;
    }
};

// 2^K n / d (K = 0 or 1) within 2 ulp of the correctly rounded quotient,
// with four FP64-pipe operations: Newton's method for the reciprocal of d,
// started from a single-precision estimate y0 and taken to third order in
// one step, y = y0 (1 + e + e^2) with e = 1 - d y0, leaves a relative error
// of e^3 (below 2^-63) before the roundings of y and of 2^K n y.  The
// estimate is rcp.approx.ftz.f32 of d truncated to single precision
// (relative error below 2^-21 in all), and both conversions are done on the
// bit patterns: for d between 2^-120 and 2^120 they only move the exponent
// and the leading mantissa bits, and the factor 2^K goes into the exponent
// of the estimate (the iteration's steps scale exactly with it).  Any other d
// (zero, subnormal, huge, infinite, NaN) takes the IEEE division.  The
// result is odd in n and in d: negating either only flips sign bits.
template <int K>
__device__ __forceinline__ double newton_quot(double n, double d)
{
    const int hi = __double2hiint(d);
    const unsigned lo = (unsigned)__double2loint(d);
    const int E = (hi >> 20) & 0x7ff;
    if ((unsigned)(E - (1023 - 120)) > 240u) return K ? (2.0 * n) / d : n / d;
    const int fb = (hi & (int)0x80000000) | ((E - 896) << 23) | ((hi & 0xfffff) << 3) | (int)(lo >> 29);
    float rf;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(rf) : "f"(__int_as_float(fb)));
    const int rb = __float_as_int(rf);
    const int rhi = (rb & (int)0x80000000) | ((((rb >> 23) & 0xff) + 896) << 20) | ((rb & 0x7fffff) >> 3);
    const int rlo = (rb & 7) << 29;
    const double y0 = __hiloint2double(rhi, rlo);
    const double yk = K ? __hiloint2double(rhi + (1 << 20), rlo) : y0;
    const double e = fma(-d, y0, 1.0);
    return n * fma(yk, fma(e, e, e), yk);
}

// 2n / d, for van Leer's slope
__device__ __forceinline__ double twice_quot(double n, double d) { return newton_quot<1>(n, d); }

// n / d, for the specific internal energy E / rho and the face velocities
// m_d / rbar that the fused 2-D tiles stage.  (The multi-pass stencil keeps
// the IEEE division: on conducting grids T = (gamma - 1) e enters the
// radiative flux through differences of neighbouring cells, whose
// cancellation in radiative equilibrium would turn a quotient 2 ulp off into
// an operator error above 1e-12 of the oracle's.)
__device__ __forceinline__ double quot(double n, double d) { return newton_quot<0>(n, d); }

// van Leer's limited slope 2ab / (a + b) of the one-sided differences a and
// b where a b > 0, else 0 (Sec. 2).  The sign test reads the bit patterns:
// a and b nonzero, neither NaN, and of one sign.  (Where a b underflows to
// zero the numerator is that zero, so the slope is zero as the product's
// test would make it.)
__device__ inline double vanleer(double a, double b)
{
    const long long ia = __double_as_longlong(a), ib = __double_as_longlong(b);
    const unsigned long long ma = (unsigned long long)ia << 1, mb = (unsigned long long)ib << 1;
    const unsigned long long inf2 = 0xffe0000000000000ull;
    if ((ia ^ ib) < 0 || ma - 1 >= inf2 || mb - 1 >= inf2) return 0.0;
    return twice_quot(a * b, a + b);
}

// Ghost mapping of cell ix (in place into j, which starts as ix): periodic
// images and mirror walls map to an interior cell; the return value is the
// direction of a hydrostatic wall ghost (Sec. 3), -1 if none, with `lower`
// telling which wall.
__device__ inline int cell_map(const GridParams &P, int j[3], int &lower)
{
    int hd = -1;
    lower = 0;
    for (int d = 0; d < P.nd; d++) {
        const int n = P.n[d];
        // tile halos of ragged edges may lie beyond the ghost layers; their
        // values are never used, so clamp wall directions into the ghost range
        const int a = (P.bc[d] == MUSIC_BC_WALL) ? min(max(j[d], -MUSIC_GHOST), n - 1 + MUSIC_GHOST) : j[d];
        if (a >= 0 && a < n) continue;
        if (P.bc[d] == MUSIC_BC_PERIODIC)
            j[d] = (a % n + n) % n;
        else if (P.ws[d] == MUSIC_WALL_MIRROR)
            j[d] = (a < 0) ? (-1 - a) : (2 * n - 1 - a);
        else {
            hd = d;
            lower = (a < 0);
        }
    }
    return hd;
}

// (rho, E) of cell ix through the ghost mapping: periodic images, mirror
// walls, or the hydrostatic extrapolation of Sec. 3; W loads a state entry
template <typename LD>
__device__ void load_cell(const GridParams &P, const LD &W, const int ix[3], double &rho, double &E)
{
    int j[3] = {ix[0], ix[1], ix[2]};
    int lower;
    const int hd = cell_map(P, j, lower);
    if (hd < 0) {
        const long long c = cell_index(P, j);
        rho = W(c);
        E = W(P.N + c);
        return;
    }
    const int n = P.n[hd];
    j[hd] = lower ? 0 : n - 1;
    const long long c0 = cell_index(P, j);
    j[hd] = lower ? 1 : n - 2;
    const long long c1 = cell_index(P, j);
    const double r0 = W(c0), r1 = W(c1);
    const double T0 = (P.gm1 * W(P.N + c0)) / r0;
    const double T1 = (P.gm1 * W(P.N + c1)) / r1;
    const double Tg = 2.0 * T0 - T1;
    const double hs = 0.5 * P.dx[hd] * face_g(P, hd, lower ? 0 : n);
    const double rg = lower ? __dmul_rn(r0, T0 - hs) / (Tg + hs) : __dmul_rn(r0, T0 + hs) / (Tg - hs);
    rho = rg;
    E = __dmul_rn(rg, Tg) / P.gm1;
}

// Ghost mapping of the d-face at ix (the face between cells ix - e_d and
// ix): false when the face lies on a wall and its velocity is zero; else
// the stored face c, its lower neighbour cl (both interior cells) and the
// sign of the mirrored velocity.
__device__ inline bool face_map(const GridParams &P, const int ix[3], int d, long long &c, long long &cl,
                                double &sgn)
{
    int j[3] = {ix[0], ix[1], ix[2]};
    sgn = 1.0;
    for (int w = 0; w < P.nd; w++) {
        const int n = P.n[w];
        const int a = (P.bc[w] == MUSIC_BC_WALL) ? min(max(j[w], -MUSIC_GHOST), n - 1 + MUSIC_GHOST) : j[w];
        j[w] = a;
        if (a >= 0 && a < n) continue;
        if (P.bc[w] == MUSIC_BC_PERIODIC) {
            j[w] = (a % n + n) % n;
        } else if (w == d) {
            if (a == n) return false;
            j[w] = (a < 0) ? -a : 2 * n - a;
            sgn = -sgn;
        } else {
            j[w] = (a < 0) ? (-1 - a) : (2 * n - 1 - a);
        }
    }
    if (P.bc[d] == MUSIC_BC_WALL && j[d] == 0) return false;
    c = cell_index(P, j);
    int l[3] = {j[0], j[1], j[2]};
    l[d] = (j[d] == 0) ? P.n[d] - 1 : j[d] - 1;
    cl = cell_index(P, l);
    return true;
}

// staggered velocity of the d-face at ix: face momentum over the mean
// density of the two cells it joins.  The fused 2-D tiles take the quotient
// by quot (NEWTON); the multi-pass stencil, which also serves the spherical
// and conducting grids, by the IEEE division.
template <bool NEWTON, typename VT>
__device__ double face_velocity(const GridParams &P, const WLoad<VT> &W, const int ix[3], int d)
{
    long long c, cl;
    double sgn;
    if (!face_map(P, ix, d, c, cl, sgn)) return 0.0;
    const double rbar = 0.5 * (W(cl) + W(c));
    const double m = W((long long)(2 + d) * P.N + c);
    return sgn * (NEWTON ? quot(m, rbar) : m / rbar);
}

// ---------------------------------------------------------------- fused 2-D
// One kernel per evaluation of R on 2-D grids.  A CTA owns a TX x TY tile of
// cells [X0, X1) x [Y0, Y1) (local coordinates) and stages the tile plus a
// halo of 3 cells below / 2 above in shared memory (RX x RY points, x
// fastest).  Each intermediate is computed once, and only on the exact
// sub-rectangle that the tile's residuals reach (the stencil is a cross, not
// a square), which keeps the FP64 quotients (E / rho, m / rbar, the slopes;
// each a Newton step for the reciprocal) near the minimum of 11 per cell:
//   1 ghost-mapped rho, e, p and face velocities u, v (global loads, L1/L2)
//   2 van Leer slopes of rho, e, u, v along x and y
//   3 upwind mass and energy fluxes on x- and y-faces
//   4 momentum fluxes: centres (Phi) and corners (Psi)
//   5 the residuals of the tile's cells, written per mode (coalesced in x).
template <int TX, int TY>
struct Tile2D {
    static constexpr int RX = TX + 5, RY = TY + 5, R = RX * RY, NARR = 16;
    static constexpr int X0 = 3, X1 = 3 + TX, Y0 = 3, Y1 = 3 + TY;
    static constexpr size_t SMEM = (size_t)NARR * R * sizeof(double);
};

// loop of the CTA's threads over the local rectangle [x0,x1) x [y0,y1)
#define TILE_RECT(x0, x1, y0, y1)                                                   \
    for (int k_ = tid, w_ = (x1) - (x0), n_ = ((x1) - (x0)) * ((y1) - (y0)); k_ < n_; \
         k_ += NT)                                                                  \
        for (int lx = (x0) + k_ % w_, ly = (y0) + k_ / w_, q = ly * RX + lx, once_ = 1; once_; once_ = 0)

// One tile (bx, by) of the fused stencil, run by a CTA of TX*TY threads with
// Tile2D<TX, TY>::SMEM bytes of shared memory at `sm`.  epsv is the finite-
// difference step (SM_JV).  Fr_out (null: none) receives the mass fluxes of
// the tile cells' lower x- and y-faces (2 planes of N) for passive scalars;
// lin (null: none; R and F modes) the linearisation planes (LinPlane).
// Callable from any kernel that owns such a CTA.
template <int MODE, typename VIN, typename VOUT, int TX, int TY>
__device__ void fused2d_tile(const GridParams &P, const double *U, const double *aux, const VIN *v, VOUT *out,
                             double *RU_out, double hdt, double sign, double epsv, int bx, int by, double *sm,
                             double *Fr_out = nullptr, float *lin = nullptr, double *Cn_out = nullptr)
{
    using TL = Tile2D<TX, TY>;
    constexpr int RX = TL::RX, RY = TL::RY, R = TL::R, NT = TX * TY;
    constexpr int X0 = TL::X0, X1 = TL::X1, Y0 = TL::Y0, Y1 = TL::Y1;
    // (no pressure plane: phase 5 forms p = (gamma - 1) E of its three cells
    // from U again, which keeps a 16 x 16 tile at four CTAs per SM)
    double *rho = sm, *ee = sm + R, *uu = sm + 2 * R, *vv = sm + 3 * R;
    double *srx = sm + 4 * R, *sry = sm + 5 * R, *sex = sm + 6 * R, *sey = sm + 7 * R;
    double *sux = sm + 8 * R, *suy = sm + 9 * R, *svx = sm + 10 * R, *svy = sm + 11 * R;
    double *Frx = sm + 12 * R, *Fry = sm + 13 * R, *FEx = sm + 14 * R, *FEy = sm + 15 * R;
    // scalar slopes are dead after phase 3: their planes hold the momentum fluxes
    double *Phx = srx, *Phy = sry, *Psxy = sex, *Psyx = sey;
    const int i0 = bx * TX - 3, j0 = by * TY - 3;
    const int tid = threadIdx.x;
    const WLoad<VIN> W{U, (MODE == SM_JV) ? v : nullptr, epsv};

    // ---- phase 1: cell scalars on the cross-shaped region, face velocities
    // (a tile whose staged region lies inside the grid indexes its cells
    // directly: no ghost, wall face or periodic image to map, so the same
    // operations on the same values as the ghost-mapping path)
    const bool inner = i0 >= 0 && i0 + RX <= P.n[0] && j0 >= 0 && j0 + RY <= P.n[1];
    const long long cs1 = P.cs[1];
    auto cix = [&](int lx, int ly) { return (long long)(i0 + lx) + cs1 * (j0 + ly); };
    auto rho_at = [&](int lx, int ly, int q) {
        if (inner) {
            rho[q] = W(cix(lx, ly));
            return;
        }
        const int ix[3] = {i0 + lx, j0 + ly, 0};
        double r, E;
        load_cell(P, W, ix, r, E);
        rho[q] = r;
    };
    auto e_at = [&](int lx, int ly, int q) {
        double r, E;
        if (inner) {
            const long long c = cix(lx, ly);
            r = W(c);
            E = W(P.N + c);
        } else {
            const int ix[3] = {i0 + lx, j0 + ly, 0};
            load_cell(P, W, ix, r, E);
        }
        ee[q] = quot(E, r);
    };
    auto u_at = [&](int lx, int ly, int q) {
        if (inner) {
            const long long c = cix(lx, ly);
            const double rbar = 0.5 * (W(c - 1) + W(c));
            uu[q] = quot(W(2 * P.N + c), rbar);
            return;
        }
        const int ix[3] = {i0 + lx, j0 + ly, 0};
        uu[q] = face_velocity<true>(P, W, ix, 0);
    };
    auto v_at = [&](int lx, int ly, int q) {
        if (inner) {
            const long long c = cix(lx, ly);
            const double rbar = 0.5 * (W(c - cs1) + W(c));
            vv[q] = quot(W(3 * P.N + c), rbar);
            return;
        }
        const int ix[3] = {i0 + lx, j0 + ly, 0};
        vv[q] = face_velocity<true>(P, W, ix, 1);
    };
    TILE_RECT(0, RX, Y0 - 1, Y1) rho_at(lx, ly, q);
    TILE_RECT(X0 - 1, X1, 0, Y0 - 1) rho_at(lx, ly, q);
    TILE_RECT(X0 - 1, X1, Y1, RY) rho_at(lx, ly, q);
    TILE_RECT(1, RX, Y0, Y1) e_at(lx, ly, q);
    TILE_RECT(X0, X1, 1, Y0) e_at(lx, ly, q);
    TILE_RECT(X0, X1, Y1, RY) e_at(lx, ly, q);
    TILE_RECT(1, RX, Y0, Y1) u_at(lx, ly, q);
    TILE_RECT(X0, X1, 1, Y0) u_at(lx, ly, q);
    TILE_RECT(X0, X1, Y1, RY) u_at(lx, ly, q);
    if (tid == 0) u_at(X0 - 1, Y0 - 1, (Y0 - 1) * RX + X0 - 1);
    if (tid == 1) u_at(X1, Y0 - 1, (Y0 - 1) * RX + X1);
    TILE_RECT(X0, X1, 1, RY) v_at(lx, ly, q);
    TILE_RECT(1, X0, Y0, Y1) v_at(lx, ly, q);
    TILE_RECT(X1, RX, Y0, Y1) v_at(lx, ly, q);
    if (tid == 2) v_at(X0 - 1, Y0 - 1, (Y0 - 1) * RX + X0 - 1);
    if (tid == 3) v_at(X0 - 1, Y1, Y1 * RX + X0 - 1);
    __syncthreads();

    // ---- phase 2: limited slopes, each on the rectangle its fluxes need
    TILE_RECT(X0 - 2, X1 + 1, Y0 - 1, Y1) srx[q] = vanleer(rho[q] - rho[q - 1], rho[q + 1] - rho[q]);
    TILE_RECT(X0 - 1, X1 + 1, Y0, Y1) sex[q] = vanleer(ee[q] - ee[q - 1], ee[q + 1] - ee[q]);
    TILE_RECT(X0 - 1, X1, Y0 - 2, Y1 + 1) sry[q] = vanleer(rho[q] - rho[q - RX], rho[q + RX] - rho[q]);
    TILE_RECT(X0, X1, Y0 - 1, Y1 + 1) sey[q] = vanleer(ee[q] - ee[q - RX], ee[q + RX] - ee[q]);
    TILE_RECT(X0 - 1, X1 + 1, Y0, Y1) {
        sux[q] = vanleer(uu[q] - uu[q - 1], uu[q + 1] - uu[q]);
        svx[q] = vanleer(vv[q] - vv[q - 1], vv[q + 1] - vv[q]);
    }
    TILE_RECT(X0, X1, Y0 - 1, Y1 + 1) {
        suy[q] = vanleer(uu[q] - uu[q - RX], uu[q + RX] - uu[q]);
        svy[q] = vanleer(vv[q] - vv[q - RX], vv[q + RX] - vv[q]);
    }
    __syncthreads();

    // ---- phase 3: upwind mass and energy fluxes
    TILE_RECT(X0 - 1, X1 + 1, Y0 - 1, Y1) {
        const double u = uu[q];
        const bool up = (u >= 0.0);
        const double rs = up ? rho[q - 1] + 0.5 * srx[q - 1] : rho[q] - 0.5 * srx[q];
        const double fr = u * rs;
        Frx[q] = fr;
        if (lx >= X0 && ly >= Y0) {
            const double es = up ? ee[q - 1] + 0.5 * sex[q - 1] : ee[q] - 0.5 * sex[q];
            FEx[q] = fr * es;
        }
    }
    TILE_RECT(X0 - 1, X1, Y0 - 1, Y1 + 1) {
        const double u = vv[q];
        const bool up = (u >= 0.0);
        const double rs = up ? rho[q - RX] + 0.5 * sry[q - RX] : rho[q] - 0.5 * sry[q];
        const double fr = u * rs;
        Fry[q] = fr;
        if (lx >= X0 && ly >= Y0) {
            const double es = up ? ee[q - RX] + 0.5 * sey[q - RX] : ee[q] - 0.5 * sey[q];
            FEy[q] = fr * es;
        }
    }
    __syncthreads();

    // ---- phase 4: momentum fluxes
    TILE_RECT(X0 - 1, X1, Y0, Y1) {
        const double fm = 0.5 * (Frx[q] + Frx[q + 1]);
        const double us = (fm >= 0.0) ? uu[q] + 0.5 * sux[q] : uu[q + 1] - 0.5 * sux[q + 1];
        Phx[q] = fm * us;
    }
    TILE_RECT(X0, X1, Y0 - 1, Y1) {
        const double fm = 0.5 * (Fry[q] + Fry[q + RX]);
        const double us = (fm >= 0.0) ? vv[q] + 0.5 * svy[q] : vv[q + RX] - 0.5 * svy[q + RX];
        Phy[q] = fm * us;
    }
    TILE_RECT(X0, X1, Y0, Y1 + 1) {
        const double fm = 0.5 * (Fry[q - 1] + Fry[q]);
        const double us = (fm >= 0.0) ? uu[q - RX] + 0.5 * suy[q - RX] : uu[q] - 0.5 * suy[q];
        Psxy[q] = fm * us;
    }
    TILE_RECT(X0, X1 + 1, Y0, Y1) {
        const double fm = 0.5 * (Frx[q - RX] + Frx[q]);
        const double us = (fm >= 0.0) ? vv[q - 1] + 0.5 * svx[q - 1] : vv[q] - 0.5 * svx[q];
        Psyx[q] = fm * us;
    }
    __syncthreads();

    // ---- phase 5: residuals of the tile
    const int tx = tid % TX, ty = tid / TX;
    const int gx = bx * TX + tx, gy = by * TY + ty;
    if (gx >= P.n[0] || gy >= P.n[1]) return;
    const int q = (ty + Y0) * RX + (tx + X0);
    const double ix0 = P.idx[0], ix1 = P.idx[1];
    // p = (gamma - 1) E of the cell offset by (dx, dy), E as phase 1 loads
    // it; the product rounded on its own, as a stored value would be (a
    // product contracted into the difference below would break the exact
    // mirror symmetry of the operator)
    auto p_at = [&](int dx, int dy) {
        double r, E;
        if (inner) {
            E = W(P.N + cix(tx + X0 + dx, ty + Y0 + dy));
        } else {
            const int ix[3] = {gx + dx, gy + dy, 0};
            load_cell(P, W, ix, r, E);
        }
        return __dmul_rn(P.gm1, E);
    };
    const double pc = p_at(0, 0);
    double Rv[4];
    {
        double accr = (Frx[q + 1] - Frx[q]) * ix0;
        accr += (Fry[q + RX] - Fry[q]) * ix1;
        double acce = (FEx[q + 1] - FEx[q]) * ix0;
        acce += (FEy[q + RX] - FEy[q]) * ix1;
        double divu = (uu[q + 1] - uu[q]) * ix0;
        divu += (vv[q + RX] - vv[q]) * ix1;
        Rv[0] = -accr;
        Rv[1] = -acce - pc * divu;
    }
    if (P.bc[0] == MUSIC_BC_WALL && gx == 0) {
        Rv[2] = 0.0;
    } else {
        double acc = (Phx[q] - Phx[q - 1]) * ix0;
        acc += (Psxy[q + RX] - Psxy[q]) * ix1;
        const double rbar = 0.5 * (rho[q - 1] + rho[q]);
        Rv[2] = (-acc - (pc - p_at(-1, 0)) * ix0) + rbar * P.g[0];
    }
    if (P.bc[1] == MUSIC_BC_WALL && gy == 0) {
        Rv[3] = 0.0;
    } else {
        double acc = (Psyx[q + 1] - Psyx[q]) * ix0;
        acc += (Phy[q] - Phy[q - RX]) * ix1;
        const double rbar = 0.5 * (rho[q - RX] + rho[q]);
        Rv[3] = (-acc - (pc - p_at(0, -1)) * ix1) + rbar * P.g[1];
    }
    const long long c = gx + (long long)P.n[0] * gy;
    if (MODE != SM_JV && Fr_out) {
        Fr_out[c] = Frx[q];
        Fr_out[P.N + c] = Fry[q];
    }
    if (MODE != SM_JV && lin) {
        const long long N = P.N;
        lin[LIN_R * N + c] = (float)rho[q];
        lin[LIN_E * N + c] = (float)ee[q];
        lin[LIN_U * N + c] = (float)uu[q];
        lin[LIN_V * N + c] = (float)vv[q];
        lin[LIN_DRX * N + c] = (float)(rho[q] - rho[q - 1]);
        lin[LIN_DRY * N + c] = (float)(rho[q] - rho[q - RX]);
        lin[LIN_DEX * N + c] = (float)(ee[q] - ee[q - 1]);
        lin[LIN_DEY * N + c] = (float)(ee[q] - ee[q - RX]);
        lin[LIN_DUX * N + c] = (float)(uu[q] - uu[q - 1]);
        lin[LIN_DUY * N + c] = (float)(uu[q] - uu[q - RX]);
        lin[LIN_DVX * N + c] = (float)(vv[q] - vv[q - 1]);
        lin[LIN_DVY * N + c] = (float)(vv[q] - vv[q - RX]);
    }
    const double c_jv = (MODE == SM_JV && epsv != 0.0) ? hdt / epsv : 0.0;
#pragma unroll
    for (int k = 0; k < 4; k++) {
        const long long i = (long long)k * P.N + c;
        if (MODE == SM_R) {
            out[i] = (VOUT)Rv[k];
        } else if (MODE == SM_CN) {
            out[i] = (VOUT)(U[i] + hdt * Rv[k]);
        } else if (MODE == SM_F) {
            out[i] = (VOUT)(sign * ((U[i] - aux[i]) - hdt * Rv[k]));
            if (RU_out) RU_out[i] = Rv[k];
        } else if (MODE == SM_CNF) {
            // the step constant as SM_CN writes it, then the residual as SM_F forms it from that value
            const double cn = U[i] + hdt * Rv[k];
            Cn_out[i] = cn;
            out[i] = (VOUT)(sign * ((U[i] - cn) - hdt * Rv[k]));
            if (RU_out) RU_out[i] = Rv[k];
        } else {
            out[i] = (epsv == 0.0) ? (VOUT)0 : (VOUT)((double)v[i] - c_jv * (Rv[k] - aux[i]));
        }
    }
}
#undef TILE_RECT

}  // namespace tile
