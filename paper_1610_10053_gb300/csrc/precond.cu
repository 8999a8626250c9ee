// Physics-based semi-implicit preconditioner (Sec. 2, after Park et al. 2009):
// the stiff acoustic subsystem of J = I - dt/2 dR/dU with coefficients frozen
// at the Newton iterate; advection and gravity are treated as absent:
//   drho + tau div(dm) = r_rho
//   dE   + tau hp div(dm / rbar) = r_E,        hp = E + p = gamma E
//   dm   + tau grad(dp) = r_m,                  dp = (gamma - 1) dE
// with tau = dt/2.  Eliminating dm gives the pressure Helmholtz problem
//   dp/gp - tau^2 div(grad(dp)/rbar) = (gamma-1) r_E/gp - tau div(r_m/rbar),
// gp = gamma p, relaxed with a fixed number of weighted-Jacobi sweeps from
// zero (so M^-1 is a fixed linear map, as GMRES needs, and commutes with the
// grid's mirror symmetries); dm, drho, dE follow by back substitution in flux
// form, which keeps sum(drho) = sum(r_rho) and sum(dm) = sum(r_m).
//
// PT is float in mixed precision and double otherwise.
#include <cmath>

#include "internal.h"
#include "tile_precond.cuh"
#include "tiles.h"

namespace {

using namespace tile;

constexpr int BS = 256;

// grid constants in the preconditioner's type, formed once per launch on the host
template <typename PT>
struct PcK {
    PT idx[3], idx2[3], gm1;
};

template <typename PT>
PcK<PT> pck_of(const GridParams &P)
{
    PcK<PT> K;
    for (int d = 0; d < 3; d++) {
        K.idx[d] = (PT)P.idx[d];
        K.idx2[d] = (PT)P.idx2[d];
    }
    K.gm1 = (PT)P.gm1;
    return K;
}

// tau and tau^2 of the launch (from the device dt when the grid has one),
// converted once per CTA
template <typename PT>
__device__ __forceinline__ void block_tau(const GridParams &P, PT &tau, PT &tau2)
{
    __shared__ PT s_t[2];
    if (threadIdx.x == 0) {
        call_tau(P, tau, tau2);
        s_t[0] = tau;
        s_t[1] = tau2;
    }
    __syncthreads();
    tau = s_t[0];
    tau2 = s_t[1];
}

template <typename PT>
__device__ inline PT a_up(const GridParams &P, const PC<PT> &C, const int ix[3], int d)
{
    return upper_wall(P, ix, d) ? (PT)0 : C.a[d][cell_nb(P, ix, d, +1)];
}

// Coefficients frozen at U and the Helmholtz diagonal, in one pass: 1/rbar on
// the lower d-faces (zero on walls), gamma p, gamma E, and
// D = 1/(gamma p) + tau^2 sum_d (a_d + a_d+) / dx_d^2, where the upper face's
// a_d+ is formed exactly as its own cell forms it as a lower face.  An FP32
// preconditioner (PT = float) forms them from the state rounded to FP32, with
// FP32 arithmetic: they are stored in FP32 either way, and FP64 divisions and
// conversions per cell run at 1/64 of the FP32 rate on this part.
// g1 = gamma (gamma - 1) and g2 = gamma in PT.
template <typename PT>
__device__ __forceinline__ PT face_coef(const GridParams &P, const double *U, long long lo, long long hi)
{
    if constexpr (sizeof(PT) == 4)
        return 2.0f / ((float)U[lo] + (float)U[hi]);
    else
        return (PT)(1.0 / (0.5 * (U[lo] + U[hi])));
}

template <typename PT>
__global__ void __launch_bounds__(BS) k_setup(GridParams P, const double *U, PC<PT> C, PcK<PT> K, PT g1, PT g2,
                                              PT tau2)
{
    pdl_entry();
    PT tau_unused = 0;
    block_tau(P, tau_unused, tau2);
    for (long long c = blockIdx.x * (long long)BS + threadIdx.x; c < P.N; c += (long long)gridDim.x * BS) {
        int ix[3];
        cell_coords(P, c, ix);
        PT gp;
        if constexpr (sizeof(PT) == 4) {
            const float E = (float)U[P.N + c];
            gp = g1 * E;
            C.hp[c] = g2 * E;
        } else {
            const double E = U[P.N + c];
            gp = (PT)(P.gamma * (P.gm1 * E));
            C.hp[c] = (PT)(P.gamma * E);
        }
        C.gp[c] = gp;
        PT diag = 0;
        for (int d = 0; d < P.nd; d++) {
            const PT am = lower_wall(P, ix, d) ? (PT)0 : face_coef<PT>(P, U, cell_nb(P, ix, d, -1), c);
            const PT ap = upper_wall(P, ix, d) ? (PT)0 : face_coef<PT>(P, U, c, cell_nb(P, ix, d, +1));
            C.a[d][c] = am;
            diag += (ap + am) * K.idx2[d];
        }
        C.D[c] = (PT)1 / gp + tau2 * diag;
    }
}

// Right-hand side of the pressure system of one cell from its r_E, gamma p,
// and per direction the upper and lower face coefficients and momentum
// residuals (shared by the per-cell and the chunked kernels: the same bits)
// (every product and fused step is spelled out, so the compiler's choice of
// contractions cannot differ between the kernels that inline it)
template <typename PT>
__device__ __forceinline__ PT rhs_value(int nd, PT rE, PT gp, const PT *ap, const PT *rp, const PT *am,
                                        const PT *rm, const PcK<PT> &K, PT tau)
{
    PT divm = 0;
#pragma unroll
    for (int d = 0; d < 3; d++) {
        if (d >= nd) break;
        divm = pfma(pfma(ap[d], rp[d], -pmul_rn(am[d], rm[d])), K.idx[d], divm);
    }
    return pfma(-tau, divm, pmul_rn(K.gm1, rE) / gp);
}

template <typename PT, typename RT>
__global__ void __launch_bounds__(BS) k_rhs(GridParams P, PC<PT> C, PcK<PT> K, const RT *r, PT *b, PT tau)
{
    pdl_entry();
    PT tau2_unused = 0;
    block_tau(P, tau, tau2_unused);
    for (long long c = blockIdx.x * (long long)BS + threadIdx.x; c < P.N; c += (long long)gridDim.x * BS) {
        int ix[3];
        cell_coords(P, c, ix);
        PT ap[3], rp[3], am[3], rm[3];
#pragma unroll
        for (int d = 0; d < 3; d++) {
            ap[d] = rp[d] = am[d] = rm[d] = (PT)0;
            if (d >= P.nd) break;
            ap[d] = a_up(P, C, ix, d);
            am[d] = C.a[d][c];
            rp[d] = (PT)r[(2 + d) * P.N + cell_nb(P, ix, d, +1)];
            rm[d] = (PT)r[(2 + d) * P.N + c];
        }
        b[c] = rhs_value<PT>(P.nd, (PT)r[P.N + c], C.gp[c], ap, rp, am, rm, K, tau);
    }
}

// dq = (1 - w) dp + w (b + tau^2 sum a dp_nb / dx^2) / D; first sweep from 0
template <typename PT, bool FIRST>
__global__ void __launch_bounds__(BS) k_jacobi(GridParams P, PC<PT> C, PcK<PT> K, const PT *b, const PT *dp,
                                               PT *dq, PT tau2)
{
    pdl_entry();
    PT tau_unused = 0;
    block_tau(P, tau_unused, tau2);
    const PT w = (PT)MUSIC_JACOBI_OMEGA;
    for (long long c = blockIdx.x * (long long)BS + threadIdx.x; c < P.N; c += (long long)gridDim.x * BS) {
        if (FIRST) {
            dq[c] = w * (b[c] / C.D[c]);
            continue;
        }
        int ix[3];
        cell_coords(P, c, ix);
        PT off = 0;
        for (int d = 0; d < P.nd; d++) {
            const PT ap = a_up(P, C, ix, d), am = C.a[d][c];
            off += (ap * dp[cell_nb(P, ix, d, +1)] + am * dp[cell_nb(P, ix, d, -1)]) * K.idx2[d];
        }
        dq[c] = ((PT)1 - w) * dp[c] + w * ((b[c] + tau2 * off) / C.D[c]);
    }
}

// The weighted-Jacobi update of one cell from its dp, its neighbours' along
// each direction (upper dpu, lower dpd), its upper and lower face
// coefficients, its right-hand side and diagonal: one expression, shared by
// the per-cell and the vectorised sweeps so that both give the same bits.
template <typename PT>
__device__ __forceinline__ PT jacobi_value(int nd, PT dpc, const PT *dpu, const PT *dpd, const PT *ap,
                                           const PT *am, PT bc, PT Dc, const PcK<PT> &K, PT tau2, PT w)
{
    PT off = 0;
#pragma unroll
    for (int d = 0; d < 3; d++) {
        if (d >= nd) break;
        off += (ap[d] * dpu[d] + am[d] * dpd[d]) * K.idx2[d];
    }
    return ((PT)1 - w) * dpc + w * ((bc + tau2 * off) / Dc);
}

// One weighted-Jacobi update of cell c (coordinates ix) from dp, with the
// neighbour rule of cell_nb (periodic wrap; at a wall the neighbour beyond it
// is the cell itself, whose wall coefficient is zero); nb(cell) returns dp at
// an interior cell index.
template <typename PT, typename NB>
__device__ __forceinline__ PT jacobi_cell(const GridParams &P, const PC<PT> &C, const PcK<PT> &K, const PT *b,
                                          const int ix[3], long long c, PT tau2, PT w, NB &&nb)
{
    PT dpu[3], dpd[3], ap[3], am[3];
#pragma unroll
    for (int d = 0; d < 3; d++) {
        dpu[d] = dpd[d] = ap[d] = am[d] = (PT)0;
        if (d >= P.nd) break;
        const int n = P.n[d], a = ix[d];
        const long long st = P.cs[d];
        const bool per = P.bc[d] == MUSIC_BC_PERIODIC;
        const long long cu = (a + 1 < n) ? c + st : (per ? c - (long long)(n - 1) * st : c);
        const long long cd = (a > 0) ? c - st : (per ? c + (long long)(n - 1) * st : c);
        ap[d] = (!per && a == n - 1) ? (PT)0 : C.a[d][cu];
        am[d] = C.a[d][c];
        dpu[d] = nb(cu, d, +1);
        dpd[d] = nb(cd, d, -1);
    }
    return jacobi_value<PT>(P.nd, nb(c, 0, 0), dpu, dpd, ap, am, b[c], C.D[c], K, tau2, w);
}

// The same sweep as k_jacobi on a 3-D launch grid: x along the threads of a
// row of XT, y and z by block, so no index is decomposed; the neighbours are
// the ones cell_nb gives (periodic wrap, walls clamped onto the cell, whose
// wall coefficient is zero), in the same expression, so both kernels give the
// same bits.
constexpr int XT = 128;

template <typename PT, bool FIRST>
__global__ void __launch_bounds__(XT) k_jacobi_rows(GridParams P, PC<PT> C, PcK<PT> K, const PT *b, const PT *dp,
                                                    PT *dq, PT tau2)
{
    pdl_entry();
    PT tau_unused = 0;
    block_tau(P, tau_unused, tau2);
    const int i = blockIdx.x * XT + threadIdx.x, j = blockIdx.y, k = blockIdx.z;
    if (i >= P.n[0]) return;
    const int ix[3] = {i, j, k};
    const long long c = i + (long long)P.n[0] * (j + (long long)P.n[1] * k);
    const PT w = (PT)MUSIC_JACOBI_OMEGA;
    if (FIRST) {
        dq[c] = w * (b[c] / C.D[c]);
        return;
    }
    dq[c] = jacobi_cell(P, C, K, b, ix, c, tau2, w, [&](long long q, int, int) { return dp[q]; });
}

// The same sweep with each thread on one 16-byte chunk of W cells adjacent in
// x (4 floats or 2 doubles; rows of a multiple of W cells): dp, the
// coefficients, b and D of the chunk and dp and the coefficients of its y and
// z neighbours in 16-byte loads, the two x neighbours beyond the chunk's ends
// in single loads, all issued before any update.  Every cell's update is
// jacobi_value on the neighbours cell_nb gives, so the bits are those of
// k_jacobi_rows; a sweep over TGV 128^3 is one chunk a thread instead of one
// cell, a quarter of the loads and blocks.
template <typename PT>
__device__ __forceinline__ void ldw(const PT *p, long long c, PT *v)
{
    if constexpr (sizeof(PT) == 4) {
        const float4 a = *reinterpret_cast<const float4 *>(p + c);
        v[0] = a.x;
        v[1] = a.y;
        v[2] = a.z;
        v[3] = a.w;
    } else {
        const double2 a = *reinterpret_cast<const double2 *>(p + c);
        v[0] = a.x;
        v[1] = a.y;
    }
}

template <typename PT>
__device__ __forceinline__ void stw(PT *p, long long c, const PT *v)
{
    if constexpr (sizeof(PT) == 4)
        *reinterpret_cast<float4 *>(p + c) = make_float4(v[0], v[1], v[2], v[3]);
    else
        *reinterpret_cast<double2 *>(p + c) = make_double2(v[0], v[1]);
}

template <typename PT, bool FIRST>
__global__ void __launch_bounds__(BS) k_jacobi_vec(GridParams P, PC<PT> C, PcK<PT> K, const PT *b, const PT *dp,
                                                   PT *dq, PT tau2)
{
    pdl_entry();
    constexpr int W = 16 / sizeof(PT);
    PT tau_unused = 0;
    block_tau(P, tau_unused, tau2);
    const PT w = (PT)MUSIC_JACOBI_OMEGA;
    const long long e = blockIdx.x * (long long)BS + threadIdx.x;
    if (e >= P.N / W) return;
    const long long c0 = e * W;
    PT bv[W], Dv[W], out[W];
    ldw(b, c0, bv);
    ldw(C.D, c0, Dv);
    if (FIRST) {
#pragma unroll
        for (int q = 0; q < W; q++) out[q] = w * (bv[q] / Dv[q]);
        stw(dq, c0, out);
        return;
    }
    int ix[3];
    cell_coords(P, c0, ix);
    // y and z: the chunk's cells share their neighbours' offsets
    PT dpc[W], dpu[3][W], dpd[3][W], apv[3][W], amv[3][W];
    ldw(dp, c0, dpc);
    bool upw[3] = {false, false, false};
#pragma unroll
    for (int d = 1; d < 3; d++) {
        if (d >= P.nd) break;
        const int n = P.n[d], a = ix[d];
        const long long st = P.cs[d];
        const bool per = P.bc[d] == MUSIC_BC_PERIODIC;
        const long long cu = (a + 1 < n) ? c0 + st : (per ? c0 - (long long)(n - 1) * st : c0);
        const long long cd = (a > 0) ? c0 - st : (per ? c0 + (long long)(n - 1) * st : c0);
        upw[d] = !per && a == n - 1;
        ldw(C.a[d], cu, apv[d]);
        ldw(C.a[d], c0, amv[d]);
        ldw(dp, cu, dpu[d]);
        ldw(dp, cd, dpd[d]);
    }
    // x: neighbours inside the chunk, and the two beyond its ends
    const int n0 = P.n[0], i0 = ix[0];
    const bool perx = P.bc[0] == MUSIC_BC_PERIODIC;
    const long long cu_end = (i0 + W < n0) ? c0 + W : (perx ? c0 + W - n0 : c0 + W - 1);
    const long long cd_end = (i0 > 0) ? c0 - 1 : (perx ? c0 + n0 - 1 : c0);
    const PT dp_after = dp[cu_end], dp_before = dp[cd_end], a_after = C.a[0][cu_end];
    PT a0[W];
    ldw(C.a[0], c0, a0);
#pragma unroll
    for (int q = 0; q < W; q++) {
        PT u[3], dn[3], ap[3], am[3];
        u[0] = (q + 1 < W) ? dpc[q + 1] : dp_after;
        dn[0] = (q > 0) ? dpc[q - 1] : dp_before;
        ap[0] = (!perx && i0 + q == n0 - 1) ? (PT)0 : ((q + 1 < W) ? a0[q + 1] : a_after);
        am[0] = a0[q];
#pragma unroll
        for (int d = 1; d < 3; d++) {
            u[d] = dn[d] = ap[d] = am[d] = (PT)0;
            if (d >= P.nd) break;
            u[d] = dpu[d][q];
            dn[d] = dpd[d][q];
            ap[d] = upw[d] ? (PT)0 : apv[d][q];
            am[d] = amv[d][q];
        }
        out[q] = jacobi_value<PT>(P.nd, dpc[q], u, dn, ap, am, bv[q], Dv[q], K, tau2, w);
    }
    stw(dq, c0, out);
}

// The momentum correction on the lower d-face of a cell: its residual, less
// tau (dp - dp of the lower neighbour) / dx; the residual alone on a wall face
template <typename PT>
__device__ __forceinline__ PT dm_value(bool lwall, PT rm, PT dpc, PT dpl, PT tau, PT idx)
{
    return lwall ? rm : pfma(-pmul_rn(tau, dpc - dpl), idx, rm);
}

template <typename PT, typename RT>
__device__ inline PT dm_face(const GridParams &P, const RT *r, const PT *dp, const int ix[3], long long c,
                             int d, PT tau, PT idx)
{
    // momentum correction on the lower d-face of cell ix (c)
    return dm_value<PT>(lower_wall(P, ix, d), (PT)r[(2 + d) * P.N + c], dp[c], dp[cell_nb(P, ix, d, -1)], tau, idx);
}

// Back substitution of one cell in flux form from its own lower-face
// momentum corrections (mm_own), those of its upper faces (mp, 0 on walls),
// whether each lower face is a wall, and the face coefficients (shared by the
// per-cell and the chunked kernels: the same bits)
template <typename PT>
__device__ __forceinline__ void back_value(int nd, PT rr, PT rE, PT hp, const PT *mm_own, const PT *mp,
                                           const bool *lwall, const PT *ap, const PT *am, const PcK<PT> &K, PT tau,
                                           PT &zr, PT &ze)
{
    PT divm = 0, divu = 0;
#pragma unroll
    for (int d = 0; d < 3; d++) {
        if (d >= nd) break;
        const PT mm = lwall[d] ? (PT)0 : mm_own[d];
        divm = pfma(mp[d] - mm, K.idx[d], divm);
        divu = pfma(pfma(ap[d], mp[d], -pmul_rn(am[d], mm)), K.idx[d], divu);
    }
    zr = pfma(-tau, divm, rr);
    ze = pfma(-pmul_rn(tau, hp), divu, rE);
}

template <typename PT, typename RT>
__global__ void __launch_bounds__(BS) k_back(GridParams P, PC<PT> C, PcK<PT> K, const RT *r, const PT *dp, RT *z,
                                             PT tau)
{
    pdl_entry();
    PT tau2_unused = 0;
    block_tau(P, tau, tau2_unused);
    for (long long c = blockIdx.x * (long long)BS + threadIdx.x; c < P.N; c += (long long)gridDim.x * BS) {
        int ix[3];
        cell_coords(P, c, ix);
        PT mm_own[3], mp[3], ap[3], am[3];
        bool lwall[3];
#pragma unroll
        for (int d = 0; d < 3; d++) {
            mm_own[d] = mp[d] = ap[d] = am[d] = (PT)0;
            lwall[d] = false;
            if (d >= P.nd) break;
            mm_own[d] = dm_face(P, r, dp, ix, c, d, tau, K.idx[d]);
            z[(2 + d) * P.N + c] = (RT)mm_own[d];
            if (!upper_wall(P, ix, d)) {
                int jx[3] = {ix[0], ix[1], ix[2]};
                jx[d] = (ix[d] + 1 == P.n[d]) ? 0 : ix[d] + 1;
                mp[d] = dm_face(P, r, dp, jx, cell_index(P, jx), d, tau, K.idx[d]);
            }
            lwall[d] = lower_wall(P, ix, d);
            ap[d] = a_up(P, C, ix, d);
            am[d] = C.a[d][c];
        }
        PT zr, ze;
        back_value<PT>(P.nd, (PT)r[c], (PT)r[P.N + c], C.hp[c], mm_own, mp, lwall, ap, am, K, tau, zr, ze);
        z[c] = (RT)zr;
        z[P.N + c] = (RT)ze;
    }
}

// The right-hand side and the back substitution on 16-byte chunks of W cells
// adjacent in x (rows of a multiple of W cells), as k_jacobi_vec: the
// chunk's own values and those of its y and z neighbours in 16-byte loads,
// the x neighbours beyond its two ends in single loads; every cell's value is
// rhs_value / dm_value / back_value on what the per-cell kernels read, so the
// bits are theirs.
template <typename PT>
__global__ void __launch_bounds__(BS) k_rhs_vec(GridParams P, PC<PT> C, PcK<PT> K, const PT *r, PT *b, PT tau)
{
    pdl_entry();
    constexpr int W = 16 / sizeof(PT);
    PT tau2_unused = 0;
    block_tau(P, tau, tau2_unused);
    const long long e = blockIdx.x * (long long)BS + threadIdx.x;
    if (e >= P.N / W) return;
    const long long c0 = e * W, N = P.N;
    int ix[3];
    cell_coords(P, c0, ix);
    PT rE[W], gp[W], am[3][W], ap[3][W], rm[3][W], rp[3][W];
    ldw(r + N, c0, rE);
    ldw(C.gp, c0, gp);
#pragma unroll
    for (int d = 1; d < 3; d++) {
        if (d >= P.nd) break;
        const int n = P.n[d], a = ix[d];
        const long long st = P.cs[d];
        const bool per = P.bc[d] == MUSIC_BC_PERIODIC;
        const long long cu = (a + 1 < n) ? c0 + st : (per ? c0 - (long long)(n - 1) * st : c0);
        ldw(C.a[d], c0, am[d]);
        ldw(C.a[d], cu, ap[d]);
        if (!per && a == n - 1)
#pragma unroll
            for (int q = 0; q < W; q++) ap[d][q] = (PT)0;
        ldw(r + (2 + d) * N, c0, rm[d]);
        ldw(r + (2 + d) * N, cu, rp[d]);
    }
    const int n0 = P.n[0], i0 = ix[0];
    const bool perx = P.bc[0] == MUSIC_BC_PERIODIC;
    const long long cu_end = (i0 + W < n0) ? c0 + W : (perx ? c0 + W - n0 : c0 + W - 1);
    ldw(C.a[0], c0, am[0]);
    ldw(r + 2 * N, c0, rm[0]);
    const PT a_after = C.a[0][cu_end], r_after = r[2 * N + cu_end];
    PT out[W];
#pragma unroll
    for (int q = 0; q < W; q++) {
        PT apq[3], rpq[3], amq[3], rmq[3];
        apq[0] = (!perx && i0 + q == n0 - 1) ? (PT)0 : ((q + 1 < W) ? am[0][q + 1] : a_after);
        rpq[0] = (q + 1 < W) ? rm[0][q + 1] : r_after;
        amq[0] = am[0][q];
        rmq[0] = rm[0][q];
#pragma unroll
        for (int d = 1; d < 3; d++) {
            apq[d] = rpq[d] = amq[d] = rmq[d] = (PT)0;
            if (d >= P.nd) break;
            apq[d] = ap[d][q];
            rpq[d] = rp[d][q];
            amq[d] = am[d][q];
            rmq[d] = rm[d][q];
        }
        out[q] = rhs_value<PT>(P.nd, rE[q], gp[q], apq, rpq, amq, rmq, K, tau);
    }
    stw(b, c0, out);
}

template <typename PT>
__global__ void __launch_bounds__(BS) k_back_vec(GridParams P, PC<PT> C, PcK<PT> K, const PT *r, const PT *dp,
                                                 PT *z, PT tau)
{
    pdl_entry();
    constexpr int W = 16 / sizeof(PT);
    PT tau2_unused = 0;
    block_tau(P, tau, tau2_unused);
    const long long e = blockIdx.x * (long long)BS + threadIdx.x;
    if (e >= P.N / W) return;
    const long long c0 = e * W, N = P.N;
    int ix[3];
    cell_coords(P, c0, ix);
    PT rr[W], rE[W], hp[W], dpc[W];
    ldw(r, c0, rr);
    ldw(r + N, c0, rE);
    ldw(C.hp, c0, hp);
    ldw(dp, c0, dpc);
    // per direction and cell: own lower-face correction, upper-face one,
    // lower wall, face coefficients
    PT mmo[3][W], mpv[3][W], apv[3][W], amv[3][W];
    bool lw[3][W];
#pragma unroll
    for (int d = 1; d < 3; d++) {
        if (d >= P.nd) break;
        const int n = P.n[d], a = ix[d];
        const long long st = P.cs[d];
        const bool per = P.bc[d] == MUSIC_BC_PERIODIC;
        const long long cu = (a + 1 < n) ? c0 + st : (per ? c0 - (long long)(n - 1) * st : c0);
        const long long cd = (a > 0) ? c0 - st : (per ? c0 + (long long)(n - 1) * st : c0);
        const bool upw = !per && a == n - 1, low = !per && a == 0;
        PT rmc[W], rmu[W], dpd[W], dpu[W];
        ldw(r + (2 + d) * N, c0, rmc);
        ldw(r + (2 + d) * N, cu, rmu);
        ldw(dp, cd, dpd);
        ldw(dp, cu, dpu);
        ldw(C.a[d], c0, amv[d]);
        ldw(C.a[d], cu, apv[d]);
        const PT idx = K.idx[d];
#pragma unroll
        for (int q = 0; q < W; q++) {
            lw[d][q] = low;
            mmo[d][q] = dm_value<PT>(low, rmc[q], dpc[q], dpd[q], tau, idx);
            mpv[d][q] = upw ? (PT)0 : dm_value<PT>(false, rmu[q], dpu[q], dpc[q], tau, idx);
            if (upw) apv[d][q] = (PT)0;
        }
        stw(z + (2 + d) * N, c0, mmo[d]);
    }
    const int n0 = P.n[0], i0 = ix[0];
    const bool perx = P.bc[0] == MUSIC_BC_PERIODIC;
    const long long cu_end = (i0 + W < n0) ? c0 + W : (perx ? c0 + W - n0 : c0 + W - 1);
    const long long cd_end = (i0 > 0) ? c0 - 1 : (perx ? c0 + n0 - 1 : c0);
    PT rm0[W];
    ldw(r + 2 * N, c0, rm0);
    ldw(C.a[0], c0, amv[0]);
    const PT dp_after = dp[cu_end], dp_before = dp[cd_end], r_after = r[2 * N + cu_end], a_after = C.a[0][cu_end];
    const PT idx0 = K.idx[0];
#pragma unroll
    for (int q = 0; q < W; q++) {
        const bool low = !perx && i0 + q == 0, upw = !perx && i0 + q == n0 - 1;
        const PT dpl = (q > 0) ? dpc[q - 1] : dp_before;
        const PT dpu = (q + 1 < W) ? dpc[q + 1] : dp_after;
        const PT rmu = (q + 1 < W) ? rm0[q + 1] : r_after;
        lw[0][q] = low;
        mmo[0][q] = dm_value<PT>(low, rm0[q], dpc[q], dpl, tau, idx0);
        mpv[0][q] = upw ? (PT)0 : dm_value<PT>(false, rmu, dpu, dpc[q], tau, idx0);
        apv[0][q] = upw ? (PT)0 : ((q + 1 < W) ? amv[0][q + 1] : a_after);
    }
    stw(z + 2 * N, c0, mmo[0]);
    PT zr[W], ze[W];
#pragma unroll
    for (int q = 0; q < W; q++) {
        PT mo[3], mq[3], aq[3], bq[3];
        bool lq[3];
#pragma unroll
        for (int d = 0; d < 3; d++) {
            mo[d] = mq[d] = aq[d] = bq[d] = (PT)0;
            lq[d] = false;
            if (d >= P.nd) break;
            mo[d] = mmo[d][q];
            mq[d] = mpv[d][q];
            aq[d] = apv[d][q];
            bq[d] = amv[d][q];
            lq[d] = lw[d][q];
        }
        back_value<PT>(P.nd, rr[q], rE[q], hp[q], mo, mq, lq, aq, bq, K, tau, zr[q], ze[q]);
    }
    stw(z, c0, zr);
    stw(z + N, c0, ze);
}

int nblocks(long long n)
{
    long long b = (n + BS - 1) / BS;
    if (b > 152 * 16) b = 152 * 16;
    return (int)(b < 1 ? 1 : b);
}

template <typename PT>
PC<PT> pc_of(music_grid *g)
{
    PC<PT> C;
    for (int d = 0; d < 3; d++) C.a[d] = (PT *)g->pa[d];
    C.gp = (PT *)g->pgp;
    C.hp = (PT *)g->php;
    C.D = (PT *)g->pD;
    return C;
}

template <typename PT>
int setup_t(music_grid *g, const double *U, double dt, cudaStream_t s)
{
    const GridParams &P = g->P;
    PC<PT> C = pc_of<PT>(g);
    const double tau = 0.5 * dt;
    k_setup<PT><<<nblocks(P.N), BS, 0, s>>>(P, U, C, pck_of<PT>(P), (PT)(P.gamma * P.gm1), (PT)P.gamma,
                                             (PT)(tau * tau));
    CHECK_LAUNCH();
    return MUSIC_OK;
}

template <typename PT>
int apply_t(music_grid *g, double dt, const PT *r, PT *z, cudaStream_t s)
{
    const GridParams &P = g->P;
    PC<PT> C = pc_of<PT>(g);
    const double tau = 0.5 * dt;
    const PT taup = (PT)tau, tau2 = (PT)(tau * tau);
    const int nb = nblocks(P.N);
    PT *b = (PT *)g->pb, *dp = (PT *)g->pdp, *dq = (PT *)g->pdq;
    const PcK<PT> pk = pck_of<PT>(P);
    // 16-byte chunks when rows hold a whole number of them; else one cell a
    // thread, the sweeps' rows launch unless an extent exceeds the grid's y /
    // z limit (65535)
    constexpr int W = 16 / sizeof(PT);
    const bool by_chunks = P.n[0] % W == 0 && g->pc_variant != PC_ROWS;
    const int nbc = (int)((P.N / W + BS - 1) / BS);
    if (by_chunks)
        k_rhs_vec<PT><<<nbc, BS, 0, s>>>(P, C, pk, r, b, taup);
    else
        k_rhs<PT, PT><<<nb, BS, 0, s>>>(P, C, pk, r, b, taup);
    CHECK_LAUNCH();
    const int K = g->desc.precond_sweeps;
    const bool by_rows = P.n[1] <= 65535 && (P.nd < 3 || P.n[2] <= 65535);
    const dim3 rows((P.n[0] + XT - 1) / XT, P.n[1], P.nd == 3 ? P.n[2] : 1);
    for (int k = 0; k < K; k++) {
        if (by_chunks && k == 0)
            k_jacobi_vec<PT, true><<<nbc, BS, 0, s>>>(P, C, pk, b, dp, dq, tau2);
        else if (by_chunks)
            k_jacobi_vec<PT, false><<<nbc, BS, 0, s>>>(P, C, pk, b, dp, dq, tau2);
        else if (by_rows && k == 0)
            k_jacobi_rows<PT, true><<<rows, XT, 0, s>>>(P, C, pk, b, dp, dq, tau2);
        else if (by_rows)
            k_jacobi_rows<PT, false><<<rows, XT, 0, s>>>(P, C, pk, b, dp, dq, tau2);
        else if (k == 0)
            k_jacobi<PT, true><<<nb, BS, 0, s>>>(P, C, pk, b, dp, dq, tau2);
        else
            k_jacobi<PT, false><<<nb, BS, 0, s>>>(P, C, pk, b, dp, dq, tau2);
        CHECK_LAUNCH();
        PT *t = dp;
        dp = dq;
        dq = t;
    }
    if (K == 0) CUDA_TRY(cudaMemsetAsync(dp, 0, P.N * sizeof(PT), s));
    if (by_chunks)
        k_back_vec<PT><<<nbc, BS, 0, s>>>(P, C, pk, r, dp, z, taup);
    else
        k_back<PT, PT><<<nb, BS, 0, s>>>(P, C, pk, r, dp, z, taup);
    CHECK_LAUNCH();
    return MUSIC_OK;
}


// ---------------------------------------------------------------- fused 2-D
// ---------------------------------------------------------------- general form
// Spherical grids and grids with radiative diffusion: every divergence is a
// weighted sum W = A/V over the cell's faces (1/dx on Cartesian grids),
// gradients divide by the distance h between cell centres, and the energy
// row gains -tau div(chi grad dT) with dT = dp / rho (coefficients frozen,
// the density change neglected).  Pressure problem:
//   dp/gp - tau^2 div(grad(dp)/rbar) - (tau (gamma-1)/gp) div(chi grad(dp/rho)) = b.
struct Geo {
    double Wm, Wp, h;  // weights of the lower / upper d-face, centre distance
};

__device__ inline Geo geo(const GridParams &P, const int ix[3], int d)
{
    Geo o;
    if (P.geom == MUSIC_GEOM_SPHERICAL) {
        const long long c = cell_index(P, ix);
        const double V = sgeo(P, SG_V, c);
        o.Wm = sgeo(P, d == 0 ? SG_ARM : SG_ATM, c) / V;
        o.Wp = sgeo(P, d == 0 ? SG_ARP : SG_ATP, c) / V;
        o.h = sph_h(P, d, ix[0]);
    } else {
        o.Wm = o.Wp = P.idx[d];
        o.h = P.dx[d];
    }
    return o;
}

template <typename PT>
struct PCG {
    PT *a[3], *kf[3];  // 1/rbar and mean chi on the lower d-face (0 on walls)
    PT *gp, *hp, *rh, *D;
    PT *chi;           // cell chi (scratch during setup)
    PT *wu[3], *wl[3]; // a sweep's weights of the upper / lower d-neighbour (metric, pressure and conduction)
};

template <typename PT>
__global__ void __launch_bounds__(BS) k_gen_cell(GridParams P, const double *U, PCG<PT> C)
{
    pdl_entry();
    for (long long c = blockIdx.x * (long long)BS + threadIdx.x; c < P.N; c += (long long)gridDim.x * BS) {
        int ix[3];
        cell_coords(P, c, ix);
        const double rho = U[c], E = U[P.N + c];
        C.gp[c] = (PT)(P.gamma * (P.gm1 * E));
        C.hp[c] = (PT)(P.gamma * E);
        C.rh[c] = (PT)rho;
        double chi = 0.0;
        if (P.conduct) {
            const double t = P.gm1 * E / rho;
            const double t3 = t * t * t;
            chi = P.chi0 * (t3 * t3 * sqrt(t)) / (rho * rho);
        }
        C.chi[c] = (PT)chi;
        for (int d = 0; d < P.nd; d++) {
            if (lower_wall(P, ix, d)) {
                C.a[d][c] = (PT)0;
            } else {
                const long long l = cell_nb(P, ix, d, -1);
                C.a[d][c] = (PT)(1.0 / (0.5 * (U[l] + U[c])));
            }
        }
    }
}

template <typename PT>
__global__ void __launch_bounds__(BS) k_gen_face(GridParams P, PCG<PT> C, double tau)
{
    pdl_entry();
    tau = call_hdt(P, tau);
    for (long long c = blockIdx.x * (long long)BS + threadIdx.x; c < P.N; c += (long long)gridDim.x * BS) {
        int ix[3];
        cell_coords(P, c, ix);
        for (int d = 0; d < P.nd; d++)
            C.kf[d][c] = lower_wall(P, ix, d) ? (PT)0 : (PT)(0.5 * ((double)C.chi[cell_nb(P, ix, d, -1)] + (double)C.chi[c]));
    }
}

template <typename PT>
__device__ inline void up_coeffs(const GridParams &P, const PCG<PT> &C, const int ix[3], int d, long long &u,
                                 double &ap, double &kp)
{
    u = cell_nb(P, ix, d, +1);
    const bool uw = upper_wall(P, ix, d);
    ap = uw ? 0.0 : (double)C.a[d][u];
    kp = uw ? 0.0 : (double)C.kf[d][u];
}

template <typename PT>
__global__ void __launch_bounds__(BS) k_gen_diag(GridParams P, PCG<PT> C, double tau)
{
    pdl_entry();
    tau = call_hdt(P, tau);
    const double tau2 = tau * tau;
    for (long long c = blockIdx.x * (long long)BS + threadIdx.x; c < P.N; c += (long long)gridDim.x * BS) {
        int ix[3];
        cell_coords(P, c, ix);
        double diag = 0.0, dth = 0.0;
        const double gp = C.gp[c];
        const double th = tau * P.gm1 / gp;
        for (int d = 0; d < P.nd; d++) {
            const Geo G = geo(P, ix, d);
            long long u;
            double ap, kp;
            up_coeffs(P, C, ix, d, u, ap, kp);
            const long long l = cell_nb(P, ix, d, -1);
            const double am = C.a[d][c], km = C.kf[d][c];
            diag += G.Wp * ap / G.h + G.Wm * am / G.h;
            dth += G.Wp * kp / G.h + G.Wm * km / G.h;
            // the sweep's off-diagonal weights, formed once per Newton iteration
            // (the metric costs FP64 trigonometry per cell)
            C.wu[d][c] = (PT)(tau2 * (G.Wp * ap / G.h) + th * (G.Wp * kp / G.h / (double)C.rh[u]));
            C.wl[d][c] = (PT)(tau2 * (G.Wm * am / G.h) + th * (G.Wm * km / G.h / (double)C.rh[l]));
        }
        C.D[c] = (PT)(1.0 / gp + tau2 * diag + th * dth / (double)C.rh[c]);
    }
}

template <typename PT>
__global__ void __launch_bounds__(BS) k_gen_rhs(GridParams P, PCG<PT> C, const PT *r, PT *b, double tau)
{
    pdl_entry();
    tau = call_hdt(P, tau);
    for (long long c = blockIdx.x * (long long)BS + threadIdx.x; c < P.N; c += (long long)gridDim.x * BS) {
        int ix[3];
        cell_coords(P, c, ix);
        double divm = 0.0;
        for (int d = 0; d < P.nd; d++) {
            const Geo G = geo(P, ix, d);
            long long u;
            double ap, kp;
            up_coeffs(P, C, ix, d, u, ap, kp);
            divm += G.Wp * ap * (double)r[(2 + d) * P.N + u] - G.Wm * (double)C.a[d][c] * (double)r[(2 + d) * P.N + c];
        }
        b[c] = (PT)(P.gm1 * (double)r[P.N + c] / (double)C.gp[c] - tau * divm);
    }
}

// One weighted-Jacobi update of the general form: the first sweep from zero,
// later ones with the set-up's neighbour weights (wu, wl along d = 0, 1, 2,
// their neighbours' dp in du, dl), in the preconditioner's type.  Shared by
// the one-kernel-per-sweep and the tile-resident variant, so both round alike.
template <typename PT>
__device__ __forceinline__ PT gen_first(PT b, PT D)
{
    return (PT)(MUSIC_JACOBI_OMEGA * ((double)b / (double)D));
}

template <typename PT>
__device__ __forceinline__ PT gen_update(int nd, const PT *wu, const PT *wl, const PT *du, const PT *dl, PT dp, PT b,
                                         PT D)
{
    const PT wp = (PT)MUSIC_JACOBI_OMEGA;
    PT off = 0;
    for (int d = 0; d < nd; d++) {
        off = pfma(wu[d], du[d], off);
        off = pfma(wl[d], dl[d], off);
    }
    return pfma((PT)1 - wp, dp, wp * ((b + off) / D));
}

template <typename PT, bool FIRST>
__global__ void __launch_bounds__(BS) k_gen_jacobi(GridParams P, PCG<PT> C, const PT *b, const PT *dp, PT *dq)
{
    pdl_entry();
    for (long long c = blockIdx.x * (long long)BS + threadIdx.x; c < P.N; c += (long long)gridDim.x * BS) {
        if (FIRST) {
            dq[c] = gen_first(b[c], C.D[c]);
            continue;
        }
        int ix[3];
        cell_coords(P, c, ix);
        PT wu[3], wl[3], du[3], dl[3];
        for (int d = 0; d < P.nd; d++) {
            wu[d] = C.wu[d][c];
            wl[d] = C.wl[d][c];
            du[d] = dp[cell_nb(P, ix, d, +1)];
            dl[d] = dp[cell_nb(P, ix, d, -1)];
        }
        dq[c] = gen_update(P.nd, wu, wl, du, dl, dp[c], b[c], C.D[c]);
    }
}

// All K sweeps of a 2-D application in one kernel (K <= GEN_KM): a CTA of
// GTX x GTY threads stages its tile and a halo of GEN_KM + 1 cells (walls
// clamp onto the edge cell, whose wall-face weight is zero; periodic
// directions wrap), sweeps in shared memory on the region that shrinks by a
// cell per sweep, and writes its tile's dp.
constexpr int GTX = 32, GTY = 16, GEN_KM = 16, GEN_H = GEN_KM + 1;
constexpr int GRX = GTX + 2 * GEN_H, GRY = GTY + 2 * GEN_H, GR = GRX * GRY;

template <typename PT>
__global__ void __launch_bounds__(GTX *GTY) k_gen_sweeps_tile(GridParams P, PCG<PT> C, const PT *b, PT *dpout,
                                                              int K)
{
    pdl_entry();
    extern __shared__ __align__(16) unsigned char smraw[];
    PT *wu0 = (PT *)smraw, *wl0 = wu0 + GR, *wu1 = wl0 + GR, *wl1 = wu1 + GR, *bb = wl1 + GR, *DD = bb + GR;
    PT *dA = DD + GR, *dB = dA + GR;
    constexpr int NT = GTX * GTY;
    const int tid = threadIdx.x;
    const int i0 = blockIdx.x * GTX - GEN_H, j0 = blockIdx.y * GTY - GEN_H;
    const int n0 = P.n[0], n1 = P.n[1];
    const bool px = P.bc[0] == MUSIC_BC_PERIODIC, py = P.bc[1] == MUSIC_BC_PERIODIC;
    for (int q = tid; q < GR; q += NT) {
        const int lx = q % GRX, ly = q / GRX;
        bool inx, iny;
        const int x = pc_wrap(i0 + lx, n0, px, inx), y = pc_wrap(j0 + ly, n1, py, iny);
        const long long c = x + (long long)n0 * y;
        wu0[q] = C.wu[0][c];
        wl0[q] = C.wl[0][c];
        wu1[q] = C.wu[1][c];
        wl1[q] = C.wl[1][c];
        bb[q] = b[c];
        DD[q] = C.D[c];
    }
    __syncthreads();
    PT *src = dA, *dst = dB;
    for (int k = 0; k < K; k++) {
        // sweep k is valid on [k, R - k) of the staged region
        const int lo = k, hx = GRX - k, hy = GRY - k;
        const int wdt = hx - lo, cnt = wdt * (hy - lo);
        for (int t = tid; t < cnt; t += NT) {
            const int lx = lo + t % wdt, ly = lo + t / wdt, q = ly * GRX + lx;
            if (k == 0) {
                dst[q] = gen_first(bb[q], DD[q]);
            } else {
                // the staged region's edge points have no outer neighbour; they
                // fall outside the next sweep's region and are never read
                const PT wu[2] = {wu0[q], wu1[q]}, wl[2] = {wl0[q], wl1[q]};
                const PT du[2] = {lx + 1 < GRX ? src[q + 1] : (PT)0, ly + 1 < GRY ? src[q + GRX] : (PT)0};
                const PT dl[2] = {lx > 0 ? src[q - 1] : (PT)0, ly > 0 ? src[q - GRX] : (PT)0};
                dst[q] = gen_update(2, wu, wl, du, dl, src[q], bb[q], DD[q]);
            }
        }
        __syncthreads();
        PT *tt = src;
        src = dst;
        dst = tt;
    }
    const int tx = tid % GTX, ty = tid / GTX;
    const int gx = blockIdx.x * GTX + tx, gy = blockIdx.y * GTY + ty;
    if (gx < n0 && gy < n1) dpout[gx + (long long)n0 * gy] = src[(ty + GEN_H) * GRX + tx + GEN_H];
}

template <typename PT>
__global__ void __launch_bounds__(BS) k_gen_back(GridParams P, PCG<PT> C, const PT *r, const PT *dp, PT *z,
                                                 double tau)
{
    pdl_entry();
    tau = call_hdt(P, tau);
    for (long long c = blockIdx.x * (long long)BS + threadIdx.x; c < P.N; c += (long long)gridDim.x * BS) {
        int ix[3];
        cell_coords(P, c, ix);
        double divm = 0.0, divu = 0.0, dth = 0.0;
        const double tc = (double)dp[c] / (double)C.rh[c];
        for (int d = 0; d < P.nd; d++) {
            const Geo G = geo(P, ix, d);
            long long u;
            double ap, kp;
            up_coeffs(P, C, ix, d, u, ap, kp);
            const long long l = cell_nb(P, ix, d, -1);
            const bool lw = lower_wall(P, ix, d), uw = upper_wall(P, ix, d);
            const double own = lw ? (double)r[(2 + d) * P.N + c]
                                  : (double)r[(2 + d) * P.N + c] - tau * ((double)dp[c] - (double)dp[l]) / G.h;
            z[(2 + d) * P.N + c] = (PT)own;
            // the upper face's correction is the next cell's own one (same h)
            int jx[3] = {ix[0], ix[1], ix[2]};
            jx[d] = (ix[d] + 1 == P.n[d]) ? 0 : ix[d] + 1;
            const double hu = (P.geom == MUSIC_GEOM_SPHERICAL) ? sph_h(P, d, jx[0]) : P.dx[d];
            const double mp = uw ? 0.0 : (double)r[(2 + d) * P.N + u] - tau * ((double)dp[u] - (double)dp[c]) / hu;
            const double mm = lw ? 0.0 : own;
            divm += G.Wp * mp - G.Wm * mm;
            divu += G.Wp * ap * mp - G.Wm * (double)C.a[d][c] * mm;
            dth += G.Wp * kp * ((double)dp[u] / (double)C.rh[u] - tc) / G.h -
                   G.Wm * (double)C.kf[d][c] * (tc - (double)dp[l] / (double)C.rh[l]) / G.h;
        }
        z[c] = (PT)((double)r[c] - tau * divm);
        z[P.N + c] = (PT)(((double)r[P.N + c] - tau * (double)C.hp[c] * divu) + tau * dth);
    }
}

template <typename PT>
PCG<PT> pcg_of(music_grid *g)
{
    PCG<PT> C;
    for (int d = 0; d < 3; d++) {
        C.a[d] = (PT *)g->pa[d];
        C.kf[d] = (PT *)g->pkf[d];
    }
    C.gp = (PT *)g->pgp;
    C.hp = (PT *)g->php;
    C.rh = (PT *)g->prh;
    C.D = (PT *)g->pD;
    C.chi = (PT *)g->pb;  // the rhs buffer is free during setup
    for (int d = 0; d < 3; d++) {
        C.wu[d] = d < g->P.nd ? (PT *)g->pgw + (size_t)(2 * d) * g->P.N : nullptr;
        C.wl[d] = d < g->P.nd ? (PT *)g->pgw + (size_t)(2 * d + 1) * g->P.N : nullptr;
    }
    return C;
}

template <typename PT>
int gen_setup(music_grid *g, const double *U, double dt, cudaStream_t s)
{
    const GridParams &P = g->P;
    PCG<PT> C = pcg_of<PT>(g);
    const int nb = nblocks(P.N);
    k_gen_cell<PT><<<nb, BS, 0, s>>>(P, U, C);
    CHECK_LAUNCH();
    k_gen_face<PT><<<nb, BS, 0, s>>>(P, C, 0.5 * dt);
    CHECK_LAUNCH();
    k_gen_diag<PT><<<nb, BS, 0, s>>>(P, C, 0.5 * dt);
    CHECK_LAUNCH();
    return MUSIC_OK;
}

template <typename PT>
int gen_apply(music_grid *g, double dt, const PT *r, PT *z, cudaStream_t s)
{
    const GridParams &P = g->P;
    PCG<PT> C = pcg_of<PT>(g);
    const double tau = 0.5 * dt;
    const int nb = nblocks(P.N);
    PT *b = (PT *)g->pb, *dp = (PT *)g->pdp, *dq = (PT *)g->pdq;
    k_gen_rhs<PT><<<nb, BS, 0, s>>>(P, C, r, b, tau);
    CHECK_LAUNCH();
    const int K = g->desc.precond_sweeps;
    if (P.nd == 2 && K >= 1 && K <= GEN_KM) {
        // the sweeps in one tile-resident launch
        constexpr size_t smem = (size_t)8 * GR * sizeof(PT);
        static std::atomic<uint64_t> attr{0};
        TRY(allow_dynamic_smem(k_gen_sweeps_tile<PT>, smem, attr));
        const dim3 grid((P.n[0] + GTX - 1) / GTX, (P.n[1] + GTY - 1) / GTY);
        k_gen_sweeps_tile<PT><<<grid, GTX * GTY, smem, s>>>(P, C, b, dp, K);
        CHECK_LAUNCH();
        k_gen_back<PT><<<nb, BS, 0, s>>>(P, C, r, dp, z, tau);
        CHECK_LAUNCH();
        return MUSIC_OK;
    }
    for (int k = 0; k < K; k++) {
        if (k == 0)
            k_gen_jacobi<PT, true><<<nb, BS, 0, s>>>(P, C, b, dp, dq);
        else
            k_gen_jacobi<PT, false><<<nb, BS, 0, s>>>(P, C, b, dp, dq);
        CHECK_LAUNCH();
        PT *t = dp;
        dp = dq;
        dq = t;
    }
    if (K == 0) CUDA_TRY(cudaMemsetAsync(dp, 0, P.N * sizeof(PT), s));
    k_gen_back<PT><<<nb, BS, 0, s>>>(P, C, r, dp, z, tau);
    CHECK_LAUNCH();
    return MUSIC_OK;
}

}  // namespace

int precond_setup(music_grid *g, const double *U, double dt, cudaStream_t s)
{
    ProfScope prof_(g, MUSIC_PROF_VECTOR, s);
    if (g->desc.precond == MUSIC_PC_NONE) return MUSIC_OK;
    if (general_grid(g->P)) return g->mixed ? gen_setup<float>(g, U, dt, s) : gen_setup<double>(g, U, dt, s);
    return g->mixed ? setup_t<float>(g, U, dt, s) : setup_t<double>(g, U, dt, s);
}

namespace {
int precond_apply_body(music_grid *g, double dt, const void *r, void *z, int want_norm, cudaStream_t s);
}

int precond_apply(music_grid *g, double dt, const void *r, void *z, int want_norm, cudaStream_t s)
{
    if (g->desc.precond == MUSIC_PC_NONE || g->in_scalar) return precond_apply_body(g, dt, r, z, want_norm, s);
    ProfScope prof_(g, MUSIC_PROF_PRECOND, s);
    return precond_apply_body(g, dt, r, z, want_norm, s);
}

namespace {
int precond_apply_body(music_grid *g, double dt, const void *r, void *z, int want_norm, cudaStream_t s)
{
    const size_t n = g->n;
    if (g->desc.precond == MUSIC_PC_NONE || g->in_scalar) {  // the scalars' solve is unpreconditioned
        const size_t es = g->mixed ? sizeof(float) : sizeof(double);
        if (r != z) CUDA_TRY(cudaMemcpyAsync(z, r, n * es, cudaMemcpyDeviceToDevice, s));
    } else if (general_grid(g->P)) {
        if (g->mixed)
            TRY(gen_apply<float>(g, dt, (const float *)r, (float *)z, s));
        else
            TRY(gen_apply<double>(g, dt, (const double *)r, (double *)z, s));
    } else if (g->P.nd == 2 && g->desc.precond_sweeps <= PC_STAGED_MAXK && g->pc_variant != PC_MULTIKERNEL) {
        return precond2d_dispatch(g, dt, r, z, want_norm, s);
    } else if (g->mixed) {
        TRY(apply_t<float>(g, dt, (const float *)r, (float *)z, s));
    } else {
        TRY(apply_t<double>(g, dt, (const double *)r, (double *)z, s));
    }
    if (want_norm) {
        TRY(dev_norm2(g, z, !g->mixed, n, &g->ds->vnorm2, s));
        TRY(dev_set_eps(g, 0.0, s));
    }
    return MUSIC_OK;
}
}  // namespace

bool precond_folds_scale(const music_grid *g)
{
    return g->desc.precond != MUSIC_PC_NONE && !g->in_scalar && !general_grid(g->P) && g->P.nd == 2 &&
           g->desc.precond_sweeps <= PC_STAGED_MAXK && g->pc_variant != PC_MULTIKERNEL;
}

int precond2d_dispatch(music_grid *g, double dt, const void *r, void *z, int want_norm, cudaStream_t s)
{
    switch (g->ptile) {
    case 0:
        return precond2d_apply_t<16, 8>(g, dt, r, z, want_norm, s);
    case 1:
        return precond2d_apply_t<16, 16>(g, dt, r, z, want_norm, s);
    case 2:
        return precond2d_apply_t<32, 8>(g, dt, r, z, want_norm, s);
    case 3:
        return precond2d_apply_t<32, 16>(g, dt, r, z, want_norm, s);
    case 4:
        return precond2d_apply_t<64, 16>(g, dt, r, z, want_norm, s);
    case 5:
        return precond2d_apply_t<32, 32>(g, dt, r, z, want_norm, s);
    }
    set_error("preconditioner: bad tile index %d", g->ptile);
    return MUSIC_E_INVAL;
}
