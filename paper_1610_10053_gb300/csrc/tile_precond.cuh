// Per-tile device code of the fused 2-D physics-based preconditioner (Sec. 2,
// after Park et al.): used by the one-launch-per-application kernel and by
// the persistent batched kernel.
#pragma once
#include "internal.h"

namespace tile {

constexpr int PTX = 32, PTY = 16;  // tile of the persistent batched kernel
constexpr int PC_FUSED_MAXK = 16;  // sweeps of a one-launch application
constexpr int PC_STAGE_MAXK = 8;   // sweeps of one stage of a split application
constexpr int PC_STAGED_MAXK = 32; // sweeps of a split application (4 stages)
constexpr int PC_BATCH_MAXK_F32 = 24;  // sweeps of the batched kernel's FP32 tiles (FP64: PC_FUSED_MAXK)
constexpr int NRX = 16, NRY = 8;  // blocks of cells of the tile-independent |z|^2 reduction

template <typename PT>
struct PC {
    PT *a[3];   // 1 / rbar on the lower d-face (0 on wall faces)
    PT *gp;     // gamma p
    PT *hp;     // gamma E
    PT *D;      // diagonal of the Helmholtz operator
};

// shared-memory planes of one stage of precond2d_tile: 5 when its sweeps
// run from registers (staged cells per thread <= MAXCPT), else 6
template <typename PT, int KM, int TX, int TY, int MAXCPT = (sizeof(PT) == 4 ? 8 : 0)>
constexpr int pc_planes()
{
    constexpr int R = (TX + 2 * (KM + 1)) * (TY + 2 * (KM + 1));
    return (R + TX * TY - 1) / (TX * TY) <= MAXCPT ? 5 : 6;
}

// a * b + c with one rounding, in the preconditioner's type
__device__ __forceinline__ float pfma(float a, float b, float c) { return fmaf(a, b, c); }
__device__ __forceinline__ double pfma(double a, double b, double c) { return fma(a, b, c); }
// a * b rounded on its own (never contracted into a later operation)
__device__ __forceinline__ float pmul_rn(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ double pmul_rn(double a, double b) { return __dmul_rn(a, b); }

// index into an interior row or column: periodic wrap, or clamp on walls
// (coefficients of faces outside a walled domain are zero, which decouples
// the clamped cells)
__device__ inline int pc_wrap(int a, int n, bool periodic, bool &inside)
{
    if (periodic) {
        while (a < 0) a += n;
        while (a >= n) a -= n;
        inside = true;
        return a;
    }
    inside = (a > 0 && a < n);
    return a < 0 ? 0 : (a >= n ? n - 1 : a);
}

// One TX x TY tile (bx, by) of the fused preconditioner, run by a CTA of
// TX*TY threads with pc_planes() (TX+2H)(TY+2H) PT of shared memory at `smraw`; returns
// the calling thread's cell's |z|^2 (thread t owns cell (t % TX, t / TX)).
// tau = dt/2 and tau2 = tau^2 are replaced by the device dt's when P has one.
//
// The K Jacobi sweeps may be split over several launches (stages) with a
// shallower halo each: a FIRST stage builds the right-hand side from r and
// starts from dp = 0; a later stage reads the right-hand side (bg) and dp
// (dpin) of the whole staged region from global memory.  A stage that is not
// the LAST writes its tile's dp to dpout; the LAST one back-substitutes into
// z.  Every sweep computes the same values whatever the split, so the result
// does not depend on it.  K <= KM sweeps per stage.  MAXCPT bounds the
// staged cells per thread kept in registers across the sweeps (0: sweep from
// shared memory only).  Measured on KH grids, registers pay for FP32 (512^2:
// 61 -> 55 us per application) and cost for FP64 (226 -> 244 us), hence the
// default.
//
// The input is rs * r (each entry rounded on its own, so the result equals
// that of r scaled in memory beforehand); a FIRST stage with vout also
// writes that scaled input of its tile to vout (the solver graph's next
// Arnoldi vector, formed here instead of by a separate pass).
template <typename PT, int KM, int TX = PTX, int TY = PTY, bool FIRST = true, bool LAST = true,
          int MAXCPT = (sizeof(PT) == 4 ? 8 : 0)>
__device__ double precond2d_tile(const GridParams &P, const PC<PT> &C, const PT *r, PT *z, PT tau, PT tau2, int K,
                                 int bx, int by, unsigned char *smraw, PT *bg = nullptr, const PT *dpin = nullptr,
                                 PT *dpout = nullptr, PT rs = (PT)1, PT *vout = nullptr)
{
    auto rin = [&](long long i) { return pmul_rn(r[i], rs); };
    constexpr int NT = TX * TY, H = KM + 1, RX = TX + 2 * H, RY = TY + 2 * H, R = RX * RY;
    // staged cells per thread; with at most MAXCPT the sweeps run from registers
    constexpr int CPT = (R + NT - 1) / NT;
    constexpr bool REG = CPT <= MAXCPT;
    // planes: face coefficients 1/rbar (x, y), the folded sweep coefficients
    // cw = w tau^2 / D and bw = w b / D, and the two dp buffers; when the
    // sweeps run from registers the coefficient planes are dead once loaded
    // and the second dp buffer takes the x-face plane (pc_planes)
    PT *ax = (PT *)smraw, *ay = ax + R, *cwp = ay + R, *bwp = cwp + R, *dA = bwp + R;
    PT *dB = REG ? ax : dA + R;
    const int i0 = bx * TX - H, j0 = by * TY - H;
    const int tid = threadIdx.x;
    const long long N = P.N;
    const int n0 = P.n[0], n1 = P.n[1];
    const bool px = P.bc[0] == MUSIC_BC_PERIODIC, py = P.bc[1] == MUSIC_BC_PERIODIC;
    const PT w = (PT)MUSIC_JACOBI_OMEGA, omw = (PT)1 - w;
    // grid constants and tau (from the device dt when the grid has one) in
    // the preconditioner's type, converted once per CTA
    __shared__ PT s_c[7];
    if (tid == 0) {
        call_tau(P, tau, tau2);
        s_c[0] = (PT)P.gm1;
        s_c[1] = (PT)P.idx[0];
        s_c[2] = (PT)P.idx[1];
        s_c[3] = (PT)P.idx2[0];
        s_c[4] = (PT)P.idx2[1];
        s_c[5] = tau;
        s_c[6] = tau2;
    }
    __syncthreads();
    const PT gm1 = s_c[0], ix0 = s_c[1], ix1 = s_c[2], i20 = s_c[3], i21 = s_c[4];
    tau = s_c[5];
    tau2 = s_c[6];
    const PT wt2 = w * tau2;
    // a tile whose staged region and its upper neighbours lie strictly inside
    // the grid needs no wrap and meets no wall face: direct indices
    const bool inner = i0 >= 1 && i0 + RX + 1 <= n0 && j0 >= 1 && j0 + RY + 1 <= n1;
    for (int q = tid; q < R; q += NT) {
        const int lx = q % RX, ly = q / RX;
        bool inx = true, iny = true;
        int x = i0 + lx, y = j0 + ly;
        if (!inner) {
            x = pc_wrap(i0 + lx, n0, px, inx);
            y = pc_wrap(j0 + ly, n1, py, iny);
        }
        const long long c = x + (long long)n0 * y;
        ax[q] = inx ? C.a[0][c] : (PT)0;
        ay[q] = iny ? C.a[1][c] : (PT)0;
        const PT iD = (PT)1 / C.D[c];
        cwp[q] = wt2 * iD;
        PT bq = (PT)0;
        if (!FIRST) {
            bq = bg[c];
            dA[q] = dpin[c];
        } else if (lx < RX - 1 && ly < RY - 1) {
            // right-hand side needs r_m on the upper faces: the next cells'
            bool inxp = true, inyp = true;
            int xp = x + 1, yp = y + 1;
            if (!inner) {
                xp = pc_wrap(i0 + lx + 1, n0, px, inxp);
                yp = pc_wrap(j0 + ly + 1, n1, py, inyp);
            }
            const long long cx = xp + (long long)n0 * y, cy = x + (long long)n0 * yp;
            const PT axp = inxp ? C.a[0][cx] : (PT)0, ayp = inyp ? C.a[1][cy] : (PT)0;
            const PT axm = inx ? C.a[0][c] : (PT)0, aym = iny ? C.a[1][c] : (PT)0;
            PT divm = (axp * rin(2 * N + cx) - axm * rin(2 * N + c)) * ix0;
            divm += (ayp * rin(3 * N + cy) - aym * rin(3 * N + c)) * ix1;
            bq = gm1 * rin(N + c) / C.gp[c] - tau * divm;
            // a first stage that is not the last hands its tile's right-hand side on
            if (!LAST && lx >= H && lx < H + TX && ly >= H && ly < H + TY && i0 + lx < n0 && j0 + ly < n1)
                bg[(i0 + lx) + (long long)n0 * (j0 + ly)] = bq;
        }
        bwp[q] = w * (bq * iD);
    }
    __syncthreads();
    const int tx = tid % TX, ty = tid / TX;
    const int gx = bx * TX + tx, gy = by * TY + ty;
    if (FIRST && vout && gx < n0 && gy < n1) {
        const long long c = gx + (long long)n0 * gy;
#pragma unroll
        for (int k = 0; k < 4; k++) vout[k * N + c] = rin(k * N + c);
    }
    PT *src = dA, *dst = dB;
    // one Jacobi update of cell q from dp in `src`: the same operations, in
    // the same order, in both variants below
    auto sweep = [&](PT cxp, PT cxm, PT cyp, PT cym, PT cw, PT bw, PT cur, const PT *sp, int q) {
        PT off = cxp * sp[q + 1];
        off = pfma(cxm, sp[q - 1], off);
        off = pfma(cyp, sp[q + RX], off);
        off = pfma(cym, sp[q - RX], off);
        return pfma(omw, cur, pfma(cw, off, bw));
    };
    // the first stage's sweep k is valid on [k, R - 1 - k) (its right-hand
    // side needs the upper neighbour); a later stage's on [k + 1, R - k - 1):
    // cell (lx, ly) is updated by the sweeps k <= kmax(lx, ly)
    auto kmax_of = [&](int lx, int ly) {
        const int e = FIRST ? 0 : 1;
        return min(min(lx - e, RX - 2 - lx), min(ly - e, RY - 2 - ly));
    };
    if constexpr (REG) {
        // each thread keeps its cells' coefficients and current dp in
        // registers across the sweeps, so a sweep reads only the four
        // neighbours from shared memory
        PT cxp[CPT], cxm[CPT], cyp[CPT], cym[CPT], cw[CPT], bw[CPT], cur[CPT];
        int km[CPT];
#pragma unroll
        for (int s = 0; s < CPT; s++) {
            const int q = tid + s * NT;
            const bool in = q < R;
            const int lx = q % RX, ly = q / RX;
            const bool nx = in && lx < RX - 1, ny = in && ly < RY - 1;
            cxp[s] = (nx ? ax[q + 1] : (PT)0) * i20;
            cxm[s] = (in ? ax[q] : (PT)0) * i20;
            cyp[s] = (ny ? ay[q + RX] : (PT)0) * i21;
            cym[s] = (in ? ay[q] : (PT)0) * i21;
            cw[s] = in ? cwp[q] : (PT)0;
            bw[s] = in ? bwp[q] : (PT)0;
            cur[s] = (!FIRST && in) ? src[q] : (PT)0;
            km[s] = in ? kmax_of(lx, ly) : -1;
        }
        __syncthreads();  // the first sweep writes over the x-face plane
        for (int k = 0; k < K; k++) {
#pragma unroll
            for (int s = 0; s < CPT; s++) {
                const int q = tid + s * NT;
                if (k <= km[s]) {
                    const PT v = (FIRST && k == 0) ? bw[s] : sweep(cxp[s], cxm[s], cyp[s], cym[s], cw[s], bw[s],
                                                                   cur[s], src, q);
                    cur[s] = v;
                    dst[q] = v;
                }
            }
            __syncthreads();
            PT *tt = src;
            src = dst;
            dst = tt;
        }
    } else {
        for (int k = 0; k < K; k++) {
            const int lo = FIRST ? k : k + 1, hx = RX - 1 - k, hy = RY - 1 - k;
            const int wdt = hx - lo, cnt = wdt * (hy - lo);
            for (int t = tid; t < cnt; t += NT) {
                const int q = (lo + t / wdt) * RX + lo + t % wdt;
                if (FIRST && k == 0)
                    dst[q] = bwp[q];
                else
                    dst[q] = sweep(ax[q + 1] * i20, ax[q] * i20, ay[q + RX] * i21, ay[q] * i21, cwp[q], bwp[q],
                                   src[q], src, q);
            }
            __syncthreads();
            PT *tt = src;
            src = dst;
            dst = tt;
        }
    }
    // src holds dp
    if (!LAST) {
        if (gx < n0 && gy < n1) dpout[gx + (long long)n0 * gy] = src[(ty + H) * RX + tx + H];
        __syncthreads();
        return 0.0;
    }
    // back substitution on the tile
    double nrm = 0.0;
    if (gx < n0 && gy < n1) {
        const int q = (ty + H) * RX + (tx + H);
        const long long c = gx + (long long)n0 * gy;
        const bool wlx = (!px && gx == 0), wux = (!px && gx == n0 - 1);
        const bool wly = (!py && gy == 0), wuy = (!py && gy == n1 - 1);
        const long long cxp = (gx + 1 == n0) ? c - gx : c + 1;
        const long long cyp = (gy + 1 == n1) ? gx : c + n0;
        const PT dp = (K > 0) ? src[q] : (PT)0;
        const PT dpxm = (K > 0) ? src[q - 1] : (PT)0, dpxp = (K > 0) ? src[q + 1] : (PT)0;
        const PT dpym = (K > 0) ? src[q - RX] : (PT)0, dpyp = (K > 0) ? src[q + RX] : (PT)0;
        const PT mx_own = wlx ? rin(2 * N + c) : rin(2 * N + c) - tau * (dp - dpxm) * ix0;
        const PT my_own = wly ? rin(3 * N + c) : rin(3 * N + c) - tau * (dp - dpym) * ix1;
        const PT mxp = wux ? (PT)0 : rin(2 * N + cxp) - tau * (dpxp - dp) * ix0;
        const PT myp = wuy ? (PT)0 : rin(3 * N + cyp) - tau * (dpyp - dp) * ix1;
        const PT mxm = wlx ? (PT)0 : mx_own, mym = wly ? (PT)0 : my_own;
        PT divm = (mxp - mxm) * ix0;
        divm += (myp - mym) * ix1;
        // face coefficients of the cell: from the staged planes, or (their
        // planes reused by the sweeps) the same values from global memory
        PT axm, axp, aym, ayp;
        if constexpr (REG) {
            axm = (px || gx > 0) ? C.a[0][c] : (PT)0;
            axp = (px || gx + 1 < n0) ? C.a[0][cxp] : (PT)0;
            aym = (py || gy > 0) ? C.a[1][c] : (PT)0;
            ayp = (py || gy + 1 < n1) ? C.a[1][cyp] : (PT)0;
        } else {
            axm = ax[q];
            axp = ax[q + 1];
            aym = ay[q];
            ayp = ay[q + RX];
        }
        PT divu = (axp * mxp - axm * mxm) * ix0;
        divu += (ayp * myp - aym * mym) * ix1;
        const PT zr = rin(c) - tau * divm;
        const PT ze = rin(N + c) - tau * C.hp[c] * divu;
        z[c] = zr;
        z[N + c] = ze;
        z[2 * N + c] = mx_own;
        z[3 * N + c] = my_own;
        if constexpr (sizeof(PT) == 4)  // the cell's square sum in FP32, one conversion
            nrm = (double)(zr * zr + ze * ze + mx_own * mx_own + my_own * my_own);
        else
            nrm = (double)zr * zr + (double)ze * ze + (double)mx_own * mx_own + (double)my_own * my_own;
    }
    __syncthreads();  // the tile's shared memory may be reused by the caller
    return nrm;
}

// |z|^2 partials on a fixed decomposition of the grid into NRX x NRY blocks
// of cells, each summed in a fixed order (lane l takes cells l, l+32, ... of
// the block, then a warp tree), so the total does not depend on the tile
// shape of the kernel that produced z.  `v` is the thread's cell value as
// returned by precond2d_tile; `buf` holds TX*TY doubles of shared memory.
template <int TX, int TY>
__device__ void norm_partials(const GridParams &P, double v, int bx, int by, double *partial, double *buf)
{
    static_assert(TX % NRX == 0 && TY % NRY == 0, "tile must be a multiple of the reduction block");
    constexpr int SX = TX / NRX, SY = TY / NRY, NS = SX * SY, NW = TX * TY / 32;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    buf[tid] = v;
    __syncthreads();
    const int nsx = (P.n[0] + NRX - 1) / NRX, nsy = (P.n[1] + NRY - 1) / NRY;
    for (int q = warp; q < NS; q += NW) {
        const int sx = q % SX, sy = q / SX;
        double a = 0.0;
        for (int c = lane; c < NRX * NRY; c += 32) a += buf[(sy * NRY + c / NRX) * TX + sx * NRX + c % NRX];
        for (int o = 16; o > 0; o >>= 1) a += __shfl_down_sync(0xffffffffu, a, o);
        const int gx = bx * SX + sx, gy = by * SY + sy;
        if (lane == 0 && gx < nsx && gy < nsy) partial[(long long)gy * nsx + gx] = a;
    }
}

// number of partials norm_partials writes for the grid
__host__ __device__ inline long long norm_partial_count(const GridParams &P)
{
    return (long long)((P.n[0] + NRX - 1) / NRX) * ((P.n[1] + NRY - 1) / NRY);
}

// In one CTA of at least 128 threads: *dst = sum of partial[0, count) in a
// fixed order (128 strided runs, then a fixed halving tree in `buf`).  Each
// run's loads are issued eight at a time, then added in the run's order: one
// L2 round trip per eight partials instead of one per partial.
__device__ inline void sum_partials_fixed(const double *partial, long long count, double *dst, double *buf)
{
    const int tid = threadIdx.x;
    if (tid < 128) {
        double a = 0.0;
        long long b = tid;
        for (; b + 7 * 128 < count; b += 8 * 128) {
            double v[8];
#pragma unroll
            for (int k = 0; k < 8; k++) v[k] = __ldcg(partial + b + 128 * k);
#pragma unroll
            for (int k = 0; k < 8; k++) a += v[k];
        }
        for (; b < count; b += 128) a += __ldcg(partial + b);
        buf[tid] = a;
    }
    __syncthreads();
    for (int w = 64; w > 0; w >>= 1) {
        if (tid < w) buf[tid] += buf[tid + w];
        __syncthreads();
    }
    if (tid == 0) *dst = buf[0];
}

}  // namespace tile
