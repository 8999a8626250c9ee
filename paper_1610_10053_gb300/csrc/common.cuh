// Shared definitions of the libmusic CUDA sources (sm_103a).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "music.h"

#define MUSIC_GHOST 3
#define MUSIC_MAXV 64          // max Krylov vectors per cycle + 1
#define MUSIC_JACOBI_OMEGA 0.8 // weight of the pressure-system Jacobi sweeps
#define MUSIC_BATCH_MAX 512    // grids per batched launch

// Grid geometry and physics, passed to kernels by value.
struct GridParams {
    int nd, nv;
    int n[3];
    long long N;          // interior cells
    int ne[3];            // extended (ghosted) extent per direction
    long long M;          // extended points
    long long es[3];      // extended strides
    long long cs[3];      // interior strides
    double dx[3], idx[3], idx2[3];
    double x0[3];
    int bc[3], ws[3];
    double gamma, gm1;
    double g[3];
    int geom;              // MUSIC_GEOM_*
    int conduct;
    double chi0, lum;
    int flux_wall[3];
    const double *gface;   // spherical: radial gravity on the n[0]+1 r-faces (device), or null
    const double *sgeo;    // spherical: the cells' metric (SG_COUNT planes of N, device), or null
    const double *dt_dev;  // launches recorded into a solver graph read dt here (device), else null
};

// dt/2 of a launch: the value passed, or the device copy for launches that
// were recorded into a solver graph (same arithmetic either way)
__device__ __forceinline__ double call_hdt(const GridParams &P, double hdt)
{
    return P.dt_dev ? 0.5 * *P.dt_dev : hdt;
}
template <typename PT>
__device__ __forceinline__ void call_tau(const GridParams &P, PT &tau, PT &tau2)
{
    if (P.dt_dev) {
        const double t = 0.5 * *P.dt_dev;
        tau = (PT)t;
        tau2 = (PT)(t * t);
    }
}

// ---- spherical (r, theta) metric, 2 pi dropped (2-D axisymmetric grids)
__host__ __device__ inline double sph_r(const GridParams &P, double i) { return P.x0[0] + i * P.dx[0]; }
__host__ __device__ inline double sph_th(const GridParams &P, double j) { return P.x0[1] + j * P.dx[1]; }
__device__ inline double sph_vol(const GridParams &P, int i, int j)
{
    const double ra = sph_r(P, i), rb = sph_r(P, i + 1);
    return (rb * rb * rb - ra * ra * ra) / 3.0 * (cos(sph_th(P, j)) - cos(sph_th(P, j + 1)));
}
// area of the lower d-face of cell (i, j)
__device__ inline double sph_area(const GridParams &P, int d, int i, int j)
{
    if (d == 0) {
        const double r = sph_r(P, i);
        return r * r * (cos(sph_th(P, j)) - cos(sph_th(P, j + 1)));
    }
    const double ra = sph_r(P, i), rb = sph_r(P, i + 1);
    return 0.5 * (rb * rb - ra * ra) * sin(sph_th(P, j));
}
// The metric of the (r, theta) cells, tabulated once per grid (the same
// expressions as above, evaluated at grid creation instead of in every
// stencil and preconditioner launch): volume, the four face areas, and the
// control volumes of the r- and theta-momenta with their face and edge areas.
enum SphGeo {
    SG_V = 0, SG_ARM, SG_ARP, SG_ATM, SG_ATP,
    SG_VR, SG_ACP, SG_ACM, SG_EM, SG_EP, SG_RF,
    SG_VT, SG_BP, SG_BM, SG_FA, SG_FB, SG_RC,
    SG_COUNT
};
__device__ inline double sgeo(const GridParams &P, int k, long long c) { return P.sgeo[(long long)k * P.N + c]; }

// distance between the centres of the two cells sharing a d-face of column i
__device__ inline double sph_h(const GridParams &P, int d, int i)
{
    return d == 0 ? P.dx[0] : sph_r(P, i + 0.5) * P.dx[1];
}
// gravity on d-face i (radial table for spherical r-faces)
__device__ inline double face_g(const GridParams &P, int d, int i)
{
    return (P.geom == MUSIC_GEOM_SPHERICAL && d == 0 && P.gface) ? P.gface[i] : P.g[d];
}

// Scalars produced and consumed on the device.
struct DevScalars {
    double unorm2;        // |U|^2 of the current Newton iterate
    double vnorm2;        // |v|^2 of the vector a Jv is about to take
    double eps;           // finite-difference step of the next Jv
    double wnorm2;        // |w|^2 after re-orthogonalisation
    double rnorm2;        // generic norm^2 slot
    double maxdrho;       // Newton test
    double rate;          // CFL rate
    double rate_adv;      // advective rate max |u_d| / h_d
    double rate_rad;      // radiative rate max D / h_d^2
    double h[MUSIC_MAXV];   // first CGS pass
    double h2[MUSIC_MAXV];  // second CGS pass
    double diag[8];
    unsigned int counters[8];  // last-block-done counters, 0 between launches
    // outputs of a batched step (music_batch_step)
    double step_dt, step_fnorm0, step_fnorm, step_maxdrho;
    int step_status, step_newton, step_gmres, step_halvings, step_unconverged, step_pad;
};

enum { CNT_DOTS = 0, CNT_UPDATE, CNT_NORMW, CNT_SUMSQ, CNT_NEWTON, CNT_PRECOND };

// Control state of one Newton attempt driven from the device (solver graph):
// loop counters, statistics and status first (the host reads these back),
// then the Hessenberg matrix with its Givens rotations.
struct SolveCtl {
    double dt;                         // step size of the attempt
    int dt_status;    // MUSIC_OK, or why the device-side choice of dt found none (k_ctl_dt)
    int dt_which;     // the limit that chose dt (0-2: CFL_hydro, advective, radiative; 3: dt_max)
    double bnorm, target, beta, resid; // |b|, eta |b|, cycle start residual, current residual
    double inv;                        // 1 / h_{j+1,j} of the pending basis scaling
    double fnorm0, fnorm, maxdrho;
    int j;            // Arnoldi index of the next iteration
    int k;            // basis vectors in the current cycle's correction
    int scale_idx;    // basis vector the pending scaling writes
    int scale;        // 1: V[scale_idx] = w * inv pending
    int cycle, converged, its;
    int newton_it, newton_its, gmres_its, unconverged;
    int cycles, restarts, solves;  // bodies run: cycles, restart residuals, corrections
    int status;       // MUSIC_OK, MUSIC_E_NONFINITE, or MUSIC_E_TIMEOUT (loop cap reached)
    int stop;         // 1: leave every loop (hard error)
    int ok;           // 1: Newton converged
    int guard;        // loop bodies run, against a hard cap
    int go;           // 1: the current cycle builds an Arnoldi basis (its kernels run)
    int nocycle;      // 1: the GMRES solve needs no cycle at all (|b| zero or not finite)
    double cs[MUSIC_MAXV], sn[MUSIC_MAXV], gv[MUSIC_MAXV + 1], y[MUSIC_MAXV];
    double H[MUSIC_MAXV * MUSIC_MAXV]; // H[i * MUSIC_MAXV + j]
};

__host__ __device__ inline long long ext_index(const GridParams &P, int i, int j, int k)
{
    return (long long)(i + MUSIC_GHOST) + P.es[1] * (j + MUSIC_GHOST) +
           P.es[2] * (k + (P.nd == 3 ? MUSIC_GHOST : 0));
}

// (64-bit integer division is emulated in software on the GPU: grids whose
// index fits 32 bits, all in practice, decompose it in 32-bit arithmetic)
__device__ inline void ext_coords(const GridParams &P, long long x, int ix[3])
{
    if (P.M <= 0x7fffffffLL) {
        const unsigned u = (unsigned)x, n0 = (unsigned)P.ne[0], n1 = (unsigned)P.ne[1];
        const unsigned q = u / n0;
        ix[0] = (int)(u - q * n0) - MUSIC_GHOST;
        ix[1] = (int)(q % n1) - MUSIC_GHOST;
        ix[2] = (int)(q / n1) - (P.nd == 3 ? MUSIC_GHOST : 0);
        return;
    }
    ix[0] = (int)(x % P.ne[0]) - MUSIC_GHOST;
    ix[1] = (int)((x / P.ne[0]) % P.ne[1]) - MUSIC_GHOST;
    ix[2] = (int)(x / P.es[2]) - (P.nd == 3 ? MUSIC_GHOST : 0);
}

__device__ inline bool ext_has(const GridParams &P, const int ix[3], int d, int off)
{
    int lo = (d < P.nd) ? -MUSIC_GHOST : 0;
    int a = ix[d] + off - lo;
    return a >= 0 && a < P.ne[d];
}

__device__ inline void cell_coords(const GridParams &P, long long c, int ix[3])
{
    if (P.N <= 0x7fffffffLL) {
        const unsigned u = (unsigned)c, n0 = (unsigned)P.n[0], n1 = (unsigned)P.n[1];
        const unsigned q = u / n0;
        ix[0] = (int)(u - q * n0);
        ix[1] = (int)(q % n1);
        ix[2] = (int)(q / n1);
        return;
    }
    ix[0] = (int)(c % P.n[0]);
    ix[1] = (int)((c / P.n[0]) % P.n[1]);
    ix[2] = (int)(c / P.cs[2]);
}

__device__ inline long long cell_index(const GridParams &P, const int ix[3])
{
    return ix[0] + P.cs[1] * ix[1] + P.cs[2] * ix[2];
}

// neighbour of an interior cell along d (periodic wrap; walls clamp, the
// coefficient of the wall face being zero wherever it is used)
__device__ inline long long cell_nb(const GridParams &P, const int ix[3], int d, int off)
{
    int j[3] = {ix[0], ix[1], ix[2]};
    int a = j[d] + off;
    if (P.bc[d] == MUSIC_BC_PERIODIC) {
        while (a < 0) a += P.n[d];  // |off| is a cell or two: at most a shift or two
        while (a >= P.n[d]) a -= P.n[d];
    } else if (a < 0)
        a = 0;
    else if (a >= P.n[d])
        a = P.n[d] - 1;
    j[d] = a;
    return cell_index(P, j);
}

__device__ inline bool lower_wall(const GridParams &P, const int ix[3], int d)
{
    return P.bc[d] == MUSIC_BC_WALL && ix[d] == 0;
}

__device__ inline bool upper_wall(const GridParams &P, const int ix[3], int d)
{
    return P.bc[d] == MUSIC_BC_WALL && ix[d] == P.n[d] - 1;
}

// ---------------------------------------------------------------- reductions
// Deterministic block sum: warp shuffles, then one warp over the warp sums.
template <int BS>
__device__ inline double block_sum(double v, double *sh)
{
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) sh[wid] = v;
    __syncthreads();
    double r = 0.0;
    if (wid == 0) {
        r = (lane < BS / 32) ? sh[lane] : 0.0;
        for (int o = 16; o > 0; o >>= 1) r += __shfl_down_sync(0xffffffffu, r, o);
    }
    return r;  // valid in thread 0
}

// NaN-propagating max of non-negative values.
__device__ inline double nanmax(double a, double b)
{
    if (a != a) return a;
    if (b != b) return b;
    return a > b ? a : b;
}

template <int BS>
__device__ inline double block_max(double v, double *sh)
{
    for (int o = 16; o > 0; o >>= 1) v = nanmax(v, __shfl_down_sync(0xffffffffu, v, o));
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) sh[wid] = v;
    __syncthreads();
    double r = 0.0;
    if (wid == 0) {
        r = (lane < BS / 32) ? sh[lane] : 0.0;
        for (int o = 16; o > 0; o >>= 1) r = nanmax(r, __shfl_down_sync(0xffffffffu, r, o));
    }
    return r;
}

template <typename T>
__device__ inline double to_d(T v) { return (double)v; }

// True in the one block of the grid that finishes last.  Every block calls it
// after writing its partials; the fence makes them visible to the last block,
// which then reads them through L2 (__ldcg).  The counter is reset for the
// next launch.  No block ever waits on another.
// Programmatic dependent launch (the recorded solver graph links
// consecutive kernels programmatically): a kernel may launch as the blocks
// of the one it depends on exit, and every kernel begins by waiting for the
// grids it depends on to complete, with their memory visible.  A no-op for
// a kernel launched without a programmatic dependency.  (Letting dependents
// launch from the start of each kernel instead, which parks their blocks on
// the SMs while they wait, measured slower: KH 512^2 3.70 -> 3.85 ms per
// step, the spherical wedge 35.5 -> 44.9.)
__device__ __forceinline__ void pdl_entry()
{
    asm volatile("griddepcontrol.wait;" ::: "memory");
}

__device__ inline bool last_block_done(unsigned int *counter)
{
    __shared__ bool last;
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) {
        const unsigned int nb = gridDim.x * gridDim.y * gridDim.z;
        last = (atomicAdd(counter, 1u) == nb - 1);
    }
    __syncthreads();
    if (last && threadIdx.x == 0) *counter = 0;
    return last;
}

// In the last block: dst[i] = sum_b partial[i * stride + b], b < nb, i < count,
// each in a fixed order (thread t takes b = t, t + BS, ..., then the tree).
template <int BS>
__device__ inline void finish_sums(const double *partial, int nb, long long stride, int count, double *dst,
                                   double *sh)
{
    for (int i = 0; i < count; i++) {
        double s = 0.0;
        for (int b = threadIdx.x; b < nb; b += BS) s += __ldcg(partial + i * stride + b);
        const double r = block_sum<BS>(s, sh);
        if (threadIdx.x == 0) dst[i] = r;
    }
}

// In the last block, several sums at once: warp w takes items w, w + BS/32,
// ..., its lanes the partials b = lane, lane + 32, ..., then a warp tree; the
// order depends on nothing but nb, so the sums are deterministic.
// (each lane issues its loads eight at a time, then adds them in the order
// of b: one L2 round trip per eight partials instead of one per partial)
template <int BS>
__device__ inline void finish_sums_warps(const double *partial, int nb, long long stride, int count, double *dst)
{
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    for (int i = wid; i < count; i += BS / 32) {
        const double *p = partial + i * stride;
        double s = 0.0;
        int b = lane;
        for (; b + 7 * 32 < nb; b += 8 * 32) {
            double v[8];
#pragma unroll
            for (int k = 0; k < 8; k++) v[k] = __ldcg(p + b + 32 * k);
#pragma unroll
            for (int k = 0; k < 8; k++) s += v[k];
        }
        for (; b < nb; b += 32) s += __ldcg(p + b);
        for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
        if (lane == 0) dst[i] = s;
    }
}

template <int BS>
__device__ inline void finish_max(const double *partial, int nb, double *dst, double *sh)
{
    double s = 0.0;
    for (int b = threadIdx.x; b < nb; b += BS) s = nanmax(s, __ldcg(partial + b));
    const double r = block_max<BS>(s, sh);
    if (threadIdx.x == 0) *dst = r;
}

// eps = sqrt(2^-52) (1 + |U|) / |v| for the next Jacobian-free product
__device__ inline double fd_eps(double unorm2, double vnorm2)
{
    const double vn = sqrt(vnorm2);
    return (vn == 0.0) ? 0.0 : (sqrt(2.220446049250313e-16) * (1.0 + sqrt(unorm2))) / vn;
}
