// Time-step rate (Sec. 2.1, Eq. 4) and the scalar diagnostics of Secs. 3-6.
//
// Deterministic: one block per row (direction 1) produces the row's sums and
// maxima in a fixed order; a single block then combines the rows in order.
#include <cmath>
#include <mutex>

#include "internal.h"

namespace {

constexpr int BS = 256;
constexpr int NR = 8;  // per-row quantities

__device__ inline double face_u(const GridParams &P, const double *U, const int ix[3], long long c, int d)
{
    if (lower_wall(P, ix, d)) return 0.0;
    const long long l = cell_nb(P, ix, d, -1);
    return U[(2 + d) * P.N + c] / (0.5 * (U[l] + U[c]));
}

// Per row j: [0] sum X_H, [1] sum KE density, [2] sum vertical KE, [3] sum v cos kx,
// [4] sum v sin kx, [5] max Mach, [6] max speed, [7] max CFL rate.
__global__ void __launch_bounds__(BS) k_rows(GridParams P, const double *U, double rho_L, double rho_H,
                                             double kmode, double *rows)
{
    pdl_entry();
    __shared__ double sh[BS / 32];
    const int j = blockIdx.x;
    const double dV = P.dx[0] * P.dx[1] * (P.nd == 3 ? P.dx[2] : 1.0);
    double s[NR] = {0, 0, 0, 0, 0, 0, 0, 0};
    const long long per_row = (long long)P.n[0] * P.n[2];
    for (long long t = threadIdx.x; t < per_row; t += BS) {
        int ix[3] = {(int)(t % P.n[0]), j, (int)(t / P.n[0])};
        const long long c = cell_index(P, ix);
        const double rho = U[c];
        const double cs = sqrt(P.gamma * (P.gm1 * U[P.N + c]) / rho);
        s[0] += (rho - rho_L) / (rho_H - rho_L);
        double u2 = 0.0;
        for (int d = 0; d < P.nd; d++) {
            const double um = face_u(P, U, ix, c, d);
            double up = 0.0;
            if (!upper_wall(P, ix, d)) {
                int jx[3] = {ix[0], ix[1], ix[2]};
                jx[d] = (ix[d] + 1 == P.n[d]) ? 0 : ix[d] + 1;
                up = face_u(P, U, jx, cell_index(P, jx), d);
            }
            const double uc = 0.5 * (um + up);
            u2 += uc * uc;
            const double rbar = lower_wall(P, ix, d) ? 0.0 : 0.5 * (U[cell_nb(P, ix, d, -1)] + rho);
            s[1] += 0.5 * rbar * um * um;
            const double q = (P.geom == MUSIC_GEOM_SPHERICAL) ? (fabs(uc) + cs) / sph_h(P, d, ix[0])
                                                              : (fabs(uc) + cs) * P.idx[d];
            s[7] = nanmax(s[7], q);
            if (d == 1) {
                s[2] += 0.5 * rbar * um * um * dV;
                const double xc = P.x0[0] + (ix[0] + 0.5) * P.dx[0];
                s[3] += um * cos(kmode * xc);
                s[4] += um * sin(kmode * xc);
            }
        }
        const double sp = sqrt(u2);
        s[5] = nanmax(s[5], sp / cs);
        s[6] = nanmax(s[6], sp);
    }
    for (int q = 0; q < 5; q++) {
        const double r = block_sum<BS>(s[q], sh);
        if (threadIdx.x == 0) rows[(long long)q * P.n[1] + j] = r;
    }
    for (int q = 5; q < NR; q++) {
        const double r = block_max<BS>(s[q], sh);
        if (threadIdx.x == 0) rows[(long long)q * P.n[1] + j] = r;
    }
}

__global__ void __launch_bounds__(BS) k_combine_rows(GridParams P, const double *rows, DevScalars *ds,
                                                      int want_diag)
{
    pdl_entry();
    // one block; thread t takes rows t, t + BS, ... and the block tree
    // combines them: a fixed order for a given grid
    __shared__ double sh[BS / 32];
    const int ny = P.n[1];
    const double per_row = (double)((long long)P.n[0] * P.n[2]);
    double a[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    for (int j = threadIdx.x; j < ny; j += BS) {
        const double xh = rows[j] / per_row;
        const double xm = (xh <= 0.5) ? 2.0 * xh : 2.0 * (1.0 - xh);
        a[0] += xm * P.dx[1];
        for (int q = 1; q < 5; q++) a[q] += rows[(long long)q * ny + j];
        for (int q = 5; q < 8; q++) a[q] = nanmax(a[q], rows[(long long)q * ny + j]);
    }
    double r[8];
    for (int q = 0; q < 5; q++) r[q] = block_sum<BS>(a[q], sh);
    for (int q = 5; q < 8; q++) r[q] = block_max<BS>(a[q], sh);
    if (threadIdx.x != 0) return;
    ds->rate = r[7];
    if (want_diag) {
        ds->diag[0] = r[0];
        ds->diag[1] = r[5];
        ds->diag[2] = 2.0 / (double)P.N * sqrt(r[3] * r[3] + r[4] * r[4]);
        ds->diag[3] = r[2];
        ds->diag[4] = r[1] / (double)P.N;
        ds->diag[5] = r[6];
    }
}

// Per row j and slab sl of its z range (gridDim.y slabs): the maxima over
// its cells and directions of (|u_d| + c_s) / h_d, |u_d| / h_d and D / h_d^2
// (D = chi / (rho c_v), 0 without radiative diffusion); the first has k_rows'
// expression, so both give the same rate.  A maximum does not depend on the
// order it is taken in, so neither do the rates on the slab count.
__global__ void __launch_bounds__(BS) k_rate_rows(GridParams P, const double *U, double *rows)
{
    pdl_entry();
    __shared__ double sh[BS / 32];
    const int j = blockIdx.x, sl = blockIdx.y, ns = gridDim.y;
    const int z0 = (int)((long long)sl * P.n[2] / ns), z1 = (int)((long long)(sl + 1) * P.n[2] / ns);
    double s[3] = {0, 0, 0};
    const long long per_slab = (long long)P.n[0] * (z1 - z0);
    for (long long t = threadIdx.x; t < per_slab; t += BS) {
        int ix[3] = {(int)(t % P.n[0]), j, z0 + (int)(t / P.n[0])};
        const long long c = cell_index(P, ix);
        const double rho = U[c];
        const double cs = sqrt(P.gamma * (P.gm1 * U[P.N + c]) / rho);
        double D = 0.0;
        if (P.conduct) {
            const double T = P.gm1 * U[P.N + c] / rho;
            const double t3 = T * T * T;
            const double chi = P.chi0 * (t3 * t3 * sqrt(T)) / (rho * rho);
            D = chi * P.gm1 / rho;
        }
        for (int d = 0; d < P.nd; d++) {
            const double um = face_u(P, U, ix, c, d);
            double up = 0.0;
            if (!upper_wall(P, ix, d)) {
                int jx[3] = {ix[0], ix[1], ix[2]};
                jx[d] = (ix[d] + 1 == P.n[d]) ? 0 : ix[d] + 1;
                up = face_u(P, U, jx, cell_index(P, jx), d);
            }
            const double a = fabs(0.5 * (um + up));
            if (P.geom == MUSIC_GEOM_SPHERICAL) {
                const double h = sph_h(P, d, ix[0]);
                s[0] = nanmax(s[0], (a + cs) / h);
                s[1] = nanmax(s[1], a / h);
                s[2] = nanmax(s[2], D / (h * h));
            } else {
                s[0] = nanmax(s[0], (a + cs) * P.idx[d]);
                s[1] = nanmax(s[1], a * P.idx[d]);
                s[2] = nanmax(s[2], D * P.idx2[d]);
            }
        }
    }
    const long long per_q = (long long)P.n[1] * ns;
    for (int q = 0; q < 3; q++) {
        const double r = block_max<BS>(s[q], sh);
        if (threadIdx.x == 0) rows[q * per_q + (long long)j * ns + sl] = r;
    }
}

// the three rates from the partial maxima of k_rate_rows (count per rate)
__global__ void __launch_bounds__(BS) k_combine_rates(GridParams P, const double *rows, DevScalars *ds, int count)
{
    pdl_entry();
    __shared__ double sh[BS / 32];
    double a[3] = {0, 0, 0};
    for (int j = threadIdx.x; j < count; j += BS)
        for (int q = 0; q < 3; q++) a[q] = nanmax(a[q], rows[(long long)q * count + j]);
    double r[3];
    for (int q = 0; q < 3; q++) r[q] = block_max<BS>(a[q], sh);
    if (threadIdx.x == 0) {
        ds->rate = r[0];
        ds->rate_adv = r[1];
        ds->rate_rad = r[2];
    }
}

int run_rows(music_grid *g, const double *U, double rho_L, double rho_H, int want_diag, cudaStream_t s)
{
    const GridParams &P = g->P;
    const double kmode = 2.0 * (2.0 * M_PI / (P.n[0] * P.dx[0]));
    k_rows<<<P.n[1], BS, 0, s>>>(P, U, rho_L, rho_H, kmode, g->diag_rows);
    CHECK_LAUNCH();
    k_combine_rows<<<1, BS, 0, s>>>(P, g->diag_rows, g->ds, want_diag);
    CHECK_LAUNCH();
    return MUSIC_OK;
}

}  // namespace

int cfl_rate(music_grid *g, const double *U, cudaStream_t s)
{
    return run_rows(g, U, 1.0, 2.0, 0, s);
}

int diagnostics(music_grid *g, const double *U, double rho_L, double rho_H, cudaStream_t s)
{
    return run_rows(g, U, rho_L, rho_H, 1, s);
}

// Convergence study of Sec. 4: one thread per coarse y-face compares the
// coarse vertical velocity with the mean of the r fine faces tiling it; the
// sums |v_c - mean| and |mean| go through a deterministic two-stage reduction.
__device__ inline double yface_v(const GridParams &P, const double *U, int i, int j)
{
    if (P.bc[1] == MUSIC_BC_WALL && j == 0) return 0.0;
    const long long c = i + (long long)P.n[0] * j;
    const long long b = i + (long long)P.n[0] * (j == 0 ? P.n[1] - 1 : j - 1);
    return U[3 * P.N + c] / (0.5 * (U[b] + U[c]));
}

__global__ void __launch_bounds__(BS) k_vy_error(GridParams Pf, const double *Uf, GridParams Pc, const double *Uc,
                                                 int r, double *partial, double *dst, unsigned int *counter)
{
    pdl_entry();
    __shared__ double sh[BS / 32];
    double a = 0.0, b = 0.0;
    for (long long f = blockIdx.x * (long long)BS + threadIdx.x; f < Pc.N; f += (long long)gridDim.x * BS) {
        const int i = (int)(f % Pc.n[0]), j = (int)(f / Pc.n[0]);
        double m = 0.0;
        for (int k = 0; k < r; k++) m += yface_v(Pf, Uf, i * r + k, j * r);
        m /= (double)r;
        a += fabs(yface_v(Pc, Uc, i, j) - m);
        b += fabs(m);
    }
    const double ra = block_sum<BS>(a, sh);
    const double rb = block_sum<BS>(b, sh);
    if (threadIdx.x == 0) {
        partial[blockIdx.x] = ra;
        partial[gridDim.x + blockIdx.x] = rb;
    }
    if (last_block_done(counter)) finish_sums<BS>(partial, gridDim.x, gridDim.x, 2, dst, sh);
}

extern "C" int music_velocity_error(music_grid *fine, music_grid *coarse, double *err, void *stream)
{
    if (!fine || !coarse || !err) {
        set_error("music_velocity_error: NULL argument");
        return MUSIC_E_INVAL;
    }
    const GridParams &Pf = fine->P, &Pc = coarse->P;
    const int r = Pc.n[0] > 0 ? Pf.n[0] / Pc.n[0] : 0;
    if (Pf.nd != 2 || Pc.nd != 2 || r < 1 || Pf.n[0] != r * Pc.n[0] || Pf.n[1] != r * Pc.n[1] ||
        Pf.bc[1] != Pc.bc[1]) {
        set_error("music_velocity_error: 2-D grids whose extents differ by one integer factor");
        return MUSIC_E_INVAL;
    }
    cudaStream_t s = (cudaStream_t)stream;
    int nb = (int)((Pc.N + BS - 1) / BS);
    if (nb > coarse->nb) nb = coarse->nb;
    k_vy_error<<<nb, BS, 0, s>>>(Pf, fine->U, Pc, coarse->U, r, coarse->partials, &coarse->ds->diag[6],
                                 &coarse->ds->counters[CNT_SUMSQ]);
    CHECK_LAUNCH();
    CUDA_TRY(cudaMemcpyAsync(coarse->hs, coarse->ds, sizeof(DevScalars), cudaMemcpyDeviceToHost, s));
    CUDA_TRY(cudaStreamSynchronize(s));
    *err = coarse->hs->diag[6] / coarse->hs->diag[7];
    return MUSIC_OK;
}

int step_rates(music_grid *g, cudaStream_t s)
{
    const GridParams &P = g->P;
    const int ns = rate_slabs(P);
    k_rate_rows<<<dim3(P.n[1], ns), BS, 0, s>>>(P, g->U, g->diag_rows);
    CHECK_LAUNCH();
    k_combine_rates<<<1, BS, 0, s>>>(P, g->diag_rows, g->ds, P.n[1] * ns);
    CHECK_LAUNCH();
    return MUSIC_OK;
}

extern "C" int music_select_dt(music_grid *g, const music_dt_limits *lim, double *dt, int *which, void *stream)
{
    if (!g || !lim || !dt) {
        set_error("music_select_dt: NULL argument");
        return MUSIC_E_INVAL;
    }
    cudaStream_t s = (cudaStream_t)stream;
    TRY(step_rates(g, s));
    CUDA_TRY(cudaMemcpyAsync(g->hs, g->ds, sizeof(DevScalars), cudaMemcpyDeviceToHost, s));
    CUDA_TRY(cudaStreamSynchronize(s));
    const double rates[3] = {g->hs->rate, g->hs->rate_adv, g->hs->rate_rad};
    const double cfl[3] = {lim->cfl_hydro, lim->cfl_adv, lim->cfl_rad};
    double best = INFINITY;
    int w = -1;
    for (int k = 0; k < 3; k++) {
        if (!std::isfinite(rates[k])) {
            set_error("music_select_dt: non-finite rate");
            return MUSIC_E_NONFINITE;
        }
        if (!(cfl[k] > 0.0) || !(rates[k] > 0.0)) continue;
        const double t = cfl[k] / rates[k];
        if (t < best) {
            best = t;
            w = k;
        }
    }
    if (lim->dt_max > 0.0 && lim->dt_max < best) {
        best = lim->dt_max;
        w = 3;
    }
    if (w < 0) {
        set_error("music_select_dt: no limit applies (all <= 0, or the state is at rest)");
        return MUSIC_E_INVAL;
    }
    *dt = best;
    if (which) *which = w;
    return MUSIC_OK;
}

// ---------------------------------------------------------------------------
// Allocation-free variant of the CFL-rate reduction (music_cfl_rate_noalloc).
//
// Its scratch -- the per-row partials of k_rows and the result slot written
// by k_combine_rows -- lives in one file-scope device array of fixed size,
// which every GPU that loads this library holds until the process exits.  In
// host code `g_noalloc_scratch` names a host-side stand-in, not device
// memory, so the kernels get the array's device address, looked up once per
// device with cudaGetSymbolAddress on the first call made with that device
// current.
namespace {

constexpr int NOALLOC_MAX_ROWS = 16384;  // grid rows (n[1]) the scratch holds
struct NoallocScratch {
    double rows[NR * NOALLOC_MAX_ROWS];  // 8 quantities per row
    DevScalars ds;                       // k_combine_rows writes ds.rate here
};
static __device__ __align__(256) NoallocScratch g_noalloc_scratch;

constexpr int NOALLOC_MAX_DEVICES = 64;
NoallocScratch *g_noalloc_ptr[NOALLOC_MAX_DEVICES];
std::mutex g_noalloc_mu;

__global__ void k_copy_rate(const NoallocScratch *S, double *rate) {
    pdl_entry(); *rate = S->ds.rate; }

}  // namespace

extern "C" int music_cfl_rate_noalloc(const music_grid_desc *desc, const double *U, double *rate, void *stream)
{
    if (!desc || !U || !rate) {
        set_error("music_cfl_rate_noalloc: NULL argument");
        return MUSIC_E_INVAL;
    }
    music_grid_desc d = *desc;
    TRY(grid_validate(&d));
    if (d.n[1] > NOALLOC_MAX_ROWS) {
        set_error("music_cfl_rate_noalloc: n[1] = %d rows exceeds the fixed scratch of %d rows", d.n[1],
                  NOALLOC_MAX_ROWS);
        return MUSIC_E_INVAL;
    }
    int dev = 0;
    CUDA_TRY(cudaGetDevice(&dev));
    if (dev < 0 || dev >= NOALLOC_MAX_DEVICES) {
        set_error("music_cfl_rate_noalloc: device %d beyond the %d supported", dev, NOALLOC_MAX_DEVICES);
        return MUSIC_E_INVAL;
    }
    NoallocScratch *S = nullptr;
    {
        std::lock_guard<std::mutex> lk(g_noalloc_mu);
        if (!g_noalloc_ptr[dev]) {
            void *p = nullptr;
            CUDA_TRY(cudaGetSymbolAddress(&p, g_noalloc_scratch));
            g_noalloc_ptr[dev] = (NoallocScratch *)p;
        }
        S = g_noalloc_ptr[dev];
    }
    GridParams P;
    fill_grid_params(d, &P);
    cudaStream_t s = (cudaStream_t)stream;
    const double kmode = 2.0 * (2.0 * M_PI / (P.n[0] * P.dx[0]));
    // every row slot k_combine_rows reads is written by k_rows first, so
    // nothing needs clearing between calls
    k_rows<<<P.n[1], BS, 0, s>>>(P, U, 1.0, 2.0, kmode, S->rows);
    CHECK_LAUNCH();
    k_combine_rows<<<1, BS, 0, s>>>(P, S->rows, &S->ds, 0);
    CHECK_LAUNCH();
    k_copy_rate<<<1, 1, 0, s>>>(S, rate);
    CHECK_LAUNCH();
    return MUSIC_OK;
}
