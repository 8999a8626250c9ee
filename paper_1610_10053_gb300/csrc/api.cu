// extern "C" entry points of libmusic (declared in include/music.h): grid
// lifetime, state transfer and the single-call operators of the JFNK loop.
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <new>
#include <vector>

#include "internal.h"
#include "tile_precond.cuh"
#include "tiles.h"

#include <atomic>

namespace {
thread_local char g_err[1024] = "";
std::atomic<unsigned long long> g_launches{0};

void fill_defaults(music_grid_desc &d)
{
    if (d.gmres_restart == 0) d.gmres_restart = 30;
    if (d.gmres_max_restarts == 0) d.gmres_max_restarts = 10;
    if (d.gmres_rtol == 0.0) d.gmres_rtol = 1e-1;
    if (d.newton_max_its == 0) d.newton_max_its = 12;
    if (d.newton_tol == 0.0) d.newton_tol = 1e-8;
    if (d.precond == 0) d.precond = MUSIC_PC_ACOUSTIC;
    else if (d.precond < 0) d.precond = MUSIC_PC_NONE;
    if (d.precond_sweeps == 0) d.precond_sweeps = 16;
    if (d.max_dt_halvings == 0) d.max_dt_halvings = 4;
    if (d.ndim == 2) d.n[2] = 1;
}

int validate(const music_grid_desc &d)
{
    if (d.ndim != 2 && d.ndim != 3) {
        set_error("ndim must be 2 or 3 (got %d)", d.ndim);
        return MUSIC_E_INVAL;
    }
    int hse = 0;
    for (int k = 0; k < d.ndim; k++) {
        if (d.n[k] < 4) {
            set_error("n[%d] = %d: every direction needs at least 4 cells", k, d.n[k]);
            return MUSIC_E_INVAL;
        }
        if (!(d.length[k] > 0.0)) {
            set_error("length[%d] must be > 0", k);
            return MUSIC_E_INVAL;
        }
        if (d.bc[k] != MUSIC_BC_PERIODIC && d.bc[k] != MUSIC_BC_WALL) {
            set_error("bc[%d] = %d is not a known boundary condition", k, d.bc[k]);
            return MUSIC_E_INVAL;
        }
        if (d.bc[k] == MUSIC_BC_WALL && d.wall_scalar[k] == MUSIC_WALL_HSE_LINEAR_T) hse++;
        if (d.bc[k] == MUSIC_BC_WALL && d.wall_scalar[k] != MUSIC_WALL_MIRROR &&
            d.wall_scalar[k] != MUSIC_WALL_HSE_LINEAR_T) {
            set_error("wall_scalar[%d] = %d unknown", k, d.wall_scalar[k]);
            return MUSIC_E_INVAL;
        }
    }
    if (hse > 1) {
        set_error("at most one direction may use hydrostatic wall ghosts");
        return MUSIC_E_INVAL;
    }
    if (!(d.gamma > 1.0)) {
        set_error("gamma must be > 1");
        return MUSIC_E_INVAL;
    }
    if (!std::isfinite(d.cfl_hydro) || !std::isfinite(d.cfl_adv) || !std::isfinite(d.cfl_rad)) {
        set_error("time-step limits must be finite");
        return MUSIC_E_INVAL;
    }
    if (d.precision != MUSIC_FP64 && d.precision != MUSIC_MIXED) {
        set_error("precision %d unknown", d.precision);
        return MUSIC_E_INVAL;
    }
    if (d.gmres_restart < 1 || d.gmres_restart > MUSIC_MAXV - 1) {
        set_error("gmres_restart must be in 1..%d", MUSIC_MAXV - 1);
        return MUSIC_E_INVAL;
    }
    if (d.precond != MUSIC_PC_NONE && d.precond != MUSIC_PC_ACOUSTIC) {
        set_error("precond %d unknown", d.precond);
        return MUSIC_E_INVAL;
    }
    if (d.precond_sweeps < 0 || d.gmres_max_restarts < 0 || d.newton_max_its < 1 || d.max_dt_halvings < 0 ||
        !(d.newton_tol > 0.0) || !(d.gmres_rtol > 0.0)) {
        set_error("invalid solver options");
        return MUSIC_E_INVAL;
    }
    if (d.geometry != MUSIC_GEOM_CARTESIAN && d.geometry != MUSIC_GEOM_SPHERICAL) {
        set_error("geometry %d unknown", d.geometry);
        return MUSIC_E_INVAL;
    }
    if (d.geometry == MUSIC_GEOM_SPHERICAL) {
        if (d.ndim != 2 || d.bc[0] != MUSIC_BC_WALL || !(d.origin[0] > 0.0) || !(d.origin[1] > 0.0) ||
            !(d.origin[1] + d.length[1] < 3.14159265358979323846)) {
            set_error("spherical grids are 2-D with walls in r, r > 0 and 0 < theta < pi");
            return MUSIC_E_INVAL;
        }
    }
    if (d.conduct && !(d.chi0 >= 0.0)) {
        set_error("chi0 must be >= 0");
        return MUSIC_E_INVAL;
    }
    if (d.nscalars < 0 || d.nscalars > 8 || (d.nscalars > 0 && d.geometry != MUSIC_GEOM_CARTESIAN)) {
        set_error("nscalars must be 0..8, on Cartesian grids");
        return MUSIC_E_INVAL;
    }
    return MUSIC_OK;
}

GridParams make_params(const music_grid_desc &d)
{
    GridParams P;
    memset(&P, 0, sizeof(P));
    P.nd = d.ndim;
    P.nv = 2 + d.ndim;
    for (int k = 0; k < 3; k++) {
        P.n[k] = (k < d.ndim) ? d.n[k] : 1;
        P.ne[k] = (k < d.ndim) ? P.n[k] + 2 * MUSIC_GHOST : 1;
        const double L = (k < d.ndim) ? d.length[k] : 1.0;
        P.dx[k] = L / P.n[k];
        P.idx[k] = 1.0 / P.dx[k];
        P.idx2[k] = 1.0 / (P.dx[k] * P.dx[k]);
        P.x0[k] = d.origin[k];
        P.bc[k] = (k < d.ndim) ? d.bc[k] : MUSIC_BC_PERIODIC;
        P.ws[k] = d.wall_scalar[k];
        P.g[k] = (k < d.ndim) ? d.g[k] : 0.0;
    }
    P.N = (long long)P.n[0] * P.n[1] * P.n[2];
    P.cs[0] = 1;
    P.cs[1] = P.n[0];
    P.cs[2] = (long long)P.n[0] * P.n[1];
    P.es[0] = 1;
    P.es[1] = P.ne[0];
    P.es[2] = (long long)P.ne[0] * P.ne[1];
    P.M = P.es[2] * P.ne[2];
    P.gamma = d.gamma;
    P.gm1 = d.gamma - 1.0;
    P.geom = d.geometry;
    P.conduct = d.conduct ? 1 : 0;
    P.chi0 = d.chi0;
    P.lum = d.lum;
    for (int k = 0; k < 3; k++) P.flux_wall[k] = (k < d.ndim && d.bc[k] == MUSIC_BC_WALL) ? d.flux_wall[k] : 0;
    P.gface = nullptr;
    P.sgeo = nullptr;
    P.dt_dev = nullptr;
    return P;
}

// The grid's device buffers, in one list shared by the footprint query and
// by creation: f(slot, bytes) is called once per buffer.
template <class F>
void alloc_plan(music_grid *g, F &&f)
{
    const music_grid_desc &d = g->desc;
    const GridParams &P = g->P;
    const size_t n = g->n, N = (size_t)P.N, M = (size_t)P.M;
    const size_t ks = g->mixed ? sizeof(float) : sizeof(double);
    for (double **p : {&g->U, &g->Un, &g->Cn, &g->RU, &g->b, &g->x, &g->t64}) f((void **)p, n * sizeof(double));
    f(&g->V, (size_t)(d.gmres_restart + 1) * n * ks);
    for (void **p : {&g->w, &g->z, &g->u, &g->q}) f(p, n * ks);
    if (d.precond != MUSIC_PC_NONE) {
        f(&g->Z, (size_t)d.gmres_restart * n * ks);
        for (int k = 0; k < P.nd; k++) f(&g->pa[k], N * ks);
        for (void **p : {&g->pgp, &g->php, &g->pD, &g->pb, &g->pdp, &g->pdq}) f(p, N * ks);
        if (general_grid(P)) {
            f(&g->prh, N * ks);
            for (int k = 0; k < P.nd; k++) f(&g->pkf[k], N * ks);
            f(&g->pgw, (size_t)2 * P.nd * N * ks);
        }
    }
    if (P.geom == MUSIC_GEOM_SPHERICAL) {
        f((void **)&g->gface, (size_t)(P.n[0] + 1) * sizeof(double));
        f((void **)&g->sgeo, (size_t)SG_COUNT * N * sizeof(double));
    }
    // linearisation planes of the difference-form Jv (mixed grids on the
    // fused 2-D stencil), written with every R and F evaluation
    if (g->mixed && P.nd == 2 && g->stencil_variant != STENCIL_MULTIPASS && !general_grid(P))
        f((void **)&g->lin, (size_t)LIN_PLANES * N * sizeof(float));
    // and on the ghosted grid for the multi-pass stencil's (3-D, or 2-D on request)
    if (g->mixed && (P.nd == 3 || g->stencil_variant == STENCIL_MULTIPASS) && !general_grid(P))
        f((void **)&g->linx, (size_t)(2 + 4 * P.nd + P.nd * P.nd) * M * sizeof(float));
    // the multi-pass stencil (3-D, spherical, conducting, or 2-D on request)
    // keeps its planes on the ghosted grid; the fused 2-D kernels need none
    if (P.nd == 3 || g->stencil_variant == STENCIL_MULTIPASS || general_grid(P)) {
        ExtScratch &X = g->ext;
        if (P.conduct) {
            f((void **)&X.Tt, M * sizeof(double));
            f((void **)&X.chi, M * sizeof(double));
            for (int k = 0; k < P.nd; k++) f((void **)&X.Gc[k], M * sizeof(double));
        }
        for (double **p : {&X.rho, &X.e, &X.p}) f((void **)p, M * sizeof(double));
        for (int k = 0; k < P.nd; k++) {
            for (double **p : {&X.uf[k], &X.srho[k], &X.se[k], &X.Frho[k], &X.FE[k], &X.Phi[k]})
                f((void **)p, M * sizeof(double));
            for (int q = 0; q < P.nd; q++) {
                f((void **)&X.su[k][q], M * sizeof(double));
                if (q != k) f((void **)&X.Psi[k][q], M * sizeof(double));
            }
        }
    }
    // reduction partials: the Krylov kernels' and the preconditioner's
    // tile-independent |z|^2 blocks (2-D)
    size_t np = (size_t)MUSIC_MAXV * (g->nb > VEC_BLOCKS_MAX ? g->nb : VEC_BLOCKS_MAX);
    if (P.nd == 2 && (size_t)tile::norm_partial_count(P) > np) np = (size_t)tile::norm_partial_count(P);
    f((void **)&g->partials, np * sizeof(double));
    f((void **)&g->hg, (size_t)(MUSIC_MAXV * MUSIC_MAXV + 4 * MUSIC_MAXV) * sizeof(double));
    f(&g->binst, 1024);  // batched-solver descriptor (sizeof checked in batched.cu)
    f((void **)&g->ds, sizeof(DevScalars));
    f((void **)&g->ctl, sizeof(SolveCtl));
    // per-row partials of the diagnostics (8 a row) and of the rates (3 a row and slab)
    const size_t nrow = (size_t)P.n[1] * (8 > 3 * rate_slabs(P) ? 8 : 3 * rate_slabs(P));
    f((void **)&g->diag_rows, nrow * sizeof(double));
    if (g->ns > 0) {
        const size_t nq = (size_t)g->ns * N;
        KSpace &S = g->sc;
        for (double **p : {&S.U, &S.RU, &S.b, &S.x, &S.t64, &g->sq_n, &g->sq_c}) f((void **)p, nq * sizeof(double));
        f(&S.V, (size_t)(d.gmres_restart + 1) * nq * ks);
        for (void **p : {&S.w, &S.z, &S.u}) f(p, nq * ks);
        f((void **)&g->sfr, (size_t)P.nd * N * sizeof(double));
        f((void **)&S.ds, sizeof(DevScalars));
    }
}

void init_grid_struct(music_grid *g, const music_grid_desc &d)
{
    memset(g, 0, sizeof(*g));
    g->desc = d;
    g->P = make_params(d);
    g->mixed = (d.precision == MUSIC_MIXED);
    // MUSIC_STENCIL=multipass selects the multi-pass stencil on 2-D grids
    const char *sv = getenv("MUSIC_STENCIL");
    g->stencil_variant = (sv && strcmp(sv, "multipass") == 0) ? STENCIL_MULTIPASS : STENCIL_AUTO;
    // MUSIC_PRECOND=multikernel selects one kernel per Jacobi sweep;
    // MUSIC_PRECOND=rows keeps those sweeps one cell a thread (no 16-byte chunks)
    const char *pv = getenv("MUSIC_PRECOND");
    g->pc_variant = !pv ? PC_AUTO
                        : strcmp(pv, "multikernel") == 0 ? PC_MULTIKERNEL
                                                         : strcmp(pv, "rows") == 0 ? PC_ROWS : PC_AUTO;
    // MUSIC_SOLVER=host sequences Newton and GMRES from the host
    const char *so = getenv("MUSIC_SOLVER");
    g->solver_variant = (so && strcmp(so, "host") == 0) ? SOLVER_HOST : SOLVER_GRAPH;
    // mixed grids take the difference form of Jv; MUSIC_JV=fd keeps FP64
    const char *jv = getenv("MUSIC_JV");
    g->jv_form = (g->mixed && !(jv && strcmp(jv, "fd") == 0)) ? JV_DIFF : JV_FD;
    // MUSIC_LOOP_CAP=<n> lowers the bound on loop bodies per Newton attempt
    // (for tests of the bound's expiry; the default is never reached)
    const char *lc = getenv("MUSIC_LOOP_CAP");
    g->loop_cap = lc ? atoi(lc) : 0;
    if (g->loop_cap < 0) g->loop_cap = 0;
    g->stile = STENCIL_TILE_DEFAULT;
    g->rtile = STENCIL_TILE_DEFAULT;
    g->ptile = PRECOND_TILE_DEFAULT;
    g->psplit = default_split(d.precond_sweeps);
    g->btile = BATCH_TILE_DEFAULT;
    tune_lookup(g);  // shapes an earlier tuning picked for this configuration
    g->n = (size_t)g->P.nv * g->P.N;
    g->ns = d.nscalars;
    g->sc.n = (size_t)g->ns * g->P.N;
    // scalar grids run the host-sequenced Newton loop
    if (g->ns > 0) g->solver_variant = SOLVER_HOST;
    // reduction blocks: enough to fill the GPU, fixed per grid
    long long nb = ((long long)g->n + 255) / 256;
    g->nb = (int)(nb > 2 * 152 ? 2 * 152 : (nb < 1 ? 1 : nb));
}

void free_grid(music_grid *g)
{
    if (!g) return;
    graph_release(g);
    alloc_plan(g, [&](void **slot, size_t) {
        if (*slot) cudaFreeAsync(*slot, g->home);
        *slot = nullptr;
    });
    cudaStreamSynchronize(g->home);
    if (g->hs) cudaFreeHost(g->hs);
    if (g->sc.hs) cudaFreeHost(g->sc.hs);
    if (g->prof_events_made)
        for (int i = 0; i < 2 * 256; i++) cudaEventDestroy(g->prof_ev[i]);
    delete g;
}

int check_grid(const music_grid *g)
{
    if (!g) {
        set_error("grid is NULL");
        return MUSIC_E_INVAL;
    }
    return MUSIC_OK;
}

}  // namespace

thread_local long long t_launches = 0;

void count_launch()
{
    g_launches.fetch_add(1, std::memory_order_relaxed);
    t_launches++;
}
void count_launches(long long k) { g_launches.fetch_add(k, std::memory_order_relaxed); }
long long capture_launches() { return t_launches; }

void fill_grid_params(const music_grid_desc &d, GridParams *P) { *P = make_params(d); }

int loop_cap_of(const music_grid *g)
{
    const music_grid_desc &d = g->desc;
    if (g->loop_cap > 0) return g->loop_cap;
    return d.newton_max_its * (d.gmres_max_restarts + 1) * (d.gmres_restart + 3) + 64;
}

int grid_validate(music_grid_desc *d)
{
    fill_defaults(*d);
    return validate(*d);
}

int grid_footprint(const music_grid_desc *desc, size_t *bytes)
{
    music_grid_desc d = *desc;
    fill_defaults(d);
    TRY(validate(d));
    music_grid *g = new (std::nothrow) music_grid;
    if (!g) {
        set_error("host allocation failed");
        return MUSIC_E_OOM;
    }
    init_grid_struct(g, d);
    size_t total = 0;
    alloc_plan(g, [&](void **, size_t b) { total += b; });
    delete g;
    *bytes = total;
    return MUSIC_OK;
}

int grid_create(const music_grid_desc *desc, cudaStream_t home, music_grid **out)
{
    if (!desc || !out) {
        set_error("music_create_grid: NULL argument");
        return MUSIC_E_INVAL;
    }
    *out = nullptr;
    music_grid_desc d = *desc;
    fill_defaults(d);
    TRY(validate(d));
    music_grid *g = new (std::nothrow) music_grid;
    if (!g) {
        set_error("host allocation failed");
        return MUSIC_E_OOM;
    }
    init_grid_struct(g, d);
    g->home = home;
    if (cudaGetDevice(&g->device) != cudaSuccess) {
        cudaGetLastError();
        delete g;
        set_error("no CUDA device");
        return MUSIC_E_CUDA;
    }
    // stream-ordered allocation on the home stream: no device-wide sync, so
    // grids created by concurrent workers do not stall one another
    int fail = 0;
    alloc_plan(g, [&](void **slot, size_t b) {
        if (fail) return;
        if (cudaMallocAsync(slot, b, home) != cudaSuccess) {
            cudaGetLastError();
            *slot = nullptr;
            fail = 1;
            return;
        }
        g->bytes += b;
        // every buffer starts at zero (the stencil scratch is read at its
        // ghosted edges before it is written)
        if (cudaMemsetAsync(*slot, 0, b, home) != cudaSuccess) {
            cudaGetLastError();
            fail = 1;
        }
    });
    if (!fail && g->gface) {
        // radial gravity on the r-faces: the table given, else the constant g[0]
        std::vector<double> tab(g->P.n[0] + 1, d.g[0]);
        if (d.g_radial)
            for (int i = 0; i <= g->P.n[0]; i++) tab[i] = d.g_radial[i];
        if (cudaMemcpyAsync(g->gface, tab.data(), tab.size() * sizeof(double), cudaMemcpyHostToDevice, home) !=
                cudaSuccess ||
            cudaStreamSynchronize(home) != cudaSuccess) {
            cudaGetLastError();
            fail = 1;
        }
        g->P.gface = g->gface;
    }
    if (!fail && g->sgeo) {
        g->P.sgeo = g->sgeo;
        if (sph_geo_build(g, home) != MUSIC_OK || cudaStreamSynchronize(home) != cudaSuccess) {
            cudaGetLastError();
            fail = 1;
        }
    }
    g->desc.g_radial = nullptr;  // copied; the caller's array is not retained
    if (!fail && cudaMallocHost(&g->hs, sizeof(DevScalars)) != cudaSuccess) {
        cudaGetLastError();
        g->hs = nullptr;
        fail = 1;
    }
    if (!fail && g->ns > 0 && cudaMallocHost(&g->sc.hs, sizeof(DevScalars)) != cudaSuccess) {
        cudaGetLastError();
        g->sc.hs = nullptr;
        fail = 1;
    }
    if (!fail && cudaStreamSynchronize(home) != cudaSuccess) {
        cudaGetLastError();
        fail = 1;
    }
    if (fail) {
        free_grid(g);
        set_error("device allocation failed");
        return MUSIC_E_OOM;
    }
    *out = g;
    return MUSIC_OK;
}

void grid_destroy(music_grid *g) { free_grid(g); }

int grid_set_state(music_grid *g, const double *U, int is_device, cudaStream_t s)
{
    CUDA_TRY(cudaMemcpyAsync(g->U, U, g->n * sizeof(double), is_device ? cudaMemcpyDeviceToDevice
                                                                        : cudaMemcpyHostToDevice, s));
    CUDA_TRY(cudaStreamSynchronize(s));
    return MUSIC_OK;
}

int grid_get_state(music_grid *g, double *U, int is_device, cudaStream_t s)
{
    CUDA_TRY(cudaMemcpyAsync(U, g->U, g->n * sizeof(double), is_device ? cudaMemcpyDeviceToDevice
                                                                        : cudaMemcpyDeviceToHost, s));
    CUDA_TRY(cudaStreamSynchronize(s));
    return MUSIC_OK;
}

void set_error(const char *fmt, ...)
{
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
}

extern "C" {

size_t music_last_error(char *buf, size_t len)
{
    size_t n = strlen(g_err);
    if (buf && len) {
        size_t k = n < len - 1 ? n : len - 1;
        memcpy(buf, g_err, k);
        buf[k] = 0;
    }
    return n;
}

const char *music_version(void) { return "libmusic 0.1 (sm_103a)"; }

uint64_t music_kernel_launches(void) { return g_launches.load(std::memory_order_relaxed); }

int music_create_grid(const music_grid_desc *desc, music_grid **out)
{
    return grid_create(desc, (cudaStream_t)0, out);
}

int music_destroy_grid(music_grid *grid)
{
    if (!grid) return MUSIC_OK;
    cudaDeviceSynchronize();  // the caller may have work on other streams
    grid_destroy(grid);
    return MUSIC_OK;
}

int music_grid_footprint(const music_grid_desc *desc, size_t *bytes)
{
    if (!desc || !bytes) {
        set_error("music_grid_footprint: NULL argument");
        return MUSIC_E_INVAL;
    }
    return grid_footprint(desc, bytes);
}

size_t music_state_size(const music_grid *grid) { return grid ? grid->n : 0; }

size_t music_grid_bytes(const music_grid *grid) { return grid ? grid->bytes : 0; }

int music_set_state(music_grid *grid, const double *U, int is_device)
{
    TRY(check_grid(grid));
    if (!U) {
        set_error("music_set_state: NULL state");
        return MUSIC_E_INVAL;
    }
    CUDA_TRY(cudaDeviceSynchronize());  // finish work queued on other streams
    return grid_set_state(grid, U, is_device, grid->home);
}

int music_get_state(music_grid *grid, double *U, int is_device)
{
    TRY(check_grid(grid));
    if (!U) {
        set_error("music_get_state: NULL buffer");
        return MUSIC_E_INVAL;
    }
    CUDA_TRY(cudaDeviceSynchronize());  // finish work queued on other streams
    return grid_get_state(grid, U, is_device, grid->home);
}

int music_spatial_operator(music_grid *grid, const double *U, double *R, void *stream)
{
    TRY(check_grid(grid));
    if (!U || !R) {
        set_error("music_spatial_operator: NULL pointer");
        return MUSIC_E_INVAL;
    }
    return stencil_apply(grid, SM_R, U, nullptr, nullptr, 1, R, 1, nullptr, 0.0, 1.0, (cudaStream_t)stream);
}

int music_residual(music_grid *grid, const double *U, const double *Un, double dt, double *F, void *stream)
{
    TRY(check_grid(grid));
    if (!U || !Un || !F) {
        set_error("music_residual: NULL pointer");
        return MUSIC_E_INVAL;
    }
    cudaStream_t s = (cudaStream_t)stream;
    // C^n in scratch, then F (RU scratch receives R(U))
    TRY(stencil_apply(grid, SM_CN, Un, nullptr, nullptr, 1, grid->t64, 1, nullptr, dt, 1.0, s));
    return stencil_apply(grid, SM_F, U, grid->t64, nullptr, 1, F, 1, grid->RU, dt, 1.0, s);
}

int music_jv(music_grid *grid, const double *U, const void *v, void *Jv, double dt, double eps, void *stream)
{
    TRY(check_grid(grid));
    if (!U || !v || !Jv) {
        set_error("music_jv: NULL pointer");
        return MUSIC_E_INVAL;
    }
    cudaStream_t s = (cudaStream_t)stream;
    const int kd = !grid->mixed;
    // R(U) into the grid's RU scratch (SM_JV reads it from there)
    TRY(stencil_apply(grid, SM_R, U, nullptr, nullptr, 1, grid->RU, 1, nullptr, dt, 1.0, s));
    if (!(eps > 0.0)) {
        TRY(dev_norm2(grid, U, 1, grid->n, &grid->ds->unorm2, s));
        TRY(dev_norm2(grid, v, kd, grid->n, &grid->ds->vnorm2, s));
    }
    TRY(dev_set_eps(grid, eps > 0.0 ? eps : 0.0, s));
    return stencil_apply(grid, SM_JV, U, grid->RU, v, kd, Jv, kd, nullptr, dt, 1.0, s);
}

int music_set_jv_form(music_grid *grid, int form)
{
    TRY(check_grid(grid));
    if ((form != MUSIC_JV_FD64 && form != MUSIC_JV_DIFF32) || (form == MUSIC_JV_DIFF32 && !grid->mixed)) {
        set_error("music_set_jv_form: form %d is not available on this grid", form);
        return MUSIC_E_INVAL;
    }
    const int f = (form == MUSIC_JV_DIFF32) ? JV_DIFF : JV_FD;
    if (f != grid->jv_form) {
        graph_release(grid);     // recorded with the other kernel
        grid->binst_ready = 0;   // the batched solver's descriptor names the form too
    }
    grid->jv_form = f;
    tune_lookup(grid);
    return MUSIC_OK;
}

int music_get_jv_form(const music_grid *grid, int *form)
{
    if (!grid || !form) {
        set_error("music_get_jv_form: NULL argument");
        return MUSIC_E_INVAL;
    }
    *form = (grid->jv_form == JV_DIFF) ? MUSIC_JV_DIFF32 : MUSIC_JV_FD64;
    return MUSIC_OK;
}

int music_precond_apply(music_grid *grid, const double *U, double dt, const void *r, void *z, void *stream)
{
    TRY(check_grid(grid));
    if (!U || !r || !z) {
        set_error("music_precond_apply: NULL pointer");
        return MUSIC_E_INVAL;
    }
    cudaStream_t s = (cudaStream_t)stream;
    TRY(precond_setup(grid, U, dt, s));
    return precond_apply(grid, dt, r, z, 0, s);
}

int music_newton_step(music_grid *grid, double dt_max, music_step_stats *st, void *stream)
{
    TRY(check_grid(grid));
    const music_grid_desc &d = grid->desc;
    if (std::isnan(dt_max) || std::isinf(dt_max)) {
        set_error("music_newton_step: dt_max must be finite");
        return MUSIC_E_INVAL;
    }
    double dt = dt_max;
    if (d.cfl_hydro > 0.0 || d.cfl_adv > 0.0 || d.cfl_rad > 0.0) {
        // the most restrictive limit, from the state at the start of the step:
        // chosen on the device when the recorded graph steps the grid (the same
        // choice, without a host round trip), else here
        const music_dt_limits lim = {d.cfl_hydro, d.cfl_adv, d.cfl_rad, dt_max};
        if (graph_driven(grid)) return newton_solve(grid, 0.0, st, (cudaStream_t)stream, &lim);
        TRY(music_select_dt(grid, &lim, &dt, nullptr, stream));
    } else if (!(dt_max > 0.0)) {
        set_error("music_newton_step: the grid has no time-step limit, so dt_max must be > 0");
        return MUSIC_E_INVAL;
    }
    return newton_solve(grid, dt, st, (cudaStream_t)stream);
}

int music_cfl_dt(music_grid *grid, double cfl, double *dt, void *stream)
{
    TRY(check_grid(grid));
    if (!dt || !(cfl > 0.0)) {
        set_error("music_cfl_dt: need cfl > 0 and an output pointer");
        return MUSIC_E_INVAL;
    }
    cudaStream_t s = (cudaStream_t)stream;
    TRY(cfl_rate(grid, grid->U, s));
    CUDA_TRY(cudaMemcpyAsync(grid->hs, grid->ds, sizeof(DevScalars), cudaMemcpyDeviceToHost, s));
    CUDA_TRY(cudaStreamSynchronize(s));
    const double rate = grid->hs->rate;
    if (!(rate > 0.0) || !std::isfinite(rate)) {
        set_error("music_cfl_dt: non-finite or zero signal speed");
        return MUSIC_E_NONFINITE;
    }
    *dt = cfl / rate;
    return MUSIC_OK;
}

int music_diagnostics(music_grid *grid, double rho_L, double rho_H, double *out, void *stream)
{
    TRY(check_grid(grid));
    if (!out || rho_H == rho_L) {
        set_error("music_diagnostics: need an output pointer and rho_H != rho_L");
        return MUSIC_E_INVAL;
    }
    cudaStream_t s = (cudaStream_t)stream;
    TRY(diagnostics(grid, grid->U, rho_L, rho_H, s));
    CUDA_TRY(cudaMemcpyAsync(grid->hs, grid->ds, sizeof(DevScalars), cudaMemcpyDeviceToHost, s));
    CUDA_TRY(cudaStreamSynchronize(s));
    for (int k = 0; k < 6; k++) out[k] = grid->hs->diag[k];
    return MUSIC_OK;
}

int music_profile_enable(music_grid *grid, int on)
{
    TRY(check_grid(grid));
    if (grid->prof_pending) TRY(prof_harvest(grid, 1));
    grid->prof_on = on ? 1 : 0;
    grid->prof_depth = 0;
    for (int c = 0; c < MUSIC_PROF_CLASSES; c++) {
        grid->prof_launches[c] = 0;
        grid->prof_ms[c] = 0.0;
    }
    return MUSIC_OK;
}

int music_profile_read(music_grid *grid, uint64_t *launches, double *ms)
{
    return music_profile_read_class(grid, MUSIC_PROF_JV, launches, ms);
}

int music_profile_read_class(music_grid *grid, int cls, uint64_t *launches, double *ms)
{
    TRY(check_grid(grid));
    if (cls < 0 || cls >= MUSIC_PROF_CLASSES) {
        set_error("music_profile_read_class: no class %d", cls);
        return MUSIC_E_INVAL;
    }
    if (grid->prof_pending) TRY(prof_harvest(grid, 1));
    if (launches) *launches = grid->prof_launches[cls];
    if (ms) *ms = grid->prof_ms[cls];
    return MUSIC_OK;
}

}  // extern "C"
