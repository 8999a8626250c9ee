// Host-side internals of libmusic shared between translation units.
#pragma once
#include <cuda_runtime.h>

#include <atomic>
#include <cstdint>
#include <string>

#include "common.cuh"

// Modes of the stencil assembly (what is written from R(W)).
enum StencilMode {
    SM_R = 0,    // out = R(U)
    SM_CN = 1,   // out = U + dt/2 R(U)                  (step constant C^n)
    SM_F = 2,    // out = sign ((U - C^n) - dt/2 R(U)), also R(U) -> RU
    SM_JV = 3,   // W = U + eps v; out = v - dt/2 (R(W) - RU) / eps
    SM_CNF = 4   // at U = U^n: C^n = U + dt/2 R(U) into aux (written), out and RU_out as SM_F
                 // (one evaluation of R(U^n) for the step constant and the first residual)
};

// Multi-pass stencil scratch on the extended grid (M doubles each).
struct ExtScratch {
    double *rho, *e, *p;
    double *uf[3], *srho[3], *se[3], *Frho[3], *FE[3], *Phi[3];
    double *su[3][3], *Psi[3][3];
    double *Tt, *chi, *Gc[3];  // radiative diffusion: T, chi per cell, chi dT/dn per face
};

enum StencilVariant { STENCIL_AUTO = 0, STENCIL_FUSED = 1, STENCIL_MULTIPASS = 2 };
enum SolverVariant { SOLVER_GRAPH = 0, SOLVER_HOST = 1 };
enum PrecondVariant { PC_AUTO = 0, PC_MULTIKERNEL = 1, PC_ROWS = 2 };
// Form of the Jacobian-free product: FP64 difference of two residual
// evaluations, or the difference form with FP32 differences (mixed-precision
// grids on the fused 2-D stencil; tile_jvdiff.cuh)
enum JvForm { JV_FD = 0, JV_DIFF = 1 };
// The linearisation planes written by the fused stencil's R and F modes for
// the difference form of Jv (tile_jvdiff.cuh): at every cell, rounded to
// FP32, the values at U of rho, e, the lower x-face velocity u and the lower
// y-face velocity v, and the backward differences of each to the cell's x-
// and y-neighbour, formed in FP64 first.  Plane k holds entry k per cell.
enum LinPlane {
    LIN_R = 0, LIN_E, LIN_U, LIN_V,
    LIN_DRX, LIN_DRY, LIN_DEX, LIN_DEY, LIN_DUX, LIN_DUY, LIN_DVX, LIN_DVY,
    LIN_PLANES
};

// grids that need the general (geometry / conduction) code paths
inline bool general_grid(const GridParams &P) { return P.geom == MUSIC_GEOM_SPHERICAL || P.conduct; }

// The vectors one GMRES solve works on.  A grid with passive scalars keeps
// a second set for the scalars' solve and swaps it in (swap_space) while that
// solve runs, so the GMRES driver and the Krylov kernels serve both.
struct KSpace {
    double *U, *RU, *b, *x, *t64;  // iterate, its operator, right-hand side, correction, scratch (FP64)
    void *V, *w, *z, *u;           // Krylov basis and work vectors (Krylov type)
    size_t n;                      // unknowns
    DevScalars *ds, *hs;           // device scalars and their pinned host mirror
};

struct music_grid {
    music_grid_desc desc;
    int stencil_variant;  // STENCIL_*: fused shared-memory kernel (2-D) or multi-pass
    int pc_variant;       // PC_*: fused 2-D preconditioner kernel or one kernel per sweep
    int solver_variant;   // SOLVER_*: device-driven graph or host-sequenced Newton/GMRES
    int stile, ptile;     // tile shapes of the fused 2-D stencil / preconditioner (indices, tiles.h)
    int rtile;            // tile shape of the stencil's R, C^n and F modes (stile: its Jv mode)
    int psplit;           // launches the fused preconditioner's sweeps are split over (1, 2 or 4)
    int btile;            // tile shape of the batched kernel (index, tiles.h)
    int jv_form;          // JV_*: form of the Krylov products of a mixed-precision grid
    int loop_cap;         // bound on the loop bodies of one Newton attempt (0: the default
                          // newton_max (restarts + 1) (m + 3) + 64, loop_cap_of)
    GridParams P;
    int mixed;
    int device;
    cudaStream_t home;  // stream of allocation, state transfer and destruction
    size_t n;         // nv * N
    size_t bytes;     // device bytes owned
    int nb;           // reduction blocks
    // FP64 state vectors
    double *U, *Un, *Cn, *RU, *b, *x, *t64, *t64b;
    // Krylov vectors (float for mixed, double otherwise)
    void *V, *w, *z, *u;
    void *q;              // copy of the current Arnoldi vector (solver graph)
    void *Z;              // preconditioned basis Z_j = M^-1 V_j (m vectors, Krylov type), or null
    // preconditioner (float for mixed, double otherwise)
    void *pa[3], *pgp, *php, *pD, *pb, *pdp, *pdq;
    void *prh, *pkf[3];    // general form: cell rho, face chi (spherical / conducting grids)
    void *pgw;             // general form: the sweeps' neighbour weights (2 nd planes)
    double *gface;         // spherical: radial gravity on the r-faces
    double *sgeo;          // spherical: the cells' metric (SG_COUNT planes of N)
    double *hg;            // Hessenberg and Givens storage of the batched solver
    void *binst;           // device copy of this grid's batched-solver descriptor
    int binst_ready;
    ExtScratch ext;
    double *partials;      // [MUSIC_MAXV][nb]
    DevScalars *ds;        // device scalars
    DevScalars *hs;        // pinned host mirror
    SolveCtl *ctl;         // device control of a graph-driven Newton attempt
    SolveCtl *hctl;        // pinned host mirror of its leading scalars
    cudaGraphExec_t gexec; // the recorded Newton attempt (null until first use)
    long long glaunch[7];  // kernels per recorded section: top, Newton iteration (with its first GMRES
                           // cycle), restarted cycle, (unused), (unused), Arnoldi step, the residual
                           // that closes a Newton iteration
    double *diag_rows;     // per-row diagnostic partials
    // passive scalars (Sec. 2.2)
    int ns;                // scalars (planes of N partial densities in sc.U)
    KSpace sc;             // the scalars' solve (swapped with the fluid's while it runs)
    int in_scalar;         // 1 while sc is swapped in
    double *sq_n, *sq_c;   // scalars at the start of the attempt, their step constant
    double *sfr;           // face mass fluxes (nd planes of N, lower faces) of the frozen fluid
    const double *srho;    // density of the frozen fluid (device, N values)
    double *fr_capture;    // when set, the stencil's non-Jv modes write their face mass fluxes here
    float *lin;            // linearisation planes (LIN_PLANES x N) of the difference-form Jv, or null
    float *linx;           // the same on the ghosted grid for the multi-pass stencil ((2+4nd+nd^2) x M), or null
    // optional timing of the main kernels by class (music_profile_*)
    int prof_on;
    int prof_pending;            // event pairs recorded, not yet harvested
    cudaEvent_t prof_ev[2 * 256];
    int prof_cls[256];           // class (MUSIC_PROF_*) of each recorded pair
    int prof_depth;              // open ProfScope nesting
    // set while the solver graph records an Arnoldi step on a grid whose
    // fused 2-D preconditioner takes the scaling of the next basis vector:
    // its input is then w * pc_scale->inv and its first stage writes
    // V[pc_scale->scale_idx] (precond_folds_scale)
    const SolveCtl *pc_scale;
    unsigned long long prof_launches[MUSIC_PROF_CLASSES];
    double prof_ms[MUSIC_PROF_CLASSES];
    int prof_events_made;
};

// record the start / end of a profiled launch; harvest completed pairs
int prof_begin_cls(music_grid *g, int cls, cudaStream_t s);  // the pair that follows is of class cls
int prof_end(music_grid *g, cudaStream_t s);
int prof_harvest(music_grid *g, int wait);
// difference-form Jv on the multi-pass stencil (jvdiff_multipass.cu): the
// linearisation arrays from the FP64 planes of the R / F evaluation just run
// at U, and the product of an FP32 direction
int lin_ext_write(music_grid *g, const double *U, cudaStream_t s);
// the spherical metric table of the grid (at creation)
int sph_geo_build(music_grid *g, cudaStream_t s);
int jvdiff_multipass(music_grid *g, const double *U, const float *v, float *out, double hdt, cudaStream_t s);
// Times the enclosing host function's launches as class cls while the grid
// is profiled (CUDA events on s around them).  Scopes do not nest: inside an
// open scope (say a norm inside a preconditioner application) the launches
// count to the outer class.
struct ProfScope {
    music_grid *g;
    cudaStream_t s;
    bool on;
    ProfScope(music_grid *g_, int cls, cudaStream_t s_) : g(g_), s(s_), on(false)
    {
        if (!g->prof_on) return;
        on = g->prof_depth == 0 && prof_begin_cls(g, cls, s) == MUSIC_OK;
        g->prof_depth++;
    }
    ~ProfScope()
    {
        if (!g->prof_on) return;
        g->prof_depth--;
        if (on) prof_end(g, s);
    }
};

// Where the Arnoldi step stores its preconditioned vector M^-1 V_j: Z, or
// null when the current solve is unpreconditioned (its Z is V itself).
inline void *krylov_zstore(const music_grid *g)
{
    return (g->desc.precond == MUSIC_PC_NONE || g->in_scalar) ? nullptr : g->Z;
}

// SMs of the part, and the most blocks a vector sweep of krylov.cu takes
// (its partials per reduced quantity): two per SM, all resident at once
constexpr int NUM_SMS = 152;
constexpr int VEC_BLOCKS_MAX = 2 * NUM_SMS;

// error reporting (thread local)
void set_error(const char *fmt, ...);
#define CUDA_TRY(call)                                                                  \
    do {                                                                                \
        cudaError_t e_ = (call);                                                        \
        if (e_ != cudaSuccess) {                                                        \
            (void)cudaGetLastError(); /* a failed call must not resurface at a later check */ \
            set_error("%s:%d %s: %s", __FILE__, __LINE__, #call, cudaGetErrorString(e_)); \
            return MUSIC_E_CUDA;                                                        \
        }                                                                               \
    } while (0)
// every kernel launch is followed by CHECK_LAUNCH, which also counts it
void count_launch();
#define CHECK_LAUNCH()               \
    do {                             \
        count_launch();              \
        CUDA_TRY(cudaGetLastError()); \
    } while (0)
#define TRY(x)                      \
    do {                            \
        int r_ = (x);               \
        if (r_ != MUSIC_OK) return r_; \
    } while (0)

// Allow a kernel `smem` bytes of dynamic shared memory on the current device,
// once per device (the attribute is per device; `done` holds one bit per
// device and may be shared by concurrent callers).
template <typename K>
int allow_dynamic_smem(K kern, size_t smem, std::atomic<uint64_t> &done)
{
    int dev = 0;
    CUDA_TRY(cudaGetDevice(&dev));
    const uint64_t bit = 1ull << (dev & 63);
    if (done.load(std::memory_order_acquire) & bit) return MUSIC_OK;
    CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    done.fetch_or(bit, std::memory_order_release);
    return MUSIC_OK;
}

// ----- stencil.cu -----
// Evaluate R at W = U (+ eps v in SM_JV) and write per `mode`.
//   U: state (device fp64); aux: C^n for SM_F, RU for SM_JV;
//   v: SM_JV input (vin_double selects its type); out: output (out_double);
//   RU_out: SM_F only, receives R(U).  eps is read from ds->eps in SM_JV.
int stencil_apply(music_grid *g, int mode, const double *U, const double *aux, const void *v,
                  int vin_double, void *out, int out_double, double *RU_out, double dt,
                  double sign, cudaStream_t s);

// ----- krylov.cu -----
// sum of squares of x (n elements) -> *dst (device), deterministic
int dev_norm2(music_grid *g, const void *x, int is_double, size_t n, double *dst, cudaStream_t s);
// *dst = sum of g->partials[0..count) in order (second stage of a reduction)
int final_sum(music_grid *g, int count, double *dst, cudaStream_t s);
// eps = sqrt(2^-52) (1 + sqrt(unorm2)) / sqrt(vnorm2), or the fixed value if > 0
int dev_set_eps(music_grid *g, double fixed, cudaStream_t s);
// the three CGS passes; jdev (device, or null) overrides j, which then bounds it
int krylov_dots(music_grid *g, int j, const int *jdev, cudaStream_t s);        // h = V[0..j]^T w; Z_j = z
int krylov_update_dots(music_grid *g, int j, const int *jdev, cudaStream_t s); // w -= V h; h2 = V^T w
// the solver graph's Arnoldi control, run by the last block of the norm pass
struct GivensCtl {
    SolveCtl *c;
    const DevScalars *ds;
    cudaGraphConditionalHandle h;  // the Arnoldi loop's condition
    int m, cap;                    // restart length, loop-body cap
};
// w -= V h2; wnorm2; with gc, then the Givens rotations of the Arnoldi step
int krylov_update_norm(music_grid *g, int j, const int *jdev, cudaStream_t s, const GivensCtl *gc = nullptr);
int krylov_scale(music_grid *g, int j, double inv, cudaStream_t s);            // V_{j+1} = w * inv
int krylov_first(music_grid *g, const double *r, double inv, cudaStream_t s);  // V_0 = r * inv
// x += sum_{i<k} y_i Z_i (Z = M^-1 V stored by krylov_dots, or V when the
// solve is unpreconditioned); kdev / ydev (device, or null) override k / y
int krylov_correct(music_grid *g, int k, const double *y, const int *kdev, const double *ydev, cudaStream_t s);
int vec_sub(music_grid *g, const double *a, const double *b, double *out, cudaStream_t s); // out = a - b
int vec_neg(music_grid *g, const double *a, double *out, cudaStream_t s);
int newton_update(music_grid *g, const int *skip, cudaStream_t s);             // U += x, maxdrho (unless *skip)
int vec_cast_copy(const void *src, int src_double, void *dst, int dst_double, size_t n, cudaStream_t s);

// ----- precond.cu -----
int precond_setup(music_grid *g, const double *U, double dt, cudaStream_t s);  // frozen coefficients
// the grid's preconditioner application is the fused 2-D kernel, which can
// take an input scale and write the scaled input (music_grid::pc_scale)
bool precond_folds_scale(const music_grid *g);
// z = M^-1 r; with want_norm also |z|^2 -> ds->vnorm2 and the Jv step
// eps(|U|, |z|) -> ds->eps
int precond_apply(music_grid *g, double dt, const void *r, void *z, int want_norm, cudaStream_t s);

// ----- diag.cu -----
int cfl_rate(music_grid *g, const double *U, cudaStream_t s);                  // -> ds->rate
// the three rates of the time-step limits at the grid's state -> ds->rate, rate_adv, rate_rad
int step_rates(music_grid *g, cudaStream_t s);
// z slabs a row of the rate reduction is split into (3-D grids: more blocks)
inline int rate_slabs(const GridParams &P) { return P.nd == 3 ? (P.n[2] < 16 ? P.n[2] : 16) : 1; }
int diagnostics(music_grid *g, const double *U, double rho_L, double rho_H, cudaStream_t s);

// ----- api.cu: grid lifetime on a given home stream (used by the server) -----
int grid_create(const music_grid_desc *desc, cudaStream_t home, music_grid **out);
void grid_destroy(music_grid *g);
int grid_footprint(const music_grid_desc *desc, size_t *bytes);
// geometry and physics of a descriptor whose defaults are filled in
void fill_grid_params(const music_grid_desc &d, GridParams *P);
// the loop-body bound of one Newton attempt (both drivers)
int loop_cap_of(const music_grid *g);
// fill in defaults and validate, allocating nothing
int grid_validate(music_grid_desc *d);
int grid_set_state(music_grid *g, const double *U, int is_device, cudaStream_t s);
int grid_get_state(music_grid *g, double *U, int is_device, cudaStream_t s);

// ----- batched.cu -----
extern "C" int music_batch_step(music_grid **grids, int count, const double *cfl, const double *dt_max,
                                music_step_stats *stats, void *stream);

// ----- scalars.cu -----
// the scalar operator in stencil_apply's modes, with the fluid frozen at
// g->srho / g->sfr (used while the scalar space is swapped in)
int scalar_apply(music_grid *g, int mode, const double *q, const double *aux, const void *v, int vin_double,
                 void *out, int out_double, double *RS_out, double dt, double sign, cudaStream_t s);
// q += x; max |x| / rho -> ds->maxdrho (scalar space swapped in)
int scalar_update(music_grid *g, cudaStream_t s);
// c_i <- c_i / sum_j c_j with the fluid density rho (device)
int scalar_renormalise(music_grid *g, const double *rho, cudaStream_t s);
// copy the multi-pass stencil's face mass fluxes to g->fr_capture
int capture_ext_fluxes(music_grid *g, cudaStream_t s);
// swap the fluid and scalar solve spaces
void swap_space(music_grid *g);

// ----- solver.cu -----
// lim (recorded-graph grids only): the first attempt's dt is chosen on the
// device from the limits, as music_select_dt would choose it; dt is then unused
int newton_solve(music_grid *g, double dt, music_step_stats *st, cudaStream_t s,
                 const music_dt_limits *lim = nullptr);
// whether newton_solve steps the grid with the recorded graph
bool graph_driven(const music_grid *g);
// J v for the current Newton iterate (eps from |U| and, with need_vnorm, |v|)
int jv_apply(music_grid *g, const void *v, int vin_double, void *out, int out_double, double dt,
             int need_vnorm, cudaStream_t s);

// ----- graph.cu -----
// One Newton attempt (Sec. 2) as a recorded CUDA graph whose Newton, restart
// and Arnoldi loops are conditional nodes driven by device-side control.
// Same arguments and results as the host-sequenced attempt.
int graph_newton_attempt(music_grid *g, double dt, music_step_stats *st, cudaStream_t s,
                         const music_dt_limits *lim = nullptr);
void graph_release(music_grid *g);

// ----- tune.cu -----
// set the grid's tile shapes from an earlier tuning of its configuration
void tune_lookup(music_grid *g);

// ----- api.cu -----
void count_launches(long long k);   // add kernels run by a graph launch
long long capture_launches();       // kernels launched by this thread so far
