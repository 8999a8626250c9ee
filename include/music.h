/*
 * libmusic - C ABI of the GB300 implicit-hydrodynamics JFNK inner loop.
 *
 * The library advances the Euler equations with gravity (paper Sec. 2,
 * Eqs. 1-3) by Crank-Nicolson implicit steps solved with Newton-Raphson,
 * restarted GMRES with Jacobian-free finite-difference matrix-vector products
 * and a physics-based semi-implicit preconditioner.  Everything on the path
 * runs as CUDA kernels on one GPU; the host code only sequences launches and
 * does the scalar Givens least-squares update of GMRES.
 *
 * Conventions shared by every call
 * --------------------------------
 *  State layout: nv planes of N = nx*ny*nz doubles, x fastest, in the order
 *    rho, E = rho e (internal energy per volume), m_x, m_y[, m_z]
 *    (nv = 2 + ndim).  m_d[c] is the momentum on the lower d-face of cell c
 *    (staggered grid, Sec. 2).  On a wall direction the lower wall face of
 *    the first layer is stored and must be 0; the upper wall face is implicit.
 *  Device pointers: every array argument documented as "device" must be a
 *    CUDA device (or managed) pointer to at least nv*N elements of the stated
 *    type, 8-byte aligned (4-byte for float).  The library never frees or
 *    retains caller pointers; they are borrowed for the duration of the call
 *    and, because work is queued asynchronously on `stream`, until the
 *    stream has passed the call.
 *  Streams: `stream` is a cudaStream_t passed as void* (NULL = the legacy
 *    default stream).  Calls queue their kernels on it and return once
 *    queued, except where a call must read a scalar result back (documented
 *    per call), in which case it synchronises `stream`.
 *  Errors: every call returns a music_status.  On failure nothing is
 *    aborted; music_last_error() gives a message for the calling thread.  A
 *    grid whose call failed with MUSIC_E_CUDA should be destroyed.
 *  Precision: MUSIC_FP64 computes everything in FP64.  MUSIC_MIXED keeps
 *    the state, the residual F(U), the finite-difference differencing
 *    U + eps v and R(U + eps v) - R(U), gravity and pressure in FP64 and
 *    stores the Krylov basis, the preconditioner and Jv results in FP32
 *    (dot products accumulate in FP64).
 *  Threads: a grid may be used by one host thread at a time.
 */
#ifndef MUSIC_H
#define MUSIC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    MUSIC_OK = 0,
    MUSIC_E_INVAL = 1,        /* bad argument or descriptor */
    MUSIC_E_OOM = 2,          /* device or host allocation failed */
    MUSIC_E_CUDA = 3,         /* a CUDA runtime call failed */
    MUSIC_E_NEWTON_FAIL = 4,  /* Newton did not converge after all dt halvings */
    MUSIC_E_GMRES_FAIL = 5,   /* reserved: GMRES non-convergence is reported in stats */
    MUSIC_E_NONFINITE = 6,    /* NaN or Inf met in a norm */
    MUSIC_E_TIMEOUT = 7,      /* a bounded wait expired */
    MUSIC_E_BUSY = 8,         /* admission refused: over the memory budget or slots full */
    MUSIC_E_NOTFOUND = 9      /* unknown ticket */
} music_status;

enum { MUSIC_BC_PERIODIC = 0, MUSIC_BC_WALL = 1 };
/* scalar ghost cells behind a wall: mirrored, or hydrostatic with the
   temperature T = (gamma-1) e extrapolated linearly and rho from the
   discrete balance p_b - p_g = -+ dx g (rho_b + rho_g)/2 (Sec. 3) */
enum { MUSIC_WALL_MIRROR = 0, MUSIC_WALL_HSE_LINEAR_T = 1 };
enum { MUSIC_FP64 = 0, MUSIC_MIXED = 1 };
enum { MUSIC_PC_NONE = 0, MUSIC_PC_ACOUSTIC = 1 };
enum { MUSIC_GEOM_CARTESIAN = 0, MUSIC_GEOM_SPHERICAL = 1 };

/* Grid, physics and solver description (copied by music_create_grid). */
typedef struct {
    int ndim;            /* 2 or 3 */
    int n[3];            /* cells per direction, n[2] = 1 when ndim = 2; each >= 4 */
    double origin[3];    /* lower corner of the box */
    double length[3];    /* box edge lengths (> 0) */
    int bc[3];           /* MUSIC_BC_* per direction */
    int wall_scalar[3];  /* MUSIC_WALL_* per wall direction; at most one HSE direction */
    double gamma;        /* ideal-gas ratio of specific heats, p = (gamma-1) E (Sec. 2) */
    double g[3];         /* constant gravitational acceleration (Sec. 2) */
    int precision;       /* MUSIC_FP64 or MUSIC_MIXED */
    /* solver options (0 selects the default in brackets) */
    int gmres_restart;        /* Krylov vectors per cycle [30], 1..63 */
    int gmres_max_restarts;   /* extra cycles [10] */
    double gmres_rtol;        /* |J d + F| <= rtol |F| [1e-1] */
    int newton_max_its;       /* [12] */
    double newton_tol;        /* converged when max |delta rho|/rho <= tol [1e-8] */
    int precond;              /* MUSIC_PC_* [ACOUSTIC]; pass -1 for NONE */
    int precond_sweeps;       /* weighted-Jacobi sweeps of the pressure system [16] */
    int max_dt_halvings;      /* retries of a failed step at dt/2 [4] */
    /* geometry and radiative diffusion (Sec. 2 Eq. 2 and the photon
       conductivity; Sec. 6) */
    int geometry;             /* MUSIC_GEOM_*; SPHERICAL is 2-D axisymmetric with
                                 direction 0 = r (walls), 1 = theta, origin and
                                 length in (r, theta) */
    const double *g_radial;   /* SPHERICAL: host array of the radial gravity on the
                                 n[0]+1 r-faces (copied at creation); NULL: g[0] */
    int conduct;              /* 1: add div(chi grad T), T = (gamma-1) e,
                                 chi = chi0 T^6.5 / rho^2 (Kramers opacity) */
    double chi0;
    int flux_wall[3];         /* 1: this direction's wall faces carry the prescribed
                                 chi dT/dn = lum (spherical r-walls: lum / r^2) */
    double lum;
    /* passive scalars (Sec. 2.2), Cartesian grids */
    int nscalars;             /* scalars carried as partial densities c_i rho, 0..8 [0] */
    int scalar_enforce;       /* 1: the Newton test also requires max |delta(c_i rho)| / rho
                                 <= newton_tol; 0: the density test alone (Sec. 2.2) [0] */
    /* time-step limits music_newton_step applies (Sec. 2, choice of the time
       step; the rates are those of music_select_dt; each <= 0 is not applied,
       and a grid with none takes the caller's dt_max as its step) */
    double cfl_hydro;         /* CFL_hydro: dt <= cfl_hydro / max (|u_d| + c_s) / h_d (Eq. 4) */
    double cfl_adv;           /* CFL_adv:   dt <= cfl_adv / max |u_d| / h_d */
    double cfl_rad;           /* CFL_rad:   dt <= cfl_rad / max D / h_d^2 (radiative diffusion) */
} music_grid_desc;

typedef struct {
    double dt;          /* step size actually taken */
    int newton_its;     /* Newton iterations of the accepted attempt */
    int gmres_its;      /* Arnoldi steps of the accepted attempt */
    int dt_halvings;    /* failed attempts before it */
    int gmres_unconverged; /* GMRES solves that hit the restart limit */
    double fnorm0;      /* |F(U^n)|_2 at the first Newton iterate */
    double fnorm;       /* |F|_2 at the last Newton iterate */
    double max_drho;    /* final max |delta rho| / rho */
    double wall_ms;     /* host wall time of the call */
    int scalar_gmres_its;  /* Arnoldi steps of the passive-scalar solves */
    int pad;
} music_step_stats;

typedef struct music_grid music_grid;

/* Service calls (the paper has no counterpart).
   Message of the last failed call on this thread (always NUL-terminated).
   Returns the full message length. */
size_t music_last_error(char *buf, size_t len);

/* Library version string. */
const char *music_version(void);

/* Number of CUDA kernels this library has launched in this process (all
   grids, all threads).  For accounting only. */
uint64_t music_kernel_launches(void);

/*
 * Create a grid: the discretised problem of Sec. 2 (Eqs. 1-3 on the
 * staggered grid, Crank-Nicolson in time) with the boundaries of Secs. 3-6
 * and the solver settings of Sec. 2 that `desc` gives.  Validates `desc`,
 * selects the current CUDA device, and
 * allocates and owns every device buffer the solver needs (state, step
 * constant, Krylov basis, preconditioner coefficients and scratch).  The
 * state starts at zero; set it with music_set_state.  Sizes: periodic
 * directions with the acoustic preconditioner need no parity constraint.
 * Errors: MUSIC_E_INVAL (descriptor), MUSIC_E_OOM, MUSIC_E_CUDA.
 */
int music_create_grid(const music_grid_desc *desc, music_grid **out);

/* Memory management of a grid (no counterpart in the paper).
   Free everything owned by the grid.  NULL is accepted.  Synchronises the
   device first (the caller may still have work using the grid queued on
   other streams). */
int music_destroy_grid(music_grid *grid);

/* Device bytes music_create_grid would allocate for `desc` (nothing is
   allocated).  Errors: MUSIC_E_INVAL for an invalid descriptor. */
int music_grid_footprint(const music_grid_desc *desc, size_t *bytes);

/* Number of state values nv*N of the grid, or 0 for NULL. */
size_t music_state_size(const music_grid *grid);

/* Device bytes owned by the grid. */
size_t music_grid_bytes(const music_grid *grid);

/* Copy a state (the conserved variables of Eqs. 1-3 in the staggered layout
   of Sec. 2, described above) into / out of the grid.  `is_device` says
   whether `U` is a device pointer (else host).  Synchronous: waits for all
   work on the device first, then copies. */
int music_set_state(music_grid *grid, const double *U, int is_device);
int music_get_state(music_grid *grid, double *U, int is_device);

/*
 * R = R(U): the spatial operator of Eqs. 1-3 on the staggered grid with
 * van Leer limited upstream reconstruction (Sec. 2), ghost cells from the
 * grid's boundary conditions.  U, R: device, float64, nv*N.  Async on
 * `stream`.  Wall faces get R = 0.
 */
int music_spatial_operator(music_grid *grid, const double *U, double *R, void *stream);

/*
 * F = U - U^n - dt/2 (R(U) + R(U^n)): the Crank-Nicolson residual (Sec. 2).
 * U, Un, F: device, float64, nv*N.  Evaluates two stencils.  Async.
 */
int music_residual(music_grid *grid, const double *U, const double *Un, double dt, double *F,
                   void *stream);

/*
 * Jv = v - dt/2 (R(U + eps v) - R(U)) / eps, the Jacobian-free product of the
 * Crank-Nicolson Jacobian (Knoll & Keyes 2004, cited in Sec. 2).  eps <= 0
 * selects eps = sqrt(2^-52) (1 + |U|_2) / |v|_2 (computed on the device);
 * v = 0 gives Jv = 0.  U: device float64.  v, Jv: device, float64 for
 * MUSIC_FP64 grids and float32 for MUSIC_MIXED grids.  On MUSIC_FP64 grids
 * U + eps v and the difference of the two residuals are formed in FP64; on
 * MUSIC_MIXED grids the form is the grid's Jv form (music_set_jv_form).
 * Async.
 */
int music_jv(music_grid *grid, const double *U, const void *v, void *Jv, double dt, double eps,
             void *stream);

/*
 * z = M^-1 r, the physics-based preconditioner (Sec. 2, after Park et al.
 * 2009) with coefficients frozen at U: the acoustic subsystem (advection and
 * gravity dropped) with the momentum eliminated into a pressure Helmholtz
 * problem, relaxed with `precond_sweeps` weighted-Jacobi sweeps (weight 0.8)
 * from zero, then density, energy and momentum by back substitution in flux
 * form.  MUSIC_PC_NONE is the identity.  U: device float64; r, z: device,
 * float64 (FP64 grids) or float32 (MIXED grids).  Async.
 */
int music_precond_apply(music_grid *grid, const double *U, double dt, const void *r, void *z,
                        void *stream);

/*
 * Advance the grid's own state by one implicit step: Newton on the
 * Crank-Nicolson system (Sec. 2) with right-preconditioned restarted GMRES.
 * The step size is chosen from the state at the start of the step: the most
 * restrictive of the grid's time-step limits (desc.cfl_hydro, cfl_adv,
 * cfl_rad, reduced on the device as in music_select_dt) and of dt_max when
 * dt_max > 0; a grid created without limits takes dt_max (> 0 then) as the
 * step.  A failed Newton solve is retried at dt/2 up to max_dt_halvings
 * times.  `st` (may be NULL) receives the step actually taken and the
 * iteration counts.  Synchronises `stream` (it reads the step size and the
 * outcome back; with the default driver the Newton and GMRES loops run on
 * the device in a recorded CUDA graph with no other host round trip).
 * Errors: MUSIC_E_INVAL (no limit and dt_max <= 0, or no limit applies),
 * MUSIC_E_NEWTON_FAIL (state restored to U^n), MUSIC_E_TIMEOUT (the bound on
 * loop bodies of an attempt was reached; state restored to U^n),
 * MUSIC_E_NONFINITE, MUSIC_E_CUDA.
 */
int music_newton_step(music_grid *grid, double dt_max, music_step_stats *st, void *stream);

/*
 * Advance `count` grids (1..512) by one implicit step each in ONE kernel
 * launch: every grid's step (CFL time step of Eq. 4 from its own state with
 * cfl[i], capped by dt_max[i] > 0 (dt_max may be NULL); Newton on the
 * Crank-Nicolson system; restarted
 * right-preconditioned GMRES with Jacobian-free products; dt halvings on
 * failure) runs in one CTA on the device with no host synchronisation, using
 * the grid's own buffers.  Meant for many small grids, which cannot fill the
 * GPU one at a time.  Every grid must be 2-D Cartesian without radiative
 * diffusion, use at most 24 preconditioner sweeps in mixed precision (16 in
 * FP64, whose planes of a deeper halo exceed shared memory), and all must
 * share one precision.  stats[i] (may be NULL) receives grid i's outcome.  Synchronises
 * `stream`.  Returns MUSIC_OK, or the first failing grid's status (its state
 * is restored to the start of the step); MUSIC_E_INVAL for a bad batch.
 */
int music_batch_step(music_grid **grids, int count, const double *cfl, const double *dt_max,
                     music_step_stats *stats, void *stream);

/*
 * Tile shapes of the fused 2-D kernels (the residual / Jacobian-free product
 * stencil of Sec. 2 and the physics-based preconditioner) and the halo depth
 * of the preconditioner (its K sweeps in 1, 2, 3 or 4 launches, halo K/stages +
 * 1), picked by timing.  The paper has no counterpart: its code ran on CPUs.
 * Every candidate gives bitwise identical results, so tuning changes speed
 * only.
 */
typedef struct {
    int tunable;              /* 0: the grid has no fused 2-D kernels (3-D, spherical, radiative
                                 diffusion, or the multi-pass stencil); nothing was timed */
    int from_cache;           /* 1: the shapes came from an earlier tuning of the same
                                 configuration in this process; nothing was timed */
    int stencil_tile[2];      /* chosen (TX, TY) of the stencil */
    int precond_tile[2];      /* chosen (TX, TY) of the preconditioner */
    int precond_stages;       /* chosen number of launches of its sweeps */
    int n_stencil, n_precond; /* candidates timed (0 when not timed) */
    int stencil_cand[8][2];   /* candidate (TX, TY) ... */
    int precond_cand[24][3];  /* candidate (TX, TY, stages) ... */
    double stencil_us[8];     /* ... and their median times in microseconds (stencil:
                                 one Jacobian-free product; preconditioner: all its launches) */
    double precond_us[24];
    int residual_tile[2];     /* chosen (TX, TY) of the stencil's R, C^n and F modes, timed as
                                 one F evaluation on the same candidates as the stencil */
    double residual_us[8];
    int batch_tile[2];        /* chosen (TX, TY) of the persistent batched kernel
                                 (music_batch_step), timed with MUSIC_TUNE_BATCH as one batched
                                 step of this grid alone, for grids of at most 65536 cells that
                                 it accepts */
    int n_batch, pad;         /* its candidates timed (0 when not timed) */
    int batch_cand[4][2];     /* candidate (TX, TY) ... */
    double batch_us[4];       /* ... and their median times in microseconds */
} music_tune_report;

#define MUSIC_TUNE_FORCE 1u   /* time the candidates even when the configuration is cached */
#define MUSIC_TUNE_BATCH 2u   /* also time the persistent batched kernel's tile shapes (grids of
                                 at most 65536 cells that music_batch_step accepts) */

/*
 * Autotuner (no counterpart in the paper: a choice of GPU tiling that
 * changes no result, every shape giving the same bits).
 * Time every candidate tile shape of the grid's fused 2-D kernels on its
 * current state at step size dt (> 0), keep the fastest for this grid, and
 * remember them for the configuration (extent, boundaries, precision,
 * preconditioner and sweeps): grids created later with the same
 * configuration start with these shapes.  Overwrites the grid's solver
 * scratch buffers (the state is unchanged).  Synchronises `stream`.
 * The environment variable MUSIC_TILES=<Jv>,<residual>,<preconditioner>,
 * <stages> (e.g. 32x16,16x16,64x16,1) pins the choice without timing when
 * it names valid candidates for the grid (a profiler slows every launch, so
 * timings taken under one are meaningless); the report's timings are then 0.
 * Errors: MUSIC_E_INVAL, MUSIC_E_CUDA.
 */
int music_autotune(music_grid *grid, double dt, unsigned flags, music_tune_report *report, void *stream);

/* (No counterpart in the paper, as for music_autotune.)
   Set the fused kernels' tile shapes to given candidates ((TX, TY) pairs;
   NULL keeps that kernel's shape; stencil_tile sets the stencil's Jv mode
   and its R / C^n / F modes alike) and the preconditioner's stage count (1, 2
   or 4; <= 0 keeps it).  MUSIC_E_INVAL for a shape that is not a candidate
   or a split that leaves more than 8 sweeps per stage.  music_get_tiles
   reads the current choice. */
int music_set_tiles(music_grid *grid, const int *stencil_tile, const int *precond_tile, int precond_stages);
int music_get_tiles(const music_grid *grid, int *stencil_tile, int *precond_tile, int *precond_stages);

/* (No counterpart in the paper, as for music_autotune.)
   Tile shape (TX, TY) of the persistent batched kernel for this grid: one of
   32 x 16, 16 x 32, 64 x 8 (a CTA of 512 threads each, so every shape gives
   bitwise the same step).  music_batch_step runs a batch with the shape of
   its first grid; music_autotune picks it by timing for small grids.
   MUSIC_E_INVAL for a shape that is not a candidate. */
int music_set_batch_tile(music_grid *grid, const int *tile);
int music_get_batch_tile(const music_grid *grid, int *tile);

/*
 * Form of the Jacobian-free product of a MUSIC_MIXED grid (Sec. 2; used by
 * music_jv and by the Arnoldi products of music_newton_step).
 *   MUSIC_JV_FD64:   R(U + eps v) and R(U) evaluated in FP64 and subtracted.
 *   MUSIC_JV_DIFF32: the same finite difference (same eps; every upwind and
 *                    limiter branch taken at U and at U + eps v) computed in
 *                    difference form: each intermediate's scaled difference
 *                    (x(U + eps v) - x(U)) / eps is carried through exact
 *                    sum, product, quotient and limiter identities in FP32,
 *                    and only the neighbour differences at U that decide the
 *                    limiter are formed in FP64.  No two nearly equal
 *                    residuals are subtracted, so FP32 rounding stays
 *                    relative to the product itself.  The default of mixed
 *                    grids.
 * The difference form covers Cartesian grids without radiative diffusion
 * (2-D on the fused stencil, 3-D and 2-D on the multi-pass stencil);
 * spherical and conducting grids, and products of FP64 vectors (the GMRES
 * restart residual), use the FP64 form whatever is set.
 * MUSIC_E_INVAL for an unknown form or MUSIC_JV_DIFF32 on a MUSIC_FP64 grid.
 * The environment variable MUSIC_JV=fd makes new mixed grids start with
 * MUSIC_JV_FD64.  music_get_jv_form reads the setting.
 */
#define MUSIC_JV_FD64 0
#define MUSIC_JV_DIFF32 1
int music_set_jv_form(music_grid *grid, int form);
int music_get_jv_form(const music_grid *grid, int *form);

/*
 * Passive scalars (Sec. 2.2).  A grid created with nscalars > 0 carries
 * their partial densities q_i = c_i rho (nscalars planes of N values, the
 * layout of the state's planes) next to the fluid state; they start at
 * zero.  music_newton_step then also advances them: every Newton iteration
 * solves the scalars' Crank-Nicolson system d q_i/dt = -div(c_i rho u) by an
 * unpreconditioned Jacobian-free Newton-Krylov step with the fluid frozen at
 * that iteration's fluid iterate (face mass flux times c_i reconstructed
 * upwind with the van Leer limiter); the loop stops on the fluid's density
 * test (and on the scalar corrections with scalar_enforce); after the step
 * the concentrations are renormalised to sum to one.  The fluid is advanced
 * exactly as without scalars.  Pointers as for music_set_state.
 */
int music_set_scalars(music_grid *grid, const double *q, int is_device, void *stream);
int music_get_scalars(music_grid *grid, double *q, int is_device, void *stream);

/* The passive scalars' operator (Sec. 2.2): S_i = -div(c_i rho u) of device
   partial densities q (nscalars planes) with the fluid frozen at the device
   state U, c_i reconstructed upwind with the van Leer limiter; S device,
   same layout.  Errors: MUSIC_E_INVAL (no scalars, NULL), MUSIC_E_CUDA. */
int music_scalar_operator(music_grid *grid, const double *U, const double *q, double *S, void *stream);

/* Mixing width of Sec. 3 from the grid's first two scalars and state:
   h = sum over rows of 2 min(<c_1>, <c_2>) dy, <.> the mean of a row of
   cells normal to direction 1.  Synchronises `stream`. */
int music_scalar_mixing_width(music_grid *grid, double *h, void *stream);

/*
 * Time-step limits (Sec. 2, choice of the time step).  Each limit <= 0 is
 * not applied; the step is the most restrictive of the others:
 *   cfl_hydro / max (|u_d| + c_s) / h_d     (Eq. 4),
 *   cfl_adv   / max |u_d| / h_d             (the paper caps it at 0.5),
 *   cfl_rad   / max D / h_d^2               (radiative diffusion grids,
 *                                            D = chi / (rho c_v)),
 *   dt_max,
 * maxima over cells and directions of the grid's state, u_d the mean of the
 * cell's two face velocities, h_d the distance between cell centres (dr, or
 * r_c dtheta on spherical grids).  *which (may be NULL) receives 0, 1, 2 or 3
 * for the limit that applied.  Synchronises `stream`.  Errors: MUSIC_E_INVAL
 * (no limit applies), MUSIC_E_NONFINITE.
 */
typedef struct {
    double cfl_hydro, cfl_adv, cfl_rad, dt_max;
} music_dt_limits;
int music_select_dt(music_grid *grid, const music_dt_limits *limits, double *dt, int *which, void *stream);

/*
 * Grid-convergence measure of Sec. 4 between two 2-D grids of the same box
 * whose extents differ by an integer factor r (fine = r x coarse): the
 * vertical velocity on the y-faces (m_y over the mean density of the two
 * cells), the fine one coarsened by averaging the r fine faces that tile each
 * coarse face, and *err = sum |v_coarse - v_fine coarsened| / sum |v_fine
 * coarsened|.  Reads both grids' states; synchronises `stream`.
 */
int music_velocity_error(music_grid *fine, music_grid *coarse, double *err, void *stream);

/* dt = cfl / max_cells,d ((|u_d| + c_s) / dx_d) of the grid's state, with
   u_d the mean of the two face velocities of the cell (Eq. 4).
   Synchronises `stream`. */
int music_cfl_dt(music_grid *grid, double cfl, double *dt, void *stream);

/*
 * Allocation-free CFL rate, for callers that cannot allocate device memory:
 * code running inside another framework's memory pool or custom allocator
 * (which forbids cudaMalloc behind its back), embedded drivers and real-time
 * loops that must never block in the allocator, and code that may run while
 * the device is nearly full.  The paper has no counterpart: it is a service
 * variant of the reduction behind music_cfl_dt that needs no music_grid.
 *
 * Writes into *rate the same rate music_cfl_dt divides by: the maximum over
 * cells and directions of (|u_d| + c_s) / h_d, u_d the mean of the cell's two
 * face velocities and h_d the cell spacing along d (dx_d on Cartesian grids;
 * dr radially and r_c dtheta tangentially on spherical grids); a caller
 * takes dt = cfl / rate.  U: device, float64, nv*N in the layout above;
 * rate: device pointer to one double.  Async on `stream`; it allocates
 * nothing: its scratch is a fixed device array inside the library, sized for
 * grids of at most 16384 rows (n[1]), held by every GPU that loads the
 * library until the process exits.  The first call on each device looks up
 * that array's address; make it before any stream capture.  Calls whose work
 * overlaps on the GPU (other streams, other threads) share the array and
 * race; serialise them.
 * The result stays on the device, so the call cannot inspect it: a state with
 * a NaN anywhere gives *rate = NaN and a state with no sound speed and no
 * motion gives 0, both with MUSIC_OK (music_cfl_dt reports both as
 * MUSIC_E_NONFINITE).  Test *rate before dividing by it.
 * Errors: MUSIC_E_INVAL (bad descriptor or pointers, n[1] > 16384),
 * MUSIC_E_CUDA.
 */
int music_cfl_rate_noalloc(const music_grid_desc *desc, const double *U, double *rate, void *stream);

/*
 * Diagnostics of the grid's state (Secs. 3-6), written to out[0..5]:
 *  0 mixing-layer height h = sum_rows X_M(<X_H>) dy with
 *    X_H = (rho - rho_L)/(rho_H - rho_L) (Cabot & Cook, Sec. 3);
 *  1 max Mach number (cell-centred velocity);
 *  2 amplitude of the two-wavelength x-mode of v_y: (2/N)|sum v e^{-ikx}|;
 *  3 vertical kinetic energy sum_{y-faces} rbar v^2 / 2 dV;
 *  4 mean kinetic energy density (1/N) sum_d sum_faces rbar u_d^2 / 2 (Sec. 5);
 *  5 max cell-centred speed (Sec. 6).
 * Synchronises `stream`.
 */
int music_diagnostics(music_grid *grid, double rho_L, double rho_H, double *out, void *stream);

/*
 * Timing of the step's main kernels: while enabled, every launch of one of
 * them is bracketed by CUDA events on the stream it is launched on, by
 * class:
 *   MUSIC_PROF_JV        the Jacobian-free product (Sec. 2), in either form;
 *   MUSIC_PROF_PRECOND   one application z = M^-1 r of the preconditioner
 *                        (all its launches);
 *   MUSIC_PROF_RESIDUAL  the stencil's other modes: R(U), the step constant
 *                        and the Crank-Nicolson residual F(U);
 *   MUSIC_PROF_VECTOR    the vector, reduction and set-up kernels of GMRES
 *                        and Newton (CGS passes, norms, the Newton update,
 *                        the preconditioner's coefficients).
 * music_profile_read_class returns the number of such launches of a class
 * and their summed device time since the last enable (it waits for
 * recorded launches to finish); music_profile_read reads MUSIC_PROF_JV.
 * Enabling resets the counters.  Off by default; costs two event records
 * per launch, and a profiled grid steps with the host-sequenced driver.
 */
#define MUSIC_PROF_JV 0
#define MUSIC_PROF_PRECOND 1
#define MUSIC_PROF_RESIDUAL 2
#define MUSIC_PROF_VECTOR 3
#define MUSIC_PROF_CLASSES 4
int music_profile_enable(music_grid *grid, int on);
int music_profile_read(music_grid *grid, uint64_t *launches, double *ms);
int music_profile_read_class(music_grid *grid, int cls, uint64_t *launches, double *ms);

/*
 * s[i] = the van Leer slope of Sec. 2 of the one-sided differences a[i] and
 * b[i] as the FP64 stencils compute it: 2ab / (a + b) where a b > 0, else
 * 0, with the quotient from one third-order Newton step for the reciprocal
 * of a + b from a single-precision estimate (within 2 ulp of the correctly
 * rounded (2a b) / (a + b)); a + b beyond 2^+-120, subnormal, infinite or
 * NaN takes the IEEE division.  It exists so that a test can hold that
 * bound against the host's arithmetic.  a, b, s: device arrays of `count`
 * doubles (the caller owns them; s may alias neither input).  Asynchronous
 * on `stream`.  Errors: MUSIC_E_INVAL (count < 0, or a NULL array with
 * count > 0), MUSIC_E_CUDA.
 */
int music_vanleer_slopes(const double *a, const double *b, double *s, long long count, void *stream);

/*
 * q[i] = n[i] / d[i] as the FP64 stencils form the quotients they stage:
 * the specific internal energy e = E / rho and the face velocities
 * u_d = m_d / rbar of Sec. 2's staggered grid (rbar the mean density of the
 * face's two cells).  The same third-order Newton step for the reciprocal
 * of d from a single-precision estimate as music_vanleer_slopes, without
 * the factor 2: within 2 ulp of the correctly rounded n / d; d beyond
 * 2^+-120, zero, subnormal, infinite or NaN takes the IEEE division.  It
 * exists so that a test can hold that bound against the host's arithmetic.
 * n, d, q: device arrays of `count` doubles (the caller owns them; q may
 * alias neither input).  Asynchronous on `stream`.  Errors: MUSIC_E_INVAL
 * (count < 0, or a NULL array with count > 0), MUSIC_E_CUDA.
 */
int music_stencil_quotients(const double *n, const double *d, double *q, long long count, void *stream);

/*
 * Measured arithmetic ceilings of the current device: FP64 and FP32 fused
 * multiply-add throughput (2 flops each) and FP64 division throughput, each
 * the best of five launches of 8 resident blocks per SM, every thread running
 * 8 independent dependency chains.  The paper has no counterpart (it reports
 * no hardware figures); the library uses none of these numbers itself.  They
 * are the denominators that the FP64-bound stencil and the FP32 kernels are
 * compared with.  Allocates a scratch buffer of 2 KB per SM, takes about
 * 50 ms, synchronises `stream`.  Errors: MUSIC_E_INVAL (NULL), MUSIC_E_CUDA.
 */
typedef struct {
    double fp64_fma_tflops;   /* FP64 FMA, 10^12 flop/s */
    double fp32_fma_tflops;   /* FP32 FMA, 10^12 flop/s */
    double fp64_div_gops;     /* FP64 IEEE divisions, 10^9 per second */
    int sms;                  /* streaming multiprocessors of the device */
    int pad;
} music_peaks;
int music_measure_peaks(music_peaks *out, void *stream);

#ifdef __cplusplus
}
#endif
#endif /* MUSIC_H */
