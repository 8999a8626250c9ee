/*
 * ORACLE - TEST INFRASTRUCTURE ONLY.
 *
 * A plain, slow, FP64 CPU restatement of the implicit time step of the MUSIC
 * code as the paper describes it (Sec. 2): the Euler equations with gravity
 * (Eqs. 1-3) on a staggered grid with upstream linear reconstruction and the
 * van Leer limiter, Crank-Nicolson in time, Newton-Raphson on the resulting
 * non-linear system, restarted GMRES (Saad & Schultz 1986) with Jacobian-free
 * matrix-vector products (Knoll & Keyes 2004) and a physics-based
 * semi-implicit preconditioner (after Park et al. 2009), and the CFL time step
 * of Sec. 2.1 (Eq. 4).
 *
 * Only the tests, the smoke check and the benchmark's CPU baseline may load
 * this file.  It shares no code with the CUDA library and must never be
 * linked into it.  Compiled with -O2 -ffp-contract=off (no fast-math): every
 * operation is the IEEE operation written here.
 *
 * Readings of points the paper leaves open (each one is also listed in the
 * design notes of the repository):
 *  - unknowns: rho and E = rho e at cell centres, momentum m_d on d-faces;
 *    face velocity u_d = m_d / (arithmetic mean of the two adjacent rho);
 *  - fluxes: mass flux = u_face * rho*, rho* from the upwind cell with a van
 *    Leer limited slope; energy flux = mass flux * e*; momentum fluxes use the
 *    mean of the two neighbouring mass fluxes times the upwind reconstructed
 *    velocity; pressure gradient and gravity act on faces, p div(u) on cells;
 *  - van Leer slope vL(a, b) = 2ab/(a+b) if ab > 0 else 0; upwind on u >= 0;
 *  - walls: no flux through the wall face, normal velocity odd and tangential
 *    velocity even (stress-free) across it; scalar ghosts either mirrored or
 *    hydrostatic (linearly extrapolated T, rho from the discrete balance);
 *  - Crank-Nicolson: F(U) = U - U^n - dt/2 (R(U) + R(U^n));
 *  - Jv = v - dt/2 (R(U + eps v) - R(U)) / eps with
 *    eps = sqrt(2^-52) (1 + |U|_2) / |v|_2;
 *  - GMRES right preconditioned, classical Gram-Schmidt with one
 *    re-orthogonalisation, Givens least squares, x0 = 0;
 *  - preconditioner: frozen coefficients, advection and gravity dropped,
 *    momentum eliminated into the energy equation, the resulting pressure
 *    Helmholtz problem relaxed with a fixed number of weighted Jacobi sweeps
 *    from zero, then back substitution in flux form;
 *  - Newton stops when max |delta rho| / rho <= tol (at least one iteration);
 *  - dt = CFL / max_cells,d ((|u_d| + c_s) / dx_d) with cell-centred u_d.
 */
#include <complex.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>

/* Loops over independent cells, points or vector entries carry OR_PAR.  The
 * oracle as tested is serial; built with -fopenmp (the multi-core CPU
 * baseline only) these loops are split over threads.  No sum, norm, maximum
 * or dot product is ever split, so both builds produce the same bits. */
#ifdef _OPENMP
#include <omp.h>
#define OR_PAR _Pragma("omp parallel for schedule(static)")
#else
#define OR_PAR
#endif

/* threads the OR_PAR loops use (1 in the serial build) */
int or_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

void or_set_threads(int n)
{
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}

#define OR_BC_PERIODIC 0
#define OR_BC_WALL 1
#define OR_WALL_MIRROR 0
#define OR_WALL_HSE 1
#define OR_PC_NONE 0
#define OR_PC_ACOUSTIC 1
#define OR_GHOST 3
#define OR_JACOBI_OMEGA 0.8
#define OR_GEOM_CARTESIAN 0
#define OR_GEOM_SPHERICAL 1   /* 2-D axisymmetric: direction 0 = r, 1 = theta */

typedef struct {
    int nd;              /* 2 or 3 */
    int n[3];            /* cells per direction (n[2] = 1 in 2-D) */
    double dx[3];        /* cell widths */
    double x0[3];        /* lower corner of the box */
    int bc[3];           /* OR_BC_* per direction */
    int wall_scalar[3];  /* OR_WALL_* per wall direction */
    double gamma;
    double g[3];         /* constant gravitational acceleration */
    /* solver options */
    int restart;         /* GMRES restart length m */
    int max_restarts;    /* restarts after the first cycle */
    double gmres_rtol;   /* linear forcing term eta */
    int newton_max;      /* Newton iterations before the step fails */
    double newton_tol;   /* max |delta rho|/rho */
    int precond;         /* OR_PC_* */
    int sweeps;          /* weighted Jacobi sweeps of the pressure system */
    int max_halvings;    /* dt halvings after a failed Newton solve */
    /* geometry and radiative diffusion (Sec. 2 Eqs. 2 and 4, Sec. 6) */
    int geom;            /* OR_GEOM_* */
    const double *gface; /* spherical: radial gravity on the n[0]+1 r-faces, else NULL */
    int conduct;         /* add div(chi grad T), chi = chi0 T^6.5 / rho^2 */
    double chi0;         /* 16 sigma / (3 kappa0) of the Kramers-law opacity */
    int flux_wall[3];    /* wall faces carry the prescribed chi dT/dn = lum (/ r^2 if spherical) */
    double lum;
} or_grid;

typedef struct {
    double dt;
    int newton_its;
    int gmres_its;
    int halvings;
    int gmres_failures;
    double fnorm0;       /* |F| at the first Newton iterate */
    double fnorm;        /* |F| at the last Newton iterate */
    double max_drho;     /* last max |delta rho|/rho */
} or_step_stats;

static long or_ncells(const or_grid *g) { return (long)g->n[0] * g->n[1] * g->n[2]; }
static int or_nvars(const or_grid *g) { return 2 + g->nd; }

/* ---------------- extended (ghosted) index space ---------------- */
typedef struct {
    int lo[3], ne[3];
    long stride[3];
    long total;
} or_ext;

static void or_ext_init(or_ext *X, const or_grid *g)
{
    for (int d = 0; d < 3; d++) {
        if (d < g->nd) {
            X->lo[d] = -OR_GHOST;
            X->ne[d] = g->n[d] + 2 * OR_GHOST;
        } else {
            X->lo[d] = 0;
            X->ne[d] = 1;
        }
    }
    X->stride[0] = 1;
    X->stride[1] = X->ne[0];
    X->stride[2] = (long)X->ne[0] * X->ne[1];
    X->total = X->stride[2] * X->ne[2];
}

static long or_ext_index(const or_ext *X, const int ix[3])
{
    return (ix[0] - X->lo[0]) + X->stride[1] * (ix[1] - X->lo[1]) + X->stride[2] * (ix[2] - X->lo[2]);
}

static void or_ext_coords(const or_ext *X, long x, int ix[3])
{
    ix[0] = (int)(x % X->ne[0]) + X->lo[0];
    ix[1] = (int)((x / X->ne[0]) % X->ne[1]) + X->lo[1];
    ix[2] = (int)(x / X->stride[2]) + X->lo[2];
}

static int or_ext_has(const or_ext *X, const int ix[3], int d, int off)
{
    int a = ix[d] + off - X->lo[d];
    return a >= 0 && a < X->ne[d];
}

static long or_ext_of_cell(const or_ext *X, const or_grid *g, long c)
{
    int ix[3];
    ix[0] = (int)(c % g->n[0]);
    ix[1] = (int)((c / g->n[0]) % g->n[1]);
    ix[2] = (int)(c / ((long)g->n[0] * g->n[1]));
    return or_ext_index(X, ix);
}

/* ---------------- spherical (r, theta) metric, 2 pi dropped throughout ---------------- */
static double or_r(const or_grid *g, double i) { return g->x0[0] + i * g->dx[0]; }
static double or_th(const or_grid *g, double j) { return g->x0[1] + j * g->dx[1]; }

/* volume of cell (i, j) */
static double or_sph_vol(const or_grid *g, int i, int j)
{
    double ra = or_r(g, i), rb = or_r(g, i + 1);
    return (rb * rb * rb - ra * ra * ra) / 3.0 * (cos(or_th(g, j)) - cos(or_th(g, j + 1)));
}

/* area of the lower d-face of cell (i, j) */
static double or_sph_area(const or_grid *g, int d, int i, int j)
{
    if (d == 0) {
        double r = or_r(g, i);
        return r * r * (cos(or_th(g, j)) - cos(or_th(g, j + 1)));
    }
    double ra = or_r(g, i), rb = or_r(g, i + 1);
    return 0.5 * (rb * rb - ra * ra) * sin(or_th(g, j));
}

/* distance between the centres of the two cells that share the lower d-face
   of cell (i, j): dr, or the arc r_c dtheta at the cell-centre radius */
static double or_sph_h(const or_grid *g, int d, int i)
{
    return d == 0 ? g->dx[0] : or_r(g, i + 0.5) * g->dx[1];
}

/* radial gravity on r-face i (spherical), or the constant component */
static double or_gface(const or_grid *g, int d, int i)
{
    if (g->geom == OR_GEOM_SPHERICAL && d == 0 && g->gface) return g->gface[i];
    return g->g[d];
}

/* ---------------- R(U): real and complex-step instantiations ---------------- */
#define FN2(a, b) a##b
#define FN1(a, b) FN2(a, b)

#define T double
#define RE(x) (x)
#define SQRT(x) sqrt(x)
#define TABS(x) fabs(x)
#define FN(name) FN1(name, _r)
#include "residual_body.h"
#undef T
#undef RE
#undef SQRT
#undef TABS
#undef FN

#define T double complex
#define RE(x) creal(x)
#define SQRT(x) csqrt(x)
#define TABS(x) cabs(x)
#define FN(name) FN1(name, _c)
#include "residual_body.h"
#undef T
#undef RE
#undef SQRT
#undef TABS
#undef FN

/* Eqs. 1-3: R(U) (spatial operator, no time discretisation). */
void or_spatial_operator(const or_grid *g, const double *U, double *R)
{
    spatial_operator_r(g, U, R);
}

/* R(U), and per cell and variable the sum of the magnitudes of the terms R
 * adds there (fluxes over the cell's faces, pressure work and gradient,
 * gravity and, on spherical grids, the curvature terms, each with its
 * geometric weight): the scale of R's rounding, for per-cell tolerances. */
void or_spatial_operator_terms(const or_grid *g, const double *U, double *R, double *A)
{
    spatial_operator_f_r(g, U, R, NULL, A);
}

/* Exact directional derivative dR = (dR/dU) V by complex-step
 * differentiation: Im R(U + i h V) / h with h = 1e-30. */
void or_spatial_operator_dir(const or_grid *g, const double *U, const double *V, double *dR)
{
    const long n = (long)or_nvars(g) * or_ncells(g);
    const double h = 1e-30;
    double complex *Uc = (double complex *)malloc(n * sizeof(double complex));
    double complex *Rc = (double complex *)malloc(n * sizeof(double complex));
        for (long i = 0; i < n; i++) Uc[i] = U[i] + I * (h * V[i]);
    spatial_operator_c(g, Uc, Rc);
        for (long i = 0; i < n; i++) dR[i] = cimag(Rc[i]) / h;
    free(Uc);
    free(Rc);
}

/* ---------------- vector helpers (fixed summation order) ---------------- */
static double or_dot(long n, const double *a, const double *b)
{
    double s = 0.0;
    for (long i = 0; i < n; i++) s += a[i] * b[i];
    return s;
}

static double or_norm(long n, const double *a) { return sqrt(or_dot(n, a, a)); }

double or_norm2(long n, const double *a) { return or_norm(n, a); }

/* ---------------- Crank-Nicolson residual (Sec. 2) ---------------- */
/* F(U) = U - C^n - dt/2 R(U) with C^n = U^n + dt/2 R(U^n). */
void or_step_constant(const or_grid *g, const double *Un, double dt, double *Cn)
{
    const long n = (long)or_nvars(g) * or_ncells(g);
    double *R = (double *)malloc(n * sizeof(double));
    spatial_operator_r(g, Un, R);
    const double hdt = 0.5 * dt;
    OR_PAR
    for (long i = 0; i < n; i++) Cn[i] = Un[i] + hdt * R[i];
    free(R);
}

void or_cn_residual_cached(const or_grid *g, const double *U, const double *Cn, double dt,
                           double *F, double *RU)
{
    const long n = (long)or_nvars(g) * or_ncells(g);
    spatial_operator_r(g, U, RU);
    const double hdt = 0.5 * dt;
    OR_PAR
    for (long i = 0; i < n; i++) F[i] = (U[i] - Cn[i]) - hdt * RU[i];
}

void or_cn_residual(const or_grid *g, const double *U, const double *Un, double dt, double *F)
{
    const long n = (long)or_nvars(g) * or_ncells(g);
    double *Cn = (double *)malloc(n * sizeof(double));
    double *RU = (double *)malloc(n * sizeof(double));
    or_step_constant(g, Un, dt, Cn);
    or_cn_residual_cached(g, U, Cn, dt, F, RU);
    free(Cn);
    free(RU);
}

/* ---------------- Jacobian-free product (Knoll & Keyes 2004) ---------------- */
double or_fd_eps(long n, double unorm, const double *v)
{
    double vn = or_norm(n, v);
    if (vn == 0.0) return 0.0;
    return sqrt(2.220446049250313e-16) * (1.0 + unorm) / vn;
}

/* Jv = v - dt/2 (R(U + eps v) - R(U)) / eps, R(U) given.  eps <= 0 selects
 * the default formula. */
void or_jv(const or_grid *g, const double *U, const double *RU, const double *v, double dt,
           double eps, double *Jv)
{
    const long n = (long)or_nvars(g) * or_ncells(g);
    if (eps <= 0.0) eps = or_fd_eps(n, or_norm(n, U), v);
    if (eps == 0.0) {
        OR_PAR
        for (long i = 0; i < n; i++) Jv[i] = 0.0;
        return;
    }
    double *W = (double *)malloc(n * sizeof(double));
    double *RW = (double *)malloc(n * sizeof(double));
    OR_PAR
    for (long i = 0; i < n; i++) W[i] = U[i] + eps * v[i];
    spatial_operator_r(g, W, RW);
    const double c = 0.5 * dt / eps;
    OR_PAR
    for (long i = 0; i < n; i++) Jv[i] = v[i] - c * (RW[i] - RU[i]);
    free(W);
    free(RW);
}

/* ---------------- physics-based preconditioner ---------------- */
static long or_cell_index(const or_grid *g, const int ix[3])
{
    return ix[0] + (long)g->n[0] * (ix[1] + (long)g->n[1] * ix[2]);
}

/* neighbour of cell ix along d by off (+-1); periodic wrap, walls clamp (the
 * coefficient of a wall face is zero so the clamped value never counts). */
static long or_nb(const or_grid *g, const int ix[3], int d, int off)
{
    int j[3] = {ix[0], ix[1], ix[2]};
    int a = j[d] + off;
    if (g->bc[d] == OR_BC_PERIODIC)
        a = ((a % g->n[d]) + g->n[d]) % g->n[d];
    else if (a < 0)
        a = 0;
    else if (a >= g->n[d])
        a = g->n[d] - 1;
    j[d] = a;
    return or_cell_index(g, j);
}

/* is the lower d-face of cell ix a wall face? */
static int or_wall_face(const or_grid *g, const int ix[3], int d)
{
    return g->bc[d] == OR_BC_WALL && ix[d] == 0;
}

static void or_cell_coords(const or_grid *g, long c, int ix[3])
{
    ix[0] = (int)(c % g->n[0]);
    ix[1] = (int)((c / g->n[0]) % g->n[1]);
    ix[2] = (int)(c / ((long)g->n[0] * g->n[1]));
}

/*
 * z = M^-1 r.  M approximates J = I - dt/2 dR/dU by the acoustic subsystem
 * with coefficients frozen at U: advection and gravity are dropped, so
 *   drho + tau div(dm) = r_rho,
 *   dE + tau hp div(dm / rbar) = r_E,       hp = E + p = gamma E,
 *   dm + tau grad(dp) = r_m,                 dp = (gamma - 1) dE,
 * with tau = dt/2.  Eliminating dm gives, per cell,
 *   dp/gp - tau^2 div(grad(dp)/rbar) = (gamma-1) r_E/gp - tau div(r_m/rbar),
 * gp = gamma p.  That system is relaxed with `sweeps` weighted Jacobi sweeps
 * (weight 0.8) from dp = 0; dm, drho and dE follow by back substitution.
 * Jacobi, unlike red-black Gauss-Seidel on an even grid, commutes with the
 * mirror reflections of the grid, so M^-1 keeps the symmetry of Sec. 3.
 */
/*
 * General form of the same preconditioner for spherical grids and for grids
 * with radiative diffusion.  With conduction, the energy row gains
 * -tau div(chi grad dT), dT = dp / rho (coefficients frozen, the density
 * change neglected), so the pressure problem becomes
 *   dp/gp - tau^2 div(grad(dp)/rbar) - (tau (gamma-1)/gp) div(chi grad(dp/rho)) = b
 * and the energy back substitution gains + tau div(chi grad(dp/rho)).  Every
 * divergence is (1/V) sum(A F) over the cell faces; gradients divide by the
 * distance between cell centres (dr, or r_c dtheta).
 */
static void or_precond_general(const or_grid *g, const double *U, double dt, const double *r, double *z)
{
    const int nd = g->nd;
    const long N = or_ncells(g);
    const double gam = g->gamma, gm1 = gam - 1.0;
    const double tau = 0.5 * dt, tau2 = tau * tau;
    const int sph = (g->geom == OR_GEOM_SPHERICAL);
    double *gp = (double *)malloc(N * sizeof(double));
    double *hp = (double *)malloc(N * sizeof(double));
    double *rh = (double *)malloc(N * sizeof(double));
    double *b = (double *)malloc(N * sizeof(double));
    double *dp = (double *)calloc(N, sizeof(double));
    double *dq = (double *)malloc(N * sizeof(double));
    double *chi = (double *)calloc(N, sizeof(double));
    OR_PAR
    for (long c = 0; c < N; c++) {
        gp[c] = gam * (gm1 * U[N + c]);
        hp[c] = gam * U[N + c];
        rh[c] = U[c];
        if (g->conduct) {
            double t = gm1 * U[N + c] / U[c];
            double t3 = t * t * t;
            chi[c] = g->chi0 * (t3 * t3 * sqrt(t)) / (U[c] * U[c]);
        }
    }
    /* per cell and direction: divergence weights W (A/V) of the lower / upper
       face, gradient lengths h, 1/rbar and face chi (0 across walls) */
#define IS_LW(d, ix) (g->bc[d] == OR_BC_WALL && (ix)[d] == 0)
#define IS_UW(d, ix) (g->bc[d] == OR_BC_WALL && (ix)[d] == g->n[d] - 1)
    double *Wm = (double *)malloc(N * 3 * sizeof(double)), *Wp = (double *)malloc(N * 3 * sizeof(double));
    double *hm = (double *)malloc(N * 3 * sizeof(double)), *hpl = (double *)malloc(N * 3 * sizeof(double));
    double *am = (double *)malloc(N * 3 * sizeof(double)), *ap = (double *)malloc(N * 3 * sizeof(double));
    double *km = (double *)malloc(N * 3 * sizeof(double)), *kp = (double *)malloc(N * 3 * sizeof(double));
    OR_PAR
    for (long c = 0; c < N; c++) {
        int ix[3];
        or_cell_coords(g, c, ix);
        const double V = sph ? or_sph_vol(g, ix[0], ix[1]) : 0.0;
        for (int d = 0; d < nd; d++) {
            const long k = c * 3 + d;
            if (sph) {
                int up[3] = {ix[0], ix[1], ix[2]};
                up[d] += 1;
                Wm[k] = or_sph_area(g, d, ix[0], ix[1]) / V;
                Wp[k] = or_sph_area(g, d, up[0], up[1]) / V;
                hm[k] = hpl[k] = or_sph_h(g, d, ix[0]);
            } else {
                Wm[k] = Wp[k] = 1.0 / g->dx[d];
                hm[k] = hpl[k] = g->dx[d];
            }
            long l = or_nb(g, ix, d, -1), u = or_nb(g, ix, d, +1);
            am[k] = IS_LW(d, ix) ? 0.0 : 1.0 / (0.5 * (U[l] + U[c]));
            ap[k] = IS_UW(d, ix) ? 0.0 : 1.0 / (0.5 * (U[c] + U[u]));
            km[k] = IS_LW(d, ix) ? 0.0 : 0.5 * (chi[l] + chi[c]);
            kp[k] = IS_UW(d, ix) ? 0.0 : 0.5 * (chi[c] + chi[u]);
        }
    }
    double *D = (double *)malloc(N * sizeof(double));
    OR_PAR
    for (long c = 0; c < N; c++) {
        int ix[3];
        or_cell_coords(g, c, ix);
        double divm = 0.0, diag = 0.0, dth = 0.0;
        for (int d = 0; d < nd; d++) {
            const long k = c * 3 + d;
            double rp = r[(2 + d) * N + or_nb(g, ix, d, +1)], rm = r[(2 + d) * N + c];
            divm += Wp[k] * ap[k] * rp - Wm[k] * am[k] * rm;
            diag += Wp[k] * ap[k] / hpl[k] + Wm[k] * am[k] / hm[k];
            dth += Wp[k] * kp[k] / hpl[k] + Wm[k] * km[k] / hm[k];
        }
        b[c] = gm1 * r[N + c] / gp[c] - tau * divm;
        D[c] = 1.0 / gp[c] + tau2 * diag + (tau * gm1 / gp[c]) * dth / rh[c];
    }
    const double omega = OR_JACOBI_OMEGA;
    for (int sw = 0; sw < g->sweeps; sw++) {
        OR_PAR
        for (long c = 0; c < N; c++) {
            int ix[3];
            or_cell_coords(g, c, ix);
            double off = 0.0;
            for (int d = 0; d < nd; d++) {
                const long k = c * 3 + d;
                long u = or_nb(g, ix, d, +1), l = or_nb(g, ix, d, -1);
                off += tau2 * (Wp[k] * ap[k] / hpl[k] * dp[u] + Wm[k] * am[k] / hm[k] * dp[l]);
                off += (tau * gm1 / gp[c]) * (Wp[k] * kp[k] / hpl[k] * dp[u] / rh[u] +
                                              Wm[k] * km[k] / hm[k] * dp[l] / rh[l]);
            }
            dq[c] = (1.0 - omega) * dp[c] + omega * ((b[c] + off) / D[c]);
        }
        memcpy(dp, dq, N * sizeof(double));
    }
    /* back substitution */
    for (int d = 0; d < nd; d++) {
        OR_PAR
        for (long c = 0; c < N; c++) {
            int ix[3];
            or_cell_coords(g, c, ix);
            if (IS_LW(d, ix))
                z[(2 + d) * N + c] = r[(2 + d) * N + c];
            else
                z[(2 + d) * N + c] = r[(2 + d) * N + c] - tau * (dp[c] - dp[or_nb(g, ix, d, -1)]) / hm[c * 3 + d];
        }
    }
    OR_PAR
    for (long c = 0; c < N; c++) {
        int ix[3];
        or_cell_coords(g, c, ix);
        double divm = 0.0, divu = 0.0, dth = 0.0;
        for (int d = 0; d < nd; d++) {
            const long k = c * 3 + d;
            long u = or_nb(g, ix, d, +1), l = or_nb(g, ix, d, -1);
            double mp = IS_UW(d, ix) ? 0.0 : z[(2 + d) * N + u];
            double mm = IS_LW(d, ix) ? 0.0 : z[(2 + d) * N + c];
            divm += Wp[k] * mp - Wm[k] * mm;
            divu += Wp[k] * ap[k] * mp - Wm[k] * am[k] * mm;
            dth += Wp[k] * kp[k] * (dp[u] / rh[u] - dp[c] / rh[c]) / hpl[k] -
                   Wm[k] * km[k] * (dp[c] / rh[c] - dp[l] / rh[l]) / hm[k];
        }
        z[c] = r[c] - tau * divm;
        z[N + c] = (r[N + c] - tau * hp[c] * divu) + tau * dth;
    }
#undef IS_LW
#undef IS_UW
    free(gp); free(hp); free(rh); free(b); free(dp); free(dq); free(chi); free(D);
    free(Wm); free(Wp); free(hm); free(hpl); free(am); free(ap); free(km); free(kp);
}

void or_precond(const or_grid *g, const double *U, double dt, const double *r, double *z)
{
    const int nd = g->nd;
    const long N = or_ncells(g);
    const long n = (long)or_nvars(g) * N;
    if (g->precond == OR_PC_NONE) {
        memcpy(z, r, n * sizeof(double));
        return;
    }
    if (g->geom == OR_GEOM_SPHERICAL || g->conduct) {
        or_precond_general(g, U, dt, r, z);
        return;
    }
    const double gam = g->gamma, gm1 = gam - 1.0;
    const double tau = 0.5 * dt, tau2 = tau * tau;
    double *a[3];
    double *gp = (double *)malloc(N * sizeof(double));
    double *hp = (double *)malloc(N * sizeof(double));
    double *b = (double *)malloc(N * sizeof(double));
    double *D = (double *)malloc(N * sizeof(double));
    double *dp = (double *)calloc(N, sizeof(double));
    for (int d = 0; d < nd; d++) a[d] = (double *)malloc(N * sizeof(double));

    /* frozen coefficients: a_d = 1/rbar on the lower d-face (0 on walls) */
    OR_PAR
    for (long c = 0; c < N; c++) {
        int ix[3];
        or_cell_coords(g, c, ix);
        gp[c] = gam * (gm1 * U[N + c]);
        hp[c] = gam * U[N + c];
        for (int d = 0; d < nd; d++) {
            if (or_wall_face(g, ix, d)) {
                a[d][c] = 0.0;
            } else {
                long l = or_nb(g, ix, d, -1);
                a[d][c] = 1.0 / (0.5 * (U[l] + U[c]));
            }
        }
    }
    /* coefficient of the upper d-face of cell c: the lower face of the next
       cell, or 0 on the implicit upper wall */
#define A_UP(d, c, ix) ((g->bc[d] == OR_BC_WALL && (ix)[d] == g->n[d] - 1) ? 0.0 : a[d][or_nb(g, ix, d, +1)])

    OR_PAR
    for (long c = 0; c < N; c++) {
        int ix[3];
        or_cell_coords(g, c, ix);
        double divm = 0.0, diag = 0.0;
        for (int d = 0; d < nd; d++) {
            double ap = A_UP(d, c, ix), am = a[d][c];
            double rp = r[(2 + d) * N + or_nb(g, ix, d, +1)];
            double rm = r[(2 + d) * N + c];
            divm += (ap * rp - am * rm) / g->dx[d];
            diag += (ap + am) / (g->dx[d] * g->dx[d]);
        }
        b[c] = gm1 * r[N + c] / gp[c] - tau * divm;
        D[c] = 1.0 / gp[c] + tau2 * diag;
    }

    /* weighted Jacobi sweeps (order free, so mirror symmetric) */
    const double omega = OR_JACOBI_OMEGA;
    double *dq = (double *)malloc(N * sizeof(double));
    for (int s = 0; s < g->sweeps; s++) {
        OR_PAR
        for (long c = 0; c < N; c++) {
            int ix[3];
            or_cell_coords(g, c, ix);
            double off = 0.0;
            for (int d = 0; d < nd; d++) {
                double ap = A_UP(d, c, ix), am = a[d][c];
                off += (ap * dp[or_nb(g, ix, d, +1)] + am * dp[or_nb(g, ix, d, -1)]) /
                       (g->dx[d] * g->dx[d]);
            }
            dq[c] = (1.0 - omega) * dp[c] + omega * ((b[c] + tau2 * off) / D[c]);
        }
        memcpy(dp, dq, N * sizeof(double));
    }
    free(dq);

    /* back substitution: dm on faces, then drho and dE in flux form */
    for (int d = 0; d < nd; d++) {
        OR_PAR
        for (long c = 0; c < N; c++) {
            int ix[3];
            or_cell_coords(g, c, ix);
            if (or_wall_face(g, ix, d))
                z[(2 + d) * N + c] = r[(2 + d) * N + c];
            else
                z[(2 + d) * N + c] =
                    r[(2 + d) * N + c] - tau * (dp[c] - dp[or_nb(g, ix, d, -1)]) / g->dx[d];
        }
    }
    OR_PAR
    for (long c = 0; c < N; c++) {
        int ix[3];
        or_cell_coords(g, c, ix);
        double divm = 0.0, divu = 0.0;
        for (int d = 0; d < nd; d++) {
            int up_wall = (g->bc[d] == OR_BC_WALL && ix[d] == g->n[d] - 1);
            double mp = up_wall ? 0.0 : z[(2 + d) * N + or_nb(g, ix, d, +1)];
            double mm = or_wall_face(g, ix, d) ? 0.0 : z[(2 + d) * N + c];
            double ap = A_UP(d, c, ix), am = a[d][c];
            divm += (mp - mm) / g->dx[d];
            divu += (ap * mp - am * mm) / g->dx[d];
        }
        z[c] = r[c] - tau * divm;
        z[N + c] = r[N + c] - tau * hp[c] * divu;
    }
#undef A_UP
    for (int d = 0; d < nd; d++) free(a[d]);
    free(gp); free(hp); free(b); free(D); free(dp);
}

/* ---------------- restarted GMRES (Saad & Schultz 1986) ---------------- */
typedef void (*or_op)(void *ctx, const double *in, double *out);

typedef struct {
    int its;        /* Arnoldi steps taken */
    int cycles;     /* restart cycles */
    int converged;
    double resid;   /* final residual estimate */
} or_gmres_stats;

/*
 * Solve A x = b with right preconditioning, A M^-1 y = b, x = M^-1 y, x0 = 0.
 * Arnoldi with classical Gram-Schmidt and one re-orthogonalisation; the
 * Hessenberg least-squares problem by Givens rotations.  Stops when the
 * residual estimate |g_{j+1}| <= rtol |b|.
 */
int or_gmres(long n, or_op A, or_op Minv, void *ctx, const double *b, double *x, int m,
             int max_restarts, double rtol, or_gmres_stats *st)
{
    OR_PAR
    for (long i = 0; i < n; i++) x[i] = 0.0;
    if (m < 1 || m > 63) return 2;
    st->its = 0;
    st->cycles = 0;
    st->converged = 0;
    const double bnorm = or_norm(n, b);
    st->resid = bnorm;
    if (bnorm == 0.0) {
        st->converged = 1;
        return 0;
    }
    const double target = rtol * bnorm;
    double *V = (double *)malloc((size_t)(m + 1) * n * sizeof(double));
    double *w = (double *)malloc(n * sizeof(double));
    double *z = (double *)malloc(n * sizeof(double));
    double *H = (double *)calloc((size_t)(m + 1) * m, sizeof(double)); /* H[i*m + j] */
    double *cs = (double *)malloc(m * sizeof(double));
    double *sn = (double *)malloc(m * sizeof(double));
    double *gv = (double *)malloc((m + 1) * sizeof(double));
    double *y = (double *)malloc(m * sizeof(double));
    double *h = (double *)malloc((m + 1) * sizeof(double));

    for (int cycle = 0; cycle <= max_restarts; cycle++) {
        st->cycles = cycle + 1;
        /* r = b - A x */
        if (cycle == 0) {
            memcpy(V, b, n * sizeof(double));
        } else {
            A(ctx, x, w);
            OR_PAR
            for (long i = 0; i < n; i++) V[i] = b[i] - w[i];
        }
        double beta = or_norm(n, V);
        st->resid = beta;
        if (beta <= target) {
            st->converged = 1;
            break;
        }
        OR_PAR
        for (long i = 0; i < n; i++) V[i] = V[i] / beta;
        for (int i = 0; i <= m; i++) gv[i] = 0.0;
        gv[0] = beta;
        int k = 0; /* number of columns built */
        for (int j = 0; j < m; j++) {
            double *Vj = V + (size_t)j * n;
            Minv(ctx, Vj, z);
            A(ctx, z, w);
            /* CGS, twice */
            for (int i = 0; i <= j; i++) h[i] = 0.0;
            for (int pass = 0; pass < 2; pass++) {
                double hp_[64];
                for (int i = 0; i <= j; i++) hp_[i] = or_dot(n, V + (size_t)i * n, w);
                for (int i = 0; i <= j; i++) {
                    const double *Vi = V + (size_t)i * n;
                    OR_PAR
                    for (long q = 0; q < n; q++) w[q] -= hp_[i] * Vi[q];
                    h[i] += hp_[i];
                }
            }
            double hn = or_norm(n, w);
            for (int i = 0; i <= j; i++) H[i * m + j] = h[i];
            H[(j + 1) * m + j] = hn;
            /* previous rotations */
            for (int i = 0; i < j; i++) {
                double t0 = H[i * m + j], t1 = H[(i + 1) * m + j];
                H[i * m + j] = cs[i] * t0 + sn[i] * t1;
                H[(i + 1) * m + j] = -sn[i] * t0 + cs[i] * t1;
            }
            /* new rotation zeroing H[j+1][j] */
            double a0 = H[j * m + j], a1 = H[(j + 1) * m + j];
            if (a1 == 0.0) {
                cs[j] = 1.0;
                sn[j] = 0.0;
            } else {
                double t = sqrt(a0 * a0 + a1 * a1);
                cs[j] = a0 / t;
                sn[j] = a1 / t;
            }
            H[j * m + j] = cs[j] * a0 + sn[j] * a1;
            H[(j + 1) * m + j] = 0.0;
            gv[j + 1] = -sn[j] * gv[j];
            gv[j] = cs[j] * gv[j];
            st->its++;
            k = j + 1;
            st->resid = fabs(gv[j + 1]);
            if (hn == 0.0 || fabs(gv[j + 1]) <= target) break;
            double *Vn = V + (size_t)(j + 1) * n;
            OR_PAR
            for (long q = 0; q < n; q++) Vn[q] = w[q] / hn;
        }
        /* y = H^-1 g (upper triangular k x k) */
        for (int i = k - 1; i >= 0; i--) {
            double s = gv[i];
            for (int l = i + 1; l < k; l++) s -= H[i * m + l] * y[l];
            y[i] = s / H[i * m + i];
        }
        /* x += M^-1 (V y) */
        OR_PAR
        for (long q = 0; q < n; q++) w[q] = 0.0;
        for (int i = 0; i < k; i++) {
            const double *Vi = V + (size_t)i * n;
            OR_PAR
            for (long q = 0; q < n; q++) w[q] += y[i] * Vi[q];
        }
        Minv(ctx, w, z);
        OR_PAR
        for (long q = 0; q < n; q++) x[q] += z[q];
        if (st->resid <= target) {
            st->converged = 1;
            break;
        }
    }
    free(V); free(w); free(z); free(H); free(cs); free(sn); free(gv); free(y); free(h);
    return st->converged ? 0 : 1;
}

/* dense test operator for the GMRES pin: out = A in, A row-major n x n */
typedef struct {
    long n;
    const double *A;
} or_dense_ctx;

static void or_dense_apply(void *ctx, const double *in, double *out)
{
    or_dense_ctx *c = (or_dense_ctx *)ctx;
    for (long i = 0; i < c->n; i++) {
        double s = 0.0;
        for (long j = 0; j < c->n; j++) s += c->A[i * c->n + j] * in[j];
        out[i] = s;
    }
}

static void or_identity(void *ctx, const double *in, double *out)
{
    or_dense_ctx *c = (or_dense_ctx *)ctx;
    memcpy(out, in, c->n * sizeof(double));
}

int or_gmres_dense(long n, const double *A, const double *b, double *x, int m, int max_restarts,
                   double rtol, int *its)
{
    or_dense_ctx ctx = {n, A};
    or_gmres_stats st;
    int rc = or_gmres(n, or_dense_apply, or_identity, &ctx, b, x, m, max_restarts, rtol, &st);
    *its = st.its;
    return rc;
}

/* ---------------- Newton-Raphson on the CN system ---------------- */
typedef struct {
    const or_grid *g;
    const double *U;
    const double *RU;
    double unorm;
    double dt;
} or_newton_ctx;

static void or_ctx_jv(void *ctx, const double *v, double *out)
{
    or_newton_ctx *c = (or_newton_ctx *)ctx;
    const long n = (long)or_nvars(c->g) * or_ncells(c->g);
    double eps = or_fd_eps(n, c->unorm, v);
    if (eps == 0.0) {
        OR_PAR
        for (long i = 0; i < n; i++) out[i] = 0.0;
        return;
    }
    or_jv(c->g, c->U, c->RU, v, c->dt, eps, out);
}

static void or_ctx_precond(void *ctx, const double *r, double *z)
{
    or_newton_ctx *c = (or_newton_ctx *)ctx;
    or_precond(c->g, c->U, c->dt, r, z);
}

/* One implicit step of size dt, in place.  Returns 0 on convergence; on
 * failure U is restored to U^n and 1 is returned. */
int or_newton_step(const or_grid *g, double *U, double dt, or_step_stats *st)
{
    const long N = or_ncells(g);
    const long n = (long)or_nvars(g) * N;
    double *Un = (double *)malloc(n * sizeof(double));
    double *Cn = (double *)malloc(n * sizeof(double));
    double *F = (double *)malloc(n * sizeof(double));
    double *RU = (double *)malloc(n * sizeof(double));
    double *x = (double *)malloc(n * sizeof(double));
    memcpy(Un, U, n * sizeof(double));
    or_step_constant(g, Un, dt, Cn);
    st->dt = dt;
    st->newton_its = 0;
    st->gmres_its = 0;
    st->gmres_failures = 0;
    int ok = 0;
    for (int k = 0; k < g->newton_max; k++) {
        or_cn_residual_cached(g, U, Cn, dt, F, RU);
        st->fnorm = or_norm(n, F);
        if (k == 0) st->fnorm0 = st->fnorm;
        OR_PAR
        for (long i = 0; i < n; i++) F[i] = -F[i];
        or_newton_ctx ctx = {g, U, RU, or_norm(n, U), dt};
        or_gmres_stats gs;
        int rc = or_gmres(n, or_ctx_jv, or_ctx_precond, &ctx, F, x, g->restart, g->max_restarts,
                          g->gmres_rtol, &gs);
        st->gmres_its += gs.its;
        st->gmres_failures += rc;
        double mx = 0.0;
        OR_PAR
        for (long i = 0; i < n; i++) U[i] += x[i];
        for (long c = 0; c < N; c++) {
            double q = fabs(x[c]) / U[c];
            if (!(q <= mx)) mx = q; /* NaN propagates */
        }
        st->max_drho = mx;
        st->newton_its = k + 1;
        if (mx <= g->newton_tol) {
            ok = 1;
            break;
        }
    }
    if (!ok) memcpy(U, Un, n * sizeof(double));
    free(Un); free(Cn); free(F); free(RU); free(x);
    return ok ? 0 : 1;
}

/* ---------------- time step (Eq. 4) ---------------- */
double or_cfl_rate(const or_grid *g, const double *U)
{
    const long N = or_ncells(g);
    double lam = 0.0;
    for (long c = 0; c < N; c++) {
        int ix[3];
        or_cell_coords(g, c, ix);
        double rho = U[c];
        double cs = sqrt(g->gamma * ((g->gamma - 1.0) * U[N + c]) / rho);
        for (int d = 0; d < g->nd; d++) {
            double um = 0.0, up = 0.0;
            if (!or_wall_face(g, ix, d)) {
                long l = or_nb(g, ix, d, -1);
                um = U[(2 + d) * N + c] / (0.5 * (U[l] + rho));
            }
            if (!(g->bc[d] == OR_BC_WALL && ix[d] == g->n[d] - 1)) {
                long r = or_nb(g, ix, d, +1);
                up = U[(2 + d) * N + r] / (0.5 * (rho + U[r]));
            }
            double h = (g->geom == OR_GEOM_SPHERICAL) ? or_sph_h(g, d, ix[0]) : g->dx[d];
            double q = (fabs(0.5 * (um + up)) + cs) / h;
            if (q > lam) lam = q;
        }
    }
    return lam;
}

/* Advance nsteps implicit steps with dt = cfl / rate (capped by dt_max > 0).
 * A failed Newton solve halves dt up to max_halvings times.  Per-step stats
 * go to st[0..nsteps).  Returns the number of steps completed. */
int or_run(const or_grid *g, double *U, int nsteps, double cfl, double dt_max, or_step_stats *st)
{
    for (int s = 0; s < nsteps; s++) {
        double dt = cfl / or_cfl_rate(g, U);
        if (dt_max > 0.0 && dt > dt_max) dt = dt_max;
        int h = 0;
        for (;;) {
            int rc = or_newton_step(g, U, dt, &st[s]);
            if (rc == 0) break;
            if (h >= g->max_halvings) return s;
            dt = 0.5 * dt;
            h++;
        }
        st[s].halvings = h;
    }
    return nsteps;
}

/* ---------------- diagnostics (Sec. 3-6) ---------------- */
/*
 * out[0] mixing-layer height h = sum_rows X_M(<X_H>_row) dy, X_H = (rho -
 *        rho_L)/(rho_H - rho_L), rows along direction 1 (Cabot & Cook);
 * out[1] max Mach number over cells (cell-centred velocity);
 * out[2] amplitude of the x-mode with two wavelengths across the box in the
 *        vertical velocity: (2 / N) |sum_{y-faces} v e^{-i k x}|;
 * out[3] vertical kinetic energy sum_{y-faces} 1/2 rbar v^2 dV;
 * out[4] mean kinetic energy density (1/N) sum_d sum_{d-faces} 1/2 rbar u_d^2;
 * out[5] max cell-centred speed.
 */
void or_diagnostics(const or_grid *g, const double *U, double rho_L, double rho_H, double *out)
{
    const int nd = g->nd;
    const long N = or_ncells(g);
    const double dV = g->dx[0] * g->dx[1] * (nd == 3 ? g->dx[2] : 1.0);
    double *uf[3];
    for (int d = 0; d < nd; d++) {
        uf[d] = (double *)malloc(N * sizeof(double));
        for (long c = 0; c < N; c++) {
            int ix[3];
            or_cell_coords(g, c, ix);
            if (or_wall_face(g, ix, d)) {
                uf[d][c] = 0.0;
            } else {
                long l = or_nb(g, ix, d, -1);
                uf[d][c] = U[(2 + d) * N + c] / (0.5 * (U[l] + U[c]));
            }
        }
    }
    /* mixing height */
    const int ny = g->n[1];
    const long per_row = N / ny;
    double hmix = 0.0;
    for (int j = 0; j < ny; j++) {
        double s = 0.0;
        for (int k = 0; k < g->n[2]; k++)
            for (int i = 0; i < g->n[0]; i++) {
                int ix[3] = {i, j, k};
                s += (U[or_cell_index(g, ix)] - rho_L) / (rho_H - rho_L);
            }
        double xh = s / (double)per_row;
        double xm = (xh <= 0.5) ? 2.0 * xh : 2.0 * (1.0 - xh);
        hmix += xm * g->dx[1];
    }
    double mach = 0.0, speed = 0.0, ekin = 0.0, ey = 0.0, cre = 0.0, cim = 0.0;
    const double k = 2.0 * (2.0 * M_PI / (g->n[0] * g->dx[0]));
    for (long c = 0; c < N; c++) {
        int ix[3];
        or_cell_coords(g, c, ix);
        double rho = U[c];
        double cs = sqrt(g->gamma * ((g->gamma - 1.0) * U[N + c]) / rho);
        double u2 = 0.0;
        for (int d = 0; d < nd; d++) {
            double up = 0.0;
            if (!(g->bc[d] == OR_BC_WALL && ix[d] == g->n[d] - 1)) up = uf[d][or_nb(g, ix, d, +1)];
            double uc = 0.5 * (uf[d][c] + up);
            u2 += uc * uc;
            double rbar = 0.0;
            if (!or_wall_face(g, ix, d)) rbar = 0.5 * (U[or_nb(g, ix, d, -1)] + rho);
            ekin += 0.5 * rbar * uf[d][c] * uf[d][c];
        }
        double sp = sqrt(u2);
        if (sp / cs > mach) mach = sp / cs;
        if (sp > speed) speed = sp;
        /* y-face quantities */
        double v = uf[1][c];
        double rbar = or_wall_face(g, ix, 1) ? 0.0 : 0.5 * (U[or_nb(g, ix, 1, -1)] + rho);
        ey += 0.5 * rbar * v * v * dV;
        double xc = g->x0[0] + (ix[0] + 0.5) * g->dx[0];
        cre += v * cos(k * xc);
        cim += v * sin(k * xc);
    }
    out[0] = hmix;
    out[1] = mach;
    out[2] = 2.0 / (double)N * sqrt(cre * cre + cim * cim);
    out[3] = ey;
    out[4] = ekin / (double)N;
    out[5] = speed;
    for (int d = 0; d < nd; d++) free(uf[d]);
}

double or_select_dt(const or_grid *g, const double *U, double cfl_hydro, double cfl_adv, double cfl_rad,
                    double dt_max, int *which);

/* ---------------- passive scalars (Sec. 2.2) ---------------- */
/*
 * ns passive scalars carried as partial densities q_i = c_i rho (ns planes
 * of N values).  Their equation d(c_i rho)/dt = -div(c_i rho u) is solved by
 * its own unpreconditioned Jacobian-free Newton-Krylov iteration, inside the
 * fluid's Newton loop: iteration k solves the scalar Crank-Nicolson system
 * linearised at q^k with the fluid frozen at the same iterate U^k that the
 * fluid residual of iteration k uses, with the fluid's GMRES settings.  The
 * loop stops on the fluid density test alone (the paper's default), or, with
 * `enforce`, also on max |delta q_i| / rho <= newton_tol.  After a step the
 * concentrations are renormalised to sum to one: c_i <- c_i / sum_j c_j.
 * Cartesian grids only.
 */

/* mass fluxes of U on the extended grid (nd arrays of the extended size) */
static double **or_mass_fluxes(const or_grid *g, const double *U)
{
    or_ext X;
    or_ext_init(&X, g);
    const long n = (long)or_nvars(g) * or_ncells(g);
    double **Fr = (double **)calloc(3, sizeof(double *));
    for (int d = 0; d < g->nd; d++) Fr[d] = (double *)calloc(X.total, sizeof(double));
    double *R = (double *)malloc(n * sizeof(double));
    spatial_operator_f_r(g, U, R, Fr, NULL);
    free(R);
    return Fr;
}

static void or_free_fluxes(const or_grid *g, double **Fr)
{
    for (int d = 0; d < g->nd; d++) free(Fr[d]);
    free(Fr);
}

/* S = scalar operator of q with the fluid frozen at U */
void or_scalar_operator(const or_grid *g, const double *U, const double *q, int ns, double *S)
{
    double **Fr = or_mass_fluxes(g, U);
    scalar_operator_r(g, U, Fr, q, ns, S);
    or_free_fluxes(g, Fr);
}

/* exact dS/dq v by complex-step differentiation (h = 1e-30) */
void or_scalar_operator_dir(const or_grid *g, const double *U, const double *q, const double *v, int ns,
                            double *dS)
{
    const long nq = (long)ns * or_ncells(g);
    double **Fr = or_mass_fluxes(g, U);
    double complex *qc = (double complex *)malloc(nq * sizeof(double complex));
    double complex *Sc = (double complex *)malloc(nq * sizeof(double complex));
    const double h = 1e-30;
        for (long i = 0; i < nq; i++) qc[i] = q[i] + I * h * v[i];
    scalar_operator_c(g, U, Fr, qc, ns, Sc);
        for (long i = 0; i < nq; i++) dS[i] = cimag(Sc[i]) / h;
    free(qc);
    free(Sc);
    or_free_fluxes(g, Fr);
}

typedef struct {
    const or_grid *g;
    const double *rho;
    double *const *Fr;
    const double *q;
    const double *Sq;
    double qnorm;
    double dt;
    int ns;
} or_scal_ctx;

/* v - dt/2 (S(q + eps v) - S(q)) / eps */
static void or_scal_jv(void *ctx, const double *v, double *out)
{
    or_scal_ctx *c = (or_scal_ctx *)ctx;
    const long nq = (long)c->ns * or_ncells(c->g);
    const double eps = or_fd_eps(nq, c->qnorm, v);
    if (eps == 0.0) {
        OR_PAR
        for (long i = 0; i < nq; i++) out[i] = 0.0;
        return;
    }
    double *W = (double *)malloc(nq * sizeof(double));
    double *SW = (double *)malloc(nq * sizeof(double));
    OR_PAR
    for (long i = 0; i < nq; i++) W[i] = c->q[i] + eps * v[i];
    scalar_operator_r(c->g, c->rho, c->Fr, W, c->ns, SW);
    const double a = 0.5 * c->dt / eps;
    OR_PAR
    for (long i = 0; i < nq; i++) out[i] = v[i] - a * (SW[i] - c->Sq[i]);
    free(W);
    free(SW);
}

/* the scalar solve is unpreconditioned: M = I */
static void or_scal_identity(void *ctx, const double *in, double *out)
{
    or_scal_ctx *c = (or_scal_ctx *)ctx;
    memcpy(out, in, (long)c->ns * or_ncells(c->g) * sizeof(double));
}

/* c_i <- c_i / sum_j c_j with the cell density rho */
static void or_scalar_renormalise(const or_grid *g, const double *rho, double *q, int ns)
{
    const long N = or_ncells(g);
    OR_PAR
    for (long k = 0; k < N; k++) {
        double s = 0.0;
        for (int i = 0; i < ns; i++) s += q[(long)i * N + k] / rho[k];
        if (!(s > 0.0)) continue;
        for (int i = 0; i < ns; i++) q[(long)i * N + k] = (q[(long)i * N + k] / rho[k] / s) * rho[k];
    }
}

/* One implicit step of the fluid and the scalars; returns 0 or 1 (Newton
 * failed: U and q restored).  scal_gmres receives the scalar GMRES steps. */
int or_newton_step_s(const or_grid *g, double *U, double *q, int ns, double dt, int enforce, or_step_stats *st,
                     int *scal_gmres)
{
    const long N = or_ncells(g);
    const long n = (long)or_nvars(g) * N;
    const long nq = (long)ns * N;
    double *Un = (double *)malloc(n * sizeof(double));
    double *qn = (double *)malloc(nq * sizeof(double));
    double *Cn = (double *)malloc(n * sizeof(double));
    double *F = (double *)malloc(n * sizeof(double));
    double *RU = (double *)malloc(n * sizeof(double));
    double *x = (double *)malloc(n * sizeof(double));
    double *Cs = (double *)malloc(nq * sizeof(double));
    double *Sq = (double *)malloc(nq * sizeof(double));
    double *bs = (double *)malloc(nq * sizeof(double));
    double *dq = (double *)malloc(nq * sizeof(double));
    memcpy(Un, U, n * sizeof(double));
    memcpy(qn, q, nq * sizeof(double));
    or_step_constant(g, Un, dt, Cn);
    {
        double **Fr = or_mass_fluxes(g, Un);
        scalar_operator_r(g, Un, Fr, qn, ns, Sq);
        OR_PAR
        for (long i = 0; i < nq; i++) Cs[i] = qn[i] + 0.5 * dt * Sq[i];
        or_free_fluxes(g, Fr);
    }
    st->dt = dt;
    st->newton_its = 0;
    st->gmres_its = 0;
    st->gmres_failures = 0;
    *scal_gmres = 0;
    int ok = 0;
    for (int k = 0; k < g->newton_max; k++) {
        /* scalars, with the fluid frozen at U^k */
        double **Fr = or_mass_fluxes(g, U);
        scalar_operator_r(g, U, Fr, q, ns, Sq);
        OR_PAR
        for (long i = 0; i < nq; i++) bs[i] = -((q[i] - Cs[i]) - 0.5 * dt * Sq[i]);
        or_scal_ctx sc = {g, U, Fr, q, Sq, or_norm(nq, q), dt, ns};
        or_gmres_stats sgs;
        or_gmres(nq, or_scal_jv, or_scal_identity, &sc, bs, dq, g->restart, g->max_restarts, g->gmres_rtol,
                 &sgs);
        *scal_gmres += sgs.its;
        double mq = 0.0;
        for (long i = 0; i < nq; i++) {
            q[i] += dq[i];
            double t = fabs(dq[i]) / U[i % N];
            if (!(t <= mq)) mq = t;
        }
        or_free_fluxes(g, Fr);
        /* the fluid, as in or_newton_step */
        or_cn_residual_cached(g, U, Cn, dt, F, RU);
        st->fnorm = or_norm(n, F);
        if (k == 0) st->fnorm0 = st->fnorm;
        OR_PAR
        for (long i = 0; i < n; i++) F[i] = -F[i];
        or_newton_ctx ctx = {g, U, RU, or_norm(n, U), dt};
        or_gmres_stats gs;
        int rc = or_gmres(n, or_ctx_jv, or_ctx_precond, &ctx, F, x, g->restart, g->max_restarts, g->gmres_rtol,
                          &gs);
        st->gmres_its += gs.its;
        st->gmres_failures += rc;
        double mx = 0.0;
        OR_PAR
        for (long i = 0; i < n; i++) U[i] += x[i];
        for (long c = 0; c < N; c++) {
            double t = fabs(x[c]) / U[c];
            if (!(t <= mx)) mx = t;
        }
        st->max_drho = mx;
        st->newton_its = k + 1;
        if (mx <= g->newton_tol && (!enforce || mq <= g->newton_tol)) {
            ok = 1;
            break;
        }
    }
    if (ok) {
        or_scalar_renormalise(g, U, q, ns);
    } else {
        memcpy(U, Un, n * sizeof(double));
        memcpy(q, qn, nq * sizeof(double));
    }
    free(Un); free(qn); free(Cn); free(F); free(RU); free(x); free(Cs); free(Sq); free(bs); free(dq);
    return ok ? 0 : 1;
}

int or_run_s(const or_grid *g, double *U, double *q, int ns, int nsteps, double cfl, double cfl_adv, double cfl_rad,
             double dt_max, int enforce, or_step_stats *st, int *scal_gmres)
{
    for (int s = 0; s < nsteps; s++) {
        int which;
        double dt = or_select_dt(g, U, cfl, cfl_adv, cfl_rad, dt_max, &which);
        int h = 0;
        for (;;) {
            int rc = or_newton_step_s(g, U, q, ns, dt, enforce, &st[s], &scal_gmres[s]);
            if (rc == 0) break;
            if (h >= g->max_halvings) return s;
            dt = 0.5 * dt;
            h++;
        }
        st[s].halvings = h;
    }
    return nsteps;
}

/* mixing width from the first two scalars: h = sum_rows 2 min(<c_1>, <c_2>) dy,
   <.> the mean over a row of cells normal to direction 1 */
double or_scalar_mixing_width(const or_grid *g, const double *U, const double *q)
{
    const long N = or_ncells(g);
    const int nx = g->n[0], ny = g->n[1], nz = g->n[2];
    double h = 0.0;
    for (int j = 0; j < ny; j++) {
        double a1 = 0.0, a2 = 0.0;
        for (int k = 0; k < nz; k++)
            for (int i = 0; i < nx; i++) {
                const long c = i + (long)nx * (j + (long)ny * k);
                a1 += q[c] / U[c];
                a2 += q[N + c] / U[c];
            }
        a1 /= (double)nx * nz;
        a2 /= (double)nx * nz;
        h += 2.0 * (a1 < a2 ? a1 : a2) * g->dx[1];
    }
    return h;
}

/* ---------------- time-step limits (Sec. 2, choice of the time step) ---------------- */
/*
 * rates[0] = max (|u_d| + c_s) / h_d   (hydrodynamic CFL, Eq. 4);
 * rates[1] = max |u_d| / h_d           (advective CFL);
 * rates[2] = max D / h_d^2             (radiative CFL; 0 without conduction)
 * over cells and directions, u_d the mean of the cell's two face velocities,
 * h_d the distance between cell centres (dr, or r_c dtheta), and D = chi /
 * (rho c_v) the radiative diffusivity, c_v = 1 / (gamma - 1) (p = rho T).
 */
void or_dt_rates(const or_grid *g, const double *U, double *rates)
{
    const long N = or_ncells(g);
    double lh = 0.0, la = 0.0, lr = 0.0;
    const double gm1 = g->gamma - 1.0;
    for (long c = 0; c < N; c++) {
        int ix[3];
        or_cell_coords(g, c, ix);
        double rho = U[c];
        double cs = sqrt(g->gamma * (gm1 * U[N + c]) / rho);
        double D = 0.0;
        if (g->conduct) {
            double T = gm1 * U[N + c] / rho;
            double t3 = T * T * T;
            double chi = g->chi0 * (t3 * t3 * sqrt(T)) / (rho * rho);
            D = chi * gm1 / rho;
        }
        for (int d = 0; d < g->nd; d++) {
            double um = 0.0, up = 0.0;
            if (!or_wall_face(g, ix, d)) {
                long l = or_nb(g, ix, d, -1);
                um = U[(2 + d) * N + c] / (0.5 * (U[l] + rho));
            }
            if (!(g->bc[d] == OR_BC_WALL && ix[d] == g->n[d] - 1)) {
                long r = or_nb(g, ix, d, +1);
                up = U[(2 + d) * N + r] / (0.5 * (rho + U[r]));
            }
            double h = (g->geom == OR_GEOM_SPHERICAL) ? or_sph_h(g, d, ix[0]) : g->dx[d];
            double a = fabs(0.5 * (um + up));
            if ((a + cs) / h > lh) lh = (a + cs) / h;
            if (a / h > la) la = a / h;
            if (D / (h * h) > lr) lr = D / (h * h);
        }
    }
    rates[0] = lh;
    rates[1] = la;
    rates[2] = lr;
}

/* The most restrictive of the limits given (each <= 0: not applied):
 * dt = min(cfl_hydro / rates[0], cfl_adv / rates[1], cfl_rad / rates[2],
 * dt_max).  *which = 0, 1, 2 or 3 names the limit that applied. */
double or_select_dt(const or_grid *g, const double *U, double cfl_hydro, double cfl_adv, double cfl_rad,
                    double dt_max, int *which)
{
    double r[3];
    or_dt_rates(g, U, r);
    const double lim[3] = {cfl_hydro, cfl_adv, cfl_rad};
    double dt = INFINITY;
    *which = -1;
    for (int k = 0; k < 3; k++) {
        if (!(lim[k] > 0.0) || !(r[k] > 0.0)) continue;
        double t = lim[k] / r[k];
        if (t < dt) {
            dt = t;
            *which = k;
        }
    }
    if (dt_max > 0.0 && dt_max < dt) {
        dt = dt_max;
        *which = 3;
    }
    return dt;
}

/* nsteps steps with the time step chosen by or_select_dt (limits <= 0 not
 * applied); returns the steps completed */
int or_run_dt(const or_grid *g, double *U, int nsteps, double cfl_hydro, double cfl_adv, double cfl_rad,
              double dt_max, or_step_stats *st)
{
    for (int s = 0; s < nsteps; s++) {
        int which;
        double dt = or_select_dt(g, U, cfl_hydro, cfl_adv, cfl_rad, dt_max, &which);
        int h = 0;
        for (;;) {
            int rc = or_newton_step(g, U, dt, &st[s]);
            if (rc == 0) break;
            if (h >= g->max_halvings) return s;
            dt = 0.5 * dt;
            h++;
        }
        st[s].halvings = h;
    }
    return nsteps;
}
