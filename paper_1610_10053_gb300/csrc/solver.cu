// Newton-Raphson on the Crank-Nicolson system with restarted, right
// preconditioned GMRES and Jacobian-free products (Sec. 2).  Two drivers run
// the same kernels: the recorded graph of graph.cu (default), whose loops
// and Givens rotations run on the device, and the host-sequenced attempt
// below, which keeps the (m+1) x m Hessenberg matrix on the host and is used
// while the Jacobian-free stencil is being timed (music_profile_enable).
#include <cmath>
#include <cstring>
#include <chrono>

#include "internal.h"

namespace {

struct GmresOut {
    int its;
    int converged;
    double bnorm;
};

// The bound on loop bodies of one Newton attempt, counted where the recorded
// graph's control kernels count them: every Arnoldi step, every GMRES cycle
// and every Newton iteration.
struct LoopGuard {
    long long bodies;
    int cap;
    bool over() { return ++bodies > cap; }
};

int loop_timeout()
{
    set_error("solver: loop-body bound reached");
    return MUSIC_E_TIMEOUT;
}

int sync_scalars(music_grid *g, cudaStream_t s)
{
    CUDA_TRY(cudaMemcpyAsync(g->hs, g->ds, sizeof(DevScalars), cudaMemcpyDeviceToHost, s));
    CUDA_TRY(cudaStreamSynchronize(s));
    if (g->prof_pending) TRY(prof_harvest(g, 0));
    return MUSIC_OK;
}

// Solve J x = b (b = g->b, FP64) into g->x (FP64).
int gmres(music_grid *g, double dt, GmresOut *o, LoopGuard &guard, cudaStream_t s)
{
    const int m = g->desc.gmres_restart;
    const double rtol = g->desc.gmres_rtol;
    const size_t n = g->n;
    const int kd = !g->mixed;  // Krylov vectors are double?
    const size_t ks = kd ? sizeof(double) : sizeof(float);
    o->its = 0;
    o->converged = 0;
    o->bnorm = 0.0;
    CUDA_TRY(cudaMemsetAsync(g->x, 0, n * sizeof(double), s));
    TRY(dev_norm2(g, g->b, 1, n, &g->ds->rnorm2, s));
    TRY(sync_scalars(g, s));
    const double bnorm = sqrt(g->hs->rnorm2);
    o->bnorm = bnorm;
    if (!std::isfinite(bnorm)) {
        set_error("GMRES: non-finite right-hand side");
        return MUSIC_E_NONFINITE;
    }
    if (bnorm == 0.0) {
        o->converged = 1;
        return MUSIC_OK;
    }
    const double target = rtol * bnorm;
    double H[MUSIC_MAXV][MUSIC_MAXV];  // H[i][j]
    double cs[MUSIC_MAXV], sn[MUSIC_MAXV], gv[MUSIC_MAXV + 1], y[MUSIC_MAXV];
    double resid = bnorm;
    for (int cycle = 0; cycle <= g->desc.gmres_max_restarts; cycle++) {
        const double *r = g->b;
        double beta = bnorm;
        if (cycle > 0) {
            // r = b - J x  (J x in FP64)
            TRY(jv_apply(g, g->x, 1, g->t64, 1, dt, 1, s));
            TRY(vec_sub(g, g->b, g->t64, g->t64, s));
            r = g->t64;
            TRY(dev_norm2(g, r, 1, n, &g->ds->rnorm2, s));
            TRY(sync_scalars(g, s));
            beta = sqrt(g->hs->rnorm2);
        }
        if (!std::isfinite(beta)) {
            set_error("GMRES: non-finite residual");
            return MUSIC_E_NONFINITE;
        }
        resid = beta;
        if (beta <= target) {
            if (guard.over()) return loop_timeout();
            o->converged = 1;
            break;
        }
        TRY(krylov_first(g, r, beta, s));
        for (int i = 0; i <= m; i++) gv[i] = 0.0;
        gv[0] = beta;
        int k = 0;
        for (int j = 0; j < m; j++) {
            void *Vj = (char *)g->V + (size_t)j * n * ks;
            TRY(precond_apply(g, dt, Vj, g->z, 1, s));
            TRY(jv_apply(g, g->z, kd, g->w, kd, dt, 0, s));
            TRY(krylov_dots(g, j, nullptr, s));
            TRY(krylov_update_dots(g, j, nullptr, s));
            TRY(krylov_update_norm(g, j, nullptr, s));
            TRY(sync_scalars(g, s));
            const DevScalars *hs = g->hs;
            const double hn = sqrt(hs->wnorm2);
            if (!std::isfinite(hn)) {
                set_error("GMRES: non-finite Arnoldi vector");
                return MUSIC_E_NONFINITE;
            }
            if (guard.over()) return loop_timeout();
            for (int i = 0; i <= j; i++) H[i][j] = hs->h[i] + hs->h2[i];
            H[j + 1][j] = hn;
            for (int i = 0; i < j; i++) {
                const double t0 = H[i][j], t1 = H[i + 1][j];
                H[i][j] = cs[i] * t0 + sn[i] * t1;
                H[i + 1][j] = -sn[i] * t0 + cs[i] * t1;
            }
            const double a0 = H[j][j], a1 = H[j + 1][j];
            if (a1 == 0.0) {
                cs[j] = 1.0;
                sn[j] = 0.0;
            } else {
                const double t = sqrt(a0 * a0 + a1 * a1);
                cs[j] = a0 / t;
                sn[j] = a1 / t;
            }
            H[j][j] = cs[j] * a0 + sn[j] * a1;
            H[j + 1][j] = 0.0;
            gv[j + 1] = -sn[j] * gv[j];
            gv[j] = cs[j] * gv[j];
            o->its++;
            k = j + 1;
            resid = fabs(gv[j + 1]);
            if (hn == 0.0 || resid <= target) break;
            TRY(krylov_scale(g, j, 1.0 / hn, s));
        }
        for (int i = k - 1; i >= 0; i--) {
            double t = gv[i];
            for (int l = i + 1; l < k; l++) t -= H[i][l] * y[l];
            y[i] = t / H[i][i];
        }
        // x += M^-1 V y as sum_i y_i Z_i: M^-1 (a fixed number of sweeps from
        // zero) is linear, and Z_i = M^-1 V_i is stored by each Arnoldi step
        TRY(krylov_correct(g, k, y, nullptr, nullptr, s));
        if (guard.over()) return loop_timeout();
        if (resid <= target) {
            o->converged = 1;
            break;
        }
    }
    return MUSIC_OK;
}

// The stencil call `call`, with its face mass fluxes captured for the
// passive scalars when the grid has any.
template <typename F>
int with_fluxes(music_grid *g, F &&call)
{
    if (g->ns > 0) g->fr_capture = g->sfr;
    const int rc = call();
    g->fr_capture = nullptr;
    return rc;
}

// Swaps the scalar solve space in for its lifetime.
struct ScalarSpace {
    music_grid *g;
    explicit ScalarSpace(music_grid *g_) : g(g_) { swap_space(g); }
    ~ScalarSpace() { swap_space(g); }
};

// One Newton iteration of the passive scalars (Sec. 2.2) with the fluid
// frozen at its current iterate, whose face mass fluxes are in g->sfr:
// b = -((q - C_s) - dt/2 S(q)), unpreconditioned GMRES, q += x.  *maxdq
// receives max |delta q| / rho.
int scalar_iteration(music_grid *g, double dt, music_step_stats *st, double *maxdq, LoopGuard &guard,
                     cudaStream_t s)
{
    g->srho = g->U;  // the fluid iterate's density plane
    ScalarSpace sp(g);
    TRY(stencil_apply(g, SM_F, g->U, g->sq_c, nullptr, 1, g->b, 1, g->RU, dt, -1.0, s));
    TRY(dev_norm2(g, g->U, 1, g->n, &g->ds->unorm2, s));
    GmresOut go;
    TRY(gmres(g, dt, &go, guard, s));
    st->scalar_gmres_its += go.its;
    TRY(scalar_update(g, s));
    TRY(sync_scalars(g, s));
    *maxdq = g->hs->maxdrho;
    return MUSIC_OK;
}

// One Newton solve of size dt from the grid's state.  Returns MUSIC_OK,
// MUSIC_E_NEWTON_FAIL (state restored) or a hard error.
int newton_attempt(music_grid *g, double dt, music_step_stats *st, cudaStream_t s)
{
    const size_t n = g->n;
    const size_t nq = g->sc.n;
    CUDA_TRY(cudaMemcpyAsync(g->Un, g->U, n * sizeof(double), cudaMemcpyDeviceToDevice, s));

    // Without scalars one evaluation of R(U^n) gives the step constant C^n and
    // the first iteration's residual (U = U^n there); with them the scalars'
    // flux captures keep the two evaluations apart.
    const bool cnf = (g->ns == 0);
    if (cnf)
        TRY(stencil_apply(g, SM_CNF, g->U, g->Cn, nullptr, 1, g->b, 1, g->RU, dt, -1.0, s));
    else
        TRY(with_fluxes(g, [&] { return stencil_apply(g, SM_CN, g->Un, nullptr, nullptr, 1, g->Cn, 1, nullptr, dt,
                                                      1.0, s); }));
    // |U|^2 for the products' eps: here for U^n, then by every Newton update
    TRY(dev_norm2(g, g->U, 1, n, &g->ds->unorm2, s));
    if (g->ns > 0) {
        // scalar step constant C_s = q^n + dt/2 S(q^n) with the fluid at U^n
        CUDA_TRY(cudaMemcpyAsync(g->sq_n, g->sc.U, nq * sizeof(double), cudaMemcpyDeviceToDevice, s));
        g->srho = g->Un;
        TRY(scalar_apply(g, SM_CN, g->sq_n, nullptr, nullptr, 1, g->sq_c, 1, nullptr, dt, 1.0, s));
    }
    st->newton_its = 0;
    st->gmres_its = 0;
    st->gmres_unconverged = 0;
    st->scalar_gmres_its = 0;
    int ok = 0;
    LoopGuard guard{0, loop_cap_of(g)};
    for (int k = 0; k < g->desc.newton_max_its; k++) {
        // b = -F(U), RU = R(U) (and the face mass fluxes of U for the scalars)
        if (!(cnf && k == 0))
            TRY(with_fluxes(g, [&] { return stencil_apply(g, SM_F, g->U, g->Cn, nullptr, 1, g->b, 1, g->RU, dt,
                                                          -1.0, s); }));
        double maxdq = 0.0;
        if (g->ns > 0) TRY(scalar_iteration(g, dt, st, &maxdq, guard, s));
        TRY(precond_setup(g, g->U, dt, s));
        GmresOut go;
        int rc = gmres(g, dt, &go, guard, s);
        if (rc != MUSIC_OK) return rc;
        st->gmres_its += go.its;
        st->gmres_unconverged += !go.converged;
        st->fnorm = go.bnorm;  // |F(U^k)|
        if (k == 0) st->fnorm0 = st->fnorm;
        TRY(newton_update(g, nullptr, s));
        TRY(sync_scalars(g, s));
        st->max_drho = g->hs->maxdrho;
        st->newton_its = k + 1;
        if (guard.over()) return loop_timeout();
        if (g->hs->maxdrho <= g->desc.newton_tol && (!g->desc.scalar_enforce || maxdq <= g->desc.newton_tol)) {
            ok = 1;
            break;
        }
        if (!std::isfinite(g->hs->maxdrho)) break;
    }
    if (!ok) {
        CUDA_TRY(cudaMemcpyAsync(g->U, g->Un, n * sizeof(double), cudaMemcpyDeviceToDevice, s));
        if (g->ns > 0)
            CUDA_TRY(cudaMemcpyAsync(g->sc.U, g->sq_n, nq * sizeof(double), cudaMemcpyDeviceToDevice, s));
        CUDA_TRY(cudaStreamSynchronize(s));
        return MUSIC_E_NEWTON_FAIL;
    }
    if (g->ns > 0) TRY(scalar_renormalise(g, g->U, s));
    return MUSIC_OK;
}

}  // namespace

// J v for the current Newton iterate: v (Krylov type, or FP64 when
// vin_double) -> out.  eps from |U| (ds->unorm2) and |v|.
int jv_apply(music_grid *g, const void *v, int vin_double, void *out, int out_double, double dt,
             int need_vnorm, cudaStream_t s)
{
    // eps comes with |v|: computed here, or already by the preconditioner
    if (need_vnorm) {
        TRY(dev_norm2(g, v, vin_double, g->n, &g->ds->vnorm2, s));
        TRY(dev_set_eps(g, 0.0, s));
    }
    return stencil_apply(g, SM_JV, g->U, g->RU, v, vin_double, out, out_double, nullptr, dt, 1.0, s);
}

// ---- timing of the Jacobian-free stencil (CUDA events on the launch stream)
int prof_begin_cls(music_grid *g, int cls, cudaStream_t s)
{
    if (!g->prof_events_made) {
        for (int i = 0; i < 2 * 256; i++) CUDA_TRY(cudaEventCreate(&g->prof_ev[i]));
        g->prof_events_made = 1;
    }
    if (g->prof_pending == 256) TRY(prof_harvest(g, 1));
    g->prof_cls[g->prof_pending] = cls;
    CUDA_TRY(cudaEventRecord(g->prof_ev[2 * g->prof_pending], s));
    return MUSIC_OK;
}

int prof_end(music_grid *g, cudaStream_t s)
{
    CUDA_TRY(cudaEventRecord(g->prof_ev[2 * g->prof_pending + 1], s));
    g->prof_pending++;
    return MUSIC_OK;
}

// Accumulate the recorded pairs; with wait = 0 only after they completed
// (the caller has synchronised the stream), with wait = 1 it waits for them.
int prof_harvest(music_grid *g, int wait)
{
    for (int i = 0; i < g->prof_pending; i++) {
        if (wait) CUDA_TRY(cudaEventSynchronize(g->prof_ev[2 * i + 1]));
        float ms = 0.0f;
        CUDA_TRY(cudaEventElapsedTime(&ms, g->prof_ev[2 * i], g->prof_ev[2 * i + 1]));
        g->prof_ms[g->prof_cls[i]] += ms;
        g->prof_launches[g->prof_cls[i]]++;
    }
    g->prof_pending = 0;
    return MUSIC_OK;
}

bool graph_driven(const music_grid *g)
{
    return g->solver_variant == SOLVER_GRAPH && !g->prof_on && g->ns == 0;
}

int newton_solve(music_grid *g, double dt, music_step_stats *st_out, cudaStream_t s, const music_dt_limits *lim)
{
    auto t0 = std::chrono::steady_clock::now();
    music_step_stats st;
    memset(&st, 0, sizeof(st));
    int rc = MUSIC_E_NEWTON_FAIL;
    int h = 0;
    for (;;) {
        st.dt = dt;
        if (graph_driven(g)) {
            // the first attempt may choose its dt on the device (st.dt receives it)
            rc = graph_newton_attempt(g, dt, &st, s, h == 0 ? lim : nullptr);
            dt = st.dt;
        } else {
            rc = newton_attempt(g, dt, &st, s);
        }
        if (rc == MUSIC_E_TIMEOUT) {
            // an attempt stopped by the loop-body bound leaves a partial
            // iterate: restore U^n (and the scalars) as a failed attempt does
            CUDA_TRY(cudaMemcpyAsync(g->U, g->Un, g->n * sizeof(double), cudaMemcpyDeviceToDevice, s));
            if (g->ns > 0)
                CUDA_TRY(cudaMemcpyAsync(g->sc.U, g->sq_n, g->sc.n * sizeof(double), cudaMemcpyDeviceToDevice, s));
            CUDA_TRY(cudaStreamSynchronize(s));
            break;
        }
        if (rc != MUSIC_E_NEWTON_FAIL) break;
        if (h >= g->desc.max_dt_halvings) break;
        dt *= 0.5;
        h++;
    }
    st.dt_halvings = h;
    st.wall_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    if (st_out) *st_out = st;
    if (rc == MUSIC_E_NEWTON_FAIL) set_error("Newton did not converge after %d dt halvings", h);
    return rc;
}
