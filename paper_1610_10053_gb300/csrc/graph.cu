// One Newton attempt of the implicit step (Sec. 2: Newton-Raphson on the
// Crank-Nicolson system, restarted right-preconditioned GMRES with
// Jacobian-free products) recorded once per grid as a CUDA graph and replayed
// for every attempt.  The Newton loop, the Arnoldi loop of each GMRES cycle
// and the loop over restarted cycles are conditional WHILE nodes, the next
// iteration's residual an IF node; tiny single-thread control kernels run the
// Givens rotations and the stopping tests and set the loop conditions, so an
// attempt needs no host round trip until it ends.  The first cycle of a solve
// sits in the Newton body itself (a solve rarely restarts, and every
// conditional node a body enters costs several microseconds); a cycle that
// builds no basis leaves its kernels to return at once on a device flag.  The vector kernels are the same as those of the
// host-sequenced attempt in solver.cu, and so is every floating-point
// operation (the control kernels use explicitly rounded, uncontracted
// arithmetic to match the host), so both drivers give identical results.
//
// Every loop is bounded by its own counter (m Arnoldi steps, max_restarts + 1
// cycles, newton_max iterations); a cap on the total number of loop bodies
// backs those bounds up and ends the attempt with MUSIC_E_TIMEOUT.
#include <cmath>
#include <cstddef>
#include <cstdlib>
#include <cstring>
#include <vector>

#include "internal.h"
#include "ctl.cuh"

namespace {

constexpr int BS = 256;

// ------------------------------------------------------------ control kernels
// All run with one thread, and each handle has one setter: these kernels, or
// (the Arnoldi loop's) thread 0 of the norm pass's last block, which runs
// ctl_givens.

// dt of the attempt from the rates at U^n (ds->rate, rate_adv, rate_rad) and
// the limits: the most restrictive cfl_k / rate_k over the limits set (> 0)
// with a positive rate, capped by dt_max > 0 — music_select_dt's choice, in
// the same correctly rounded FP64 operations.  A non-finite rate, or no
// limit that applies, leaves dt_status set and the attempt does nothing.
__global__ void k_ctl_dt(SolveCtl *c, const DevScalars *ds, double cfl_h, double cfl_a, double cfl_r, double dt_max)
{
    pdl_entry();
    const double rates[3] = {ds->rate, ds->rate_adv, ds->rate_rad};
    const double cfl[3] = {cfl_h, cfl_a, cfl_r};
    double best = __longlong_as_double(0x7ff0000000000000LL);  // +infinity
    int w = -1, status = MUSIC_OK;
    for (int k = 0; k < 3; k++) {
        if (!isfinite(rates[k])) {
            status = MUSIC_E_NONFINITE;
            break;
        }
        if (!(cfl[k] > 0.0) || !(rates[k] > 0.0)) continue;
        const double t = __ddiv_rn(cfl[k], rates[k]);
        if (t < best) {
            best = t;
            w = k;
        }
    }
    if (status == MUSIC_OK && dt_max > 0.0 && dt_max < best) {
        best = dt_max;
        w = 3;
    }
    if (status == MUSIC_OK && w < 0) status = MUSIC_E_INVAL;
    c->dt = best;
    c->dt_which = w;
    c->dt_status = status;
}

__global__ void k_ctl_attempt(SolveCtl *c, cudaGraphConditionalHandle h_newton, int newton_max)
{
    pdl_entry();
    c->newton_it = 0;
    c->newton_its = 0;
    c->gmres_its = 0;
    c->unconverged = 0;
    c->cycles = 0;
    c->restarts = 0;
    c->solves = 0;
    c->fnorm0 = 0.0;
    c->fnorm = 0.0;
    c->maxdrho = 0.0;
    c->status = MUSIC_OK;
    c->stop = 0;
    c->ok = 0;
    c->guard = 0;
    // no dt (the device-side choice found none): no Newton iteration
    cudaGraphSetConditional(h_newton, (newton_max > 0 && c->dt_status == MUSIC_OK) ? 1u : 0u);
}

// GMRES set-up after |b|^2 -> ds->rnorm2 (b = -F(U), x = 0), and the start
// of its first cycle (beta = |b|): the condition of that cycle's Arnoldi loop
__global__ void k_ctl_gmres(SolveCtl *c, const DevScalars *ds, cudaGraphConditionalHandle h_arnoldi, double rtol,
                            int m)
{
    pdl_entry();
    const double bnorm = sqrt(ds->rnorm2);
    c->bnorm = bnorm;
    c->its = 0;
    c->converged = 0;
    c->cycle = 0;
    c->j = 0;
    c->k = 0;
    c->scale = 0;
    c->resid = bnorm;
    c->target = __dmul_rn(rtol, bnorm);
    c->go = 0;
    c->nocycle = 0;
    if (!isfinite(bnorm)) {
        c->status = MUSIC_E_NONFINITE;
        c->stop = 1;
        c->nocycle = 1;
    } else if (bnorm == 0.0) {
        c->converged = 1;
        c->nocycle = 1;
    } else {
        c->cycles++;
        c->beta = bnorm;
        if (!(bnorm <= c->target)) {
            c->go = 1;
            for (int i = 0; i <= m; i++) c->gv[i] = 0.0;
            c->gv[0] = bnorm;
            c->solves++;
        }
    }
    cudaGraphSetConditional(h_arnoldi, c->go ? 1u : 0u);
}

// a cycle after the first starts from the true residual b - J x
__global__ void k_ctl_cycle_pre(SolveCtl *c)
{
    pdl_entry();
    c->cycles++;
    c->restarts++;
}

// beta = |b - J x| (ds->rnorm2) of a restarted cycle; build its basis (the
// condition of its Arnoldi loop) or stop
__global__ void k_ctl_cycle_start(SolveCtl *c, const DevScalars *ds, cudaGraphConditionalHandle h_arnoldi, int m)
{
    pdl_entry();
    const double beta = sqrt(ds->rnorm2);
    c->beta = beta;
    c->j = 0;
    c->k = 0;
    c->scale = 0;
    c->go = 0;
    if (!isfinite(beta)) {
        c->status = MUSIC_E_NONFINITE;
        c->stop = 1;
    } else {
        c->resid = beta;
        if (!(beta <= c->target)) {
            c->go = 1;
            for (int i = 0; i <= m; i++) c->gv[i] = 0.0;
            c->gv[0] = beta;
            c->solves++;
        }
    }
    cudaGraphSetConditional(h_arnoldi, c->go ? 1u : 0u);
}

// y from the k x k upper triangle: H y = g
__global__ void k_ctl_solve(SolveCtl *c)
{
    pdl_entry();
    constexpr int L = MUSIC_MAXV;
    const int k = c->k;
    for (int i = k - 1; i >= 0; i--) {
        double t = c->gv[i];
        for (int l = i + 1; l < k; l++) t = __dsub_rn(t, __dmul_rn(c->H[i * L + l], c->y[l]));
        c->y[i] = __ddiv_rn(t, c->H[i * L + i]);
    }
}

__global__ void k_ctl_cycle_end(SolveCtl *c, cudaGraphConditionalHandle h_cycle, int max_restarts, int cap)
{
    pdl_entry();
    unsigned go = 0u;
    if (!c->nocycle && !c->stop && !over_cap(c, cap)) {
        if (c->resid <= c->target) {
            c->converged = 1;
        } else {
            c->cycle++;
            go = c->cycle <= max_restarts ? 1u : 0u;
        }
    }
    cudaGraphSetConditional(h_cycle, go);
}

// after the update U += x: statistics and the density-correction test
__global__ void k_ctl_newton(SolveCtl *c, const DevScalars *ds, cudaGraphConditionalHandle h_newton,
                             cudaGraphConditionalHandle h_next, int newton_max, double tol, int cap)
{
    pdl_entry();
    unsigned go = 0u;
    if (!c->stop && !over_cap(c, cap)) {
        c->gmres_its += c->its;
        c->unconverged += c->converged ? 0 : 1;
        c->fnorm = c->bnorm;
        if (c->newton_it == 0) c->fnorm0 = c->bnorm;
        const double md = ds->maxdrho;
        c->maxdrho = md;
        c->newton_it++;
        c->newton_its = c->newton_it;
        if (md <= tol)
            c->ok = 1;
        else if (isfinite(md) && c->newton_it < newton_max)
            go = 1u;
    }
    cudaGraphSetConditional(h_newton, go);
    cudaGraphSetConditional(h_next, go);  // the next iteration's residual, when there is one
}

// --------------------------------------------------------------- vector kernels
// V_0 = r / beta, r = b on the first cycle and b - J x after a restart; the
// same values go to q, the fixed-address copy the preconditioner reads.
// With fold (the preconditioner takes the scaling, precond_folds_scale) it
// writes r to w unscaled instead, and 1 / beta and index 0 as the scaling
// the preconditioner applies and stores.
template <typename KT>
__global__ void __launch_bounds__(BS) k_first_dev(const double *b, const double *t64, KT *V, KT *q, long long n,
                                                  SolveCtl *c, KT *w, int fold)
{
    pdl_entry();
    if (!c->go) return;  // the cycle builds no basis
    const double *r = c->cycle == 0 ? b : t64;
    if (fold) {
        for (long long e = blockIdx.x * (long long)BS + threadIdx.x; e < n; e += (long long)gridDim.x * BS)
            w[e] = (KT)r[e];
        if (blockIdx.x == 0 && threadIdx.x == 0) {
            c->inv = 1.0 / c->beta;
            c->scale_idx = 0;
        }
        return;
    }
    // r / beta as r times 1 / beta (formed once per CTA), as the host driver does
    __shared__ KT s_rinv;
    if (threadIdx.x == 0) s_rinv = (KT)(1.0 / c->beta);
    __syncthreads();
    const KT rinv = s_rinv;
    const long long stride = (long long)gridDim.x * BS, t0 = blockIdx.x * (long long)BS + threadIdx.x;
    long long e0 = t0;
    if constexpr (sizeof(KT) == 4) {
        // four elements a step when the vectors start 16-byte aligned
        const long long n4 = (n & 3) ? 0 : (n >> 2);
        for (long long e = t0; e < n4; e += stride) {
            const double2 a = reinterpret_cast<const double2 *>(r)[2 * e], b = reinterpret_cast<const double2 *>(r)[2 * e + 1];
            const float4 v = make_float4((float)a.x * rinv, (float)a.y * rinv, (float)b.x * rinv, (float)b.y * rinv);
            reinterpret_cast<float4 *>(V)[e] = v;
            reinterpret_cast<float4 *>(q)[e] = v;
        }
        e0 = 4 * n4 + t0;
    }
    for (long long e = e0; e < n; e += stride) {
        const KT v = (KT)r[e] * rinv;
        V[e] = v;
        q[e] = v;
    }
}

// V_{j+1} = w / h_{j+1,j} (and q) when the Arnoldi step asked for it
template <typename KT>
__global__ void __launch_bounds__(BS) k_scale_dev(const KT *w, KT *V, KT *q, long long n, const SolveCtl *c)
{
    pdl_entry();
    if (!c->scale) return;
    KT *dst = V + (long long)c->scale_idx * n;
    const KT inv = (KT)c->inv;
    const long long stride = (long long)gridDim.x * BS, t0 = blockIdx.x * (long long)BS + threadIdx.x;
    long long e0 = t0;
    if constexpr (sizeof(KT) == 4) {
        // four elements a step when the vectors start 16-byte aligned
        const long long n4 = (n & 3) ? 0 : (n >> 2);
        for (long long e = t0; e < n4; e += stride) {
            const float4 a = reinterpret_cast<const float4 *>(w)[e];
            const float4 v = make_float4(a.x * inv, a.y * inv, a.z * inv, a.w * inv);
            reinterpret_cast<float4 *>(dst)[e] = v;
            reinterpret_cast<float4 *>(q)[e] = v;
        }
        e0 = 4 * n4 + t0;
    }
    for (long long e = e0; e < n; e += stride) {
        const KT v = w[e] * inv;
        dst[e] = v;
        q[e] = v;
    }
}

}  // namespace

namespace {

// The capture graph of stream s and its current dependencies.
int capture_info(cudaStream_t s, cudaGraph_t *graph, const cudaGraphNode_t **deps, size_t *ndeps)
{
    cudaStreamCaptureStatus st;
    CUDA_TRY(cudaStreamGetCaptureInfo(s, &st, nullptr, graph, deps, nullptr, ndeps));
    if (st != cudaStreamCaptureStatusActive) {
        set_error("solver graph: stream is not capturing");
        return MUSIC_E_CUDA;
    }
    return MUSIC_OK;
}

// A handle for a conditional node that will follow in the graph captured on s.
int new_handle(cudaStream_t s, cudaGraphConditionalHandle *h)
{
    cudaGraph_t graph;
    const cudaGraphNode_t *deps;
    size_t nd;
    TRY(capture_info(s, &graph, &deps, &nd));
    CUDA_TRY(cudaGraphConditionalHandleCreate(h, graph, 0, 0));
    return MUSIC_OK;
}

// Append a conditional node after everything captured on s so far; later
// work on s follows it.  *body receives the graph it runs.
int add_conditional(cudaStream_t s, cudaGraphConditionalHandle h, cudaGraphConditionalNodeType type,
                    cudaGraph_t *body)
{
    cudaGraph_t graph;
    const cudaGraphNode_t *deps;
    size_t nd;
    TRY(capture_info(s, &graph, &deps, &nd));
    cudaGraphNodeParams p = {};
    p.type = cudaGraphNodeTypeConditional;
    p.conditional.handle = h;
    p.conditional.type = type;
    p.conditional.size = 1;
    cudaGraphNode_t node;
    CUDA_TRY(cudaGraphAddNode(&node, graph, deps, nullptr, nd, &p));
    CUDA_TRY(cudaStreamUpdateCaptureDependencies(s, &node, nullptr, 1, cudaStreamSetCaptureDependencies));
    *body = p.conditional.phGraph_out[0];
    return MUSIC_OK;
}

// record_attempt's status when the driver refuses the programmatic edges
constexpr int PDL_REFUSED = 1000;

// Every kernel-to-kernel edge of graph gr made programmatic: the downstream
// kernel may launch as the upstream's blocks exit, ahead of the upstream's
// completion, and waits for that completion (pdl_entry) before it reads
// anything, so its launch overlaps the upstream's tail.
int programmatic_edges(cudaGraph_t gr)
{
    size_t ne = 0;
    CUDA_TRY(cudaGraphGetEdges(gr, nullptr, nullptr, nullptr, &ne));
    if (ne == 0) return MUSIC_OK;
    std::vector<cudaGraphNode_t> from(ne), to(ne);
    std::vector<cudaGraphEdgeData> ed(ne);
    CUDA_TRY(cudaGraphGetEdges(gr, from.data(), to.data(), ed.data(), &ne));
    for (size_t i = 0; i < ne; i++) {
        cudaGraphNodeType a, b;
        CUDA_TRY(cudaGraphNodeGetType(from[i], &a));
        CUDA_TRY(cudaGraphNodeGetType(to[i], &b));
        if (a != cudaGraphNodeTypeKernel || b != cudaGraphNodeTypeKernel || ed[i].type != cudaGraphDependencyTypeDefault ||
            ed[i].from_port != cudaGraphKernelNodePortDefault)
            continue;
        cudaGraphEdgeData pe;
        memset(&pe, 0, sizeof(pe));
        pe.from_port = cudaGraphKernelNodePortProgrammatic;
        pe.type = cudaGraphDependencyTypeProgrammatic;
        CUDA_TRY(cudaGraphRemoveDependencies(gr, &from[i], &to[i], &ed[i], 1));
        CUDA_TRY(cudaGraphAddDependencies(gr, &from[i], &to[i], &pe, 1));
    }
    return MUSIC_OK;
}

// Streams capturing nested bodies; every capture still open when recording
// fails is ended (innermost first) so the streams stay usable.
// Streams 5 and 6 only join captures (side branches forked by events).
struct Capture {
    cudaStream_t st[7] = {};
    bool open[5] = {};
    cudaEvent_t ev[4] = {};
    std::vector<cudaGraph_t> bodies;  // the conditional nodes' body graphs
    ~Capture()
    {
        for (int i = 4; i >= 0; i--) {
            if (open[i]) {
                cudaGraph_t gr = nullptr;
                cudaStreamEndCapture(st[i], &gr);
                if (gr && i == 0) cudaGraphDestroy(gr);
            }
        }
        for (int i = 6; i >= 0; i--)
            if (st[i]) cudaStreamDestroy(st[i]);
        for (cudaEvent_t e : ev)
            if (e) cudaEventDestroy(e);
        cudaGetLastError();
    }
    int begin_body(int i, cudaGraph_t body)
    {
        CUDA_TRY(cudaStreamBeginCaptureToGraph(st[i], body, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed));
        open[i] = true;
        return MUSIC_OK;
    }
    int end_body(int i)
    {
        open[i] = false;
        CUDA_TRY(cudaStreamEndCapture(st[i], nullptr));
        return MUSIC_OK;
    }
};

// kernels launched by this thread since `from`
long long since(long long from) { return capture_launches() - from; }

// The preconditioner's coefficients at U on side stream a, forked from s
// with event ef: they depend on U alone, so they overlap the residual
// evaluation that s runs next (FP64-bound, while the set-up is a memory
// pass).  join() merges the branch back into s.
int fork_setup(music_grid *g, cudaStream_t s, cudaStream_t a, cudaEvent_t ef, double dt)
{
    CUDA_TRY(cudaEventRecord(ef, s));
    CUDA_TRY(cudaStreamWaitEvent(a, ef, 0));
    return precond_setup(g, g->U, dt, a);
}

int join(cudaStream_t s, cudaStream_t a, cudaEvent_t ej)
{
    CUDA_TRY(cudaEventRecord(ej, a));
    CUDA_TRY(cudaStreamWaitEvent(s, ej, 0));
    return MUSIC_OK;
}

// One GMRES cycle on stream s (capturing body level `lvl`): the first basis
// vector, the Arnoldi loop (WHILE on hA, set by the cycle's start), the
// small solve and the correction x += M^-1 V y.  The Arnoldi body's kernels
// per step go to g->glaunch[5].
int record_cycle(music_grid *g, Capture &C, cudaStream_t s, int lvl, cudaGraphConditionalHandle hA, SolveCtl *ctl,
                 int nb, int fold, int cap, int m)
{
    const long long n = (long long)g->n;
    const int kd = !g->mixed;
    const double dt = 1.0;  // every recorded kernel reads dt from g->ctl->dt instead
    DevScalars *ds = g->ds;
    cudaStream_t sa = C.st[lvl + 1];
    if (g->mixed)
        k_first_dev<float><<<nb, BS, 0, s>>>(g->b, g->t64, (float *)g->V, (float *)g->q, n, ctl, (float *)g->w, fold);
    else
        k_first_dev<double><<<nb, BS, 0, s>>>(g->b, g->t64, (double *)g->V, (double *)g->q, n, ctl, (double *)g->w,
                                              fold);
    CHECK_LAUNCH();
    cudaGraph_t bA;
    TRY(add_conditional(s, hA, cudaGraphCondTypeWhile, &bA));
    C.bodies.push_back(bA);
    {
        TRY(C.begin_body(lvl + 1, bA));
        const long long a0 = capture_launches();
        // on grids whose preconditioner takes the scaling of the next basis
        // vector, it reads w and writes V_j (no scaling pass)
        if (fold) {
            g->pc_scale = ctl;
            const int rc = precond_apply(g, dt, g->w, g->z, 1, sa);
            g->pc_scale = nullptr;
            TRY(rc);
        } else {
            TRY(precond_apply(g, dt, g->q, g->z, 1, sa));
        }
        TRY(jv_apply(g, g->z, kd, g->w, kd, dt, 0, sa));
        // the last block of the norm pass runs the Givens rotations
        const GivensCtl gc{ctl, ds, hA, m, cap};
        TRY(krylov_dots(g, m - 1, &ctl->j, sa));
        TRY(krylov_update_dots(g, m - 1, &ctl->j, sa));
        TRY(krylov_update_norm(g, m - 1, &ctl->j, sa, &gc));
        if (!fold) {
            if (g->mixed)
                k_scale_dev<float><<<nb, BS, 0, sa>>>((const float *)g->w, (float *)g->V, (float *)g->q, n, ctl);
            else
                k_scale_dev<double><<<nb, BS, 0, sa>>>((const double *)g->w, (double *)g->V, (double *)g->q, n,
                                                       ctl);
            CHECK_LAUNCH();
        }
        g->glaunch[5] = since(a0);
        TRY(C.end_body(lvl + 1));
    }
    k_ctl_solve<<<1, 1, 0, s>>>(ctl);
    CHECK_LAUNCH();
    TRY(krylov_correct(g, 0, nullptr, &ctl->k, ctl->y, s));
    return MUSIC_OK;
}

int record(music_grid *g, Capture &C, cudaGraph_t *out)
{
    const music_grid_desc &d = g->desc;
    const int m = d.gmres_restart;
    const long long n = (long long)g->n;
    const int nb = (int)((n + BS - 1) / BS < 152 * 16 ? (n + BS - 1) / BS : 152 * 16);
    const int cap = loop_cap_of(g);
    const double dt = 1.0;  // every recorded kernel reads dt from g->ctl->dt instead
    // on grids whose preconditioner takes the scaling of the next basis
    // vector, it reads w and writes V_j (no scaling pass)
    const int fold = precond_folds_scale(g) ? 1 : 0;
    SolveCtl *ctl = g->ctl;
    DevScalars *ds = g->ds;
    cudaStream_t s0 = C.st[0], s1 = C.st[1], s2 = C.st[2];
    cudaStream_t sa0 = C.st[5], sa2 = C.st[6];
    cudaGraph_t bN, bC, bF;
    cudaGraphConditionalHandle hN, hC, hA, hA2, hF;
    long long t0;
    g->glaunch[3] = g->glaunch[4] = 0;

    CUDA_TRY(cudaStreamBeginCapture(s0, cudaStreamCaptureModeRelaxed));
    C.open[0] = true;
    // ---- attempt: U^n; the step constant C^n with the first residual b = -F(U^n)
    // and R(U^n) from one evaluation; then the Newton loop, each iteration
    // closed by the residual of the next (an IF node, skipped after the last)
    t0 = capture_launches();
    CUDA_TRY(cudaMemcpyAsync(g->Un, g->U, n * sizeof(double), cudaMemcpyDeviceToDevice, s0));
    TRY(fork_setup(g, s0, sa0, C.ev[0], dt));
    TRY(stencil_apply(g, SM_CNF, g->U, g->Cn, nullptr, 1, g->b, 1, g->RU, dt, -1.0, s0));
    // |U^n|^2 for the products' eps (each Newton update forms the next one)
    TRY(dev_norm2(g, g->U, 1, (size_t)n, &ds->unorm2, s0));
    TRY(join(s0, sa0, C.ev[1]));
    TRY(new_handle(s0, &hN));
    k_ctl_attempt<<<1, 1, 0, s0>>>(ctl, hN, d.newton_max_its);
    CHECK_LAUNCH();
    g->glaunch[0] = since(t0);
    TRY(add_conditional(s0, hN, cudaGraphCondTypeWhile, &bN));
    C.bodies.push_back(bN);
    {
        // ---- Newton iteration (b = -F(U), R(U), |U| and the preconditioner's
        // coefficients at U ready): |b|
        TRY(C.begin_body(1, bN));
        t0 = capture_launches();
        CUDA_TRY(cudaMemsetAsync(g->x, 0, n * sizeof(double), s1));
        TRY(dev_norm2(g, g->b, 1, (size_t)n, &ds->rnorm2, s1));
        // the first cycle (beta = |b|): its Arnoldi loop's condition comes
        // from the set-up, its kernels return at once when it builds no basis
        TRY(new_handle(s1, &hA));
        k_ctl_gmres<<<1, 1, 0, s1>>>(ctl, ds, hA, d.gmres_rtol, m);
        CHECK_LAUNCH();
        TRY(record_cycle(g, C, s1, 2, hA, ctl, nb, fold, cap, m));
        TRY(new_handle(s1, &hC));
        k_ctl_cycle_end<<<1, 1, 0, s1>>>(ctl, hC, d.gmres_max_restarts, cap);
        CHECK_LAUNCH();
        long long nN = since(t0) - g->glaunch[5];  // the Arnoldi body is counted per step
        TRY(add_conditional(s1, hC, cudaGraphCondTypeWhile, &bC));
        C.bodies.push_back(bC);
        {
            // ---- a restarted cycle: t64 = b - J x, |t64|^2, then as the first
            TRY(C.begin_body(2, bC));
            const long long r0 = capture_launches();
            k_ctl_cycle_pre<<<1, 1, 0, s2>>>(ctl);
            CHECK_LAUNCH();
            TRY(jv_apply(g, g->x, 1, g->t64, 1, dt, 1, s2));
            TRY(vec_sub(g, g->b, g->t64, g->t64, s2));
            TRY(dev_norm2(g, g->t64, 1, (size_t)n, &ds->rnorm2, s2));
            TRY(new_handle(s2, &hA2));
            k_ctl_cycle_start<<<1, 1, 0, s2>>>(ctl, ds, hA2, m);
            CHECK_LAUNCH();
            TRY(record_cycle(g, C, s2, 3, hA2, ctl, nb, fold, cap, m));
            k_ctl_cycle_end<<<1, 1, 0, s2>>>(ctl, hC, d.gmres_max_restarts, cap);
            CHECK_LAUNCH();
            g->glaunch[2] = since(r0) - g->glaunch[5];
            TRY(C.end_body(2));
        }
        const long long u0 = capture_launches();
        TRY(newton_update(g, &ctl->stop, s1));
        TRY(new_handle(s1, &hF));
        k_ctl_newton<<<1, 1, 0, s1>>>(ctl, ds, hN, hF, d.newton_max_its, d.newton_tol, cap);
        CHECK_LAUNCH();
        g->glaunch[1] = nN + since(u0);
        TRY(add_conditional(s1, hF, cudaGraphCondTypeIf, &bF));
        C.bodies.push_back(bF);
        {
            // b = -F(U), R(U) and the coefficients of the updated iterate, for
            // the next iteration
            TRY(C.begin_body(2, bF));
            const long long f0 = capture_launches();
            TRY(fork_setup(g, s2, sa2, C.ev[2], dt));
            TRY(stencil_apply(g, SM_F, g->U, g->Cn, nullptr, 1, g->b, 1, g->RU, dt, -1.0, s2));
            TRY(join(s2, sa2, C.ev[3]));
            g->glaunch[6] = since(f0);
            TRY(C.end_body(2));
        }
        TRY(C.end_body(1));
    }
    C.open[0] = false;
    CUDA_TRY(cudaStreamEndCapture(s0, out));
    return MUSIC_OK;
}

int record_attempt(music_grid *g, bool pdl_ok)
{
    if (!g->hctl) CUDA_TRY(cudaMallocHost((void **)&g->hctl, offsetof(SolveCtl, cs)));
    Capture C;
    for (int i = 0; i < 7; i++) CUDA_TRY(cudaStreamCreateWithFlags(&C.st[i], cudaStreamNonBlocking));
    for (int i = 0; i < 4; i++) CUDA_TRY(cudaEventCreateWithFlags(&C.ev[i], cudaEventDisableTiming));
    const long long before = capture_launches();
    const GridParams saved = g->P;
    g->P.dt_dev = &g->ctl->dt;
    cudaGraph_t graph = nullptr;
    const int rc = record(g, C, &graph);
    g->P = saved;
    // recording launches nothing: take the captured kernels off the count
    count_launches(-(capture_launches() - before));
    if (rc != MUSIC_OK) {
        if (graph) cudaGraphDestroy(graph);
        return rc;
    }
    // programmatic launches between consecutive kernels (MUSIC_PDL=0: plain
    // edges); a graph the driver will not instantiate with them is recorded
    // again without
    const char *pv = getenv("MUSIC_PDL");
    const bool pdl = pdl_ok && !(pv && strcmp(pv, "0") == 0);
    int prc = MUSIC_OK;
    if (pdl) {
        prc = programmatic_edges(graph);
        for (cudaGraph_t b : C.bodies)
            if (prc == MUSIC_OK) prc = programmatic_edges(b);
    }
    cudaGraphExec_t exec = nullptr;
    const cudaError_t e = prc == MUSIC_OK ? cudaGraphInstantiate(&exec, graph, 0) : cudaErrorNotSupported;
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) {
        cudaGetLastError();
        if (pdl) return PDL_REFUSED;
        set_error("solver graph: instantiation failed: %s", cudaGetErrorString(e));
        return MUSIC_E_CUDA;
    }
    g->gexec = exec;
    return MUSIC_OK;
}

}  // namespace

void graph_release(music_grid *g)
{
    if (g->gexec) cudaGraphExecDestroy(g->gexec);
    g->gexec = nullptr;
    if (g->hctl) cudaFreeHost(g->hctl);
    g->hctl = nullptr;
}

int graph_newton_attempt(music_grid *g, double dt, music_step_stats *st, cudaStream_t s, const music_dt_limits *lim)
{
    if (!g->gexec) {
        int rc = record_attempt(g, true);
        if (rc == PDL_REFUSED) rc = record_attempt(g, false);
        TRY(rc);
    }
    SolveCtl *h = g->hctl;
    if (lim) {
        // dt chosen on the device from the rates at U^n: no host round trip
        // between the step's start and its graph
        TRY(step_rates(g, s));
        k_ctl_dt<<<1, 1, 0, s>>>(g->ctl, g->ds, lim->cfl_hydro, lim->cfl_adv, lim->cfl_rad, lim->dt_max);
        CHECK_LAUNCH();
    } else {
        h->dt = dt;
        h->dt_status = MUSIC_OK;
        h->dt_which = -1;
        CUDA_TRY(cudaMemcpyAsync(&g->ctl->dt, &h->dt, offsetof(SolveCtl, bnorm), cudaMemcpyHostToDevice, s));
    }
    CUDA_TRY(cudaGraphLaunch(g->gexec, s));
    CUDA_TRY(cudaMemcpyAsync(h, g->ctl, offsetof(SolveCtl, cs), cudaMemcpyDeviceToHost, s));
    CUDA_TRY(cudaStreamSynchronize(s));
    st->dt = h->dt;
    if (h->dt_status == MUSIC_E_NONFINITE) {
        set_error("music_select_dt: non-finite rate");
        return MUSIC_E_NONFINITE;
    }
    if (h->dt_status != MUSIC_OK) {
        set_error("music_select_dt: no limit applies (all <= 0, or the state is at rest)");
        return MUSIC_E_INVAL;
    }
    // kernels the replay ran, from the bodies each loop executed (the closing
    // residual runs after every Newton iteration but the last)
    const long long nextres = h->newton_it > 0 ? h->newton_it - 1 : 0;
    count_launches(g->glaunch[0] + g->glaunch[1] * h->newton_it + g->glaunch[2] * h->restarts +
                   g->glaunch[5] * h->gmres_its + g->glaunch[6] * nextres);
    st->newton_its = h->newton_its;
    st->gmres_its = h->gmres_its;
    st->gmres_unconverged = h->unconverged;
    st->fnorm0 = h->fnorm0;
    st->fnorm = h->fnorm;
    st->max_drho = h->maxdrho;
    if (h->status == MUSIC_E_NONFINITE) {
        set_error("GMRES: non-finite residual or Arnoldi vector");
        return MUSIC_E_NONFINITE;
    }
    if (h->status != MUSIC_OK) {
        set_error("solver graph: loop cap reached (status %d)", h->status);
        return h->status;
    }
    if (!h->ok) {
        CUDA_TRY(cudaMemcpyAsync(g->U, g->Un, g->n * sizeof(double), cudaMemcpyDeviceToDevice, s));
        CUDA_TRY(cudaStreamSynchronize(s));
        return MUSIC_E_NEWTON_FAIL;
    }
    return MUSIC_OK;
}
