// Solve server: continuous batching of independent implicit solves on one GPU.
//
// Requests queue on the host; worker threads admit them first-fit in arrival
// order while the admitted solves' device footprints (music_grid_footprint)
// fit the memory budget and a worker is free.  Each worker owns a CUDA stream
// and runs its solve's steps there, so kernels of concurrent solves overlap
// on the device; a finished solve frees its memory and its worker admits the
// next request at once.  A solve's state and Krylov basis stay resident from
// admission to completion.  Every kernel reduction is deterministic, so a
// solve's result does not depend on what runs beside it.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <memory>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "internal.h"
#include "music_server.h"

namespace {

using clk = std::chrono::steady_clock;

double ms_between(clk::time_point a, clk::time_point b)
{
    return std::chrono::duration<double, std::milli>(b - a).count();
}

double percentile(std::vector<double> v, double p)
{
    if (v.empty()) return 0.0;
    std::sort(v.begin(), v.end());
    const double pos = p / 100.0 * (double)(v.size() - 1);
    const size_t lo = (size_t)pos;
    const size_t hi = std::min(lo + 1, v.size() - 1);
    return v[lo] + (pos - (double)lo) * (v[hi] - v[lo]);
}

struct Job {
    uint64_t ticket = 0;
    music_grid_desc desc;
    std::vector<double> U0, Ufinal;
    int n_steps = 0;
    double cfl = 1.0, dt_max = 0.0, rho_L = 1.0, rho_H = 2.0, cfl_adv = 0.0, cfl_rad = 0.0;
    size_t footprint = 0;
    bool done = false;
    bool failed = false;
    int autotune = 0;
    int graph = 0;
    music_solve_result res;
    std::vector<double> step_ms;
    clk::time_point t_submit, t_admit, t_done;
};

}  // namespace

struct music_server {
    music_server_opts opts;
    size_t budget = 0, used = 0;
    int device = 0;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<uint64_t> pending;
    std::unordered_map<uint64_t, std::unique_ptr<Job>> jobs;
    std::vector<std::thread> workers;
    std::vector<cudaStream_t> streams;
    bool stop = false;
    uint64_t next_ticket = 1;
    int active = 0;
    double cell_steps = 0.0;
    double busy_ms = 0.0;
    clk::time_point busy_since;
    std::vector<double> all_step_ms;
    // batch lane
    bool lane = false;
    int lane_cells = 16384, lane_size = 152;
    std::thread lane_thread;
    cudaStream_t lane_stream = nullptr;
};

namespace {

bool lane_eligible(const music_server *S, const Job *j)
{
    const music_grid_desc &d = j->desc;
    const long long cells = (long long)d.n[0] * d.n[1] * (d.ndim == 3 ? d.n[2] : 1);
    return S->lane && d.ndim == 2 && d.geometry == MUSIC_GEOM_CARTESIAN && !d.conduct && d.nscalars == 0 &&
           !(j->cfl_adv > 0.0) && !(j->cfl_rad > 0.0) &&
           d.precond_sweeps <= (d.precision == MUSIC_MIXED ? 24 : 16) && cells <= S->lane_cells;
}

// Take the first pending job that fits (the lane takes only its own kind,
// the workers only the other); caller holds the lock.
Job *admit_locked(music_server *S, bool for_lane = false)
{
    for (auto it = S->pending.begin(); it != S->pending.end(); ++it) {
        Job *j = S->jobs[*it].get();
        if (lane_eligible(S, j) != for_lane) continue;
        if (S->used + j->footprint <= S->budget) {
            S->pending.erase(it);
            S->used += j->footprint;
            if (S->active == 0) S->busy_since = clk::now();
            S->active++;
            j->t_admit = clk::now();
            return j;
        }
    }
    return nullptr;
}

// the job's initial state (fluid, then scalar planes) into the grid, and back
int set_job_state(music_grid *g, Job *j, cudaStream_t s)
{
    TRY(grid_set_state(g, j->U0.data(), 0, s));
    if (g->ns > 0) TRY(music_set_scalars(g, j->U0.data() + g->n, 0, s));
    return MUSIC_OK;
}

int get_job_state(music_grid *g, Job *j, cudaStream_t s)
{
    j->Ufinal.resize(g->n + g->sc.n);
    TRY(grid_get_state(g, j->Ufinal.data(), 0, s));
    if (g->ns > 0) TRY(music_get_scalars(g, j->Ufinal.data() + g->n, 0, s));
    return MUSIC_OK;
}

int run_job(Job *j, cudaStream_t s)
{
    music_grid *g = nullptr;
    TRY(grid_create(&j->desc, s, &g));
    g->solver_variant = j->graph ? SOLVER_GRAPH : SOLVER_HOST;
    int rc = set_job_state(g, j, s);
    if (rc == MUSIC_OK && j->autotune && j->n_steps > 0) {
        // tile shapes for this configuration (timed once per process, then cached)
        double dt = 0.0;
        rc = music_cfl_dt(g, j->cfl, &dt, s);
        if (rc == MUSIC_OK && j->dt_max > 0.0 && dt > j->dt_max) dt = j->dt_max;
        music_tune_report rep;
        if (rc == MUSIC_OK) rc = music_autotune(g, dt, 0, &rep, s);
    }
    double t = 0.0;
    for (int k = 0; rc == MUSIC_OK && k < j->n_steps; k++) {
        const auto t0 = clk::now();
        music_step_stats st;
        rc = music_newton_step(g, j->dt_max, &st, s);
        if (rc != MUSIC_OK) break;
        j->step_ms.push_back(ms_between(t0, clk::now()));
        t += st.dt;
        j->res.steps_done = k + 1;
        j->res.newton_its += st.newton_its;
        j->res.gmres_its += st.gmres_its;
    }
    j->res.sim_time = t;
    if (rc == MUSIC_OK) rc = music_diagnostics(g, j->rho_L, j->rho_H, j->res.diag, s);
    if (rc == MUSIC_OK) {
        rc = get_job_state(g, j, s);
    }
    grid_destroy(g);
    return rc;
}

// Record a finished solve and free its budget; caller holds the lock.
void finish_locked(music_server *S, Job *j, int rc)
{
    j->res.status = rc;
    j->t_done = clk::now();
    j->res.queue_ms = ms_between(j->t_submit, j->t_admit);
    j->res.total_ms = ms_between(j->t_submit, j->t_done);
    j->res.step_ms_p50 = percentile(j->step_ms, 50.0);
    j->res.step_ms_p99 = percentile(j->step_ms, 99.0);
    j->done = true;
    const double cells = (double)j->desc.n[0] * j->desc.n[1] * (j->desc.ndim == 3 ? j->desc.n[2] : 1);
    S->cell_steps += cells * j->res.steps_done;
    S->all_step_ms.insert(S->all_step_ms.end(), j->step_ms.begin(), j->step_ms.end());
    S->used -= j->footprint;
    S->active--;
    if (S->active == 0) S->busy_ms += ms_between(S->busy_since, clk::now());
    S->cv_done.notify_all();
    S->cv_work.notify_all();  // memory freed: someone may fit now
}

// The batch lane: all resident small solves advance together, one batched
// launch per round per precision; new solves join between rounds.
void lane_main(music_server *S)
{
    cudaSetDevice(S->device);
    cudaStream_t s = S->lane_stream;
    struct Slot {
        Job *j;
        music_grid *g;
    };
    std::vector<Slot> act;
    for (;;) {
        std::vector<Job *> fresh;
        {
            std::unique_lock<std::mutex> lk(S->mu);
            for (;;) {
                while ((int)(act.size() + fresh.size()) < S->lane_size) {
                    Job *j = admit_locked(S, true);
                    if (!j) break;
                    fresh.push_back(j);
                }
                if (!act.empty() || !fresh.empty() || S->stop) break;
                S->cv_work.wait(lk);
            }
            if (S->stop && act.empty() && fresh.empty()) return;
        }
        for (Job *j : fresh) {
            music_grid *g = nullptr;
            int rc = grid_create(&j->desc, s, &g);
            if (rc == MUSIC_OK) rc = grid_set_state(g, j->U0.data(), 0, s);
            // (the lane's grids run the batched kernel only: they take the
            // batched tile shape cached for their configuration by an earlier
            // music_autotune with MUSIC_TUNE_BATCH, if any; timing the shapes
            // here would cost a batched step per candidate inside the service)
            if (rc != MUSIC_OK) {
                if (g) grid_destroy(g);
                std::lock_guard<std::mutex> lk(S->mu);
                finish_locked(S, j, rc);
                continue;
            }
            act.push_back({j, g});
        }
        // one round: a batched step per precision present
        for (int mixed = 0; mixed < 2; mixed++) {
            std::vector<music_grid *> gs;
            std::vector<double> cf, dm;
            std::vector<size_t> idx;
            for (size_t k = 0; k < act.size(); k++)
                if (act[k].g->mixed == mixed && act[k].j->res.steps_done < act[k].j->n_steps) {
                    gs.push_back(act[k].g);
                    cf.push_back(act[k].j->cfl);
                    dm.push_back(act[k].j->dt_max);
                    idx.push_back(k);
                }
            if (gs.empty()) continue;
            const auto t0 = clk::now();
            std::vector<music_step_stats> st(gs.size());
            const int rc = music_batch_step(gs.data(), (int)gs.size(), cf.data(), dm.data(), st.data(), s);
            const double ms = ms_between(t0, clk::now());
            // a bad batch or a CUDA failure fails the whole group; otherwise each
            // grid's own status (read back by the call) decides
            const bool group_err = (rc == MUSIC_E_INVAL || rc == MUSIC_E_OOM || rc == MUSIC_E_CUDA);
            for (size_t q = 0; q < gs.size(); q++) {
                Job *j = act[idx[q]].j;
                const int srcode = group_err ? rc : gs[q]->hs->step_status;
                if (srcode != MUSIC_OK) {
                    j->res.status = srcode;
                    j->n_steps = j->res.steps_done;  // stop here; reported below
                    j->failed = true;
                    continue;
                }
                j->step_ms.push_back(ms);
                j->res.sim_time += st[q].dt;
                j->res.steps_done++;
                j->res.newton_its += st[q].newton_its;
                j->res.gmres_its += st[q].gmres_its;
            }
        }
        // retire finished solves
        for (size_t k = 0; k < act.size();) {
            Job *j = act[k].j;
            if (j->res.steps_done < j->n_steps) {
                k++;
                continue;
            }
            music_grid *g = act[k].g;
            int rc = j->failed ? j->res.status : MUSIC_OK;
            if (rc == MUSIC_OK) rc = music_diagnostics(g, j->rho_L, j->rho_H, j->res.diag, s);
            if (rc == MUSIC_OK) {
                j->Ufinal.resize(g->n);
                rc = grid_get_state(g, j->Ufinal.data(), 0, s);
            }
            grid_destroy(g);
            {
                std::lock_guard<std::mutex> lk(S->mu);
                finish_locked(S, j, rc);
            }
            act[k] = act.back();
            act.pop_back();
        }
    }
}

void worker_main(music_server *S, int w)
{
    cudaSetDevice(S->device);
    cudaStream_t s = S->streams[w];
    for (;;) {
        Job *j = nullptr;
        {
            std::unique_lock<std::mutex> lk(S->mu);
            S->cv_work.wait(lk, [&] { return S->stop || (j = admit_locked(S)) != nullptr; });
            if (!j) return;  // stopping
        }
        const int rc = run_job(j, s);
        std::lock_guard<std::mutex> lk(S->mu);
        finish_locked(S, j, rc);
    }
}

int check_server(const music_server *S)
{
    if (!S) {
        set_error("server is NULL");
        return MUSIC_E_INVAL;
    }
    return MUSIC_OK;
}

}  // namespace

extern "C" {

int music_server_create(const music_server_opts *opts, music_server **out)
{
    if (!out) {
        set_error("music_server_create: NULL output");
        return MUSIC_E_INVAL;
    }
    *out = nullptr;
    music_server *S = new (std::nothrow) music_server;
    if (!S) {
        set_error("host allocation failed");
        return MUSIC_E_OOM;
    }
    music_server_opts o;
    memset(&o, 0, sizeof(o));
    if (opts) o = *opts;
    if (o.max_active <= 0) o.max_active = 16;
    if (o.max_active > 256) o.max_active = 256;
    S->opts = o;
    CUDA_TRY(cudaGetDevice(&S->device));
    if (o.mem_budget_bytes == 0) {
        size_t fr = 0, tot = 0;
        CUDA_TRY(cudaMemGetInfo(&fr, &tot));
        S->budget = (size_t)(0.6 * (double)fr);
    } else {
        S->budget = o.mem_budget_bytes;
    }
    for (int w = 0; w < o.max_active; w++) {
        cudaStream_t st;
        if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) {
            cudaGetLastError();
            for (cudaStream_t x : S->streams) cudaStreamDestroy(x);
            delete S;
            set_error("cudaStreamCreate failed");
            return MUSIC_E_CUDA;
        }
        S->streams.push_back(st);
    }
    S->lane = (o.batch_max_cells > 0);
    S->lane_cells = o.batch_max_cells;
    S->lane_size = o.batch_size > 0 ? (o.batch_size > MUSIC_BATCH_MAX ? MUSIC_BATCH_MAX : o.batch_size) : 152;
    if (S->lane) {
        if (cudaStreamCreateWithFlags(&S->lane_stream, cudaStreamNonBlocking) != cudaSuccess) {
            cudaGetLastError();
            for (cudaStream_t x : S->streams) cudaStreamDestroy(x);
            delete S;
            set_error("cudaStreamCreate failed");
            return MUSIC_E_CUDA;
        }
        S->lane_thread = std::thread(lane_main, S);
    }
    for (int w = 0; w < o.max_active; w++) S->workers.emplace_back(worker_main, S, w);
    *out = S;
    return MUSIC_OK;
}

int music_submit_solve(music_server *S, const music_solve_req *req, uint64_t *ticket)
{
    TRY(check_server(S));
    if (!req || !ticket || !req->U0 || req->n_steps < 0 || !(req->cfl > 0.0)) {
        set_error("music_submit_solve: need a request with U0, n_steps >= 0 and cfl > 0");
        return MUSIC_E_INVAL;
    }
    size_t fp = 0;
    TRY(grid_footprint(&req->desc, &fp));
    if (fp > S->budget) {
        set_error("solve needs %zu device bytes, more than the whole budget of %zu", fp, S->budget);
        return MUSIC_E_BUSY;
    }
    std::unique_ptr<Job> j(new (std::nothrow) Job);
    if (!j) {
        set_error("host allocation failed");
        return MUSIC_E_OOM;
    }
    j->desc = req->desc;
    const size_t ncell = (size_t)req->desc.n[0] * req->desc.n[1] * (req->desc.ndim == 3 ? req->desc.n[2] : 1);
    j->U0.assign(req->U0, req->U0 + (2 + req->desc.ndim + (size_t)req->desc.nscalars) * ncell);
    j->n_steps = req->n_steps;
    j->cfl = req->cfl;
    j->dt_max = req->dt_max;
    j->cfl_adv = req->cfl_adv;
    j->cfl_rad = req->cfl_rad;
    // the request's limits are the grid's: music_newton_step applies them
    j->desc.cfl_hydro = req->cfl;
    j->desc.cfl_adv = req->cfl_adv;
    j->desc.cfl_rad = req->cfl_rad;
    j->rho_L = req->rho_L;
    j->rho_H = (req->rho_H == req->rho_L) ? req->rho_L + 1.0 : req->rho_H;
    j->footprint = fp;
    j->autotune = S->opts.autotune;
    j->graph = S->opts.graph;
    memset(&j->res, 0, sizeof(j->res));
    j->res.status = MUSIC_E_BUSY;
    j->t_submit = clk::now();
    std::lock_guard<std::mutex> lk(S->mu);
    const uint64_t t = S->next_ticket++;
    j->ticket = t;
    S->jobs[t] = std::move(j);
    S->pending.push_back(t);
    *ticket = t;
    S->cv_work.notify_all();  // the lane and the workers take different kinds
    return MUSIC_OK;
}

int music_poll(music_server *S, uint64_t ticket, music_solve_result *res)
{
    TRY(check_server(S));
    std::lock_guard<std::mutex> lk(S->mu);
    auto it = S->jobs.find(ticket);
    if (it == S->jobs.end()) {
        set_error("unknown ticket %llu", (unsigned long long)ticket);
        return MUSIC_E_NOTFOUND;
    }
    if (!it->second->done) return MUSIC_E_BUSY;
    if (res) *res = it->second->res;
    return MUSIC_OK;
}

int music_wait(music_server *S, uint64_t ticket, int timeout_ms, music_solve_result *res)
{
    TRY(check_server(S));
    std::unique_lock<std::mutex> lk(S->mu);
    auto it = S->jobs.find(ticket);
    if (it == S->jobs.end()) {
        set_error("unknown ticket %llu", (unsigned long long)ticket);
        return MUSIC_E_NOTFOUND;
    }
    Job *j = it->second.get();
    if (timeout_ms < 0) {
        S->cv_done.wait(lk, [&] { return j->done; });
    } else if (!S->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms), [&] { return j->done; })) {
        set_error("solve %llu still running after %d ms", (unsigned long long)ticket, timeout_ms);
        return MUSIC_E_TIMEOUT;
    }
    if (res) *res = j->res;
    return MUSIC_OK;
}

int music_result_state(music_server *S, uint64_t ticket, double *U)
{
    TRY(check_server(S));
    std::lock_guard<std::mutex> lk(S->mu);
    auto it = S->jobs.find(ticket);
    if (it == S->jobs.end()) {
        set_error("unknown ticket %llu", (unsigned long long)ticket);
        return MUSIC_E_NOTFOUND;
    }
    Job *j = it->second.get();
    if (!j->done) return MUSIC_E_BUSY;
    if (j->Ufinal.empty()) {
        set_error("solve %llu ended without a state (status %d)", (unsigned long long)ticket, j->res.status);
        return j->res.status ? j->res.status : MUSIC_E_INVAL;
    }
    if (!U) {
        set_error("music_result_state: NULL buffer");
        return MUSIC_E_INVAL;
    }
    memcpy(U, j->Ufinal.data(), j->Ufinal.size() * sizeof(double));
    return MUSIC_OK;
}

int music_release(music_server *S, uint64_t ticket)
{
    TRY(check_server(S));
    std::lock_guard<std::mutex> lk(S->mu);
    auto it = S->jobs.find(ticket);
    if (it == S->jobs.end()) {
        set_error("unknown ticket %llu", (unsigned long long)ticket);
        return MUSIC_E_NOTFOUND;
    }
    if (!it->second->done) {
        set_error("solve %llu is still queued or running", (unsigned long long)ticket);
        return MUSIC_E_BUSY;
    }
    S->jobs.erase(it);
    return MUSIC_OK;
}

int music_server_stats(music_server *S, double *cell_steps, double *busy_ms, int *active, int *queued)
{
    TRY(check_server(S));
    std::lock_guard<std::mutex> lk(S->mu);
    if (cell_steps) *cell_steps = S->cell_steps;
    if (busy_ms) *busy_ms = S->busy_ms + (S->active ? ms_between(S->busy_since, clk::now()) : 0.0);
    if (active) *active = S->active;
    if (queued) *queued = (int)S->pending.size();
    return MUSIC_OK;
}

int music_server_step_times(music_server *S, double *out, size_t cap, size_t *count)
{
    TRY(check_server(S));
    std::lock_guard<std::mutex> lk(S->mu);
    if (count) *count = S->all_step_ms.size();
    if (out) {
        const size_t k = std::min(cap, S->all_step_ms.size());
        memcpy(out, S->all_step_ms.data(), k * sizeof(double));
    }
    return MUSIC_OK;
}

int music_server_destroy(music_server *S)
{
    if (!S) return MUSIC_OK;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        S->stop = true;
        // queued requests are dropped; running solves finish their step loop
        S->pending.clear();
    }
    S->cv_work.notify_all();
    for (std::thread &t : S->workers) t.join();
    if (S->lane_thread.joinable()) S->lane_thread.join();
    for (cudaStream_t st : S->streams) cudaStreamDestroy(st);
    if (S->lane_stream) cudaStreamDestroy(S->lane_stream);
    delete S;
    return MUSIC_OK;
}

}  // extern "C"
