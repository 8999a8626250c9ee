/*
 * libmusic solve server: continuous batching of independent implicit solves
 * (the Crank-Nicolson JFNK steps of music.h) on one GPU.
 *
 * The paper runs one solve per job on CPU clusters; this service layer has
 * no counterpart there.  Requests are copied at submission and queued on the
 * host and admitted first-fit in arrival order while the device footprint of
 * the admitted solves (see music_grid_footprint) stays within the memory
 * budget.  Small solves go to the batch lane: one thread advances all of its
 * resident solves together, one music_batch_step launch per round, and new
 * solves join between rounds (continuous batching at step granularity).
 * Larger solves go to per-stream workers, so their kernels overlap on the
 * device.  A solve keeps its state and Krylov basis resident until it
 * finishes, then frees them and the next request is admitted.  Every reduction in the
 * library is deterministic, so a solve gives the same result alone and in a
 * mix.  All calls are thread safe and never abort.
 */
#ifndef MUSIC_SERVER_H
#define MUSIC_SERVER_H

#include "music.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct music_server music_server;

typedef struct {
    size_t mem_budget_bytes;  /* device bytes the admitted solves may own (0: 60% of free memory) */
    int max_active;           /* per-stream workers = concurrently resident solves off the batch
                                 lane [16], <= 256 */
    int batch_max_cells;      /* > 0: solves of at most this many cells (2-D Cartesian, no radiative
                                 diffusion, <= 24 preconditioner sweeps in mixed precision, <= 16
                                 in FP64) join the batch lane; <= 0: no batch lane [0] */
    int batch_size;           /* solves per batched launch [152], <= 512 */
    int autotune;             /* 1: a worker tunes the tile shapes of each new grid configuration
                                 (music_autotune) before its first step; later solves of that
                                 configuration reuse them [0] */
    int graph;                /* 1: workers run each Newton attempt as the recorded solver graph;
                                 0: host-sequenced kernels, which overlap better across many
                                 concurrent solves on this hardware [0] */
} music_server_opts;

typedef struct {
    music_grid_desc desc;     /* problem and solver options (copied) */
    const double *U0;         /* host initial state, nv*N doubles followed by the nscalars
                                 planes of partial densities when desc.nscalars > 0 (copied at
                                 submission) */
    int n_steps;              /* implicit steps to take (>= 0) */
    double cfl;               /* each step: dt = cfl-limited (Eq. 4), > 0; with cfl_adv and
                                 cfl_rad it replaces desc's time-step limits, and every step is
                                 music_newton_step(grid, dt_max) */
    double dt_max;            /* optional cap on dt (<= 0: none) */
    double rho_L, rho_H;      /* densities of the mixing-height diagnostic */
    double cfl_adv, cfl_rad;  /* optional advective / radiative CFL limits (<= 0: none); the step
                                 is the most restrictive limit (music_select_dt) */
} music_solve_req;

typedef struct {
    int status;               /* music_status of the solve; MUSIC_E_BUSY while queued or running */
    int steps_done;
    double sim_time;          /* sum of the steps' dt */
    double diag[6];           /* music_diagnostics of the final state */
    double step_ms_p50;       /* per-step wall latency of this solve (dt choice + Newton solve) */
    double step_ms_p99;
    double queue_ms;          /* submission -> admission */
    double total_ms;          /* submission -> completion */
    int newton_its, gmres_its;/* totals over the steps */
} music_solve_result;

/* Start the workers.  `opts` may be NULL for the defaults.
   Errors: MUSIC_E_OOM, MUSIC_E_CUDA. */
int music_server_create(const music_server_opts *opts, music_server **out);

/* Queue a solve; returns at once with a ticket.  MUSIC_E_INVAL for a bad
   request or descriptor, MUSIC_E_BUSY if the solve alone needs more device
   memory than the whole budget (it could never be admitted). */
int music_submit_solve(music_server *s, const music_solve_req *req, uint64_t *ticket);

/* Non-blocking: MUSIC_OK and *res once the solve is done (its own outcome is
   res->status), MUSIC_E_BUSY while queued or running, MUSIC_E_NOTFOUND for
   an unknown ticket. */
int music_poll(music_server *s, uint64_t ticket, music_solve_result *res);

/* Wait up to timeout_ms (< 0: no limit) for the solve; MUSIC_E_TIMEOUT if it
   is still pending then. */
int music_wait(music_server *s, uint64_t ticket, int timeout_ms, music_solve_result *res);

/* Copy the final state of a finished solve into host memory (nv*N doubles,
   then the scalar planes when the solve carries passive scalars). */
int music_result_state(music_server *s, uint64_t ticket, double *U);

/* Forget a finished solve (MUSIC_E_BUSY if it has not finished). */
int music_release(music_server *s, uint64_t ticket);

/* Aggregates since creation: cell-steps completed, wall time with at least
   one solve resident, solves resident now, requests waiting now. */
int music_server_stats(music_server *s, double *cell_steps, double *busy_ms, int *active, int *queued);

/* Per-step wall latencies (ms) of all completed solves, in completion order:
   copies min(cap, count) values to out (may be NULL) and the total to *count. */
int music_server_step_times(music_server *s, double *out, size_t cap, size_t *count);

/* Stop: requests still queued are dropped, running solves finish, workers
   join, streams are destroyed.  NULL is accepted. */
int music_server_destroy(music_server *s);

#ifdef __cplusplus
}
#endif
#endif /* MUSIC_SERVER_H */
