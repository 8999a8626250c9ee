// Device-side control of the recorded solver graph shared by the control
// kernels (graph.cu) and the vector kernel that closes an Arnoldi step
// (krylov.cu).  One thread runs each; the arithmetic is explicitly rounded
// and uncontracted so that it matches the host-sequenced driver.
#pragma once
#include "internal.h"

__device__ inline bool over_cap(SolveCtl *c, int cap)
{
    if (++c->guard <= cap) return false;
    c->status = MUSIC_E_TIMEOUT;
    c->stop = 1;
    return true;
}

// Arnoldi step j: column j of H from the two CGS passes and |w|, the earlier
// rotations, a new rotation, the residual estimate |g_{j+1}|, the next index.
__device__ inline void ctl_givens(SolveCtl *c, const DevScalars *ds, cudaGraphConditionalHandle h_arnoldi, int m,
                                  int cap)
{
    const int j = c->j;
    const double hn = sqrt(ds->wnorm2);
    c->scale = 0;
    if (!isfinite(hn)) {
        c->status = MUSIC_E_NONFINITE;
        c->stop = 1;
    }
    if (c->stop || over_cap(c, cap)) {
        cudaGraphSetConditional(h_arnoldi, 0u);
        return;
    }
    double *H = c->H;
    constexpr int L = MUSIC_MAXV;
    for (int i = 0; i <= j; i++) H[i * L + j] = __dadd_rn(ds->h[i], ds->h2[i]);
    H[(j + 1) * L + j] = hn;
    for (int i = 0; i < j; i++) {
        const double t0 = H[i * L + j], t1 = H[(i + 1) * L + j];
        H[i * L + j] = __dadd_rn(__dmul_rn(c->cs[i], t0), __dmul_rn(c->sn[i], t1));
        H[(i + 1) * L + j] = __dadd_rn(__dmul_rn(-c->sn[i], t0), __dmul_rn(c->cs[i], t1));
    }
    const double a0 = H[j * L + j], a1 = H[(j + 1) * L + j];
    if (a1 == 0.0) {
        c->cs[j] = 1.0;
        c->sn[j] = 0.0;
    } else {
        const double t = __dsqrt_rn(__dadd_rn(__dmul_rn(a0, a0), __dmul_rn(a1, a1)));
        c->cs[j] = __ddiv_rn(a0, t);
        c->sn[j] = __ddiv_rn(a1, t);
    }
    H[j * L + j] = __dadd_rn(__dmul_rn(c->cs[j], a0), __dmul_rn(c->sn[j], a1));
    H[(j + 1) * L + j] = 0.0;
    c->gv[j + 1] = __dmul_rn(-c->sn[j], c->gv[j]);
    c->gv[j] = __dmul_rn(c->cs[j], c->gv[j]);
    c->its++;
    c->k = j + 1;
    const double resid = fabs(c->gv[j + 1]);
    c->resid = resid;
    const bool done = (hn == 0.0 || resid <= c->target);
    if (!done) {
        c->scale = 1;
        c->scale_idx = j + 1;
        c->inv = __ddiv_rn(1.0, hn);
    }
    c->j = j + 1;
    cudaGraphSetConditional(h_arnoldi, (!done && j + 1 < m) ? 1u : 0u);
}

