// Passive scalars (Sec. 2.2): partial densities q_i = c_i rho advected by
// S_i(q) = -div(c_i rho u) with the fluid frozen.  The flux on a face is the
// fluid's face mass flux times c_i reconstructed upwind with the van Leer
// limiter (the form of the internal-energy flux, so a uniform c_i is carried
// exactly like rho); ghost values of c_i wrap on periodic directions and
// mirror at walls, whose faces carry no mass flux.
//
// The kernels read the frozen fluid as the cell density rho and the mass
// fluxes of the cells' lower faces (nd planes of N, written by the stencil's
// non-Jacobian modes into g->fr_capture); the upper face of the last cell of
// a periodic direction is the lower face of the first, of a walled one zero.
#include <cmath>
#include <utility>

#include "internal.h"

namespace {

constexpr int BS = 256;

__device__ inline double vl(double a, double b) { return (a * b > 0.0) ? (2.0 * a) * b / (a + b) : 0.0; }

template <typename VIN>
struct QLoad {
    const double *q;
    const VIN *v;   // Jv direction or null
    double eps;
    __device__ inline double operator()(long long i) const
    {
        double x = q[i];
        if (v) x = x + eps * (double)v[i];
        return x;
    }
};

// c_i of the cell `off` cells from ix along d (periodic wrap, mirror at walls)
template <typename VIN>
__device__ inline double c_at(const GridParams &P, const QLoad<VIN> &W, const double *rho, long long base,
                              const int ix[3], int d, int off)
{
    int j[3] = {ix[0], ix[1], ix[2]};
    const int n = P.n[d];
    int a = ix[d] + off;
    if (P.bc[d] == MUSIC_BC_PERIODIC)
        a = (a % n + n) % n;
    else if (a < 0)
        a = -1 - a;
    else if (a >= n)
        a = 2 * n - 1 - a;
    j[d] = a;
    const long long c = cell_index(P, j);
    return W(base + c) / rho[c];
}

// S_i of cell c (index ix) for scalar i
template <typename VIN>
__device__ double scalar_S(const GridParams &P, const QLoad<VIN> &W, const double *rho, const double *Fr, int i,
                           long long c, const int ix[3])
{
    const long long base = (long long)i * P.N;
    double acc = 0.0;
    for (int d = 0; d < P.nd; d++) {
        const double cm2 = c_at(P, W, rho, base, ix, d, -2), cm1 = c_at(P, W, rho, base, ix, d, -1);
        const double c0 = W(base + c) / rho[c];
        const double cp1 = c_at(P, W, rho, base, ix, d, +1), cp2 = c_at(P, W, rho, base, ix, d, +2);
        const double sm1 = vl(cm1 - cm2, c0 - cm1), s0 = vl(c0 - cm1, cp1 - c0), sp1 = vl(cp1 - c0, cp2 - cp1);
        // lower face (between cells -1 and 0) and upper face (0 and +1)
        const double fl = Fr[(long long)d * P.N + c];
        double fu = 0.0;
        if (ix[d] + 1 < P.n[d]) {
            int j[3] = {ix[0], ix[1], ix[2]};
            j[d] = ix[d] + 1;
            fu = Fr[(long long)d * P.N + cell_index(P, j)];
        } else if (P.bc[d] == MUSIC_BC_PERIODIC) {
            int j[3] = {ix[0], ix[1], ix[2]};
            j[d] = 0;
            fu = Fr[(long long)d * P.N + cell_index(P, j)];
        }
        const double gl = fl * ((fl >= 0.0) ? cm1 + 0.5 * sm1 : c0 - 0.5 * s0);
        const double gu = fu * ((fu >= 0.0) ? c0 + 0.5 * s0 : cp1 - 0.5 * sp1);
        acc += (gu - gl) * P.idx[d];
    }
    return -acc;
}

// modes as the fluid stencil's: R out = S; CN out = q + dt/2 S; F out =
// sign ((q - C) - dt/2 S) and RS_out = S; JV out = v - dt/2 (S(q + eps v) - RS) / eps
template <int MODE, typename VIN, typename VOUT>
__global__ void __launch_bounds__(BS) k_scalar_op(GridParams P, int ns, const double *q, const double *aux,
                                                  const VIN *v, VOUT *out, double *RS_out, const double *rho,
                                                  const double *Fr, double hdt, double sign, const double *eps)
{
    pdl_entry();
    const double e = (MODE == SM_JV) ? *eps : 0.0;
    const QLoad<VIN> W{q, (MODE == SM_JV) ? v : nullptr, e};
    const double c_jv = (MODE == SM_JV && e != 0.0) ? hdt / e : 0.0;
    for (long long c = blockIdx.x * (long long)BS + threadIdx.x; c < P.N; c += (long long)gridDim.x * BS) {
        int ix[3];
        cell_coords(P, c, ix);
        for (int i = 0; i < ns; i++) {
            const double S = scalar_S(P, W, rho, Fr, i, c, ix);
            const long long k = (long long)i * P.N + c;
            if (MODE == SM_R) {
                out[k] = (VOUT)S;
            } else if (MODE == SM_CN) {
                out[k] = (VOUT)(q[k] + hdt * S);
            } else if (MODE == SM_F) {
                out[k] = (VOUT)(sign * ((q[k] - aux[k]) - hdt * S));
                if (RS_out) RS_out[k] = S;
            } else {
                out[k] = (e == 0.0) ? (VOUT)0 : (VOUT)((double)v[k] - c_jv * (S - aux[k]));
            }
        }
    }
}

// q += x over all scalars; partial max of |x| / rho over their entries
__global__ void __launch_bounds__(BS) k_scalar_update(double *q, const double *x, const double *rho, long long N,
                                                      int ns, double *partial, double *dst, unsigned int *counter)
{
    pdl_entry();
    __shared__ double sh[BS / 32];
    double m = 0.0;
    const long long n = (long long)ns * N;
    for (long long e = blockIdx.x * (long long)BS + threadIdx.x; e < n; e += (long long)gridDim.x * BS) {
        q[e] = q[e] + x[e];
        m = nanmax(m, fabs(x[e]) / rho[e % N]);
    }
    const double r = block_max<BS>(m, sh);
    if (threadIdx.x == 0) partial[blockIdx.x] = r;
    if (last_block_done(counter)) finish_max<BS>(partial, gridDim.x, dst, sh);
}

// c_i <- c_i / sum_j c_j per cell (cells whose sum is not positive are left)
__global__ void __launch_bounds__(BS) k_renormalise(double *q, const double *rho, long long N, int ns)
{
    pdl_entry();
    for (long long c = blockIdx.x * (long long)BS + threadIdx.x; c < N; c += (long long)gridDim.x * BS) {
        const double r = rho[c];
        double s = 0.0;
        for (int i = 0; i < ns; i++) s += q[(long long)i * N + c] / r;
        if (!(s > 0.0)) continue;
        for (int i = 0; i < ns; i++) q[(long long)i * N + c] = (q[(long long)i * N + c] / r / s) * r;
    }
}

// lower-face mass fluxes of the multi-pass stencil (extended grid) -> nd planes of N
__global__ void __launch_bounds__(BS) k_copy_fluxes(GridParams P, const double *F0, const double *F1,
                                                    const double *F2, double *out)
{
    pdl_entry();
    for (long long c = blockIdx.x * (long long)BS + threadIdx.x; c < P.N; c += (long long)gridDim.x * BS) {
        int ix[3];
        cell_coords(P, c, ix);
        const long long x = ext_index(P, ix[0], ix[1], ix[2]);
        out[c] = F0[x];
        out[P.N + c] = F1[x];
        if (P.nd == 3) out[2 * P.N + c] = F2[x];
    }
}

// one block per row normal to direction 1: 2 min(<c_1>, <c_2>) dy
__global__ void __launch_bounds__(BS) k_mix_rows(GridParams P, const double *q, const double *rho, double *rows)
{
    pdl_entry();
    __shared__ double sh[BS / 32];
    const int j = blockIdx.x;
    const long long cnt = (long long)P.n[0] * P.n[2];
    double a1 = 0.0, a2 = 0.0;
    for (long long t = threadIdx.x; t < cnt; t += BS) {
        const int i = (int)(t % P.n[0]), k = (int)(t / P.n[0]);
        const long long c = i + (long long)P.n[0] * (j + (long long)P.n[1] * k);
        a1 += q[c] / rho[c];
        a2 += q[P.N + c] / rho[c];
    }
    const double s1 = block_sum<BS>(a1, sh);
    const double s2 = block_sum<BS>(a2, sh);
    if (threadIdx.x == 0) {
        const double m1 = s1 / (double)cnt, m2 = s2 / (double)cnt;
        rows[j] = 2.0 * (m1 < m2 ? m1 : m2) * P.dx[1];
    }
}

__global__ void __launch_bounds__(BS) k_sum_rows(const double *rows, int n, double *dst)
{
    pdl_entry();
    __shared__ double sh[BS / 32];
    double s = 0.0;
    for (int i = threadIdx.x; i < n; i += BS) s += rows[i];
    const double r = block_sum<BS>(s, sh);
    if (threadIdx.x == 0) *dst = r;
}

int blocks(long long n)
{
    long long b = (n + BS - 1) / BS;
    if (b > 152 * 8) b = 152 * 8;
    return (int)(b < 1 ? 1 : b);
}

template <int MODE, typename VIN, typename VOUT>
int launch_sop(music_grid *g, const double *q, const double *aux, const VIN *v, VOUT *out, double *RS_out,
               double hdt, double sign, cudaStream_t s)
{
    k_scalar_op<MODE, VIN, VOUT><<<blocks(g->P.N), BS, 0, s>>>(g->P, g->ns, q, aux, v, out, RS_out, g->srho, g->sfr,
                                                               hdt, sign, &g->ds->eps);
    CHECK_LAUNCH();
    return MUSIC_OK;
}

int check_scalar_grid(music_grid *g)
{
    if (!g) {
        set_error("grid is NULL");
        return MUSIC_E_INVAL;
    }
    if (g->ns < 1) {
        set_error("the grid carries no passive scalars");
        return MUSIC_E_INVAL;
    }
    return MUSIC_OK;
}

}  // namespace

void swap_space(music_grid *g)
{
    KSpace &S = g->sc;
    std::swap(g->U, S.U);
    std::swap(g->RU, S.RU);
    std::swap(g->b, S.b);
    std::swap(g->x, S.x);
    std::swap(g->t64, S.t64);
    std::swap(g->V, S.V);
    std::swap(g->w, S.w);
    std::swap(g->z, S.z);
    std::swap(g->u, S.u);
    std::swap(g->n, S.n);
    std::swap(g->ds, S.ds);
    std::swap(g->hs, S.hs);
    g->in_scalar = !g->in_scalar;
}

int scalar_apply(music_grid *g, int mode, const double *q, const double *aux, const void *v, int vin_double,
                 void *out, int out_double, double *RS_out, double dt, double sign, cudaStream_t s)
{
    const double hdt = 0.5 * dt;
    switch (mode) {
    case SM_R:
        return launch_sop<SM_R, double, double>(g, q, aux, nullptr, (double *)out, nullptr, hdt, sign, s);
    case SM_CN:
        return launch_sop<SM_CN, double, double>(g, q, aux, nullptr, (double *)out, nullptr, hdt, sign, s);
    case SM_F:
        return launch_sop<SM_F, double, double>(g, q, aux, nullptr, (double *)out, RS_out, hdt, sign, s);
    case SM_JV:
        if (vin_double && out_double)
            return launch_sop<SM_JV, double, double>(g, q, aux, (const double *)v, (double *)out, nullptr, hdt,
                                                     sign, s);
        if (!vin_double && !out_double)
            return launch_sop<SM_JV, float, float>(g, q, aux, (const float *)v, (float *)out, nullptr, hdt, sign,
                                                   s);
        if (vin_double)
            return launch_sop<SM_JV, double, float>(g, q, aux, (const double *)v, (float *)out, nullptr, hdt, sign,
                                                    s);
        return launch_sop<SM_JV, float, double>(g, q, aux, (const float *)v, (double *)out, nullptr, hdt, sign, s);
    }
    set_error("scalars: bad mode %d", mode);
    return MUSIC_E_INVAL;
}

int scalar_update(music_grid *g, cudaStream_t s)
{
    k_scalar_update<<<g->nb, BS, 0, s>>>(g->U, g->x, g->srho, g->P.N, g->ns, g->partials, &g->ds->maxdrho,
                                         &g->ds->counters[CNT_NEWTON]);
    CHECK_LAUNCH();
    return MUSIC_OK;
}

int scalar_renormalise(music_grid *g, const double *rho, cudaStream_t s)
{
    double *q = g->in_scalar ? g->U : g->sc.U;
    k_renormalise<<<blocks(g->P.N), BS, 0, s>>>(q, rho, g->P.N, g->ns);
    CHECK_LAUNCH();
    return MUSIC_OK;
}

int capture_ext_fluxes(music_grid *g, cudaStream_t s)
{
    const ExtScratch &X = g->ext;
    k_copy_fluxes<<<blocks(g->P.N), BS, 0, s>>>(g->P, X.Frho[0], X.Frho[1], g->P.nd == 3 ? X.Frho[2] : X.Frho[1],
                                                g->fr_capture);
    CHECK_LAUNCH();
    return MUSIC_OK;
}

extern "C" {

int music_set_scalars(music_grid *grid, const double *q, int is_device, void *stream)
{
    TRY(check_scalar_grid(grid));
    if (!q) {
        set_error("music_set_scalars: q is NULL");
        return MUSIC_E_INVAL;
    }
    cudaStream_t s = (cudaStream_t)stream;
    CUDA_TRY(cudaMemcpyAsync(grid->sc.U, q, grid->sc.n * sizeof(double),
                             is_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, s));
    CUDA_TRY(cudaStreamSynchronize(s));
    return MUSIC_OK;
}

int music_get_scalars(music_grid *grid, double *q, int is_device, void *stream)
{
    TRY(check_scalar_grid(grid));
    if (!q) {
        set_error("music_get_scalars: q is NULL");
        return MUSIC_E_INVAL;
    }
    cudaStream_t s = (cudaStream_t)stream;
    CUDA_TRY(cudaMemcpyAsync(q, grid->sc.U, grid->sc.n * sizeof(double),
                             is_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, s));
    CUDA_TRY(cudaStreamSynchronize(s));
    return MUSIC_OK;
}

int music_scalar_operator(music_grid *grid, const double *U, const double *q, double *S, void *stream)
{
    TRY(check_scalar_grid(grid));
    if (!U || !q || !S) {
        set_error("music_scalar_operator: NULL pointer");
        return MUSIC_E_INVAL;
    }
    cudaStream_t s = (cudaStream_t)stream;
    // the face mass fluxes of U, then S with the fluid frozen there
    grid->fr_capture = grid->sfr;
    const int rc = stencil_apply(grid, SM_R, U, nullptr, nullptr, 1, grid->t64, 1, nullptr, 0.0, 1.0, s);
    grid->fr_capture = nullptr;
    TRY(rc);
    grid->srho = U;
    TRY((launch_sop<SM_R, double, double>(grid, q, nullptr, nullptr, S, nullptr, 0.0, 1.0, s)));
    return MUSIC_OK;
}

int music_scalar_mixing_width(music_grid *grid, double *h, void *stream)
{
    TRY(check_scalar_grid(grid));
    if (!h || grid->ns < 2) {
        set_error("music_scalar_mixing_width: needs two scalars and an output");
        return MUSIC_E_INVAL;
    }
    cudaStream_t s = (cudaStream_t)stream;
    double *rows = grid->sc.t64;  // scratch, n[1] values
    k_mix_rows<<<grid->P.n[1], BS, 0, s>>>(grid->P, grid->sc.U, grid->U, rows);
    CHECK_LAUNCH();
    k_sum_rows<<<1, BS, 0, s>>>(rows, grid->P.n[1], &grid->ds->diag[7]);
    CHECK_LAUNCH();
    CUDA_TRY(cudaMemcpyAsync(grid->hs, grid->ds, sizeof(DevScalars), cudaMemcpyDeviceToHost, s));
    CUDA_TRY(cudaStreamSynchronize(s));
    *h = grid->hs->diag[7];
    return MUSIC_OK;
}

}  // extern "C"
