// Vector kernels of the GMRES / Newton loop (Saad & Schultz 1986, cited in
// Sec. 2): classical Gram-Schmidt with one re-orthogonalisation, each pass a
// sweep over w and up to eight basis vectors (more in further sweeps) with
// FP64 accumulation; norms; the cycle's correction from the stored
// preconditioned basis; the Newton update with its density-correction test.
//
// Reductions are two-stage and deterministic: every block writes one partial
// per quantity, then the last block to finish sums the partials in block
// order.  The block count per grid is fixed, so results do not depend on
// timing.
#include <cmath>

#include "internal.h"
#include "ctl.cuh"

namespace {

constexpr int BS = 256;
constexpr int RUN = 4;  // float4 chunks summed in FP32 before an FP64 add (16 elements)

struct Coef {
    double c[MUSIC_MAXV];
};

template <typename T>
__global__ void __launch_bounds__(BS) k_sumsq(const T *x, long long n, double *partial, double *dst,
                                              unsigned int *counter)
{
    pdl_entry();
    __shared__ double sh[BS / 32];
    double s = 0.0;
    // four elements' loads in flight per step, summed in element order; an
    // FP32 vector's squares are summed in FP32 over each step's four, then
    // added in FP64 (as the dot products do: FP64 adds run at 1/73 of the FP32
    // rate on this part)
    const long long stride = (long long)gridDim.x * BS;
    long long i = blockIdx.x * (long long)BS + threadIdx.x;
    for (; i + 3 * stride < n; i += 4 * stride) {
        T v[4];
#pragma unroll
        for (int r = 0; r < 4; r++) v[r] = x[i + r * stride];
        if constexpr (sizeof(T) == 4) {
            float q = v[0] * v[0];
#pragma unroll
            for (int r = 1; r < 4; r++) q = fmaf(v[r], v[r], q);
            s += (double)q;
        } else {
#pragma unroll
            for (int r = 0; r < 4; r++) s += v[r] * v[r];
        }
    }
    for (; i < n; i += stride) {
        const double v = (double)x[i];
        s += v * v;
    }
    const double r = block_sum<BS>(s, sh);
    if (threadIdx.x == 0) partial[blockIdx.x] = r;
    if (last_block_done(counter)) finish_sums<BS>(partial, gridDim.x, 0, 1, dst, sh);
}

// dst[k] = sum_b partial[k * nb + b], one block per k, fixed order.
__global__ void __launch_bounds__(BS) k_final_sum(const double *partial, int nb, double *dst)
{
    pdl_entry();
    __shared__ double sh[BS / 32];
    const double *p = partial + (long long)blockIdx.x * nb;
    double s = 0.0;
    for (int i = threadIdx.x; i < nb; i += BS) s += p[i];
    const double r = block_sum<BS>(s, sh);
    if (threadIdx.x == 0) dst[blockIdx.x] = r;
}

__global__ void k_set_eps(DevScalars *ds, double fixed)
{
    pdl_entry();
    if (fixed > 0.0) {
        ds->eps = fixed;
        return;
    }
    ds->eps = fd_eps(ds->unorm2, ds->vnorm2);
}

// The CGS passes hold NG accumulators per thread: a pass over more basis
// vectors runs in groups of NG, each group one more sweep over w and its
// NG basis vectors, so the register count (and the occupancy) does not grow
// with the Arnoldi index.  Every group visits the thread's elements in the
// same order, so each product is summed exactly as one sweep would sum it.
constexpr int NG = 8;

// acc[i] = <V_{i0+i}, w> over the thread's elements in FP64, i < cnt <= NG
template <typename KT>
__device__ __forceinline__ void dots_pass(const KT *V, const KT *w, long long n, int i0, int cnt, double acc[NG])
{
#pragma unroll
    for (int i = 0; i < NG; i++) acc[i] = 0.0;
    for (long long e = blockIdx.x * (long long)BS + threadIdx.x; e < n; e += (long long)gridDim.x * BS) {
        const double we = (double)w[e];
#pragma unroll
        for (int i = 0; i < NG; i++)
            if (i < cnt) acc[i] += (double)V[(long long)(i0 + i) * n + e] * we;
    }
}

// block partials of acc[0, cnt) into partial[(i0 + i) * nb + block]
__device__ __forceinline__ void write_partials(const double acc[NG], int i0, int cnt, double *partial, int nb,
                                               double *sh)
{
#pragma unroll
    for (int i = 0; i < NG; i++) {
        if (i < cnt) {
            const double r = block_sum<BS>(acc[i], sh);
            if (threadIdx.x == 0) partial[(long long)(i0 + i) * nb + blockIdx.x] = r;
        }
    }
}

template <typename KT>
__global__ void __launch_bounds__(BS) k_scale_into(const KT *w, KT *dst, long long n, double inv)
{
    pdl_entry();
    for (long long e = blockIdx.x * (long long)BS + threadIdx.x; e < n; e += (long long)gridDim.x * BS)
        dst[e] = (KT)((double)w[e] * inv);
}

// V_0 = r / beta as r times 1 / beta (formed once, rounded to the Krylov type)
template <typename KT>
__global__ void __launch_bounds__(BS) k_first(const double *r, KT *dst, long long n, KT rinv)
{
    pdl_entry();
    const long long stride = (long long)gridDim.x * BS, t0 = blockIdx.x * (long long)BS + threadIdx.x;
    long long e0 = t0;
    if constexpr (sizeof(KT) == 4) {
        // four elements a step when the vectors start 16-byte aligned
        const long long n4 = (n & 3) ? 0 : (n >> 2);
        for (long long e = t0; e < n4; e += stride) {
            const double2 a = reinterpret_cast<const double2 *>(r)[2 * e], b = reinterpret_cast<const double2 *>(r)[2 * e + 1];
            reinterpret_cast<float4 *>(dst)[e] =
                make_float4((float)a.x * rinv, (float)a.y * rinv, (float)b.x * rinv, (float)b.y * rinv);
        }
        e0 = 4 * n4 + t0;
    }
    for (long long e = e0; e < n; e += stride) dst[e] = (KT)r[e] * rinv;
}

// x += sum_{i<k} y_i Z_i: the cycle's correction M^-1 V y from the stored
// preconditioned basis Z_i = M^-1 V_i (V itself when unpreconditioned)
template <typename KT>
__global__ void __launch_bounds__(BS) k_correct(const KT *Z, double *x, long long n, int k, Coef y, const int *kdev,
                                                const double *ydev)
{
    pdl_entry();
    __shared__ double ys[MUSIC_MAXV];
    if (kdev) k = *kdev;
    for (int i = threadIdx.x; i < k; i += BS) ys[i] = ydev ? ydev[i] : y.c[i];
    __syncthreads();
    for (long long e = blockIdx.x * (long long)BS + threadIdx.x; e < n; e += (long long)gridDim.x * BS) {
        double s = 0.0;
        for (int i = 0; i < k; i++) s += ys[i] * (double)Z[(long long)i * n + e];
        x[e] += (double)(KT)s;
    }
}

__global__ void __launch_bounds__(BS) k_sub(const double *a, const double *b, double *o, long long n)
{
    pdl_entry();
    for (long long e = blockIdx.x * (long long)BS + threadIdx.x; e < n; e += (long long)gridDim.x * BS)
        o[e] = a[e] - b[e];
}

__global__ void __launch_bounds__(BS) k_neg(const double *a, double *o, long long n)
{
    pdl_entry();
    for (long long e = blockIdx.x * (long long)BS + threadIdx.x; e < n; e += (long long)gridDim.x * BS)
        o[e] = -a[e];
}

template <typename S, typename D>
__global__ void __launch_bounds__(BS) k_cast(const S *a, D *o, long long n)
{
    pdl_entry();
    for (long long e = blockIdx.x * (long long)BS + threadIdx.x; e < n; e += (long long)gridDim.x * BS)
        o[e] = (D)a[e];
}

// U += x over all unknowns; partial max of |x_rho| / rho_new over cells.  On
// mixed grids (F32) the ratio is formed in FP32: it only meets the Newton
// tolerance, and an FP64 division per cell costs more than the update itself.
template <bool F32>
__global__ void __launch_bounds__(BS) k_newton_update(double *U, const double *x, long long n, long long N,
                                                      double *partial, double *dst, double *unorm2,
                                                      unsigned int *counter, const int *skip)
{
    pdl_entry();
    if (skip && *skip) return;  // a hard error ended the linear solve: U stays as it is
    __shared__ double sh[BS / 32];
    double m = 0.0, q = 0.0;
    float m32 = 0.0f;
    auto one = [&](long long e, double Ue, double xe) {
        const double u = Ue + xe;
        U[e] = u;
        q = fma(u, u, q);  // |U|^2 of the new iterate, for the next product's eps
        if (e < N) {
            if (F32) {
                const float t = fabsf((float)xe) / (float)u;
                m32 = (t > m32 || t != t) ? t : m32;  // NaN-propagating, as nanmax
            } else {
                m = nanmax(m, fabs(xe) / u);
            }
        }
    };
    // four elements' loads in flight per step, processed in element order
    const long long stride = (long long)gridDim.x * BS;
    long long e = blockIdx.x * (long long)BS + threadIdx.x;
    for (; e + 3 * stride < n; e += 4 * stride) {
        double Ue[4], xe[4];
#pragma unroll
        for (int r = 0; r < 4; r++) {
            Ue[r] = U[e + r * stride];
            xe[r] = x[e + r * stride];
        }
#pragma unroll
        for (int r = 0; r < 4; r++) one(e + r * stride, Ue[r], xe[r]);
    }
    for (; e < n; e += stride) one(e, U[e], x[e]);
    if (F32) m = (double)m32;
    const double r = block_max<BS>(m, sh);
    if (threadIdx.x == 0) partial[blockIdx.x] = r;
    const double t = block_sum<BS>(q, sh);
    if (threadIdx.x == 0) partial[gridDim.x + blockIdx.x] = t;
    if (last_block_done(counter)) {
        finish_max<BS>(partial, gridDim.x, dst, sh);
        __syncthreads();
        finish_sums<BS>(partial + gridDim.x, gridDim.x, 0, 1, unorm2, sh);
    }
}


// ---- mixed precision: FP32 basis, FP32 arithmetic inside a 4-element chunk
// (float4 loads), FP64 accumulation across chunks and in the reductions.

// Block partials of cnt <= NVM per-thread sums: each warp adds its lanes'
// values in FP32 (a fixed tree of five levels), then one thread per sum adds
// the warps' results in FP64 in warp order and writes partial[i * nb + block].
// FP64 work and barriers stay per block, not per thread and sum: FP64 runs at
// 1/64 of the FP32 rate on this part, and a thread of these kernels holds only
// a few chunks on the grids the step is timed on.
template <int NVM>
__device__ __forceinline__ void block_partials_mixed(const double *acc, int cnt, double *partial, int nb)
{
    __shared__ double ws[NVM][BS / 32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int i = 0; i < NVM; i++) {
        if (i < cnt) {
            float v = (float)acc[i];
            for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
            if (lane == 0) ws[i][wid] = (double)v;
        }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < cnt; i += BS) {
        double t = 0.0;
        for (int w = 0; w < BS / 32; w++) t += ws[i][w];
        partial[(long long)i * nb + blockIdx.x] = t;
    }
}
__device__ inline float dot4(const float4 a, const float4 b)
{
    float s = a.x * b.x;
    s = fmaf(a.y, b.y, s);
    s = fmaf(a.z, b.z, s);
    return fmaf(a.w, b.w, s);
}

// acc[i] = <V_{i0+i}, w> over the thread's elements, i < cnt <= NG: FP32
// runs of RUN float4 chunks, then FP64 (FP64 adds and conversions run at
// 1/74 of the FP32 rate on this part)
__device__ __forceinline__ void dots_pass_f32(const float *V, const float *w, long long n, int i0, int cnt,
                                              double acc[NG])
{
    float run[NG];
#pragma unroll
    for (int i = 0; i < NG; i++) {
        acc[i] = 0.0;
        run[i] = 0.0f;
    }
    // float4 path only when every basis vector starts 16-byte aligned
    const long long n4 = (n & 3) ? 0 : (n >> 2);
    const long long stride = (long long)gridDim.x * BS;
    const long long t0 = blockIdx.x * (long long)BS + threadIdx.x;
    int k = 0;
    for (long long e = t0; e < n4; e += stride) {
        const float4 we = reinterpret_cast<const float4 *>(w)[e];
#pragma unroll
        for (int i = 0; i < NG; i++)
            if (i < cnt) run[i] += dot4(reinterpret_cast<const float4 *>(V + (long long)(i0 + i) * n)[e], we);
        if (++k == RUN) {
#pragma unroll
            for (int i = 0; i < NG; i++) {
                if (i < cnt) acc[i] += (double)run[i];
                run[i] = 0.0f;
            }
            k = 0;
        }
    }
#pragma unroll
    for (int i = 0; i < NG; i++)
        if (i < cnt) acc[i] += (double)run[i];
    for (long long e = 4 * n4 + t0; e < n; e += stride) {
        const float we = w[e];
#pragma unroll
        for (int i = 0; i < NG; i++)
            if (i < cnt) acc[i] += (double)(V[(long long)(i0 + i) * n + e] * we);
    }
}

// ---- the passes of one Arnoldi step's CGS2 (classical Gram-Schmidt with one
// re-orthogonalisation), as block partials, one kernel each.

// Pass 1: Z_j = zs (with Zb) and the block partials of h_i = <V_i, w>, i <= j,
// at partial[i * nb + block].
template <typename KT>
__device__ __forceinline__ void cgs_dots_pass(const KT *V, const KT *w, long long n, int j, double *partial, int nb,
                                              const KT *zs, KT *Zb, double *sh)
{
    const long long stride = (long long)gridDim.x * BS, t0 = blockIdx.x * (long long)BS + threadIdx.x;
    if (Zb) {
        KT *Zj = Zb + (long long)j * n;
        long long e0 = t0;
        if constexpr (sizeof(KT) == 4) {
            const long long n4 = (n & 3) ? 0 : (n >> 2);
            for (long long e = t0; e < n4; e += stride)
                reinterpret_cast<float4 *>(Zj)[e] = reinterpret_cast<const float4 *>(zs)[e];
            e0 = 4 * n4 + t0;
        }
        for (long long e = e0; e < n; e += stride) Zj[e] = zs[e];
    }
    for (int i0 = 0; i0 <= j; i0 += NG) {
        const int cnt = min(NG, j + 1 - i0);
        double acc[NG];
        if constexpr (sizeof(KT) == 4) {
            dots_pass_f32(V, w, n, i0, cnt, acc);
            block_partials_mixed<NG>(acc, cnt, partial + (long long)i0 * nb, nb);
            __syncthreads();  // the block's warp sums are reused by the next group
        } else {
            dots_pass<KT>(V, w, n, i0, cnt, acc);
            write_partials(acc, i0, cnt, partial, nb, sh);
        }
    }
}

// Passes 2 and 3: w <- w - sum_i h_i V_i (FP32 coefficients on an FP32
// basis), then the block partials of h2_i = <V_i, w> or, with NORM, of |w|^2.
// Up to NG products ride on the update sweep; beyond that the updated w is
// swept again in groups.  h: the j + 1 coefficients (device or shared memory).
template <bool NORM, typename KT>
__device__ __forceinline__ void cgs_update_pass(const KT *V, KT *w, long long n, int j, const double *h,
                                                double *partial, int nb, double *sh)
{
    using CT = KT;  // coefficient type
    __shared__ CT hs[MUSIC_MAXV];
    for (int i = threadIdx.x; i <= j; i += BS) hs[i] = (CT)h[i];
    __syncthreads();
    const bool fused = NORM || j < NG;
    double acc[NG];
    const long long stride = (long long)gridDim.x * BS;
    const long long t0 = blockIdx.x * (long long)BS + threadIdx.x;
    if constexpr (sizeof(KT) == 4) {
        float run[NG];
#pragma unroll
        for (int i = 0; i < NG; i++) {
            acc[i] = 0.0;
            run[i] = 0.0f;
        }
        int k = 0;
        // float4 path only when every basis vector starts 16-byte aligned
        const long long n4 = (n & 3) ? 0 : (n >> 2);
        for (long long e = t0; e < n4; e += stride) {
            float4 we = reinterpret_cast<const float4 *>(w)[e];
            for (int i = 0; i <= j; i++) {
                const float4 v = reinterpret_cast<const float4 *>(V + (long long)i * n)[e];
                const float c = -hs[i];
                we.x = fmaf(c, v.x, we.x);
                we.y = fmaf(c, v.y, we.y);
                we.z = fmaf(c, v.z, we.z);
                we.w = fmaf(c, v.w, we.w);
            }
            reinterpret_cast<float4 *>(w)[e] = we;
            if (NORM) {
                run[0] += dot4(we, we);
            } else if (fused) {
#pragma unroll
                for (int i = 0; i < NG; i++)
                    if (i <= j) run[i] += dot4(reinterpret_cast<const float4 *>(V + (long long)i * n)[e], we);
            }
            if (fused && ++k == RUN) {
#pragma unroll
                for (int i = 0; i < NG; i++) {
                    if (NORM ? i == 0 : i <= j) acc[i] += (double)run[i];
                    run[i] = 0.0f;
                }
                k = 0;
            }
        }
#pragma unroll
        for (int i = 0; i < NG; i++)
            if (fused && (NORM ? i == 0 : i <= j)) acc[i] += (double)run[i];
        for (long long e = 4 * n4 + t0; e < n; e += stride) {
            float we = w[e];
            for (int i = 0; i <= j; i++) we = fmaf(-hs[i], V[(long long)i * n + e], we);
            w[e] = we;
            if (NORM) {
                acc[0] += (double)(we * we);
            } else if (fused) {
#pragma unroll
                for (int i = 0; i < NG; i++)
                    if (i <= j) acc[i] += (double)(V[(long long)i * n + e] * we);
            }
        }
        if (NORM) {
            block_partials_mixed<1>(acc, 1, partial, nb);
        } else if (fused) {
            block_partials_mixed<NG>(acc, j + 1, partial, nb);
        } else {
            for (int i0 = 0; i0 <= j; i0 += NG) {
                const int cnt = min(NG, j + 1 - i0);
                dots_pass_f32(V, w, n, i0, cnt, acc);
                block_partials_mixed<NG>(acc, cnt, partial + (long long)i0 * nb, nb);
                __syncthreads();
            }
        }
    } else {
#pragma unroll
        for (int i = 0; i < NG; i++) acc[i] = 0.0;
        for (long long e = t0; e < n; e += stride) {
            double we = (double)w[e];
            for (int i = 0; i <= j; i++) we -= hs[i] * (double)V[(long long)i * n + e];
            const KT ws = (KT)we;
            w[e] = ws;
            const double wr = (double)ws;
            if (NORM) {
                acc[0] += wr * wr;
            } else if (fused) {
#pragma unroll
                for (int i = 0; i < NG; i++)
                    if (i <= j) acc[i] += (double)V[(long long)i * n + e] * wr;
            }
        }
        if (NORM) {
            write_partials(acc, 0, 1, partial, nb, sh);
        } else if (fused) {
            write_partials(acc, 0, j + 1, partial, nb, sh);
        } else {
            for (int i0 = 0; i0 <= j; i0 += NG) {
                const int cnt = min(NG, j + 1 - i0);
                dots_pass<KT>(V, w, n, i0, cnt, acc);
                write_partials(acc, i0, cnt, partial, nb, sh);
            }
        }
    }
}

// h_i = <V_i, w>, i <= j (j read from jdev when given); with Zb, also Z_j = zs
template <typename KT>
__global__ void __launch_bounds__(BS, sizeof(KT) == 4 ? 4 : 1) k_dots(const KT *V, const KT *w, long long n, int j, double *partial,
                                                int nb, double *dst, unsigned int *counter, const int *jdev,
                                                const KT *zs, KT *Zb)
{
    pdl_entry();
    __shared__ double sh[BS / 32];
    if (jdev) j = *jdev;
    cgs_dots_pass<KT>(V, w, n, j, partial, nb, zs, Zb, sh);
    if (last_block_done(counter)) finish_sums_warps<BS>(partial, nb, nb, j + 1, dst);
}

// w <- w - sum_i h_i V_i, then h2_i = <V_i, w> (second CGS pass) or, with
// NORM, |w|^2 only; with gc.c the last block then runs the Arnoldi step's
// Givens control
template <bool NORM, typename KT>
__global__ void __launch_bounds__(BS, sizeof(KT) == 4 ? 4 : 1) k_update(const KT *V, KT *w, long long n, int j, const double *h,
                                                  double *partial, int nb, double *dst, unsigned int *counter,
                                                  const int *jdev, GivensCtl gc)
{
    pdl_entry();
    __shared__ double sh[BS / 32];
    if (jdev) j = *jdev;
    cgs_update_pass<NORM, KT>(V, w, n, j, h, partial, nb, sh);
    if (last_block_done(counter)) {
        if (NORM)
            finish_sums<BS>(partial, nb, nb, 1, dst, sh);
        else
            finish_sums_warps<BS>(partial, nb, nb, j + 1, dst);
        // |w| is in *dst (written by thread 0): the Arnoldi step's control
        if (NORM && gc.c && threadIdx.x == 0) ctl_givens(gc.c, gc.ds, gc.h, gc.m, gc.cap);
    }
}

__global__ void __launch_bounds__(BS) k_correct_f32(const float *Z, double *x, long long n, int k, Coef y,
                                                    const int *kdev, const double *ydev)
{
    pdl_entry();
    __shared__ float ys[MUSIC_MAXV];
    if (kdev) k = *kdev;
    for (int i = threadIdx.x; i < k; i += BS) ys[i] = (float)(ydev ? ydev[i] : y.c[i]);
    __syncthreads();
    // four elements a step (float4 loads of the basis) when every vector
    // starts 16-byte aligned; each element summed as the scalar loop sums it
    const long long n4 = (n & 3) ? 0 : (n >> 2);
    const long long stride = (long long)gridDim.x * BS, t0 = blockIdx.x * (long long)BS + threadIdx.x;
    for (long long e = t0; e < n4; e += stride) {
        float4 s = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
        for (int i = 0; i < k; i++) {
            const float4 z = reinterpret_cast<const float4 *>(Z + (long long)i * n)[e];
            s.x = fmaf(ys[i], z.x, s.x);
            s.y = fmaf(ys[i], z.y, s.y);
            s.z = fmaf(ys[i], z.z, s.z);
            s.w = fmaf(ys[i], z.w, s.w);
        }
        double2 *x2 = reinterpret_cast<double2 *>(x) + 2 * e;
        double2 a = x2[0], b = x2[1];
        a.x += (double)s.x;
        a.y += (double)s.y;
        b.x += (double)s.z;
        b.y += (double)s.w;
        x2[0] = a;
        x2[1] = b;
    }
    for (long long e = 4 * n4 + t0; e < n; e += stride) {
        float s = 0.0f;
        for (int i = 0; i < k; i++) s = fmaf(ys[i], Z[(long long)i * n + e], s);
        x[e] += (double)s;
    }
}

__global__ void __launch_bounds__(BS) k_scale_f32(const float *w, float *dst, long long n, float inv)
{
    pdl_entry();
    // four elements a step when the vectors start 16-byte aligned
    const long long n4 = (n & 3) ? 0 : (n >> 2);
    const long long stride = (long long)gridDim.x * BS, t0 = blockIdx.x * (long long)BS + threadIdx.x;
    for (long long e = t0; e < n4; e += stride) {
        const float4 a = reinterpret_cast<const float4 *>(w)[e];
        reinterpret_cast<float4 *>(dst)[e] = make_float4(a.x * inv, a.y * inv, a.z * inv, a.w * inv);
    }
    for (long long e = 4 * n4 + t0; e < n; e += stride) dst[e] = w[e] * inv;
}

int grid_blocks(long long n, int cap)
{
    long long b = (n + BS - 1) / BS;
    if (b > cap) b = cap;
    if (b < 1) b = 1;
    return (int)b;
}

int launch_dots(music_grid *g, int j, const int *jdev, cudaStream_t s)
{
    const long long n = (long long)g->n;
    unsigned int *cnt = &g->ds->counters[CNT_DOTS];
    void *Zb = krylov_zstore(g);
    if (g->mixed)
        k_dots<float><<<g->nb, BS, 0, s>>>((const float *)g->V, (const float *)g->w, n, j, g->partials, g->nb,
                                           g->ds->h, cnt, jdev, (const float *)g->z, (float *)Zb);
    else
        k_dots<double><<<g->nb, BS, 0, s>>>((const double *)g->V, (const double *)g->w, n, j, g->partials, g->nb,
                                            g->ds->h, cnt, jdev, (const double *)g->z, (double *)Zb);
    CHECK_LAUNCH();
    return MUSIC_OK;
}

template <bool NORM>
int launch_update(music_grid *g, int j, const int *jdev, const double *h, cudaStream_t s, const GivensCtl *gcp)
{
    const GivensCtl gc = gcp ? *gcp : GivensCtl{};
    const long long n = (long long)g->n;
    double *dst = NORM ? &g->ds->wnorm2 : g->ds->h2;
    unsigned int *cnt = &g->ds->counters[NORM ? CNT_NORMW : CNT_UPDATE];
    if (g->mixed)
        k_update<NORM, float><<<g->nb, BS, 0, s>>>((const float *)g->V, (float *)g->w, n, j, h, g->partials, g->nb,
                                                   dst, cnt, jdev, gc);
    else
        k_update<NORM, double><<<g->nb, BS, 0, s>>>((const double *)g->V, (double *)g->w, n, j, h, g->partials,
                                                    g->nb, dst, cnt, jdev, gc);
    CHECK_LAUNCH();
    return MUSIC_OK;
}

}  // namespace

int dev_norm2(music_grid *g, const void *x, int is_double, size_t n, double *dst, cudaStream_t s)
{
    ProfScope prof_(g, MUSIC_PROF_VECTOR, s);
    unsigned int *cnt = &g->ds->counters[CNT_SUMSQ];
    if (is_double)
        k_sumsq<double><<<g->nb, BS, 0, s>>>((const double *)x, (long long)n, g->partials, dst, cnt);
    else
        k_sumsq<float><<<g->nb, BS, 0, s>>>((const float *)x, (long long)n, g->partials, dst, cnt);
    CHECK_LAUNCH();
    return MUSIC_OK;
}

int final_sum(music_grid *g, int count, double *dst, cudaStream_t s)
{
    k_final_sum<<<1, BS, 0, s>>>(g->partials, count, dst);
    CHECK_LAUNCH();
    return MUSIC_OK;
}

int dev_set_eps(music_grid *g, double fixed, cudaStream_t s)
{
    ProfScope prof_(g, MUSIC_PROF_VECTOR, s);
    k_set_eps<<<1, 1, 0, s>>>(g->ds, fixed);
    CHECK_LAUNCH();
    return MUSIC_OK;
}

// With jdev the Arnoldi index is read on the device (j then bounds it).
int krylov_dots(music_grid *g, int j, const int *jdev, cudaStream_t s)
{
    ProfScope prof_(g, MUSIC_PROF_VECTOR, s);
    return launch_dots(g, j, jdev, s);
}

template <bool NORM>
int update_any(music_grid *g, int j, const int *jdev, cudaStream_t s, const GivensCtl *gc)
{
    ProfScope prof_(g, MUSIC_PROF_VECTOR, s);
    return launch_update<NORM>(g, j, jdev, NORM ? g->ds->h2 : g->ds->h, s, gc);
}

int krylov_update_dots(music_grid *g, int j, const int *jdev, cudaStream_t s)
{
    return update_any<false>(g, j, jdev, s, nullptr);
}

int krylov_update_norm(music_grid *g, int j, const int *jdev, cudaStream_t s, const GivensCtl *gc)
{
    return update_any<true>(g, j, jdev, s, gc);
}

int krylov_scale(music_grid *g, int j, double inv, cudaStream_t s)
{
    ProfScope prof_(g, MUSIC_PROF_VECTOR, s);
    const long long n = (long long)g->n;
    const int nb = grid_blocks(n, 152 * 16);
    if (g->mixed)
        k_scale_f32<<<nb, BS, 0, s>>>((const float *)g->w, (float *)g->V + (long long)(j + 1) * n, n, (float)inv);
    else
        k_scale_into<double><<<nb, BS, 0, s>>>((const double *)g->w, (double *)g->V + (long long)(j + 1) * n, n,
                                              inv);
    CHECK_LAUNCH();
    return MUSIC_OK;
}

// V_0 = r / beta  (the division keeps the oracle's rounding)
int krylov_first(music_grid *g, const double *r, double beta, cudaStream_t s)
{
    ProfScope prof_(g, MUSIC_PROF_VECTOR, s);
    const long long n = (long long)g->n;
    const int nb = grid_blocks(n, 152 * 16);
    const double rinv = 1.0 / beta;
    if (g->mixed)
        k_first<float><<<nb, BS, 0, s>>>(r, (float *)g->V, n, (float)rinv);
    else
        k_first<double><<<nb, BS, 0, s>>>(r, (double *)g->V, n, rinv);
    CHECK_LAUNCH();
    return MUSIC_OK;
}

int krylov_correct(music_grid *g, int k, const double *y, const int *kdev, const double *ydev, cudaStream_t s)
{
    ProfScope prof_(g, MUSIC_PROF_VECTOR, s);
    Coef c;
    for (int i = 0; i < MUSIC_MAXV; i++) c.c[i] = (y && i < k) ? y[i] : 0.0;
    const long long n = (long long)g->n;
    const int nb = grid_blocks(n, 152 * 16);
    const void *Z = krylov_zstore(g) ? krylov_zstore(g) : g->V;
    if (g->mixed)
        k_correct_f32<<<nb, BS, 0, s>>>((const float *)Z, g->x, n, k, c, kdev, ydev);
    else
        k_correct<double><<<nb, BS, 0, s>>>((const double *)Z, g->x, n, k, c, kdev, ydev);
    CHECK_LAUNCH();
    return MUSIC_OK;
}

int vec_sub(music_grid *g, const double *a, const double *b, double *out, cudaStream_t s)
{
    ProfScope prof_(g, MUSIC_PROF_VECTOR, s);
    const long long n = (long long)g->n;
    k_sub<<<grid_blocks(n, 152 * 16), BS, 0, s>>>(a, b, out, n);
    CHECK_LAUNCH();
    return MUSIC_OK;
}

int vec_neg(music_grid *g, const double *a, double *out, cudaStream_t s)
{
    ProfScope prof_(g, MUSIC_PROF_VECTOR, s);
    const long long n = (long long)g->n;
    k_neg<<<grid_blocks(n, 152 * 16), BS, 0, s>>>(a, out, n);
    CHECK_LAUNCH();
    return MUSIC_OK;
}

int vec_cast_copy(const void *src, int src_double, void *dst, int dst_double, size_t n, cudaStream_t s)
{
    const int nb = grid_blocks((long long)n, 152 * 16);
    if (src_double && dst_double)
        CUDA_TRY(cudaMemcpyAsync(dst, src, n * sizeof(double), cudaMemcpyDeviceToDevice, s));
    else if (!src_double && !dst_double)
        CUDA_TRY(cudaMemcpyAsync(dst, src, n * sizeof(float), cudaMemcpyDeviceToDevice, s));
    else if (src_double)
        k_cast<double, float><<<nb, BS, 0, s>>>((const double *)src, (float *)dst, (long long)n);
    else
        k_cast<float, double><<<nb, BS, 0, s>>>((const float *)src, (double *)dst, (long long)n);
    CHECK_LAUNCH();
    return MUSIC_OK;
}

int newton_update(music_grid *g, const int *skip, cudaStream_t s)
{
    ProfScope prof_(g, MUSIC_PROF_VECTOR, s);
    if (g->mixed)
        k_newton_update<true><<<g->nb, BS, 0, s>>>(g->U, g->x, (long long)g->n, g->P.N, g->partials,
                                                    &g->ds->maxdrho, &g->ds->unorm2, &g->ds->counters[CNT_NEWTON],
                                                    skip);
    else
        k_newton_update<false><<<g->nb, BS, 0, s>>>(g->U, g->x, (long long)g->n, g->P.N, g->partials,
                                                     &g->ds->maxdrho, &g->ds->unorm2, &g->ds->counters[CNT_NEWTON],
                                                     skip);
    CHECK_LAUNCH();
    return MUSIC_OK;
}
