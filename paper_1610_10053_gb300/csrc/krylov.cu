// Vector kernels of the GMRES / Newton loop (Saad & Schultz 1986, cited in
// Sec. 2): classical Gram-Schmidt with one re-orthogonalisation, each pass a
// sweep over w and up to eight basis vectors (more in further sweeps) with
// FP64 accumulation; norms; the cycle's correction from the stored
// preconditioned basis; the Newton update with its density-correction test.
//
// Every sweep takes its vectors in 16-byte chunks (4 floats or 2 doubles;
// element by element when a vector's length is not a multiple of 16 bytes).
// A thread owns a fixed set of chunks and issues the loads of K of them, in
// every vector the pass reads, before it uses any: at the few chunks a
// thread owns here, a pass is bound by the latency of its loads, and one
// round trip per K chunks instead of one per chunk and vector is what makes
// it fast.  The passes are specialised on the number of basis vectors they
// read together (1 to 8), so those loads are independent instructions.
//
// Reductions are two-stage and deterministic: every block writes one partial
// per quantity, then the last block to finish sums the partials in block
// order.  The block count and the chunks of every thread depend on the
// vector length alone, so results do not depend on timing.
#include <cmath>

#include "internal.h"
#include "ctl.cuh"

namespace {

constexpr int BS = 256;
constexpr int NG = 8;  // basis vectors a sweep reads together

struct Coef {
    double c[MUSIC_MAXV];
};

// ---------------------------------------------------------------- chunks
template <typename T, int W>
struct Ch {
    T v[W];
};

template <typename T, int W>
__device__ __forceinline__ Ch<T, W> ldch(const T *p, long long c)
{
    static_assert(W == 1 || W * sizeof(T) == 16, "a chunk is one element or 16 bytes");
    Ch<T, W> r;
    if constexpr (W == 1) {
        r.v[0] = p[c];
    } else if constexpr (sizeof(T) == 4) {
        const float4 a = reinterpret_cast<const float4 *>(p)[c];
        r.v[0] = a.x;
        r.v[1] = a.y;
        r.v[2] = a.z;
        r.v[3] = a.w;
    } else {
        const double2 a = reinterpret_cast<const double2 *>(p)[c];
        r.v[0] = a.x;
        r.v[1] = a.y;
    }
    return r;
}

template <typename T, int W>
__device__ __forceinline__ void stch(T *p, long long c, const Ch<T, W> &r)
{
    if constexpr (W == 1) {
        p[c] = r.v[0];
    } else if constexpr (sizeof(T) == 4) {
        reinterpret_cast<float4 *>(p)[c] = make_float4(r.v[0], r.v[1], r.v[2], r.v[3]);
    } else {
        reinterpret_cast<double2 *>(p)[c] = make_double2(r.v[0], r.v[1]);
    }
}

template <typename T, int W>
__device__ __forceinline__ Ch<T, W> zero_ch()
{
    Ch<T, W> r;
#pragma unroll
    for (int e = 0; e < W; e++) r.v[e] = (T)0;
    return r;
}

// chunk c of a load that may lie beyond the last chunk (then zero)
template <typename T, int W>
__device__ __forceinline__ Ch<T, W> ldch_or0(const T *p, long long c, bool in)
{
    return in ? ldch<T, W>(p, c) : zero_ch<T, W>();
}

__device__ __forceinline__ float fmat(float a, float b, float c) { return fmaf(a, b, c); }
__device__ __forceinline__ double fmat(double a, double b, double c) { return fma(a, b, c); }

// The chunks of a sweep: step s of thread t (of T in the grid) takes chunks
// s K T + k T + t, k < K, consecutive threads reading consecutive chunks.
struct Sweep {
    long long T, t;
    __device__ Sweep() : T((long long)gridDim.x * BS), t(blockIdx.x * (long long)BS + threadIdx.x) {}
};

// Block partials of cnt <= NG per-thread sums: each warp adds its lanes'
// values (in FP32 for an FP32 basis, a fixed tree of five levels), then one
// thread per sum adds the warps' results in FP64 in warp order and writes
// partial[i * nb + block].  Ends with a barrier, so it may be called again.
template <typename KT>
__device__ __forceinline__ void block_partials(const double *acc, int cnt, double *partial, int nb)
{
    __shared__ double ws[NG][BS / 32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int i = 0; i < NG; i++) {
        if (i < cnt) {
            if constexpr (sizeof(KT) == 4) {
                float v = (float)acc[i];
                for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
                if (lane == 0) ws[i][wid] = (double)v;
            } else {
                double v = acc[i];
                for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
                if (lane == 0) ws[i][wid] = v;
            }
        }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < cnt; i += BS) {
        double t = 0.0;
        for (int w = 0; w < BS / 32; w++) t += ws[i][w];
        partial[(long long)i * nb + blockIdx.x] = t;
    }
    __syncthreads();
}

// |x|^2: squares summed in T over each step's K chunks, then in FP64
template <typename T, int W>
__global__ void __launch_bounds__(BS, 2) k_sumsq(const T *x, long long n, double *partial, double *dst,
                                              unsigned int *counter)
{
    pdl_entry();
    constexpr int K = 4;
    __shared__ double sh[BS / 32];
    const Sweep S;
    const long long nc = n / W;
    double s = 0.0;
    for (long long base = 0; base < nc; base += K * S.T) {
        Ch<T, W> xc[K];
#pragma unroll
        for (int k = 0; k < K; k++) {
            const long long c = base + k * S.T + S.t;
            xc[k] = ldch_or0<T, W>(x, c, c < nc);
        }
        T r = (T)0;
#pragma unroll
        for (int k = 0; k < K; k++)
#pragma unroll
            for (int e = 0; e < W; e++) r = fmat(xc[k].v[e], xc[k].v[e], r);
        s += (double)r;
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

// ---------------------------------------------------------------- CGS passes
// The passes of one Arnoldi step's CGS2 (classical Gram-Schmidt with one
// re-orthogonalisation), as block partials, one kernel each.  Products are
// summed in KT over each step's chunks, then in FP64.

// acc[i] = <V_{i0+i}, w> over the thread's chunks, i < J; with Zj, also
// Zj = zs over the same chunks (pass 1 stores the preconditioned vector)
template <typename KT, int W, int J, int K>
__device__ __forceinline__ void dots_group(const KT *V, const KT *w, long long n, int i0, double *acc,
                                           const KT *zs, KT *Zj)
{
    const Sweep S;
    const long long nc = n / W;
#pragma unroll
    for (int i = 0; i < J; i++) acc[i] = 0.0;
    for (long long base = 0; base < nc; base += K * S.T) {
        Ch<KT, W> wc[K], vc[J][K];
#pragma unroll
        for (int k = 0; k < K; k++) {
            const long long c = base + k * S.T + S.t;
            const bool in = c < nc;
            wc[k] = ldch_or0<KT, W>(w, c, in);
#pragma unroll
            for (int i = 0; i < J; i++) vc[i][k] = ldch_or0<KT, W>(V + (long long)(i0 + i) * n, c, in);
            if (Zj && in) stch<KT, W>(Zj, c, ldch<KT, W>(zs, c));
        }
#pragma unroll
        for (int i = 0; i < J; i++) {
            KT r = (KT)0;
#pragma unroll
            for (int k = 0; k < K; k++)
#pragma unroll
                for (int e = 0; e < W; e++) r = fmat(vc[i][k].v[e], wc[k].v[e], r);
            acc[i] += (double)r;
        }
    }
}

// chunks a step of a pass reading J basis vectors: fewer when more vectors
// come with each chunk (registers)
template <int J>
constexpr int steps_k() { return J <= 3 ? 4 : 2; }

// dots_group for cnt = 1..NG vectors (cnt known on the device only)
template <typename KT, int W>
__device__ __forceinline__ void dots_any(int cnt, const KT *V, const KT *w, long long n, int i0, double *acc,
                                         const KT *zs, KT *Zj)
{
    switch (cnt) {
    case 1: dots_group<KT, W, 1, steps_k<1>()>(V, w, n, i0, acc, zs, Zj); break;
    case 2: dots_group<KT, W, 2, steps_k<2>()>(V, w, n, i0, acc, zs, Zj); break;
    case 3: dots_group<KT, W, 3, steps_k<3>()>(V, w, n, i0, acc, zs, Zj); break;
    case 4: dots_group<KT, W, 4, steps_k<4>()>(V, w, n, i0, acc, zs, Zj); break;
    case 5: dots_group<KT, W, 5, steps_k<5>()>(V, w, n, i0, acc, zs, Zj); break;
    case 6: dots_group<KT, W, 6, steps_k<6>()>(V, w, n, i0, acc, zs, Zj); break;
    case 7: dots_group<KT, W, 7, steps_k<7>()>(V, w, n, i0, acc, zs, Zj); break;
    default: dots_group<KT, W, 8, steps_k<8>()>(V, w, n, i0, acc, zs, Zj); break;
    }
}

// Pass 1: h_i = <V_i, w>, i <= j, in groups of NG vectors (each group one
// sweep over w), block partials at partial[i * nb + block]; the first group
// also stores Z_j = zs when Zb is given.
template <typename KT, int W>
__device__ __forceinline__ void cgs_dots_pass(const KT *V, const KT *w, long long n, int j, double *partial, int nb,
                                              const KT *zs, KT *Zb)
{
    for (int i0 = 0; i0 <= j; i0 += NG) {
        const int cnt = min(NG, j + 1 - i0);
        double acc[NG];
        dots_any<KT, W>(cnt, V, w, n, i0, acc, zs, (Zb && i0 == 0) ? Zb + (long long)j * n : nullptr);
        block_partials<KT>(acc, cnt, partial + (long long)i0 * nb, nb);
    }
}

// w <- w - sum_{i<J} h_i V_i (J <= NG), in the order of i, then the products
// <V_i, w> (acc[0, J)) or, with NORM, |w|^2 (acc[0]) from the values in
// registers
template <typename KT, int W, int J, int K, bool NORM>
__device__ __forceinline__ void update_group(const KT *V, KT *w, long long n, const KT *hs, double *acc)
{
    const Sweep S;
    const long long nc = n / W;
#pragma unroll
    for (int i = 0; i < J; i++) acc[i] = 0.0;
    for (long long base = 0; base < nc; base += K * S.T) {
        Ch<KT, W> wc[K], vc[J][K];
#pragma unroll
        for (int k = 0; k < K; k++) {
            const long long c = base + k * S.T + S.t;
            const bool in = c < nc;
            wc[k] = ldch_or0<KT, W>(w, c, in);
#pragma unroll
            for (int i = 0; i < J; i++) vc[i][k] = ldch_or0<KT, W>(V + (long long)i * n, c, in);
        }
#pragma unroll
        for (int k = 0; k < K; k++) {
#pragma unroll
            for (int i = 0; i < J; i++) {
                const KT cf = -hs[i];
#pragma unroll
                for (int e = 0; e < W; e++) wc[k].v[e] = fmat(cf, vc[i][k].v[e], wc[k].v[e]);
            }
            const long long c = base + k * S.T + S.t;
            if (c < nc) stch<KT, W>(w, c, wc[k]);
        }
        if (NORM) {
            KT r = (KT)0;
#pragma unroll
            for (int k = 0; k < K; k++)
#pragma unroll
                for (int e = 0; e < W; e++) r = fmat(wc[k].v[e], wc[k].v[e], r);
            acc[0] += (double)r;
        } else {
#pragma unroll
            for (int i = 0; i < J; i++) {
                KT r = (KT)0;
#pragma unroll
                for (int k = 0; k < K; k++)
#pragma unroll
                    for (int e = 0; e < W; e++) r = fmat(vc[i][k].v[e], wc[k].v[e], r);
                acc[i] += (double)r;
            }
        }
    }
}

// The same update for jp1 > NG vectors: per step, the basis in groups of NG
// (each group's loads issued together), the coefficients still applied in
// the order of i; with NORM also |w|^2 (acc[0])
template <typename KT, int W, int K, bool NORM>
__device__ __forceinline__ void update_long(const KT *V, KT *w, long long n, int jp1, const KT *hs, double *acc)
{
    const Sweep S;
    const long long nc = n / W;
    acc[0] = 0.0;
    for (long long base = 0; base < nc; base += K * S.T) {
        Ch<KT, W> wc[K];
#pragma unroll
        for (int k = 0; k < K; k++) {
            const long long c = base + k * S.T + S.t;
            wc[k] = ldch_or0<KT, W>(w, c, c < nc);
        }
        for (int g0 = 0; g0 < jp1; g0 += NG) {
            const int cnt = min(NG, jp1 - g0);
            Ch<KT, W> vc[NG][K];
#pragma unroll
            for (int k = 0; k < K; k++) {
                const long long c = base + k * S.T + S.t;
#pragma unroll
                for (int i = 0; i < NG; i++)
                    vc[i][k] = ldch_or0<KT, W>(V + (long long)(g0 + i) * n, c, c < nc && i < cnt);
            }
#pragma unroll
            for (int k = 0; k < K; k++)
#pragma unroll
                for (int i = 0; i < NG; i++) {
                    if (i < cnt) {
                        const KT cf = -hs[g0 + i];
#pragma unroll
                        for (int e = 0; e < W; e++) wc[k].v[e] = fmat(cf, vc[i][k].v[e], wc[k].v[e]);
                    }
                }
        }
#pragma unroll
        for (int k = 0; k < K; k++) {
            const long long c = base + k * S.T + S.t;
            if (c < nc) stch<KT, W>(w, c, wc[k]);
        }
        if (NORM) {
            KT r = (KT)0;
#pragma unroll
            for (int k = 0; k < K; k++)
#pragma unroll
                for (int e = 0; e < W; e++) r = fmat(wc[k].v[e], wc[k].v[e], r);
            acc[0] += (double)r;
        }
    }
}

template <typename KT, int W, bool NORM>
__device__ __forceinline__ void update_any(int jp1, const KT *V, KT *w, long long n, const KT *hs, double *acc)
{
    switch (jp1) {
    case 1: update_group<KT, W, 1, steps_k<1>(), NORM>(V, w, n, hs, acc); break;
    case 2: update_group<KT, W, 2, steps_k<2>(), NORM>(V, w, n, hs, acc); break;
    case 3: update_group<KT, W, 3, steps_k<3>(), NORM>(V, w, n, hs, acc); break;
    case 4: update_group<KT, W, 4, steps_k<4>(), NORM>(V, w, n, hs, acc); break;
    case 5: update_group<KT, W, 5, steps_k<5>(), NORM>(V, w, n, hs, acc); break;
    case 6: update_group<KT, W, 6, steps_k<6>(), NORM>(V, w, n, hs, acc); break;
    case 7: update_group<KT, W, 7, steps_k<7>(), NORM>(V, w, n, hs, acc); break;
    case 8: update_group<KT, W, 8, steps_k<8>(), NORM>(V, w, n, hs, acc); break;
    default: update_long<KT, W, 2, NORM>(V, w, n, jp1, hs, acc); break;
    }
}

// Passes 2 and 3: w <- w - sum_i h_i V_i (coefficients rounded to the
// Krylov type), then the block partials of h2_i = <V_i, w> or, with NORM, of
// |w|^2.  Up to NG products ride on the update sweep; beyond that the
// updated w is swept again in groups.  h: the j + 1 coefficients.
template <bool NORM, typename KT, int W>
__device__ __forceinline__ void cgs_update_pass(const KT *V, KT *w, long long n, int j, const double *h,
                                                double *partial, int nb)
{
    __shared__ KT hs[MUSIC_MAXV];
    for (int i = threadIdx.x; i <= j; i += BS) hs[i] = (KT)h[i];
    __syncthreads();
    const int jp1 = j + 1;
    double acc[NG];
    update_any<KT, W, NORM>(jp1, V, w, n, hs, acc);
    if (NORM) {
        block_partials<KT>(acc, 1, partial, nb);
    } else if (jp1 <= NG) {
        block_partials<KT>(acc, jp1, partial, nb);
    } else {
        for (int i0 = 0; i0 < jp1; i0 += NG) {
            const int cnt = min(NG, jp1 - i0);
            dots_any<KT, W>(cnt, V, w, n, i0, acc, nullptr, nullptr);
            block_partials<KT>(acc, cnt, partial + (long long)i0 * nb, nb);
        }
    }
}

// h_i = <V_i, w>, i <= j (j read from jdev when given); with Zb, also Z_j = zs
template <typename KT, int W>
__global__ void __launch_bounds__(BS, 2) k_dots(const KT *V, const KT *w, long long n, int j, double *partial,
                                                double *dst, unsigned int *counter, const int *jdev, const KT *zs,
                                                KT *Zb)
{
    pdl_entry();
    if (jdev) j = *jdev;
    const int nb = gridDim.x;
    cgs_dots_pass<KT, W>(V, w, n, j, partial, nb, zs, Zb);
    if (last_block_done(counter)) finish_sums_warps<BS>(partial, nb, nb, j + 1, dst);
}

// w <- w - sum_i h_i V_i, then h2_i = <V_i, w> (second CGS pass) or, with
// NORM, |w|^2 only; with gc.c the last block then runs the Arnoldi step's
// Givens control
template <bool NORM, typename KT, int W>
__global__ void __launch_bounds__(BS, 2) k_update(const KT *V, KT *w, long long n, int j, const double *h,
                                                  double *partial, double *dst, unsigned int *counter,
                                                  const int *jdev, GivensCtl gc)
{
    pdl_entry();
    __shared__ double sh[BS / 32];
    if (jdev) j = *jdev;
    const int nb = gridDim.x;
    cgs_update_pass<NORM, KT, W>(V, w, n, j, h, partial, nb);
    if (last_block_done(counter)) {
        if (NORM)
            finish_sums<BS>(partial, nb, nb, 1, dst, sh);
        else
            finish_sums_warps<BS>(partial, nb, nb, j + 1, dst);
        // |w| is in *dst (written by thread 0): the Arnoldi step's control
        if (NORM && gc.c && threadIdx.x == 0) ctl_givens(gc.c, gc.ds, gc.h, gc.m, gc.cap);
    }
}

// ---------------------------------------------------------------- the rest
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

// the W FP64 values of x at the elements of chunk c (W of them, 16-byte
// aligned pairs when W > 1)
template <int W>
__device__ __forceinline__ void ldx(const double *x, long long c, double *out)
{
    if constexpr (W == 1) {
        out[0] = x[c];
    } else {
#pragma unroll
        for (int h = 0; h < W / 2; h++) {
            const double2 a = reinterpret_cast<const double2 *>(x)[c * (W / 2) + h];
            out[2 * h] = a.x;
            out[2 * h + 1] = a.y;
        }
    }
}

template <int W>
__device__ __forceinline__ void stx(double *x, long long c, const double *in)
{
    if constexpr (W == 1) {
        x[c] = in[0];
    } else {
#pragma unroll
        for (int h = 0; h < W / 2; h++) reinterpret_cast<double2 *>(x)[c * (W / 2) + h] = make_double2(in[2 * h], in[2 * h + 1]);
    }
}

// x += sum_{i<k} y_i Z_i: the cycle's correction M^-1 V y from the stored
// preconditioned basis Z_i = M^-1 V_i (V itself when unpreconditioned).
// Each element's sum runs over i in order in the Krylov type (coefficients
// rounded to it), then is added to x in FP64; the basis is read in groups of
// NG vectors whose loads are issued together.
template <typename KT, int W>
__global__ void __launch_bounds__(BS) k_correct(const KT *Z, double *x, long long n, int k, Coef y,
                                                const int *kdev, const double *ydev)
{
    pdl_entry();
    constexpr int K = 2;
    __shared__ KT ys[MUSIC_MAXV];
    if (kdev) k = *kdev;
    for (int i = threadIdx.x; i < k; i += BS) ys[i] = (KT)(ydev ? ydev[i] : y.c[i]);
    __syncthreads();
    const Sweep S;
    const long long nc = n / W;
    for (long long base = 0; base < nc; base += K * S.T) {
        KT s[K][W];
#pragma unroll
        for (int kk = 0; kk < K; kk++)
#pragma unroll
            for (int e = 0; e < W; e++) s[kk][e] = (KT)0;
        for (int g0 = 0; g0 < k; g0 += NG) {
            const int cnt = min(NG, k - g0);
            Ch<KT, W> zc[NG][K];
#pragma unroll
            for (int kk = 0; kk < K; kk++) {
                const long long c = base + kk * S.T + S.t;
#pragma unroll
                for (int i = 0; i < NG; i++)
                    zc[i][kk] = ldch_or0<KT, W>(Z + (long long)(g0 + i) * n, c, c < nc && i < cnt);
            }
#pragma unroll
            for (int kk = 0; kk < K; kk++)
#pragma unroll
                for (int i = 0; i < NG; i++)
                    if (i < cnt) {
#pragma unroll
                        for (int e = 0; e < W; e++) s[kk][e] = fmat(ys[g0 + i], zc[i][kk].v[e], s[kk][e]);
                    }
        }
#pragma unroll
        for (int kk = 0; kk < K; kk++) {
            const long long c = base + kk * S.T + S.t;
            if (c < nc) {
                double xv[W];
                ldx<W>(x, c, xv);
#pragma unroll
                for (int e = 0; e < W; e++) xv[e] += (double)s[kk][e];
                stx<W>(x, c, xv);
            }
        }
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
template <bool F32, int W>
__global__ void __launch_bounds__(BS, 2) k_newton_update(double *U, const double *x, long long n, long long N,
                                                      double *partial, double *dst, double *unorm2,
                                                      unsigned int *counter, const int *skip)
{
    pdl_entry();
    if (skip && *skip) return;  // a hard error ended the linear solve: U stays as it is
    constexpr int K = 4;
    __shared__ double sh[BS / 32];
    const Sweep S;
    const long long nc = n / W;
    double m = 0.0, q = 0.0;
    float m32 = 0.0f;
    for (long long base = 0; base < nc; base += K * S.T) {
        Ch<double, W> uc[K], xc[K];
#pragma unroll
        for (int k = 0; k < K; k++) {
            const long long c = base + k * S.T + S.t;
            const bool in = c < nc;
            uc[k] = ldch_or0<double, W>(U, c, in);
            xc[k] = ldch_or0<double, W>(x, c, in);
        }
#pragma unroll
        for (int k = 0; k < K; k++) {
            const long long c = base + k * S.T + S.t;
            if (c >= nc) continue;
#pragma unroll
            for (int e = 0; e < W; e++) {
                const double xe = xc[k].v[e], u = uc[k].v[e] + xe;
                uc[k].v[e] = u;
                q = fma(u, u, q);  // |U|^2 of the new iterate, for the next product's eps
                if (c * W + e < N) {
                    if (F32) {
                        const float t = fabsf((float)xe) / (float)u;
                        m32 = (t > m32 || t != t) ? t : m32;  // NaN-propagating, as nanmax
                    } else {
                        m = nanmax(m, fabs(xe) / u);
                    }
                }
            }
            stch<double, W>(U, c, uc[k]);
        }
    }
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

// Is a vector of n elements of T swept in 16-byte chunks?
template <typename T>
bool chunked(long long n)
{
    return (n * (long long)sizeof(T)) % 16 == 0;
}

// Blocks of a sweep over nc chunks taking K a step: enough for one step to
// cover the vector, rounded up to a whole number of blocks per SM beyond
// one per SM, at most VEC_BLOCKS_MAX (more steps then).  Depends on nc alone.
int sweep_blocks(long long nc, int K)
{
    long long b = (nc + (long long)BS * K - 1) / ((long long)BS * K);
    if (b > NUM_SMS) b = (b + NUM_SMS - 1) / NUM_SMS * NUM_SMS;
    if (b > VEC_BLOCKS_MAX) b = VEC_BLOCKS_MAX;
    if (b < 1) b = 1;
    return (int)b;
}

template <typename KT>
int launch_dots_t(music_grid *g, int j, const int *jdev, cudaStream_t s)
{
    const long long n = (long long)g->n;
    unsigned int *cnt = &g->ds->counters[CNT_DOTS];
    const KT *V = (const KT *)g->V, *w = (const KT *)g->w, *z = (const KT *)g->z;
    KT *Zb = (KT *)krylov_zstore(g);
    if (chunked<KT>(n)) {
        constexpr int W = 16 / sizeof(KT);
        k_dots<KT, W><<<sweep_blocks(n / W, 4), BS, 0, s>>>(V, w, n, j, g->partials, g->ds->h, cnt, jdev, z, Zb);
    } else {
        k_dots<KT, 1><<<sweep_blocks(n, 4), BS, 0, s>>>(V, w, n, j, g->partials, g->ds->h, cnt, jdev, z, Zb);
    }
    CHECK_LAUNCH();
    return MUSIC_OK;
}

int launch_dots(music_grid *g, int j, const int *jdev, cudaStream_t s)
{
    return g->mixed ? launch_dots_t<float>(g, j, jdev, s) : launch_dots_t<double>(g, j, jdev, s);
}

template <bool NORM, typename KT>
int launch_update_t(music_grid *g, int j, const int *jdev, const double *h, cudaStream_t s, const GivensCtl &gc)
{
    const long long n = (long long)g->n;
    double *dst = NORM ? &g->ds->wnorm2 : g->ds->h2;
    unsigned int *cnt = &g->ds->counters[NORM ? CNT_NORMW : CNT_UPDATE];
    const KT *V = (const KT *)g->V;
    KT *w = (KT *)g->w;
    if (chunked<KT>(n)) {
        constexpr int W = 16 / sizeof(KT);
        k_update<NORM, KT, W><<<sweep_blocks(n / W, 4), BS, 0, s>>>(V, w, n, j, h, g->partials, dst, cnt, jdev, gc);
    } else {
        k_update<NORM, KT, 1><<<sweep_blocks(n, 4), BS, 0, s>>>(V, w, n, j, h, g->partials, dst, cnt, jdev, gc);
    }
    CHECK_LAUNCH();
    return MUSIC_OK;
}

template <bool NORM>
int launch_update(music_grid *g, int j, const int *jdev, const double *h, cudaStream_t s, const GivensCtl *gcp)
{
    const GivensCtl gc = gcp ? *gcp : GivensCtl{};
    return g->mixed ? launch_update_t<NORM, float>(g, j, jdev, h, s, gc)
                    : launch_update_t<NORM, double>(g, j, jdev, h, s, gc);
}

template <typename T>
int launch_sumsq(music_grid *g, const T *x, long long n, double *dst, cudaStream_t s)
{
    unsigned int *cnt = &g->ds->counters[CNT_SUMSQ];
    if (chunked<T>(n)) {
        constexpr int W = 16 / sizeof(T);
        k_sumsq<T, W><<<sweep_blocks(n / W, 4), BS, 0, s>>>(x, n, g->partials, dst, cnt);
    } else {
        k_sumsq<T, 1><<<sweep_blocks(n, 4), BS, 0, s>>>(x, n, g->partials, dst, cnt);
    }
    CHECK_LAUNCH();
    return MUSIC_OK;
}

}  // namespace

int dev_norm2(music_grid *g, const void *x, int is_double, size_t n, double *dst, cudaStream_t s)
{
    ProfScope prof_(g, MUSIC_PROF_VECTOR, s);
    return is_double ? launch_sumsq<double>(g, (const double *)x, (long long)n, dst, s)
                     : launch_sumsq<float>(g, (const float *)x, (long long)n, dst, s);
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
int update_pass(music_grid *g, int j, const int *jdev, cudaStream_t s, const GivensCtl *gc)
{
    ProfScope prof_(g, MUSIC_PROF_VECTOR, s);
    return launch_update<NORM>(g, j, jdev, NORM ? g->ds->h2 : g->ds->h, s, gc);
}

int krylov_update_dots(music_grid *g, int j, const int *jdev, cudaStream_t s)
{
    return update_pass<false>(g, j, jdev, s, nullptr);
}

int krylov_update_norm(music_grid *g, int j, const int *jdev, cudaStream_t s, const GivensCtl *gc)
{
    return update_pass<true>(g, j, jdev, s, gc);
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
    const void *Z = krylov_zstore(g) ? krylov_zstore(g) : g->V;
    if (g->mixed) {
        if (chunked<float>(n))
            k_correct<float, 4><<<grid_blocks((n / 4 + 1) / 2, 152 * 16), BS, 0, s>>>((const float *)Z, g->x, n, k, c,
                                                                                    kdev, ydev);
        else
            k_correct<float, 1><<<grid_blocks((n + 1) / 2, 152 * 16), BS, 0, s>>>((const float *)Z, g->x, n, k, c, kdev,
                                                                                ydev);
    } else {
        if (chunked<double>(n))
            k_correct<double, 2><<<grid_blocks((n / 2 + 1) / 2, 152 * 16), BS, 0, s>>>((const double *)Z, g->x, n, k,
                                                                                     c, kdev, ydev);
        else
            k_correct<double, 1><<<grid_blocks((n + 1) / 2, 152 * 16), BS, 0, s>>>((const double *)Z, g->x, n, k, c,
                                                                                 kdev, ydev);
    }
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

template <bool F32>
int newton_update_t(music_grid *g, const int *skip, cudaStream_t s)
{
    const long long n = (long long)g->n;
    double *const dst = &g->ds->maxdrho, *const un = &g->ds->unorm2;
    unsigned int *cnt = &g->ds->counters[CNT_NEWTON];
    if (chunked<double>(n))
        k_newton_update<F32, 2><<<sweep_blocks(n / 2, 4), BS, 0, s>>>(g->U, g->x, n, g->P.N, g->partials, dst, un,
                                                                      cnt, skip);
    else
        k_newton_update<F32, 1><<<sweep_blocks(n, 4), BS, 0, s>>>(g->U, g->x, n, g->P.N, g->partials, dst, un, cnt,
                                                                  skip);
    CHECK_LAUNCH();
    return MUSIC_OK;
}

int newton_update(music_grid *g, const int *skip, cudaStream_t s)
{
    ProfScope prof_(g, MUSIC_PROF_VECTOR, s);
    return g->mixed ? newton_update_t<true>(g, skip, s) : newton_update_t<false>(g, skip, s);
}
