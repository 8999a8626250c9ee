// Arithmetic throughput of the GPU the library runs on, measured: FP64 and
// FP32 fused multiply-adds and FP64 divisions per second.  These are the
// ceilings the FP64-bound stencil and the FP32 kernels are judged against;
// the GPU's vendor figures are not published for every part, and a clock
// under load differs from the nominal one.
#include "internal.h"

namespace {

constexpr int PB = 256;      // threads per block
constexpr int PCH = 8;       // independent chains per thread
constexpr int PITER = 4096;  // dependent operations per chain

template <typename T>
__global__ void __launch_bounds__(PB) k_peak_fma(T *out, T a, T b)
{
    pdl_entry();
    T x[PCH];
#pragma unroll
    for (int k = 0; k < PCH; k++) x[k] = (T)(threadIdx.x & 7) + (T)k;
    for (int i = 0; i < PITER; i++)
#pragma unroll
        for (int k = 0; k < PCH; k++) x[k] = fma(x[k], a, b);
    T s = 0;
#pragma unroll
    for (int k = 0; k < PCH; k++) s += x[k];
    out[blockIdx.x * PB + threadIdx.x] = s;  // keeps every chain live
}

// x <- b / (x + c): one IEEE division per step
__global__ void __launch_bounds__(PB) k_peak_div(double *out, double b, double c)
{
    pdl_entry();
    double x[PCH];
#pragma unroll
    for (int k = 0; k < PCH; k++) x[k] = 1.0 + (double)(threadIdx.x & 7) + k;
    for (int i = 0; i < PITER / 8; i++)
#pragma unroll
        for (int k = 0; k < PCH; k++) x[k] = b / (x[k] + c);
    double s = 0;
#pragma unroll
    for (int k = 0; k < PCH; k++) s += x[k];
    out[blockIdx.x * PB + threadIdx.x] = s;
}

// best of `reps` timed launches (after one warm-up), in ms
template <typename L>
int time_best(L launch, int reps, cudaStream_t s, cudaEvent_t e0, cudaEvent_t e1, float *best)
{
    TRY(launch());
    *best = 1e30f;
    for (int r = 0; r < reps; r++) {
        CUDA_TRY(cudaEventRecord(e0, s));
        TRY(launch());
        CUDA_TRY(cudaEventRecord(e1, s));
        CUDA_TRY(cudaEventSynchronize(e1));
        float ms = 0.0f;
        CUDA_TRY(cudaEventElapsedTime(&ms, e0, e1));
        if (ms < *best) *best = ms;
    }
    return MUSIC_OK;
}

}  // namespace

extern "C" int music_measure_peaks(music_peaks *out, void *stream)
{
    if (!out) {
        set_error("music_measure_peaks: NULL argument");
        return MUSIC_E_INVAL;
    }
    cudaStream_t s = (cudaStream_t)stream;
    int dev = 0, sms = 0;
    CUDA_TRY(cudaGetDevice(&dev));
    CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const int blocks = sms * 8;  // eight resident blocks of 256 threads per SM
    const double threads = (double)blocks * PB;
    void *buf = nullptr;
    CUDA_TRY(cudaMallocAsync(&buf, (size_t)blocks * PB * sizeof(double), s));
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    int rc = MUSIC_OK;
    float ms_d = 0.0f, ms_f = 0.0f, ms_v = 0.0f;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
        cudaGetLastError();
        set_error("music_measure_peaks: event creation failed");
        rc = MUSIC_E_CUDA;
    }
    auto dfma = [&] {
        k_peak_fma<double><<<blocks, PB, 0, s>>>((double *)buf, 0.999999, 1e-7);
        CHECK_LAUNCH();
        return MUSIC_OK;
    };
    auto ffma = [&] {
        k_peak_fma<float><<<blocks, PB, 0, s>>>((float *)buf, 0.999999f, 1e-7f);
        CHECK_LAUNCH();
        return MUSIC_OK;
    };
    auto ddiv = [&] {
        k_peak_div<<<blocks, PB, 0, s>>>((double *)buf, 1.5, 0.25);
        CHECK_LAUNCH();
        return MUSIC_OK;
    };
    if (rc == MUSIC_OK) rc = time_best(dfma, 5, s, e0, e1, &ms_d);
    if (rc == MUSIC_OK) rc = time_best(ffma, 5, s, e0, e1, &ms_f);
    if (rc == MUSIC_OK) rc = time_best(ddiv, 5, s, e0, e1, &ms_v);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaFreeAsync(buf, s);
    if (cudaStreamSynchronize(s) != cudaSuccess && rc == MUSIC_OK) {
        cudaGetLastError();
        set_error("music_measure_peaks: stream failed");
        rc = MUSIC_E_CUDA;
    }
    if (rc != MUSIC_OK) return rc;
    const double fma_ops = threads * PCH * PITER;
    out->fp64_fma_tflops = 2.0 * fma_ops / (ms_d * 1e-3) / 1e12;
    out->fp32_fma_tflops = 2.0 * fma_ops / (ms_f * 1e-3) / 1e12;
    out->fp64_div_gops = threads * PCH * (PITER / 8) / (ms_v * 1e-3) / 1e9;
    out->sms = sms;
    return MUSIC_OK;
}
