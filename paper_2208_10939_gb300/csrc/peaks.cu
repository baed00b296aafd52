// Arithmetic-pipe peak microbenchmarks (bart_measure_peaks): the rates the
// echo-synthesis roofline is quoted against.  Each kernel keeps eight
// independent dependency chains per thread in registers (no memory traffic
// inside the timed loop), runs 2048 threads on every SM, and is timed with
// CUDA events; the best of several runs is kept.
//   fp32      : scalar fmaf                       one FMA-pipe operation each
//   fp32x2    : packed fma.rn.f32x2 (sm_100+)     two operations each (one per lane)
//   sincos    : __sincosf (MUFU sin + cos)        one sincos pair each
//   fp64      : fma on doubles                    one FP64 operation each
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <cstring>

#include "bart_internal.cuh"
#include "bartsim.h"

namespace {

constexpr int kThreads = 256;
constexpr int kChains = 8;

__global__ void __launch_bounds__(kThreads) peak_fp32_kernel(float *out, int iters, float a, float b)
{
    float x[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = (float)(threadIdx.x + c) * 1e-3f;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int u = 0; u < 16; ++u)
#pragma unroll
            for (int c = 0; c < kChains; ++c) x[c] = fmaf(x[c], a, b);
    }
    float s = 0.f;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += x[c];
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

__global__ void __launch_bounds__(kThreads) peak_fp32x2_kernel(float *out, int iters, float a, float b)
{
    uint64_t x[kChains], A, B;
    asm("mov.b64 %0, {%1, %2};" : "=l"(A) : "f"(a), "f"(a));
    asm("mov.b64 %0, {%1, %2};" : "=l"(B) : "f"(b), "f"(b));
#pragma unroll
    for (int c = 0; c < kChains; ++c) {
        const float v0 = (float)(threadIdx.x + c) * 1e-3f, v1 = v0 + 0.5f;
        asm("mov.b64 %0, {%1, %2};" : "=l"(x[c]) : "f"(v0), "f"(v1));
    }
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int u = 0; u < 16; ++u)
#pragma unroll
            for (int c = 0; c < kChains; ++c)
                asm volatile("fma.rn.f32x2 %0, %0, %1, %2;" : "+l"(x[c]) : "l"(A), "l"(B));
    }
    float s = 0.f;
#pragma unroll
    for (int c = 0; c < kChains; ++c) {
        float lo, hi;
        asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(x[c]));
        s += lo + hi;
    }
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

__global__ void __launch_bounds__(kThreads) peak_sincos_kernel(float *out, int iters, float a, float b)
{
    float x[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = (float)(threadIdx.x + c) * 1e-3f;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
            for (int c = 0; c < kChains; ++c) {
                float sn, cs;
                __sincosf(x[c], &sn, &cs);
                x[c] = fmaf(sn, a, cs * b);
            }
    }
    float s = 0.f;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += x[c];
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

__global__ void __launch_bounds__(kThreads) peak_fp64_kernel(float *out, int iters, double a, double b)
{
    double x[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = (double)(threadIdx.x + c) * 1e-3;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
            for (int c = 0; c < kChains; ++c) x[c] = fma(x[c], a, b);
    }
    double s = 0.0;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += x[c];
    out[blockIdx.x * blockDim.x + threadIdx.x] = (float)s;
}

// best time (s) of reps runs of one launch, after one warm-up run
template <typename L>
int time_best(L launch, int reps, cudaEvent_t e0, cudaEvent_t e1, double *best)
{
    *best = 1e30;
    for (int r = 0; r <= reps; ++r) {
        if (cudaEventRecord(e0) != cudaSuccess) return BART_ECUDA;
        launch();
        if (cudaEventRecord(e1) != cudaSuccess) return BART_ECUDA;
        if (cudaEventSynchronize(e1) != cudaSuccess) return BART_ECUDA;
        if (cudaGetLastError() != cudaSuccess) return BART_ECUDA;
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) return BART_ECUDA;
        if (r > 0) *best = std::min(*best, (double)ms * 1e-3);
    }
    return BART_OK;
}

}  // namespace

extern "C" int bart_measure_peaks(int32_t device, int32_t reps, bart_peaks *out)
{
    using bart::set_last_error;
    if (!out || reps < 1 || reps > 100)
        return set_last_error(BART_EINVAL, "bart_measure_peaks: NULL out or reps outside [1, 100]");
    std::memset(out, 0, sizeof *out);
    int n = 0;
    if (cudaGetDeviceCount(&n) != cudaSuccess || device < 0 || device >= n) {
        cudaGetLastError();
        return set_last_error(BART_EINVAL, "bart_measure_peaks: no such CUDA device");
    }
    if (cudaSetDevice(device) != cudaSuccess)
        return set_last_error(BART_ECUDA, "bart_measure_peaks: cudaSetDevice failed");
    int sms = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess)
        return set_last_error(BART_ECUDA, "bart_measure_peaks: cudaDeviceGetAttribute failed");
    const int blocks = sms * (2048 / kThreads);
    const int64_t threads = (int64_t)blocks * kThreads;
    float *buf = nullptr;
    if (cudaMalloc(&buf, (size_t)threads * sizeof(float)) != cudaSuccess) {
        cudaGetLastError();
        return set_last_error(BART_ENOMEM, "bart_measure_peaks: cudaMalloc failed");
    }
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    int rc = BART_OK;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) rc = BART_ECUDA;
    const int it32 = 8192, itmufu = 2048, it64 = 256;
    double t = 0.0;
    if (rc == BART_OK)
        rc = time_best([&] { peak_fp32_kernel<<<blocks, kThreads>>>(buf, it32, 0.999999f, 1e-7f); },
                       reps, e0, e1, &t);
    if (rc == BART_OK) out->fp32_fma_per_s = (double)threads * it32 * 16 * kChains / t;
    if (rc == BART_OK)
        rc = time_best([&] { peak_fp32x2_kernel<<<blocks, kThreads>>>(buf, it32, 0.999999f, 1e-7f); },
                       reps, e0, e1, &t);
    if (rc == BART_OK) out->fp32x2_fma_per_s = 2.0 * (double)threads * it32 * 16 * kChains / t;
    if (rc == BART_OK)
        rc = time_best([&] { peak_sincos_kernel<<<blocks, kThreads>>>(buf, itmufu, 0.7f, 0.6f); },
                       reps, e0, e1, &t);
    if (rc == BART_OK) out->sincos_per_s = (double)threads * itmufu * 4 * kChains / t;
    if (rc == BART_OK)
        rc = time_best([&] { peak_fp64_kernel<<<blocks, kThreads>>>(buf, it64, 0.999999, 1e-7); },
                       reps, e0, e1, &t);
    if (rc == BART_OK) out->fp64_fma_per_s = (double)threads * it64 * 4 * kChains / t;
    out->sms = sms;
    out->threads = (int32_t)threads;
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaFree(buf);
    cudaGetLastError();
    if (rc != BART_OK) return set_last_error(rc, "bart_measure_peaks: a timed launch failed");
    set_last_error(BART_OK, "");
    return BART_OK;
}
