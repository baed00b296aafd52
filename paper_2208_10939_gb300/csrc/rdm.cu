// Range-Doppler map (Sec. 3.3): per channel, a windowed forward FFT over the
// M fast-time samples of every chirp (range), then a windowed forward FFT
// over the N chirps of every range bin (Doppler); |.|^2 summed over the O
// channels; the Doppler axis shifted so that zero velocity is bin N/2.
//
// Mixed-radix (2, 3) Stockham autosort FFTs in shared memory
// (fft_stockham.cuh).  Both passes are HBM-bound: each reads and writes the
// cube once.
#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <type_traits>

#include "bart_internal.cuh"
#include "fft_reg.cuh"
#include "fft_stockham.cuh"

namespace bart {

// one block per (channel, chirp) row
template <typename T>
__global__ void range_fft_kernel(const typename Cplx<T>::type *__restrict__ adc,
                                 typename Cplx<T>::type *__restrict__ X, int M, int window)
{
    using C = typename Cplx<T>::type;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C *buf0 = reinterpret_cast<C *>(smem_raw);
    C *buf1 = buf0 + M;
    C *tw = buf1 + M;
    fill_twiddles<T>(tw, M);
    const int64_t row = blockIdx.x;
    const C *in = adc + row * M;
    for (int i = threadIdx.x; i < M; i += blockDim.x) {
        const T w = window_val<T>(i, M, window);
        C v = in[i];
        v.x *= w;
        v.y *= w;
        buf0[i] = v;
    }
    __syncthreads();
    const C *res = stockham<C, T>(buf0, buf1, tw, M, 1);
    C *out = X + row * M;
    for (int i = threadIdx.x; i < M; i += blockDim.x) out[i] = res[i];
}

// one block per (RB consecutive range bins, channel): Doppler FFT of the
// channel's RB columns, the complex Y written, [o][r][d'] (summed by
// rdm_cube_sum_kernel and kept for the angle spectrum and the adjoint); d' is
// the Doppler bin after the N/2 shift.
template <typename T>
__global__ void doppler_kernel(const typename Cplx<T>::type *__restrict__ X, int N, int M,
                               int RB, int window, typename Cplx<T>::type *__restrict__ cube_out)
{
    using C = typename Cplx<T>::type;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C *buf0 = reinterpret_cast<C *>(smem_raw);
    C *buf1 = buf0 + RB * N;
    C *tw = buf1 + RB * N;
    fill_twiddles<T>(tw, N);
    const int r0 = blockIdx.x * RB;
    const int o = blockIdx.y;
    // load X[o][n][r0 + c] into column-major buf0[c * N + n]
    for (int i = threadIdx.x; i < RB * N; i += blockDim.x) {
        const int n = i / RB, c = i % RB;
        const T w = window_val<T>(n, N, window);
        C v = X[((int64_t)o * N + n) * M + r0 + c];
        v.x *= w;
        v.y *= w;
        buf0[c * N + n] = v;
    }
    __syncthreads();
    const C *res = stockham<C, T>(buf0, buf1, tw, N, RB);
    for (int i = threadIdx.x; i < RB * N; i += blockDim.x) {
        const int c = i / N, d = i % N;
        const C v = res[i];
        const int ds = d + (N >> 1);
        cube_out[((int64_t)o * M + r0 + c) * N + (ds >= N ? ds - N : ds)] = v;
    }
}

// RDM[g][r][d] = sum over the O partial maps of group g, in order
template <typename T>
__global__ void rdm_sum_kernel(const T *__restrict__ pw, int O, int64_t MN, int groups,
                               float *__restrict__ rdm)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= MN * groups) return;
    const int64_t g = i / MN, j = i - g * MN;
    const T *src = pw + g * O * MN + j;
    T acc = (T)0;
    for (int o = 0; o < O; ++o) acc += src[(int64_t)o * MN];
    rdm[i] = (float)acc;
}

// RDM[r][d'] = sum over channels of |Y[o][r][d']|^2, in channel order
template <typename T>
__global__ void rdm_cube_sum_kernel(const typename Cplx<T>::type *__restrict__ Y, int O,
                                    int64_t MN, float *__restrict__ rdm)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= MN) return;
    T acc = (T)0;
    for (int o = 0; o < O; ++o) {
        const typename Cplx<T>::type v = Y[(int64_t)o * MN + i];
        acc += v.x * v.x + v.y * v.y;
    }
    rdm[i] = (float)acc;
}

// -------------------------------------------------------------------------
// The RDM without the complex range-Doppler cube (bart_form_rdm): the range
// pass transforms TN consecutive chirps of one channel per block and writes
// them transposed, Xt[o][r][n], so that the Doppler pass reads every range
// bin's N chirps as one contiguous run; the Doppler pass transforms RB range
// bins of a group of channels per block and sums |Y|^2 over the group's
// channels in shared memory, in channel order; the groups' partial maps are
// then added in group order.  HBM traffic per sample: ADC read, Xt write, Xt
// read (3 x 8 bytes for complex64) against 4 x 8 for a per-channel power
// array.
// -------------------------------------------------------------------------
template <typename T>
__global__ void range_fft_t_kernel(const typename Cplx<T>::type *__restrict__ adc,
                                   typename Cplx<T>::type *__restrict__ Xt, int N, int M, int TN,
                                   int window)
{
    using C = typename Cplx<T>::type;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C *buf0 = reinterpret_cast<C *>(smem_raw);
    C *buf1 = buf0 + TN * M;
    C *tw = buf1 + TN * M;
    fill_twiddles<T>(tw, M);
    const int o = blockIdx.y;
    const int n0 = blockIdx.x * TN;
    const int rows = min(TN, N - n0);
    const C *in = adc + ((int64_t)o * N + n0) * M;
    for (int i = threadIdx.x; i < TN * M; i += blockDim.x) {
        const int c = i / M, m = i % M;
        C v;
        if (c < rows) {
            v = in[i];
            const T w = window_val<T>(m, M, window);
            v.x *= w;
            v.y *= w;
        } else {
            v.x = v.y = (T)0;
        }
        buf0[i] = v;
    }
    __syncthreads();
    const C *res = stockham<C, T>(buf0, buf1, tw, M, TN);
    C *out = Xt + (int64_t)o * M * N + n0;
    for (int i = threadIdx.x; i < M * TN; i += blockDim.x) {
        const int r = i / TN, c = i % TN;
        if (c < rows) out[(int64_t)r * N + c] = res[c * M + r];
    }
}

template <typename T>
__global__ void doppler_sum_kernel(const typename Cplx<T>::type *__restrict__ Xt, int N, int M,
                                   int RB, int CPB, int O, int window, T *__restrict__ part)
{
    using C = typename Cplx<T>::type;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C *buf0 = reinterpret_cast<C *>(smem_raw);
    C *buf1 = buf0 + RB * N;
    C *tw = buf1 + RB * N;
    T *acc = reinterpret_cast<T *>(tw + tw_len(N));
    fill_twiddles<T>(tw, N);
    const int r0 = blockIdx.x * RB;
    const int gg = blockIdx.y;                       // group of channels (over all scenes)
    const int G = (O + CPB - 1) / CPB;               // groups per scene
    const int scene = gg / G, g = gg % G;
    const int o0 = scene * O + g * CPB, o1 = scene * O + min(O, (g + 1) * CPB);
    for (int i = threadIdx.x; i < RB * N; i += blockDim.x) acc[i] = (T)0;
    for (int o = o0; o < o1; ++o) {
        const C *src = Xt + ((int64_t)o * M + r0) * N;
        for (int i = threadIdx.x; i < RB * N; i += blockDim.x) {
            const int n = i % N;
            const T w = window_val<T>(n, N, window);
            C v = src[i];
            v.x *= w;
            v.y *= w;
            buf0[i] = v;
        }
        __syncthreads();
        const C *res = stockham<C, T>(buf0, buf1, tw, N, RB);
        for (int i = threadIdx.x; i < RB * N; i += blockDim.x) {
            const C v = res[i];
            acc[i] += v.x * v.x + v.y * v.y;
        }
        __syncthreads();
    }
    T *dst = part + (int64_t)gg * M * N;
    for (int i = threadIdx.x; i < RB * N; i += blockDim.x) {
        const int c = i / N, d = i % N;
        const int ds = d + (N >> 1);
        dst[(int64_t)(r0 + c) * N + (ds >= N ? ds - N : ds)] = acc[i];
    }
}

// -------------------------------------------------------------------------
// Register-resident variant (complex64, power-of-two M and N, fft_reg.cuh):
// the same two passes without the transposed intermediate.  The range pass
// keeps X[o][n][r] in natural order (each thread holds R0 samples of a row,
// loaded and stored with unit stride across the row's T threads); the
// Doppler pass gives each of RB consecutive range bins T threads (bins
// fastest, so a warp's loads of one chirp are RB consecutive complex) and
// sums |Y|^2 over its channel group in registers, each thread owning the
// same R0 cells for every channel.  Blocks loop over rows (range) or
// channels (Doppler) so that the per-thread twiddles and window values,
// computed once, serve many transforms.
// -------------------------------------------------------------------------
constexpr int kRegThreads = 256;

template <int M>
__global__ void __launch_bounds__(kRegThreads, 2)
range_fft_reg_kernel(const float2 *__restrict__ adc, float2 *__restrict__ X, int64_t rows,
                     int window)
{
    using namespace fftr;
    constexpr int R0 = Plan<M>::R0, T = M / R0, RPB = kRegThreads / T;
    __shared__ float2 buf[RPB * M];
    const int g = threadIdx.x / T, tid = threadIdx.x % T;
    FftTw<M> tw;
    tw.init(tid);
    float wv[R0];
#pragma unroll
    for (int k = 0; k < R0; ++k) wv[k] = window_val<float>(tid + T * k, M, window);
    const int64_t stride = (int64_t)gridDim.x * RPB;
    int64_t row = (int64_t)blockIdx.x * RPB + g;
    // the next row's samples are loaded while the current one is transformed
    float2 nx[R0];
#pragma unroll
    for (int k = 0; k < R0; ++k)
        nx[k] = row < rows ? adc[row * M + tid + T * k] : make_float2(0.f, 0.f);
    for (int64_t row0 = (int64_t)blockIdx.x * RPB; row0 < rows; row0 += stride, row += stride) {
        float2 a[R0];
#pragma unroll
        for (int k = 0; k < R0; ++k) a[k] = make_float2(nx[k].x * wv[k], nx[k].y * wv[k]);
        const int64_t next = row + stride;
#pragma unroll
        for (int k = 0; k < R0; ++k)
            nx[k] = next < rows ? adc[next * M + tid + T * k] : make_float2(0.f, 0.f);
        fft<M>(a, tid, buf + g * M, tw);
        if (row < rows) {
            float2 *out = X + row * M;
#pragma unroll
            for (int i = 0; i < R0; ++i) out[fft_out_index<M>(tid, i)] = a[i];
        }
        __syncthreads();      // buf is reused by the next row
    }
}

__device__ __forceinline__ void cp_async8(void *smem, const void *gmem)
{
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(
                     (unsigned)__cvta_generic_to_shared(smem)),
                 "l"(gmem)
                 : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int NPEND>
__device__ __forceinline__ void cp_async_wait()
{
    asm volatile("cp.async.wait_group %0;" ::"n"(NPEND) : "memory");
}

// Doppler pass over channels o0 .. o1 - 1 of the cube X ([o][n][r], rows of
// M range bins); the next channel's tile is copied into shared memory
// (cp.async, two stages) while the current one is transformed.
template <int N>
__global__ void __launch_bounds__(kRegThreads, 2)
doppler_sum_reg_kernel(const float2 *__restrict__ X, int M, int CPB, int O, int window,
                       float *__restrict__ part)
{
    using namespace fftr;
    constexpr int R0 = Plan<N>::R0, T = N / R0, RB = kRegThreads / T;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float2 *buf = reinterpret_cast<float2 *>(smem_raw);                 // RB (N + 1)
    float2 *stage = buf + RB * (N + 1);                                  // 2 x R0 x 256
    const int c = threadIdx.x % RB, tid = threadIdx.x / RB;
    FftTw<N> tw;
    tw.init(tid);
    float wv[R0];
#pragma unroll
    for (int k = 0; k < R0; ++k) wv[k] = window_val<float>(tid + T * k, N, window);
    const int r = blockIdx.x * RB + c;
    const int gg = blockIdx.y;                       // group of channels (over all scenes)
    const int G = (O + CPB - 1) / CPB;               // groups per scene
    const int scene = gg / G, gi = gg % G;
    const int o0 = scene * O + gi * CPB, o1 = scene * O + min(O, (gi + 1) * CPB);
    // a thread's own R0 samples of channel o into stage s: slot k at
    // (s R0 + k) 256 + threadIdx.x (a warp's slots are consecutive)
    auto issue = [&](int o, int st) {
        const float2 *in = X + ((int64_t)o * N + tid) * M + r;
#pragma unroll
        for (int k = 0; k < R0; ++k)
            cp_async8(stage + (st * R0 + k) * kRegThreads + threadIdx.x, in + (int64_t)T * k * M);
        cp_async_commit();
    };
    float acc[R0];
#pragma unroll
    for (int i = 0; i < R0; ++i) acc[i] = 0.f;
    if (o0 < o1) issue(o0, 0);
    for (int o = o0; o < o1; ++o) {
        const int st = (o - o0) & 1;
        if (o + 1 < o1) {
            issue(o + 1, st ^ 1);
            cp_async_wait<1>();
        } else {
            cp_async_wait<0>();
        }
        float2 a[R0];
#pragma unroll
        for (int k = 0; k < R0; ++k) {
            const float2 v = stage[(st * R0 + k) * kRegThreads + threadIdx.x];
            a[k] = make_float2(v.x * wv[k], v.y * wv[k]);
        }
        fft<N>(a, tid, buf + c * (N + 1), tw);
#pragma unroll
        for (int i = 0; i < R0; ++i) acc[i] = fmaf(a[i].x, a[i].x, fmaf(a[i].y, a[i].y, acc[i]));
        __syncthreads();
    }
    // the block's RB x N map through shared memory (the exchange buffer,
    // free after the last transform), then written row by row
    float *tile = reinterpret_cast<float *>(buf);
#pragma unroll
    for (int i = 0; i < R0; ++i) {
        const int d = fft_out_index<N>(tid, i);
        const int ds = d + (N >> 1);
        tile[c * (N + 1) + (ds >= N ? ds - N : ds)] = acc[i];
    }
    __syncthreads();
    float *dst = part + (int64_t)gg * M * N + (int64_t)blockIdx.x * RB * N;
    for (int j = threadIdx.x; j < RB * N; j += kRegThreads) {
        const float v = tile[(j / N) * (N + 1) + j % N];
        dst[j] = v;
    }
}

// -------------------------------------------------------------------------
// Doppler pass with TMA tile loads (N <= 256): the block's tile of channel o
// -- its RB range bins over the N chirps, a 2-D box of the cube X viewed as
// [O N] rows x [2 M] floats -- comes in by one cp.async.bulk.tensor copy,
// double-buffered and completed on an mbarrier.  One thread issues, every
// thread waits on the stage's barrier (bounded: on expiry the block records
// kStatusWaitTimeout, waits -- again bounded -- for its copy in flight and
// stops).  Otherwise as doppler_sum_reg_kernel.  A box dimension holds at
// most 256 elements, so the tile's 2 RB floats and N rows limit it to
// 32 <= N <= 256.
// -------------------------------------------------------------------------
constexpr int kTmaWaitLimit = 1 << 22;

__device__ __forceinline__ uint32_t smem_u32(const void *p)
{
    return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count)
                 : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
                 "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
// bounded wait for the phase `parity` of `bar`; false if the limit expired
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, uint32_t parity,
                                                  int limit = kTmaWaitLimit)
{
    for (int i = 0; i < limit; ++i)
        if (mbar_try_wait(bar, parity)) return true;
    return false;
}
__device__ __forceinline__ void tma_load_2d(void *dst, const CUtensorMap *map, int x, int y,
                                            uint64_t *bar)
{
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3}], [%4];" ::"r"(smem_u32(dst)),
        "l"(map), "r"(x), "r"(y), "r"(smem_u32(bar))
        : "memory");
}

// The expiry path of the bounded mbarrier wait, exercised on purpose: a
// barrier expecting one arrival that never comes, waited on by every thread
// for `polls` polls; on expiry the status word gets kStatusWaitTimeout, as
// in the Doppler pass.  The barrier is invalidated before the block exits.
__global__ void wait_selftest_kernel(int polls, int *status)
{
    __shared__ __align__(8) uint64_t bar;
    __shared__ int s_expired;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        s_expired = 0;
    }
    __syncthreads();
    if (!mbar_wait_bounded(&bar, 0u, polls)) s_expired = 1;
    __syncthreads();
    if (threadIdx.x == 0) {
        if (s_expired && status) atomicOr(status, kStatusWaitTimeout);
        asm volatile("mbarrier.inval.shared::cta.b64 [%0];" ::"r"(smem_u32(&bar)) : "memory");
    }
}

void launch_wait_selftest(int polls, int *status, cudaStream_t s)
{
    wait_selftest_kernel<<<1, 64, 0, s>>>(polls, status);
}

template <int N>
struct TmaDoppler {
    static constexpr int R0 = fftr::Plan<N>::R0, T = N / R0, RB = kRegThreads / T;
    static constexpr uint32_t kTileBytes = (uint32_t)N * RB * 8;
    // stage tiles (two, 1024-byte aligned), the exchange buffer, two barriers
    static constexpr size_t kStageOff = 0;
    static constexpr size_t kBufOff = 2 * (size_t)kTileBytes;
    static constexpr size_t kBarOff = kBufOff + (size_t)RB * (N + 1) * 8;
    static constexpr size_t kSmem = kBarOff + 16 + 1024;     // + alignment slack
};

template <int N>
__global__ void __launch_bounds__(kRegThreads, 2)
doppler_sum_tma_kernel(const __grid_constant__ CUtensorMap tmap, int M, int CPB, int O,
                       int window, int *status, float *__restrict__ part)
{
    using namespace fftr;
    using Q = TmaDoppler<N>;
    constexpr int R0 = Q::R0, T = Q::T, RB = Q::RB;
    extern __shared__ unsigned char smem_dyn[];
    unsigned char *base = reinterpret_cast<unsigned char *>(
        (reinterpret_cast<uintptr_t>(smem_dyn) + 1023) & ~uintptr_t(1023));
    float2 *stage = reinterpret_cast<float2 *>(base + Q::kStageOff);      // [2][N][RB]
    float2 *buf = reinterpret_cast<float2 *>(base + Q::kBufOff);          // RB (N + 1)
    uint64_t *bar = reinterpret_cast<uint64_t *>(base + Q::kBarOff);      // [2]
    __shared__ int s_err;
    const int c = threadIdx.x % RB, tid = threadIdx.x / RB;
    const int r0 = blockIdx.x * RB;
    const int gg = blockIdx.y;
    const int G = (O + CPB - 1) / CPB;
    const int scene = gg / G, gi = gg % G;
    const int o0 = scene * O + gi * CPB, o1 = scene * O + min(O, (gi + 1) * CPB);
    if (threadIdx.x == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        s_err = 0;
    }
    __syncthreads();
    // thread 0: the tile of channel o into stage st (x in floats: 2 r0)
    auto issue = [&](int o, int st) {
        mbar_expect_tx(&bar[st], Q::kTileBytes);
        tma_load_2d(stage + (size_t)st * N * RB, &tmap, 2 * r0, o * N, &bar[st]);
    };
    if (threadIdx.x == 0 && o0 < o1) issue(o0, 0);
    FftTw<N> tw;
    tw.init(tid);
    float wv[R0];
#pragma unroll
    for (int k = 0; k < R0; ++k) wv[k] = window_val<float>(tid + T * k, N, window);
    float acc[R0];
#pragma unroll
    for (int i = 0; i < R0; ++i) acc[i] = 0.f;
    int o = o0;
    for (; o < o1; ++o) {
        const int it = o - o0, st = it & 1;
        // the other stage was released by the barrier that ended the last
        // iteration: its next tile goes in while this one is transformed
        if (threadIdx.x == 0 && o + 1 < o1) issue(o + 1, st ^ 1);
        if (!mbar_wait_bounded(&bar[st], (uint32_t)(it >> 1) & 1u)) s_err = 1;
        __syncthreads();
        if (s_err) break;
        const float2 *tile = stage + (size_t)st * N * RB;
        float2 a[R0];
#pragma unroll
        for (int k = 0; k < R0; ++k) {
            const float2 v = tile[(tid + T * k) * RB + c];
            a[k] = make_float2(v.x * wv[k], v.y * wv[k]);
        }
        fft<N>(a, tid, buf + c * (N + 1), tw);
#pragma unroll
        for (int i = 0; i < R0; ++i) acc[i] = fmaf(a[i].x, a[i].x, fmaf(a[i].y, a[i].y, acc[i]));
        __syncthreads();
    }
    if (s_err) {
        // stop: record the expiry, let the copy in flight (if any) land first
        if (threadIdx.x == 0) {
            if (status) atomicOr(status, kStatusWaitTimeout);
            const int it = o - o0;
            mbar_wait_bounded(&bar[it & 1], (uint32_t)(it >> 1) & 1u);
            if (o + 1 < o1) mbar_wait_bounded(&bar[(it + 1) & 1], (uint32_t)((it + 1) >> 1) & 1u);
        }
        __syncthreads();
        return;
    }
    float *tilem = reinterpret_cast<float *>(buf);
#pragma unroll
    for (int i = 0; i < R0; ++i) {
        const int d = fft_out_index<N>(tid, i);
        const int ds = d + (N >> 1);
        tilem[c * (N + 1) + (ds >= N ? ds - N : ds)] = acc[i];
    }
    __syncthreads();
    float *dst = part + (int64_t)gg * M * N + (int64_t)r0 * N;
    for (int j = threadIdx.x; j < RB * N; j += kRegThreads) dst[j] = tilem[(j / N) * (N + 1) + j % N];
}

using EncodeTiledFn = CUresult (*)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *,
                                   const cuuint64_t *, const cuuint64_t *, const cuuint32_t *,
                                   const cuuint32_t *, CUtensorMapInterleave, CUtensorMapSwizzle,
                                   CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

// the driver's tensor-map encoder, through the runtime's entry-point query
static EncodeTiledFn tensor_map_encoder()
{
    static const EncodeTiledFn fn = [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000,
                                             cudaEnableDefault, &q) != cudaSuccess ||
            q != cudaDriverEntryPointSuccess) {
            cudaGetLastError();
            return static_cast<EncodeTiledFn>(nullptr);
        }
        return reinterpret_cast<EncodeTiledFn>(p);
    }();
    return fn;
}

// TMA Doppler pass over X ([rows][M] complex64, rows = O groups N); false
// (nothing launched) when the tensor map cannot be made
template <int N>
static bool doppler_tma_launch(const float2 *X, int M, int O, int groups, int window, float *part,
                               int CPB, int *status, cudaStream_t s)
{
    using Q = TmaDoppler<N>;
    const EncodeTiledFn enc = tensor_map_encoder();
    if (!enc || (reinterpret_cast<uintptr_t>(X) & 15u) != 0) return false;
    CUtensorMap map;
    const cuuint64_t dims[2] = {(cuuint64_t)2 * M, (cuuint64_t)O * groups * N};
    const cuuint64_t strides[1] = {(cuuint64_t)M * sizeof(float2)};
    const cuuint32_t box[2] = {(cuuint32_t)(2 * Q::RB), (cuuint32_t)N};
    const cuuint32_t estr[2] = {1, 1};
    if (enc(&map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float2 *>(X), dims, strides, box,
            estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
            CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
        return false;
    const int G = (O + CPB - 1) / CPB;
    cudaFuncSetAttribute(doppler_sum_tma_kernel<N>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)Q::kSmem);
    doppler_sum_tma_kernel<N><<<dim3((unsigned int)(M / Q::RB), (unsigned int)(G * groups)),
                                kRegThreads, Q::kSmem, s>>>(map, M, CPB, O, window, status, part);
    return true;
}

template <int N>
static size_t doppler_reg_smem()
{
    constexpr int R0 = fftr::Plan<N>::R0, T = N / R0, RB = kRegThreads / T;
    return (size_t)(RB * (N + 1) + 2 * R0 * kRegThreads) * sizeof(float2);
}

// range bins per Doppler block: the largest power of two RB with RB N <= 512
// that divides M
// -------------------------------------------------------------------------
// adjoint of the RDM: for a real loss L(RDM) with dL/dRDM = G[r][d'],
//   Ybar[o][r][d'] = 2 G[r][d'] Y[o][r][d']            (|Y|^2 = Y conj(Y))
//   Xbar[o][n][r]  = w_d[n] sum_d exp(+2 pi i n d / N) Ybar[o][r][d]
//   xbar[o][n][m]  = w_r[m] sum_r exp(+2 pi i m r / M) Xbar[o][n][r]
// i.e. the conjugate transposes of the two windowed DFTs; gradients of
// complex tensors as d/dRe + i d/dIm.
// -------------------------------------------------------------------------
template <typename T>
__global__ void doppler_adjoint_kernel(const typename Cplx<T>::type *__restrict__ Y,
                                       const float *__restrict__ G, int O, int N, int M, int RB,
                                       int window, typename Cplx<T>::type *__restrict__ Xbar)
{
    using C = typename Cplx<T>::type;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C *buf0 = reinterpret_cast<C *>(smem_raw);
    C *buf1 = buf0 + RB * N;
    C *tw = buf1 + RB * N;
    fill_twiddles<T>(tw, N, -1);
    const int r0 = blockIdx.x * RB;
    const int o = blockIdx.y;              // group * O + channel
    const int g = o / O;
    // Ybar of range bins r0 .. r0 + RB - 1, unshifted Doppler order, column-major
    for (int i = threadIdx.x; i < RB * N; i += blockDim.x) {
        const int c = i / N, d = i % N;
        const int ds = d + (N >> 1) >= N ? d + (N >> 1) - N : d + (N >> 1);
        const int64_t cell = (int64_t)(r0 + c) * N + ds;
        const C y = Y[(int64_t)o * M * N + cell];
        const T w = (T)2 * (T)G[(int64_t)g * M * N + cell];
        C v;
        v.x = w * y.x;
        v.y = w * y.y;
        buf0[c * N + d] = v;
    }
    __syncthreads();
    const C *res = stockham<C, T>(buf0, buf1, tw, N, RB, -1);
    for (int i = threadIdx.x; i < RB * N; i += blockDim.x) {
        const int n = i / RB, c = i % RB;
        const T w = window_val<T>(n, N, window);
        C v = res[c * N + n];
        v.x *= w;
        v.y *= w;
        Xbar[((int64_t)o * N + n) * M + r0 + c] = v;
    }
}

template <typename T>
__global__ void range_adjoint_kernel(const typename Cplx<T>::type *__restrict__ Xbar, int M,
                                     int window, typename Cplx<T>::type *__restrict__ xbar)
{
    using C = typename Cplx<T>::type;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C *buf0 = reinterpret_cast<C *>(smem_raw);
    C *buf1 = buf0 + M;
    C *tw = buf1 + M;
    fill_twiddles<T>(tw, M, -1);
    const int64_t row = blockIdx.x;
    for (int i = threadIdx.x; i < M; i += blockDim.x) buf0[i] = Xbar[row * M + i];
    __syncthreads();
    const C *res = stockham<C, T>(buf0, buf1, tw, M, 1, -1);
    for (int i = threadIdx.x; i < M; i += blockDim.x) {
        const T w = window_val<T>(i, M, window);
        C v = res[i];
        v.x *= w;
        v.y *= w;
        xbar[row * M + i] = v;
    }
}

static int rdm_rb(int N, int M)
{
    int rb = 1;
    while (2 * rb * N <= 512 && M % (2 * rb) == 0) rb *= 2;
    return rb;
}

// workspace: the range-FFT output (O N M complex) followed by the channel
// groups' partial maps (at most O M N reals of the same precision)
int64_t rdm_workspace_bytes(const RadarDev &rd, int dtype)
{
    const int64_t e = dtype == BART_C64 ? 8 : 16;
    return (int64_t)rd.O * rd.N * rd.M * (e + e / 2);
}

template <typename T>
static void range_fft(const void *adc, const RadarDev &rd, void *X, cudaStream_t s)
{
    using C = typename Cplx<T>::type;
    const int M = rd.M;
    const size_t sm1 = (size_t)(2 * M + tw_len(M)) * sizeof(C);
    const int t1 = M / 2 < 1024 ? (M / 2 < 32 ? 32 : M / 2) : 1024;
    cudaFuncSetAttribute(range_fft_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)sm1);
    range_fft_kernel<T><<<(unsigned int)((int64_t)rd.O * rd.N), t1, sm1, s>>>(
        reinterpret_cast<const C *>(adc), reinterpret_cast<C *>(X), M, rd.window);
}

template <typename T>
static void doppler(const void *X, const RadarDev &rd, void *cube, cudaStream_t s)
{
    using C = typename Cplx<T>::type;
    const int M = rd.M, N = rd.N;
    const int RB = rdm_rb(N, M);
    const size_t sm2 = (size_t)(2 * RB * N + tw_len(N)) * sizeof(C);
    cudaFuncSetAttribute(doppler_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)sm2);
    doppler_kernel<T><<<dim3((unsigned int)(M / RB), (unsigned int)rd.O), 256, sm2, s>>>(
        reinterpret_cast<const C *>(X), N, M, RB, rd.window, reinterpret_cast<C *>(cube));
}

// chirps per range-FFT block: the largest power of two TN <= N whose two
// ping-pong buffers fit in ~128 KB of shared memory
static int rdm_tn(int N, int M, size_t csize)
{
    int tn = 1;
    while (2 * tn <= N && (size_t)2 * (2 * tn) * M * csize <= (128u << 10)) tn *= 2;
    return tn;
}

// channels summed per Doppler block: the whole scene's channels when they
// fill the GPU, else fewer, as a divisor-free split (the last group shorter)
static int rdm_cpb(int O, int blocks_per_channel_group, int scenes)
{
    int cpb = O;
    while (cpb > 1 && (int64_t)blocks_per_channel_group * scenes * ((O + cpb - 1) / cpb) < 4 * 152)
        cpb = (cpb + 1) / 2;
    return cpb;
}

// the register-resident kernels of lengths M (range) and N (Doppler)
template <int M>
static void range_reg_launch(const float2 *adc, float2 *X, int64_t rows, int window,
                             cudaStream_t s)
{
    constexpr int RPB = kRegThreads / (M / fftr::Plan<M>::R0);
    int dev = 0, sms = 0, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, range_fft_reg_kernel<M>, kRegThreads, 0);
    const int64_t need = (rows + RPB - 1) / RPB;
    const int64_t grid = std::max<int64_t>(1, std::min<int64_t>(need, (int64_t)sms * std::max(1, per_sm)));
    range_fft_reg_kernel<M><<<(unsigned int)grid, kRegThreads, 0, s>>>(adc, X, rows, window);
}

template <int N>
static void doppler_reg_launch(const float2 *X, int M, int O, int groups, int window, float *part,
                               int CPB, cudaStream_t s)
{
    constexpr int RB = kRegThreads / (N / fftr::Plan<N>::R0);
    const int G = (O + CPB - 1) / CPB;
    const size_t sm = doppler_reg_smem<N>();
    cudaFuncSetAttribute(doppler_sum_reg_kernel<N>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)sm);
    doppler_sum_reg_kernel<N><<<dim3((unsigned int)(M / RB), (unsigned int)(G * groups)),
                                kRegThreads, sm, s>>>(X, M, CPB, O, window, part);
}

static bool reg_len_ok(int L) { return L >= 16 && L <= 1024 && is_pow2_len(L); }

// columns per Doppler block of the register kernels
static int reg_rb(int N) { return kRegThreads / (N / (N == 32 || N == 64 || N == 512 ? 8 : 16)); }

static bool rdm_reg_supported(const RadarDev &rd)
{
    return reg_len_ok(rd.M) && reg_len_ok(rd.N) && rd.M % reg_rb(rd.N) == 0;
}

static void range_reg_dispatch(const float2 *adc, float2 *X, int64_t rows, int M, int window,
                               cudaStream_t s)
{
    switch (M) {
    case 16: range_reg_launch<16>(adc, X, rows, window, s); break;
    case 32: range_reg_launch<32>(adc, X, rows, window, s); break;
    case 64: range_reg_launch<64>(adc, X, rows, window, s); break;
    case 128: range_reg_launch<128>(adc, X, rows, window, s); break;
    case 256: range_reg_launch<256>(adc, X, rows, window, s); break;
    case 512: range_reg_launch<512>(adc, X, rows, window, s); break;
    default: range_reg_launch<1024>(adc, X, rows, window, s); break;
    }
}

static void doppler_reg_dispatch(const float2 *X, int N, int M, int O, int groups, int window,
                                 float *part, int CPB, int *status,
                                 cudaStream_t s)
{
    // TMA tile loads where one box covers the tile (32 <= N <= 256 chirps)
    {
        bool done = false;
        switch (N) {
        case 32: done = doppler_tma_launch<32>(X, M, O, groups, window, part, CPB, status, s); break;
        case 64: done = doppler_tma_launch<64>(X, M, O, groups, window, part, CPB, status, s); break;
        case 128: done = doppler_tma_launch<128>(X, M, O, groups, window, part, CPB, status, s); break;
        case 256: done = doppler_tma_launch<256>(X, M, O, groups, window, part, CPB, status, s); break;
        default: break;
        }
        if (done) return;
    }
    switch (N) {
    case 16: doppler_reg_launch<16>(X, M, O, groups, window, part, CPB, s); break;
    case 32: doppler_reg_launch<32>(X, M, O, groups, window, part, CPB, s); break;
    case 64: doppler_reg_launch<64>(X, M, O, groups, window, part, CPB, s); break;
    case 128: doppler_reg_launch<128>(X, M, O, groups, window, part, CPB, s); break;
    case 256: doppler_reg_launch<256>(X, M, O, groups, window, part, CPB, s); break;
    case 512: doppler_reg_launch<512>(X, M, O, groups, window, part, CPB, s); break;
    default: doppler_reg_launch<1024>(X, M, O, groups, window, part, CPB, s); break;
    }
}

// Returns the number of partial maps per scene left in `part`.  (A
// channel-chunked schedule -- range and Doppler passes over chunks of ~32
// MiB so that the range output is read back from L2 -- measured 5x slower
// on the 192 x 256 x 512 cube: twelve short launches, each a fraction of a
// wave, and the chunks' partial maps added in place.)
static int run_rdm_reg(const float2 *adc, const RadarDev &rd, int groups, float2 *X, float *part,
                       int *status, cudaStream_t s)
{
    const int M = rd.M, N = rd.N, O = rd.O;
    const int RB = reg_rb(N);
    range_reg_dispatch(adc, X, (int64_t)O * groups * N, M, rd.window, s);
    const int CPB = rdm_cpb(O, M / RB, groups);
    doppler_reg_dispatch(X, N, M, O, groups, rd.window, part, CPB, status, s);
    return (O + CPB - 1) / CPB;
}

template <typename T>
static void run_rdm(const void *adc, const RadarDev &rd, int groups, void *ws, float *rdm,
                    int *status, cudaStream_t s)
{
    using C = typename Cplx<T>::type;
    const int M = rd.M, N = rd.N, O = rd.O;
    const int64_t Oall = (int64_t)O * groups;
    const int64_t MN = (int64_t)M * N;
    if (std::is_same<T, float>::value && rdm_reg_supported(rd)) {
        float2 *X = reinterpret_cast<float2 *>(ws);
        float *part = reinterpret_cast<float *>(X + Oall * N * M);
        const int G =
            run_rdm_reg(reinterpret_cast<const float2 *>(adc), rd, groups, X, part, status, s);
        rdm_sum_kernel<float><<<(unsigned int)((MN * groups + 255) / 256), 256, 0, s>>>(
            part, G, MN, groups, rdm);
        return;
    }
    // range pass, transposed output Xt[o][r][n]
    const int TN = rdm_tn(N, M, sizeof(C));
    const size_t sm1 = (size_t)(2 * TN * M + tw_len(M)) * sizeof(C);
    cudaFuncSetAttribute(range_fft_t_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)sm1);
    const int t1 = std::min(1024, std::max(128, TN * M / 4));
    range_fft_t_kernel<T><<<dim3((unsigned int)((N + TN - 1) / TN), (unsigned int)Oall), t1, sm1,
                            s>>>(reinterpret_cast<const C *>(adc), reinterpret_cast<C *>(ws), N,
                                 M, TN, rd.window);
    // Doppler pass and the per-group channel sums
    const int RB = rdm_rb(N, M);
    const int CPB = rdm_cpb(O, M / RB, groups);
    const int G = (O + CPB - 1) / CPB;
    T *part = reinterpret_cast<T *>(reinterpret_cast<C *>(ws) + Oall * N * M);
    const size_t sm2 = (size_t)(2 * RB * N + tw_len(N)) * sizeof(C) + (size_t)RB * N * sizeof(T);
    cudaFuncSetAttribute(doppler_sum_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)sm2);
    doppler_sum_kernel<T><<<dim3((unsigned int)(M / RB), (unsigned int)(G * groups)), 256, sm2,
                            s>>>(reinterpret_cast<const C *>(ws), N, M, RB, CPB, O, rd.window,
                                 part);
    rdm_sum_kernel<T><<<(unsigned int)((MN * groups + 255) / 256), 256, 0, s>>>(part, G, MN,
                                                                               groups, rdm);
}

template <typename T>
static void run_rdm_cube(const void *adc, const RadarDev &rd, void *X, void *cube, float *rdm,
                         cudaStream_t s)
{
    using C = typename Cplx<T>::type;
    range_fft<T>(adc, rd, X, s);
    doppler<T>(X, rd, cube, s);
    const int64_t MN = (int64_t)rd.M * rd.N;
    rdm_cube_sum_kernel<T><<<(unsigned int)((MN + 255) / 256), 256, 0, s>>>(
        reinterpret_cast<const C *>(cube), rd.O, MN, rdm);
}

template <typename T>
static void run_rdm_adjoint(const void *adc, const float *grad_rdm, const RadarDev &rd,
                            int groups, void *X, void *cube, float *rdm, void *grad_adc,
                            cudaStream_t s)
{
    using C = typename Cplx<T>::type;
    RadarDev all = rd;
    all.O = rd.O * groups;
    const int M = rd.M, N = rd.N;
    // forward cube Y (and the RDM, unused) into `cube`
    range_fft<T>(adc, all, X, s);
    doppler<T>(X, all, cube, s);
    const int RB = rdm_rb(N, M);
    const size_t sm2 = (size_t)(2 * RB * N + tw_len(N)) * sizeof(C);
    cudaFuncSetAttribute(doppler_adjoint_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)sm2);
    doppler_adjoint_kernel<T><<<dim3((unsigned int)(M / RB), (unsigned int)all.O), 256, sm2, s>>>(
        reinterpret_cast<const C *>(cube), grad_rdm, rd.O, N, M, RB, rd.window,
        reinterpret_cast<C *>(X));
    const size_t sm1 = (size_t)(2 * M + tw_len(M)) * sizeof(C);
    const int t1 = M / 2 < 1024 ? (M / 2 < 32 ? 32 : M / 2) : 1024;
    cudaFuncSetAttribute(range_adjoint_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)sm1);
    range_adjoint_kernel<T><<<(unsigned int)((int64_t)all.O * N), t1, sm1, s>>>(
        reinterpret_cast<const C *>(X), M, rd.window, reinterpret_cast<C *>(grad_adc));
    (void)rdm;
}

void launch_rdm_adjoint(const void *adc, int dtype, const float *grad_rdm, const RadarDev &rd,
                        int groups, void *X, void *cube, void *grad_adc, cudaStream_t s)
{
    if (dtype == BART_C64)
        run_rdm_adjoint<float>(adc, grad_rdm, rd, groups, X, cube, nullptr, grad_adc, s);
    else
        run_rdm_adjoint<double>(adc, grad_rdm, rd, groups, X, cube, nullptr, grad_adc, s);
}

void launch_rdm_cube(const void *adc, int dtype, const RadarDev &rd, void *X, void *cube,
                     float *rdm, cudaStream_t s)
{
    if (dtype == BART_C64) run_rdm_cube<float>(adc, rd, X, cube, rdm, s);
    else run_rdm_cube<double>(adc, rd, X, cube, rdm, s);
}

void launch_rdm(const void *adc, int dtype, const RadarDev &rd, int groups, void *ws, float *rdm,
                int *status, cudaStream_t s)
{
    if (dtype == BART_C64) run_rdm<float>(adc, rd, groups, ws, rdm, status, s);
    else run_rdm<double>(adc, rd, groups, ws, rdm, status, s);
}

// -------------------------------------------------------------------------
// Fixed workspace for bart_form_rdm_static: a statically sized device array
// that exists on every GPU that loads this library, for as long as the
// process lives.  Host code may not use its name as an address; the device
// address is looked up with cudaGetSymbolAddress on every call, with the
// target device current (the lookup allocates nothing, and a fresh lookup
// stays valid after cudaDeviceReset or under another context).
// -------------------------------------------------------------------------
static __device__ __align__(256) unsigned char g_rdm_static_ws[kRdmStaticWorkspaceBytes];

int rdm_static_workspace(void **ws, const char **err)
{
    void *p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_rdm_static_ws);
    if (e != cudaSuccess || !p) {
        cudaGetLastError();
        *err = "cudaGetSymbolAddress of the static RDM workspace failed";
        return BART_ECUDA;
    }
    *ws = p;
    return BART_OK;
}

}  // namespace bart
