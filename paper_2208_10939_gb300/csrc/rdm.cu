// Range-Doppler map (Sec. 3.3): per channel, a windowed forward FFT over the
// M fast-time samples of every chirp (range), then a windowed forward FFT
// over the N chirps of every range bin (Doppler); |.|^2 summed over the O
// channels; the Doppler axis shifted so that zero velocity is bin N/2.
//
// Radix-2 Stockham autosort FFTs in shared memory (no bit reversal): stage
// with current length n and stride s = L/n maps
//   y[q + s(2p)] = x[q + s p] + x[q + s(p + n/2)]
//   y[q + s(2p+1)] = (x[q + s p] - x[q + s(p + n/2)]) * exp(-2 pi i p s / L)
// Both passes are HBM-bound: each reads and writes the cube once.
#include <cuda_runtime.h>
#include <stdint.h>

#include <mutex>

#include "bart_internal.cuh"

namespace bart {

template <typename T> struct Cplx;
template <> struct Cplx<float> { using type = float2; };
template <> struct Cplx<double> { using type = double2; };

__device__ __forceinline__ void sincospi_t(float x, float *s, float *c) { sincospif(x, s, c); }
__device__ __forceinline__ void sincospi_t(double x, double *s, double *c) { sincospi(x, s, c); }
__device__ __forceinline__ float cospi_t(float x) { return cospif(x); }
__device__ __forceinline__ double cospi_t(double x) { return cospi(x); }

// symmetric Hann: 0.5 - 0.5 cos(2 pi i / (L-1)), evaluated in the FFT's own
// precision (cospif / cospi)
template <typename T>
__device__ __forceinline__ T window_val(int i, int L, int kind)
{
    if (kind == BART_WINDOW_RECT || L < 2) return (T)1;
    return (T)0.5 - (T)0.5 * cospi_t((T)(2 * i) / (T)(L - 1));
}

// Stockham stages over `cols` interleaved transforms of length L stored as
// buf[col * L + idx]; `tw` holds exp(-2 pi i j / L), j < L/2.
template <typename C>
__device__ C *stockham(C *x, C *y, const C *tw, int L, int cols)
{
    const int half_tot = (L >> 1) * cols;
    for (int n = L, s = 1; n > 1; n >>= 1, s <<= 1) {
        const int h = n >> 1;
        for (int t = threadIdx.x; t < half_tot; t += blockDim.x) {
            const int col = t / (L >> 1), b = t % (L >> 1);
            const int p = b / s, q = b % s;
            const C *xc = x + col * L;
            C *yc = y + col * L;
            const C a = xc[q + s * p], c = xc[q + s * (p + h)];
            const C w = tw[p * s];
            C sum, dif;
            sum.x = a.x + c.x;
            sum.y = a.y + c.y;
            dif.x = a.x - c.x;
            dif.y = a.y - c.y;
            yc[q + s * (2 * p)] = sum;
            C r;
            r.x = dif.x * w.x - dif.y * w.y;
            r.y = dif.x * w.y + dif.y * w.x;
            yc[q + s * (2 * p + 1)] = r;
        }
        __syncthreads();
        C *tmp = x;
        x = y;
        y = tmp;
    }
    return x;
}

template <typename T>
__device__ void fill_twiddles(typename Cplx<T>::type *tw, int L)
{
    for (int j = threadIdx.x; j < (L >> 1); j += blockDim.x) {
        T s, c;
        sincospi_t((T)(-2 * j) / (T)L, &s, &c);
        tw[j].x = c;
        tw[j].y = s;
    }
}

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
    const C *res = stockham<C>(buf0, buf1, tw, M, 1);
    C *out = X + row * M;
    for (int i = threadIdx.x; i < M; i += blockDim.x) out[i] = res[i];
}

// one block per (RB consecutive range bins, channel): Doppler FFT of the
// channel's RB columns.  CUBE = false: |Y|^2 written per channel, [o][r][d']
// (summed by rdm_sum_kernel); CUBE = true: the complex Y written, [o][r][d']
// (summed by rdm_cube_sum_kernel and kept for the angle spectrum).  d' is the
// Doppler bin after the N/2 shift.
template <typename T, bool CUBE>
__global__ void doppler_kernel(const typename Cplx<T>::type *__restrict__ X, int N, int M,
                               int RB, int window, T *__restrict__ pw_out,
                               typename Cplx<T>::type *__restrict__ cube_out)
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
    const C *res = stockham<C>(buf0, buf1, tw, N, RB);
    for (int i = threadIdx.x; i < RB * N; i += blockDim.x) {
        const int c = i / N, d = i % N;
        const C v = res[i];
        const int64_t at = ((int64_t)o * M + r0 + c) * N + ((d + (N >> 1)) & (N - 1));
        if (CUBE) cube_out[at] = v;
        else pw_out[at] = v.x * v.x + v.y * v.y;
    }
}

// RDM[r][d] = sum over channels, in channel order
template <typename T>
__global__ void rdm_sum_kernel(const T *__restrict__ pw, int O, int64_t MN, float *__restrict__ rdm)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= MN) return;
    T acc = (T)0;
    for (int o = 0; o < O; ++o) acc += pw[(int64_t)o * MN + i];
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

static int rdm_rb(int N) { return N >= 512 ? 1 : 512 / N; }

// workspace: the range-FFT output (O N M complex) followed by the
// per-channel Doppler power (O M N reals of the same precision)
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
    const size_t sm1 = (size_t)(2 * M + M / 2) * sizeof(C);
    const int t1 = M / 2 < 1024 ? (M / 2 < 32 ? 32 : M / 2) : 1024;
    cudaFuncSetAttribute(range_fft_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)sm1);
    range_fft_kernel<T><<<(unsigned int)((int64_t)rd.O * rd.N), t1, sm1, s>>>(
        reinterpret_cast<const C *>(adc), reinterpret_cast<C *>(X), M, rd.window);
}

template <typename T, bool CUBE>
static void doppler(const void *X, const RadarDev &rd, T *pw, void *cube, cudaStream_t s)
{
    using C = typename Cplx<T>::type;
    const int M = rd.M, N = rd.N;
    int RB = rdm_rb(N);
    if (RB > M) RB = M;
    const size_t sm2 = (size_t)(2 * RB * N + N / 2) * sizeof(C);
    cudaFuncSetAttribute(doppler_kernel<T, CUBE>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)sm2);
    doppler_kernel<T, CUBE><<<dim3((unsigned int)(M / RB), (unsigned int)rd.O), 256, sm2, s>>>(
        reinterpret_cast<const C *>(X), N, M, RB, rd.window, pw, reinterpret_cast<C *>(cube));
}

template <typename T>
static void run_rdm(const void *adc, const RadarDev &rd, void *ws, float *rdm, cudaStream_t s)
{
    using C = typename Cplx<T>::type;
    range_fft<T>(adc, rd, ws, s);
    T *pw = reinterpret_cast<T *>(reinterpret_cast<C *>(ws) + (int64_t)rd.O * rd.N * rd.M);
    doppler<T, false>(ws, rd, pw, nullptr, s);
    const int64_t MN = (int64_t)rd.M * rd.N;
    rdm_sum_kernel<T><<<(unsigned int)((MN + 255) / 256), 256, 0, s>>>(pw, rd.O, MN, rdm);
}

template <typename T>
static void run_rdm_cube(const void *adc, const RadarDev &rd, void *X, void *cube, float *rdm,
                         cudaStream_t s)
{
    using C = typename Cplx<T>::type;
    range_fft<T>(adc, rd, X, s);
    doppler<T, true>(X, rd, nullptr, cube, s);
    const int64_t MN = (int64_t)rd.M * rd.N;
    rdm_cube_sum_kernel<T><<<(unsigned int)((MN + 255) / 256), 256, 0, s>>>(
        reinterpret_cast<const C *>(cube), rd.O, MN, rdm);
}

void launch_rdm_cube(const void *adc, int dtype, const RadarDev &rd, void *X, void *cube,
                     float *rdm, cudaStream_t s)
{
    if (dtype == BART_C64) run_rdm_cube<float>(adc, rd, X, cube, rdm, s);
    else run_rdm_cube<double>(adc, rd, X, cube, rdm, s);
}

void launch_rdm(const void *adc, int dtype, const RadarDev &rd, void *ws, float *rdm,
                cudaStream_t s)
{
    if (dtype == BART_C64) run_rdm<float>(adc, rd, ws, rdm, s);
    else run_rdm<double>(adc, rd, ws, rdm, s);
}

// -------------------------------------------------------------------------
// Fixed workspace for bart_form_rdm_static: a statically sized device array
// that exists on every GPU that loads this library, for as long as the
// process lives.  Host code may not use its name as an address; the device
// address is looked up once per device with cudaGetSymbolAddress.
// -------------------------------------------------------------------------
static __device__ __align__(256) unsigned char g_rdm_static_ws[kRdmStaticWorkspaceBytes];

constexpr int kMaxDevices = 64;

int rdm_static_workspace(void **ws, const char **err)
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
        cudaGetLastError();
        *err = "no usable current CUDA device";
        return BART_ECUDA;
    }
    static std::mutex mu;
    static void *addr[kMaxDevices] = {nullptr};
    std::lock_guard<std::mutex> lock(mu);
    if (!addr[dev]) {
        void *p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_rdm_static_ws);
        if (e != cudaSuccess || !p) {
            cudaGetLastError();
            *err = "cudaGetSymbolAddress of the static RDM workspace failed";
            return BART_ECUDA;
        }
        addr[dev] = p;
    }
    *ws = addr[dev];
    return BART_OK;
}

}  // namespace bart
