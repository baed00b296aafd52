// Range-Doppler map (Sec. 3.3): per channel, a windowed forward FFT over the
// M fast-time samples of every chirp (range), then a windowed forward FFT
// over the N chirps of every range bin (Doppler); |.|^2 summed over the O
// channels; the Doppler axis shifted so that zero velocity is bin N/2.
//
// Mixed-radix (2, 3) Stockham autosort FFTs in shared memory (no digit
// reversal), lengths L = 2^a 3^b.  A stage with current length n, radix p
// (2 while n is even, else 3), m = n/p and stride s = L/n maps, for
// j < m, q < s and k' < p,
//   y[q + s(p j + k')] = exp(-2 pi i j k' / n) sum_k x[q + s(j + k m)] exp(-2 pi i k k' / p)
// Both passes are HBM-bound: each reads and writes the cube once.
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>

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

__host__ __device__ __forceinline__ bool is_pow2_len(int L) { return (L & (L - 1)) == 0; }

// twiddle table length: exp(-2 pi i t / L) for t < L/2 (radix 2 only) or
// t < L (a radix-3 stage reaches t = 2 j s < 2L/3)
__host__ __device__ __forceinline__ int tw_len(int L) { return is_pow2_len(L) ? L / 2 : L; }

// Stockham stages over `cols` interleaved transforms of length L stored as
// buf[col * L + idx]; `tw` holds exp(-2 pi i t / L), t < tw_len(L).
template <typename C, typename T>
__device__ C *stockham(C *x, C *y, const C *tw, int L, int cols, int sgn = 1)
{
    // sgn = +1: forward transform (exp(-i ...)); -1: unnormalised inverse
    // (exp(+i ...), with `tw` holding the conjugate twiddles)
    const T h3 = (T)sgn * (T)0.86602540378443864676;    // sin(2 pi / 3)
    for (int n = L, s = 1; n > 1;) {
        const int p = (n & 1) ? 3 : 2;
        const int m = n / p;
        const int per_col = m * s;
        for (int t = threadIdx.x; t < per_col * cols; t += blockDim.x) {
            const int col = t / per_col, b = t % per_col;
            const int j = b / s, q = b % s;
            const C *xc = x + col * L;
            C *yc = y + col * L;
            if (p == 2) {
                const C a = xc[q + s * j], c = xc[q + s * (j + m)];
                const C w = tw[j * s];
                C sum, dif, r;
                sum.x = a.x + c.x;
                sum.y = a.y + c.y;
                dif.x = a.x - c.x;
                dif.y = a.y - c.y;
                r.x = dif.x * w.x - dif.y * w.y;
                r.y = dif.x * w.y + dif.y * w.x;
                yc[q + s * (2 * j)] = sum;
                yc[q + s * (2 * j + 1)] = r;
            } else {
                const C a0 = xc[q + s * j], a1 = xc[q + s * (j + m)], a2 = xc[q + s * (j + 2 * m)];
                const T t1x = a1.x + a2.x, t1y = a1.y + a2.y;
                const T t2x = a0.x - (T)0.5 * t1x, t2y = a0.y - (T)0.5 * t1y;
                // -i sin(2 pi/3) (a1 - a2)
                const T t3x = h3 * (a1.y - a2.y), t3y = -h3 * (a1.x - a2.x);
                C y0, u1, u2, r1, r2;
                y0.x = a0.x + t1x;
                y0.y = a0.y + t1y;
                u1.x = t2x + t3x;
                u1.y = t2y + t3y;
                u2.x = t2x - t3x;
                u2.y = t2y - t3y;
                const C w1 = tw[j * s], w2 = tw[2 * j * s];
                r1.x = u1.x * w1.x - u1.y * w1.y;
                r1.y = u1.x * w1.y + u1.y * w1.x;
                r2.x = u2.x * w2.x - u2.y * w2.y;
                r2.y = u2.x * w2.y + u2.y * w2.x;
                yc[q + s * (3 * j)] = y0;
                yc[q + s * (3 * j + 1)] = r1;
                yc[q + s * (3 * j + 2)] = r2;
            }
        }
        __syncthreads();
        C *tmp = x;
        x = y;
        y = tmp;
        n = m;
        s *= p;
    }
    return x;
}

template <typename T>
__device__ void fill_twiddles(typename Cplx<T>::type *tw, int L, int sgn = 1)
{
    for (int j = threadIdx.x; j < tw_len(L); j += blockDim.x) {
        T s, c;
        sincospi_t((T)(-2 * j) / (T)L, &s, &c);
        tw[j].x = c;
        tw[j].y = (T)sgn * s;
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

template <typename T>
static void run_rdm(const void *adc, const RadarDev &rd, int groups, void *ws, float *rdm,
                    cudaStream_t s)
{
    using C = typename Cplx<T>::type;
    const int M = rd.M, N = rd.N, O = rd.O;
    const int64_t Oall = (int64_t)O * groups;
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
    const int64_t MN = (int64_t)M * N;
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
                cudaStream_t s)
{
    if (dtype == BART_C64) run_rdm<float>(adc, rd, groups, ws, rdm, s);
    else run_rdm<double>(adc, rd, groups, ws, rdm, s);
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
