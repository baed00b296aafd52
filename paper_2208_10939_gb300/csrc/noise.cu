// Additive white complex Gaussian noise at a given signal-to-noise ratio
// (Sec. 3.2: Gaussian white noise "with a certain signal-to-noise ratio").
//
//   x[e] += sigma * n[e],   sigma^2 = P / 10^(SNR/10),   P = mean |x|^2 of the cube
//   n[e] = (g1 + j g2) / sqrt(2),  (g1, g2) = Box-Muller(u1, u2)
//   u_i = (w_i + 1) 2^-32,  (w0, w1, w2, w3) = Philox4x32-10(ctr, key)
//   ctr = (e mod 2^32, e div 2^32, frame, 0),  key = (seed mod 2^32, seed div 2^32)
//
// Philox4x32-10 is the counter-based generator of Salmon, Moraes, Dror and
// Shaw (SC 2011), written here from its published round function.
#include <cuda_runtime.h>
#include <stdint.h>

#include "bart_internal.cuh"

namespace bart {

__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint2 k)
{
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const unsigned int hi0 = __umulhi(0xD2511F53u, c.x), lo0 = 0xD2511F53u * c.x;
        const unsigned int hi1 = __umulhi(0xCD9E8D57u, c.z), lo1 = 0xCD9E8D57u * c.z;
        c = make_uint4(hi1 ^ c.y ^ k.x, lo1, hi0 ^ c.w ^ k.y, lo0);
        k.x += 0x9E3779B9u;
        k.y += 0xBB67AE85u;
    }
    return c;
}

constexpr int kPowBlocks = 1024;
constexpr int kPowThreads = 256;

template <typename C>
__global__ void noise_power_kernel(const C *__restrict__ x, int64_t n, double *__restrict__ part)
{
    __shared__ double s[kPowThreads];
    double acc = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * kPowThreads + threadIdx.x; i < n;
         i += (int64_t)kPowBlocks * kPowThreads) {
        const C v = x[i];
        acc += (double)v.x * (double)v.x + (double)v.y * (double)v.y;
    }
    s[threadIdx.x] = acc;
    __syncthreads();
    for (int w = kPowThreads / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) s[threadIdx.x] += s[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) part[blockIdx.x] = s[0];
}

// sigma from the block partials, summed in block order (deterministic)
__global__ void noise_sigma_kernel(const double *__restrict__ part, int64_t n, double inv_snr,
                                   double *__restrict__ sigma)
{
    if (threadIdx.x != 0) return;
    double p = 0.0;
    for (int b = 0; b < kPowBlocks; ++b) p += part[b];
    sigma[0] = n > 0 ? sqrt(p / (double)n * inv_snr) : 0.0;
}

__global__ void noise_add_c64(float2 *__restrict__ x, int64_t n, uint2 key, unsigned int frame,
                              const double *__restrict__ sigma)
{
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n) return;
    const uint4 w = philox4x32_10(
        make_uint4((unsigned int)e, (unsigned int)((uint64_t)e >> 32), frame, 0u), key);
    const float u1 = ((float)w.x + 1.f) * 2.3283064e-10f;     // (w + 1) 2^-32
    const float u2 = ((float)w.y + 1.f) * 2.3283064e-10f;
    const float r = sqrtf(-2.f * logf(u1));
    float sn, cs;
    sincospif(2.f * u2, &sn, &cs);
    const float sg = (float)sigma[0] * 0.70710678f;
    float2 v = x[e];
    v.x = fmaf(sg * r, cs, v.x);
    v.y = fmaf(sg * r, sn, v.y);
    x[e] = v;
}

__global__ void noise_add_c128(double2 *__restrict__ x, int64_t n, uint2 key, unsigned int frame,
                               const double *__restrict__ sigma)
{
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n) return;
    const uint4 w = philox4x32_10(
        make_uint4((unsigned int)e, (unsigned int)((uint64_t)e >> 32), frame, 0u), key);
    const double u1 = ((double)w.x + 1.0) * 2.3283064365386963e-10;
    const double u2 = ((double)w.y + 1.0) * 2.3283064365386963e-10;
    const double r = sqrt(-2.0 * log(u1));
    double sn, cs;
    sincospi(2.0 * u2, &sn, &cs);
    const double sg = sigma[0] * 0.70710678118654752;
    double2 v = x[e];
    v.x += sg * r * cs;
    v.y += sg * r * sn;
    x[e] = v;
}

int64_t noise_scratch_words() { return kPowBlocks + 2; }

void launch_add_noise(void *adc, int dtype, int64_t n, double snr_db, uint64_t seed,
                      unsigned int frame, double *scratch, cudaStream_t s)
{
    const uint2 key = make_uint2((unsigned int)seed, (unsigned int)(seed >> 32));
    const double inv = pow(10.0, -snr_db / 10.0);
    double *sigma = scratch + kPowBlocks;
    const unsigned int g = (unsigned int)((n + 255) / 256);
    if (dtype == BART_C64) {
        noise_power_kernel<float2><<<kPowBlocks, kPowThreads, 0, s>>>(
            reinterpret_cast<const float2 *>(adc), n, scratch);
        noise_sigma_kernel<<<1, 32, 0, s>>>(scratch, n, inv, sigma);
        noise_add_c64<<<g, 256, 0, s>>>(reinterpret_cast<float2 *>(adc), n, key, frame, sigma);
    } else {
        noise_power_kernel<double2><<<kPowBlocks, kPowThreads, 0, s>>>(
            reinterpret_cast<const double2 *>(adc), n, scratch);
        noise_sigma_kernel<<<1, 32, 0, s>>>(scratch, n, inv, sigma);
        noise_add_c128<<<g, 256, 0, s>>>(reinterpret_cast<double2 *>(adc), n, key, frame, sigma);
    }
}

}  // namespace bart
