// Mixed-radix (2, 3) Stockham autosort FFTs in shared memory (no digit
// reversal), lengths L = 2^a 3^b, used by the range-Doppler map (rdm.cu) and
// the spectral echo synthesis (spectral.cu).  A stage with current length n,
// radix p (2 while n is even, else 3), m = n/p and stride s = L/n maps, for
// j < m, q < s and k' < p,
//   y[q + s(p j + k')] = exp(-2 pi i j k' / n) sum_k x[q + s(j + k m)] exp(-2 pi i k k' / p)
#pragma once

#include <cuda_runtime.h>

#include "bartsim.h"

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
    if (is_pow2_len(L)) {
        // radix 2 throughout: L/2 butterflies per column at every stage, all
        // index arithmetic by shifts and masks
        const int lh = __ffs(L) - 2;                      // log2(L / 2)
        for (int n = L, ls = 0; n > 1; n >>= 1, ++ls) {
            const int s = 1 << ls, m = n >> 1;
            for (int t = threadIdx.x; t < (cols << lh); t += blockDim.x) {
                const int col = t >> lh, b = t & ((1 << lh) - 1);
                const int j = b >> ls, q = b & (s - 1);
                const C *xc = x + col * L;
                C *yc = y + col * L;
                const C a = xc[q + s * j], c = xc[q + s * (j + m)];
                const C w = tw[j * s];
                C sum, r;
                sum.x = a.x + c.x;
                sum.y = a.y + c.y;
                const T dx = a.x - c.x, dy = a.y - c.y;
                r.x = dx * w.x - dy * w.y;
                r.y = dx * w.y + dy * w.x;
                yc[q + s * (2 * j)] = sum;
                yc[q + s * (2 * j + 1)] = r;
            }
            __syncthreads();
            C *tmp = x;
            x = y;
            y = tmp;
        }
        return x;
    }
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

}  // namespace bart
