// Power-of-two FFTs held in registers (complex64), for the range-Doppler map
// (rdm.cu).  A length-L transform is spread over T = L / R0 threads, each
// holding R0 points; it runs as P = 1..3 radix passes (the plans below),
// each pass an R-point DFT per butterfly in registers followed by the
// pass's twiddles, with the data exchanged between passes through L
// complex of shared memory.  The pass is the Stockham autosort step (no
// digit reversal): with current stride S (the product of the earlier
// radices), n = L / S, m = n / R, butterfly b = q + S j (q < S, j < m)
//   y[q + S (R j + k')] = W_n^{j k'} sum_k x[b + (L / R) k] W_R^{k k'},
// W_n = exp(-2 pi i / n).  Every thread's butterflies, and so its
// twiddles, are the same for every transform it runs: they are computed
// once (FftTw) and kept in registers.
//
// Entry layout: a[k] = x[tid + T k], k < R0 (coalesced loads of a row).
// Exit layout: a[u R + k'] = X[tid + T u + (L / R) k'] for the last pass's
// radix R (U = R0 / R butterflies u per thread); fft_out_index() gives it.
//
// Shared-memory exchanges are swizzled per pass (an XOR of the low four
// index bits with the butterfly's j bits) so that the writes of a
// half-warp's 16 consecutive butterflies hit 16 distinct 8-byte bank
// pairs; the next pass's reads (16 consecutive indices) stay
// conflict-free under any such XOR.
#pragma once

#include <cuda_runtime.h>

namespace bart {
namespace fftr {

template <int L> struct Plan;
template <> struct Plan<16> { static constexpr int P = 1, R0 = 16, R1 = 1, R2 = 1; };
template <> struct Plan<32> { static constexpr int P = 2, R0 = 8, R1 = 4, R2 = 1; };
template <> struct Plan<64> { static constexpr int P = 2, R0 = 8, R1 = 8, R2 = 1; };
template <> struct Plan<128> { static constexpr int P = 2, R0 = 16, R1 = 8, R2 = 1; };
template <> struct Plan<256> { static constexpr int P = 2, R0 = 16, R1 = 16, R2 = 1; };
template <> struct Plan<512> { static constexpr int P = 3, R0 = 8, R1 = 8, R2 = 8; };
template <> struct Plan<1024> { static constexpr int P = 3, R0 = 16, R1 = 8, R2 = 8; };

__host__ __device__ constexpr int ilog2(int x) { return x <= 1 ? 0 : 1 + ilog2(x / 2); }

__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 cmul(float2 a, float2 w)
{
    return make_float2(fmaf(a.x, w.x, -a.y * w.y), fmaf(a.x, w.y, a.y * w.x));
}
// a (-i): a quarter turn of the forward transform
__device__ __forceinline__ float2 mnj(float2 a) { return make_float2(a.y, -a.x); }

constexpr float kS2 = 0.70710678118654752440f;    // sqrt(2) / 2
constexpr float kC8 = 0.92387953251128675613f;    // cos(pi / 8)
constexpr float kS8 = 0.38268343236508977173f;    // sin(pi / 8)

// forward DFTs of R points, natural order in and out
__device__ __forceinline__ void dft2(float2 &a0, float2 &a1)
{
    const float2 t = a0;
    a0 = cadd(t, a1);
    a1 = csub(t, a1);
}

__device__ __forceinline__ void dft4(float2 &a0, float2 &a1, float2 &a2, float2 &a3)
{
    const float2 t0 = cadd(a0, a2), t1 = csub(a0, a2);
    const float2 t2 = cadd(a1, a3), t3 = mnj(csub(a1, a3));
    a0 = cadd(t0, t2);
    a2 = csub(t0, t2);
    a1 = cadd(t1, t3);
    a3 = csub(t1, t3);
}

template <int R> __device__ __forceinline__ void dft(float2 *a);

template <> __device__ __forceinline__ void dft<1>(float2 *) {}
template <> __device__ __forceinline__ void dft<2>(float2 *a) { dft2(a[0], a[1]); }
template <> __device__ __forceinline__ void dft<4>(float2 *a) { dft4(a[0], a[1], a[2], a[3]); }

template <> __device__ __forceinline__ void dft<8>(float2 *a)
{
    // even and odd halves, then X_k = E_k + W8^k O_k, X_{k+4} = E_k - W8^k O_k
    dft4(a[0], a[2], a[4], a[6]);
    dft4(a[1], a[3], a[5], a[7]);
    const float2 o1 = make_float2(kS2 * (a[3].x + a[3].y), kS2 * (a[3].y - a[3].x));
    const float2 o2 = mnj(a[5]);
    const float2 o3 = make_float2(kS2 * (a[7].y - a[7].x), -kS2 * (a[7].x + a[7].y));
    const float2 e0 = a[0], e1 = a[2], e2 = a[4], e3 = a[6], o0 = a[1];
    a[0] = cadd(e0, o0);
    a[4] = csub(e0, o0);
    a[1] = cadd(e1, o1);
    a[5] = csub(e1, o1);
    a[2] = cadd(e2, o2);
    a[6] = csub(e2, o2);
    a[3] = cadd(e3, o3);
    a[7] = csub(e3, o3);
}

template <> __device__ __forceinline__ void dft<16>(float2 *a)
{
    // n = n1 + 4 n2, k = k2 + 4 k1: DFT4 over n2, twiddle W16^{n1 k2}, DFT4 over n1
#pragma unroll
    for (int n1 = 0; n1 < 4; ++n1) dft4(a[n1], a[n1 + 4], a[n1 + 8], a[n1 + 12]);
    // b[n1][k2] sits in a[n1 + 4 k2]
    const float2 w1 = make_float2(kC8, -kS8), w2 = make_float2(kS2, -kS2),
                 w3 = make_float2(kS8, -kC8), w6 = make_float2(-kS2, -kS2),
                 w9 = make_float2(-kC8, kS8);
    a[5] = cmul(a[5], w1);      // n1 = 1, k2 = 1
    a[9] = cmul(a[9], w2);      // n1 = 1, k2 = 2
    a[13] = cmul(a[13], w3);    // n1 = 1, k2 = 3
    a[6] = cmul(a[6], w2);      // n1 = 2, k2 = 1
    a[10] = mnj(a[10]);         // n1 = 2, k2 = 2
    a[14] = cmul(a[14], w6);    // n1 = 2, k2 = 3
    a[7] = cmul(a[7], w3);      // n1 = 3, k2 = 1
    a[11] = cmul(a[11], w6);    // n1 = 3, k2 = 2
    a[15] = cmul(a[15], w9);    // n1 = 3, k2 = 3
    float2 c[16];
#pragma unroll
    for (int k2 = 0; k2 < 4; ++k2) {
        float2 b0 = a[4 * k2], b1 = a[4 * k2 + 1], b2 = a[4 * k2 + 2], b3 = a[4 * k2 + 3];
        dft4(b0, b1, b2, b3);
        c[k2] = b0;
        c[k2 + 4] = b1;
        c[k2 + 8] = b2;
        c[k2 + 12] = b3;
    }
#pragma unroll
    for (int i = 0; i < 16; ++i) a[i] = c[i];
}

// the radix, stride and butterflies per thread of pass p
template <int L, int p> struct PassOf {
    using PL = Plan<L>;
    static constexpr int R = p == 0 ? PL::R0 : (p == 1 ? PL::R1 : PL::R2);
    static constexpr int S = p == 0 ? 1 : (p == 1 ? PL::R0 : PL::R0 * PL::R1);
    static constexpr int U = PL::R0 / R;
    static constexpr int T = L / PL::R0;
    static constexpr int NTW = U * (R - 1);     // twiddles per thread
};

// swizzled shared-memory index of the exchange written by a pass (S, R)
template <int S, int R>
__device__ __forceinline__ int swz(int i)
{
    constexpr int sh = ilog2(S) + ilog2(R);
    return i ^ (((i >> sh) << ilog2(S)) & 15);
}

// per-thread twiddles of the passes that apply them (all but the last)
template <int L> struct FftTw {
    static constexpr int P = Plan<L>::P;
    static constexpr int N0 = P > 1 ? PassOf<L, 0>::NTW : 1;
    static constexpr int N1 = P > 2 ? PassOf<L, 1>::NTW : 1;
    float2 w0[N0], w1[N1];

    template <int p>
    __device__ __forceinline__ void fill(float2 *w, int tid)
    {
        using Q = PassOf<L, p>;
#pragma unroll
        for (int u = 0; u < Q::U; ++u) {
            const int b = tid + Q::T * u;
            const int j = b >> ilog2(Q::S);
#pragma unroll
            for (int k = 1; k < Q::R; ++k) {
                // W_L^{S j k}, S j k < L
                float s, c;
                sincospif(-2.f * (float)(Q::S * j * k) / (float)L, &s, &c);
                w[u * (Q::R - 1) + k - 1] = make_float2(c, s);
            }
        }
    }
    __device__ __forceinline__ void init(int tid)
    {
        if constexpr (P > 1) fill<0>(w0, tid);
        if constexpr (P > 2) fill<1>(w1, tid);
    }
};

// DFT, twiddles (unless last) and, unless last, the swizzled store of pass p
template <int L, int p>
__device__ __forceinline__ void pass_compute_store(float2 (&a)[Plan<L>::R0], int tid,
                                                   float2 *buf, const float2 *w)
{
    using Q = PassOf<L, p>;
    constexpr bool last = p == Plan<L>::P - 1;
#pragma unroll
    for (int u = 0; u < Q::U; ++u) {
        dft<Q::R>(a + u * Q::R);
        if constexpr (!last) {
#pragma unroll
            for (int k = 1; k < Q::R; ++k)
                a[u * Q::R + k] = cmul(a[u * Q::R + k], w[u * (Q::R - 1) + k - 1]);
            const int b = tid + Q::T * u;
            const int j = b >> ilog2(Q::S), q = b & (Q::S - 1);
#pragma unroll
            for (int k = 0; k < Q::R; ++k)
                buf[swz<Q::S, Q::R>(q + Q::S * (Q::R * j + k))] = a[u * Q::R + k];
        }
    }
}

// the loads of pass p (> 0) from the exchange written by pass p - 1
template <int L, int p>
__device__ __forceinline__ void pass_load(float2 (&a)[Plan<L>::R0], int tid, const float2 *buf)
{
    using Q = PassOf<L, p>;
    using Pv = PassOf<L, p - 1>;
#pragma unroll
    for (int u = 0; u < Q::U; ++u) {
        const int b = tid + Q::T * u;
#pragma unroll
        for (int k = 0; k < Q::R; ++k)
            a[u * Q::R + k] = buf[swz<Pv::S, Pv::R>(b + (L / Q::R) * k)];
    }
}

// The whole transform.  Every thread of the block must call it together
// (it synchronises the block); buf: L complex of this transform.
template <int L>
__device__ __forceinline__ void fft(float2 (&a)[Plan<L>::R0], int tid, float2 *buf,
                                    const FftTw<L> &tw)
{
    constexpr int P = Plan<L>::P;
    pass_compute_store<L, 0>(a, tid, buf, tw.w0);
    if constexpr (P > 1) {
        __syncthreads();
        pass_load<L, 1>(a, tid, buf);
        __syncthreads();
        pass_compute_store<L, 1>(a, tid, buf, tw.w1);
    }
    if constexpr (P > 2) {
        __syncthreads();
        pass_load<L, 2>(a, tid, buf);
        __syncthreads();
        pass_compute_store<L, 2>(a, tid, buf, nullptr);
    }
}

// the output bin held in a[i] after fft<L>
template <int L>
__device__ __forceinline__ int fft_out_index(int tid, int i)
{
    using Q = PassOf<L, Plan<L>::P - 1>;
    const int u = i / Q::R, k = i % Q::R;
    return tid + Q::T * u + (L / Q::R) * k;
}

}  // namespace fftr
}  // namespace bart
