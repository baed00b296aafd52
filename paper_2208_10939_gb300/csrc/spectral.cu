// Spectral echo synthesis (BART_PATH_SPECTRAL): the coherent sum of Eq. 13
// over the lit facets of a chirp row, evaluated through the inverse-FFT
// route of Sec. 3.2 (Eqs. 9-11) instead of sample by sample.
//
// A vertex-form record (see mixed_record.cuh) contributes three terms
//   w_v exp{j 2 pi (ph0_v + alpha_v m + p2 m^2)},   alpha_v = hi + lo_v,
// each a spectral line at the beat frequency alpha_v (cycles per sample).
// With m = m' + M/2 (m' in [-M/2, M/2)) a term is
//   c_v exp{j 2 pi x_v m' / G} exp{j 2 pi p2 m'^2},
//   c_v = w_v exp{j 2 pi (ph0_v + alpha_v M/2 + p2 M^2/4)},
//   x_v = G (alpha_v + p2 M) mod G,
// and the row is a type-1 non-uniform discrete Fourier transform: every
// line is spread onto a uniform grid of G = 2M beat-frequency cells with a
// compact kernel psi, one inverse FFT per grid gives the row at the M
// samples, and dividing by psi's Fourier transform undoes the spreading
// (Dutt & Rokhlin 1993; the "exponential of semicircle" kernel
// psi(z) = exp(beta (sqrt(1 - (2z/W)^2) - 1)) of Barnett, Magland & af
// Klinteberg 2019).  The within-chirp quadratic phase, |2 pi p2 m'^2| < 0.02
// rad at 15 m/s, enters as exp(j 2 pi p2 m'^2) = 1 + j 2 pi p2 m'^2 -
// 2 pi^2 p2^2 m'^4 + O(1e-6): two more grids with strengths j 2 pi p2 c_v
// and -2 pi^2 p2^2 c_v, multiplied by m'^2 and m'^4 after their FFTs (both
// spread with one narrower kernel; static facets have p2 = 0 and skip them).
// Series- and edge-form records (a few in 1e4 of a frame) are added sample
// by sample: a lane that meets one queues its list position, and after the
// spreading each warp evaluates queued records with its lanes over the
// samples.  Work per record ~ W grid cells instead of M samples.
//
// One CTA per chirp row.  The row's record list is cut into 64 blocks that
// the warps take from a shared counter; a warp's lanes take consecutive runs
// of a block (neighbouring facets sit at neighbouring beat frequencies, so
// lane runs apart rarely add to the same grid cell at once, while a warp
// stays mostly within one mesh and its record forms).  Measured on the
// intersection frame: lanes on consecutive list entries 2.4x slower (a
// warp's shared-memory adds collide); 32 list-wide lane segments with the
// warps interleaved 1.23x slower (warps mixing the ground's and the
// vehicles' record forms diverge); blocks dealt to the warps in turn 1.08x
// slower (the warps finish at different times).
#include <cuda_runtime.h>
#include <stdint.h>

#include <cmath>
#include <vector>

#include "bart_internal.cuh"
#include "fft_stockham.cuh"
#include "mixed_record.cuh"

namespace bart {

namespace {

constexpr int kSpecThreads = 256;
constexpr int kQueue = 2048;      // series / edge records of a row deferred to the CTA
constexpr int kSpecBlocksPerWarp = 8;   // list blocks per warp (interleaved over the warps)
constexpr int kW0 = 8;            // taps of the main grid's kernel
constexpr int kW1 = 4;            // taps of the two quadratic-phase grids
constexpr int kD0 = 9;            // degree of the main kernel's tap polynomials
constexpr int kD1 = 5;            // degree of the narrow kernel's
constexpr double kBetaPerTap = 2.30;   // beta = 2.30 W at oversampling 2

// The kernel at the W taps around a position x = xi + u (xi integer,
// u in [0, 1)): tap j (cell xi - W/2 + 1 + j, offset z = j - W/2 + 1 - u)
// as a degree-D polynomial in t = 2u - 1, fitted once on the host
// (Chebyshev interpolation, converted to monomials; FP32 Horner evaluation
// within 1e-7 of the kernel's peak for W = 8, D = 9).
struct SpecConsts {
    int M, G;
    float halfM, quarterM2;       // M / 2, M^2 / 4
    float fM, fG;                 // M, G as floats
    float c0[kW0][kD0 + 1];
    float c1[kW1][kD1 + 1];
};

template <int W, int D>
__device__ __forceinline__ void kernel_taps(const float (&c)[W][D + 1], float t, float (&k)[W])
{
#pragma unroll
    for (int j = 0; j < W; ++j) {
        float a = c[j][D];
#pragma unroll
        for (int d = D - 1; d >= 0; --d) a = fmaf(a, t, c[j][d]);
        k[j] = a;
    }
}

// cell of tap j for a line whose taps start at cell g0 (within a few cells of [0, G))
__device__ __forceinline__ int wrap_cell(int g, int G)
{
    return g < 0 ? g + G : (g >= G ? g - G : g);
}

// shared-memory reduction without a returned value
__device__ __forceinline__ void red_add(float *a, float v)
{
    asm volatile("red.shared.add.f32 [%0], %1;" ::"r"((unsigned)__cvta_generic_to_shared(a)),
                 "f"(v)
                 : "memory");
}

__global__ void __launch_bounds__(kSpecThreads, 2)
synth_spectral_kernel(SynthArgs A, MixConsts K, SpecConsts C, const float *__restrict__ inv_psi)
{
    using C2 = float2;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int G = C.G, M = C.M;
    // grids as separate real / imaginary arrays (for float atomics), then
    // the complex FFT buffers: buf1 reuses the grids' space after the copy
    float *gr0 = reinterpret_cast<float *>(smem_raw);
    float *gi0 = gr0 + G, *gr1 = gi0 + G, *gi1 = gr1 + G, *gr2 = gi1 + G, *gi2 = gr2 + G;
    C2 *buf1 = reinterpret_cast<C2 *>(smem_raw);                 // 3 G complex
    C2 *buf0 = reinterpret_cast<C2 *>(smem_raw + 6 * G * sizeof(float));   // 3 G complex
    C2 *tw = buf0 + 3 * G;
    float *dre = reinterpret_cast<float *>(tw + tw_len(G));
    float *dim = dre + M;
    int *queue = reinterpret_cast<int *>(dim + M);
    __shared__ int s_qn, s_next;

    const int row = blockIdx.x;
    const int nc = A.nc;
    const int vrow = row / nc, nl = row % nc;
    const int n = A.n0 + nl;
    const int O = A.rd.O, P = A.rd.P, Q = A.rd.Q;
    const int o = vrow % O;
    const int tx = o / Q, rx = o % Q;
    const int64_t F = A.F;
    for (int i = threadIdx.x; i < 6 * G; i += blockDim.x) gr0[i] = 0.f;
    for (int i = threadIdx.x; i < 2 * M; i += blockDim.x) dre[i] = 0.f;
    if (threadIdx.x == 0) s_qn = s_next = 0;
    fill_twiddles<float>(tw, G, -1);
    __syncthreads();

    const int slot = A.rd.tdm ? tx : 0;
    MixRow w;
    w.kin_t = A.kin + (int64_t)tx * F * kKinRow;
    w.kin_r = A.kin + (int64_t)(P + rx) * F * kKinRow;
    w.quad_t = A.kquad + (int64_t)tx * F * kKinQuadWords;
    w.quad_r = A.kquad + (int64_t)(P + rx) * F * kKinQuadWords;
    w.sl = n * A.rd.slots + slot;
    w.ant_t = tx;
    w.ant_r = P + rx;
    w.tau_s = (float)w.sl - K.s_mid;
    w.tn = (float)w.sl * K.tc;
#pragma unroll
    for (int r = 0; r < 3; ++r) {
        w.ptx[r] = K.ant[tx][r];
        w.prx[r] = K.ant[P + rx][r];
    }
    const int32_t *list = A.vis_idx + (int64_t)o * F + (A.vstart ? A.vstart[vrow] : 0);
    const int cnt = A.vcnt[vrow];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
    unsigned long long nV = 0, nSr = 0, nE = 0;
    const float twopi = 6.283185307179586f;
    auto process = [&](int i) {
        float R[24];
        const int cls = build_mixed_record(A, K, w, list[i], R);
        if (cls == kRecVertex) {
            ++nV;
            const float hi = R[15], p2 = R[16];
            // the common part of the lines' positions (exact: hi is a
            // multiple of 2^-14) and of their centred phases
            const float xh = hi * C.fG;
            const int gi = (int)floorf(xh);
            const float xh_f = xh - (float)gi;
            const float ph_h = red1(hi * C.halfM);
            const float a1 = twopi * p2, a2 = -0.5f * a1 * a1;
            // the three lines: strengths, tap polynomials' argument, base cells
            float cr[3], ci[3], t[3];
            int xi[3];
#pragma unroll
            for (int v = 0; v < 3; ++v) {
                const float lo = R[3 + v], wv = R[6 + v];
                const float Cv = red1(R[v] + ph_h + fmaf(lo, C.halfM, p2 * C.quarterM2));
                const float xf = xh_f + fmaf(lo, C.fG, p2 * C.fM * C.fG);
                float s_, c_;
                sincospif(2.f * Cv, &s_, &c_);
                cr[v] = wv * c_;
                ci[v] = wv * s_;
                const float xfl = floorf(xf);
                t[v] = 2.f * (xf - xfl) - 1.f;
                xi[v] = gi + (int)xfl;
            }
            const int xmin = min(min(xi[0], xi[1]), xi[2]);
            const int xmax = max(max(xi[0], xi[1]), xi[2]);
            if (xmax - xmin <= 1) {
                // the lines share a window of W + 1 taps: sum them per tap in
                // registers, one reduction per cell (a third of the adds, and
                // the facet's cancellation done before rounding into the grid)
                float ar[kW0 + 1], ai[kW0 + 1];
#pragma unroll
                for (int j = 0; j <= kW0; ++j) ar[j] = ai[j] = 0.f;
#pragma unroll
                for (int v = 0; v < 3; ++v) {
                    float k0[kW0];
                    kernel_taps<kW0, kD0>(C.c0, t[v], k0);
                    const bool up = xi[v] != xmin;       // window starts one cell later
#pragma unroll
                    for (int j = 0; j <= kW0; ++j) {
                        const float kk = up ? (j > 0 ? k0[j - 1] : 0.f) : (j < kW0 ? k0[j] : 0.f);
                        ar[j] = fmaf(kk, cr[v], ar[j]);
                        ai[j] = fmaf(kk, ci[v], ai[j]);
                    }
                }
#pragma unroll
                for (int j = 0; j <= kW0; ++j) {
                    const int g = wrap_cell(xmin - kW0 / 2 + 1 + j, G);
                    red_add(gr0 + g, ar[j]);
                    red_add(gi0 + g, ai[j]);
                }
                if (p2 != 0.f) {                   // moving facet: quadratic-phase grids
                    float br[kW1 + 1], bi[kW1 + 1];
#pragma unroll
                    for (int j = 0; j <= kW1; ++j) br[j] = bi[j] = 0.f;
#pragma unroll
                    for (int v = 0; v < 3; ++v) {
                        float k1[kW1];
                        kernel_taps<kW1, kD1>(C.c1, t[v], k1);
                        const bool up = xi[v] != xmin;
#pragma unroll
                        for (int j = 0; j <= kW1; ++j) {
                            const float kk = up ? (j > 0 ? k1[j - 1] : 0.f) : (j < kW1 ? k1[j] : 0.f);
                            br[j] = fmaf(kk, cr[v], br[j]);
                            bi[j] = fmaf(kk, ci[v], bi[j]);
                        }
                    }
#pragma unroll
                    for (int j = 0; j <= kW1; ++j) {
                        const int g = wrap_cell(xmin - kW1 / 2 + 1 + j, G);
                        // j 2 pi p2 (br + j bi) and -2 pi^2 p2^2 (br + j bi)
                        red_add(gr1 + g, -a1 * bi[j]);
                        red_add(gi1 + g, a1 * br[j]);
                        red_add(gr2 + g, a2 * br[j]);
                        red_add(gi2 + g, a2 * bi[j]);
                    }
                }
            } else {
                // lines in separate windows (a facet spanning cells): each alone
#pragma unroll
                for (int v = 0; v < 3; ++v) {
                    float k0[kW0];
                    kernel_taps<kW0, kD0>(C.c0, t[v], k0);
#pragma unroll
                    for (int j = 0; j < kW0; ++j) {
                        const int g = wrap_cell(xi[v] - kW0 / 2 + 1 + j, G);
                        red_add(gr0 + g, k0[j] * cr[v]);
                        red_add(gi0 + g, k0[j] * ci[v]);
                    }
                    if (p2 != 0.f) {
                        float k1[kW1];
                        kernel_taps<kW1, kD1>(C.c1, t[v], k1);
                        const float r1 = -a1 * ci[v], i1 = a1 * cr[v], r2 = a2 * cr[v],
                                    i2 = a2 * ci[v];
#pragma unroll
                        for (int j = 0; j < kW1; ++j) {
                            const int g = wrap_cell(xi[v] - kW1 / 2 + 1 + j, G);
                            red_add(gr1 + g, k1[j] * r1);
                            red_add(gi1 + g, k1[j] * i1);
                            red_add(gr2 + g, k1[j] * r2);
                            red_add(gi2 + g, k1[j] * i2);
                        }
                    }
                }
            }
        } else {
            if (cls == kRecSeries) ++nSr;
            else ++nE;
            const int q = atomicAdd(&s_qn, 1);
            if (q < kQueue) {
                queue[q] = i;
            } else {                           // queue full: this lane alone
                const bool series = cls == kRecSeries;
                for (int m = 0; m < M; ++m) {
                    float dr, di;
                    series_edge_term(R, series, (float)m, K, dr, di);
                    red_add(dre + m, dr);
                    red_add(dim + m, di);
                }
            }
        }
        };
    // the list in kSpecBlocksPerWarp x nwarp blocks, which the warps take in
    // turn from a shared counter (a warp whose blocks hold cheaper records
    // takes more of them), its lanes consecutive runs of each block: a warp
    // stays mostly within one mesh (fewer divergent record forms, e.g. the
    // ground's large static facets apart from the vehicles'), while the
    // lanes, runs apart, rarely add to the same grid cell at once
    {
        const int nb = kSpecBlocksPerWarp * nwarp;
        const int bs = (cnt + nb - 1) / nb, lseg = (bs + 31) / 32;
        for (;;) {
            int b = 0;
            if (lane == 0) b = atomicAdd(&s_next, 1);
            b = __shfl_sync(0xffffffffu, b, 0);
            if (b >= nb) break;
            const int i0 = b * bs + lane * lseg;
            const int i1 = min(cnt, min((b + 1) * bs, i0 + lseg));
            for (int i = i0; i < i1; ++i) process(i);
        }
    }
    __syncthreads();
    // queued series / edge records: a warp per record, its lanes over the samples
    const int nq = min(s_qn, kQueue);
    for (int q = warp; q < nq; q += nwarp) {
        float R[24];
        const int cls = build_mixed_record(A, K, w, list[queue[q]], R);
        const bool series = cls == kRecSeries;
        for (int m = lane; m < M; m += 32) {
            float dr, di;
            series_edge_term(R, series, (float)m, K, dr, di);
            red_add(dre + m, dr);
            red_add(dim + m, di);
        }
    }
    __syncthreads();
    // the three grids into interleaved complex transforms, inverse FFTs
    for (int i = threadIdx.x; i < 3 * G; i += blockDim.x) {
        const int c = i / G, g = i % G;
        const float *re = c == 0 ? gr0 : c == 1 ? gr1 : gr2;
        const float *im = c == 0 ? gi0 : c == 1 ? gi1 : gi2;
        buf0[i] = make_float2(re[g], im[g]);
    }
    __syncthreads();
    const C2 *res = stockham<C2, float>(buf0, buf1, tw, G, 3, -1);
    // deconvolve, add the quadratic-phase terms and the direct records,
    // scale by C / k_m^2 and write the row
    const int64_t out_row = ((int64_t)vrow * A.rd.N + n) * M;
    for (int m = threadIdx.x; m < M; m += blockDim.x) {
        const int mp = m - (M >> 1);
        const int k = mp < 0 ? mp + G : mp;
        const float q0 = inv_psi[m], q1 = inv_psi[M + m];
        const float m2 = (float)mp * (float)mp;
        const C2 y0 = res[k], y1 = res[G + k], y2 = res[2 * G + k];
        const float xr = fmaf(y0.x, q0, q1 * m2 * fmaf(y2.x, m2, y1.x)) + dre[m];
        const float xi = fmaf(y0.y, q0, q1 * m2 * fmaf(y2.y, m2, y1.y)) + dim[m];
        const float kp = fmaf((float)m, K.kap_step, 1.f);
        const float sc = K.out_scale / (kp * kp);
        if (A.out_c64) reinterpret_cast<float2 *>(A.out)[out_row + m] = make_float2(xr * sc, xi * sc);
        else reinterpret_cast<double2 *>(A.out)[out_row + m] =
                 make_double2((double)xr * sc, (double)xi * sc);
    }
    if (A.counters) {
        for (int off = 16; off > 0; off >>= 1) {
            nV += __shfl_xor_sync(0xffffffffu, nV, off);
            nSr += __shfl_xor_sync(0xffffffffu, nSr, off);
            nE += __shfl_xor_sync(0xffffffffu, nE, off);
        }
        if (lane == 0) {
            atomicAdd(A.counters + 0, nV);
            atomicAdd(A.counters + 1, nSr);
            atomicAdd(A.counters + 2, nE);
        }
    }
}

double es_value(double z, int W, double beta)
{
    const double sv = 2.0 * z / W, t = 1.0 - sv * sv;
    return t > 0.0 ? exp(beta * (sqrt(t) - 1.0)) : 0.0;
}

// continuous Fourier transform of the kernel at m' cycles over the grid:
// int psi(z) cos(2 pi z m' / G) dz over |z| < W/2, with z = (W/2) sin(theta)
// (the integrand is then smooth on [-pi/2, pi/2]); midpoint rule
double es_hat(int W, double beta, double mp, double G)
{
    const int n = 4096;
    const double hw = 0.5 * W, h = kPi / n;
    double s = 0.0;
    for (int i = 0; i < n; ++i) {
        const double th = -0.5 * kPi + (i + 0.5) * h;
        const double z = hw * sin(th);
        s += exp(beta * (cos(th) - 1.0)) * cos(2.0 * kPi * z * mp / G) * hw * cos(th);
    }
    return s * h;
}

// tap polynomials: Chebyshev interpolation of psi(j - W/2 + 1 - u), u in
// [0, 1), at D + 1 Chebyshev nodes of t = 2u - 1, converted to monomials in t
template <int W, int D>
void fit_taps(double beta, float (&out)[W][D + 1])
{
    const int n = D + 1;
    double T[D + 1][D + 1] = {};          // monomial coefficients of T_0 .. T_D
    T[0][0] = 1.0;
    if (D >= 1) T[1][1] = 1.0;
    for (int d = 2; d <= D; ++d)
        for (int e = 0; e <= d; ++e)
            T[d][e] = (e > 0 ? 2.0 * T[d - 1][e - 1] : 0.0) - T[d - 2][e];
    for (int j = 0; j < W; ++j) {
        double f[D + 1], cheb[D + 1];
        for (int k = 0; k < n; ++k) {
            const double t = cos(kPi * (k + 0.5) / n);
            f[k] = es_value(j - 0.5 * W + 1.0 - 0.5 * (t + 1.0), W, beta);
        }
        for (int m = 0; m < n; ++m) {
            double a = 0.0;
            for (int k = 0; k < n; ++k) a += f[k] * cos(kPi * m * (k + 0.5) / n);
            cheb[m] = (m == 0 ? 1.0 : 2.0) * a / n;
        }
        for (int e = 0; e <= D; ++e) {
            double a = 0.0;
            for (int d = 0; d <= D; ++d) a += cheb[d] * T[d][e];
            out[j][e] = (float)a;
        }
    }
}

size_t spectral_smem(int M)
{
    const int G = 2 * M;
    return (size_t)6 * G * sizeof(float) + (size_t)(3 * G + tw_len(G)) * sizeof(float2) +
           (size_t)2 * M * sizeof(float) + (size_t)kQueue * sizeof(int);
}

}  // namespace

bool spectral_supported(int M) { return spectral_smem(M) <= (size_t)200 * 1024; }

void spectral_tables(int M, float *host)
{
    const int G = 2 * M;
    for (int m = 0; m < M; ++m) {
        const double mp = (double)(m - M / 2);
        host[m] = (float)(1.0 / es_hat(kW0, kBetaPerTap * kW0, mp, G));
        host[M + m] = (float)(1.0 / es_hat(kW1, kBetaPerTap * kW1, mp, G));
    }
}

void launch_synth_spectral(const SynthArgs &a, const float *inv_psi, cudaStream_t s)
{
    const MixConsts K = mix_consts(a.rd);
    static const SpecConsts base = [] {      // the tap polynomials, fitted once
        SpecConsts b{};
        fit_taps<kW0, kD0>(kBetaPerTap * kW0, b.c0);
        fit_taps<kW1, kD1>(kBetaPerTap * kW1, b.c1);
        return b;
    }();
    SpecConsts C = base;
    C.M = a.rd.M;
    C.G = 2 * a.rd.M;
    C.halfM = 0.5f * (float)C.M;
    C.quarterM2 = 0.25f * (float)C.M * (float)C.M;
    C.fM = (float)C.M;
    C.fG = (float)C.G;
    const size_t sm = spectral_smem(C.M);
    const unsigned int rows = (unsigned int)((int64_t)a.VO * a.nc);
    cudaFuncSetAttribute(synth_spectral_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)sm);
    synth_spectral_kernel<<<rows, kSpecThreads, sm, s>>>(a, K, C, inv_psi);
}

}  // namespace bart
