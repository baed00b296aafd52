// Adjoint of the plain FP64 echo synthesis (differentiable echo).
//
// For a real loss L of the ADC cube x with G = dL/dRe(x) + i dL/dIm(x), the
// gradient with respect to a real facet parameter p (a world vertex
// coordinate at the frame start, or the reflectivity) is
//   dL/dp = sum_{rows, samples} Re( conj(G) dx/dp ),
// the visibility mask held fixed.  Two reverse stages:
//   1. per sample, the partial derivatives of the sample's term with respect
//      to the record entries (path-length polynomial qt/qr and the form
//      coefficients d, see record_fp64.cuh) are weighted by conj(G) and
//      summed over the row's samples (lanes, then a warp reduction): the
//      record adjoint rbar;
//   2. per record, each of the 10 parameters is pushed through the record
//      construction in forward-mode dual numbers and dotted with rbar.
// Facet gradients are then mapped to mesh-local vertices (transpose of the
// instance rotation) and reflectivities.
#include <cuda_runtime.h>
#include <stdint.h>

#include "bart_internal.cuh"
#include "record_fp64.cuh"

namespace bart {

namespace {

constexpr int kAdjWarps = 4;
constexpr int kAdjS = 8;            // samples per lane

struct __align__(16) RecA {
    int kind, flags;
    double r[kRecEntries];
};

__device__ __forceinline__ double warp_sum(double v)
{
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

template <int S>
__global__ void __launch_bounds__(kAdjWarps * 32)
adjoint_fp64_kernel(SynthArgs A, int W, const void *__restrict__ grad, int grad_c64,
                    double *__restrict__ gfac)
{
    __shared__ RecA sR[kAdjWarps][32];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t gw = (int64_t)blockIdx.x * kAdjWarps + warp;
    const int N = A.rd.N, M = A.rd.M;
    const int64_t unit = gw / W;
    const int seg = (int)(gw % W);
    if (unit >= (int64_t)A.VO * N) return;
    const int vrow = (int)(unit / N), n = (int)(unit % N);
    const int o = vrow % A.rd.O;
    const int P = A.rd.P, Q = A.rd.Q;
    const int tx = o / Q, rx = o % Q;
    const int64_t F = A.F;
    const int m0 = (seg * 32 + lane) * S;
    const double c = kC0, f0 = A.rd.f0, mu = A.rd.slope, fs = A.rd.fs;
    const double f_max = f0 + mu * (M - 1) / fs;
    const double k0 = 2.0 * kPi * f0 / c, kmax = 2.0 * kPi * f_max / c;
    const double tn = (double)((int64_t)n * A.rd.slots + (A.rd.tdm ? tx : 0)) * A.rd.Tc;
    const double *ptx = A.rd.ant[tx];
    const double *prx = A.rd.ant[P + rx];
    const double twopi = 2.0 * kPi;

    // conj(G) times the output scale of each of this lane's samples
    const double camp = 2.0 * sqrt(kPi) / pow(4.0 * kPi, 1.5);
    double gr[S], gi[S];
    const int64_t row = ((int64_t)vrow * N + n) * M + m0;
#pragma unroll
    for (int j = 0; j < S; ++j) {
        const double fm = f0 + mu * (double)(m0 + j) / fs;
        const double km = 2.0 * kPi * fm / c;
        const double sc = camp / (km * km);
        double x, y;
        if (grad_c64) {
            const float2 v = reinterpret_cast<const float2 *>(grad)[row + j];
            x = v.x;
            y = v.y;
        } else {
            const double2 v = reinterpret_cast<const double2 *>(grad)[row + j];
            x = v.x;
            y = v.y;
        }
        gr[j] = x * sc;
        gi[j] = -y * sc;
    }

    const int32_t *list = A.vis_idx + (int64_t)o * F + (A.vstart ? A.vstart[vrow] : 0);
    const int cnt = A.vcnt[vrow];

    for (int base = 0; base < cnt; base += 32) {
        const bool valid = base + lane < cnt;
        int64_t k = 0;
        double vel[3] = {0.0, 0.0, 0.0};
        if (valid) {
            k = list[base + lane];
            const int inst = A.fac[k].inst;
            for (int r = 0; r < 3; ++r) vel[r] = A.vel64[3 * inst + r];
            double tri[9], c0[3];
            for (int i = 0; i < 9; ++i) tri[i] = A.tri64[9 * k + i];
            for (int r = 0; r < 3; ++r) c0[r] = A.c64[3 * k + r];
            RecA &R = sR[warp][lane];
            int flags = 0;
            R.kind = build_record<double>(tri, c0, vel, tn, ptx, prx, (double)A.fac[k].rho,
                                          A.rd.intra, k0, kmax,
                                          A.rd.delay_ref ? A.ref64 + 3 * inst : nullptr, R.r,
                                          &flags);
            R.flags = flags;
        }
        __syncwarp();
        double mine[kRecEntries];
#pragma unroll
        for (int e = 0; e < kRecEntries; ++e) mine[e] = 0.0;
        unsigned int mask = __ballot_sync(0xffffffffu, valid);
        while (mask) {
            const int i = __ffs(mask) - 1;
            mask &= mask - 1;
            const RecA &R = sR[warp][i];
            const double *d = R.r + kRecD;
            double ab[kRecEntries];
#pragma unroll
            for (int e = 0; e < kRecEntries; ++e) ab[e] = 0.0;
            // Per lane (samples m0 .. m0 + S - 1, t = t0 + tau):
            //  - sqrt(Q(t)) and 0.5 / sqrt(Q(t)) from their expansions in
            //    u = (Q(t) - Q(t0)) / Q(t0): sqrt(1+u) = 1 + u/2 - u^2/8 + u^3/16,
            //    (1+u)^(-1/2) = 1 - u/2 + 3u^2/8 - 5u^3/16; |u| <= 2|dR/dt| tau / R
            //    stays below 1e-4 (R >= 1 m, |v| <= 30 m/s, tau <= S / fs), so the
            //    truncation is below 4e-18 relative;
            //  - each phasor slot (three vertices, the series term, or three
            //    edges) exp(j 2 pi phi(j)): one sincospi at j = 0 and one for
            //    the first-step increment delta = red(phi(1) - phi(0)); sample j
            //    is the rotated start times exp(j 2 pi r), r = red(phi(j) -
            //    phi(0) - j delta) the phase's curvature residual (|r| < 1e-4
            //    cycles, four series terms: error below 1e-17)
            const int nslot = R.kind == kRecSeries ? 1 : 3;
            const int sstride = R.kind == kRecVertex ? 1 : 3;
            // reciprocals formed once (products instead of FP64 divisions per sample)
            const double inv_fs = 1.0 / fs, inv_c = 1.0 / c, inv_f0 = 1.0 / f0;
            const double mu_2c2 = mu / (2.0 * c * c), mu_c2 = mu / (c * c);
            const double t0 = (double)m0 * inv_fs;
            const double Qt0 = R.r[0] + t0 * (R.r[1] + t0 * R.r[2]);
            const double Qr0 = R.r[3] + t0 * (R.r[4] + t0 * R.r[2]);
            const double st0 = sqrt(Qt0), sr0 = sqrt(Qr0);
            const double ht0 = 0.5 / st0, hr0 = 0.5 / sr0;
            const double at1 = (R.r[1] + 2.0 * R.r[2] * t0) / Qt0, at2 = R.r[2] / Qt0;
            const double ar1 = (R.r[4] + 2.0 * R.r[2] * t0) / Qr0, ar2 = R.r[2] / Qr0;
            double ph0[3], dl[3], zc[3], zs[3], cd[3], sd[3];
#pragma unroll 1
            for (int j = 0; j < S; ++j) {
                const double tau = (double)j * inv_fs;
                const double t = t0 + tau;
                const double fm = f0 + mu * t;
                const double ut = tau * (at1 + tau * at2), ur = tau * (ar1 + tau * ar2);
                const double sQt = st0 * (1.0 + ut * (0.5 + ut * (-0.125 + ut * 0.0625)));
                const double sQr = sr0 * (1.0 + ur * (0.5 + ur * (-0.125 + ur * 0.0625)));
                const double it = ht0 * (1.0 + ut * (-0.5 + ut * (0.375 - ut * 0.3125)));
                const double ir = hr0 * (1.0 + ur * (-0.5 + ur * (0.375 - ur * 0.3125)));
                const double L = sQt + sQr;
                const double fmc = fm * inv_c;
                const double kp = fm * inv_f0;
                double thc = fmc * (L + R.r[kRecLs]) - mu_2c2 * L * L;
                thc -= rint(thc);
                // the phasor of each slot at this sample
                double pc[3], ps[3];
#pragma unroll
                for (int q = 0; q < 3; ++q) {
                    if (q >= nslot) break;
                    double ph = thc - fmc * d[q * sstride];
                    ph -= rint(ph);
                    if (j == 0) {
                        ph0[q] = ph;
                        sincospi(2.0 * ph, &zs[q], &zc[q]);
                        pc[q] = zc[q];
                        ps[q] = zs[q];
                    } else {
                        if (j == 1) {
                            dl[q] = ph - ph0[q];
                            dl[q] -= rint(dl[q]);
                            sincospi(2.0 * dl[q], &sd[q], &cd[q]);
                        }
                        const double nc = zc[q] * cd[q] - zs[q] * sd[q];
                        zs[q] = zc[q] * sd[q] + zs[q] * cd[q];
                        zc[q] = nc;
                        double r = ph - ph0[q] - (double)j * dl[q];
                        r -= rint(r);
                        const double x = twopi * r, x2 = x * x;
                        const double ec = 1.0 - 0.5 * x2 * (1.0 - x2 * (1.0 / 12.0));
                        const double es = x * (1.0 - x2 * (1.0 / 6.0));
                        pc[q] = zc[q] * ec - zs[q] * es;
                        ps[q] = zc[q] * es + zs[q] * ec;
                    }
                }
                double a_thc = 0.0;
                if (R.kind == kRecVertex) {
                    for (int v = 0; v < 3; ++v) {
                        const double c_ = pc[v], s_ = ps[v];
                        const double zr = gr[j] * c_ - gi[j] * s_, zi = gr[j] * s_ + gi[j] * c_;
                        ab[kRecD + 3 + v] += zr;
                        ab[kRecD + v] += twopi * fmc * d[3 + v] * zi;
                        a_thc -= twopi * d[3 + v] * zi;
                    }
                } else if (R.kind == kRecSeries) {
                    const double c_ = pc[0], s_ = ps[0];
                    const double zr = gr[j] * c_ - gi[j] * s_, zi = gr[j] * s_ + gi[j] * c_;
                    const double k2 = kp * kp;
                    double a = d[8], bb = d[15];
                    for (int q = 6; q >= 0; --q) a = a * k2 + d[1 + q];
                    for (int q = 5; q >= 0; --q) bb = bb * k2 + d[9 + q];
                    const double pr_ = a * k2, pi_ = bb * k2 * kp;
                    double pw = k2;
                    for (int q = 0; q < 8; ++q) {
                        ab[kRecD + 1 + q] += zr * pw;
                        if (q < 7) ab[kRecD + 9 + q] -= zi * kp * pw;
                        pw *= k2;
                    }
                    const double wi = zr * pi_ + zi * pr_;
                    ab[kRecD] += twopi * fmc * wi;
                    a_thc -= twopi * wi;
                } else {
                    for (int e = 0; e < 3; ++e) {
                        const double c_ = pc[e], s_ = ps[e];
                        const double zr = gr[j] * c_ - gi[j] * s_, zi = gr[j] * s_ + gi[j] * c_;
                        const double x = kp * d[3 * e + 1];
                        double sn, snp;
                        if (R.flags & (1 << e)) {
                            const double x2 = x * x;
                            sn = 1.0 + x2 * (-1.0 / 6 + x2 * (1.0 / 120 + x2 * (-1.0 / 5040 +
                                 x2 * (1.0 / 362880 + x2 * (-1.0 / 39916800)))));
                            snp = x * (-1.0 / 3 + x2 * (1.0 / 30 + x2 * (-1.0 / 840 +
                                  x2 * (1.0 / 45360 + x2 * (-1.0 / 3991680)))));
                        } else {
                            double sx, cx;
                            sincos(x, &sx, &cx);
                            sn = sx / x;
                            snp = (x * cx - sx) / (x * x);
                        }
                        const double coef = kp * d[3 * e + 2] * sn;
                        ab[kRecD + 3 * e + 2] -= zi * kp * sn;
                        ab[kRecD + 3 * e + 1] -= zi * kp * d[3 * e + 2] * snp * kp;
                        ab[kRecD + 3 * e] += twopi * fmc * coef * zr;
                        a_thc -= twopi * coef * zr;
                    }
                }
                // thc -> L -> path-length polynomial coefficients; thc -> shift
                ab[kRecLs] += a_thc * fmc;
                const double aL = a_thc * (fmc - mu_c2 * L);
                ab[0] += aL * it;
                ab[1] += aL * it * t;
                ab[2] += aL * (it + ir) * t * t;
                ab[3] += aL * ir;
                ab[4] += aL * ir * t;
            }
            // entries each form uses: qt, qr and 6 / 16 / 9 coefficients
            const int used = kRecD + (R.kind == kRecVertex ? 6 : R.kind == kRecSeries ? 16 : 9);
#pragma unroll
            for (int e = 0; e < kRecEntries; ++e) {
                if (e < used) {
                    const double tot = warp_sum(ab[e]);
                    if (lane == i) mine[e] = tot;
                }
            }
        }
        // reverse through the record construction, one parameter at a time
        if (valid) {
            const RecA &R = sR[warp][lane];
            double tri[9], c0[3];
            for (int q = 0; q < 9; ++q) tri[q] = A.tri64[9 * k + q];
            for (int r = 0; r < 3; ++r) c0[r] = A.c64[3 * k + r];
            const double rho = (double)A.fac[k].rho;
            const double *ref = A.rd.delay_ref ? A.ref64 + 3 * A.fac[k].inst : nullptr;
            for (int p = 0; p < 10; ++p) {
                Dual dtri[9], dc0[3], out[kRecEntries];
                for (int e = 0; e < kRecEntries; ++e) out[e] = Dual(0.0, 0.0);
                for (int q = 0; q < 9; ++q) dtri[q] = Dual(tri[q], q == p ? 1.0 : 0.0);
                for (int r = 0; r < 3; ++r)
                    dc0[r] = Dual(c0[r], (p < 9 && p % 3 == r) ? 1.0 / 3.0 : 0.0);
                const Dual drho(rho, p == 9 ? 1.0 : 0.0);
                int flags = 0;
                const int kind = build_record<Dual>(dtri, dc0, vel, tn, ptx, prx, drho, A.rd.intra,
                                                    k0, kmax, ref, out, &flags);
                double gsum = 0.0;
                if (kind == R.kind)
                    for (int e = 0; e < kRecEntries; ++e) gsum += mine[e] * out[e].d;
                atomicAdd(gfac + 10 * k + p, gsum);
            }
        }
        __syncwarp();
    }
}

// facet gradients -> mesh-local vertex and reflectivity gradients
__global__ void adjoint_scatter_kernel(const double *__restrict__ gfac, const FacetRec *__restrict__ fac,
                                       const InstDev *__restrict__ insts, const MeshDesc *__restrict__ meshes,
                                       const int64_t *__restrict__ voff, int64_t F,
                                       double *__restrict__ gverts, double *__restrict__ grho)
{
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= F) return;
    const int inst = fac[k].inst;
    const InstDev &in = insts[inst];
    const MeshDesc &m = meshes[in.mesh];
    const int64_t j = k - in.off;
    for (int v = 0; v < 3; ++v) {
        const int64_t vi = m.tris[3 * j + v];
        for (int cc = 0; cc < 3; ++cc) {
            // world_r = sum_c rot[r][c] local_c
            double g = 0.0;
            for (int r = 0; r < 3; ++r) g += in.rot[3 * r + cc] * gfac[10 * k + 3 * v + r];
            atomicAdd(gverts + 3 * (voff[inst] + vi) + cc, g);
        }
    }
    if (grho) grho[k] = gfac[10 * k + 9] * (double)in.rho_scale;
}

}  // namespace

int64_t adjoint_facet_words(int64_t F) { return 10 * F; }

void launch_adjoint_fp64(const SynthArgs &a, const void *grad, int grad_c64, double *gfac,
                         cudaStream_t s)
{
    const int M = a.rd.M;
    int S = kAdjS;
    while (S > 1 && M % (32 * S) != 0) S >>= 1;
    const int W = M / (32 * S);
    cudaMemsetAsync(gfac, 0, (size_t)a.F * 10 * sizeof(double), s);
    const int64_t warps = (int64_t)a.VO * a.rd.N * W;
    const unsigned int grid = (unsigned int)((warps + kAdjWarps - 1) / kAdjWarps);
    switch (S) {
    case 8: adjoint_fp64_kernel<8><<<grid, kAdjWarps * 32, 0, s>>>(a, W, grad, grad_c64, gfac); break;
    case 4: adjoint_fp64_kernel<4><<<grid, kAdjWarps * 32, 0, s>>>(a, W, grad, grad_c64, gfac); break;
    case 2: adjoint_fp64_kernel<2><<<grid, kAdjWarps * 32, 0, s>>>(a, W, grad, grad_c64, gfac); break;
    default: adjoint_fp64_kernel<1><<<grid, kAdjWarps * 32, 0, s>>>(a, W, grad, grad_c64, gfac); break;
    }
}

void launch_adjoint_scatter(const double *gfac, const FacetRec *fac, const InstDev *insts,
                            const MeshDesc *meshes, const int64_t *voff, int64_t F, double *gverts,
                            int64_t n_vert_words, double *grho, cudaStream_t s)
{
    cudaMemsetAsync(gverts, 0, (size_t)n_vert_words * sizeof(double), s);
    const int T = 256;
    adjoint_scatter_kernel<<<(unsigned int)((F + T - 1) / T), T, 0, s>>>(gfac, fac, insts, meshes,
                                                                        voff, F, gverts, grho);
}

}  // namespace bart
