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
//
// The mixed variant (bart_simulate_adjoint_mixed) takes vertex-form records
// of the per-facet delay form (all but ~1e-3 of a frame) through FP32 only:
// stage 1 from the forward mixed record (mixed_record.cuh: the vertex
// phases, beat frequencies and weights the forward mixed and spectral paths
// use) with the lanes' phasors advanced by rotation (adj_vertex_f32), and
// stage 2 as one hand-derived reverse pass through the record construction
// (vertex_reverse_f32) instead of ten dual-number passes.  FP64 runs at
// 1/64 of the FP32 rate on this GPU, so the FP64 route of the plain adjoint
// is kept for the other records (series and edge forms, the reference-point
// and far-field delay forms) only.
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <type_traits>

#include "bart_internal.cuh"
#include "mixed_record.cuh"
#include "record_fp64.cuh"

namespace bart {

namespace {

constexpr int kAdjWarps = 4;
constexpr int kAdjS = 8;            // samples per lane

struct __align__(16) RecA {
    int kind, flags;
    double r[kRecEntries];
};

// The mixed adjoint's record adds, about the row's middle sample t_c
// (tau = t - t_c), the path length L(tau) = sqrt(Qt) + sqrt(Qr) and the
// phase thc(tau) = fmc (L + shift) - mu L^2 / (2 c^2) as degree-4
// polynomials (from L^2 = Q term by term; the series ratio |v| |tau| / R is
// below 1e-3, so the truncation is ~1e-16 relative), and the quadratics'
// normalised coefficients for 0.5 / sqrt(Q) = (0.5 / s)(1 + u)^(-1/2),
// u = tau (a1 + a2 tau).  Formed once per record: no lane takes an FP64
// square root or division.
struct __align__(16) RecAX : RecA {
    double tc, st, sr, at1, at2, ar1, ar2;
    double Lk[5], thk[5];
};

__device__ __forceinline__ double warp_sum(double v)
{
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Record adjoint of a vertex-form record over one lane's S samples with the
// per-sample work in FP32 (the mixed adjoint).  FP64 gives each vertex's
// phase at the lane's samples 0, 1 and S - 1 (from the record's path-length
// and phase polynomials); the phasors then advance by an FP32 rotation along the chord
// of those phases (the phase's curvature over the lane, p2 (S - 1)^2 / 4
// cycles, is left out: ~1e-5 rad on a moving car), and the sums over the
// lane's samples run in FP32:
//   rbar(w_v) = sum zr_v,   rbar(u_v) = 2 pi w_v sum fmc zi_v,
//   a = -2 pi sum_v w_v zi_v,   rbar(shift) = sum a fmc,
//   rbar(qt_i), rbar(qr_i) from sum a (fmc - mu L / c^2) t^i,
// with z = conj(G) exp(j 2 pi phase); 0.5 / sqrt(Q) is held at the lane's
// first sample (it moves by ~5e-7 of itself over 8 samples).
// (1 + u)^(-1/2) to fourth order in u: with |u| <= 2 |dR/dt|
// |tau| / R below 1.5e-3 (R >= 1 m, |v| <= 30 m/s, |tau| <= 25 us) the
// truncation is below 2e-16 relative
__device__ __forceinline__ double rsqrt1p4(double u)
{
    return 1.0 + u * (-0.5 + u * (0.375 + u * (-0.3125 + u * 0.2734375)));
}

template <int S>
__device__ __forceinline__ void adj_vertex_mixed(const RecAX &X, int m0, double f0, double mu,
                                                 double fs, double c, const double *gr,
                                                 const double *gi, float *fb)
{
    const double *rr = X.r;
    const double *d = rr + kRecD;
    const double inv_fs = 1.0 / fs, inv_c = 1.0 / c;
    const double t0 = (double)m0 * inv_fs;
    const int jp[3] = {0, 1, S - 1};
    double th[3][3], Lp[3];
#pragma unroll
    for (int p = 0; p < 3; ++p) {
        const double t = t0 + (double)jp[p] * inv_fs;
        const double tau = t - X.tc;
        double thc = X.thk[4], L = X.Lk[4];
#pragma unroll
        for (int q = 3; q >= 0; --q) {
            thc = fma(thc, tau, X.thk[q]);
            L = fma(L, tau, X.Lk[q]);
        }
        thc -= rint(thc);
        const double fmc = (f0 + mu * t) * inv_c;
#pragma unroll
        for (int v = 0; v < 3; ++v) {
            double ph = thc - fmc * d[v];
            th[p][v] = ph - rint(ph);
        }
        Lp[p] = L;
    }
    float zc[3], zs[3], cst[3], sst[3], wv[3], Sw[3], Su[3];
#pragma unroll
    for (int v = 0; v < 3; ++v) {
        double d1 = th[1][v] - th[0][v];
        d1 -= rint(d1);
        double slope = d1;
        if (S > 2) {
            double r = th[2][v] - th[0][v] - (double)(S - 1) * d1;
            r -= rint(r);
            slope += r / (double)(S > 2 ? S - 1 : 1);
        }
        sincospif(2.f * (float)th[0][v], &zs[v], &zc[v]);
        sincospif(2.f * (float)slope, &sst[v], &cst[v]);
        wv[v] = (float)d[3 + v];
        Sw[v] = Su[v] = 0.f;
    }
    const float fmc0 = (float)((f0 + mu * t0) * inv_c), dfmc = (float)(mu * inv_fs * inv_c);
    const float L0 = (float)Lp[0];
    const float dL = S > 1 ? (float)((Lp[2] - Lp[0]) / (double)(S - 1)) : 0.f;
    const float muc2 = (float)(mu * inv_c * inv_c);
    const float t0f = (float)t0, dt = (float)inv_fs;
    float A0 = 0.f, A1 = 0.f, A2 = 0.f, Ash = 0.f;
#pragma unroll
    for (int j = 0; j < S; ++j) {
        const float fmc = fmaf((float)j, dfmc, fmc0);
        const float t = fmaf((float)j, dt, t0f);
        const float L = fmaf((float)j, dL, L0);
        const float g_r = (float)gr[j], g_i = (float)gi[j];
        float a = 0.f;
#pragma unroll
        for (int v = 0; v < 3; ++v) {
            const float zr = fmaf(g_r, zc[v], -g_i * zs[v]);
            const float zi = fmaf(g_r, zs[v], g_i * zc[v]);
            Sw[v] += zr;
            Su[v] = fmaf(fmc, zi, Su[v]);
            a = fmaf(-wv[v], zi, a);
            const float nc = fmaf(zc[v], cst[v], -zs[v] * sst[v]);
            zs[v] = fmaf(zc[v], sst[v], zs[v] * cst[v]);
            zc[v] = nc;
        }
        Ash = fmaf(a, fmc, Ash);
        const float aL = a * fmaf(-muc2, L, fmc);
        A0 += aL;
        A1 = fmaf(aL, t, A1);
        A2 = fmaf(aL * t, t, A2);
    }
    // 0.5 / sqrt(Q) at the lane's first sample
    const double tau0 = t0 - X.tc;
    const float twopi = 6.283185307179586f;
    const float it = (float)(0.5 / X.st * rsqrt1p4(tau0 * (X.at1 + tau0 * X.at2)));
    const float ir = (float)(0.5 / X.sr * rsqrt1p4(tau0 * (X.ar1 + tau0 * X.ar2)));
    // the record adjoint's entries in record order (qt[3], qr[2], shift, u[3], w[3])
    fb[0] = twopi * it * A0;
    fb[1] = twopi * it * A1;
    fb[2] = twopi * (it + ir) * A2;
    fb[3] = twopi * ir * A0;
    fb[4] = twopi * ir * A1;
    fb[kRecLs] = twopi * Ash;
#pragma unroll
    for (int v = 0; v < 3; ++v) {
        fb[kRecD + v] = twopi * (float)d[3 + v] * Su[v];
        fb[kRecD + 3 + v] = Sw[v];
    }
}

// FP32 vertex-form record of the mixed adjoint: the forward mixed record's
// phase model ph_v(m) = ph0_v + (hi + lo_v) m + p2 m^2 (cycles) and weights
// w_v, the chirp-start path L0 = R_t + R_r and its rate Ld, and the
// adjoint's d sqrt(Q) / dQ = 0.5 / R(t) = it + itd t (TX; ir, ird for the
// RX) to first order in the fast time t
struct RecF {
    int kind, pad;          // kind = kRouteF32 (the same leading member as RecA)
    float ph0[3], lo[3], w[3];
    float hi, p2, L0, Ld, it, ir, itd, ird;
};
constexpr int kRouteF32 = -1;

// Stage 1 of a RecF record over one lane's S samples m0 .. m0 + S - 1: the
// phasors start from sincospi at m0 and rotate by the chord step of the
// lane (the curvature p2 (S - 1)^2 / 4 cycles, below 1e-6, is left out);
// out = {sum zr_v (3), sum fmc zi_v (3), sum aL, sum aL t, sum aL t^2} with
// z_v = conj(G) exp(j 2 pi ph_v), a = -sum_v w_v zi_v,
// aL = a (fmc - mu L / c^2), fmc = f_m / c, t = m / fs.
template <int S>
__device__ __forceinline__ void adj_vertex_f32(const RecF &F, int m0, const MixConsts &K,
                                               float muc2, float inv_fs, const float *gr,
                                               const float *gi, float *out)
{
    const float fm0 = (float)m0;
    const float hm = red1(F.hi * fm0);             // exact: hi is a multiple of 2^-14
    float zc[3], zs[3], cs[3], ss[3];
#pragma unroll
    for (int v = 0; v < 3; ++v) {
        const float ph = red1(F.ph0[v] + hm + fmaf(F.lo[v], fm0, F.p2 * fm0 * fm0));
        sincospif(2.f * ph, &zs[v], &zc[v]);
        const float st = red1(F.hi + fmaf(F.p2, 2.f * fm0 + (float)(S - 1), F.lo[v]));
        sincospif(2.f * st, &ss[v], &cs[v]);
    }
    float Sw[3] = {0.f, 0.f, 0.f}, Su[3] = {0.f, 0.f, 0.f}, A0 = 0.f, A1 = 0.f, A2 = 0.f;
#pragma unroll
    for (int j = 0; j < S; ++j) {
        const float m = fm0 + (float)j;
        const float fmc = fmaf(m, K.muc, K.f0c);
        const float t = m * inv_fs;
        const float L = fmaf(F.Ld, t, F.L0);
        float a = 0.f;
#pragma unroll
        for (int v = 0; v < 3; ++v) {
            const float zr = fmaf(gr[j], zc[v], -gi[j] * zs[v]);
            const float zi = fmaf(gr[j], zs[v], gi[j] * zc[v]);
            Sw[v] += zr;
            Su[v] = fmaf(fmc, zi, Su[v]);
            a = fmaf(-F.w[v], zi, a);
            const float nc = fmaf(zc[v], cs[v], -zs[v] * ss[v]);
            zs[v] = fmaf(zc[v], ss[v], zs[v] * cs[v]);
            zc[v] = nc;
        }
        const float aL = a * fmaf(-muc2, L, fmc);
        A0 += aL;
        A1 = fmaf(aL, t, A1);
        A2 = fmaf(aL * t, t, A2);
    }
#pragma unroll
    for (int v = 0; v < 3; ++v) {
        out[v] = Sw[v];
        out[3 + v] = Su[v];
    }
    out[6] = A0;
    out[7] = A1;
    out[8] = A2;
}

__device__ __forceinline__ void cross3(const float *a, const float *b, float *c)
{
    c[0] = a[1] * b[2] - a[2] * b[1];
    c[1] = a[2] * b[0] - a[0] * b[2];
    c[2] = a[0] * b[1] - a[1] * b[0];
}
__device__ __forceinline__ float dot3(const float *a, const float *b)
{
    return fmaf(a[0], b[0], fmaf(a[1], b[1], a[2] * b[2]));
}

// Stage 2 of a vertex-form record, per-facet delay form: the record entries
// (record_fp64.cuh)
//   qt0 = |p_t - c(t_n)|^2, qt1 = -2 (p_t - c(t_n)).v (intra-chirp motion),
//   the same for the RX, u_v = b_t . dv_v, w_v = -A2 / ((u_v - u_a)(u_v - u_b)),
//   b = t + r, b_t its part in the facet plane, A2 = 2 area rho o / (R_t R_r),
//   o = n.b / 2 (|.| for two-sided facets),
// are reversed in FP32 from their adjoints bar = {qt0, qt1, qr0, qr1, u (3),
// w (3)} to the adjoints of the nine world vertex coordinates at the frame
// start (c = their mean, dv_v = vertex_v - c) and of rho: g[10].
__device__ __forceinline__ void vertex_reverse_f32(const FacetRec &fr, const float *vel, float tn,
                                                   const float *pt, const float *pr, int intra,
                                                   const float *bar, float *g)
{
    float dv[9];
#pragma unroll
    for (int i = 0; i < 9; ++i) dv[i] = fr.dv[i];
    float dt[3], dr[3];
#pragma unroll
    for (int r = 0; r < 3; ++r) {
        const float cc = fmaf(vel[r], tn, fr.c[r]);
        dt[r] = pt[r] - cc;
        dr[r] = pr[r] - cc;
    }
    const float Rt = sqrtf(dot3(dt, dt)), Rr = sqrtf(dot3(dr, dr));
    const float iRt = 1.f / Rt, iRr = 1.f / Rr;
    float b[3];
#pragma unroll
    for (int r = 0; r < 3; ++r) b[r] = fmaf(dt[r], iRt, dr[r] * iRr);
    const float e1[3] = {dv[3] - dv[0], dv[4] - dv[1], dv[5] - dv[2]};
    const float e2[3] = {dv[6] - dv[0], dv[7] - dv[1], dv[8] - dv[2]};
    float nr[3];
    cross3(e1, e2, nr);
    const float nl = sqrtf(dot3(nr, nr)), inl = 1.f / nl;
    const float nn[3] = {nr[0] * inl, nr[1] * inl, nr[2] * inl};
    const float area = 0.5f * nl;
    const float okr = 0.5f * dot3(nn, b);
    const float sg = (fr.two_sided && okr < 0.f) ? -1.f : 1.f;
    const float ok = sg * okr;
    const float iRR = iRt * iRr;
    const float gg = fr.rho * ok * iRR;
    const float bn = dot3(b, nn);
    const float bt[3] = {b[0] - bn * nn[0], b[1] - bn * nn[1], b[2] - bn * nn[2]};
    float u[3];
#pragma unroll
    for (int v = 0; v < 3; ++v) u[v] = dot3(bt, dv + 3 * v);
    const float A2 = 2.f * area * gg;
    // w_v = -A2 / D_v, D_v = (u_v - u_a)(u_v - u_b)
    float ub[3] = {bar[4], bar[5], bar[6]};
    float A2b = 0.f;
#pragma unroll
    for (int v = 0; v < 3; ++v) {
        const int a = (v + 1) % 3, c = (v + 2) % 3;
        const float da = u[v] - u[a], dc = u[v] - u[c];
        const float iD = 1.f / (da * dc);
        const float wb = bar[7 + v];
        A2b -= wb * iD;
        const float Db = wb * A2 * iD * iD;
        ub[v] += Db * (dc + da);
        ub[a] -= Db * dc;
        ub[c] -= Db * da;
    }
    const float areab = 2.f * gg * A2b, gb = 2.f * area * A2b;
    g[9] = gb * ok * iRR;
    const float okb = gb * fr.rho * iRR;
    float Rtb = -gb * gg * iRt, Rrb = -gb * gg * iRr;
    // u_v = bt . dv_v
    float btb[3] = {0.f, 0.f, 0.f}, dvb[9];
#pragma unroll
    for (int v = 0; v < 3; ++v)
#pragma unroll
        for (int r = 0; r < 3; ++r) {
            btb[r] = fmaf(ub[v], dv[3 * v + r], btb[r]);
            dvb[3 * v + r] = ub[v] * bt[r];
        }
    // bt = b - (b.n) n, o = s (n.b) / 2
    const float bnb = -dot3(nn, btb);
    float bb[3], nnb[3];
#pragma unroll
    for (int r = 0; r < 3; ++r) {
        bb[r] = btb[r] + bnb * nn[r] + 0.5f * sg * okb * nn[r];
        nnb[r] = -bn * btb[r] + bnb * b[r] + 0.5f * sg * okb * b[r];
    }
    // n = nr / |nr|, area = |nr| / 2
    const float nnd = dot3(nn, nnb);
    float nrb[3];
#pragma unroll
    for (int r = 0; r < 3; ++r) nrb[r] = (nnb[r] - nn[r] * nnd) * inl + 0.5f * areab * nn[r];
    // nr = e1 x e2
    float e1b[3], e2b[3];
    cross3(e2, nrb, e1b);
    cross3(nrb, e1, e2b);
#pragma unroll
    for (int r = 0; r < 3; ++r) {
        dvb[3 + r] += e1b[r];
        dvb[6 + r] += e2b[r];
        dvb[r] -= e1b[r] + e2b[r];
    }
    // b = dt / R_t + dr / R_r; R = |d|; qt0 = |dt|^2, qt1 = -2 dt.v
    const float bdt = dot3(bb, dt), bdr = dot3(bb, dr);
    float ccb[3];
#pragma unroll
    for (int r = 0; r < 3; ++r) {
        float dtb = bb[r] * iRt - dt[r] * (bdt * iRt * iRt * iRt) + Rtb * iRt * dt[r] +
                    2.f * bar[0] * dt[r];
        float drb = bb[r] * iRr - dr[r] * (bdr * iRr * iRr * iRr) + Rrb * iRr * dr[r] +
                    2.f * bar[2] * dr[r];
        if (intra) {
            dtb -= 2.f * bar[1] * vel[r];
            drb -= 2.f * bar[3] * vel[r];
        }
        ccb[r] = -(dtb + drb);
    }
    // c(t_n) = c + v t_n, dv_v = vertex_v - c, c = mean of the vertices
#pragma unroll
    for (int r = 0; r < 3; ++r) {
        const float cb = ccb[r] - (dvb[r] + dvb[3 + r] + dvb[6 + r]);
#pragma unroll
        for (int v = 0; v < 3; ++v) g[3 * v + r] = dvb[3 * v + r] + cb * (1.f / 3.f);
    }
}

__device__ __forceinline__ float warp_sum_f(float v)
{
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

constexpr int kAdjMixMinBlocks = 4;   // resident blocks the mixed variant's register budget targets

template <int S, bool MX>
__global__ void __launch_bounds__(kAdjWarps * 32, MX ? kAdjMixMinBlocks : 1)
adjoint_fp64_kernel(SynthArgs A, MixConsts K, int W, int NCH, const void *__restrict__ grad,
                    int grad_c64, double *__restrict__ gfac)
{
    using Rec = typename std::conditional<MX, RecAX, RecA>::type;
    // a lane's record: FP64 (Rec) or, in the mixed variant's FP32 route, RecF
    union RecU {
        Rec x;
        RecF f;
    };
    __shared__ RecU sU[kAdjWarps][32];          // .x.kind == kRouteF32: the FP32 route
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t gw = (int64_t)blockIdx.x * kAdjWarps + warp;
    const int N = A.rd.N, M = A.rd.M;
    // warp = (row unit, sample segment, chunk of the row's facet list)
    const int64_t unit = gw / ((int64_t)W * NCH);
    const int seg = (int)(gw / NCH % W), chunk = (int)(gw % NCH);
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

    // the mixed variant's FP32 route: per-facet delay form, near field
    const bool f32_route = MX && !A.rd.delay_ref && !A.rd.far_field;
    float gfr[S], gfi[S];
    MixRow w;
    float muc2 = 0.f, inv_fs = 0.f;
    if constexpr (MX) {
#pragma unroll
        for (int j = 0; j < S; ++j) {
            gfr[j] = (float)gr[j];
            gfi[j] = (float)gi[j];
        }
        const int slot = A.rd.tdm ? tx : 0;
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
        muc2 = (float)(mu / (c * c));
        inv_fs = (float)(1.0 / fs);
    }

    const int nbat = (cnt + 31) / 32;
    const int bat0 = (int)((int64_t)nbat * chunk / NCH);
    const int bat1 = (int)((int64_t)nbat * (chunk + 1) / NCH);
    for (int base = bat0 * 32; base < bat1 * 32; base += 32) {
        const bool valid = base + lane < cnt;
        int64_t k = 0;
        double vel[3] = {0.0, 0.0, 0.0};
        int f32 = 0;
        if (valid) {
            k = list[base + lane];
            const int inst = A.fac[k].inst;
            for (int r = 0; r < 3; ++r) vel[r] = A.vel64[3 * inst + r];
            if constexpr (MX) {
                if (f32_route) {
                    float Rm[24];
                    // (a stricter vertex-form limit for this route, k_max d_min
                    // >= kd instead of kEdgeKd = 0.03, trades speed for accuracy
                    // on the sedan: kd 0.1 / 0.25 / 0.5 / 1.0 gave 19 / 32 / 51 /
                    // 76 ms at 4.7e-5 / 2.9e-5 / 4.6e-6 / 2.3e-6 from the FP64
                    // adjoint, against 13 ms at 5.7e-5: the derivative of a
                    // nearly equal projection pair cancels as 1 / (k d), which
                    // amplifies the FP32 phase steps' rounding)
                    if (build_mixed_record(A, K, w, (int)k, Rm, true) == kRecVertex) {
                        f32 = 1;
                        RecF &Fr = sU[warp][lane].f;
                        Fr.kind = kRouteF32;
#pragma unroll
                        for (int v = 0; v < 3; ++v) {
                            Fr.ph0[v] = Rm[v];
                            Fr.lo[v] = Rm[3 + v];
                            Fr.w[v] = Rm[6 + v];
                        }
                        Fr.hi = Rm[15];
                        Fr.p2 = Rm[16];
                        // chirp-start ranges and the path's rate (FP32 suffices
                        // for the factors d sqrt(Q) / dQ and fmc - mu L / c^2)
                        const FacetRec fr = A.fac[k];
                        const float4 vv = reinterpret_cast<const float4 *>(A.vel32)[fr.inst];
                        const float vf[3] = {vv.x, vv.y, vv.z};
                        float dt[3], dr[3];
                        for (int r = 0; r < 3; ++r) {
                            const float cc = fmaf(vf[r], w.tn, fr.c[r]);
                            dt[r] = w.ptx[r] - cc;
                            dr[r] = w.prx[r] - cc;
                        }
                        const float Rt = sqrtf(dot3(dt, dt)), Rr = sqrtf(dot3(dr, dr));
                        const float Rtd = A.rd.intra ? -dot3(vf, dt) / Rt : 0.f;
                        const float Rrd = A.rd.intra ? -dot3(vf, dr) / Rr : 0.f;
                        Fr.L0 = Rt + Rr;
                        Fr.Ld = Rtd + Rrd;
                        Fr.it = 0.5f / Rt;
                        Fr.ir = 0.5f / Rr;
                        Fr.itd = -Fr.it * Rtd / Rt;
                        Fr.ird = -Fr.ir * Rrd / Rr;
                    }
                }
            }
        }
        if (valid && !f32) {
            const int inst = A.fac[k].inst;
            double tri[9], c0[3];
            for (int i = 0; i < 9; ++i) tri[i] = A.tri64[9 * k + i];
            for (int r = 0; r < 3; ++r) c0[r] = A.c64[3 * k + r];
            Rec &R = sU[warp][lane].x;
            int flags = 0;
            R.kind = build_record<double>(tri, c0, vel, tn, ptx, prx, (double)A.fac[k].rho,
                                          A.rd.intra, k0, kmax,
                                          A.rd.delay_ref ? kDelayRef : kDelayFacet,
                                          A.ref64 + 3 * inst, A.fac[k].two_sided, R.r, &flags);
            R.flags = flags;
            if constexpr (MX) {
                // the path lengths' expansion about the row's middle sample
                R.tc = 0.5 * (double)(M - 1) / fs;
                const double Qt = R.r[0] + R.tc * (R.r[1] + R.tc * R.r[2]);
                const double Qr = R.r[3] + R.tc * (R.r[4] + R.tc * R.r[2]);
                R.st = sqrt(Qt);
                R.sr = sqrt(Qr);
                R.at1 = (R.r[1] + 2.0 * R.r[2] * R.tc) / Qt;
                R.at2 = R.r[2] / Qt;
                R.ar1 = (R.r[4] + 2.0 * R.r[2] * R.tc) / Qr;
                R.ar2 = R.r[2] / Qr;
                // sqrt(q0 + q1 tau + q2 tau^2) = sum_k l_k tau^k: 2 l0 l1 = q1,
                // 2 l0 l2 + l1^2 = q2, 2 l0 l3 + 2 l1 l2 = 0, 2 l0 l4 + 2 l1 l3 + l2^2 = 0
                double lt[5], lr[5];
                const double q1t = R.r[1] + 2.0 * R.r[2] * R.tc, q1r = R.r[4] + 2.0 * R.r[2] * R.tc;
                lt[0] = R.st;
                lr[0] = R.sr;
                const double ht = 0.5 / R.st, hr = 0.5 / R.sr;
                lt[1] = q1t * ht;
                lr[1] = q1r * hr;
                lt[2] = (R.r[2] - lt[1] * lt[1]) * ht;
                lr[2] = (R.r[2] - lr[1] * lr[1]) * hr;
                lt[3] = -2.0 * lt[1] * lt[2] * ht;
                lr[3] = -2.0 * lr[1] * lr[2] * hr;
                lt[4] = -(2.0 * lt[1] * lt[3] + lt[2] * lt[2]) * ht;
                lr[4] = -(2.0 * lr[1] * lr[3] + lr[2] * lr[2]) * hr;
                for (int q = 0; q < 5; ++q) R.Lk[q] = lt[q] + lr[q];
                // thc = (fmc_c + mu/c tau)(L + shift) - mu / (2 c^2) L^2, degree 4
                const double fmcc = (A.rd.f0 + A.rd.slope * R.tc) / kC0;
                const double muc = A.rd.slope / kC0, mu2 = A.rd.slope / (2.0 * kC0 * kC0);
                for (int q = 0; q < 5; ++q) {
                    const double aq = R.Lk[q] + (q == 0 ? R.r[kRecLs] : 0.0);
                    const double aq1 = q > 0 ? R.Lk[q - 1] + (q == 1 ? R.r[kRecLs] : 0.0) : 0.0;
                    double sq = 0.0;
                    for (int i = 0; i <= q; ++i) sq += R.Lk[i] * R.Lk[q - i];
                    R.thk[q] = fmcc * aq + muc * aq1 - mu2 * sq;
                }
            }
        }
        __syncwarp();
        double mine[kRecEntries];
#pragma unroll
        for (int e = 0; e < kRecEntries; ++e) mine[e] = 0.0;
        float mine_f[9];
#pragma unroll
        for (int e = 0; e < 9; ++e) mine_f[e] = 0.f;
        unsigned int mask = __ballot_sync(0xffffffffu, valid);
        while (mask) {
            const int i = __ffs(mask) - 1;
            mask &= mask - 1;
            if constexpr (MX) {
                if (sU[warp][i].x.kind == kRouteF32) {   // uniform over the warp (record i)
                    float part[9];
                    adj_vertex_f32<S>(sU[warp][i].f, m0, K, muc2, inv_fs, gfr, gfi, part);
#pragma unroll
                    for (int e = 0; e < 9; ++e) {
                        const float tot = warp_sum_f(part[e]);
                        if (lane == i) mine_f[e] = tot;
                    }
                    continue;
                }
            }
            const Rec &R = sU[warp][i].x;
            const double *d = R.r + kRecD;
            bool mixed_done = false;
            if constexpr (MX) {
                if (R.kind == kRecVertex) {          // uniform over the warp (record i)
                    float fb[kRecD + 6];
                    adj_vertex_mixed<S>(R, m0, f0, mu, fs, c, gr, gi, fb);
#pragma unroll
                    for (int e = 0; e < kRecD + 6; ++e) {
                        const float tot = warp_sum_f(fb[e]);
                        if (lane == i) mine[e] = (double)tot;
                    }
                    mixed_done = true;
                }
            }
            if (!mixed_done) {
            double ab[kRecEntries];
#pragma unroll
            for (int e = 0; e < kRecEntries; ++e) ab[e] = 0.0;
            {
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
        }
        // the FP32 route: one reverse pass of the vertex-form record
        if (valid && f32) {
            const RecF &Fr = sU[warp][lane].f;
            const float twopi = 6.283185307179586f;
            float bar[10], gp[10];
            bar[0] = twopi * fmaf(Fr.it, mine_f[6], Fr.itd * mine_f[7]);
            bar[1] = twopi * fmaf(Fr.it, mine_f[7], Fr.itd * mine_f[8]);
            bar[2] = twopi * fmaf(Fr.ir, mine_f[6], Fr.ird * mine_f[7]);
            bar[3] = twopi * fmaf(Fr.ir, mine_f[7], Fr.ird * mine_f[8]);
#pragma unroll
            for (int v = 0; v < 3; ++v) {
                bar[4 + v] = twopi * Fr.w[v] * mine_f[3 + v];
                bar[7 + v] = mine_f[v];
            }
            const FacetRec fr = A.fac[k];
            const float4 vv = reinterpret_cast<const float4 *>(A.vel32)[fr.inst];
            const float vf[3] = {vv.x, vv.y, vv.z};
            vertex_reverse_f32(fr, vf, w.tn, w.ptx, w.prx, A.rd.intra, bar, gp);
#pragma unroll
            for (int p = 0; p < 10; ++p) atomicAdd(gfac + 10 * k + p, (double)gp[p]);
        }
        // reverse through the record construction, one parameter at a time
        if (valid && !f32) {
            const Rec &R = sU[warp][lane].x;
            double tri[9], c0[3];
            for (int q = 0; q < 9; ++q) tri[q] = A.tri64[9 * k + q];
            for (int r = 0; r < 3; ++r) c0[r] = A.c64[3 * k + r];
            const double rho = (double)A.fac[k].rho;
            const double *ref = A.rd.delay_ref ? A.ref64 + 3 * A.fac[k].inst : nullptr;
            const int two_sided = A.fac[k].two_sided;
            for (int p = 0; p < 10; ++p) {
                Dual dtri[9], dc0[3], out[kRecEntries];
                for (int e = 0; e < kRecEntries; ++e) out[e] = Dual(0.0, 0.0);
                for (int q = 0; q < 9; ++q) dtri[q] = Dual(tri[q], q == p ? 1.0 : 0.0);
                for (int r = 0; r < 3; ++r)
                    dc0[r] = Dual(c0[r], (p < 9 && p % 3 == r) ? 1.0 / 3.0 : 0.0);
                const Dual drho(rho, p == 9 ? 1.0 : 0.0);
                int flags = 0;
                const int kind = build_record<Dual>(dtri, dc0, vel, tn, ptx, prx, drho, A.rd.intra,
                                                    k0, kmax, ref ? kDelayRef : kDelayFacet,
                                                    ref, two_sided, out, &flags);
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

template <bool MX>
static void launch_adjoint(const SynthArgs &a, const void *grad, int grad_c64, double *gfac,
                           cudaStream_t s)
{
    const MixConsts K = mix_consts(a.rd);

    const int M = a.rd.M;
    int S = kAdjS;
    while (S > 1 && M % (32 * S) != 0) S >>= 1;
    const int W = M / (32 * S);
    cudaMemsetAsync(gfac, 0, (size_t)a.F * 10 * sizeof(double), s);
    // each row's facet list in NCH chunks: about four waves of resident
    // blocks (a row per warp alone leaves the GPU a fraction of a wave on a
    // single sedan: 1536 rows), at most one 32-facet batch per chunk
    const int64_t rows = (int64_t)a.VO * a.rd.N * W;
    static int sms = 0;
    if (sms <= 0) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (sms <= 0) sms = 1;
    }
    const int64_t target = 4 * (int64_t)sms * 3 * kAdjWarps;
    const int64_t maxb = std::max<int64_t>(1, (a.F + 31) / 32);
    const int NCH = (int)std::max<int64_t>(1, std::min<int64_t>(maxb, (target + rows - 1) / rows));
    const int64_t warps = rows * NCH;
    const unsigned int grid = (unsigned int)((warps + kAdjWarps - 1) / kAdjWarps);
    switch (S) {
    case 8: adjoint_fp64_kernel<8, MX><<<grid, kAdjWarps * 32, 0, s>>>(a, K, W, NCH, grad, grad_c64, gfac); break;
    case 4: adjoint_fp64_kernel<4, MX><<<grid, kAdjWarps * 32, 0, s>>>(a, K, W, NCH, grad, grad_c64, gfac); break;
    case 2: adjoint_fp64_kernel<2, MX><<<grid, kAdjWarps * 32, 0, s>>>(a, K, W, NCH, grad, grad_c64, gfac); break;
    default: adjoint_fp64_kernel<1, MX><<<grid, kAdjWarps * 32, 0, s>>>(a, K, W, NCH, grad, grad_c64, gfac); break;
    }
}

void launch_adjoint_fp64(const SynthArgs &a, const void *grad, int grad_c64, double *gfac,
                         cudaStream_t s)
{
    launch_adjoint<false>(a, grad, grad_c64, gfac, s);
}

void launch_adjoint_mixed(const SynthArgs &a, const void *grad, int grad_c64, double *gfac,
                          cudaStream_t s)
{
    launch_adjoint<true>(a, grad, grad_c64, gfac, s);
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
