// The mixed-precision per-(facet, channel, chirp) record shared by the
// direct echo-synthesis kernel (synth.cu) and the spectral one
// (spectral.cu): FP64 path-length Taylor rows evaluated in double-float
// arithmetic, reduced mod 1, and the facet-integral form's coefficients in
// FP32.  See synth.cu for the definitions.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <cmath>

#include "bart_internal.cuh"
#include "record_fp64.cuh"

namespace bart {

constexpr int kKinMaxDeg = 8;
constexpr int kKinRow = kKinMaxDeg + 1;    // float4 per antenna-facet row

// double-float helpers: values xh + xl with |xl| <= ulp(xh) / 2; every
// operation rounds once (explicit _rn intrinsics: no contraction)
__device__ __forceinline__ void df_horner_step(float &xh, float &xl, float t, float ch, float cl)
{
    // (xh + xl) t + (ch + cl)
    const float ph = __fmul_rn(xh, t);
    float pl = __fmaf_rn(xh, t, -ph);                // exact product error
    pl = __fmaf_rn(xl, t, pl);
    const float sh = __fadd_rn(ph, ch);              // two-sum of ph and ch
    const float bb = __fsub_rn(sh, ph);
    float sl = __fadd_rn(__fsub_rn(ph, __fsub_rn(sh, bb)), __fsub_rn(ch, bb));
    sl = __fadd_rn(sl, __fadd_rn(pl, cl));
    xh = __fadd_rn(sh, sl);                          // renormalise
    xl = __fsub_rn(sl, __fsub_rn(xh, sh));
}

// (x0, hi, lo, R) from the double-float cycles x0u = xh + xl and R:
// x0 = frac(x0u), hi + lo = frac(x0u mu / (fs f0)), hi a multiple of 2^-14
__device__ __forceinline__ float4 kin_finish(float xh, float xl, float R, float mfh, float mfl)
{
    // xh - floor(xh) is exact (Sterbenz), then + xl
    const float x0 = __fadd_rn(__fsub_rn(xh, floorf(xh)), xl);
    const float ph = __fmul_rn(xh, mfh);
    float pl = __fmaf_rn(xh, mfh, -ph);
    pl = __fmaf_rn(xh, mfl, pl);
    pl = __fmaf_rn(xl, mfh, pl);
    const float yh = __fadd_rn(ph, pl);
    const float yl = __fsub_rn(pl, __fsub_rn(yh, ph));
    const float x1h = __fsub_rn(yh, floorf(yh));
    float hi = __fmul_rn(rintf(__fmul_rn(x1h, 16384.f)), 1.f / 16384.f);
    const float lo = __fadd_rn(__fsub_rn(x1h, hi), yl);
    if (hi >= 1.f) hi -= 1.f;
    return make_float4(x0, hi, lo, R);
}

// a row without a convergent expansion: FP64 square root at slot s (far
// field: R + l / R)
__device__ __forceinline__ float4 kin_fallback(const double *__restrict__ quad, int s, double Tc,
                                               double f0c, double mu_f0)
{
    const double t = (double)s * Tc;
    double R = sqrt(quad[0] + t * (quad[1] + t * quad[2]));
    R += (quad[3] + t * quad[4]) / R;
    const double x0u = R * f0c;
    double x1 = x0u * mu_f0;
    x1 -= floor(x1);
    const double hi = rint(x1 * 16384.0) * (1.0 / 16384.0);
    return make_float4((float)(x0u - floor(x0u)), (float)hi, (float)(x1 - hi), (float)R);
}

// the TX and RX rows of one record at chirp slot s (tau = s - s_mid), in one
// Horner loop: each iteration loads the two rows' coefficients together
__device__ __forceinline__ void kin_eval2(const float4 *__restrict__ rt,
                                          const float4 *__restrict__ rr,
                                          const double *__restrict__ qt,
                                          const double *__restrict__ qr, int s, float tau,
                                          double Tc, double f0c, double mu_f0, float mfh,
                                          float mfl, float4 &kt, float4 &kr)
{
    const float4 t0 = rt[0], r0 = rr[0];
    const int dt = __float_as_int(t0.w), dr = __float_as_int(r0.w);
    const int D = max(dt, dr);
    float th = 0.f, tl = 0.f, tR = 0.f, rh = 0.f, rl = 0.f, rR = 0.f;
    if (D > 0) {
        const float4 ct = rt[D], cr = rr[D];   // zero above each row's own degree
        th = ct.x; tl = ct.y; tR = ct.z;
        rh = cr.x; rl = cr.y; rR = cr.z;
    }
#pragma unroll 2
    for (int j = D - 1; j >= 0; --j) {
        const float4 ct = j == 0 ? t0 : rt[j];
        const float4 cr = j == 0 ? r0 : rr[j];
        df_horner_step(th, tl, tau, ct.x, ct.y);
        tR = __fmaf_rn(tR, tau, ct.z);
        df_horner_step(rh, rl, tau, cr.x, cr.y);
        rR = __fmaf_rn(rR, tau, cr.z);
    }
    kt = dt < 0 ? kin_fallback(qt, s, Tc, f0c, mu_f0) : kin_finish(th, tl, tR, mfh, mfl);
    kr = dr < 0 ? kin_fallback(qr, s, Tc, f0c, mu_f0) : kin_finish(rh, rl, rR, mfh, mfl);
}

struct MixConsts {
    float f0c;            // f0 / c                    cycles per metre at f0
    float muc;            // mu / (fs c)               cycles per metre per sample
    float f0c_fs;         // f0 / (c fs)
    float mu_c2fs;        // mu / (c^2 fs)
    float half_f0c_fs2;   // f0 / (2 c fs^2)
    float mu_c_fs2;       // mu / (c fs^2)
    float mu_2c2;         // mu / (2 c^2)
    float k0, kmax;       // 2 pi f0 / c, 2 pi f_max / c
    float kap_step;       // mu / (fs f0): kappa_m = f_m / f0 = 1 + m kap_step
    float mfh, mfl;       // mu / (fs f0) as a double-float (high, low)
    double f0c_d, mu_f0_d;  // f0 / c and mu / (fs f0) in FP64 (fallback rows)
    float s_mid;          // middle chirp slot of the frame (expansion point)
    float out_scale;      // C (c / (2 pi f0))^2
    float tc;
    float ant[kMaxAnt][3];
};

// One record per (facet, channel, chirp), 24 words in shared memory; the
// layout depends on its form:
//   vertex (V): [0..2] ph0_v  [3..5] lo_v  [6..8] w_v  [9..11] step re
//               [12..14] step im  [15] hi  [16] p2  [17..19] 2 cos(2 step)
//               [20..22] 4 sin(2 step)
//   series (S): [0] ph0c [1] hi [2] loc [3] p2 [4] po [5] pl [6..13] cr [14..20] ci
//   edge (E):   [0] ph0c [1] hi [2] loc [3] p2 [4+4e] po [5+4e] pl [6+4e] G [7+4e] K
//               [16] sinc-series flags (int bits)
// Phases are in cycles.  ph0 is reduced to [-0.5, 0.5]; hi is a
// multiple of 2^-14 so that frac(hi m) is exact in FP32.
struct __align__(16) RecM {
    float f[24];
};

__device__ __forceinline__ float red1(float x) { return x - rintf(x); }

// The record of facet k for one chirp row (see RecM): kinematics rows
// evaluated at the row's chirp slot, directions, obliquity, amplitude, the
// in-plane projections u_v and the form's coefficients.  Returns the form.
struct MixRow {
    const float4 *kin_t, *kin_r;     // kinematics rows of the row's TX and RX
    const double *quad_t, *quad_r;   // their FP64 fallback data
    int sl;                          // chirp slot
    int ant_t, ant_r;                // antenna indices of the row's TX and RX
    float tau_s, tn;                 // slot offset from the expansion point; chirp start (s)
    float ptx[3], prx[3];            // antenna positions
};

__device__ __forceinline__ int build_mixed_record(const SynthArgs &A, const MixConsts &K,
                                                  const MixRow &w, int k, float *R)
{
    const FacetRec fr = A.fac[k];
    const float4 vv = reinterpret_cast<const float4 *>(A.vel32)[fr.inst];
    float4 kt, kr;
    kin_eval2(w.kin_t + (int64_t)k * kKinRow, w.kin_r + (int64_t)k * kKinRow,
              w.quad_t + kKinQuadWords * (int64_t)k, w.quad_r + kKinQuadWords * (int64_t)k,
              w.sl, w.tau_s, A.rd.Tc, K.f0c_d, K.mu_f0_d, K.mfh, K.mfl, kt, kr);
    // directions t, r and the amplitude's ranges: from the facet
    // centroid, or (far field) from the instance origin, whose
    // plane waves every facet of the instance sees
    float th[3], rh[3], Rt, Rr;
    if (A.rd.far_field) {
        const float4 rf = reinterpret_cast<const float4 *>(A.ref32)[fr.inst];
        const float ox = fmaf(vv.x, w.tn, rf.x), oy = fmaf(vv.y, w.tn, rf.y),
                    oz = fmaf(vv.z, w.tn, rf.z);
        th[0] = w.ptx[0] - ox; th[1] = w.ptx[1] - oy; th[2] = w.ptx[2] - oz;
        rh[0] = w.prx[0] - ox; rh[1] = w.prx[1] - oy; rh[2] = w.prx[2] - oz;
        Rt = sqrtf(th[0] * th[0] + th[1] * th[1] + th[2] * th[2]);
        Rr = sqrtf(rh[0] * rh[0] + rh[1] * rh[1] + rh[2] * rh[2]);
#pragma unroll
        for (int r = 0; r < 3; ++r) {
            th[r] /= Rt;
            rh[r] /= Rr;
        }
    } else {
        const float cx = fmaf(vv.x, w.tn, fr.c[0]);
        const float cy = fmaf(vv.y, w.tn, fr.c[1]);
        const float cz = fmaf(vv.z, w.tn, fr.c[2]);
        th[0] = w.ptx[0] - cx; th[1] = w.ptx[1] - cy; th[2] = w.ptx[2] - cz;
        rh[0] = w.prx[0] - cx; rh[1] = w.prx[1] - cy; rh[2] = w.prx[2] - cz;
        const float it = rsqrtf(th[0] * th[0] + th[1] * th[1] + th[2] * th[2]);
        const float ir = rsqrtf(rh[0] * rh[0] + rh[1] * rh[1] + rh[2] * rh[2]);
#pragma unroll
        for (int r = 0; r < 3; ++r) {
            th[r] *= it;
            rh[r] *= ir;
        }
        Rt = kt.w;
        Rr = kr.w;
    }
    float b[3];
#pragma unroll
    for (int r = 0; r < 3; ++r) b[r] = th[r] + rh[r];
    const float L = kt.w + kr.w;            // the facet's path at the chirp start
    float o_k = 0.5f * (fr.n[0] * b[0] + fr.n[1] * b[1] + fr.n[2] * b[2]);
    if (fr.two_sided) o_k = fabsf(o_k);    // the side both antennas light
    const float g = __fdividef(fr.rho * o_k, Rt * Rr);
    // in-plane part of b, formed once: u_v, |b_t|^2 and n x b_t all derive
    // from it, so every form evaluates J exactly at one wave vector
    // (|b|^2 - (b.n)^2 would cancel catastrophically near specular)
    const float bn = fr.n[0] * b[0] + fr.n[1] * b[1] + fr.n[2] * b[2];
    const float bt[3] = {b[0] - bn * fr.n[0], b[1] - bn * fr.n[1], b[2] - bn * fr.n[2]};
    float u[3];
#pragma unroll
    for (int v = 0; v < 3; ++v)
        u[v] = bt[0] * fr.dv[3 * v] + bt[1] * fr.dv[3 * v + 1] + bt[2] * fr.dv[3 * v + 2];
    // the delay's motion within the chirp and the residual video phase
    // follow the facet centroid, or (reference-point form) the
    // instance origin: path Lp, its first and second time derivatives
    // (far field: the origin's motion, the facet's plane-wave path)
    float Lp = L, Ld = 0.f, Ldd = 0.f;
    {
        float ut[3] = {th[0], th[1], th[2]}, ur[3] = {rh[0], rh[1], rh[2]};
        float Rtp = Rt, Rrp = Rr;
        if (A.rd.delay_ref) {
            const float4 rf = reinterpret_cast<const float4 *>(A.ref32)[fr.inst];
            const float ox = fmaf(vv.x, w.tn, rf.x), oy = fmaf(vv.y, w.tn, rf.y),
                        oz = fmaf(vv.z, w.tn, rf.z);
            float gt[3] = {w.ptx[0] - ox, w.ptx[1] - oy, w.ptx[2] - oz};
            float gr[3] = {w.prx[0] - ox, w.prx[1] - oy, w.prx[2] - oz};
            Rtp = sqrtf(gt[0] * gt[0] + gt[1] * gt[1] + gt[2] * gt[2]);
            Rrp = sqrtf(gr[0] * gr[0] + gr[1] * gr[1] + gr[2] * gr[2]);
            Lp = Rtp + Rrp;
#pragma unroll
            for (int r = 0; r < 3; ++r) {
                ut[r] = gt[r] / Rtp;
                ur[r] = gr[r] / Rrp;
            }
        }
        if (A.rd.intra) {
            const float v2 = vv.x * vv.x + vv.y * vv.y + vv.z * vv.z;
            const float vt = vv.x * ut[0] + vv.y * ut[1] + vv.z * ut[2];
            const float vr = vv.x * ur[0] + vv.y * ur[1] + vv.z * ur[2];
            Ld = -(vt + vr);
            Ldd = __fdividef(v2 - vt * vt, Rtp) + __fdividef(v2 - vr * vr, Rrp);
        }
    }
    float hi = kt.y + kr.y;
    hi = hi >= 1.f ? hi - 1.f : hi;
    const float loc = (kt.z + kr.z) + K.f0c_fs * Ld - K.mu_c2fs * Lp * Ld;
    const float p2 = K.half_f0c_fs2 * Ldd + K.mu_c_fs2 * Ld;
    const float ph0c = red1((kt.x + kr.x) - K.mu_2c2 * Lp * Lp);
    // Large facets (f0 |u_v| / c beyond 64 cycles, |u| over ~0.25 m): the
    // FP32 offsets, directions and the product f0 u / c would put ~1e-4 rad
    // into the vertex phases, so u_v and the phases derived from it are
    // formed in FP64 from the FP64 world vertices (the FP32 values remain
    // for the weights and steps, which need only relative accuracy).
    double ud[3];
    const bool large = K.f0c * fmaxf(fmaxf(fabsf(u[0]), fabsf(u[1])), fabsf(u[2])) > 64.f;
    if (large) {
        const double vx = A.vel64[3 * fr.inst], vy = A.vel64[3 * fr.inst + 1],
                     vz = A.vel64[3 * fr.inst + 2];
        const double tnd = (double)w.sl * A.rd.Tc;
        const double *c0 = A.c64 + 3 * (int64_t)k;
        const double c[3] = {c0[0] + vx * tnd, c0[1] + vy * tnd, c0[2] + vz * tnd};
        double from[3] = {c[0], c[1], c[2]};
        if (A.rd.far_field) {
            const double *r0 = A.ref64 + 3 * fr.inst;
            from[0] = r0[0] + vx * tnd;
            from[1] = r0[1] + vy * tnd;
            from[2] = r0[2] + vz * tnd;
        }
        const int tx = w.ant_t, rx = w.ant_r;
        double bd[3], dt[3], dr[3];
        for (int r = 0; r < 3; ++r) {
            dt[r] = A.rd.ant[tx][r] - from[r];
            dr[r] = A.rd.ant[rx][r] - from[r];
        }
        const double it = 1.0 / sqrt(dt[0] * dt[0] + dt[1] * dt[1] + dt[2] * dt[2]);
        const double ir = 1.0 / sqrt(dr[0] * dr[0] + dr[1] * dr[1] + dr[2] * dr[2]);
        for (int r = 0; r < 3; ++r) bd[r] = dt[r] * it + dr[r] * ir;
        const double *tv = A.tri64 + 9 * (int64_t)k;
        const double e1[3] = {tv[3] - tv[0], tv[4] - tv[1], tv[5] - tv[2]};
        const double e2[3] = {tv[6] - tv[0], tv[7] - tv[1], tv[8] - tv[2]};
        double nd[3] = {e1[1] * e2[2] - e1[2] * e2[1], e1[2] * e2[0] - e1[0] * e2[2],
                        e1[0] * e2[1] - e1[1] * e2[0]};
        const double in = 1.0 / sqrt(nd[0] * nd[0] + nd[1] * nd[1] + nd[2] * nd[2]);
        const double bn = (bd[0] * nd[0] + bd[1] * nd[1] + bd[2] * nd[2]) * in * in;
        for (int r = 0; r < 3; ++r) bd[r] -= bn * nd[r];
        for (int v = 0; v < 3; ++v) {
            ud[v] = bd[0] * (tv[3 * v] - c0[0]) + bd[1] * (tv[3 * v + 1] - c0[1]) +
                    bd[2] * (tv[3 * v + 2] - c0[2]);
            u[v] = (float)ud[v];
        }
    }
    // frac(x0 - f0 u / c) for a u of the record: FP64 on large facets
    auto vphase = [&](float x0, float uf, double udv) -> float {
        if (!large) return red1(x0 - K.f0c * uf);
        const double y = (double)x0 - K.f0c_d * udv;
        return (float)(y - rint(y));
    };
    const float umin = fminf(fminf(u[0], u[1]), u[2]);
    const float umax = fmaxf(fmaxf(u[0], u[1]), u[2]);
    const float dmin = fminf(fminf(fabsf(u[0] - u[1]), fabsf(u[1] - u[2])),
                             fabsf(u[0] - u[2]));
    const float A2 = 2.f * fr.area * g;
    if (K.kmax * (umax - umin) < (float)kSeriesKD) {
        R[0] = ph0c;
        R[1] = hi;
        R[2] = loc;
        R[3] = p2;
        const float ub = (u[0] + u[1] + u[2]) * (1.f / 3.f);
        R[4] = red1(-K.f0c * ub);
        R[5] = -K.muc * ub;
        const float y0 = K.k0 * (u[0] - ub), y1 = K.k0 * (u[1] - ub),
                    y2 = K.k0 * (u[2] - ub);
        const float e2 = y0 * y1 + y0 * y2 + y1 * y2, e3 = y0 * y1 * y2;
        float h[kSeriesTerms];
        h[0] = 1.f;
        h[1] = 0.f;
        h[2] = -e2;
#pragma unroll
        for (int p = 3; p < kSeriesTerms; ++p) h[p] = -e2 * h[p - 2] + e3 * h[p - 3];
        const float sc = A2 * K.k0 * K.k0;
#pragma unroll
        for (int i = 0; i < 8; ++i)
            R[6 + i] = ((i & 1) ? -sc : sc) * h[2 * i] * (float)c_inv_fact[2 * i + 2];
#pragma unroll
        for (int i = 0; i < 7; ++i)
            R[14 + i] = ((i & 1) ? sc : -sc) * h[2 * i + 1] * (float)c_inv_fact[2 * i + 3];
        return kRecSeries;
    } else if (K.kmax * dmin < (float)kEdgeKd) {
        R[0] = ph0c;
        R[1] = hi;
        R[2] = loc;
        R[3] = p2;
        const float bt2 = bt[0] * bt[0] + bt[1] * bt[1] + bt[2] * bt[2];
        const float nxb[3] = {fr.n[1] * bt[2] - fr.n[2] * bt[1],
                              fr.n[2] * bt[0] - fr.n[0] * bt[2],
                              fr.n[0] * bt[1] - fr.n[1] * bt[0]};
        int flags = 0;
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            const int i1 = (i + 1) % 3;
            const float e[3] = {fr.dv[3 * i1] - fr.dv[3 * i],
                                fr.dv[3 * i1 + 1] - fr.dv[3 * i + 1],
                                fr.dv[3 * i1 + 2] - fr.dv[3 * i + 2]};
            const float beta = 0.5f * (u[i] + u[i1]);
            const float gam = 0.5f * (u[i1] - u[i]);
            const float ci = (e[0] * nxb[0] + e[1] * nxb[1] + e[2] * nxb[2]) / bt2;
            R[4 + 4 * i] = vphase(0.f, beta, 0.5 * (ud[i] + ud[i1]));
            R[5 + 4 * i] = -K.muc * beta;
            R[6 + 4 * i] = K.k0 * gam;
            R[7 + 4 * i] = K.k0 * ci * g;
            if (K.kmax * fabsf(gam) < (float)kSincSeries) flags |= 1 << i;
        }
        R[16] = __int_as_float(flags);
        return kRecEdge;
    } else {
        R[15] = hi;
        R[16] = p2;
        // vertex steps = the centroid's step times e^{j x_v},
        // x_v = -2 pi mu/(fs c) u_v, from its Taylor series (error
        // below x^6/720 = 1.4e-9 for |x| < 0.1), else sincospi
        float sc_, cc_;
        sincospif(2.f * red1(hi + loc), &sc_, &cc_);
#pragma unroll
        for (int v = 0; v < 3; ++v) {
            const float ua = u[v], ub_ = u[(v + 1) % 3], uc = u[(v + 2) % 3];
            R[v] = vphase(ph0c, ua, ud[v]);
            const float lo = loc - K.muc * ua;
            R[3 + v] = lo;
            R[6 + v] = __fdividef(-A2, (ua - ub_) * (ua - uc));
            float s_, c_;
            const float x = -6.283185307179586f * K.muc * ua;
            if (fabsf(x) < 0.1f) {
                const float x2 = x * x;
                const float cx = fmaf(x2, fmaf(x2, 1.f / 24.f, -0.5f), 1.f);
                const float sx = x * fmaf(x2, fmaf(x2, 1.f / 120.f, -1.f / 6.f), 1.f);
                c_ = fmaf(cc_, cx, -sc_ * sx);
                s_ = fmaf(sc_, cx, cc_ * sx);
            } else {
                sincospif(2.f * red1(hi + lo), &s_, &c_);
            }
            R[9 + v] = c_;
            R[12 + v] = s_;
            // 2 cos(2 step) = 2 - 4 sin^2 = 4 cos^2 - 2, taken from the
            // smaller of sin and cos so that only its own rounding remains
            // (the recurrence is most sensitive to it near angle 0 and pi)
            R[17 + v] = fabsf(s_) < fabsf(c_) ? fmaf(-4.f * s_, s_, 2.f)
                                              : fmaf(4.f * c_, c_, -2.f);
            R[20 + v] = 8.f * c_ * s_;                // 4 sin(2 step)
        }
    }
    return kRecVertex;
}

// The term of a series- or edge-form record (see RecM) at fast-time sample
// m: the facet integral's k-dependence evaluated per sample, times the
// phasor of the record's phase (Eq. 13); unscaled (times C / k_m^2 later).
__device__ __forceinline__ void series_edge_term(const float *R, bool series, float fm,
                                                 const MixConsts &K, float &dr, float &di)
{
    const float thc = fmaf(R[3], fm * fm, fmaf(R[2], fm, R[0] + red1(R[1] * fm)));
    const float kp = fmaf(fm, K.kap_step, 1.f);
    dr = 0.f;
    di = 0.f;
    if (series) {
        const float th = red1(thc + fmaf(R[5], fm, R[4]));
        float zs, zc;
        __sincosf(6.283185307179586f * th, &zs, &zc);
        const float k2 = kp * kp;
        float a = R[13], bb = R[20];
#pragma unroll
        for (int q = 6; q >= 0; --q) a = fmaf(a, k2, R[6 + q]);
#pragma unroll
        for (int q = 5; q >= 0; --q) bb = fmaf(bb, k2, R[14 + q]);
        const float re = a * k2, im = bb * k2 * kp;
        dr = zc * re - zs * im;
        di = zc * im + zs * re;
    } else {
        const int flags = __float_as_int(R[16]);
#pragma unroll
        for (int e = 0; e < 3; ++e) {
            const float th = red1(thc + fmaf(R[5 + 4 * e], fm, R[4 + 4 * e]));
            float zs, zc;
            __sincosf(6.283185307179586f * th, &zs, &zc);
            const float x = kp * R[6 + 4 * e];
            float sn;
            if (flags & (1 << e)) {
                const float x2 = x * x;
                sn = fmaf(x2, fmaf(x2, fmaf(x2, fmaf(x2, 1.f / 362880.f, -1.f / 5040.f),
                                            1.f / 120.f), -1.f / 6.f), 1.f);
            } else {
                sn = sinf(x) / x;   // accurate sinf: |x| may reach ~1e3
            }
            const float coef = kp * R[7 + 4 * e] * sn;
            dr = fmaf(-coef, zs, dr);
            di = fmaf(coef, zc, di);
        }
    }
}

inline MixConsts mix_consts(const RadarDev &rd)
{
    MixConsts K;
    const double c = kC0, fs = rd.fs, mu = rd.slope, f0 = rd.f0;
    const double f_max = f0 + mu * (rd.M - 1) / fs;
    K.f0c = (float)(f0 / c);
    K.muc = (float)(mu / (fs * c));
    K.f0c_fs = (float)(f0 / (c * fs));
    K.mu_c2fs = (float)(mu / (c * c * fs));
    K.half_f0c_fs2 = (float)(0.5 * f0 / (c * fs * fs));
    K.mu_c_fs2 = (float)(mu / (c * fs * fs));
    K.mu_2c2 = (float)(mu / (2.0 * c * c));
    K.k0 = (float)(2.0 * kPi * f0 / c);
    K.kmax = (float)(2.0 * kPi * f_max / c);
    K.kap_step = (float)(mu / (fs * f0));
    K.mu_f0_d = mu / (fs * f0);
    K.f0c_d = f0 / c;
    K.mfh = (float)K.mu_f0_d;
    K.mfl = (float)(K.mu_f0_d - (double)K.mfh);
    K.s_mid = (float)(0.5 * (double)(rd.N * rd.slots - 1));
    const double camp = 2.0 * sqrt(kPi) / pow(4.0 * kPi, 1.5);
    const double lk = c / (2.0 * kPi * f0);
    K.out_scale = (float)(camp * lk * lk);
    K.tc = (float)rd.Tc;
    for (int a = 0; a < kMaxAnt; ++a)
        for (int r = 0; r < 3; ++r) K.ant[a][r] = (float)rd.ant[a][r];
    return K;
}

}  // namespace bart
