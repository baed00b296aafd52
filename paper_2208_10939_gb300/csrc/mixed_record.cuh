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

// a + b = s + e exactly (Knuth's two-sum)
__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e)
{
    s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

// unit vector of d = sh + sl (|sl| ~ ulp(sh)) as double-float pairs: the
// norm's square in double-float, 1/sqrt by rsqrtf and one Newton step on
// its double-float residual h = 1 - |d|^2 r0^2 (|h| ~ 1e-7, so the step
// leaves ~h^2), then d r
__device__ __forceinline__ void df_unit(const float sh[3], const float sl[3], float uh[3],
                                        float ul[3])
{
    float p[3], pe = 0.f, cross = 0.f;
#pragma unroll
    for (int r = 0; r < 3; ++r) {
        p[r] = __fmul_rn(sh[r], sh[r]);
        pe += __fmaf_rn(sh[r], sh[r], -p[r]);
        cross += sh[r] * sl[r];
    }
    float q1, e1, qh, e2;
    two_sum(p[0], p[1], q1, e1);
    two_sum(q1, p[2], qh, e2);
    const float ql = (e1 + e2) + pe + 2.f * cross;
    const float r0 = rsqrtf(qh);
    const float y = __fmul_rn(r0, r0), yl = __fmaf_rn(r0, r0, -y);
    const float z = __fmul_rn(qh, y);
    const float zl = __fmaf_rn(qh, y, -z) + (qh * yl + ql * y);
    const float h = __fsub_rn(1.f, z) - zl;     // 1 - z exact: z is within 1e-6 of 1
    const float rl = 0.5f * r0 * h;
#pragma unroll
    for (int r = 0; r < 3; ++r) {
        uh[r] = __fmul_rn(sh[r], r0);
        ul[r] = __fmaf_rn(sh[r], r0, -uh[r]) + (sh[r] * rl + sl[r] * r0);
    }
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
    float f0c_lo;         // its rounding residue (f0 / c = f0c + f0c_lo in double-float)
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
    float ant_lo[kMaxAnt][3];   // rounding residues of ant
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
                                                  const MixRow &w, int k, float *R,
                                                  bool exact_u = false)
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
    // The origin o(t_n) = o0 + v t_n is never formed in FP32: at tens of
    // metres its rounding would repeat with the instance's per-chirp step
    // v T_c (the same for every facet of the instance, so coherent across
    // them: a Doppler spur).  Each direction is normalised from the
    // constant B = p - o0 and the small D = -v t_n instead.
    float th[3], rh[3], Rt, Rr;
    const float D[3] = {-vv.x * w.tn, -vv.y * w.tn, -vv.z * w.tn};
    float o0[3];
    if (A.rd.far_field) {
        const float4 rf = reinterpret_cast<const float4 *>(A.ref32)[fr.inst];
        o0[0] = rf.x; o0[1] = rf.y; o0[2] = rf.z;
    } else {
        o0[0] = fr.c[0]; o0[1] = fr.c[1]; o0[2] = fr.c[2];
    }
    {
        float Bt[3], Br[3];
#pragma unroll
        for (int r = 0; r < 3; ++r) {
            Bt[r] = w.ptx[r] - o0[r];
            Br[r] = w.prx[r] - o0[r];
        }
        const float dd = D[0] * D[0] + D[1] * D[1] + D[2] * D[2];
        const float qt = (Bt[0] * Bt[0] + Bt[1] * Bt[1] + Bt[2] * Bt[2]) +
                         fmaf(2.f, Bt[0] * D[0] + Bt[1] * D[1] + Bt[2] * D[2], dd);
        const float qr = (Br[0] * Br[0] + Br[1] * Br[1] + Br[2] * Br[2]) +
                         fmaf(2.f, Br[0] * D[0] + Br[1] * D[1] + Br[2] * D[2], dd);
        const float it = rsqrtf(qt), ir = rsqrtf(qr);
#pragma unroll
        for (int r = 0; r < 3; ++r) {
            th[r] = fmaf(Bt[r], it, D[r] * it);
            rh[r] = fmaf(Br[r], ir, D[r] * ir);
        }
        if (A.rd.far_field) {
            Rt = qt * it;
            Rr = qr * ir;
        } else {
            Rt = kt.w;
            Rr = kr.w;
        }
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
    // formed in double-float arithmetic (FP32 pairs, ~1e-12 relative) from
    // the FP32 centroid, offsets and antenna positions and their rounding
    // residues; the FP32 u_v remain for the weights and steps, which need
    // only relative accuracy.  u_v = b . dv_v with b = t + r the sum of the
    // unit vectors toward the antennas (dv_v lies in the facet plane, so
    // b's in-plane part gives the same product).
    float ul[3] = {0.f, 0.f, 0.f};
    // (exact_u: every facet, for the adjoint, whose vertex-sum cancellation
    // amplifies the FP32 rounding of f0 u / c)
    const bool large =
        exact_u || K.f0c * fmaxf(fmaxf(fabsf(u[0]), fabsf(u[1])), fabsf(u[2])) > 64.f;
    if (large) {
        const float *res = A.fac_lo + 12 * (int64_t)k;
        // the origin of the directions at the chirp start: the centroid,
        // or (far field) the instance origin
        float oh[3], ol[3];
        if (A.rd.far_field) {
            const float4 rf = reinterpret_cast<const float4 *>(A.ref32)[fr.inst];
            oh[0] = rf.x; oh[1] = rf.y; oh[2] = rf.z;
#pragma unroll
            for (int r = 0; r < 3; ++r)
                ol[r] = (float)(A.ref64[3 * fr.inst + r] - (double)oh[r]);
        } else {
#pragma unroll
            for (int r = 0; r < 3; ++r) {
                oh[r] = fr.c[r];
                ol[r] = res[r];
            }
        }
        const float vel[3] = {vv.x, vv.y, vv.z};
        float bh[3] = {0.f, 0.f, 0.f}, bl[3] = {0.f, 0.f, 0.f};
#pragma unroll
        for (int e = 0; e < 2; ++e) {
            const int ant = e == 0 ? w.ant_t : w.ant_r;
            float sh[3], sl[3];
#pragma unroll
            for (int r = 0; r < 3; ++r) {
                // antenna - origin - v t_n, as sh + sl
                float d1, e1, d2, e2;
                two_sum(K.ant[ant][r], -oh[r], d1, e1);
                two_sum(d1, -(vel[r] * w.tn), d2, e2);
                sh[r] = d2;
                sl[r] = (e1 + e2) + (K.ant_lo[ant][r] - ol[r]);
            }
            float th_[3], tl_[3];
            df_unit(sh, sl, th_, tl_);
#pragma unroll
            for (int r = 0; r < 3; ++r) {
                float s_, e_;
                two_sum(bh[r], th_[r], s_, e_);
                bh[r] = s_;
                bl[r] = bl[r] + tl_[r] + e_;
            }
        }
#pragma unroll
        for (int v = 0; v < 3; ++v) {
            float p[3], pe = 0.f;
#pragma unroll
            for (int r = 0; r < 3; ++r) {
                const float dh = fr.dv[3 * v + r], dl = res[3 + 3 * v + r];
                p[r] = __fmul_rn(bh[r], dh);
                pe += __fmaf_rn(bh[r], dh, -p[r]) + bh[r] * dl + bl[r] * dh;
            }
            float q, e1, uh_, e2;
            two_sum(p[0], p[1], q, e1);
            two_sum(q, p[2], uh_, e2);
            const float ulo = (e1 + e2) + pe;
            u[v] = uh_ + ulo;
            ul[v] = ulo - (u[v] - uh_);
        }
    }
    // frac(x0 - f0 u / c) for a u of the record (u + ul in double-float on
    // large facets; ul = 0 otherwise)
    auto vphase = [&](float x0, float uh, float ulo) -> float {
        if (!large) return red1(x0 - K.f0c * uh);
        float y = __fmul_rn(K.f0c, uh);
        const float yl = __fmaf_rn(K.f0c, uh, -y) + (K.f0c * ulo + K.f0c_lo * uh);
        y = __fsub_rn(y, rintf(y));               // exact
        return red1(__fsub_rn(x0, y) - yl);
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
            // the mid-edge projection in double-float: halving is exact
            float bs, be;
            two_sum(u[i], u[i1], bs, be);
            R[4 + 4 * i] = vphase(0.f, 0.5f * bs, 0.5f * (be + ul[i] + ul[i1]));
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
            R[v] = vphase(ph0c, ua, ul[v]);
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
    K.f0c_lo = (float)(f0 / c - (double)K.f0c);
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
        for (int r = 0; r < 3; ++r) {
            K.ant[a][r] = (float)rd.ant[a][r];
            K.ant_lo[a][r] = (float)(rd.ant[a][r] - (double)K.ant[a][r]);
        }
    return K;
}

}  // namespace bart
