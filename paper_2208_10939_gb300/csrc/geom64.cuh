// FP64 geometry shared by the visibility and double-bounce kernels: vector
// steps with one IEEE rounding per operation in a fixed order (explicit
// __d*_rn intrinsics, no FMA contraction), so that their decisions are
// reproducible bit for bit by any IEEE-754 implementation of the same
// steps; the Moller-Trumbore (1997) segment/triangle test; the slab test of
// a segment against an FP32 box (boxes rounded outward and padded, so the
// test never drops a candidate).
#pragma once

#include <cuda_runtime.h>

#include "bart_internal.cuh"

namespace bart {

constexpr int kStack = 64;   // BVH traversal stack depth

__device__ __forceinline__ void sub3(const double *a, const double *b, double *o)
{
    o[0] = __dsub_rn(a[0], b[0]);
    o[1] = __dsub_rn(a[1], b[1]);
    o[2] = __dsub_rn(a[2], b[2]);
}
__device__ __forceinline__ double dot3(const double *a, const double *b)
{
    double s = __dmul_rn(a[0], b[0]);
    s = __dadd_rn(s, __dmul_rn(a[1], b[1]));
    s = __dadd_rn(s, __dmul_rn(a[2], b[2]));
    return s;
}
__device__ __forceinline__ void cross3(const double *a, const double *b, double *o)
{
    o[0] = __dsub_rn(__dmul_rn(a[1], b[2]), __dmul_rn(a[2], b[1]));
    o[1] = __dsub_rn(__dmul_rn(a[2], b[0]), __dmul_rn(a[0], b[2]));
    o[2] = __dsub_rn(__dmul_rn(a[0], b[1]), __dmul_rn(a[1], b[0]));
}

// 2 = hit with margin, 1 = grazing (inside the margins), 0 = miss
__device__ __forceinline__ int mt_segment(const double *O, const double *D, const double *tri)
{
    double e1[3], e2[3], P[3], T[3], Qv[3];
    sub3(tri + 3, tri, e1);
    sub3(tri + 6, tri, e2);
    cross3(D, e2, P);
    const double det = dot3(e1, P);
    if (det == 0.0) return 0;
    const double inv = __ddiv_rn(1.0, det);
    sub3(O, tri, T);
    const double u = __dmul_rn(dot3(T, P), inv);
    if (u < -kEpsB || u > __dadd_rn(1.0, kEpsB)) return 0;
    cross3(T, e1, Qv);
    const double v = __dmul_rn(dot3(D, Qv), inv);
    const double uv = __dadd_rn(u, v);
    if (v < -kEpsB || uv > __dadd_rn(1.0, kEpsB)) return 0;
    const double t = __dmul_rn(dot3(e2, Qv), inv);
    if (t < -kEpsT || t > __dadd_rn(1.0, kEpsT)) return 0;
    if (u >= kEpsB && v >= kEpsB && uv <= __dsub_rn(1.0, kEpsB) && t >= kEpsT &&
        t <= __dsub_rn(1.0, kEpsT))
        return 2;
    return 1;
}

// FP32 pre-test of the FP64 test above: 0 when it certainly returns 0 (a
// miss), 2 when it certainly returns 2 (a hit inside every margin), 1 when
// undecided (the FP64 test then runs).
// tri: FP32 vertices (rounded from the FP64 ones) + X = max |coordinate|;
// O, D: the segment rounded to FP32, Dm = max |D_i|, Om = max |O_i|.
// Every FP32 quantity carries a first-order bound on its distance to the
// exact value (inputs rounded: |dx| <= 2^-24 |x|; each operation rounds);
// a miss is certain when u, v, u + v or t lie beyond [0, 1] by more than
// twice that bound plus 1e-6, a hit when all of them lie inside (0, 1) by
// more than twice the bound plus 1e-6 (the FP64 test's margins are 1e-9,
// its own rounding error is < 2^-29 of the FP32 bound, which is capped at
// 100).
__device__ __forceinline__ int mt_fp32_classify(const float4 t0, const float4 t1,
                                                const float4 t2, const float *O,
                                                const float *D, float Dm, float Om)
{
    constexpr float u = 5.9604645e-8f;   // 2^-24
    const float v0[3] = {t0.x, t0.y, t0.z}, v1[3] = {t0.w, t1.x, t1.y},
                v2[3] = {t1.z, t1.w, t2.x};
    const float X = fmaxf(t2.y, Om) * 1.000001f;
    const float ein = 4.f * u * X;       // error of each component of e1, e2, T
    float e1[3], e2[3], T[3];
#pragma unroll
    for (int r = 0; r < 3; ++r) {
        e1[r] = v1[r] - v0[r];
        e2[r] = v2[r] - v0[r];
        T[r] = O[r] - v0[r];
    }
    const float e1m = fmaxf(fmaxf(fabsf(e1[0]), fabsf(e1[1])), fabsf(e1[2])) + ein;
    const float e2m = fmaxf(fmaxf(fabsf(e2[0]), fabsf(e2[1])), fabsf(e2[2])) + ein;
    const float Tm = fmaxf(fmaxf(fabsf(T[0]), fabsf(T[1])), fabsf(T[2])) + ein;
    const float P[3] = {D[1] * e2[2] - D[2] * e2[1], D[2] * e2[0] - D[0] * e2[2],
                        D[0] * e2[1] - D[1] * e2[0]};
    const float dP = Dm * (2.f * ein + 6.f * u * e2m);
    const float Pm = fmaxf(fmaxf(fabsf(P[0]), fabsf(P[1])), fabsf(P[2])) + dP;
    const float det = e1[0] * P[0] + e1[1] * P[1] + e1[2] * P[2];
    const float dDet = 3.f * (ein * Pm + e1m * dP) + 9.f * u * e1m * Pm;
    const float adet = fabsf(det);
    if (adet <= 4.f * dDet) return 1;
    const float den = adet - dDet;
    const float nu = T[0] * P[0] + T[1] * P[1] + T[2] * P[2];
    const float dNu = 3.f * (ein * Pm + Tm * dP) + 9.f * u * Tm * Pm;
    const float uu = nu / det;
    const float Bu = 2.f * ((dNu + fabsf(uu) * dDet) / den + 2.f * u * fabsf(uu));
    if (Bu > 100.f) return 1;
    if (uu + Bu < -1e-6f || uu - Bu > 1.f + 1e-6f) return 0;
    const float Qv[3] = {T[1] * e1[2] - T[2] * e1[1], T[2] * e1[0] - T[0] * e1[2],
                         T[0] * e1[1] - T[1] * e1[0]};
    const float dQ = 2.f * ein * (e1m + Tm) + 6.f * u * Tm * e1m;
    const float Qm = fmaxf(fmaxf(fabsf(Qv[0]), fabsf(Qv[1])), fabsf(Qv[2])) + dQ;
    const float nv = D[0] * Qv[0] + D[1] * Qv[1] + D[2] * Qv[2];
    const float dNv = 3.f * (u * Dm * Qm + Dm * dQ) + 9.f * u * Dm * Qm;
    const float vv = nv / det;
    const float Bv = 2.f * ((dNv + fabsf(vv) * dDet) / den + 2.f * u * fabsf(vv));
    if (Bv > 100.f) return 1;
    if (vv + Bv < -1e-6f || uu + vv - Bu - Bv > 1.f + 1e-6f) return 0;
    const float nt = e2[0] * Qv[0] + e2[1] * Qv[1] + e2[2] * Qv[2];
    const float dNt = 3.f * (ein * Qm + e2m * dQ) + 9.f * u * e2m * Qm;
    const float tt = nt / det;
    const float Bt = 2.f * ((dNt + fabsf(tt) * dDet) / den + 2.f * u * fabsf(tt));
    if (Bt > 100.f) return 1;
    if (tt + Bt < -1e-6f || tt - Bt > 1.f + 1e-6f) return 0;
    const bool inside = uu - Bu > 1e-6f && vv - Bv > 1e-6f && uu + vv + Bu + Bv < 1.f - 1e-6f &&
                        tt - Bt > 1e-6f && tt + Bt < 1.f - 1e-6f;
    return inside ? 2 : 1;
}

__device__ __forceinline__ bool slab_hit(const float *bmin, const float *bmax, const float *o,
                                         const float *inv)
{
    float tn = -1e-3f, tf = 1.0f + 1e-3f;
#pragma unroll
    for (int r = 0; r < 3; ++r) {
        const float t0 = (bmin[r] - o[r]) * inv[r];
        const float t1 = (bmax[r] - o[r]) * inv[r];
        tn = fmaxf(tn, fminf(t0, t1));
        tf = fminf(tf, fmaxf(t0, t1));
    }
    return tn <= tf;
}

}  // namespace bart
