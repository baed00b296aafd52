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
