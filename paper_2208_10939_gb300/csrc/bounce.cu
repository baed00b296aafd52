// Double-bounce paths (Sec. 2.2: the forward ray from a TX and the backward
// ray from an RX joined through two facets).  The paper names such paths
// but gives no formula; the reading implemented here is geometric optics at
// the first facet a and physical optics at the second facet b:
//
//  * a is lit from TX p (single-bounce state LIT or LIT_REV, side s_a);
//    beyond a, the reflected field is that of the image source
//    p' = p - 2 ((p - x0_a).n_a / |n_a|^2) n_a, confined to the beam of rays
//    from p' through the triangle a;
//  * Pi_ab = b clipped by a's front half-space (s_a n_a.(x - x0_a) >= 0) and
//    the three planes through p' and a's edges (each keeping a's third
//    vertex) is the part of b that the reflection lights; b must face p'
//    (cos >= eps_face; <= -eps_face on a two-sided b, side s_b = -1);
//  * the a -> b leg, from the specular point s (where the line p' -> c_Pi
//    meets a's plane; c_Pi the mean of Pi's vertices) to c_Pi, must not hit
//    or graze any facet other than a and b (the Moller-Trumbore test and
//    margins of the single-bounce visibility);
//  * Pi_ab is split into the fan (Pi_0, Pi_i, Pi_i+1) without clip slivers
//    (|cross| <= 1e-6 |n_b|); each piece is a virtual facet that scatters
//    toward RX q like a single-bounce facet, with the TX replaced by p' and
//    the reflectivity by -rho_a rho_b, when b is seen from RX q on side s_b;
//  * pairs, clips and the leg are decided on the frame-start geometry; a
//    virtual facet then moves with b, and p' with a's plane:
//    p'(t) = p'_0 + u t, u = 2 (v_a.n_a / |n_a|^2) n_a.
//
// Discovery, in two passes of count / scan / fill: one thread per (TX,
// facet a lit from it, LBVH subtree) casts a's beam through the subtree and
// lists the facets b facing the image in boxes that meet the beam (FP32
// culling with a rounding margin); one thread per candidate then clips b,
// drops slivers and casts the leg's segment.  Every decision takes one IEEE
// rounding per operation in a fixed order (geom64.cuh), so the virtual
// facets are reproducible bit for bit, in (TX, a, subtree, traversal, fan)
// order.  Synthesis: one warp per (channel, chirp, sample segment) adds into
// the cube the single-bounce synthesis wrote; the FP64 path evaluates the
// FP64 path's record forms sample by sample (the TX leg with its own
// quadratic in fast time), the mixed and spectral paths build each record
// from per-frame slow-time rows of the virtual facet's legs and evaluate it
// with FP32 phasors.
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <climits>

#include "bart_internal.cuh"
#include "bounce.cuh"
#include "geom64.cuh"
#include "record_fp64.cuh"

namespace bart {

namespace {

constexpr int kDbMaxV = 7;          // a triangle clipped by four half-spaces

// the middle chirp slot's start time (the rows' expansion point)
__host__ __device__ inline double bounce_mid_time(const RadarDev &rd)
{
    return 0.5 * (double)(rd.N * rd.slots - 1) * rd.Tc;
}
constexpr double kDbSliver = 1e-6;  // fan pieces with |cross| <= this |n_b| are dropped

__device__ __forceinline__ void centroid3(const double *t, double *c)
{
    for (int r = 0; r < 3; ++r)
        c[r] = __ddiv_rn(__dadd_rn(__dadd_rn(t[r], t[3 + r]), t[6 + r]), 3.0);
}

// Sutherland-Hodgman step: the part of the convex polygon with
// g.(x - base) >= 0
__device__ int clip_keep(const double *in, int n, const double *g, const double *base,
                         double *out)
{
    int k = 0;
    for (int i = 0; i < n; ++i) {
        const double *P = in + 3 * i, *Q = in + 3 * ((i + 1) % n);
        double d[3];
        sub3(P, base, d);
        const double fP = dot3(g, d);
        sub3(Q, base, d);
        const double fQ = dot3(g, d);
        if (fP >= 0.0) {
            for (int r = 0; r < 3; ++r) out[3 * k + r] = P[r];
            ++k;
        }
        if ((fP >= 0.0) != (fQ >= 0.0)) {
            const double t = __ddiv_rn(fP, __dsub_rn(fP, fQ));
            for (int r = 0; r < 3; ++r)
                out[3 * k + r] = __dadd_rn(P[r], __dmul_rn(t, __dsub_rn(Q[r], P[r])));
            ++k;
        }
    }
    return k;
}

// The beam of a from the image source img: a's front half-space and the
// three planes through img and a's edges, as (g, base) pairs
__device__ void beam_planes(const double *ta, int side_a, const double *img, double *g,
                            double *base)
{
    double e1[3], e2[3], n[3];
    sub3(ta + 3, ta, e1);
    sub3(ta + 6, ta, e2);
    cross3(e1, e2, n);
    for (int r = 0; r < 3; ++r) {
        g[r] = side_a > 0 ? n[r] : -n[r];
        base[r] = ta[r];
    }
    for (int i = 0; i < 3; ++i) {
        const double *xi = ta + 3 * i, *xj = ta + 3 * ((i + 1) % 3), *xk = ta + 3 * ((i + 2) % 3);
        double u[3], v[3], m[3], d[3];
        sub3(xi, img, u);
        sub3(xj, img, v);
        cross3(u, v, m);
        sub3(xk, img, d);
        const bool flip = dot3(m, d) < 0.0;
        for (int r = 0; r < 3; ++r) {
            g[3 * (i + 1) + r] = flip ? -m[r] : m[r];
            base[3 * (i + 1) + r] = img[r];
        }
    }
}

// The beam's four half-spaces rounded to FP32 for the traversal's box
// culling, each with the size sum_r |g_r| that scales its margin
struct Beam32 {
    float g[12], base[12], gs[4];
};

__device__ __forceinline__ void beam_to_f32(const double *g, const double *base, Beam32 &b)
{
    for (int i = 0; i < 12; ++i) {
        b.g[i] = (float)g[i];
        b.base[i] = (float)base[i];
    }
    for (int h = 0; h < 4; ++h)
        b.gs[h] = fabsf(b.g[3 * h]) + fabsf(b.g[3 * h + 1]) + fabsf(b.g[3 * h + 2]);
}

// box_meets_beam in FP32: a box is skipped only when its farthest corner
// lies outside a half-space by more than 1e-5 sum_r |g_r| (|x_r| + |base_r|),
// which covers the FP32 rounding of g, base and the sum (a few 1e-7 of that
// size) and the FP64 test's own margin with room to spare
__device__ __forceinline__ bool box_meets_beam32(const float *bmin, const float *bmax,
                                                 const Beam32 &B)
{
#pragma unroll
    for (int h = 0; h < 4; ++h) {
        const float *gh = B.g + 3 * h, *bh = B.base + 3 * h;
        float f = 0.f, scale = 1.f;
#pragma unroll
        for (int r = 0; r < 3; ++r) {
            const float x = gh[r] >= 0.f ? bmax[r] : bmin[r];
            f = fmaf(gh[r], x - bh[r], f);
            scale = fmaxf(scale, fabsf(x) + fabsf(bh[r]));
        }
        if (f < -1e-5f * B.gs[h] * scale) return false;
    }
    return true;
}

// a's image of TX p and its velocity (the mirror moving with a's plane),
// a's normal (|n_a|^2 = nn)
__device__ __forceinline__ void image_of(const double *ta, const double *pt, const double *va,
                                         double *na, double &nn, double *img, double *u)
{
    double e1[3], e2[3], d[3];
    sub3(ta + 3, ta, e1);
    sub3(ta + 6, ta, e2);
    cross3(e1, e2, na);
    nn = dot3(na, na);
    sub3(pt, ta, d);
    const double sc = __ddiv_rn(__dmul_rn(2.0, dot3(d, na)), nn);
    for (int r = 0; r < 3; ++r) img[r] = __dsub_rn(pt[r], __dmul_rn(sc, na[r]));
    const double su = __ddiv_rn(__dmul_rn(2.0, dot3(va, na)), nn);
    for (int r = 0; r < 3; ++r) u[r] = __dmul_rn(su, na[r]);
}

// facing_image's decision when FP32 makes it certain, else 2: FP32 from
// the rounded unit normal and centroid of the facet record, whose errors
// (~1e-7 in the normal, ~1e-7 relative in the centroid, so ~2e-6 / |D| in
// the direction) stay far inside the margin; slivers always take the FP64
// test
__device__ __forceinline__ int facing_image32(const FacetRec &fr, const double *img,
                                              double eps_face)
{
    float L2 = 0.f;
#pragma unroll
    for (int v = 0; v < 3; ++v) {
        const float x = fr.dv[3 * v], y = fr.dv[3 * v + 1], z = fr.dv[3 * v + 2];
        L2 = fmaxf(L2, fmaf(x, x, fmaf(y, y, z * z)));
    }
    if (2.f * fr.area < 4e-6f * L2) return 2;
    const float D[3] = {(float)img[0] - fr.c[0], (float)img[1] - fr.c[1], (float)img[2] - fr.c[2]};
    const float dd = fmaf(D[0], D[0], fmaf(D[1], D[1], D[2] * D[2]));
    if (!(dd > 0.f)) return 2;
    const float inv = rsqrtf(dd);
    const float cs = fmaf(fr.n[0], D[0], fmaf(fr.n[1], D[1], fr.n[2] * D[2])) * inv;
    const float scale = fmaxf(fmaxf(fabsf(fr.c[0]), fabsf(fr.c[1])), fabsf(fr.c[2])) +
                        fmaxf(fmaxf(fabsf((float)img[0]), fabsf((float)img[1])),
                              fabsf((float)img[2]));
    const float m = 2e-5f + 4e-7f * scale * inv;
    const float e = (float)eps_face;
    if (cs >= e + m) return 1;
    if (cs <= -e - m) return fr.two_sided ? -1 : 0;
    if (fabsf(cs) <= e - m) return 0;
    return 2;
}

// the side of b that faces the image (+1 front, -1 reverse of a two-sided
// b), 0 when it does not face it beyond eps_face
__device__ __forceinline__ int facing_image(const double *tb, const double *img, bool two_sided,
                                            double eps_face, double *nbb_out)
{
    double f1[3], f2[3], nb[3], cb[3], D[3];
    sub3(tb + 3, tb, f1);
    sub3(tb + 6, tb, f2);
    cross3(f1, f2, nb);
    const double nbb = dot3(nb, nb);
    *nbb_out = nbb;
    if (nbb == 0.0) return 0;
    centroid3(tb, cb);
    sub3(img, cb, D);
    const double cosang =
        __ddiv_rn(dot3(nb, D), __dmul_rn(__dsqrt_rn(nbb), __dsqrt_rn(dot3(D, D))));
    if (cosang >= eps_face) return 1;
    if (two_sided && cosang <= -eps_face) return -1;
    return 0;
}

// Pi = tb clipped by the beam; returns its vertex count and the fan pieces
// kept (bit q: piece (Pi_0, Pi_q, Pi_q+1) is not a sliver)
__device__ __forceinline__ int clip_to_beam(const double *tb, const double *g, const double *base,
                                            double nbb, double *poly, unsigned *keep)
{
    double buf[3 * kDbMaxV];
    int K = 3;
    for (int q = 0; q < 9; ++q) poly[q] = tb[q];
    for (int h = 0; h < 4 && K >= 3; ++h) {
        K = clip_keep(poly, K, g + 3 * h, base + 3 * h, buf);
        for (int q = 0; q < 3 * K; ++q) poly[q] = buf[q];
    }
    *keep = 0;
    if (K < 3) return K;
    const double thr = __dmul_rn(kDbSliver, __dsqrt_rn(nbb));
    for (int q = 1; q + 1 < K; ++q) {
        double x1[3], x2[3], cr[3];
        sub3(poly + 3 * q, poly, x1);
        sub3(poly + 3 * (q + 1), poly, x2);
        cross3(x1, x2, cr);
        if (__dsqrt_rn(dot3(cr, cr)) > thr) *keep |= 1u << q;
    }
    return K;
}

// whether the a -> b leg (specular point on a's plane -> mean of Pi's
// vertices) hits or grazes a facet other than a and b
__device__ bool leg_blocked(const double *poly, int K, const double *ta, const double *na,
                            const double *img, const double *__restrict__ tri64,
                            const float4 *__restrict__ tri32, const BvhNode *__restrict__ nodes,
                            int64_t a, int64_t b, int *status)
{
    double cp[3] = {0.0, 0.0, 0.0}, spt[3], Dl[3], t1[3], t2[3];
    for (int q = 0; q < K; ++q)
        for (int r = 0; r < 3; ++r) cp[r] = __dadd_rn(cp[r], poly[3 * q + r]);
    for (int r = 0; r < 3; ++r) cp[r] = __ddiv_rn(cp[r], (double)K);
    sub3(ta, img, t1);
    sub3(cp, img, t2);
    const double lam = __ddiv_rn(dot3(na, t1), dot3(na, t2));
    for (int r = 0; r < 3; ++r) spt[r] = __dadd_rn(img[r], __dmul_rn(lam, t2[r]));
    sub3(cp, spt, Dl);
    const float o[3] = {(float)spt[0], (float)spt[1], (float)spt[2]};
    const float Df[3] = {(float)Dl[0], (float)Dl[1], (float)Dl[2]};
    const float Dm = fmaxf(fmaxf(fabsf(Df[0]), fabsf(Df[1])), fabsf(Df[2]));
    const float Om = fmaxf(fmaxf(fabsf(o[0]), fabsf(o[1])), fabsf(o[2]));
    float inv[3];
    for (int r = 0; r < 3; ++r) {
        float dd = Df[r];
        if (fabsf(dd) < 1e-30f) dd = copysignf(1e-30f, dd);
        inv[r] = 1.0f / dd;
    }
    int st[kStack];
    int sp = 0;
    st[sp++] = 0;
    while (sp > 0) {
        const BvhNode m = nodes[st[--sp]];
        const int c[2] = {m.left, m.right};
        const bool h[2] = {slab_hit(m.lmin, m.lmax, o, inv), slab_hit(m.rmin, m.rmax, o, inv)};
        for (int e = 0; e < 2; ++e) {
            if (!h[e]) continue;
            if (c[e] >= 0) {
                if (sp < kStack) {
                    st[sp++] = c[e];
                } else {
                    atomicOr(status, kStatusStackOverflow);
                    return true;
                }
                continue;
            }
            const int64_t j = ~c[e];
            if (j == a || j == b) continue;
            // the FP32 pre-test decides certain misses and certain hits
            // exactly as the FP64 test would; the rest take the FP64 test
            const int pre = mt_fp32_classify(tri32[3 * j], tri32[3 * j + 1], tri32[3 * j + 2], o,
                                             Df, Dm, Om);
            if (pre == 0) continue;
            if (pre == 2) return true;
            double tj[9];
            for (int q = 0; q < 9; ++q) tj[q] = tri64[9 * j + q];
            if (mt_segment(spt, Dl, tj) != 0) return true;
        }
    }
    return false;
}

// the roots of the NS subtrees the candidate traversal splits the LBVH
// into: the nodes log2(NS) levels below the root, a leaf standing in for
// itself and leaving its missing descendants kNoNode
constexpr int kNoNode = INT32_MIN;
__global__ void bounce_roots_kernel(const BvhNode *__restrict__ nodes, int64_t F, int NS,
                                    int32_t *__restrict__ roots)
{
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    int32_t cur[8], nxt[8];
    cur[0] = F >= 2 ? 0 : kNoNode;
    int n = 1;
    while (n < NS) {
        for (int k = 0; k < n; ++k) {
            const int32_t r = cur[k];
            if (r >= 0) {
                nxt[2 * k] = nodes[r].left;
                nxt[2 * k + 1] = nodes[r].right;
            } else {
                nxt[2 * k] = r;
                nxt[2 * k + 1] = kNoNode;
            }
        }
        n *= 2;
        for (int k = 0; k < n; ++k) cur[k] = nxt[k];
    }
    for (int k = 0; k < NS; ++k) roots[k] = cur[k];
}

// Pass 1, one thread per item (p, i, s): TX p, a = the i-th facet lit from
// TX p, subtree s of the LBVH.  a's beam through the subtree; every facet
// b != a in a box that meets the beam and facing the image is a candidate
// (count, or write (a, b, p, side) at the item's offset).  Several subtrees
// per facet spread the long traversals of facets whose beams cross many
// boxes over several threads when the items alone would not fill the GPU.
template <bool FILL>
__global__ void __launch_bounds__(128)
bounce_cand_kernel(const double *__restrict__ tri64, const FacetRec *__restrict__ fac,
                   const double *__restrict__ vel64, const BvhNode *__restrict__ nodes,
                   const uint8_t *__restrict__ state, const int32_t *__restrict__ vis_idx,
                   const int32_t *__restrict__ vis_cnt, int64_t F, RadarDev rd, int NS,
                   const int32_t *__restrict__ roots, int32_t *__restrict__ cnt,
                   const int64_t *__restrict__ off, BounceCand *__restrict__ cand, int *status)
{
    const int p = blockIdx.y;
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= F * NS) return;
    const int64_t i = idx / NS;
    const int sub = (int)(idx % NS);
    const int64_t item = ((int64_t)p * F + i) * NS + sub;   // (TX, facet, subtree)
    const int root = roots[sub];
    if (i >= vis_cnt[rd.O + p] || F < 2 || root == kNoNode) {
        if (!FILL) cnt[item] = 0;
        return;
    }
    const int64_t a = vis_idx[(int64_t)(rd.O + p) * F + i];
    const double *ta = tri64 + 9 * a;
    const double pt[3] = {rd.ant[p][0], rd.ant[p][1], rd.ant[p][2]};
    double na[3], nn, img[3], u[3];
    image_of(ta, pt, vel64 + 3 * fac[a].inst, na, nn, img, u);
    const int side_a = state[(int64_t)p * F + a] == BART_VIS_LIT ? 1 : -1;
    double g[12], base[12];
    beam_planes(ta, side_a, img, g, base);
    Beam32 bm;
    beam_to_f32(g, base, bm);
    int32_t count = 0;
    int64_t slot = FILL ? off[item] : 0;
    // a leaf b met by the beam: a candidate when it faces the image
    auto leaf = [&](int64_t b) {
        if (b == a) return;
        int side_b = facing_image32(fac[b], img, rd.eps_face);
        if (side_b == 2) {
            double nbb;
            side_b = facing_image(tri64 + 9 * b, img, fac[b].two_sided != 0, rd.eps_face, &nbb);
        }
        if (!side_b) return;
        if (FILL) cand[slot++] = BounceCand{(int32_t)a, (int32_t)b, p, side_b};
        ++count;
    };
    if (root < 0) {
        leaf(~(int64_t)root);            // a subtree that is one facet (no box test)
    } else {
        int stack[kStack];
        int sp = 0;
        stack[sp++] = root;
        while (sp > 0) {
            const BvhNode nd = nodes[stack[--sp]];
            const int ch[2] = {nd.left, nd.right};
            const bool hh[2] = {box_meets_beam32(nd.lmin, nd.lmax, bm),
                                box_meets_beam32(nd.rmin, nd.rmax, bm)};
            for (int c = 0; c < 2; ++c) {
                if (!hh[c]) continue;
                if (ch[c] >= 0) {
                    if (sp < kStack) stack[sp++] = ch[c];
                    else atomicOr(status, kStatusStackOverflow);
                    continue;
                }
                leaf(~(int64_t)ch[c]);
            }
        }
    }
    if (!FILL) cnt[item] = count;
}

// Pass 2, one thread per candidate: b clipped to a's beam, the fan's
// non-sliver pieces and the a -> b leg.  Count pass: pieces (0 when the leg
// is blocked or nothing is lit); fill pass: writes them at the candidate's
// offset (the leg already decided).
template <bool FILL>
__global__ void __launch_bounds__(128)
bounce_pair_kernel(const double *__restrict__ tri64, const float4 *__restrict__ tri32,
                   const FacetRec *__restrict__ fac,
                   const double *__restrict__ vel64, const BvhNode *__restrict__ nodes,
                   const uint8_t *__restrict__ state, const BounceCand *__restrict__ cand,
                   int64_t ncand, int64_t F, RadarDev rd, int32_t *__restrict__ pcnt, const int64_t *__restrict__ poff,
                   BounceFacet *__restrict__ vf, int *status)
{
    const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= ncand) return;
    if (FILL && pcnt[c] == 0) return;
    const BounceCand C = cand[c];
    const double *ta = tri64 + 9 * (int64_t)C.a, *tb = tri64 + 9 * (int64_t)C.b;
    const double pt[3] = {rd.ant[C.p][0], rd.ant[C.p][1], rd.ant[C.p][2]};
    double na[3], nn, img[3], u[3];
    image_of(ta, pt, vel64 + 3 * fac[C.a].inst, na, nn, img, u);
    const int side_a = state[(int64_t)C.p * F + C.a] == BART_VIS_LIT ? 1 : -1;
    double g[12], base[12];
    beam_planes(ta, side_a, img, g, base);
    double f1[3], f2[3], nb[3];
    sub3(tb + 3, tb, f1);
    sub3(tb + 6, tb, f2);
    cross3(f1, f2, nb);
    const double nbb = dot3(nb, nb);
    double poly[3 * kDbMaxV];
    unsigned keep;
    const int K = clip_to_beam(tb, g, base, nbb, poly, &keep);
    if (!FILL) {
        const bool lit = K >= 3 && keep != 0 &&
                         !leg_blocked(poly, K, ta, na, img, tri64, tri32, nodes, C.a, C.b, status);
        pcnt[c] = lit ? __popc(keep) : 0;
        return;
    }
    int64_t slot = poff[c];
    const double w = -__dmul_rn((double)fac[C.a].rho, (double)fac[C.b].rho);
    for (int q = 1; q + 1 < K; ++q) {
        if (!(keep & (1u << q))) continue;
        BounceFacet &v = vf[slot++];
        v.p = C.p;
        v.a = C.a;
        v.b = C.b;
        v.side = C.side;
        for (int r = 0; r < 3; ++r) {
            v.tri[r] = poly[r];
            v.tri[3 + r] = poly[3 * q + r];
            v.tri[6 + r] = poly[3 * (q + 1) + r];
            v.src[r] = img[r];
            v.usrc[r] = u[r];
        }
        v.w = w;
    }
}

// first virtual facet of each TX: the pieces of its first candidate
__global__ void bounce_tx_offsets_kernel(const int64_t *__restrict__ cand_off,
                                         const int64_t *__restrict__ ncand,
                                         const int64_t *__restrict__ poff,
                                         const int64_t *__restrict__ npieces, int64_t F, int P,
                                         int NS, int64_t *__restrict__ txoff)
{
    const int p = threadIdx.x;
    if (p > P) return;
    const int64_t c = p < P ? cand_off[(int64_t)p * F * NS] : *ncand;
    txoff[p] = c < *ncand ? poff[c] : *npieces;
}

// ---- exclusive scan of int32 counts into int64 offsets -------------------
constexpr int kScanBlk = 1024;

__global__ void scan_blocks_kernel(const int32_t *__restrict__ in, int64_t n,
                                   int64_t *__restrict__ out, int64_t *__restrict__ blk)
{
    __shared__ int64_t s_w[kScanBlk / 32];
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    const int64_t k = (int64_t)blockIdx.x * kScanBlk + t;
    const int64_t v = k < n ? in[k] : 0;
    int64_t x = v;
    for (int o = 1; o < 32; o <<= 1) {
        const int64_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) s_w[warp] = x;
    __syncthreads();
    if (warp == 0) {
        const int64_t wv = s_w[lane];
        int64_t wx = wv;
        for (int o = 1; o < 32; o <<= 1) {
            const int64_t y = __shfl_up_sync(0xffffffffu, wx, o);
            if (lane >= o) wx += y;
        }
        s_w[lane] = wx - wv;
        if (lane == 31) blk[blockIdx.x] = wx;
    }
    __syncthreads();
    if (k < n) out[k] = s_w[warp] + x - v;
}

// one warp: exclusive scan of the block totals; blk[nblk] = the grand total
__global__ void scan_totals_kernel(int64_t *__restrict__ blk, int64_t nblk)
{
    const int lane = threadIdx.x;
    int64_t run = 0;
    for (int64_t b0 = 0; b0 < nblk; b0 += 32) {
        const int64_t b = b0 + lane;
        const int64_t v = b < nblk ? blk[b] : 0;
        int64_t x = v;
        for (int o = 1; o < 32; o <<= 1) {
            const int64_t y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        if (b < nblk) blk[b] = run + x - v;
        run += __shfl_sync(0xffffffffu, x, 31);
    }
    if (lane == 0) blk[nblk] = run;
}

__global__ void scan_add_kernel(int64_t *__restrict__ out, int64_t n,
                                const int64_t *__restrict__ blk)
{
    const int64_t k = (int64_t)blockIdx.x * kScanBlk + threadIdx.x;
    if (k < n) out[k] += blk[blockIdx.x];
}

// ---- synthesis ----------------------------------------------------------
constexpr int kDbWarps = 4;
// resident blocks per SM the FP32 synthesis is compiled for (a register
// cap): measured on the sedan-over-ground frame, 2 (218 registers) 78 ms,
// 3 (168) 69 ms, 4 (128, a few spills) 64 ms, 5 and 6 no faster
constexpr int kDbF32Blocks = 4;

struct RecB {
    double qt[3], qr[3];       // R_t(t)^2 and R_r(t)^2 over the fast time
    double d[22];              // form coefficients (record_fp64.cuh)
    int kind, flags;
};

// one sample (fast time t, frequency fm) of an FP64 record, before the
// common factor C / k_m^2
__device__ __forceinline__ void eval_rec64(const RecB &R, double t, double fm, double inv_c,
                                           double inv_f0, double mu_2c2, double &re, double &im)
{
    const double L = sqrt(R.qt[0] + t * (R.qt[1] + t * R.qt[2])) +
                     sqrt(R.qr[0] + t * (R.qr[1] + t * R.qr[2]));
    const double fmc = fm * inv_c;
    const double kp = fm * inv_f0;
    double thc = fmc * L - mu_2c2 * L * L;
    thc -= rint(thc);
    re = 0.0;
    im = 0.0;
    if (R.kind == kRecVertex) {
        for (int e = 0; e < 3; ++e) {
            double s_, c_;
            sincospi(2.0 * (thc - fmc * R.d[e]), &s_, &c_);
            re += R.d[3 + e] * c_;
            im += R.d[3 + e] * s_;
        }
    } else if (R.kind == kRecSeries) {
        double s_, c_;
        sincospi(2.0 * (thc - fmc * R.d[0]), &s_, &c_);
        const double k2 = kp * kp;
        double aa = R.d[8], bb = R.d[15];
        for (int e = 6; e >= 0; --e) aa = aa * k2 + R.d[1 + e];
        for (int e = 5; e >= 0; --e) bb = bb * k2 + R.d[9 + e];
        const double pr_ = aa * k2, pi_ = bb * k2 * kp;
        re = c_ * pr_ - s_ * pi_;
        im = c_ * pi_ + s_ * pr_;
    } else {
        for (int e = 0; e < 3; ++e) {
            double s_, c_;
            sincospi(2.0 * (thc - fmc * R.d[3 * e]), &s_, &c_);
            const double x = kp * R.d[3 * e + 1];
            double sn;
            if (R.flags & (1 << e)) {
                const double x2 = x * x;
                sn = 1.0 + x2 * (-1.0 / 6 + x2 * (1.0 / 120 + x2 * (-1.0 / 5040 +
                     x2 * (1.0 / 362880 + x2 * (-1.0 / 39916800)))));
            } else {
                sn = sin(x) / x;
            }
            const double coef = kp * R.d[3 * e + 2] * sn;
            re -= coef * s_;
            im += coef * c_;
        }
    }
}

// The FP64 record of virtual facet B for one (channel, chirp): the FP64
// path's record (record_fp64.cuh) from the facet's position at the chirp
// start tn, with the image source in place of the TX and, for the delay's
// motion within the chirp, the TX leg's own relative velocity v_b - u
__device__ void build_rec64(const BounceFacet &B, const double *vb, double tn, const double *prx,
                            const RadarDev &rd, double k0, double kmax, int two_sided, RecB &R)
{
    double tri[9], c0[3], ptx[3], rec[kRecEntries];
    for (int r = 0; r < 9; ++r) tri[r] = B.tri[r];
    centroid3(tri, c0);
    for (int r = 0; r < 3; ++r) ptx[r] = B.src[r] + B.usrc[r] * tn;
    int flags = 0;
    R.kind = build_record<double>(tri, c0, vb, tn, ptx, prx, B.w, rd.intra, k0, kmax,
                                  kDelayFacet, nullptr, two_sided, rec,
                                  &flags);
    R.flags = flags;
    R.qt[0] = rec[0];
    R.qr[0] = rec[3];
    if (rd.intra) {
        // the TX leg runs from the moving image: relative velocity v_b - u
        double dt[3], wv[3];
        for (int r = 0; r < 3; ++r) {
            dt[r] = ptx[r] - (c0[r] + vb[r] * tn);
            wv[r] = vb[r] - B.usrc[r];
        }
        R.qt[1] = -2.0 * (dt[0] * wv[0] + dt[1] * wv[1] + dt[2] * wv[2]);
        R.qt[2] = wv[0] * wv[0] + wv[1] * wv[1] + wv[2] * wv[2];
        R.qr[1] = rec[4];
        R.qr[2] = rec[2];
    } else {
        R.qt[1] = R.qt[2] = R.qr[1] = R.qr[2] = 0.0;
    }
    for (int r = 0; r < 22; ++r) R.d[r] = rec[kRecD + r];
}

template <int S>
__global__ void __launch_bounds__(kDbWarps * 32)
bounce_synth_kernel(const BounceFacet *__restrict__ vf, const int64_t *__restrict__ txoff,
                    const FacetRec *__restrict__ fac, const double *__restrict__ vel64,
                    const uint8_t *__restrict__ state, int64_t F, RadarDev rd, int W, void *out,
                    int out_c64, unsigned long long *records)
{
    __shared__ RecB sR[kDbWarps][32];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t gw = (int64_t)blockIdx.x * kDbWarps + warp;
    const int N = rd.N;
    if (gw >= (int64_t)rd.O * N * W) return;
    const int seg = (int)(gw % W);
    const int64_t unit = gw / W;
    const int o = (int)(unit / N), n = (int)(unit % N);
    const int p = o / rd.Q, q = o % rd.Q;
    const int m0 = (seg * 32 + lane) * S;
    const double c = kC0, f0 = rd.f0, mu = rd.slope, fs = rd.fs;
    const double f_max = f0 + mu * (rd.M - 1) / fs;
    const double k0 = 2.0 * kPi * f0 / c, kmax = 2.0 * kPi * f_max / c;
    const double tn = (double)((int64_t)n * rd.slots + (rd.tdm ? p : 0)) * rd.Tc;
    const double *prx = rd.ant[rd.P + q];
    const uint8_t *st_r = state + (int64_t)(rd.P + q) * F;
    const int64_t v0 = txoff[p], v1 = txoff[p + 1];      // the virtual facets of TX p

    double accr[S], acci[S];
#pragma unroll
    for (int j = 0; j < S; ++j) accr[j] = acci[j] = 0.0;
    unsigned long long nrec = 0;
    const double inv_fs = 1.0 / fs, inv_c = 1.0 / c, inv_f0 = 1.0 / f0;
    const double mu_2c2 = mu / (2.0 * c * c);
    for (int64_t base = v0; base < v1; base += 32) {
        const int64_t v = base + lane;
        bool valid = false;
        if (v < v1) {
            const BounceFacet &B = vf[v];
            valid = st_r[B.b] == (B.side > 0 ? BART_VIS_LIT : BART_VIS_LIT_REV);
            if (valid) {
                build_rec64(B, vel64 + 3 * fac[B.b].inst, tn, prx, rd, k0, kmax,
                            fac[B.b].two_sided, sR[warp][lane]);
            }
        }
        __syncwarp();
        unsigned int mask = __ballot_sync(0xffffffffu, valid);
        nrec += __popc(mask);
        while (mask) {
            const int i = __ffs(mask) - 1;
            mask &= mask - 1;
            const RecB &R = sR[warp][i];
#pragma unroll 1
            for (int j = 0; j < S; ++j) {
                const double t = (double)(m0 + j) * inv_fs;
                const double fm = f0 + mu * t;
                double re, im;
                eval_rec64(R, t, fm, inv_c, inv_f0, mu_2c2, re, im);
                accr[j] += re;
                acci[j] += im;
            }
        }
        __syncwarp();
    }
    if (lane == 0 && seg == 0 && records) atomicAdd(records, nrec);
    const double camp = 2.0 * sqrt(kPi) / pow(4.0 * kPi, 1.5);
    const int64_t row = ((int64_t)o * N + n) * rd.M + m0;
#pragma unroll
    for (int j = 0; j < S; ++j) {
        const double fm = f0 + mu * (double)(m0 + j) / fs;
        const double km = 2.0 * kPi * fm / c;
        const double sc = camp / (km * km);
        if (out_c64) {
            float2 &y = reinterpret_cast<float2 *>(out)[row + j];
            y.x += (float)(accr[j] * sc);
            y.y += (float)(acci[j] * sc);
        } else {
            double2 &y = reinterpret_cast<double2 *>(out)[row + j];
            y.x += accr[j] * sc;
            y.y += acci[j] * sc;
        }
    }
}

__device__ __forceinline__ double red1d(double x) { return x - rint(x); }
__device__ __forceinline__ float red1f(float x) { return x - rintf(x); }

// FP32 form of a record for one (channel, chirp).  Every form is a sum of
// phasors exp{j 2 pi (theta(m) - f_m u_c / c)} over its centres u_c (the
// vertex form: the vertices; the edge form: the edge midpoints; the series
// form: the vertices' mean) with amplitudes from x; the phase of centre c at
// sample m is A_c + B_c m + C m^2 cycles (the path to second order in fast
// time; the third-order term stays below 1e-12 m over a chirp), B_c = Bhi_c
// + Blo_c with Bhi_c a multiple of 2^-14 (so that Bhi_c m is exact in FP32
// for m < 2^10) and |Blo_c| <= 2^-15.  x: vertex form, the vertex weights
// (x[0..2]); series form, the 15 coefficients of the polynomials in k_m^2
// (record_fp64.cuh's d[1..15]); edge form, k0 gamma_e (x[0..2]) and the edge
// amplitudes (x[3..5]), with flags bit e: sinc by its series.
struct RecV {
    float A[3], Bhi[3], Blo[3];
    float C;
    float sc[3], ss[3];      // the chord step of each centre at m0 = 0 (cos, sin)
    float x[15];
    int kind, flags;
};

// the centres' chord steps exp{j 2 pi (B_c + C (S - 1))} of a lane that
// starts at m0 = 0 (a lane at m0 multiplies them by exp{j 4 pi C m0})
__device__ __forceinline__ void chord_steps(RecV &V, float chord0)
{
    const int nc = V.kind == kRecSeries ? 1 : 3;
    for (int c = 0; c < nc; ++c)
        sincospif(2.f * red1f(V.Bhi[c] + fmaf(V.C, chord0, V.Blo[c])), &V.ss[c], &V.sc[c]);
}


// the phase constants of Eq. 13 for the quadratics, formed once
struct PhaseK {
    double f0c, muc, mu2c2, inv_fs, inv_fs2, mucfs;
};
__device__ __forceinline__ PhaseK phase_consts(const RadarDev &rd)
{
    PhaseK P;
    P.f0c = rd.f0 / kC0;
    P.muc = rd.slope / kC0;
    P.mu2c2 = rd.slope / (2.0 * kC0 * kC0);
    P.inv_fs = 1.0 / rd.fs;
    P.inv_fs2 = P.inv_fs * P.inv_fs;
    P.mucfs = P.muc * P.inv_fs;
    return P;
}

// the phase f(t) L(t) / c - mu L(t)^2 / (2 c^2) of Eq. 13 over the fast
// time, L = L0 + L1 t + L2 t^2, as th0 + th1 m + th2 m^2 (cycles, samples m);
// then centre c's A_c, Bhi_c, Blo_c and the common C
__device__ __forceinline__ void path_phase(double L0, double L1, double L2, const PhaseK &K,
                                           double &th0, double &th1, double &th2)
{
    th0 = K.f0c * L0 - K.mu2c2 * L0 * L0;
    th1 = (K.f0c * L1 + K.muc * L0 - 2.0 * K.mu2c2 * L0 * L1) * K.inv_fs;
    th2 = (K.f0c * L2 + K.muc * L1 - K.mu2c2 * (L1 * L1 + 2.0 * L0 * L2)) * K.inv_fs2;
}
__device__ __forceinline__ void centre_phase(double th0, double th1, double u, const PhaseK &K,
                                             RecV &V, int c)
{
    V.A[c] = (float)red1d(th0 - K.f0c * u);
    const double b = red1d(th1 - K.mucfs * u);
    const double bhi = rint(b * 16384.0) * 0x1p-14;
    V.Bhi[c] = (float)bhi;
    V.Blo[c] = (float)(b - bhi);
}

// RecV of a full FP64 record: each leg's path sqrt(q0 + q1 t + q2 t^2)
// expanded to second order, the centres and amplitudes rounded to FP32
__device__ __forceinline__ void rec64_to_v(const RecB &R, const PhaseK &K, RecV &V)
{
    double L0 = 0.0, L1 = 0.0, L2 = 0.0;
    const double *qs[2] = {R.qt, R.qr};
    for (int l = 0; l < 2; ++l) {
        const double *q = qs[l];
        const double a0 = sqrt(q[0]);
        const double inv = 0.5 / a0;
        const double a1 = q[1] * inv;
        L0 += a0;
        L1 += a1;
        L2 += (q[2] - a1 * a1) * inv;
    }
    double th0, th1, th2;
    path_phase(L0, L1, L2, K, th0, th1, th2);
    V.C = (float)th2;
    V.kind = R.kind;
    V.flags = R.flags;
    if (R.kind == kRecVertex) {
        for (int v = 0; v < 3; ++v) {
            centre_phase(th0, th1, R.d[v], K, V, v);
            V.x[v] = (float)R.d[3 + v];
        }
    } else if (R.kind == kRecSeries) {
        centre_phase(th0, th1, R.d[0], K, V, 0);
        for (int i = 0; i < 15; ++i) V.x[i] = (float)R.d[1 + i];
    } else {
        for (int e = 0; e < 3; ++e) {
            centre_phase(th0, th1, R.d[3 * e], K, V, e);
            V.x[e] = (float)R.d[3 * e + 1];
            V.x[3 + e] = (float)R.d[3 * e + 2];
        }
    }
}

// Slow-time row of one leg of a virtual facet: the path from the facet's
// centroid to the leg's antenna (the image source for the TX leg, RX q for
// leg 1 + q) as R(t_c + tau) = sum_j a_j tau^j about the frame's middle
// chirp slot t_c.  R^2 is exactly the quadratic |D_c + w tau|^2 (both ends
// move linearly), so the a_j follow from the square-root recursion, and
// with rho = tau_max |w| / R(t_c) the terms beyond degree 6 are bounded by
// R rho^7 / (1 - rho); a row whose bound exceeds 1e-11 m is marked a[0] = -1
// (its records take the full FP64 build).  B = antenna - centroid at the
// frame start and w = centroid velocity relative to the antenna give the
// directions in FP32 from the constant B and the small drift -w t.
constexpr int kDbDeg = 6;
// the projections of the vertex offsets on the leg's unit vector toward its
// antenna, p_v(t_c + tau) = sum_j pu[v][j] tau^j; a row is used only where
// the terms beyond degree 3, at most |dv| rho^4 / (1 - rho), stay below 1e-9 m
constexpr int kDbPDeg = 3;
struct BounceRow {
    double a[kDbDeg + 1];
    double pu[3][kDbPDeg + 1];
    float af[kDbDeg + 1];    // a in FP32 (for the derivatives)
    float B[3], w[3];
};
// per virtual facet: unit normal, area and vertex offsets from the centroid
struct BounceGeo {
    float n[3], area, dv[9], pad[3];
};

__global__ void bounce_rows_kernel(const BounceFacet *__restrict__ vf, int64_t V,
                                   const FacetRec *__restrict__ fac,
                                   const double *__restrict__ vel64, RadarDev rd, double tc,
                                   double tmax, BounceRow *__restrict__ rows,
                                   BounceGeo *__restrict__ geo)
{
    const int L = 1 + rd.Q;
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= V * L) return;
    const int64_t v = i / L;
    const int l = (int)(i % L);
    const BounceFacet &B = vf[v];
    double c0[3];
    for (int r = 0; r < 3; ++r) c0[r] = (B.tri[r] + B.tri[3 + r] + B.tri[6 + r]) / 3.0;
    const double *vb = vel64 + 3 * fac[B.b].inst;
    double P[3], w[3];
    for (int r = 0; r < 3; ++r) {
        P[r] = l == 0 ? B.src[r] : rd.ant[rd.P + l - 1][r];
        w[r] = l == 0 ? vb[r] - B.usrc[r] : vb[r];
    }
    double Dc[3];
    for (int r = 0; r < 3; ++r) Dc[r] = (c0[r] - P[r]) + w[r] * tc;
    const double q0 = Dc[0] * Dc[0] + Dc[1] * Dc[1] + Dc[2] * Dc[2];
    const double q1 = 2.0 * (Dc[0] * w[0] + Dc[1] * w[1] + Dc[2] * w[2]);
    const double q2 = w[0] * w[0] + w[1] * w[1] + w[2] * w[2];
    BounceRow &R = rows[i];
    const double a0 = sqrt(q0);
    const double rho = tmax * sqrt(q2 / q0);
    double dvmax = 0.0;              // the largest vertex offset (projection series bound)
    for (int v = 0; v < 3; ++v) {
        double q = 0.0;
        for (int r = 0; r < 3; ++r) {
            const double d = B.tri[3 * v + r] - c0[r];
            q += d * d;
        }
        dvmax = fmax(dvmax, sqrt(q));
    }
    bool ok = q0 > 0.0 && rho < 0.25;
    if (ok) {
        double b = a0, bp = dvmax;
        for (int j = 0; j <= kDbDeg; ++j) b *= rho;
        for (int j = 0; j <= kDbPDeg; ++j) bp *= rho;
        ok = b / (1.0 - rho) <= 1e-11 && bp / (1.0 - rho) <= 1e-9;
    }
    double a[kDbDeg + 1];
    a[0] = ok ? a0 : -1.0;
    const double inv2a0 = 0.5 / a0;
    for (int j = 1; j <= kDbDeg; ++j) {
        double s = j == 1 ? q1 : (j == 2 ? q2 : 0.0);
        for (int k = 1; k < j; ++k) s -= a[k] * a[j - k];
        a[j] = ok ? s * inv2a0 : 0.0;
    }
    for (int j = 0; j <= kDbDeg; ++j) {
        R.a[j] = a[j];
        R.af[j] = (float)a[j];
    }
    // 1 / R as a series (b_0 = 1 / a_0, b_j = -sum_i a_i b_{j - i} / a_0), and
    // p_v = -(D_c + w tau).dv_v / R: the phase's projections in FP64
    double rb[kDbPDeg + 1];
    rb[0] = ok ? 1.0 / a0 : 0.0;
    for (int j = 1; j <= kDbPDeg; ++j) {
        double sacc = 0.0;
        for (int k = 1; k <= j; ++k) sacc += a[k] * rb[j - k];
        rb[j] = ok ? -sacc * rb[0] : 0.0;
    }
    for (int v = 0; v < 3; ++v) {
        double dv[3];
        for (int r = 0; r < 3; ++r) dv[r] = B.tri[3 * v + r] - c0[r];
        const double n0 = -(Dc[0] * dv[0] + Dc[1] * dv[1] + Dc[2] * dv[2]);
        const double n1 = -(w[0] * dv[0] + w[1] * dv[1] + w[2] * dv[2]);
        for (int j = 0; j <= kDbPDeg; ++j) R.pu[v][j] = n0 * rb[j] + (j > 0 ? n1 * rb[j - 1] : 0.0);
    }
    for (int r = 0; r < 3; ++r) {
        R.B[r] = (float)(P[r] - c0[r]);
        R.w[r] = (float)w[r];
    }
    if (l == 0) {
        BounceGeo &G = geo[v];
        double e1[3], e2[3], n[3];
        for (int r = 0; r < 3; ++r) {
            e1[r] = B.tri[3 + r] - B.tri[r];
            e2[r] = B.tri[6 + r] - B.tri[r];
        }
        n[0] = e1[1] * e2[2] - e1[2] * e2[1];
        n[1] = e1[2] * e2[0] - e1[0] * e2[2];
        n[2] = e1[0] * e2[1] - e1[1] * e2[0];
        const double nl = sqrt(n[0] * n[0] + n[1] * n[1] + n[2] * n[2]);
        for (int r = 0; r < 3; ++r) G.n[r] = (float)(n[r] / nl);
        G.area = (float)(0.5 * nl);
        for (int k = 0; k < 9; ++k) G.dv[k] = (float)(B.tri[k] - c0[k % 3]);
        G.pad[0] = G.pad[1] = G.pad[2] = 0.f;
    }
}

// R (FP64), dR/dt and d2R/dt2 (FP32: they enter the phase only through
// the slope's small velocity part and the curvature) of a row at tau
__device__ __forceinline__ void row_eval(const BounceRow &R, double tau, double &r0, float &r1,
                                         float &r2)
{
    r0 = R.a[kDbDeg];
#pragma unroll
    for (int j = kDbDeg - 1; j >= 0; --j) r0 = fma(r0, tau, R.a[j]);
    const float t = (float)tau;
    r1 = kDbDeg * R.af[kDbDeg];
    r2 = kDbDeg * (kDbDeg - 1) * R.af[kDbDeg];
#pragma unroll
    for (int j = kDbDeg - 1; j >= 1; --j) {
        r1 = fmaf(r1, t, j * R.af[j]);
        if (j >= 2) r2 = fmaf(r2, t, j * (j - 1) * R.af[j]);
    }
}

// 1 / n! in FP32 for the series form (n = 2 .. 16)
__device__ __forceinline__ float inv_fact_f(int n)
{
    float f = 1.f;
    for (int i = 2; i <= n; ++i) f *= (float)i;
    return 1.f / f;
}

// The FP32 record of a virtual facet from its rows: FP64 for the path, the
// phase quadratics and the projections u_v (from the rows' series of
// th.dv_v and rh.dv_v; u_v = b.dv_v as dv_v lies in the facet's plane), from
// which the form switches and the weights' pair differences come too;
// directions, obliquity and every form's amplitudes in FP32
// (record_fp64.cuh's forms).  Returns false when a row has
// no expansion (the record then takes the full FP64 build).
__device__ __forceinline__ bool lean_record(const BounceRow &Rt, const BounceRow &Rr,
                                            const BounceGeo &G, float wrho, int two_sided,
                                            double tau, float tn, const RadarDev &rd,
                                            const PhaseK &K, float k0, float kmax,
                                            float chord0, RecV &V)
{
    if (Rt.a[0] < 0.0 || Rr.a[0] < 0.0) return false;
    double t0, s0;
    float t1, t2, s1, s2;
    row_eval(Rt, tau, t0, t1, t2);
    row_eval(Rr, tau, s0, s1, s2);
    float th[3], rh[3];
    {
        float dt[3], dr[3];
#pragma unroll
        for (int r = 0; r < 3; ++r) {
            dt[r] = fmaf(-Rt.w[r], tn, Rt.B[r]);
            dr[r] = fmaf(-Rr.w[r], tn, Rr.B[r]);
        }
        const float it = rsqrtf(dt[0] * dt[0] + dt[1] * dt[1] + dt[2] * dt[2]);
        const float ir = rsqrtf(dr[0] * dr[0] + dr[1] * dr[1] + dr[2] * dr[2]);
#pragma unroll
        for (int r = 0; r < 3; ++r) {
            th[r] = dt[r] * it;
            rh[r] = dr[r] * ir;
        }
    }
    const float b[3] = {th[0] + rh[0], th[1] + rh[1], th[2] + rh[2]};
    const float bn = G.n[0] * b[0] + G.n[1] * b[1] + G.n[2] * b[2];
    float ok = 0.5f * bn;
    if (two_sided) ok = fabsf(ok);
    const float g = __fdividef(wrho * ok, (float)t0 * (float)s0);
    const float bt[3] = {b[0] - bn * G.n[0], b[1] - bn * G.n[1], b[2] - bn * G.n[2]};
    const float A2 = 2.f * G.area * g;
    double th0, th1, th2;
    path_phase(t0 + s0, rd.intra ? (double)(t1 + s1) : 0.0,
               rd.intra ? (double)(0.5f * (t2 + s2)) : 0.0, K, th0, th1, th2);
    double ud[3];                    // u_v in FP64 for the phases
#pragma unroll
    for (int v = 0; v < 3; ++v) {
        double pt = Rt.pu[v][kDbPDeg], pr = Rr.pu[v][kDbPDeg];
#pragma unroll
        for (int j = kDbPDeg - 1; j >= 0; --j) {
            pt = fma(pt, tau, Rt.pu[v][j]);
            pr = fma(pr, tau, Rr.pu[v][j]);
        }
        ud[v] = pt + pr;
    }
    // the forms' weights must use the u_v of their phases: a mismatch of
    // delta between them is amplified by the vertex terms' cancellation
    // (~delta / |u_a - u_b| relative), so the pair differences d_v =
    // u_v - u_{v+1} and the form switches come from the FP64 projections
    float d[3];
#pragma unroll
    for (int v = 0; v < 3; ++v) d[v] = (float)(ud[v] - ud[(v + 1) % 3]);
    const float urange = (float)(fmax(fmax(ud[0], ud[1]), ud[2]) - fmin(fmin(ud[0], ud[1]), ud[2]));
    const float dmin = fminf(fminf(fabsf(d[0]), fabsf(d[1])), fabsf(d[2]));
    V.C = (float)th2;
    V.flags = 0;
    if (kmax * urange < (float)kSeriesKD) {
        // series form: J = sum_p j^p h_p(y) / (p + 2)!  with y_v = k (u_v - ub)
        const float y0 = k0 * (d[0] - d[2]) * (1.f / 3.f);
        const float y1 = k0 * (d[1] - d[0]) * (1.f / 3.f);
        const float y2 = k0 * (d[2] - d[1]) * (1.f / 3.f);
        const float e2s = y0 * y1 + y0 * y2 + y1 * y2, e3s = y0 * y1 * y2;
        float h[kSeriesTerms];
        h[0] = 1.f;
        h[1] = 0.f;
        h[2] = -e2s;
#pragma unroll
        for (int q = 3; q < kSeriesTerms; ++q) h[q] = -e2s * h[q - 2] + e3s * h[q - 3];
        const float sc = A2 * k0 * k0;
#pragma unroll
        for (int i = 0; i < 8; ++i) V.x[i] = ((i & 1) ? -sc : sc) * h[2 * i] * inv_fact_f(2 * i + 2);
#pragma unroll
        for (int i = 0; i < 7; ++i)
            V.x[8 + i] = ((i & 1) ? sc : -sc) * h[2 * i + 1] * inv_fact_f(2 * i + 3);
        centre_phase(th0, th1, (ud[0] + ud[1] + ud[2]) * (1.0 / 3.0), K, V, 0);
        V.kind = kRecSeries;
        chord_steps(V, chord0);
        return true;
    }
    if (kmax * dmin < (float)kEdgeKd) {
        // edge form: J = sum_e (-j) k gamma_e-scaled sinc terms at the edge midpoints
        const float bt2 = bt[0] * bt[0] + bt[1] * bt[1] + bt[2] * bt[2];
        const float nxb[3] = {G.n[1] * bt[2] - G.n[2] * bt[1], G.n[2] * bt[0] - G.n[0] * bt[2],
                              G.n[0] * bt[1] - G.n[1] * bt[0]};
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            const int i1 = (i + 1) % 3;
            const float e[3] = {G.dv[3 * i1] - G.dv[3 * i], G.dv[3 * i1 + 1] - G.dv[3 * i + 1],
                                G.dv[3 * i1 + 2] - G.dv[3 * i + 2]};
            const float gam = -0.5f * d[i];
            V.x[i] = k0 * gam;
            V.x[3 + i] = k0 * g * (e[0] * nxb[0] + e[1] * nxb[1] + e[2] * nxb[2]) / bt2;
            if (kmax * fabsf(gam) < (float)kSincSeries) V.flags |= 1 << i;
            centre_phase(th0, th1, 0.5 * (ud[i] + ud[i1]), K, V, i);
        }
        V.kind = kRecEdge;
        chord_steps(V, chord0);
        return true;
    }
    // vertex form: -A2 / ((u_v - u_{v+1}) (u_v - u_{v+2})) = A2 / (d_v d_{v+2})
    V.x[0] = A2 / (d[0] * d[2]);
    V.x[1] = A2 / (d[1] * d[0]);
    V.x[2] = A2 / (d[2] * d[1]);
#pragma unroll
    for (int v = 0; v < 3; ++v) centre_phase(th0, th1, ud[v], K, V, v);
    V.kind = kRecVertex;
    chord_steps(V, chord0);
    return true;
}

// The double-bounce synthesis with the per-sample work in FP32: records
// from the virtual facets' slow-time rows (lean_record; the full FP64 build,
// rounded to the same FP32 form, where a row has no expansion), one per
// lane, 32 per batch, records of every form evaluated
// by every lane over its S samples from an FP32 start phasor and its chord
// step (the curvature C (S - 1)^2 / 4 cycles, below 1e-5, is left out),
// the amplitudes of the series and edge forms per sample; batch sums in
// FP32 added to FP64 totals.
template <int S>
__global__ void __launch_bounds__(kDbWarps * 32, kDbF32Blocks)
bounce_synth_f32_kernel(const BounceFacet *__restrict__ vf, const int64_t *__restrict__ txoff,
                        const FacetRec *__restrict__ fac, const double *__restrict__ vel64,
                        const uint8_t *__restrict__ state, int64_t F, RadarDev rd, int W,
                        void *out, int out_c64, unsigned long long *records,
                        const BounceRow *__restrict__ rows, const BounceGeo *__restrict__ geo,
                        double tc, int NCH, double2 *__restrict__ partial)
{
    __shared__ RecV sV[kDbWarps][32];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t gw = (int64_t)blockIdx.x * kDbWarps + warp;
    const int N = rd.N;
    if (gw >= (int64_t)rd.O * N * W * NCH) return;
    const int chunk = (int)(gw % NCH);
    const int seg = (int)(gw / NCH % W);
    const int64_t unit = gw / ((int64_t)NCH * W);
    const int o = (int)(unit / N), n = (int)(unit % N);
    const int p = o / rd.Q, q = o % rd.Q;
    const int m0 = (seg * 32 + lane) * S;
    const double c = kC0, f0 = rd.f0, mu = rd.slope, fs = rd.fs;
    const double f_max = f0 + mu * (rd.M - 1) / fs;
    const double k0 = 2.0 * kPi * f0 / c, kmax = 2.0 * kPi * f_max / c;
    const double tn = (double)((int64_t)n * rd.slots + (rd.tdm ? p : 0)) * rd.Tc;
    const double *prx = rd.ant[rd.P + q];
    const uint8_t *st_r = state + (int64_t)(rd.P + q) * F;
    // this warp's chunk of the virtual facets of TX p
    const int64_t vt0 = txoff[p], nv = txoff[p + 1] - vt0;
    const int64_t v0 = vt0 + nv * chunk / NCH, v1 = vt0 + nv * (chunk + 1) / NCH;
    const float fm0 = (float)m0, fm0sq = fm0 * fm0;
    const PhaseK PK = phase_consts(rd);

    const float kps = (float)(mu / (f0 * fs));       // k_m / k_0 = 1 + kps m
    const float k0f = (float)k0, kmaxf = (float)kmax;

    double accr[S], acci[S];
#pragma unroll
    for (int j = 0; j < S; ++j) accr[j] = acci[j] = 0.0;
    unsigned long long nrec = 0;
    for (int64_t base = v0; base < v1; base += 32) {
        const int64_t v = base + lane;
        bool valid = false;
        if (v < v1) {
            const BounceFacet &B = vf[v];
            valid = st_r[B.b] == (B.side > 0 ? BART_VIS_LIT : BART_VIS_LIT_REV);
            if (valid) {
                const int L = 1 + rd.Q;
                const bool lean = lean_record(rows[v * L], rows[v * L + 1 + q], geo[v],
                                              (float)B.w, fac[B.b].two_sided, tn - tc,
                                              (float)tn, rd, PK, k0f, kmaxf, (float)(S - 1),
                                              sV[warp][lane]);
                if (!lean) {
                    RecB R64;
                    build_rec64(B, vel64 + 3 * fac[B.b].inst, tn, prx, rd, k0, kmax,
                                fac[B.b].two_sided, R64);
                    rec64_to_v(R64, PK, sV[warp][lane]);
                    chord_steps(sV[warp][lane], (float)(S - 1));
                }
            }
        }
        __syncwarp();
        unsigned int mask = __ballot_sync(0xffffffffu, valid);
        nrec += __popc(mask);
        float ar[S], ai[S];
#pragma unroll
        for (int j = 0; j < S; ++j) ar[j] = ai[j] = 0.f;
        while (mask) {
            const int i = __ffs(mask) - 1;
            mask &= mask - 1;
            const RecV &V = sV[warp][i];
            const int nc = V.kind == kRecSeries ? 1 : 3;
            float zc[3], zs[3], cs[3], ss[3];
            // the lane's chord step: the record's at m0 = 0 times
            // exp{j 4 pi C m0} ~ (1 - x^2 / 2, x), |x| < 1e-2, error x^3 / 6
            const float x = 12.566370614359172f * V.C * fm0;
            const float xr = fmaf(-0.5f * x, x, 1.f);
#pragma unroll
            for (int e = 0; e < 3; ++e) {
                if (e >= nc) break;
                // the phase reduced to [-1/2, 1/2] cycle: the SFU's sine and
                // cosine over [-pi, pi] (absolute error ~4e-7)
                const float ph = red1f(red1f(V.Bhi[e] * fm0) +
                                       (V.A[e] + fmaf(V.Blo[e], fm0, V.C * fm0sq)));
                __sincosf(6.283185307179586f * ph, &zs[e], &zc[e]);
                cs[e] = fmaf(V.sc[e], xr, -V.ss[e] * x);
                ss[e] = fmaf(V.sc[e], x, V.ss[e] * xr);
            }
            if (V.kind == kRecVertex) {
#pragma unroll
                for (int j = 0; j < S; ++j) {
                    float tr = 0.f, ti = 0.f;
#pragma unroll
                    for (int e = 0; e < 3; ++e) {
                        tr = fmaf(V.x[e], zc[e], tr);
                        ti = fmaf(V.x[e], zs[e], ti);
                        const float ncs = fmaf(zc[e], cs[e], -zs[e] * ss[e]);
                        zs[e] = fmaf(zc[e], ss[e], zs[e] * cs[e]);
                        zc[e] = ncs;
                    }
                    ar[j] += tr;
                    ai[j] += ti;
                }
            } else if (V.kind == kRecSeries) {
#pragma unroll
                for (int j = 0; j < S; ++j) {
                    const float kp = fmaf(kps, fm0 + (float)j, 1.f), k2 = kp * kp;
                    float a = V.x[7], bb = V.x[14];
#pragma unroll
                    for (int e = 6; e >= 0; --e) a = fmaf(a, k2, V.x[e]);
#pragma unroll
                    for (int e = 5; e >= 0; --e) bb = fmaf(bb, k2, V.x[8 + e]);
                    const float pr = a * k2, pi = bb * k2 * kp;
                    ar[j] += fmaf(zc[0], pr, -zs[0] * pi);
                    ai[j] += fmaf(zc[0], pi, zs[0] * pr);
                    const float ncs = fmaf(zc[0], cs[0], -zs[0] * ss[0]);
                    zs[0] = fmaf(zc[0], ss[0], zs[0] * cs[0]);
                    zc[0] = ncs;
                }
            } else {
#pragma unroll 1
                for (int j = 0; j < S; ++j) {
                    const float kp = fmaf(kps, fm0 + (float)j, 1.f);
                    float tr = 0.f, ti = 0.f;
#pragma unroll
                    for (int e = 0; e < 3; ++e) {
                        const float xx = kp * V.x[e];
                        float sn;
                        if (V.flags & (1 << e)) {
                            const float x2 = xx * xx;
                            sn = 1.f + x2 * (-1.f / 6 + x2 * (1.f / 120 + x2 * (-1.f / 5040 +
                                 x2 * (1.f / 362880))));
                        } else {
                            sn = sinf(xx) / xx;
                        }
                        const float coef = kp * V.x[3 + e] * sn;
                        tr = fmaf(-coef, zs[e], tr);
                        ti = fmaf(coef, zc[e], ti);
                        const float ncs = fmaf(zc[e], cs[e], -zs[e] * ss[e]);
                        zs[e] = fmaf(zc[e], ss[e], zs[e] * cs[e]);
                        zc[e] = ncs;
                    }
                    ar[j] += tr;
                    ai[j] += ti;
                }
            }
        }
#pragma unroll
        for (int j = 0; j < S; ++j) {
            accr[j] += (double)ar[j];
            acci[j] += (double)ai[j];
        }
        __syncwarp();
    }
    if (lane == 0 && seg == 0 && records) atomicAdd(records, nrec);
    const double camp = 2.0 * sqrt(kPi) / pow(4.0 * kPi, 1.5);
    const int64_t row = ((int64_t)o * N + n) * rd.M + m0;
#pragma unroll
    for (int j = 0; j < S; ++j) {
        const double fm = f0 + mu * (double)(m0 + j) / fs;
        const double km = 2.0 * kPi * fm / c;
        const double sc = camp / (km * km);
        if (NCH > 1) {         // this chunk's scaled partial sums, added in order later
            partial[(int64_t)chunk * rd.O * N * rd.M + row + j] =
                make_double2(accr[j] * sc, acci[j] * sc);
        } else if (out_c64) {
            float2 &y = reinterpret_cast<float2 *>(out)[row + j];
            y.x += (float)(accr[j] * sc);
            y.y += (float)(acci[j] * sc);
        } else {
            double2 &y = reinterpret_cast<double2 *>(out)[row + j];
            y.x += accr[j] * sc;
            y.y += acci[j] * sc;
        }
    }
}

// adds the chunks' partial sums of each sample, in chunk order, into the cube
__global__ void bounce_reduce_kernel(const double2 *__restrict__ partial, int64_t n, int NCH,
                                     void *out, int out_c64)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    double re = 0.0, im = 0.0;
    for (int ch = 0; ch < NCH; ++ch) {
        const double2 v = partial[(int64_t)ch * n + i];
        re += v.x;
        im += v.y;
    }
    if (out_c64) {
        float2 &y = reinterpret_cast<float2 *>(out)[i];
        y.x += (float)re;
        y.y += (float)im;
    } else {
        double2 &y = reinterpret_cast<double2 *>(out)[i];
        y.x += re;
        y.y += im;
    }
}

}  // namespace

int64_t bounce_scan_words(int64_t n) { return (n + kScanBlk - 1) / kScanBlk + 1; }

int64_t bounce_row_bytes(const RadarDev &rd) { return (int64_t)sizeof(BounceRow) * (1 + rd.Q); }
int64_t bounce_geo_bytes() { return (int64_t)sizeof(BounceGeo); }

void launch_bounce_scan(const int32_t *cnt, int64_t n, int64_t *off, int64_t *blk,
                        cudaStream_t s)
{
    const int64_t nblk = (n + kScanBlk - 1) / kScanBlk;
    if (nblk > 0) scan_blocks_kernel<<<(unsigned int)nblk, kScanBlk, 0, s>>>(cnt, n, off, blk);
    scan_totals_kernel<<<1, 32, 0, s>>>(blk, nblk);
    if (nblk > 0) scan_add_kernel<<<(unsigned int)nblk, kScanBlk, 0, s>>>(off, n, blk);
}

int bounce_subtrees(const RadarDev &rd, int64_t F)
{
    const int64_t items = (int64_t)rd.P * F;
    int NS = 1;
    while (NS < 8 && items * NS < (1 << 21)) NS *= 2;
    return NS;
}

void launch_bounce_roots(const BvhNode *nodes, int64_t F, int NS, int32_t *roots, cudaStream_t s)
{
    bounce_roots_kernel<<<1, 32, 0, s>>>(nodes, F, NS, roots);
}

void launch_bounce_candidates(bool fill, const double *tri64, const FacetRec *fac,
                              const double *vel64, const BvhNode *nodes, const uint8_t *state,
                              const int32_t *vis_idx, const int32_t *vis_cnt, int64_t F,
                              const RadarDev &rd, int NS, const int32_t *roots, int32_t *cnt,
                              const int64_t *off, BounceCand *cand, int *status, cudaStream_t s)
{
    const int T = 128;
    dim3 grid((unsigned int)((F * NS + T - 1) / T), (unsigned int)rd.P);
    if (fill)
        bounce_cand_kernel<true><<<grid, T, 0, s>>>(tri64, fac, vel64, nodes, state, vis_idx,
                                                    vis_cnt, F, rd, NS, roots, cnt, off, cand,
                                                    status);
    else
        bounce_cand_kernel<false><<<grid, T, 0, s>>>(tri64, fac, vel64, nodes, state, vis_idx,
                                                     vis_cnt, F, rd, NS, roots, cnt, off, cand,
                                                     status);
}

void launch_bounce_pairs(bool fill, const double *tri64, const float *tri32, const FacetRec *fac,
                         const double *vel64, const BvhNode *nodes, const uint8_t *state,
                         const BounceCand *cand, int64_t ncand, int64_t F, const RadarDev &rd,
                         int32_t *pcnt, const int64_t *poff, BounceFacet *vf, int *status,
                         cudaStream_t s)
{
    if (ncand <= 0) return;
    const float4 *t32 = reinterpret_cast<const float4 *>(tri32);
    const int T = 128;
    const unsigned int grid = (unsigned int)((ncand + T - 1) / T);
    if (fill)
        bounce_pair_kernel<true><<<grid, T, 0, s>>>(tri64, t32, fac, vel64, nodes, state, cand, ncand,
                                                    F, rd, pcnt, poff, vf, status);
    else
        bounce_pair_kernel<false><<<grid, T, 0, s>>>(tri64, t32, fac, vel64, nodes, state, cand,
                                                     ncand, F, rd, pcnt, poff, vf, status);
}

void launch_bounce_tx_offsets(const int64_t *cand_off, const int64_t *ncand, const int64_t *poff,
                              const int64_t *npieces, int64_t F, int P, int NS, int64_t *txoff,
                              cudaStream_t s)
{
    bounce_tx_offsets_kernel<<<1, 64, 0, s>>>(cand_off, ncand, poff, npieces, F, P, NS, txoff);
}

void launch_bounce_rows(const BounceFacet *vf, int64_t V, const FacetRec *fac,
                        const double *vel64, const RadarDev &rd, void *rows, void *geo,
                        cudaStream_t s)
{
    if (V <= 0) return;
    const double tc = bounce_mid_time(rd);
    const int64_t n = V * (1 + rd.Q);
    bounce_rows_kernel<<<(unsigned int)((n + 127) / 128), 128, 0, s>>>(
        vf, V, fac, vel64, rd, tc, tc > 0.0 ? tc : rd.Tc, static_cast<BounceRow *>(rows),
        static_cast<BounceGeo *>(geo));
}

// chunks of each (channel, chirp, segment) record list of the FP32
// evaluation: about four waves of resident warps (a sedan frame has a few
// thousand (channel, chirp) rows), at most 16
int bounce_synth_chunks(const RadarDev &rd)
{
    static int sms = 0;
    if (sms <= 0) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (sms <= 0) sms = 1;
    }
    int S = 16;
    while ((rd.M / 32) % S) S /= 2;
    const int64_t rows = (int64_t)rd.O * rd.N * (rd.M / (32 * S));
    const int64_t target = 4 * (int64_t)sms * 12;     // ~12 resident warps per SM
    return (int)std::max<int64_t>(1, std::min<int64_t>(16, (target + rows - 1) / rows));
}

void launch_bounce_synth(const BounceFacet *vf, const int64_t *txoff, const FacetRec *fac,
                         const double *vel64, const uint8_t *state, int64_t F,
                         const RadarDev &rd, void *out, int out_c64, bool fp32_eval,
                         const void *rows, const void *geo, int NCH, double2 *partial,
                         unsigned long long *records, cudaStream_t s)
{
    const int M = rd.M;                // a multiple of 32
    // samples per lane: the largest power of two up to 16 (FP32 evaluation)
    // or 8 (FP64) that divides M / 32
    int S = fp32_eval ? 16 : 8;
    while ((M / 32) % S) S /= 2;
    const int W = M / (32 * S);
    const int64_t warps = (int64_t)rd.O * rd.N * W;
    const dim3 blk(kDbWarps * 32);
    if (!fp32_eval) {
        const unsigned int grid = (unsigned int)((warps + kDbWarps - 1) / kDbWarps);
#define BART_DB_LAUNCH64(SS) bounce_synth_kernel<SS><<<grid, blk, 0, s>>>(vf, txoff, fac, vel64, state, F, rd, W, out, out_c64, records)
        switch (S) {
        case 8: BART_DB_LAUNCH64(8); break;
        case 4: BART_DB_LAUNCH64(4); break;
        case 2: BART_DB_LAUNCH64(2); break;
        default: BART_DB_LAUNCH64(1); break;
        }
#undef BART_DB_LAUNCH64
        return;
    }
    if (NCH < 1 || !partial) NCH = 1;
    const BounceRow *R = static_cast<const BounceRow *>(rows);
    const BounceGeo *G = static_cast<const BounceGeo *>(geo);
    const double tc = bounce_mid_time(rd);
    const unsigned int grid = (unsigned int)((warps * NCH + kDbWarps - 1) / kDbWarps);
#define BART_DB_LAUNCH32(SS) bounce_synth_f32_kernel<SS><<<grid, blk, 0, s>>>(vf, txoff, fac, vel64, state, F, rd, W, out, out_c64, records, R, G, tc, NCH, partial)
    switch (S) {
    case 16: BART_DB_LAUNCH32(16); break;
    case 8: BART_DB_LAUNCH32(8); break;
    case 4: BART_DB_LAUNCH32(4); break;
    case 2: BART_DB_LAUNCH32(2); break;
    default: BART_DB_LAUNCH32(1); break;
    }
#undef BART_DB_LAUNCH32
    if (NCH > 1) {
        const int64_t n = (int64_t)rd.O * rd.N * M;
        bounce_reduce_kernel<<<(unsigned int)((n + 255) / 256), 256, 0, s>>>(partial, n, NCH,
                                                                           out, out_c64);
    }
}

}  // namespace bart
