// BART single-bounce visibility (Sec. 2.2): the forward ray from a TX and the
// backward ray from an RX "meet" on a facet when the facet is lit from the
// TX and seen from the RX.  Each (antenna, facet) pair gets a state from the
// facet-centroid -> antenna segment cast through the LBVH:
//   BACK  (facing away), LIT, GRAZE (within margins: excluded, counted),
//   OCCL  (a robust hit on another facet), LIT_REV (a two-sided facet lit on
//   its reverse side).
// In far-field mode the segment ends at p_a + (c_k - r), r the instance
// origin at the frame start: every facet of an instance looks along the same
// plane-wave direction, over the origin's range.
// The segment/triangle decision is Moller-Trumbore (1997) in FP64 with one
// IEEE rounding per operation in a fixed order (explicit __d*_rn intrinsics:
// no FMA contraction), so states are reproducible bit for bit by any
// IEEE-754 implementation of the same steps.  The BVH boxes are FP32,
// rounded outward and padded, so box culling never drops a candidate.
#include <cuda_runtime.h>
#include <stdint.h>

#include "bart_internal.cuh"
#include "geom64.cuh"

namespace bart {

__global__ void __launch_bounds__(128)
visibility_kernel(const double *__restrict__ tri64, const float4 *__restrict__ tri32,
                  const double *__restrict__ c64, const FacetRec *__restrict__ fac,
                  const double *__restrict__ ref64, const BvhNode *__restrict__ nodes,
                  const int32_t *__restrict__ order, int64_t F, RadarDev rd, SceneSplit sc,
                  uint8_t *__restrict__ state, unsigned long long *n_graze, int *status)
{
    const int64_t gid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int a = blockIdx.y;
    bool graze_flag = false;
    if (gid < F) {
        // threads walk the facets in Morton order so that a warp's segments
        // start close together and traverse similar BVH paths
        const int64_t k = order ? (int64_t)order[gid] : gid;
        const double c[3] = {c64[3 * k], c64[3 * k + 1], c64[3 * k + 2]};
        double pa[3] = {rd.ant[a][0], rd.ant[a][1], rd.ant[a][2]};
        if (rd.far_field) {                 // end = p_a + (c - r): the plane-wave segment
            const double *r0 = ref64 + 3 * fac[k].inst;
            for (int r = 0; r < 3; ++r) pa[r] = __dadd_rn(pa[r], __dsub_rn(c[r], r0[r]));
        }
        double D[3];
        sub3(pa, c, D);
        const float Df[3] = {(float)D[0], (float)D[1], (float)D[2]};
        // FP32 pre-test of the facing test below.  n32 is the unit normal
        // formed in FP64 and rounded (error < 2e-7), Df the rounded segment
        // (relative error 2^-24 per component); with the dot product's and
        // rsqrt's rounding, |cos32 - cos| < 6e-7, so beyond +-(eps_face + 2e-6)
        // the FP64 decision is certain.  Slivers (2A below 1e-6 of the
        // squared edge scale), whose FP64 normal direction is ill-conditioned,
        // always take the FP64 test.
        const bool two = fac[k].two_sided != 0;
        int face = 1;                        // 0 back, 2 front, 3 reverse (two-sided), 1 undecided
        {
            const FacetRec *fr = fac + k;
            const float n0 = fr->n[0], n1 = fr->n[1], n2 = fr->n[2];
            float L2 = 0.f;
#pragma unroll
            for (int v = 0; v < 3; ++v) {
                const float x = fr->dv[3 * v], y = fr->dv[3 * v + 1], z = fr->dv[3 * v + 2];
                L2 = fmaxf(L2, fmaf(x, x, fmaf(y, y, z * z)));
            }
            const float dd = fmaf(Df[0], Df[0], fmaf(Df[1], Df[1], Df[2] * Df[2]));
            const float cos32 = fmaf(n0, Df[0], fmaf(n1, Df[1], n2 * Df[2])) * rsqrtf(dd);
            const float thr = (float)rd.eps_face + 2e-6f;
            if (2.f * fr->area >= 4e-6f * L2 && dd > 0.f) {
                if (cos32 >= thr) face = 2;
                else if (cos32 <= -thr) face = two ? 3 : 0;
            }
        }
        uint8_t st;
        bool graze = false;
        if (face == 1) {
            const double *tk = tri64 + 9 * k;
            double tri[9];
            for (int i = 0; i < 9; ++i) tri[i] = tk[i];
            double e1[3], e2[3], n[3];
            sub3(tri + 3, tri, e1);
            sub3(tri + 6, tri, e2);
            cross3(e1, e2, n);
            const double cosang = __ddiv_rn(
                dot3(n, D), __dmul_rn(__dsqrt_rn(dot3(n, n)), __dsqrt_rn(dot3(D, D))));
            if (dot3(n, n) == 0.0) face = 0;                  // zero area: no normal
            else if (cosang <= -rd.eps_face) face = two ? 3 : 0;
            else graze = fabs(cosang) < rd.eps_face;
        }
        if (face == 0) {
            st = BART_VIS_BACK;
        } else {
            bool hit = false;
            // traversal root: the whole tree, or the subtree of the facet's scene
            int root = F >= 2 ? 0 : -1;
            if (sc.B > 1) {
                int lo = 0, hi = sc.B - 1;          // last scene with foff <= k
                while (lo < hi) {
                    const int mid = (lo + hi + 1) >> 1;
                    if (sc.foff[mid] <= k) lo = mid;
                    else hi = mid - 1;
                }
                root = sc.root[lo];             // < 0: a one-facet scene, nothing to meet
            }
            if (root >= 0) {
                const float o[3] = {(float)c[0], (float)c[1], (float)c[2]};
                const float Dm = fmaxf(fmaxf(fabsf(Df[0]), fabsf(Df[1])), fabsf(Df[2]));
                const float Om = fmaxf(fmaxf(fabsf(o[0]), fabsf(o[1])), fabsf(o[2]));
                float inv[3];
                for (int r = 0; r < 3; ++r) {
                    float d = Df[r];
                    if (fabsf(d) < 1e-30f) d = copysignf(1e-30f, d);
                    inv[r] = 1.0f / d;
                }
                int stack[kStack];
                int sp = 0;
                stack[sp++] = root;
                while (sp > 0 && !hit) {
                    const BvhNode nd = nodes[stack[--sp]];
                    const bool hl = slab_hit(nd.lmin, nd.lmax, o, inv);
                    const bool hr = slab_hit(nd.rmin, nd.rmax, o, inv);
                    const int ch[2] = {nd.left, nd.right};
                    const bool hh[2] = {hl, hr};
                    for (int q = 0; q < 2 && !hit; ++q) {
                        if (!hh[q]) continue;
                        const int cc = ch[q];
                        if (cc < 0) {
                            const int64_t j = ~cc;
                            if (j == k) continue;
                            const int pre = mt_fp32_classify(tri32[3 * j], tri32[3 * j + 1],
                                                             tri32[3 * j + 2], o, Df, Dm, Om);
                            if (pre == 0) continue;
                            if (pre == 2) {             // a certain hit: occluded
                                hit = true;
                                continue;
                            }
                            double tj[9];
                            for (int i = 0; i < 9; ++i) tj[i] = tri64[9 * j + i];
                            const int r = mt_segment(c, D, tj);
                            if (r == 2) hit = true;
                            else if (r == 1) graze = true;
                        } else if (sp < kStack) {
                            stack[sp++] = cc;
                        } else {
                            atomicOr(status, kStatusStackOverflow);
                            graze = true;
                        }
                    }
                }
            }
            st = hit ? BART_VIS_OCCL
                     : (graze ? BART_VIS_GRAZE : (face == 3 ? BART_VIS_LIT_REV : BART_VIS_LIT));
        }
        state[(int64_t)a * F + k] = st;
        graze_flag = (st == BART_VIS_GRAZE);
    }
    const unsigned int b = __ballot_sync(0xffffffffu, graze_flag);
    if ((threadIdx.x & 31) == 0 && b) atomicAdd(n_graze, (unsigned long long)__popc(b));
}

void launch_visibility(const double *tri64, const float *tri32, const double *c64,
                       const FacetRec *fac, const double *ref64, const BvhNode *nodes,
                       const int32_t *order, int64_t F, const RadarDev &rd,
                       const SceneSplit &sc, uint8_t *state, unsigned long long *n_graze,
                       int *status, cudaStream_t s)
{
    const int T = 128;
    dim3 grid((unsigned int)((F + T - 1) / T), (unsigned int)rd.A);
    visibility_kernel<<<grid, T, 0, s>>>(tri64, reinterpret_cast<const float4 *>(tri32), c64,
                                         fac, ref64, nodes, order, F, rd, sc, state, n_graze,
                                         status);
}

// -------------------------------------------------------------------------
// compaction into ascending facet lists: list l < O holds the facets lit
// from TX p AND RX q of channel l = p Q + q on the same side (both LIT, or
// both LIT_REV); list O + a holds the facets lit from antenna a
// -------------------------------------------------------------------------
constexpr int kCompactBlk = 1024;

int64_t compact_blk_words(int64_t F, int L) { return (int64_t)L * ((F + kCompactBlk - 1) / kCompactBlk); }

__device__ __forceinline__ bool in_list(const uint8_t *state, int64_t F, int l, int O, int P,
                                        int Q, int64_t k)
{
    if (l >= O) {
        const uint8_t s = state[(int64_t)(l - O) * F + k];
        return s == BART_VIS_LIT || s == BART_VIS_LIT_REV;
    }
    const int p = l / Q, q = l % Q;
    const uint8_t st = state[(int64_t)p * F + k], sr = state[(int64_t)(P + q) * F + k];
    return st == sr && (st == BART_VIS_LIT || st == BART_VIS_LIT_REV);
}

__global__ void compact_count_kernel(const uint8_t *__restrict__ state, int64_t F, int O, int P,
                                     int Q, int32_t *__restrict__ blk_cnt, int64_t nblk)
{
    const int o = blockIdx.y;
    const int64_t k = (int64_t)blockIdx.x * kCompactBlk + threadIdx.x;
    const bool lit = k < F && in_list(state, F, o, O, P, Q, k);
    const int c = __syncthreads_count(lit);
    if (threadIdx.x == 0) blk_cnt[(int64_t)o * nblk + blockIdx.x] = c;
}

// exclusive scan of each channel's block counts (one warp per channel)
__global__ void compact_scan_kernel(int32_t *__restrict__ blk_cnt, int64_t nblk,
                                    int32_t *__restrict__ vis_cnt)
{
    const int o = blockIdx.x, lane = threadIdx.x;
    int32_t *c = blk_cnt + (int64_t)o * nblk;
    int32_t run = 0;
    for (int64_t b0 = 0; b0 < nblk; b0 += 32) {
        const int64_t b = b0 + lane;
        const int32_t v = b < nblk ? c[b] : 0;
        int32_t x = v;
        for (int off = 1; off < 32; off <<= 1) {
            const int32_t y = __shfl_up_sync(0xffffffffu, x, off);
            if (lane >= off) x += y;
        }
        if (b < nblk) c[b] = run + x - v;
        run += __shfl_sync(0xffffffffu, x, 31);
    }
    if (lane == 0) vis_cnt[o] = run;
}

__global__ void compact_write_kernel(const uint8_t *__restrict__ state, int64_t F, int O, int P,
                                     int Q, const int32_t *__restrict__ blk_cnt, int64_t nblk,
                                     int32_t *__restrict__ vis_idx)
{
    __shared__ int32_t s_w[kCompactBlk / 32];
    const int o = blockIdx.y;
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    const int64_t k = (int64_t)blockIdx.x * kCompactBlk + t;
    const bool lit = k < F && in_list(state, F, o, O, P, Q, k);
    const unsigned int b = __ballot_sync(0xffffffffu, lit);
    if (lane == 0) s_w[warp] = __popc(b);
    __syncthreads();
    if (warp == 0) {
        const int32_t v = s_w[lane];
        int32_t x = v;
        for (int off = 1; off < 32; off <<= 1) {
            const int32_t y = __shfl_up_sync(0xffffffffu, x, off);
            if (lane >= off) x += y;
        }
        s_w[lane] = x - v;
    }
    __syncthreads();
    if (lit) {
        const int32_t pos = blk_cnt[(int64_t)o * nblk + blockIdx.x] + s_w[warp] +
                            __popc(b & ((1u << lane) - 1u));
        vis_idx[(int64_t)o * F + pos] = (int32_t)k;
    }
}

void launch_compact(const uint8_t *state, int64_t F, const RadarDev &rd, int32_t *blk_cnt,
                    int32_t *vis_idx, int32_t *vis_cnt, cudaStream_t s)
{
    const int64_t nblk = (F + kCompactBlk - 1) / kCompactBlk;
    const int L = rd.O + rd.A;
    dim3 grid((unsigned int)nblk, (unsigned int)L);
    compact_count_kernel<<<grid, kCompactBlk, 0, s>>>(state, F, rd.O, rd.P, rd.Q, blk_cnt, nblk);
    compact_scan_kernel<<<L, 32, 0, s>>>(blk_cnt, nblk, vis_cnt);
    compact_write_kernel<<<grid, kCompactBlk, 0, s>>>(state, F, rd.O, rd.P, rd.Q, blk_cnt, nblk,
                                                      vis_idx);
}

// lists are ascending in facet index and scenes own consecutive facets, so
// each (scene, channel) part of list o is one contiguous run
__global__ void scene_lists_kernel(const int32_t *__restrict__ vis_idx,
                                   const int32_t *__restrict__ vis_cnt, int64_t F, int O,
                                   const int64_t *__restrict__ foff, int B,
                                   int32_t *__restrict__ vstart, int32_t *__restrict__ vcnt)
{
    const int v = blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= B * O) return;
    const int b = v / O, o = v % O;
    const int32_t *list = vis_idx + (int64_t)o * F;
    const int n = vis_cnt[o];
    int lim[2];
    for (int e = 0; e < 2; ++e) {           // first entry with facet >= foff[b + e]
        const int64_t key = foff[b + e];
        int lo = 0, hi = n;
        while (lo < hi) {
            const int mid = (lo + hi) >> 1;
            if (list[mid] < key) lo = mid + 1;
            else hi = mid;
        }
        lim[e] = lo;
    }
    vstart[v] = lim[0];
    vcnt[v] = lim[1] - lim[0];
}

void launch_scene_lists(const int32_t *vis_idx, const int32_t *vis_cnt, int64_t F, int O,
                        const int64_t *foff, int B, int32_t *vstart, int32_t *vcnt,
                        cudaStream_t s)
{
    const int T = 128;
    scene_lists_kernel<<<(B * O + T - 1) / T, T, 0, s>>>(vis_idx, vis_cnt, F, O, foff, B, vstart,
                                                         vcnt);
}

}  // namespace bart
