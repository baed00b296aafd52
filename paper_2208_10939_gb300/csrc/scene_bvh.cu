// Scene flattening (world facets at the frame start) and the LBVH builder
// used by the BART visibility rays (Sec. 2.2 ray tracing).
//
// LBVH: 30-bit Morton codes of facet centroids, a stable LSD radix sort,
// the hierarchy of Karras (2012, "Maximizing parallelism in the construction
// of BVHs, octrees, and k-d trees"), and a bottom-up refit with atomics.
#include <cuda_runtime.h>
#include <stdint.h>

#include "bart_internal.cuh"

namespace bart {

// -------------------------------------------------------------------------
// world facets
// -------------------------------------------------------------------------
__device__ __forceinline__ unsigned int f2ord(float x)
{
    unsigned int b = __float_as_uint(x);
    return (b & 0x80000000u) ? ~b : (b | 0x80000000u);
}
__device__ __forceinline__ float ord2f(unsigned int u)
{
    return __uint_as_float((u & 0x80000000u) ? (u & 0x7fffffffu) : ~u);
}

// Rigid transform with one IEEE rounding per operation, in a fixed order:
//   w = ((r0 x + r1 y) + r2 z) + p;  w = w + v t
__device__ __forceinline__ double world_coord(const double *r, double x, double y, double z,
                                              double p, double v, double t)
{
    double w = __dmul_rn(r[0], x);
    w = __dadd_rn(w, __dmul_rn(r[1], y));
    w = __dadd_rn(w, __dmul_rn(r[2], z));
    w = __dadd_rn(w, p);
    w = __dadd_rn(w, __dmul_rn(v, t));
    return w;
}

__global__ void build_facets_kernel(const MeshDesc *__restrict__ meshes,
                                    const InstDev *__restrict__ insts, int n_inst, int64_t F,
                                    double t0, double *__restrict__ tri64,
                                    float *__restrict__ tri32,
                                    double *__restrict__ c64, FacetRec *__restrict__ fac,
                                    float *__restrict__ aabb, float *__restrict__ vel32,
                                    unsigned int *__restrict__ bounds,
                                    double *__restrict__ ref64, float *__restrict__ ref32,
                                    float *__restrict__ fac_lo)
{
    const int64_t f = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    float cf[3] = {0.f, 0.f, 0.f};
    const bool valid = f < F;
    if (valid) {
        int lo = 0, hi = n_inst - 1;            // last instance with off <= f
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (insts[mid].off <= f) lo = mid;
            else hi = mid - 1;
        }
        const InstDev &in = insts[lo];
        const MeshDesc &m = meshes[in.mesh];
        const int64_t j = f - in.off;
        double v[9];
        for (int k = 0; k < 3; ++k) {
            const int64_t vi = m.tris[3 * j + k];
            const double x = m.verts[3 * vi], y = m.verts[3 * vi + 1], z = m.verts[3 * vi + 2];
            for (int r = 0; r < 3; ++r)
                v[3 * k + r] = world_coord(in.rot + 3 * r, x, y, z, in.pos[r], in.vel[r], t0);
        }
        float vmax = 0.f;
        for (int i = 0; i < 9; ++i) {
            tri64[9 * f + i] = v[i];
            const float vf = (float)v[i];
            tri32[12 * f + i] = vf;
            vmax = fmaxf(vmax, fabsf(vf));
        }
        tri32[12 * f + 9] = vmax;
        tri32[12 * f + 10] = 0.f;
        tri32[12 * f + 11] = 0.f;
        double c[3];
        for (int r = 0; r < 3; ++r) {
            c[r] = __ddiv_rn(__dadd_rn(__dadd_rn(v[r], v[3 + r]), v[6 + r]), 3.0);
            c64[3 * f + r] = c[r];
        }
        const double e1[3] = {v[3] - v[0], v[4] - v[1], v[5] - v[2]};
        const double e2[3] = {v[6] - v[0], v[7] - v[1], v[8] - v[2]};
        const double nx = e1[1] * e2[2] - e1[2] * e2[1];
        const double ny = e1[2] * e2[0] - e1[0] * e2[2];
        const double nz = e1[0] * e2[1] - e1[1] * e2[0];
        const double nl = sqrt(nx * nx + ny * ny + nz * nz);
        FacetRec rec;
        for (int r = 0; r < 3; ++r) {
            rec.c[r] = (float)c[r];
            cf[r] = rec.c[r];
        }
        rec.area = (float)(0.5 * nl);
        for (int r = 0; r < 3; ++r) fac_lo[12 * f + r] = (float)(c[r] - (double)rec.c[r]);
        for (int k = 0; k < 3; ++k)
            for (int r = 0; r < 3; ++r) {
                const double d = v[3 * k + r] - c[r];
                rec.dv[3 * k + r] = (float)d;
                fac_lo[12 * f + 3 + 3 * k + r] = (float)(d - (double)rec.dv[3 * k + r]);
            }
        const double inl = nl > 0.0 ? 1.0 / nl : 0.0;
        rec.n[0] = (float)(nx * inl);
        rec.n[1] = (float)(ny * inl);
        rec.n[2] = (float)(nz * inl);
        rec.rho = m.rho ? m.rho[j] * in.rho_scale : in.rho_scale;
        rec.inst = lo;
        rec.two_sided = m.two_sided;
        rec.pad = 0.f;
        fac[f] = rec;
        // conservative FP32 box: outward rounding plus a pad covering the
        // FP32 slab test of a segment of <= ~200 m length
        float mx = 0.f;
        for (int r = 0; r < 3; ++r) {
            double lo_ = fmin(fmin(v[r], v[3 + r]), v[6 + r]);
            double hi_ = fmax(fmax(v[r], v[3 + r]), v[6 + r]);
            mx = fmaxf(mx, fmaxf(fabsf((float)lo_), fabsf((float)hi_)));
            aabb[6 * f + r] = __double2float_rd(lo_);
            aabb[6 * f + 3 + r] = __double2float_ru(hi_);
        }
        const float pad = 1e-4f + 4e-6f * mx;
        for (int r = 0; r < 3; ++r) {
            aabb[6 * f + r] -= pad;
            aabb[6 * f + 3 + r] += pad;
        }
        if (j == 0) {
            for (int r = 0; r < 3; ++r) {
                vel32[4 * lo + r] = (float)in.vel[r];
                // the instance origin at t0 (reference point of the delay form)
                const double o = world_coord(in.rot + 3 * r, 0.0, 0.0, 0.0, in.pos[r], in.vel[r], t0);
                ref64[3 * lo + r] = o;
                ref32[4 * lo + r] = (float)o;
            }
            vel32[4 * lo + 3] = 0.f;
            ref32[4 * lo + 3] = 0.f;
        }
    }
    // centroid bounds for the Morton grid
    __shared__ unsigned int s_b[6];
    if (threadIdx.x < 6) s_b[threadIdx.x] = threadIdx.x < 3 ? 0xffffffffu : 0u;
    __syncthreads();
    if (valid)
        for (int r = 0; r < 3; ++r) {
            atomicMin(&s_b[r], f2ord(cf[r]));
            atomicMax(&s_b[3 + r], f2ord(cf[r]));
        }
    __syncthreads();
    if (threadIdx.x < 3) atomicMin(&bounds[threadIdx.x], s_b[threadIdx.x]);
    else if (threadIdx.x < 6) atomicMax(&bounds[threadIdx.x], s_b[threadIdx.x]);
}

const void *build_facets_kernel_fn(int *t0_arg_index, int *n_args)
{
    *t0_arg_index = 4;      // meshes, insts, n_inst, F, t0, tri64, tri32, c64, fac, aabb,
    *n_args = 15;           // vel32, bounds, ref64, ref32, fac_lo
    return reinterpret_cast<const void *>(build_facets_kernel);
}

void launch_build_facets(const MeshDesc *meshes, const InstDev *insts, int n_inst, int64_t F,
                         double t0, double *tri64, float *tri32, double *c64, FacetRec *fac,
                         float *aabb, float *vel32, unsigned int *bounds, double *ref64,
                         float *ref32, float *fac_lo, cudaStream_t s)
{
    cudaMemsetAsync(bounds, 0xff, 3 * sizeof(unsigned int), s);
    cudaMemsetAsync(bounds + 3, 0, 3 * sizeof(unsigned int), s);
    const int T = 256;
    const unsigned int G = (unsigned int)((F + T - 1) / T);
    build_facets_kernel<<<G, T, 0, s>>>(meshes, insts, n_inst, F, t0, tri64, tri32, c64, fac,
                                        aabb, vel32, bounds, ref64, ref32, fac_lo);
}

// -------------------------------------------------------------------------
// Morton codes
// -------------------------------------------------------------------------
__device__ __forceinline__ uint32_t spread10(uint32_t x)
{
    x &= 0x3ffu;
    x = (x | (x << 16)) & 0x030000ffu;
    x = (x | (x << 8)) & 0x0300f00fu;
    x = (x | (x << 4)) & 0x030c30c3u;
    x = (x | (x << 2)) & 0x09249249u;
    return x;
}

__global__ void morton_kernel(const FacetRec *__restrict__ fac, int64_t F,
                              const unsigned int *__restrict__ bounds,
                              uint32_t *__restrict__ keys, int32_t *__restrict__ vals)
{
    const int64_t f = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (f >= F) return;
    uint32_t code = 0;
    for (int r = 0; r < 3; ++r) {
        const float lo = ord2f(bounds[r]), hi = ord2f(bounds[3 + r]);
        const float ext = hi - lo;
        float u = ext > 0.f ? (fac[f].c[r] - lo) / ext : 0.f;
        u = fminf(fmaxf(u, 0.f), 1.f);
        const uint32_t q = (uint32_t)fminf(u * 1024.f, 1023.f);
        code |= spread10(q) << (2 - r);
    }
    keys[f] = code;
    vals[f] = (int32_t)f;
}

void launch_morton(const FacetRec *fac, int64_t F, const unsigned int *bounds, uint32_t *keys,
                   int32_t *vals, cudaStream_t s)
{
    const int T = 256;
    morton_kernel<<<(unsigned int)((F + T - 1) / T), T, 0, s>>>(fac, F, bounds, keys, vals);
}

// -------------------------------------------------------------------------
// stable LSD radix sort, 8-bit digits
// -------------------------------------------------------------------------
constexpr int kSortThreads = 256;
constexpr int kSortTile = 2048;     // keys per block

static inline int64_t sort_blocks(int64_t n) { return (n + kSortTile - 1) / kSortTile; }

int64_t radix_sort_temp_words(int64_t n) { return 256 * sort_blocks(n) + 1; }

__global__ void rs_hist_kernel(const uint32_t *__restrict__ keys, int64_t n, int shift,
                               uint32_t *__restrict__ hist, int64_t nblk)
{
    __shared__ uint32_t h[256];
    h[threadIdx.x] = 0;
    __syncthreads();
    const int64_t base = (int64_t)blockIdx.x * kSortTile;
    for (int i = threadIdx.x; i < kSortTile; i += kSortThreads) {
        const int64_t idx = base + i;
        if (idx < n) atomicAdd(&h[(keys[idx] >> shift) & 0xffu], 1u);
    }
    __syncthreads();
    hist[(int64_t)threadIdx.x * nblk + blockIdx.x] = h[threadIdx.x];
}

// exclusive scan of `len` words in place, one block of 1024 threads
__global__ void rs_scan_kernel(uint32_t *__restrict__ data, int64_t len)
{
    __shared__ uint32_t s_part[1024];
    const int t = threadIdx.x;
    const int64_t chunk = (len + 1023) / 1024;
    const int64_t b = t * chunk, e = b + chunk < len ? b + chunk : len;
    uint32_t sum = 0;
    for (int64_t i = b; i < e; ++i) sum += data[i];
    s_part[t] = sum;
    __syncthreads();
    for (int off = 1; off < 1024; off <<= 1) {
        const uint32_t v = t >= off ? s_part[t - off] : 0u;
        __syncthreads();
        s_part[t] += v;
        __syncthreads();
    }
    uint32_t run = s_part[t] - sum;     // exclusive prefix of this chunk
    for (int64_t i = b; i < e; ++i) {
        const uint32_t v = data[i];
        data[i] = run;
        run += v;
    }
}

__global__ void rs_scatter_kernel(const uint32_t *__restrict__ keys_in,
                                  const int32_t *__restrict__ vals_in, int64_t n, int shift,
                                  const uint32_t *__restrict__ hist, int64_t nblk,
                                  uint32_t *__restrict__ keys_out, int32_t *__restrict__ vals_out)
{
    constexpr int W = kSortThreads / 32;
    __shared__ uint32_t s_base[256];
    __shared__ uint32_t s_wcnt[W][256];
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    s_base[t] = hist[(int64_t)t * nblk + blockIdx.x];
    const int64_t base = (int64_t)blockIdx.x * kSortTile;
    const unsigned int lt = (1u << lane) - 1u;
    for (int r = 0; r < kSortTile / kSortThreads; ++r) {
        for (int w = 0; w < W; ++w) s_wcnt[w][t] = 0;
        __syncthreads();
        const int64_t idx = base + (int64_t)r * kSortThreads + t;
        const bool valid = idx < n;
        uint32_t key = 0;
        int32_t val = 0;
        int d = 256;                                   // invalid items form their own group
        if (valid) {
            key = keys_in[idx];
            val = vals_in[idx];
            d = (key >> shift) & 0xff;
        }
        const unsigned int peers = __match_any_sync(0xffffffffu, d);
        const int rank = __popc(peers & lt);
        if (valid && rank == 0) s_wcnt[warp][d] = __popc(peers);
        __syncthreads();
        if (valid) {
            uint32_t pos = s_base[d] + rank;
            for (int w = 0; w < warp; ++w) pos += s_wcnt[w][d];
            keys_out[pos] = key;
            vals_out[pos] = val;
        }
        __syncthreads();
        uint32_t tot = 0;
        for (int w = 0; w < W; ++w) tot += s_wcnt[w][t];
        s_base[t] += tot;
        __syncthreads();
    }
}

void radix_sort_pairs(uint32_t *keys, int32_t *vals, uint32_t *keys_tmp, int32_t *vals_tmp,
                      uint32_t *temp, int64_t n, int bits, cudaStream_t s)
{
    const int64_t nblk = sort_blocks(n);
    uint32_t *ka = keys, *kb = keys_tmp;
    int32_t *va = vals, *vb = vals_tmp;
    int passes = (bits + 7) / 8;
    if (passes & 1) passes += 1;                      // even: result lands in `keys`
    for (int p = 0; p < passes; ++p) {
        const int shift = 8 * p;
        rs_hist_kernel<<<(unsigned int)nblk, kSortThreads, 0, s>>>(ka, n, shift, temp, nblk);
        rs_scan_kernel<<<1, 1024, 0, s>>>(temp, 256 * nblk);
        rs_scatter_kernel<<<(unsigned int)nblk, kSortThreads, 0, s>>>(ka, va, n, shift, temp,
                                                                      nblk, kb, vb);
        uint32_t *tk = ka; ka = kb; kb = tk;
        int32_t *tv = va; va = vb; vb = tv;
    }
}

// -------------------------------------------------------------------------
// Karras hierarchy
// -------------------------------------------------------------------------
// Common-prefix length of sorted leaves i and j (-1 outside [0, n)).  With
// batched scenes the key is (scene, Morton code, index): leaves of
// different scenes compare on the scene id alone (0..31), so every scene's
// leaves form one subtree; equal codes fall back to the index.
__device__ __forceinline__ int delta(const uint32_t *keys, const uint32_t *scene, int64_t n,
                                     int64_t i, int64_t j)
{
    if (j < 0 || j >= n) return -1;
    if (scene) {
        const uint32_t sa = scene[i], sb = scene[j];
        if (sa != sb) return __clz((int)(sa ^ sb));
    }
    const uint32_t a = keys[i], b = keys[j];
    if (a == b) return 64 + __clz((int)(i ^ j));      // index tie-break for equal codes
    return 32 + __clz((int)(a ^ b));
}

__global__ void lbvh_build_kernel(const uint32_t *__restrict__ keys,
                                  const uint32_t *__restrict__ scene,
                                  const int32_t *__restrict__ vals, int64_t n,
                                  BvhNode *__restrict__ nodes, int32_t *__restrict__ parent,
                                  int32_t *__restrict__ leaf_parent, int32_t *__restrict__ root)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n - 1) return;
    const int d = (delta(keys, scene, n, i, i + 1) - delta(keys, scene, n, i, i - 1)) >= 0 ? 1 : -1;
    const int dmin = delta(keys, scene, n, i, i - d);
    int64_t lmax = 2;
    while (delta(keys, scene, n, i, i + lmax * d) > dmin) lmax <<= 1;
    int64_t l = 0;
    for (int64_t t = lmax >> 1; t >= 1; t >>= 1)
        if (delta(keys, scene, n, i, i + (l + t) * d) > dmin) l += t;
    const int64_t j = i + l * d;
    const int dnode = delta(keys, scene, n, i, j);
    int64_t sp = 0;
    int64_t t = l;
    do {
        t = (t + 1) >> 1;
        if (delta(keys, scene, n, i, i + (sp + t) * d) > dnode) sp += t;
    } while (t > 1);
    const int64_t gamma = i + sp * d + (d < 0 ? -1 : 0);
    const int64_t lo = i < j ? i : j, hi = i < j ? j : i;
    int left, right;
    if (lo == gamma) {
        left = ~vals[gamma];
        leaf_parent[gamma] = (int32_t)i;
    } else {
        left = (int)gamma;
        parent[gamma] = (int32_t)i;
    }
    if (hi == gamma + 1) {
        right = ~vals[gamma + 1];
        leaf_parent[gamma + 1] = (int32_t)i;
    } else {
        right = (int)(gamma + 1);
        parent[gamma + 1] = (int32_t)i;
    }
    nodes[i].left = left;
    nodes[i].right = right;
    if (i == 0) parent[0] = -1;
    if (scene) {
        // the node covering exactly one scene's leaves is that scene's root
        const uint32_t sc = scene[lo];
        if (scene[hi] == sc && (lo == 0 || scene[lo - 1] != sc) && (hi == n - 1 || scene[hi + 1] != sc))
            root[sc] = (int32_t)i;
    }
}

void launch_lbvh_build(const uint32_t *keys, const int32_t *vals, int64_t n, BvhNode *nodes,
                       int32_t *parent, int32_t *leaf_parent, cudaStream_t s)
{
    if (n < 2) return;
    const int T = 256;
    lbvh_build_kernel<<<(unsigned int)((n - 1 + T - 1) / T), T, 0, s>>>(
        keys, nullptr, vals, n, nodes, parent, leaf_parent, nullptr);
}

// scene of each sorted leaf: facets [foff[b], foff[b+1]) belong to scene b
__global__ void scene_keys_kernel(const int32_t *__restrict__ vals, int64_t n,
                                  const int64_t *__restrict__ foff, int B,
                                  uint32_t *__restrict__ skeys)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int64_t f = vals[i];
    int lo = 0, hi = B - 1;                 // last scene with foff <= f
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (foff[mid] <= f) lo = mid;
        else hi = mid - 1;
    }
    skeys[i] = (uint32_t)lo;
}

__global__ void gather_keys_kernel(const int32_t *__restrict__ vals, int64_t n,
                                   const uint32_t *__restrict__ by_facet, uint32_t *__restrict__ keys)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) keys[i] = by_facet[vals[i]];
}

// one-facet scenes have their leaf as root; the others get theirs from the build
__global__ void scene_root_init_kernel(const int64_t *__restrict__ foff, int B,
                                       int32_t *__restrict__ root)
{
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b < B) root[b] = foff[b + 1] - foff[b] == 1 ? ~(int32_t)foff[b] : 0;
}

void launch_lbvh_batched(const FacetRec *fac, int64_t F, const unsigned int *bounds,
                         const int64_t *foff, int B, uint32_t *keys, int32_t *vals,
                         uint32_t *keys_tmp, int32_t *vals_tmp, uint32_t *temp, uint32_t *mkeys,
                         uint32_t *skeys, BvhNode *nodes, int32_t *parent, int32_t *leaf_parent,
                         int32_t *root, cudaStream_t s)
{
    const int T = 256;
    const unsigned int G = (unsigned int)((F + T - 1) / T);
    launch_morton(fac, F, bounds, keys, vals, s);
    cudaMemcpyAsync(mkeys, keys, (size_t)F * sizeof(uint32_t), cudaMemcpyDeviceToDevice, s);
    radix_sort_pairs(keys, vals, keys_tmp, vals_tmp, temp, F, 30, s);
    scene_keys_kernel<<<G, T, 0, s>>>(vals, F, foff, B, skeys);
    int sbits = 1;
    while ((1 << sbits) < B) ++sbits;
    radix_sort_pairs(skeys, vals, keys_tmp, vals_tmp, temp, F, sbits, s);   // stable
    gather_keys_kernel<<<G, T, 0, s>>>(vals, F, mkeys, keys);
    scene_root_init_kernel<<<(B + T - 1) / T, T, 0, s>>>(foff, B, root);
    if (F < 2) return;
    lbvh_build_kernel<<<(unsigned int)((F - 1 + T - 1) / T), T, 0, s>>>(
        keys, skeys, vals, F, nodes, parent, leaf_parent, root);
}

int lbvh_batched_launches(int B)
{
    int sbits = 1;
    while ((1 << sbits) < B) ++sbits;
    int p2 = (sbits + 7) / 8;
    if (p2 & 1) ++p2;
    return 1 + 3 * 4 + 1 + 3 * p2 + 1 + 1 + 1;
}

// bottom-up refit: each leaf writes its box into its parent's slot; the
// second thread to reach a node merges both slots and climbs on.
__global__ void lbvh_refit_kernel(const int32_t *__restrict__ vals,
                                  const float *__restrict__ aabb, int64_t n,
                                  BvhNode *nodes, const int32_t *__restrict__ parent,
                                  const int32_t *__restrict__ leaf_parent, int32_t *flags)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int32_t f = vals[i];
    float bmin[3], bmax[3];
    for (int r = 0; r < 3; ++r) {
        bmin[r] = aabb[6 * (int64_t)f + r];
        bmax[r] = aabb[6 * (int64_t)f + 3 + r];
    }
    int child_code = ~f;
    int p = leaf_parent[i];
    while (p >= 0) {
        BvhNode *nd = nodes + p;
        const bool is_left = (nd->left == child_code);
        float *smin = is_left ? nd->lmin : nd->rmin;
        float *smax = is_left ? nd->lmax : nd->rmax;
        for (int r = 0; r < 3; ++r) {
            __stcg(smin + r, bmin[r]);
            __stcg(smax + r, bmax[r]);
        }
        __threadfence();
        if (atomicAdd(flags + p, 1) == 0) return;      // sibling not done yet
        __threadfence();
        for (int r = 0; r < 3; ++r) {
            bmin[r] = fminf(__ldcg(nd->lmin + r), __ldcg(nd->rmin + r));
            bmax[r] = fmaxf(__ldcg(nd->lmax + r), __ldcg(nd->rmax + r));
        }
        child_code = p;
        p = parent[p];
    }
}

void launch_lbvh_refit(const int32_t *vals, const float *aabb, int64_t n, BvhNode *nodes,
                       const int32_t *parent, const int32_t *leaf_parent, int32_t *flags,
                       cudaStream_t s)
{
    if (n < 2) return;
    cudaMemsetAsync(flags, 0, (size_t)(n - 1) * sizeof(int32_t), s);
    const int T = 256;
    lbvh_refit_kernel<<<(unsigned int)((n + T - 1) / T), T, 0, s>>>(vals, aabb, n, nodes, parent,
                                                                   leaf_parent, flags);
}

}  // namespace bart
