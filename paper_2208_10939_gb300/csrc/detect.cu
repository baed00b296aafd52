// Radar point cloud from the range-Doppler map (Sec. 3.3, Eqs. 4-6).
//
//  1. RDM with the complex cube kept: Y[o][r][d'] (rdm.cu).
//  2. cfar_kernel: cell-averaging CFAR.  A block owns TR whole range rows
//     (TR * N <= 1024 cells, TR | M), so the cyclic Doppler neighbourhood of every
//     cell is inside the block.  Vertical partial sums first, per column:
//       vout[r][c] = sum_{gr < |u| <= hr} P[r+u][c]   (rows outside the guard)
//       vmid[r][c] = sum_{|u| <= gr}       P[r+u][c]   (rows of the guard)
//     then per cell the training sum
//       T = sum_{|k| <= hd} vout[r][c+k] + sum_{gd < |k| <= hd} vmid[r][c+k],
//     every term a training cell, no cancellation.  FP64 sums of the FP32
//     RDM; detection when (double)P > alpha * (T / n_train).
//  3. emit_kernel: ordered compaction of the flags into row-major cell
//     indices (per-block counts, block-local scan).
//  4. steer_kernel: steering table E[o][i] = exp(+j 2 pi a_o s_i) with
//     a_o = x_o / lambda_c, s_i = -1 + 2 i / bins; the phase 2 a_o s_i is
//     formed and reduced mod 2 in FP64, the sine/cosine taken in the FFT's
//     precision.
//  5. angle_kernel: per detection, S_i = |sum_o E[o][i] Y_o|^2 over the
//     grid, first maximum -> azimuth; range and rate from the bins.
#include <cuda_runtime.h>
#include <stdint.h>

#include "bart_internal.cuh"

namespace bart {

namespace {

template <typename T> struct Cx;
template <> struct Cx<float> { using type = float2; };
template <> struct Cx<double> { using type = double2; };

__device__ __forceinline__ void sincospi_p(float x, float *s, float *c) { sincospif(x, s, c); }
__device__ __forceinline__ void sincospi_p(double x, double *s, double *c) { sincospi(x, s, c); }

constexpr int kCfarThreads = 256;
constexpr int kCfarCells = 1024;      // cells per CFAR block (TR * N)
constexpr int kAngleThreads = 256;
constexpr int kAngleBlocks = 4 * 152;

// whole range rows per CFAR block: the largest power of two TR with
// TR N <= kCfarCells that divides M
int rows_per_block(int M, int N)
{
    int tr = 1;
    while (2 * tr * N <= kCfarCells && M % (2 * tr) == 0) tr *= 2;
    return tr;
}

__global__ void __launch_bounds__(kCfarThreads)
cfar_kernel(const float *__restrict__ P, int M, int N, int TR, DetectDev dd,
            uint8_t *__restrict__ flag, int32_t *__restrict__ blk_cnt)
{
    __shared__ double vout[kCfarCells];
    __shared__ double vmid[kCfarCells];
    const int r0 = blockIdx.x * TR;
    const int cells = TR * N;
    const int gr = dd.guard_r, hr = dd.hr, gd = dd.guard_d, hd = dd.hd;
    for (int i = threadIdx.x; i < cells; i += blockDim.x) {
        const int r = r0 + i / N, c = i % N;
        if (r < hr || r >= M - hr) continue;
        const float *col = P + c;
        double sm = (double)col[(int64_t)r * N];
        for (int u = 1; u <= gr; ++u)
            sm += (double)col[(int64_t)(r - u) * N] + (double)col[(int64_t)(r + u) * N];
        double so = 0.0;
        for (int u = gr + 1; u <= hr; ++u)
            so += (double)col[(int64_t)(r - u) * N] + (double)col[(int64_t)(r + u) * N];
        vout[i] = so;
        vmid[i] = sm;
    }
    __syncthreads();
    int found = 0;
    for (int base = 0; base < cells; base += blockDim.x) {
        const int i = base + threadIdx.x;
        int det = 0;
        if (i < cells) {
            const int j = i / N, c = i % N, r = r0 + j;
            if (r >= hr && r < M - hr) {
                const double *vo = vout + j * N;
                const double *vm = vmid + j * N;
                double t = vo[c];
                // cyclic Doppler neighbours (hd < N/2)
                for (int k = 1; k <= hd; ++k) {
                    const int lo = c - k < 0 ? c - k + N : c - k, hi = c + k >= N ? c + k - N : c + k;
                    t += vo[lo] + vo[hi];
                }
                for (int k = gd + 1; k <= hd; ++k) {
                    const int lo = c - k < 0 ? c - k + N : c - k, hi = c + k >= N ? c + k - N : c + k;
                    t += vm[lo] + vm[hi];
                }
                const double thr = dd.alpha * (t / (double)dd.n_train);
                det = (double)P[(int64_t)r * N + c] > thr;
            }
            flag[(int64_t)r0 * N + i] = (uint8_t)det;
        }
        found += __syncthreads_count(det);
    }
    if (threadIdx.x == 0) blk_cnt[blockIdx.x] = found;
}

// exclusive prefix sum of one int per thread over the block (blockDim 256)
__device__ int block_exclusive_scan(int v, int *total)
{
    __shared__ int warp_sum[32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int x = v;
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) warp_sum[warp] = x;
    __syncthreads();
    if (warp == 0) {
        const int nw = blockDim.x >> 5;
        int w = lane < nw ? warp_sum[lane] : 0;
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o) w += y;
        }
        if (lane < nw) warp_sum[lane] = w;
    }
    __syncthreads();
    const int before = (warp > 0 ? warp_sum[warp - 1] : 0) + x - v;
    *total = warp_sum[(blockDim.x >> 5) - 1];
    __syncthreads();
    return before;
}

// one block per CFAR block: row-major ranks of its detections
__global__ void __launch_bounds__(kCfarThreads)
emit_kernel(const uint8_t *__restrict__ flag, const int32_t *__restrict__ blk_cnt, int nblk,
            int cells, int32_t *__restrict__ list, int32_t *__restrict__ count)
{
    __shared__ int off_s;
    if (threadIdx.x == 0) {
        int off = 0;
        for (int b = 0; b < blockIdx.x; ++b) off += blk_cnt[b];
        off_s = off;
        if (blockIdx.x == nblk - 1) *count = off + blk_cnt[blockIdx.x];
    }
    __syncthreads();
    if (blk_cnt[blockIdx.x] == 0) return;
    const int per = (cells + blockDim.x - 1) / blockDim.x;   // consecutive cells per thread
    const int64_t base = (int64_t)blockIdx.x * cells;
    const int c0 = threadIdx.x * per;
    int mine = 0;
    for (int k = 0; k < per; ++k)
        if (c0 + k < cells) mine += flag[base + c0 + k];
    int total = 0;
    int at = off_s + block_exclusive_scan(mine, &total);
    for (int k = 0; k < per && mine; ++k)
        if (c0 + k < cells && flag[base + c0 + k]) {
            list[at++] = (int32_t)(base + c0 + k);
            --mine;
        }
}

template <typename T>
__global__ void steer_kernel(RadarDev rd, double lam_c, int bins,
                             typename Cx<T>::type *__restrict__ E)
{
    const int64_t n = (int64_t)rd.O * bins;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int o = (int)(i / bins), b = (int)(i % bins);
        const int p = o / rd.Q, q = o % rd.Q;
        const double a = (rd.ant[p][0] + rd.ant[rd.P + q][0]) / lam_c;
        const double sv = -1.0 + 2.0 * (double)b / (double)bins;
        double t = 2.0 * a * sv;            // phase / pi
        t -= 2.0 * rint(0.5 * t);           // into [-1, 1]
        T s, c;
        sincospi_p((T)t, &s, &c);
        typename Cx<T>::type e;
        e.x = c;
        e.y = s;
        E[i] = e;
    }
}

template <typename T>
__global__ void __launch_bounds__(kAngleThreads)
angle_kernel(const typename Cx<T>::type *__restrict__ Y, const typename Cx<T>::type *__restrict__ E,
             const float *__restrict__ rdm, const int32_t *__restrict__ list,
             const int32_t *__restrict__ count, int max_points, int O, int M, int N,
             DetectDev dd, bart_point *__restrict__ pts)
{
    using C = typename Cx<T>::type;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C *yo = reinterpret_cast<C *>(smem_raw);
    __shared__ T best_v[kAngleThreads / 32];
    __shared__ int best_i[kAngleThreads / 32];
    const int n = min(*count, max_points);
    const int64_t MN = (int64_t)M * N;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int det = blockIdx.x; det < n; det += gridDim.x) {
        const int cell = list[det];
        for (int o = threadIdx.x; o < O; o += blockDim.x) yo[o] = Y[(int64_t)o * MN + cell];
        __syncthreads();
        T bv = (T)-1;
        int bi = 0;
        for (int i = threadIdx.x; i < dd.bins; i += blockDim.x) {
            T re = (T)0, im = (T)0;
            for (int o = 0; o < O; ++o) {
                const C e = E[(int64_t)o * dd.bins + i], y = yo[o];
                re += e.x * y.x - e.y * y.y;
                im += e.x * y.y + e.y * y.x;
            }
            const T pw = re * re + im * im;
            if (pw > bv) {          // strict: first maximum of this thread's bins
                bv = pw;
                bi = i;
            }
        }
        // larger power wins; equal power: lower bin
        for (int o = 16; o > 0; o >>= 1) {
            const T v2 = __shfl_down_sync(0xffffffffu, bv, o);
            const int i2 = __shfl_down_sync(0xffffffffu, bi, o);
            if (v2 > bv || (v2 == bv && i2 < bi)) {
                bv = v2;
                bi = i2;
            }
        }
        if (lane == 0) {
            best_v[warp] = bv;
            best_i[warp] = bi;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            for (int w = 1; w < (int)(blockDim.x >> 5); ++w)
                if (best_v[w] > bv || (best_v[w] == bv && best_i[w] < bi)) {
                    bv = best_v[w];
                    bi = best_i[w];
                }
            const int r = cell / N, d = cell % N;
            const double sv = -1.0 + 2.0 * (double)bi / (double)dd.bins;
            const double az = asin(fmin(1.0, fmax(-1.0, sv)));
            bart_point pt;
            pt.range = dd.range_scale * (double)r;
            pt.rate = dd.rate_scale * (double)(d - N / 2);
            pt.azimuth = az;
            pt.x = pt.range * sin(az);
            pt.y = pt.range * cos(az);
            pt.power = (double)rdm[cell];
            pt.r_bin = r;
            pt.d_bin = d;
            pts[det] = pt;
        }
        __syncthreads();
    }
}

int64_t align256(int64_t b) { return (b + 255) & ~(int64_t)255; }

}  // namespace

int64_t detect_workspace_bytes(const RadarDev &rd, int dtype, int bins)
{
    const int64_t ce = dtype == BART_C64 ? 8 : 16;
    const int64_t MN = (int64_t)rd.M * rd.N, cube = (int64_t)rd.O * MN * ce;
    const int64_t nblk = MN / ((int64_t)rows_per_block(rd.M, rd.N) * rd.N);
    return 2 * align256(cube) + align256(MN * 4) + align256((int64_t)rd.O * bins * ce) +
           align256(MN) + align256(nblk * 4) + align256(MN * 4) + align256(4);
}

void detect_carve(void *ws, const RadarDev &rd, int dtype, int bins, DetectBufs *b)
{
    const int64_t ce = dtype == BART_C64 ? 8 : 16;
    const int64_t MN = (int64_t)rd.M * rd.N, cube = (int64_t)rd.O * MN * ce;
    const int64_t nblk = MN / ((int64_t)rows_per_block(rd.M, rd.N) * rd.N);
    unsigned char *p = static_cast<unsigned char *>(ws);
    b->X = p;                                   p += align256(cube);
    b->cube = p;                                p += align256(cube);
    b->rdm = reinterpret_cast<float *>(p);      p += align256(MN * 4);
    b->steer = p;                               p += align256((int64_t)rd.O * bins * ce);
    b->flag = p;                                p += align256(MN);
    b->blk_cnt = reinterpret_cast<int32_t *>(p); p += align256(nblk * 4);
    b->list = reinterpret_cast<int32_t *>(p);   p += align256(MN * 4);
    b->count = reinterpret_cast<int32_t *>(p);
}

template <typename T>
static void run_angle(const RadarDev &rd, const DetectDev &dd, const DetectBufs &b,
                      const float *rdm, bart_point *points, int max_points, cudaStream_t s)
{
    using C = typename Cx<T>::type;
    const int64_t ne = (int64_t)rd.O * dd.bins;
    const int sb = (int)((ne + 255) / 256 < 4 * 152 ? (ne + 255) / 256 : 4 * 152);
    steer_kernel<T><<<sb, 256, 0, s>>>(rd, dd.lam_c, dd.bins, reinterpret_cast<C *>(b.steer));
    if (max_points <= 0) return;
    const size_t smem = (size_t)rd.O * sizeof(C);
    angle_kernel<T><<<kAngleBlocks, kAngleThreads, smem, s>>>(
        reinterpret_cast<const C *>(b.cube), reinterpret_cast<const C *>(b.steer), rdm, b.list,
        b.count, max_points, rd.O, rd.M, rd.N, dd, points);
}

int launch_detect(const void *adc, int dtype, const RadarDev &rd, const DetectDev &dd,
                  const DetectBufs &b, bart_point *points, int max_points, cudaStream_t s)
{
    launch_rdm_cube(adc, dtype, rd, b.X, b.cube, b.rdm, s);
    const int TR = rows_per_block(rd.M, rd.N);
    const int nblk = rd.M / TR;
    cfar_kernel<<<nblk, kCfarThreads, 0, s>>>(b.rdm, rd.M, rd.N, TR, dd, b.flag, b.blk_cnt);
    emit_kernel<<<nblk, kCfarThreads, 0, s>>>(b.flag, b.blk_cnt, nblk, TR * rd.N, b.list,
                                             b.count);
    if (dtype == BART_C64) run_angle<float>(rd, dd, b, b.rdm, points, max_points, s);
    else run_angle<double>(rd, dd, b, b.rdm, points, max_points, s);
    return 3 + 3 + (max_points > 0 ? 1 : 0);
}

}  // namespace bart
