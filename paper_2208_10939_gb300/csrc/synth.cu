// Coherent MIMO FMCW echo synthesis (Sec. 3.2, Eqs. 7, 9-13).
//
// For channel o = (p, q), chirp n and fast-time sample m the dechirped IF
// sample is the coherent sum over the facets k lit from TX p and RX q:
//
//   x[o][n][m] = C / k_m^2 * sum_k g_k * F_k(k_m) * exp{j 2 pi theta_k(m)}
//
//   theta_k(m) = f_m L_k(t)/c - mu L_k(t)^2 / (2 c^2)     (Eq. 13 bracket,
//                tau = L/c, f_m = f0 + mu t, t = m/fs, L = R_t + R_r at
//                t_n + t: Eq. 12 with continuous time and the bistatic path)
//   g_k = rho_k o_k / (R_t R_r),  o_k = n_k . (t + r) / 2         (Eq. 7, PO)
//   F_k(k) = k^2 conj(J_k(k b)),   b = t + r,
//   J_k(w) = integral over facet k of exp(j w.(r' - c_k)) dA
//   C = lambda k / (sqrt(pi) (4 pi)^{3/2}) = 2 sqrt(pi) / (4 pi)^{3/2}
//
// The Eq. 9-11 "IFFT route" is read as the time-domain product: sample m
// sees the instantaneous frequency f_m, so sigma_f at f_m multiplies the
// dechirp phase directly.  Directions, R_t R_r in the amplitude and the
// facet integral are held at the chirp start t_n; only the delay moves.
//
// With u_v = b.(v_v - c_k) the facet integral is a divided difference of the
// exponential (Hermite-Genocchi), giving three evaluation forms, chosen per
// (facet, channel, chirp) record with k_max = 2 pi f_max / c:
//   vertex : F = sum_v w_v e^{-j k u_v},  w_v = -2A / prod_{l != v}(u_v - u_l)
//   series : k_max (u_max - u_min) < 1:  F = 2A e^{-j k ubar}
//              * sum_{p<=14} (-j)^p k^{p+2} h_p(u - ubar) / (p+2)!
//   edge   : some k_max |u_i - u_j| < 0.03 (an edge nearly normal to b_t):
//              F = sum_i j k c_i e^{-j k beta_i} sinc(k gamma_i),
//              c_i = e_i.(n x b)/|b_t|^2, beta_i = b.(m_i - c), gamma_i = b.e_i/2
//
// Two paths:
//   mixed : FP64 only where the phase spans ~1e5 cycles -- per-chirp
//           positions, |c(t_n) - p_a| and its reduction mod 1 (kinematics
//           kernel); everything else in FP32.  Per lane, S consecutive
//           samples: one MUFU sincos per vertex, then an FMA-only phasor
//           recurrence; partial sums per 32-record tile, Kahan-compensated
//           into the running sum.
//   fp64  : every quantity in FP64, the exact per-sample delay
//           sqrt(|c(t_n) + v t - p|^2), one sincospi per phasor per sample.
#include <cuda_runtime.h>
#include <stdint.h>

#include "bart_internal.cuh"

namespace bart {

// 1/n! for n = 0..17
__constant__ double c_inv_fact[18] = {
    1.0, 1.0, 1.0 / 2, 1.0 / 6, 1.0 / 24, 1.0 / 120, 1.0 / 720, 1.0 / 5040, 1.0 / 40320,
    1.0 / 362880, 1.0 / 3628800, 1.0 / 39916800, 1.0 / 479001600, 1.0 / 6227020800.0,
    1.0 / 87178291200.0, 1.0 / 1307674368000.0, 1.0 / 20922789888000.0,
    1.0 / 355687428096000.0};

// -------------------------------------------------------------------------
// kinematics (FP64): per antenna a, facet k lit from a, chirp n of the chunk
//   R = |c_k + v t_n - p_a|,  x0 = frac(R f0/c),  x1 = frac(R mu/(fs c))
//   hi = x1 rounded to a multiple of 2^-14, lo = x1 - hi
// stored as float4 (x0, hi, lo, R).  Since m is an integer, frac(L q m) =
// frac(frac(L q) m) and frac(hi m) is exact in FP32 for m < 1024.
// -------------------------------------------------------------------------
__global__ void kin_kernel(const double *__restrict__ c64, const FacetRec *__restrict__ fac,
                           const double *__restrict__ vel64, const uint8_t *__restrict__ state,
                           int64_t F, RadarDev rd, int n0, int nc, float4 *__restrict__ kin)
{
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int a = blockIdx.y;
    if (k >= F || state[(int64_t)a * F + k] != BART_VIS_LIT) return;
    const int inst = fac[k].inst;
    const double vx = vel64[3 * inst], vy = vel64[3 * inst + 1], vz = vel64[3 * inst + 2];
    const double dx = c64[3 * k] - rd.ant[a][0];
    const double dy = c64[3 * k + 1] - rd.ant[a][1];
    const double dz = c64[3 * k + 2] - rd.ant[a][2];
    const double A = dx * dx + dy * dy + dz * dz;
    const double B = 2.0 * (dx * vx + dy * vy + dz * vz);
    const double Cq = vx * vx + vy * vy + vz * vz;
    const double f0c = rd.f0 / kC0;
    const double muc = rd.slope / (rd.fs * kC0);
    for (int nl = 0; nl < nc; ++nl) {
        const double t = (double)(n0 + nl) * rd.Tc;
        const double R = sqrt(A + t * (B + t * Cq));
        double x0 = R * f0c;
        x0 -= floor(x0);
        double x1 = R * muc;
        x1 -= floor(x1);
        const double hi = rint(x1 * 16384.0) * (1.0 / 16384.0);
        kin[((int64_t)nl * rd.A + a) * F + k] =
            make_float4((float)x0, (float)hi, (float)(x1 - hi), (float)R);
    }
}

void launch_kinematics(const double *c64, const FacetRec *fac, const double *vel64,
                       const uint8_t *state, int64_t F, const RadarDev &rd, int n0, int nc,
                       float4 *kin, cudaStream_t s)
{
    const int T = 256;
    dim3 grid((unsigned int)((F + T - 1) / T), (unsigned int)rd.A);
    kin_kernel<<<grid, T, 0, s>>>(c64, fac, vel64, state, F, rd, n0, nc, kin);
}

// -------------------------------------------------------------------------
// mixed path
// -------------------------------------------------------------------------
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
    float out_scale;      // C (c / (2 pi f0))^2
    float tc;
    float ant[kMaxAnt][3];
};

struct __align__(16) RecV {   // vertex form
    float ph0[3];             // static phase per vertex, cycles in [-0.5, 0.5)
    float lo[3];              // per-sample rate remainder per vertex, cycles/sample
    float w[3];               // weight g w_v
    float sre[3], sim[3];     // step phasor exp(j 2 pi (hi + lo_v))
    float hi;                 // quantised rate, multiple of 2^-14
    float p2;                 // cycles / sample^2
    float pad;
};
struct __align__(16) RecS {   // series / edge form
    int kind;                 // kRecSeries or kRecEdge
    int flags;                // edge: bit i = sinc of edge i by its series
    float ph0c, hi, loc, p2;  // centroid phase terms
    float d[18];
};

constexpr int kMixWarps = 4;

__device__ __forceinline__ float red1(float x) { return x - rintf(x); }

template <int S>
__global__ void __launch_bounds__(kMixWarps * 32)
synth_mixed_kernel(SynthArgs A, MixConsts K, int W)
{
    __shared__ RecV sV[kMixWarps][32];
    __shared__ RecS sS[kMixWarps][32];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t gw = (int64_t)blockIdx.x * kMixWarps + warp;
    const int nc = A.nc;
    const int64_t unit = gw / W;
    const int seg = (int)(gw % W);
    if (unit >= (int64_t)A.rd.O * nc) return;
    const int o = (int)(unit / nc), nl = (int)(unit % nc);
    const int n = A.n0 + nl;
    const int P = A.rd.P, Q = A.rd.Q, AA = A.rd.A;
    const int tx = o / Q, rx = o % Q;
    const int64_t F = A.F;
    const int m0 = (seg * 32 + lane) * S;
    const float fm0 = (float)m0;
    const float fm0sq = fm0 * fm0;
    const float eps_lane = 6.283185307179586f * (2.f * fm0 + 1.f);   // times p2
    const float ptx[3] = {K.ant[tx][0], K.ant[tx][1], K.ant[tx][2]};
    const float prx[3] = {K.ant[P + rx][0], K.ant[P + rx][1], K.ant[P + rx][2]};
    const float tn = (float)n * K.tc;

    float kap[S];
#pragma unroll
    for (int j = 0; j < S; ++j) kap[j] = fmaf((float)(m0 + j), K.kap_step, 1.f);

    float sr[S], si[S], cr_[S], ci_[S], pr[S], pi[S];
#pragma unroll
    for (int j = 0; j < S; ++j) sr[j] = si[j] = cr_[j] = ci_[j] = pr[j] = pi[j] = 0.f;

    const int32_t *list = A.vis_idx + (int64_t)o * F;
    const int cnt = A.vis_cnt[o];
    const float4 *kin_t = A.kin + ((int64_t)nl * AA + tx) * F;
    const float4 *kin_r = A.kin + ((int64_t)nl * AA + P + rx) * F;
    unsigned long long nV = 0, nSr = 0, nE = 0;

    for (int base = 0; base < cnt; base += 32) {
        // ---------------- build one record per lane ----------------
        const bool valid = base + lane < cnt;
        int cls = -1;
        if (valid) {
            const int k = list[base + lane];
            const FacetRec fr = A.fac[k];
            const float4 vv = reinterpret_cast<const float4 *>(A.vel32)[fr.inst];
            const float4 kt = kin_t[k], kr = kin_r[k];
            const float cx = fmaf(vv.x, tn, fr.c[0]);
            const float cy = fmaf(vv.y, tn, fr.c[1]);
            const float cz = fmaf(vv.z, tn, fr.c[2]);
            float th[3] = {ptx[0] - cx, ptx[1] - cy, ptx[2] - cz};
            float rh[3] = {prx[0] - cx, prx[1] - cy, prx[2] - cz};
            const float it = rsqrtf(th[0] * th[0] + th[1] * th[1] + th[2] * th[2]);
            const float ir = rsqrtf(rh[0] * rh[0] + rh[1] * rh[1] + rh[2] * rh[2]);
            float b[3];
#pragma unroll
            for (int r = 0; r < 3; ++r) {
                th[r] *= it;
                rh[r] *= ir;
                b[r] = th[r] + rh[r];
            }
            const float Rt = kt.w, Rr = kr.w, L = Rt + Rr;
            const float o_k = 0.5f * (fr.n[0] * b[0] + fr.n[1] * b[1] + fr.n[2] * b[2]);
            const float g = fr.rho * o_k / (Rt * Rr);
            // in-plane part of b, formed once: u_v, |b_t|^2 and n x b_t all derive
            // from it, so the forms below evaluate J exactly at one wave vector
            // (|b|^2 - (b.n)^2 would cancel catastrophically near specular)
            const float bn = fr.n[0] * b[0] + fr.n[1] * b[1] + fr.n[2] * b[2];
            const float bt[3] = {b[0] - bn * fr.n[0], b[1] - bn * fr.n[1], b[2] - bn * fr.n[2]};
            float u[3];
#pragma unroll
            for (int v = 0; v < 3; ++v)
                u[v] = bt[0] * fr.dv[3 * v] + bt[1] * fr.dv[3 * v + 1] + bt[2] * fr.dv[3 * v + 2];
            float Ld = 0.f, Ldd = 0.f;
            if (A.rd.intra) {
                const float v2 = vv.x * vv.x + vv.y * vv.y + vv.z * vv.z;
                const float vt = vv.x * th[0] + vv.y * th[1] + vv.z * th[2];
                const float vr = vv.x * rh[0] + vv.y * rh[1] + vv.z * rh[2];
                Ld = -(vt + vr);
                Ldd = (v2 - vt * vt) / Rt + (v2 - vr * vr) / Rr;
            }
            float hi = kt.y + kr.y;
            hi = hi >= 1.f ? hi - 1.f : hi;
            const float loc = (kt.z + kr.z) + K.f0c_fs * Ld - K.mu_c2fs * L * Ld;
            const float p2 = K.half_f0c_fs2 * Ldd + K.mu_c_fs2 * Ld;
            const float ph0c = red1((kt.x + kr.x) - K.mu_2c2 * L * L);
            const float umin = fminf(fminf(u[0], u[1]), u[2]);
            const float umax = fmaxf(fmaxf(u[0], u[1]), u[2]);
            const float dmin = fminf(fminf(fabsf(u[0] - u[1]), fabsf(u[1] - u[2])),
                                     fabsf(u[0] - u[2]));
            const float A2 = 2.f * fr.area * g;
            if (K.kmax * (umax - umin) < (float)kSeriesKD) {
                cls = kRecSeries;
                RecS &R = sS[warp][lane];
                R.kind = kRecSeries;
                R.flags = 0;
                R.ph0c = ph0c;
                R.hi = hi;
                R.loc = loc;
                R.p2 = p2;
                const float ub = (u[0] + u[1] + u[2]) * (1.f / 3.f);
                R.d[0] = red1(-K.f0c * ub);
                R.d[1] = -K.muc * ub;
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
                    R.d[2 + i] = ((i & 1) ? -sc : sc) * h[2 * i] * (float)c_inv_fact[2 * i + 2];
#pragma unroll
                for (int i = 0; i < 7; ++i)
                    R.d[10 + i] = ((i & 1) ? sc : -sc) * h[2 * i + 1] *
                                  (float)c_inv_fact[2 * i + 3];
            } else if (K.kmax * dmin < (float)kEdgeKd) {
                cls = kRecEdge;
                RecS &R = sS[warp][lane];
                R.kind = kRecEdge;
                R.ph0c = ph0c;
                R.hi = hi;
                R.loc = loc;
                R.p2 = p2;
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
                    R.d[4 * i] = red1(-K.f0c * beta);
                    R.d[4 * i + 1] = -K.muc * beta;
                    R.d[4 * i + 2] = K.k0 * gam;
                    R.d[4 * i + 3] = K.k0 * ci * g;
                    if (K.kmax * fabsf(gam) < (float)kSincSeries) flags |= 1 << i;
                }
                R.flags = flags;
            } else {
                cls = kRecVertex;
                RecV &R = sV[warp][lane];
                R.hi = hi;
                R.p2 = p2;
                R.pad = 0.f;
#pragma unroll
                for (int v = 0; v < 3; ++v) {
                    const float ua = u[v], ub_ = u[(v + 1) % 3], uc = u[(v + 2) % 3];
                    R.ph0[v] = red1(ph0c - K.f0c * ua);
                    const float lo = loc - K.muc * ua;
                    R.lo[v] = lo;
                    R.w[v] = -A2 / ((ua - ub_) * (ua - uc));
                    float s, c;
                    sincospif(2.f * red1(hi + lo), &s, &c);
                    R.sre[v] = c;
                    R.sim[v] = s;
                }
            }
        }
        __syncwarp();
        unsigned int mv = __ballot_sync(0xffffffffu, cls == kRecVertex);
        unsigned int ms = __ballot_sync(0xffffffffu, cls == kRecSeries || cls == kRecEdge);
        const unsigned int mser = __ballot_sync(0xffffffffu, cls == kRecSeries);
        nV += __popc(mv);
        nSr += __popc(mser);
        nE += __popc(ms & ~mser);
        // ---------------- vertex records: recurrence ----------------
        while (mv) {
            const int i = __ffs(mv) - 1;
            mv &= mv - 1;
            const RecV &R = sV[warp][i];
            const float t1 = red1(R.hi * fm0);
            const float q2 = R.p2 * fm0sq;
            const float eps = R.p2 * eps_lane;
#pragma unroll
            for (int v = 0; v < 3; ++v) {
                const float thv = red1(fmaf(R.lo[v], fm0, R.ph0[v] + t1) + q2);
                float zs, zc;
                __sincosf(6.283185307179586f * thv, &zs, &zc);
                const float stc = fmaf(-eps, R.sim[v], R.sre[v]);
                const float sts = fmaf(eps, R.sre[v], R.sim[v]);
                const float w = R.w[v];
#pragma unroll
                for (int j = 0; j < S; ++j) {
                    pr[j] = fmaf(w, zc, pr[j]);
                    pi[j] = fmaf(w, zs, pi[j]);
                    if (j + 1 < S) {
                        const float nc_ = fmaf(zc, stc, -zs * sts);
                        zs = fmaf(zc, sts, zs * stc);
                        zc = nc_;
                    }
                }
            }
        }
        // ---------------- series / edge records: per sample ----------------
        while (ms) {
            const int i = __ffs(ms) - 1;
            ms &= ms - 1;
            const RecS &R = sS[warp][i];
#pragma unroll
            for (int j = 0; j < S; ++j) {
                const float fm = (float)(m0 + j);
                const float thc = fmaf(R.p2, fm * fm, fmaf(R.loc, fm, R.ph0c + red1(R.hi * fm)));
                const float kp = kap[j];
                if (R.kind == kRecSeries) {
                    const float th = red1(thc + fmaf(R.d[1], fm, R.d[0]));
                    float zs, zc;
                    __sincosf(6.283185307179586f * th, &zs, &zc);
                    const float k2 = kp * kp;
                    float a = R.d[9], bb = R.d[16];
#pragma unroll
                    for (int q = 6; q >= 0; --q) a = fmaf(a, k2, R.d[2 + q]);
#pragma unroll
                    for (int q = 5; q >= 0; --q) bb = fmaf(bb, k2, R.d[10 + q]);
                    const float re = a * k2, im = bb * k2 * kp;
                    pr[j] += zc * re - zs * im;
                    pi[j] += zc * im + zs * re;
                } else {
#pragma unroll
                    for (int e = 0; e < 3; ++e) {
                        const float th = red1(thc + fmaf(R.d[4 * e + 1], fm, R.d[4 * e]));
                        float zs, zc;
                        __sincosf(6.283185307179586f * th, &zs, &zc);
                        const float x = kp * R.d[4 * e + 2];
                        float sn;
                        if (R.flags & (1 << e)) {
                            const float x2 = x * x;
                            sn = fmaf(x2, fmaf(x2, fmaf(x2, fmaf(x2, 1.f / 362880.f, -1.f / 5040.f),
                                                        1.f / 120.f), -1.f / 6.f), 1.f);
                        } else {
                            sn = sinf(x) / x;   // accurate sinf: |x| may reach ~1e3
                        }
                        const float coef = kp * R.d[4 * e + 3] * sn;
                        pr[j] = fmaf(-coef, zs, pr[j]);
                        pi[j] = fmaf(coef, zc, pi[j]);
                    }
                }
            }
        }
        // ---------------- Kahan-compensated tile accumulation ----------------
#pragma unroll
        for (int j = 0; j < S; ++j) {
            float y = pr[j] - cr_[j];
            float t = sr[j] + y;
            cr_[j] = (t - sr[j]) - y;
            sr[j] = t;
            y = pi[j] - ci_[j];
            t = si[j] + y;
            ci_[j] = (t - si[j]) - y;
            si[j] = t;
            pr[j] = pi[j] = 0.f;
        }
        __syncwarp();
    }
    if (lane == 0 && seg == 0 && A.counters) {
        atomicAdd(A.counters + 0, nV);
        atomicAdd(A.counters + 1, nSr);
        atomicAdd(A.counters + 2, nE);
    }
    const int64_t row = ((int64_t)o * A.rd.N + n) * A.rd.M + m0;
#pragma unroll
    for (int j = 0; j < S; ++j) {
        const float sc = K.out_scale / (kap[j] * kap[j]);
        if (A.out_c64) {
            reinterpret_cast<float2 *>(A.out)[row + j] = make_float2(sr[j] * sc, si[j] * sc);
        } else {
            reinterpret_cast<double2 *>(A.out)[row + j] =
                make_double2((double)sr[j] * sc, (double)si[j] * sc);
        }
    }
}

// consecutive samples per lane: the largest S in {8, 4, 2, 1} with 32 S | M;
// a (channel, chirp) row of M samples then takes W = M / (32 S) warps
static int samples_per_lane(int M)
{
    for (int S = 8; S > 1; S >>= 1)
        if (M % (32 * S) == 0) return S;
    return 1;
}

static MixConsts mix_consts(const RadarDev &rd)
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
    const double camp = 2.0 * sqrt(kPi) / pow(4.0 * kPi, 1.5);
    const double lk = c / (2.0 * kPi * f0);
    K.out_scale = (float)(camp * lk * lk);
    K.tc = (float)rd.Tc;
    for (int a = 0; a < kMaxAnt; ++a)
        for (int r = 0; r < 3; ++r) K.ant[a][r] = (float)rd.ant[a][r];
    return K;
}

void launch_synth_mixed(const SynthArgs &a, cudaStream_t s)
{
    const MixConsts K = mix_consts(a.rd);
    const int M = a.rd.M;
    const int S = samples_per_lane(M);
    const int W = M / (32 * S);
    const int64_t warps = (int64_t)a.rd.O * a.nc * W;
    const unsigned int grid = (unsigned int)((warps + kMixWarps - 1) / kMixWarps);
    switch (S) {
    case 8: synth_mixed_kernel<8><<<grid, kMixWarps * 32, 0, s>>>(a, K, W); break;
    case 4: synth_mixed_kernel<4><<<grid, kMixWarps * 32, 0, s>>>(a, K, W); break;
    case 2: synth_mixed_kernel<2><<<grid, kMixWarps * 32, 0, s>>>(a, K, W); break;
    default: synth_mixed_kernel<1><<<grid, kMixWarps * 32, 0, s>>>(a, K, W); break;
    }
}

// -------------------------------------------------------------------------
// plain FP64 path
// -------------------------------------------------------------------------
struct __align__(16) RecD {
    int kind, flags;
    double qt[3];     // R_t(t)^2 = qt0 + t (qt1 + t qt2), t = fast time
    double qr[2];     // R_r(t)^2 = qr0 + t (qr1 + t qt2)
    double d[22];
};

constexpr int kF64Warps = 4;

template <int S>
__global__ void __launch_bounds__(kF64Warps * 32)
synth_fp64_kernel(SynthArgs A, int W)
{
    __shared__ RecD sR[kF64Warps][32];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t gw = (int64_t)blockIdx.x * kF64Warps + warp;
    const int N = A.rd.N;
    const int64_t unit = gw / W;
    const int seg = (int)(gw % W);
    if (unit >= (int64_t)A.rd.O * N) return;
    const int o = (int)(unit / N), n = (int)(unit % N);
    const int P = A.rd.P, Q = A.rd.Q;
    const int tx = o / Q, rx = o % Q;
    const int64_t F = A.F;
    const int m0 = (seg * 32 + lane) * S;
    const double c = kC0, f0 = A.rd.f0, mu = A.rd.slope, fs = A.rd.fs;
    const double f_max = f0 + mu * (A.rd.M - 1) / fs;
    const double k0 = 2.0 * kPi * f0 / c, kmax = 2.0 * kPi * f_max / c;
    const double tn = (double)n * A.rd.Tc;
    const double *ptx = A.rd.ant[tx];
    const double *prx = A.rd.ant[P + rx];

    double accr[S], acci[S];
#pragma unroll
    for (int j = 0; j < S; ++j) accr[j] = acci[j] = 0.0;

    const int32_t *list = A.vis_idx + (int64_t)o * F;
    const int cnt = A.vis_cnt[o];
    unsigned long long nV = 0, nSr = 0, nE = 0;

    for (int base = 0; base < cnt; base += 32) {
        const bool valid = base + lane < cnt;
        int cls = -1;
        if (valid) {
            const int64_t k = list[base + lane];
            RecD &R = sR[warp][lane];
            const int inst = A.fac[k].inst;
            const double vel[3] = {A.vel64[3 * inst], A.vel64[3 * inst + 1],
                                   A.vel64[3 * inst + 2]};
            double cc[3], dv[9];
            for (int r = 0; r < 3; ++r) cc[r] = A.c64[3 * k + r];
            for (int i = 0; i < 9; ++i) dv[i] = A.tri64[9 * k + i] - cc[i % 3];
            for (int r = 0; r < 3; ++r) cc[r] += vel[r] * tn;
            const double e1[3] = {dv[3] - dv[0], dv[4] - dv[1], dv[5] - dv[2]};
            const double e2[3] = {dv[6] - dv[0], dv[7] - dv[1], dv[8] - dv[2]};
            double nn[3] = {e1[1] * e2[2] - e1[2] * e2[1], e1[2] * e2[0] - e1[0] * e2[2],
                            e1[0] * e2[1] - e1[1] * e2[0]};
            const double nl = sqrt(nn[0] * nn[0] + nn[1] * nn[1] + nn[2] * nn[2]);
            const double area = 0.5 * nl;
            for (int r = 0; r < 3; ++r) nn[r] /= nl;
            double dt[3], dr[3];
            for (int r = 0; r < 3; ++r) {
                dt[r] = ptx[r] - cc[r];
                dr[r] = prx[r] - cc[r];
            }
            const double Rt2 = dt[0] * dt[0] + dt[1] * dt[1] + dt[2] * dt[2];
            const double Rr2 = dr[0] * dr[0] + dr[1] * dr[1] + dr[2] * dr[2];
            const double Rt = sqrt(Rt2), Rr = sqrt(Rr2);
            double b[3];
            for (int r = 0; r < 3; ++r) b[r] = dt[r] / Rt + dr[r] / Rr;
            const double ok = 0.5 * (nn[0] * b[0] + nn[1] * b[1] + nn[2] * b[2]);
            const double g = (double)A.fac[k].rho * ok / (Rt * Rr);
            R.qt[0] = Rt2;
            R.qr[0] = Rr2;
            if (A.rd.intra) {
                R.qt[1] = -2.0 * (dt[0] * vel[0] + dt[1] * vel[1] + dt[2] * vel[2]);
                R.qr[1] = -2.0 * (dr[0] * vel[0] + dr[1] * vel[1] + dr[2] * vel[2]);
                R.qt[2] = vel[0] * vel[0] + vel[1] * vel[1] + vel[2] * vel[2];
            } else {
                R.qt[1] = R.qr[1] = R.qt[2] = 0.0;
            }
            const double bn = b[0] * nn[0] + b[1] * nn[1] + b[2] * nn[2];
            const double bt[3] = {b[0] - bn * nn[0], b[1] - bn * nn[1], b[2] - bn * nn[2]};
            double u[3];
            for (int v = 0; v < 3; ++v)
                u[v] = bt[0] * dv[3 * v] + bt[1] * dv[3 * v + 1] + bt[2] * dv[3 * v + 2];
            const double umin = fmin(fmin(u[0], u[1]), u[2]);
            const double umax = fmax(fmax(u[0], u[1]), u[2]);
            const double dmin = fmin(fmin(fabs(u[0] - u[1]), fabs(u[1] - u[2])),
                                     fabs(u[0] - u[2]));
            const double A2 = 2.0 * area * g;
            if (kmax * (umax - umin) < kSeriesKD) {
                cls = R.kind = kRecSeries;
                const double ub = (u[0] + u[1] + u[2]) / 3.0;
                R.d[0] = ub;
                const double y0 = k0 * (u[0] - ub), y1 = k0 * (u[1] - ub), y2 = k0 * (u[2] - ub);
                const double e2s = y0 * y1 + y0 * y2 + y1 * y2, e3s = y0 * y1 * y2;
                double h[kSeriesTerms];
                h[0] = 1.0;
                h[1] = 0.0;
                h[2] = -e2s;
                for (int p = 3; p < kSeriesTerms; ++p) h[p] = -e2s * h[p - 2] + e3s * h[p - 3];
                const double sc = A2 * k0 * k0;
                for (int i = 0; i < 8; ++i)
                    R.d[1 + i] = ((i & 1) ? -sc : sc) * h[2 * i] * c_inv_fact[2 * i + 2];
                for (int i = 0; i < 7; ++i)
                    R.d[9 + i] = ((i & 1) ? sc : -sc) * h[2 * i + 1] * c_inv_fact[2 * i + 3];
            } else if (kmax * dmin < kEdgeKd) {
                cls = R.kind = kRecEdge;
                const double bt2 = bt[0] * bt[0] + bt[1] * bt[1] + bt[2] * bt[2];
                const double nxb[3] = {nn[1] * bt[2] - nn[2] * bt[1], nn[2] * bt[0] - nn[0] * bt[2],
                                       nn[0] * bt[1] - nn[1] * bt[0]};
                int flags = 0;
                for (int i = 0; i < 3; ++i) {
                    const int i1 = (i + 1) % 3;
                    const double e[3] = {dv[3 * i1] - dv[3 * i], dv[3 * i1 + 1] - dv[3 * i + 1],
                                         dv[3 * i1 + 2] - dv[3 * i + 2]};
                    const double gam = 0.5 * (u[i1] - u[i]);
                    R.d[3 * i] = 0.5 * (u[i] + u[i1]);
                    R.d[3 * i + 1] = k0 * gam;
                    R.d[3 * i + 2] = k0 * g * (e[0] * nxb[0] + e[1] * nxb[1] + e[2] * nxb[2]) / bt2;
                    if (kmax * fabs(gam) < kSincSeries) flags |= 1 << i;
                }
                R.flags = flags;
            } else {
                cls = R.kind = kRecVertex;
                for (int v = 0; v < 3; ++v) {
                    const double ua = u[v], ub_ = u[(v + 1) % 3], uc = u[(v + 2) % 3];
                    R.d[v] = ua;
                    R.d[3 + v] = -A2 / ((ua - ub_) * (ua - uc));
                }
            }
        }
        __syncwarp();
        unsigned int mask = __ballot_sync(0xffffffffu, valid);
        const unsigned int a1 = __ballot_sync(0xffffffffu, cls == kRecVertex);
        const unsigned int a2 = __ballot_sync(0xffffffffu, cls == kRecSeries);
        nV += __popc(a1);
        nSr += __popc(a2);
        nE += __popc(mask & ~a1 & ~a2);
        while (mask) {
            const int i = __ffs(mask) - 1;
            mask &= mask - 1;
            const RecD &R = sR[warp][i];
#pragma unroll 1
            for (int j = 0; j < S; ++j) {
                const double t = (double)(m0 + j) / fs;
                const double fm = f0 + mu * t;
                const double L = sqrt(R.qt[0] + t * (R.qt[1] + t * R.qt[2])) +
                                 sqrt(R.qr[0] + t * (R.qr[1] + t * R.qt[2]));
                double thc = fm * L / c - mu * L * L / (2.0 * c * c);
                thc -= rint(thc);
                const double fmc = fm / c;
                const double kp = fm / f0;
                double re = 0.0, im = 0.0;
                if (R.kind == kRecVertex) {
                    for (int v = 0; v < 3; ++v) {
                        double s_, c_;
                        sincospi(2.0 * (thc - fmc * R.d[v]), &s_, &c_);
                        re += R.d[3 + v] * c_;
                        im += R.d[3 + v] * s_;
                    }
                } else if (R.kind == kRecSeries) {
                    double s_, c_;
                    sincospi(2.0 * (thc - fmc * R.d[0]), &s_, &c_);
                    const double k2 = kp * kp;
                    double a = R.d[8], bb = R.d[15];
                    for (int q = 6; q >= 0; --q) a = a * k2 + R.d[1 + q];
                    for (int q = 5; q >= 0; --q) bb = bb * k2 + R.d[9 + q];
                    const double pr_ = a * k2, pi_ = bb * k2 * kp;
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
                accr[j] += re;
                acci[j] += im;
            }
        }
        __syncwarp();
    }
    if (lane == 0 && seg == 0 && A.counters) {
        atomicAdd(A.counters + 0, nV);
        atomicAdd(A.counters + 1, nSr);
        atomicAdd(A.counters + 2, nE);
    }
    const double camp = 2.0 * sqrt(kPi) / pow(4.0 * kPi, 1.5);
    const int64_t row = ((int64_t)o * N + n) * A.rd.M + m0;
#pragma unroll
    for (int j = 0; j < S; ++j) {
        const double fm = f0 + mu * (double)(m0 + j) / fs;
        const double km = 2.0 * kPi * fm / c;
        const double sc = camp / (km * km);
        if (A.out_c64) {
            reinterpret_cast<float2 *>(A.out)[row + j] =
                make_float2((float)(accr[j] * sc), (float)(acci[j] * sc));
        } else {
            reinterpret_cast<double2 *>(A.out)[row + j] = make_double2(accr[j] * sc, acci[j] * sc);
        }
    }
}

void launch_synth_fp64(const SynthArgs &a, cudaStream_t s)
{
    const int M = a.rd.M;
    const int S = samples_per_lane(M);
    const int W = M / (32 * S);
    const int64_t warps = (int64_t)a.rd.O * a.rd.N * W;
    const unsigned int grid = (unsigned int)((warps + kF64Warps - 1) / kF64Warps);
    switch (S) {
    case 8: synth_fp64_kernel<8><<<grid, kF64Warps * 32, 0, s>>>(a, W); break;
    case 4: synth_fp64_kernel<4><<<grid, kF64Warps * 32, 0, s>>>(a, W); break;
    case 2: synth_fp64_kernel<2><<<grid, kF64Warps * 32, 0, s>>>(a, W); break;
    default: synth_fp64_kernel<1><<<grid, kF64Warps * 32, 0, s>>>(a, W); break;
    }
}

}  // namespace bart
