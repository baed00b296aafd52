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
//           samples: one MUFU sincos per vertex, then the FMA-only
//           three-term phasor recurrence on sample pairs; partial sums per
//           32-record tile, Kahan-compensated into the running sum.
//   fp64  : every quantity in FP64, the exact per-sample delay
//           sqrt(|c(t_n) + v t - p|^2), one sincospi per phasor per sample.
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>

#include "bart_internal.cuh"
#include "mixed_record.cuh"
#include "record_fp64.cuh"

namespace bart {

// -------------------------------------------------------------------------
// kinematics: per antenna a and facet k lit from a, the one-way distance
// R(t) = |c_k + v t - p_a| over the frame, as Taylor coefficients in the
// chirp-slot index s (time s Tc; one slot per chirp, P with time-division
// MIMO).  R^2 = A + B t + C t^2 is expanded about the middle slot s_c,
// R = sum_j a_j tau^j with tau = s - s_c, a_0 = sqrt(q_0) and
// a_j = (q_j - sum_{i=1}^{j-1} a_i a_{j-i}) / (2 a_0)  (from R^2 = q).  The
// series converges with ratio rho = tau_max |v| Tc / R (the roots of q lie at
// |tau| = R / (|v| Tc)); the degree is the smallest d <= 8 with
// R rho^(d+1) / (1 - rho) <= 1e-11 m, else the record build takes an FP64
// square root.  Computed once per frame in FP64 and stored per (a, k) as
// kKinRow float4: (f0/c a_j split into a high and a low float, a_j in FP32);
// the degree rides in row 0's w.  The mixed kernel evaluates the cycles
// x0u = R f0 / c in double-float arithmetic (float pairs, error-free
// transformations, Dekker 1971 / Knuth), reduces frac(x0u) and
// frac(x0u mu / (fs f0)) (split into hi, a multiple of 2^-14, and lo) and R.
// -------------------------------------------------------------------------

// Rows are formed for every facet that is not certainly back-facing (a
// superset of the lit ones): the kernel then needs only the world facets and
// runs beside the hierarchy build and visibility.  The facing decision is
// the visibility kernel's FP32 pre-test: |cos32 - cos| < 6e-7 (two-sided
// facets always get rows).
// Far field: the row is the facet's plane-wave path from the instance
// origin r, g(t) = |r(t) - p_a| + l(t) / |r(t) - p_a| with
// l(t) = (r(t) - p_a).(c_k - r), expanded from the series of R = |r - p_a|
// and of 1/R (b_0 = 1/a_0, b_j = -sum_{i=1}^{j} a_i b_{j-i} / a_0).
__global__ void kin_coef_kernel(const double *__restrict__ c64, const FacetRec *__restrict__ fac,
                                const double *__restrict__ vel64,
                                const double *__restrict__ ref64, int64_t F, RadarDev rd,
                                float4 *__restrict__ coef, double *__restrict__ quad)
{
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int a = blockIdx.y;
    if (k >= F) return;
    const int inst = fac[k].inst;
    const double *from = rd.far_field ? ref64 + 3 * inst : c64 + 3 * k;
    if (!fac[k].two_sided) {
        const float D0 = (float)(rd.ant[a][0] - from[0]);
        const float D1 = (float)(rd.ant[a][1] - from[1]);
        const float D2 = (float)(rd.ant[a][2] - from[2]);
        const float dd = fmaf(D0, D0, fmaf(D1, D1, D2 * D2));
        const float cs = fmaf(fac[k].n[0], D0, fmaf(fac[k].n[1], D1, fac[k].n[2] * D2)) *
                         rsqrtf(dd);
        if (dd > 0.f && cs <= -((float)rd.eps_face + 2e-6f)) return;   // certainly BACK
    }
    const double vx = vel64[3 * inst], vy = vel64[3 * inst + 1], vz = vel64[3 * inst + 2];
    const double dx = from[0] - rd.ant[a][0];
    const double dy = from[1] - rd.ant[a][1];
    const double dz = from[2] - rd.ant[a][2];
    const double A = dx * dx + dy * dy + dz * dz;
    const double B = 2.0 * (dx * vx + dy * vy + dz * vz);
    const double Cq = vx * vx + vy * vy + vz * vz;
    // far field: l(t) = l0 + l1 t, the facet's offset from the origin
    // projected on r(t) - p_a
    double l0 = 0.0, l1 = 0.0, doff = 0.0;
    if (rd.far_field) {
        const double ox = c64[3 * k] - from[0], oy = c64[3 * k + 1] - from[1],
                     oz = c64[3 * k + 2] - from[2];
        l0 = dx * ox + dy * oy + dz * oz;
        l1 = vx * ox + vy * oy + vz * oz;
        doff = sqrt(ox * ox + oy * oy + oz * oz);
    }
    const double f0c = rd.f0 / kC0;
    const int64_t row = (int64_t)a * F + k;
    double *qd = quad + kKinQuadWords * row;
    qd[0] = A;
    qd[1] = B;
    qd[2] = Cq;
    qd[3] = l0;
    qd[4] = l1;
    // expansion point: the middle chirp slot; tau in slots
    const double sc = 0.5 * (double)(rd.N * rd.slots - 1);
    const double tc = sc * rd.Tc;
    const double tmax = sc > 0.0 ? sc : 1.0;
    const double q0 = A + tc * (B + tc * Cq);
    const double q1 = (B + 2.0 * Cq * tc) * rd.Tc, q2 = Cq * rd.Tc * rd.Tc;
    const double a0 = sqrt(q0);
    const double rho = tmax * sqrt(q2 / q0);
    int deg = -1;
    if (rho < 0.25) {
        double bound = (a0 + doff) * rho * rho / (1.0 - rho);
        for (int d = 1; d <= kKinMaxDeg; ++d, bound *= rho)
            if (bound <= 1e-11) { deg = d; break; }
    }
    float4 *out = coef + row * kKinRow;
    if (deg < 0) {
        out[0] = make_float4(0.f, 0.f, 0.f, __int_as_float(-1));
        for (int j = 1; j <= kKinMaxDeg; ++j) out[j] = make_float4(0.f, 0.f, 0.f, 0.f);
        return;
    }
    double aj[kKinMaxDeg + 1];
    aj[0] = a0;
    const double inv2a0 = 0.5 / a0;
#pragma unroll
    for (int j = 1; j <= kKinMaxDeg; ++j) {
        double sacc = j == 1 ? q1 : (j == 2 ? q2 : 0.0);
#pragma unroll
        for (int l = 1; l < j; ++l) sacc -= aj[l] * aj[j - l];
        aj[j] = sacc * inv2a0;
    }
    if (rd.far_field) {
        // g = R + (L0 + L1 tau) / R, tau in slots about the middle one
        const double L0 = l0 + l1 * tc, L1 = l1 * rd.Tc;
        double bj[kKinMaxDeg + 1];
        bj[0] = 1.0 / a0;
#pragma unroll
        for (int j = 1; j <= kKinMaxDeg; ++j) {
            double sacc = 0.0;
#pragma unroll
            for (int i = 1; i <= j; ++i) sacc += aj[i] * bj[j - i];
            bj[j] = -sacc * bj[0];
        }
#pragma unroll
        for (int j = kKinMaxDeg; j >= 0; --j) aj[j] += L0 * bj[j] + (j > 0 ? L1 * bj[j - 1] : 0.0);
    }
    // rows above the degree are zero, so two rows of different degrees can
    // share one Horner loop
    for (int j = 0; j <= kKinMaxDeg; ++j) {
        if (j > deg) {
            out[j] = make_float4(0.f, 0.f, 0.f, 0.f);
            continue;
        }
        const double cf = f0c * aj[j];
        const float hi = (float)cf;
        out[j] = make_float4(hi, (float)(cf - (double)hi), (float)aj[j],
                             j == 0 ? __int_as_float(deg) : 0.f);
    }
}

void launch_kin_coef(const double *c64, const FacetRec *fac, const double *vel64,
                     const double *ref64, int64_t F, const RadarDev &rd, float4 *coef,
                     double *quad, cudaStream_t s)
{
    const int T = 128;
    dim3 grid((unsigned int)((F + T - 1) / T), (unsigned int)rd.A);
    kin_coef_kernel<<<grid, T, 0, s>>>(c64, fac, vel64, ref64, F, rd, coef, quad);
}

// -------------------------------------------------------------------------
// mixed path
// -------------------------------------------------------------------------
constexpr int kMixWarps = 2;         // 2-warp CTAs: 22 KB of shared memory at S = 16
constexpr int kMixMinBlocks = 8;     // resident CTAs per SM: 16 warps, 128 registers a thread

// Packed FP32 pairs (sm_100+ f32x2 arithmetic): two floats in one 64-bit
// register pair, one instruction for both lanes of a pair.  The mixed
// kernel keeps two consecutive samples of a lane in one pair.
__device__ __forceinline__ uint64_t pk2(float lo, float hi)
{
    uint64_t r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
    return r;
}
__device__ __forceinline__ void upk2(uint64_t r, float &lo, float &hi)
{
    asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(r));
}
__device__ __forceinline__ uint64_t ffma2(uint64_t a, uint64_t b, uint64_t c)
{
    uint64_t d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}
__device__ __forceinline__ uint64_t fmul2(uint64_t a, uint64_t b)
{
    uint64_t d;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ uint64_t fadd2(uint64_t a, uint64_t b)
{
    uint64_t d;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ uint64_t fsub2(uint64_t a, uint64_t b)
{
    uint64_t d;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}

// S: consecutive samples per lane; LPR: lanes per chirp row (RPW = 32/LPR
// rows of the same channel share a warp, e.g. two 256-sample chirps at
// S = 16).  A 32-record tile holds LPR facets x RPW chirps: lane l builds
// the record of facet (l mod LPR) for its own row.
template <int S, int LPR>
__global__ void __launch_bounds__(kMixWarps * 32, S >= 32 ? 6 : kMixMinBlocks)
synth_mixed_kernel(SynthArgs A, MixConsts K, int W)
{
    constexpr int RPW = 32 / LPR;
    __shared__ RecM sRec[kMixWarps][32];
    // running sums and Kahan compensations: [warp][re, im, c_re, c_im][S][lane]
    constexpr int S2 = (S + 1) / 2;
    // running sums and Kahan compensations of the sample pairs:
    // [warp][re, im, c_re, c_im][pair][lane]
    __shared__ uint64_t sAcc[kMixWarps][4][S2][32];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int row = lane / LPR, col = lane % LPR;
    const int O = A.rd.O, P = A.rd.P, Q = A.rd.Q;
    const int TPI = A.tiles_per_item;
    const int64_t F = A.F;
    const int nc = A.nc;
    const int ngroups = (nc + RPW - 1) / RPW;
    const int VO = A.VO;
    const int total = A.item_off[VO];
    unsigned long long nV = 0, nSr = 0, nE = 0;

    // persistent warps: each pulls (channel, chirp group, sample segment,
    // record chunk) items from a device counter until none remain
    for (;;) {
    int item = 0;
    if (lane == 0) item = atomicAdd(A.item_counter, 1);
    item = __shfl_sync(0xffffffffu, item, 0);
    if (item >= total) break;
    int clo = 0, chi = VO - 1;                 // row: last v with item_off[v] <= item
    while (clo < chi) {
        const int mid = (clo + chi + 1) >> 1;
        if (A.item_off[mid] <= item) clo = mid;
        else chi = mid - 1;
    }
    const int vrow = clo;                      // scene * O + channel
    const int o = vrow % O;
    const int cnt = A.vcnt[vrow];
    const int ipu = max(1, ((cnt + 31) / 32 + TPI - 1) / TPI);
    const int local = item - A.item_off[vrow];
    // consecutive items take one record chunk through the row's chirp groups
    // and sample segments, so that the chunk's facet records and kinematics
    // rows, read from HBM by the first of them, are L2 hits for the others;
    // the partial sums keep their (chirp group, segment)-major slots, which
    // the reduction adds in chunk order
    const int nrs = ngroups * W;
    const int jchunk = local / nrs;
    const int rowseg = local % nrs;
    const int64_t pslot = (int64_t)A.item_off[vrow] + (int64_t)rowseg * ipu + jchunk;
    const int seg = rowseg % W, grp = rowseg / W;
    const int rbeg = jchunk * TPI * 32;
    const int rend = min(cnt, rbeg + TPI * 32);
    const int nl_raw = grp * RPW + row;
    const bool row_ok = nl_raw < nc;
    const int nl = row_ok ? nl_raw : 0;
    const int n = A.n0 + nl;
    const int tx = o / Q, rx = o % Q;
    const int m0 = (seg * LPR + col) * S;
    const float fm0 = (float)m0;
    const float fm0sq = fm0 * fm0;
    // the within-chirp quadratic phase p2 ((m0 + s)^2 - m0^2) is followed by a
    // constant step of p2 (2 m0 + S - 1) per sample: exact at s = 0 and
    // s = S - 1, off by at most p2 (S - 1)^2 / 4 cycles in between
    const float eps_lane = 6.283185307179586f * (2.f * fm0 + (float)(S - 1));   // times p2
    const float ptx[3] = {K.ant[tx][0], K.ant[tx][1], K.ant[tx][2]};
    const float prx[3] = {K.ant[P + rx][0], K.ant[P + rx][1], K.ant[P + rx][2]};
    const int slot = A.rd.tdm ? tx : 0;        // time-division MIMO: TX p in slot p
    const float tn = (float)(n * A.rd.slots + slot) * K.tc;

    // per-tile partial sums: samples (2k, 2k+1) of the lane packed in one pair
    // (an odd S computes one extra sample in the last pair and drops it)
    uint64_t PR[S2], PI[S2];
    const uint64_t zero2 = pk2(0.f, 0.f);
#pragma unroll
    for (int k = 0; k < S2; ++k) {
        PR[k] = PI[k] = zero2;
        sAcc[warp][0][k][lane] = zero2;
        sAcc[warp][1][k][lane] = zero2;
        sAcc[warp][2][k][lane] = zero2;
        sAcc[warp][3][k][lane] = zero2;
    }

    const int32_t *list = A.vis_idx + (int64_t)o * F + (A.vstart ? A.vstart[vrow] : 0);
    // kinematics rows of this channel's TX and RX, evaluated at chirp slot sl
    const int sl = n * A.rd.slots + slot;
    const float tau_s = (float)sl - K.s_mid;
    const float4 *kin_t = A.kin + (int64_t)tx * F * kKinRow;
    const float4 *kin_r = A.kin + (int64_t)(P + rx) * F * kKinRow;
    const double *quad_t = A.kquad + (int64_t)tx * F * kKinQuadWords;
    const double *quad_r = A.kquad + (int64_t)(P + rx) * F * kKinQuadWords;
    MixRow wrow;
    wrow.kin_t = kin_t;
    wrow.kin_r = kin_r;
    wrow.quad_t = quad_t;
    wrow.quad_r = quad_r;
    wrow.sl = sl;
    wrow.ant_t = tx;
    wrow.ant_r = P + rx;
    wrow.tau_s = tau_s;
    wrow.tn = tn;
#pragma unroll
    for (int r = 0; r < 3; ++r) {
        wrow.ptx[r] = ptx[r];
        wrow.prx[r] = prx[r];
    }

    for (int base = rbeg; base < rend; base += LPR) {
        // ---------------- build one record per lane ----------------
        const bool valid = row_ok && base + col < rend;
        int cls = -1;
        if (valid) cls = build_mixed_record(A, K, wrow, list[base + col], sRec[warp][lane].f);
        __syncwarp();
        const unsigned int mv = __ballot_sync(0xffffffffu, cls == kRecVertex);
        const unsigned int ms = __ballot_sync(0xffffffffu, cls == kRecSeries || cls == kRecEdge);
        const unsigned int mser = __ballot_sync(0xffffffffu, cls == kRecSeries);
        nV += __popc(mv);
        nSr += __popc(mser);
        nE += __popc(ms & ~mser);
        // each lane walks its row's records; rows of one warp normally share
        // the record forms (same facets, neighbouring chirps), so the
        // branches below rarely diverge
        for (int ii = 0; ii < LPR; ++ii) {
            const int i = row * LPR + ii;
            if ((mv >> i) & 1u) {
                // ------- vertex form: a three-term recurrence per vertex -------
                // e^{j(phi + (s+2) a)} = 2 cos(a) e^{j(phi + (s+1) a)} - e^{j(phi + s a)}:
                // on sample pairs (2k, 2k+1) with the two-sample angle, one FMA
                // per pair and component.  Pair k is held times sg(k) = +1 for
                // k mod 4 in {0, 1}, else -1, so that the recurrence needs no
                // negated addend: held(k) = sg(k) sg(k-1) c2 held(k-1) + held(k-2).
                // 128-bit broadcast loads of the record
                const float4 *R4 = reinterpret_cast<const float4 *>(sRec[warp][i].f);
                const float4 q0 = R4[0], q1 = R4[1], q2v = R4[2], q3 = R4[3], q4 = R4[4],
                             q5 = R4[5];
                const float ph0[3] = {q0.x, q0.y, q0.z};
                const float lo[3] = {q0.w, q1.x, q1.y};
                const float wv[3] = {q1.z, q1.w, q2v.x};
                const float sre[3] = {q2v.y, q2v.z, q2v.w};
                const float sim[3] = {q3.x, q3.y, q3.z};
                const float c2x2[3] = {q4.y, q4.z, q4.w};     // 2 cos(2 step)
                const float s2x4[3] = {q5.x, q5.y, q5.z};     // 4 sin(2 step)
                const float hi = q3.w, p2 = q4.x;
                // the vertices' common phase at the lane's first sample
                const float tq = red1(hi * fm0) + p2 * fm0sq;
                const float eps = p2 * eps_lane;
    #pragma unroll
                for (int v = 0; v < 3; ++v) {
                    const float thv = red1(fmaf(lo[v], fm0, ph0[v] + tq));
                    float zs, zc;
                    __sincosf(6.283185307179586f * thv, &zs, &zc);
                    zc *= wv[v];
                    zs *= wv[v];
                    // the lane's step (angle + eps) and its doubled cosines
                    const float stc = fmaf(-eps, sim[v], sre[v]);
                    const float sts = fmaf(eps, sre[v], sim[v]);
                    const float a1 = 2.f * stc;
                    const float a2 = fmaf(-eps, s2x4[v], c2x2[v]);
                    // samples m0 + 1 (rotation), m0 + 2 and m0 + 3 (recurrence)
                    const float zc1 = fmaf(zc, stc, -zs * sts), zs1 = fmaf(zc, sts, zs * stc);
                    const float zc2 = fmaf(a1, zc1, -zc), zs2 = fmaf(a1, zs1, -zs);
                    const float zc3 = fmaf(a1, zc2, -zc1), zs3 = fmaf(a1, zs2, -zs1);
                    uint64_t XC = pk2(zc, zc1), XS = pk2(zs, zs1);       // held(k - 1)
                    uint64_t YC = pk2(zc2, zc3), YS = pk2(zs2, zs3);     // held(k)
                    const uint64_t A2 = pk2(a2, a2), NA2 = pk2(-a2, -a2);
                    PR[0] = fadd2(PR[0], XC);
                    PI[0] = fadd2(PI[0], XS);
                    if (S2 > 1) {
                        PR[1] = fadd2(PR[1], YC);
                        PI[1] = fadd2(PI[1], YS);
                    }
    #pragma unroll
                    for (int k = 2; k < S2; ++k) {
                        const bool neg = (k & 2) != 0;                   // sg(k) = -1
                        const uint64_t A = (((k - 1) & 2) != 0) != neg ? NA2 : A2;
                        const uint64_t NC = ffma2(A, YC, XC), NS = ffma2(A, YS, XS);
                        XC = YC;
                        XS = YS;
                        YC = NC;
                        YS = NS;
                        if (neg) {
                            PR[k] = fsub2(PR[k], YC);
                            PI[k] = fsub2(PI[k], YS);
                        } else {
                            PR[k] = fadd2(PR[k], YC);
                            PI[k] = fadd2(PI[k], YS);
                        }
                    }
                }
        
            } else if ((ms >> i) & 1u) {
                // ---------------- series / edge forms: per sample ----------------
                const bool series = (mser >> i) & 1u;
                const float *R = sRec[warp][i].f;
    #pragma unroll
                for (int j = 0; j < S; ++j) {
                    float dr, di;
                    series_edge_term(R, series, (float)(m0 + j), K, dr, di);
                    // into sample j's half of its pair
                    const uint64_t DR = (j & 1) ? pk2(0.f, dr) : pk2(dr, 0.f);
                    const uint64_t DI = (j & 1) ? pk2(0.f, di) : pk2(di, 0.f);
                    PR[j >> 1] = fadd2(PR[j >> 1], DR);
                    PI[j >> 1] = fadd2(PI[j >> 1], DI);
                }
        
            }
        }
        // ---------------- Kahan-compensated tile accumulation ----------------
#pragma unroll
        for (int k = 0; k < S2; ++k) {
            uint64_t sr = sAcc[warp][0][k][lane], si = sAcc[warp][1][k][lane];
            uint64_t cr = sAcc[warp][2][k][lane], ci = sAcc[warp][3][k][lane];
            uint64_t y = fsub2(PR[k], cr);
            uint64_t t = fadd2(sr, y);
            cr = fsub2(fsub2(t, sr), y);
            sr = t;
            y = fsub2(PI[k], ci);
            t = fadd2(si, y);
            ci = fsub2(fsub2(t, si), y);
            si = t;
            sAcc[warp][0][k][lane] = sr;
            sAcc[warp][1][k][lane] = si;
            sAcc[warp][2][k][lane] = cr;
            sAcc[warp][3][k][lane] = ci;
            PR[k] = PI[k] = zero2;
        }
        __syncwarp();
    }
    // unscaled partial sums of this item
    float2 *dst = A.partial + pslot * (32 * S) + lane * S;
#pragma unroll
    for (int k = 0; k < S2; ++k) {
        float r0, r1, i0, i1;
        upk2(sAcc[warp][0][k][lane], r0, r1);
        upk2(sAcc[warp][1][k][lane], i0, i1);
        dst[2 * k] = make_float2(r0, i0);
        if (2 * k + 1 < S) dst[2 * k + 1] = make_float2(r1, i1);
    }
    __syncwarp();
    }   // item loop
    if (lane == 0 && A.counters) {
        atomicAdd(A.counters + 0, nV);
        atomicAdd(A.counters + 1, nSr);
        atomicAdd(A.counters + 2, nE);
    }
}

// item table: row v (scene * O + channel) owns ipu_v = ceil(ceil(cnt_v / 32)
// / TPI) record chunks (at least one) per (chirp group, sample segment);
// item_off is their prefix (one block-wide scan)
__global__ void synth_items_kernel(const int32_t *__restrict__ vcnt, int VO, int TPI, int nc,
                                   int RPW, int W, int32_t *__restrict__ item_off, int *counter)
{
    __shared__ int s_warp[32];
    __shared__ int s_run;
    const int ngroups = (nc + RPW - 1) / RPW;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    if (threadIdx.x == 0) s_run = 0;
    __syncthreads();
    for (int v0 = 0; v0 < VO; v0 += blockDim.x) {
        const int v = v0 + threadIdx.x;
        const int mine = v < VO ? max(1, ((vcnt[v] + 31) / 32 + TPI - 1) / TPI) * ngroups * W : 0;
        int x = mine;
        for (int off = 1; off < 32; off <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, x, off);
            if (lane >= off) x += y;
        }
        if (lane == 31) s_warp[warp] = x;
        __syncthreads();
        if (warp == 0) {
            int w = lane < nw ? s_warp[lane] : 0;
            for (int off = 1; off < 32; off <<= 1) {
                const int y = __shfl_up_sync(0xffffffffu, w, off);
                if (lane >= off) w += y;
            }
            if (lane < nw) s_warp[lane] = w;
        }
        __syncthreads();
        const int before = s_run + (warp > 0 ? s_warp[warp - 1] : 0) + x - mine;
        if (v < VO) item_off[v] = before;
        __syncthreads();
        if (threadIdx.x == 0) s_run += s_warp[nw - 1];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        item_off[VO] = s_run;
        *counter = 0;
    }
}

// sums the item partials of each (channel, chirp, sample) in item order with
// Kahan compensation, and applies C / k_m^2 = out_scale / kappa_m^2
__global__ void synth_reduce_kernel(const float2 *__restrict__ partial,
                                    const int32_t *__restrict__ item_off,
                                    const int32_t *__restrict__ vcnt, int TPI, int W, int S,
                                    int LPR, int O, int N, int M, int n0, float out_scale,
                                    float kap_step, void *out, int out_c64)
{
    const int m = blockIdx.x * blockDim.x + threadIdx.x;
    const int nl = blockIdx.y, o = blockIdx.z;
    if (m >= M) return;
    const int RPW = 32 / LPR;
    const int grp = nl / RPW, row = nl % RPW;
    const int seg = m / (LPR * S), ml = m % (LPR * S);
    const int slot = (row * LPR + ml / S) * S + ml % S;     // lane * S + j
    const int ipu = max(1, ((vcnt[o] + 31) / 32 + TPI - 1) / TPI);
    const int64_t it0 = (int64_t)item_off[o] + (int64_t)(grp * W + seg) * ipu;
    const float2 *src = partial + it0 * (32 * S) + slot;
    float sr = 0.f, si = 0.f, cr = 0.f, ci = 0.f;
    for (int j = 0; j < ipu; ++j) {
        const float2 p = src[(int64_t)j * (32 * S)];
        float y = p.x - cr, t = sr + y;
        cr = (t - sr) - y;
        sr = t;
        y = p.y - ci;
        t = si + y;
        ci = (t - si) - y;
        si = t;
    }
    const float kp = fmaf((float)m, kap_step, 1.f);
    const float sc = out_scale / (kp * kp);
    const int64_t idx = ((int64_t)o * N + n0 + nl) * M + m;
    if (out_c64) reinterpret_cast<float2 *>(out)[idx] = make_float2(sr * sc, si * sc);
    else reinterpret_cast<double2 *>(out)[idx] = make_double2((double)sr * sc, (double)si * sc);
}

// consecutive samples per lane: the largest S in {8, 4, 2, 1} with 32 S | M;
// a (channel, chirp) row of M samples then takes W = M / (32 S) warps
static int samples_per_lane(int M)
{
    for (int S = 8; S > 1; S >>= 1)
        if (M % (32 * S) == 0) return S;
    return 1;
}


// 32-record tiles per work item: at least 16 (512 records), more for large
// scenes so that a channel row splits into at most 64 items; the partial
// sums cost one 8-byte store and load per sample and item
int synth_tiles_per_item(int64_t F) { return (int)std::max<int64_t>(16, ((F + 31) / 32 + 63) / 64); }

// lane layout of the mixed kernel: S samples per lane, LPR lanes per chirp
// row, W warps per row.  16 samples per lane halve the per-lane start-up
// work (MUFU start phasors, the first samples of each recurrence) against
// 8; S_req = 8 asks for the 8-sample layout where M allows it, S_req = 32
// for 32 samples per lane (M = 256, 512, 1024: half the per-lane start-up
// work again, at fewer resident warps; autotuner candidates).
struct MixLayout {
    int S, LPR, W;
};
static MixLayout mix_layout(int M, int S_req)
{
    if (S_req == 32 && (M == 256 || M == 512 || M == 1024)) return {32, M / 32, 1};
    if (S_req == 8) {
        if (M <= 256 && 256 % M == 0) return {8, M / 8, 1};
        if (M % 256 == 0) return {8, 32, M / 256};
    }
    if (M <= 512 && 512 % M == 0) return {16, M / 16, 1};
    if (M % 512 == 0) return {16, 32, M / 512};
    const int S = samples_per_lane(M);
    return {S, 32, M / (32 * S)};
}

int synth_layout_samples(int M, int S_req) { return mix_layout(M, S_req).S; }

int64_t synth_max_items(const int64_t *scene_F, int n_scene, const RadarDev &rd, int nc, int tpi,
                        int S_req)
{
    const MixLayout L = mix_layout(rd.M, S_req);
    const int RPW = 32 / L.LPR;
    int64_t per_group = 0;
    for (int b = 0; b < n_scene; ++b) {
        const int64_t tiles = (scene_F[b] + 31) / 32;
        per_group += std::max<int64_t>(1, (tiles + tpi - 1) / tpi);
    }
    return (int64_t)rd.O * per_group * ((nc + RPW - 1) / RPW) * L.W;
}

int64_t synth_partial_words(const int64_t *scene_F, int n_scene, const RadarDev &rd, int nc,
                            int tpi, int S_req)
{
    return synth_max_items(scene_F, n_scene, rd, nc, tpi, S_req) * 32 * mix_layout(rd.M, S_req).S;
}

template <int S, int LPR> static int mixed_grid(int64_t items)
{
    static int blocks_per_sm = -1, sms = 0;
    if (blocks_per_sm < 0) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks_per_sm, synth_mixed_kernel<S, LPR>,
                                                      kMixWarps * 32, 0);
        if (blocks_per_sm < 1) blocks_per_sm = 1;
    }
    const int64_t need = (items + kMixWarps - 1) / kMixWarps;
    return (int)std::max<int64_t>(1, std::min<int64_t>(need, (int64_t)blocks_per_sm * sms));
}

template <int S, int LPR>
static void run_mixed(const SynthArgs &a, const MixConsts &K, int W, int64_t items, cudaStream_t s)
{
    synth_mixed_kernel<S, LPR><<<mixed_grid<S, LPR>(items), kMixWarps * 32, 0, s>>>(a, K, W);
}

void launch_synth_mixed(const SynthArgs &a0, cudaStream_t s)
{
    SynthArgs a = a0;
    const MixConsts K = mix_consts(a.rd);
    const int M = a.rd.M;
    const MixLayout L = mix_layout(M, a.layout_S);
    synth_items_kernel<<<1, 1024, 0, s>>>(a.vcnt, a.VO, a.tiles_per_item, a.nc, 32 / L.LPR,
                                          L.W, a.item_off, a.item_counter);
    const int64_t items = a.max_items;
    if (L.S == 32) {
        switch (L.LPR) {
        case 8: run_mixed<32, 8>(a, K, L.W, items, s); break;
        case 16: run_mixed<32, 16>(a, K, L.W, items, s); break;
        default: run_mixed<32, 32>(a, K, L.W, items, s); break;
        }
    } else if (L.S == 16) {
        switch (L.LPR) {
        case 2: run_mixed<16, 2>(a, K, L.W, items, s); break;
        case 4: run_mixed<16, 4>(a, K, L.W, items, s); break;
        case 8: run_mixed<16, 8>(a, K, L.W, items, s); break;
        case 16: run_mixed<16, 16>(a, K, L.W, items, s); break;
        default: run_mixed<16, 32>(a, K, L.W, items, s); break;
        }
    } else if (L.S == 8) {
        switch (L.LPR) {
        case 4: run_mixed<8, 4>(a, K, L.W, items, s); break;
        case 8: run_mixed<8, 8>(a, K, L.W, items, s); break;
        case 16: run_mixed<8, 16>(a, K, L.W, items, s); break;
        default: run_mixed<8, 32>(a, K, L.W, items, s); break;
        }
    } else {
        switch (L.S) {
        case 4: run_mixed<4, 32>(a, K, L.W, items, s); break;
        case 2: run_mixed<2, 32>(a, K, L.W, items, s); break;
        default: run_mixed<1, 32>(a, K, L.W, items, s); break;
        }
    }
    dim3 rg((unsigned int)((M + 255) / 256), (unsigned int)a.nc, (unsigned int)a.VO);
    synth_reduce_kernel<<<rg, 256, 0, s>>>(a.partial, a.item_off, a.vcnt, a.tiles_per_item, L.W,
                                           L.S, L.LPR, a.rd.O, a.rd.N, M, a.n0, K.out_scale,
                                           K.kap_step, a.out, a.out_c64);
}

// -------------------------------------------------------------------------
// plain FP64 path
// -------------------------------------------------------------------------
struct __align__(16) RecD {
    int kind, flags;
    double qt[3];     // R_t(t)^2 = qt0 + t (qt1 + t qt2), t = fast time
    double qr[2];     // R_r(t)^2 = qr0 + t (qr1 + t qt2)
    double ls;        // path-length shift of the delay (reference-point form)
    double d[22];
};

constexpr int kF64Warps = 4;

template <int S>
__global__ void __launch_bounds__(kF64Warps * 32)
synth_fp64_kernel(SynthArgs A, int W, int NCH)
{
    __shared__ RecD sR[kF64Warps][32];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t gw = (int64_t)blockIdx.x * kF64Warps + warp;
    const int N = A.rd.N;
    // warp = (row unit, sample segment, chunk of the row's facet list)
    const int64_t unit = gw / ((int64_t)W * NCH);
    const int seg = (int)(gw / NCH % W), chunk = (int)(gw % NCH);
    if (unit >= (int64_t)A.VO * N) return;
    const int vrow = (int)(unit / N), n = (int)(unit % N);   // scene * O + channel
    const int o = vrow % A.rd.O;
    const int P = A.rd.P, Q = A.rd.Q;
    const int tx = o / Q, rx = o % Q;
    const int64_t F = A.F;
    const int m0 = (seg * 32 + lane) * S;
    const double c = kC0, f0 = A.rd.f0, mu = A.rd.slope, fs = A.rd.fs;
    const double f_max = f0 + mu * (A.rd.M - 1) / fs;
    const double k0 = 2.0 * kPi * f0 / c, kmax = 2.0 * kPi * f_max / c;
    // chirp start of this channel: time-division MIMO puts TX p in slot p
    const double tn = (double)((int64_t)n * A.rd.slots + (A.rd.tdm ? tx : 0)) * A.rd.Tc;
    const double *ptx = A.rd.ant[tx];
    const double *prx = A.rd.ant[P + rx];

    double accr[S], acci[S];
#pragma unroll
    for (int j = 0; j < S; ++j) accr[j] = acci[j] = 0.0;

    const int32_t *list = A.vis_idx + (int64_t)o * F + (A.vstart ? A.vstart[vrow] : 0);
    const int cnt = A.vcnt[vrow];
    unsigned long long nV = 0, nSr = 0, nE = 0;

    const int nbat = (cnt + 31) / 32;
    const int bat0 = (int)((int64_t)nbat * chunk / NCH);
    const int bat1 = (int)((int64_t)nbat * (chunk + 1) / NCH);
    for (int base = bat0 * 32; base < bat1 * 32; base += 32) {
        const bool valid = base + lane < cnt;
        int cls = -1;
        if (valid) {
            const int64_t k = list[base + lane];
            RecD &R = sR[warp][lane];
            const int inst = A.fac[k].inst;
            const double vel[3] = {A.vel64[3 * inst], A.vel64[3 * inst + 1],
                                   A.vel64[3 * inst + 2]};
            double tri[9], c0[3], rec[kRecEntries];
            for (int i = 0; i < 9; ++i) tri[i] = A.tri64[9 * k + i];
            for (int r = 0; r < 3; ++r) c0[r] = A.c64[3 * k + r];
            int flags = 0;
            cls = R.kind = build_record<double>(
                tri, c0, vel, tn, ptx, prx, (double)A.fac[k].rho, A.rd.intra, k0, kmax,
                A.rd.far_field ? kDelayFarField : A.rd.delay_ref ? kDelayRef : kDelayFacet,
                A.ref64 + 3 * inst, A.fac[k].two_sided, rec, &flags);
            R.flags = flags;
            R.qt[0] = rec[0];
            R.qt[1] = rec[1];
            R.qt[2] = rec[2];
            R.qr[0] = rec[3];
            R.qr[1] = rec[4];
            R.ls = rec[kRecLs];
            for (int i = 0; i < 22; ++i) R.d[i] = rec[kRecD + i];
        }
        __syncwarp();
        unsigned int mask = __ballot_sync(0xffffffffu, valid);
        const unsigned int a1 = __ballot_sync(0xffffffffu, cls == kRecVertex);
        const unsigned int a2 = __ballot_sync(0xffffffffu, cls == kRecSeries);
        nV += __popc(a1);
        nSr += __popc(a2);
        nE += __popc(mask & ~a1 & ~a2);
        // reciprocals formed once: products instead of FP64 divisions per sample
        const double inv_fs = 1.0 / fs, inv_c = 1.0 / c, inv_f0 = 1.0 / f0;
        const double mu_2c2 = mu / (2.0 * c * c);
        while (mask) {
            const int i = __ffs(mask) - 1;
            mask &= mask - 1;
            const RecD &R = sR[warp][i];
#pragma unroll 1
            for (int j = 0; j < S; ++j) {
                const double t = (double)(m0 + j) * inv_fs;
                const double fm = f0 + mu * t;
                const double L = sqrt(R.qt[0] + t * (R.qt[1] + t * R.qt[2])) +
                                 sqrt(R.qr[0] + t * (R.qr[1] + t * R.qt[2]));
                const double fmc = fm * inv_c;
                const double kp = fm * inv_f0;
                // residual video phase: the origin's path (reference-point
                // form), else the facet's own, plane-wave in the far field
                const double Lv = A.rd.far_field ? L + R.ls : L;
                double thc = fmc * (L + R.ls) - mu_2c2 * Lv * Lv;
                thc -= rint(thc);
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
    const int64_t row = ((int64_t)vrow * N + n) * A.rd.M + m0;
#pragma unroll
    for (int j = 0; j < S; ++j) {
        const double fm = f0 + mu * (double)(m0 + j) / fs;
        const double km = 2.0 * kPi * fm / c;
        const double sc = camp / (km * km);
        if (NCH > 1) {           // this chunk's scaled partial sums, added in order later
            reinterpret_cast<double2 *>(A.partial)[(int64_t)chunk * A.VO * N * A.rd.M + row + j] =
                make_double2(accr[j] * sc, acci[j] * sc);
        } else if (A.out_c64) {
            reinterpret_cast<float2 *>(A.out)[row + j] =
                make_float2((float)(accr[j] * sc), (float)(acci[j] * sc));
        } else {
            reinterpret_cast<double2 *>(A.out)[row + j] = make_double2(accr[j] * sc, acci[j] * sc);
        }
    }
}

// sums the chunks' partial sums of each (row, sample) in chunk order
__global__ void synth_fp64_reduce_kernel(const double2 *__restrict__ partial, int64_t n, int NCH,
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
    if (out_c64) reinterpret_cast<float2 *>(out)[i] = make_float2((float)re, (float)im);
    else reinterpret_cast<double2 *>(out)[i] = make_double2(re, im);
}

template <int S> static int fp64_blocks_per_sm()
{
    static int b = -1;
    if (b < 0) {
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, synth_fp64_kernel<S>, kF64Warps * 32, 0);
        if (b < 1) b = 1;
    }
    return b;
}

// chunks of each row's facet list: about four waves of resident blocks (a
// warp per chirp row alone leaves a single sedan, 1536 rows, a fraction of
// a wave), at most one 32-facet batch per chunk and 64 chunks
int synth_fp64_chunks(const RadarDev &rd, int VO, int64_t F)
{
    const int M = rd.M;
    const int S = samples_per_lane(M);
    const int W = M / (32 * S);
    static int sms = 0;
    if (sms <= 0) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (sms <= 0) sms = 1;
    }
    const int bps = S == 8 ? fp64_blocks_per_sm<8>() : S == 4 ? fp64_blocks_per_sm<4>()
                  : S == 2 ? fp64_blocks_per_sm<2>() : fp64_blocks_per_sm<1>();
    const int64_t rows = (int64_t)VO * rd.N * W;
    const int64_t target = 4 * (int64_t)sms * bps * kF64Warps;
    const int64_t maxb = std::min<int64_t>(64, std::max<int64_t>(1, (F + 31) / 32));
    return (int)std::max<int64_t>(1, std::min<int64_t>(maxb, (target + rows - 1) / rows));
}

void launch_synth_fp64(const SynthArgs &a, cudaStream_t s)
{
    const int M = a.rd.M;
    const int S = samples_per_lane(M);
    const int W = M / (32 * S);
    const int NCH = a.partial ? synth_fp64_chunks(a.rd, a.VO, a.F) : 1;
    const int64_t warps = (int64_t)a.VO * a.rd.N * W * NCH;
    const unsigned int grid = (unsigned int)((warps + kF64Warps - 1) / kF64Warps);
    switch (S) {
    case 8: synth_fp64_kernel<8><<<grid, kF64Warps * 32, 0, s>>>(a, W, NCH); break;
    case 4: synth_fp64_kernel<4><<<grid, kF64Warps * 32, 0, s>>>(a, W, NCH); break;
    case 2: synth_fp64_kernel<2><<<grid, kF64Warps * 32, 0, s>>>(a, W, NCH); break;
    default: synth_fp64_kernel<1><<<grid, kF64Warps * 32, 0, s>>>(a, W, NCH); break;
    }
    if (NCH > 1) {
        const int64_t n = (int64_t)a.VO * a.rd.N * M;
        synth_fp64_reduce_kernel<<<(unsigned int)((n + 255) / 256), 256, 0, s>>>(
            reinterpret_cast<const double2 *>(a.partial), n, NCH, a.out, a.out_c64);
    }
}

}  // namespace bart
