// The per-(facet, channel, chirp) record of the plain FP64 echo synthesis,
// built by one templated routine: in double for the forward synthesis, and
// in forward-mode dual numbers for the adjoint (derivative of every record
// entry with respect to one facet parameter: a world vertex coordinate at
// the frame start, or the reflectivity).
//
// Record entries (kRecEntries doubles):
//   [0..2] qt: R_t(t)^2 = qt0 + t (qt1 + t qt2), t = fast time
//   [3..4] qr: R_r(t)^2 = qr0 + t (qr1 + t qt2)
//   [5]    ls: path-length shift; the delay path is L(t) + ls, the residual
//              video phase uses L(t) alone
//   [6..]  d:  form coefficients (vertex / series / edge, see synth.cu)
// Per-facet delay form: qt, qr from the facet centroid, ls = 0.  Reference-
// point form (Eqs. 11-13 per target): qt, qr from the instance origin and
// ls = L_facet - L_origin at the chirp start.  Far field: directions, ranges
// and qt, qr from the instance origin, ls = -(t + r).(c - origin), the
// plane-wave path shift (the residual video phase then uses L(t) + ls too).
#pragma once

#include "bart_internal.cuh"

namespace bart {

constexpr int kRecEntries = 28;
constexpr int kRecLs = 5;           // path-length shift entry
constexpr int kRecD = 6;            // first d[] entry

// 1/n!, n = 0..17 (series form of the facet integral)
static __constant__ double c_inv_fact[18] = {
    1.0, 1.0, 1.0 / 2, 1.0 / 6, 1.0 / 24, 1.0 / 120, 1.0 / 720, 1.0 / 5040, 1.0 / 40320,
    1.0 / 362880, 1.0 / 3628800, 1.0 / 39916800, 1.0 / 479001600, 1.0 / 6227020800.0,
    1.0 / 87178291200.0, 1.0 / 1307674368000.0, 1.0 / 20922789888000.0,
    1.0 / 355687428096000.0};

// value + one directional derivative
struct Dual {
    double v, d;
    __device__ Dual() {}
    __device__ explicit Dual(double x) : v(x), d(0.0) {}
    __device__ Dual(double x, double y) : v(x), d(y) {}
};
__device__ __forceinline__ Dual operator+(Dual a, Dual b) { return Dual{a.v + b.v, a.d + b.d}; }
__device__ __forceinline__ Dual operator-(Dual a, Dual b) { return Dual{a.v - b.v, a.d - b.d}; }
__device__ __forceinline__ Dual operator-(Dual a) { return Dual{-a.v, -a.d}; }
__device__ __forceinline__ Dual operator*(Dual a, Dual b) { return Dual{a.v * b.v, a.d * b.v + a.v * b.d}; }
__device__ __forceinline__ Dual operator/(Dual a, Dual b)
{
    const double q = a.v / b.v;
    return Dual{q, (a.d - q * b.d) / b.v};
}
__device__ __forceinline__ Dual operator+(Dual a, double b) { return Dual{a.v + b, a.d}; }
__device__ __forceinline__ Dual operator-(Dual a, double b) { return Dual{a.v - b, a.d}; }
__device__ __forceinline__ Dual operator-(double a, Dual b) { return Dual{a - b.v, -b.d}; }
__device__ __forceinline__ Dual operator*(Dual a, double b) { return Dual{a.v * b, a.d * b}; }
__device__ __forceinline__ Dual operator*(double a, Dual b) { return Dual{a * b.v, a * b.d}; }
__device__ __forceinline__ Dual operator/(Dual a, double b) { return Dual{a.v / b, a.d / b}; }
// square root of a double or a dual number
__device__ __forceinline__ double sqrt_s(double a) { return ::sqrt(a); }
__device__ __forceinline__ Dual sqrt_s(Dual a)
{
    const double r = ::sqrt(a.v);
    return Dual{r, a.d / (2.0 * r)};
}
__device__ __forceinline__ double val(double a) { return a; }
__device__ __forceinline__ double val(Dual a) { return a.v; }

// delay forms of build_record
constexpr int kDelayFacet = 0;      // spherical waves from the facet centroid
constexpr int kDelayRef = 1;        // reference-point form (Eqs. 11-13 per target)
constexpr int kDelayFarField = 2;   // plane waves from the instance origin

__device__ __forceinline__ double abs_s(double a) { return fabs(a); }
__device__ __forceinline__ Dual abs_s(Dual a) { return a.v < 0.0 ? -a : a; }

// Builds the record of one facet for channel antennas ptx/prx at chirp time
// tn.  tri: world vertices at t0 (9), c0: the stored centroid at t0 (3), vel:
// instance velocity, rho: reflectivity, form: kDelay*, ref: the instance
// origin at t0 (used by the reference-point and far-field forms), two_sided:
// obliquity |n.(t + r)|/2 (the side the antennas light).  Returns the form
// (kRec*), the sinc flags of the edge form in *flags.  Branches depend on
// values only, so the double and dual builds take the same path.
template <typename Sc>
__device__ __forceinline__ int build_record(const Sc *tri, const Sc *c0, const double *vel,
                                            double tn, const double *ptx, const double *prx,
                                            Sc rho, int intra, double k0, double kmax,
                                            int form, const double *ref, int two_sided, Sc *out,
                                            int *flags)
{
    Sc cc[3], dv[9];
    for (int r = 0; r < 3; ++r) cc[r] = c0[r];
    for (int i = 0; i < 9; ++i) dv[i] = tri[i] - cc[i % 3];
    for (int r = 0; r < 3; ++r) cc[r] = cc[r] + vel[r] * tn;
    const Sc e1[3] = {dv[3] - dv[0], dv[4] - dv[1], dv[5] - dv[2]};
    const Sc e2[3] = {dv[6] - dv[0], dv[7] - dv[1], dv[8] - dv[2]};
    Sc nn[3] = {e1[1] * e2[2] - e1[2] * e2[1], e1[2] * e2[0] - e1[0] * e2[2],
                e1[0] * e2[1] - e1[1] * e2[0]};
    const Sc nl = sqrt_s(nn[0] * nn[0] + nn[1] * nn[1] + nn[2] * nn[2]);
    const Sc area = 0.5 * nl;
    for (int r = 0; r < 3; ++r) nn[r] = nn[r] / nl;
    // the instance origin at the chirp start (a constant of the facet
    // parameters) and the channel's vectors from it
    double gt[3] = {0.0, 0.0, 0.0}, gr[3] = {0.0, 0.0, 0.0}, ro[3] = {0.0, 0.0, 0.0};
    if (form != kDelayFacet)
        for (int r = 0; r < 3; ++r) {
            ro[r] = ref[r] + vel[r] * tn;
            gt[r] = ptx[r] - ro[r];
            gr[r] = prx[r] - ro[r];
        }
    const double qt0 = gt[0] * gt[0] + gt[1] * gt[1] + gt[2] * gt[2];
    const double qr0 = gr[0] * gr[0] + gr[1] * gr[1] + gr[2] * gr[2];
    Sc dt[3], dr[3];
    for (int r = 0; r < 3; ++r) {
        dt[r] = form == kDelayFarField ? Sc(gt[r]) : ptx[r] - cc[r];
        dr[r] = form == kDelayFarField ? Sc(gr[r]) : prx[r] - cc[r];
    }
    const Sc Rt2 = dt[0] * dt[0] + dt[1] * dt[1] + dt[2] * dt[2];
    const Sc Rr2 = dr[0] * dr[0] + dr[1] * dr[1] + dr[2] * dr[2];
    const Sc Rt = sqrt_s(Rt2), Rr = sqrt_s(Rr2);
    Sc b[3];
    for (int r = 0; r < 3; ++r) b[r] = dt[r] / Rt + dr[r] / Rr;
    Sc ok = 0.5 * (nn[0] * b[0] + nn[1] * b[1] + nn[2] * b[2]);
    if (two_sided) ok = abs_s(ok);
    const Sc g = rho * ok / (Rt * Rr);
    if (form == kDelayFacet) {
        out[0] = Rt2;
        out[3] = Rr2;
        out[kRecLs] = Sc(0.0);
        if (intra) {
            out[1] = -2.0 * (dt[0] * vel[0] + dt[1] * vel[1] + dt[2] * vel[2]);
            out[4] = -2.0 * (dr[0] * vel[0] + dr[1] * vel[1] + dr[2] * vel[2]);
        }
    } else {
        // the origin's path polynomial; the facet enters through ls
        out[0] = Sc(qt0);
        out[3] = Sc(qr0);
        if (form == kDelayRef) {
            out[kRecLs] = (Rt + Rr) - (::sqrt(qt0) + ::sqrt(qr0));
        } else {
            out[kRecLs] = -(b[0] * (cc[0] - ro[0]) + b[1] * (cc[1] - ro[1]) +
                            b[2] * (cc[2] - ro[2]));
        }
        if (intra) {
            out[1] = Sc(-2.0 * (gt[0] * vel[0] + gt[1] * vel[1] + gt[2] * vel[2]));
            out[4] = Sc(-2.0 * (gr[0] * vel[0] + gr[1] * vel[1] + gr[2] * vel[2]));
        }
    }
    if (intra) {
        out[2] = Sc(vel[0] * vel[0] + vel[1] * vel[1] + vel[2] * vel[2]);
    } else {
        out[1] = out[4] = out[2] = Sc(0.0);
    }
    const Sc bn = b[0] * nn[0] + b[1] * nn[1] + b[2] * nn[2];
    const Sc bt[3] = {b[0] - bn * nn[0], b[1] - bn * nn[1], b[2] - bn * nn[2]};
    Sc u[3];
    for (int v = 0; v < 3; ++v)
        u[v] = bt[0] * dv[3 * v] + bt[1] * dv[3 * v + 1] + bt[2] * dv[3 * v + 2];
    const double umin = fmin(fmin(val(u[0]), val(u[1])), val(u[2]));
    const double umax = fmax(fmax(val(u[0]), val(u[1])), val(u[2]));
    const double dmin = fmin(fmin(fabs(val(u[0]) - val(u[1])), fabs(val(u[1]) - val(u[2]))),
                             fabs(val(u[0]) - val(u[2])));
    const Sc A2 = 2.0 * area * g;
    Sc *d = out + kRecD;
    *flags = 0;
    if (kmax * (umax - umin) < kSeriesKD) {
        const Sc ub = (u[0] + u[1] + u[2]) / 3.0;
        d[0] = ub;
        const Sc y0 = k0 * (u[0] - ub), y1 = k0 * (u[1] - ub), y2 = k0 * (u[2] - ub);
        const Sc e2s = y0 * y1 + y0 * y2 + y1 * y2, e3s = y0 * y1 * y2;
        Sc h[kSeriesTerms];
        h[0] = Sc(1.0);
        h[1] = Sc(0.0);
        h[2] = -e2s;
        for (int p = 3; p < kSeriesTerms; ++p) h[p] = -e2s * h[p - 2] + e3s * h[p - 3];
        const Sc sc = A2 * k0 * k0;
        for (int i = 0; i < 8; ++i)
            d[1 + i] = ((i & 1) ? -sc : sc) * h[2 * i] * c_inv_fact[2 * i + 2];
        for (int i = 0; i < 7; ++i)
            d[9 + i] = ((i & 1) ? sc : -sc) * h[2 * i + 1] * c_inv_fact[2 * i + 3];
        return kRecSeries;
    }
    if (kmax * dmin < kEdgeKd) {
        const Sc bt2 = bt[0] * bt[0] + bt[1] * bt[1] + bt[2] * bt[2];
        const Sc nxb[3] = {nn[1] * bt[2] - nn[2] * bt[1], nn[2] * bt[0] - nn[0] * bt[2],
                           nn[0] * bt[1] - nn[1] * bt[0]};
        for (int i = 0; i < 3; ++i) {
            const int i1 = (i + 1) % 3;
            const Sc e[3] = {dv[3 * i1] - dv[3 * i], dv[3 * i1 + 1] - dv[3 * i + 1],
                             dv[3 * i1 + 2] - dv[3 * i + 2]};
            const Sc gam = 0.5 * (u[i1] - u[i]);
            d[3 * i] = 0.5 * (u[i] + u[i1]);
            d[3 * i + 1] = k0 * gam;
            d[3 * i + 2] = k0 * g * (e[0] * nxb[0] + e[1] * nxb[1] + e[2] * nxb[2]) / bt2;
            if (kmax * fabs(val(gam)) < kSincSeries) *flags |= 1 << i;
        }
        return kRecEdge;
    }
    for (int v = 0; v < 3; ++v) {
        const Sc ua = u[v], ub_ = u[(v + 1) % 3], uc = u[(v + 2) % 3];
        d[v] = ua;
        d[3 + v] = -A2 / ((ua - ub_) * (ua - uc));
    }
    return kRecVertex;
}

}  // namespace bart
