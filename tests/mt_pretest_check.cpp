// Host check of the FP32 pre-test of the segment/triangle test (geom64.cuh):
// whenever mt_fp32_classify decides -- 0, a certain miss, or 2, a certain
// hit inside every margin -- the FP64 test mt_segment must return the same.
// Both functions are compiled here, unchanged, as host code: the header's
// FP64 steps name CUDA's round-to-nearest intrinsics, which are plain IEEE
// operations on the host (built with -ffp-contract=off, so every operation
// rounds once, the case the pre-test's error bounds are derived for; the
// device may fuse some FP32 multiply-adds, which only shrinks their error).
//
// Cases (seeded splitmix64): random segments around triangles of 1 mm to
// 5 m at up to 150 m from the origin, and adversarial ones through points at
// barycentric distance 1e-13 .. 1e-3 from an edge or a vertex, with a
// segment end 1e-13 .. 1e-3 (in the segment parameter) from the triangle's
// plane, and nearly parallel to the plane.
// Prints: cases, violations, decided (certain) cases, and the wrong
// decisions of a plain FP32 Moller-Trumbore without error bounds on cases
// the FP64 test does not call grazing (the adversarial cases must provoke
// them, or they would not probe the margins).
// Also: the FP32 slab test (slab_hit) against the triangle's box -- rounded
// outward from the FP64 vertices and padded by 1e-4 + 4e-6 max|coordinate|,
// as the world-facet kernel builds it -- never drops a segment that the
// FP64 test finds hitting or grazing the triangle (printed: slab_drops of
// the hitting or grazing cases).
#include <cmath>
#include <cstdint>
#include <cstdio>

static inline double __dadd_rn(double a, double b) { return a + b; }
static inline double __dsub_rn(double a, double b) { return a - b; }
static inline double __dmul_rn(double a, double b) { return a * b; }
static inline double __ddiv_rn(double a, double b) { return a / b; }

#include "geom64.cuh"

using namespace bart;

static uint64_t g_state = 0x2208109390001ull;
static uint64_t next_u64()
{
    uint64_t z = (g_state += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}
static double uni() { return (double)(next_u64() >> 11) * 0x1.0p-53; }       // [0, 1)
static double sym() { return 2.0 * uni() - 1.0; }                            // [-1, 1)
static double logu(double lo, double hi) { return lo * std::pow(hi / lo, uni()); }

struct Tally {
    long cases = 0, violations = 0, decided = 0, naive_wrong = 0, slab_drops = 0, slab_checked = 0;
};

// plain FP32 test: 0 outside, 2 strictly inside, no rounding bounds
static int naive_fp32(const float *v0, const float *v1, const float *v2, const float *o,
                      const float *d)
{
    float e1[3], e2[3], T[3];
    for (int r = 0; r < 3; ++r) {
        e1[r] = v1[r] - v0[r];
        e2[r] = v2[r] - v0[r];
        T[r] = o[r] - v0[r];
    }
    const float P[3] = {d[1] * e2[2] - d[2] * e2[1], d[2] * e2[0] - d[0] * e2[2],
                        d[0] * e2[1] - d[1] * e2[0]};
    const float det = e1[0] * P[0] + e1[1] * P[1] + e1[2] * P[2];
    if (det == 0.f) return 0;
    const float u = (T[0] * P[0] + T[1] * P[1] + T[2] * P[2]) / det;
    const float Q[3] = {T[1] * e1[2] - T[2] * e1[1], T[2] * e1[0] - T[0] * e1[2],
                        T[0] * e1[1] - T[1] * e1[0]};
    const float v = (d[0] * Q[0] + d[1] * Q[1] + d[2] * Q[2]) / det;
    const float t = (e2[0] * Q[0] + e2[1] * Q[1] + e2[2] * Q[2]) / det;
    const bool in = u > 0.f && v > 0.f && u + v < 1.f && t > 0.f && t < 1.f;
    return in ? 2 : 0;
}

static void check(const double *tri, const double *O, const double *D, Tally &t)
{
    float f[12];
    float X = 0.f;
    for (int i = 0; i < 9; ++i) {
        f[i] = (float)tri[i];
        X = std::fmax(X, std::fabs(f[i]));
    }
    f[9] = X;
    f[10] = f[11] = 0.f;
    const float4 t0 = make_float4(f[0], f[1], f[2], f[3]);
    const float4 t1 = make_float4(f[4], f[5], f[6], f[7]);
    const float4 t2 = make_float4(f[8], f[9], f[10], f[11]);
    const float o[3] = {(float)O[0], (float)O[1], (float)O[2]};
    const float d[3] = {(float)D[0], (float)D[1], (float)D[2]};
    const float Dm = std::fmax(std::fmax(std::fabs(d[0]), std::fabs(d[1])), std::fabs(d[2]));
    const float Om = std::fmax(std::fmax(std::fabs(o[0]), std::fabs(o[1])), std::fabs(o[2]));
    const int pre = mt_fp32_classify(t0, t1, t2, o, d, Dm, Om);
    const int exact = mt_segment(O, D, tri);
    if (exact != 1 && naive_fp32(f, f + 3, f + 6, o, d) != exact) ++t.naive_wrong;
    if (exact != 0) {
        float bmin[3], bmax[3], inv[3], mx = 0.f;
        for (int r = 0; r < 3; ++r) {
            const double lo = std::fmin(std::fmin(tri[r], tri[3 + r]), tri[6 + r]);
            const double hi = std::fmax(std::fmax(tri[r], tri[3 + r]), tri[6 + r]);
            float a = (float)lo, b = (float)hi;
            mx = std::fmax(mx, std::fmax(std::fabs(a), std::fabs(b)));
            if ((double)a > lo) a = std::nextafter(a, -INFINITY);
            if ((double)b < hi) b = std::nextafter(b, INFINITY);
            bmin[r] = a;
            bmax[r] = b;
        }
        const float pad = 1e-4f + 4e-6f * mx;
        for (int r = 0; r < 3; ++r) {
            bmin[r] -= pad;
            bmax[r] += pad;
            float dd = d[r];
            if (std::fabs(dd) < 1e-30f) dd = std::copysign(1e-30f, dd);
            inv[r] = 1.0f / dd;
        }
        ++t.slab_checked;
        if (!slab_hit(bmin, bmax, o, inv)) ++t.slab_drops;
    }
    ++t.cases;
    if (pre != 1) {
        ++t.decided;
        if (pre != exact) {
            if (t.violations < 5)
                std::printf("violation: pre %d exact %d O %.17g %.17g %.17g D %.17g %.17g %.17g\n",
                            pre, exact, O[0], O[1], O[2], D[0], D[1], D[2]);
            ++t.violations;
        }
    }
}

static void random_triangle(double *tri, double size)
{
    const double c[3] = {150.0 * sym(), 150.0 * sym(), 20.0 * sym()};
    for (int k = 0; k < 3; ++k)
        for (int r = 0; r < 3; ++r) tri[3 * k + r] = c[r] + size * sym();
}

static void random_dir(double *d, double len)
{
    double n = 0.0;
    do {
        for (int r = 0; r < 3; ++r) d[r] = sym();
        n = std::sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
    } while (n < 1e-3 || n > 1.0);
    for (int r = 0; r < 3; ++r) d[r] *= len / n;
}

int main()
{
    Tally t;
    double tri[9], O[3], D[3];
    // random segments around the triangle
    for (int i = 0; i < 400000; ++i) {
        const double s = logu(1e-3, 5.0);
        random_triangle(tri, s);
        random_dir(D, logu(0.05, 150.0));
        for (int r = 0; r < 3; ++r) O[r] = tri[r] + 3.0 * s * sym() - 0.5 * D[r];
        check(tri, O, D, t);
    }
    // through a point near an edge or a vertex, ends near the plane
    for (int i = 0; i < 1200000; ++i) {
        random_triangle(tri, logu(1e-3, 5.0));
        double e1[3], e2[3];
        for (int r = 0; r < 3; ++r) {
            e1[r] = tri[3 + r] - tri[r];
            e2[r] = tri[6 + r] - tri[r];
        }
        const double dlt = (next_u64() & 1 ? 1.0 : -1.0) * logu(1e-13, 1e-3);
        double u = uni(), v = uni() * (1.0 - u);
        switch (next_u64() % 5) {
        case 0: u = dlt; break;                              // edge u = 0
        case 1: v = dlt; break;                              // edge v = 0
        case 2: v = 1.0 - u - dlt; break;                    // edge u + v = 1
        case 3: u = dlt; v = (next_u64() & 1) ? dlt : 1.0 - dlt; break;   // near a vertex
        default: break;                                      // interior
        }
        double tp = uni();
        const int end = (int)(next_u64() % 3);
        if (end == 1) tp = dlt;                              // start on the plane
        if (end == 2) tp = 1.0 - dlt;                        // end on the plane
        if ((next_u64() % 4) == 0) {                         // nearly parallel to the plane
            double n[3] = {e1[1] * e2[2] - e1[2] * e2[1], e1[2] * e2[0] - e1[0] * e2[2],
                           e1[0] * e2[1] - e1[1] * e2[0]};
            const double nn = std::sqrt(n[0] * n[0] + n[1] * n[1] + n[2] * n[2]);
            const double len = logu(0.05, 150.0), tilt = logu(1e-9, 1e-2);
            for (int r = 0; r < 3; ++r) D[r] = len * (e1[r] / std::sqrt(e1[0] * e1[0] + e1[1] * e1[1] + e1[2] * e1[2]) + tilt * n[r] / nn);
        } else {
            random_dir(D, logu(0.05, 150.0));
        }
        for (int r = 0; r < 3; ++r) O[r] = tri[r] + u * e1[r] + v * e2[r] - tp * D[r];
        check(tri, O, D, t);
    }
    std::printf("cases %ld violations %ld decided %ld naive_wrong %ld slab_drops %ld of %ld\n",
                t.cases, t.violations, t.decided, t.naive_wrong, t.slab_drops, t.slab_checked);
    return t.violations == 0 && t.slab_drops == 0 ? 0 : 1;
}
