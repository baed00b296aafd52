/*
 * FP64 CPU oracle for the BART single-bounce scattering, coherent MIMO FMCW
 * echo synthesis and range-Doppler map of arXiv 2208.10939.
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the
 * cpu_baseline / reference legs of bench.py load this library.  It shares no
 * code with the CUDA path and is deliberately plain: no blocking, no caching
 * of per-facet quantities across samples, every term recomputed from the
 * frame-start geometry.
 *
 * Build: gcc -O2 -fopenmp -ffp-contract=off -fPIC -shared (no fast-math):
 * the visibility predicate must round exactly like IEEE-754 binary64 with
 * one rounding per operation.
 *
 * Definitions followed (paper sections / equations):
 *   - rigid vehicle motion, position at every chirp time (Sec. 3.2, Eq. 12)
 *   - BART single bounce: a scattering path exists where the forward ray
 *     from TX and the backward ray from RX meet on the same facet (Sec. 2.2)
 *     -> facet lit from TX AND seen from RX, decided at frame start
 *   - radar equation amplitude (Eq. 7), read as an amplitude sqrt(P)
 *   - physical-optics RCS of each lit facet over the swept frequency,
 *     sigma_f (Sec. 3.2); scalar PO with the flat-triangle integral
 *   - dechirped IF sample (Eq. 13) per facet with the exact bistatic
 *     round-trip delay (Eq. 12 with continuous t)
 * Readings of what the paper leaves silent or garbled are listed where used.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_C0 299792458.0
#define ORC_PI 3.14159265358979323846

enum { ORC_BACK = 0, ORC_LIT = 1, ORC_GRAZE = 2, ORC_OCCL = 3, ORC_LIT_REV = 4 };

int orc_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

void orc_set_threads(int n)
{
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}

/* ------------------------------------------------------------------ */
/* geometry                                                            */
/* ------------------------------------------------------------------ */

/* World vertices of every facet at time t (rigid instances):
 *   x = ((R00 lx + R01 ly) + R02 lz) + p ;  x = x + v t
 * lv: F x 9 local vertex triples; inst: F instance indices.
 * pos/vel: I x 3, rot: I x 9 (row-major).  out: F x 9. */
void orc_world_vertices(const double *lv, const int32_t *inst, int64_t F,
                        const double *pos, const double *rot, const double *vel,
                        double t, double *out)
{
    for (int64_t f = 0; f < F; ++f) {
        const int i = inst[f];
        for (int v = 0; v < 3; ++v) {
            const double x = lv[9 * f + 3 * v + 0];
            const double y = lv[9 * f + 3 * v + 1];
            const double z = lv[9 * f + 3 * v + 2];
            for (int r = 0; r < 3; ++r) {
                double w = rot[9 * i + 3 * r + 0] * x;
                w = w + rot[9 * i + 3 * r + 1] * y;
                w = w + rot[9 * i + 3 * r + 2] * z;
                w = w + pos[3 * i + r];
                w = w + vel[3 * i + r] * t;
                out[9 * f + 3 * v + r] = w;
            }
        }
    }
}

static void sub3(const double *a, const double *b, double *o)
{
    o[0] = a[0] - b[0];
    o[1] = a[1] - b[1];
    o[2] = a[2] - b[2];
}

static double dot3(const double *a, const double *b)
{
    double s = a[0] * b[0];
    s = s + a[1] * b[1];
    s = s + a[2] * b[2];
    return s;
}

static void cross3(const double *a, const double *b, double *o)
{
    o[0] = a[1] * b[2] - a[2] * b[1];
    o[1] = a[2] * b[0] - a[0] * b[2];
    o[2] = a[0] * b[1] - a[1] * b[0];
}

static void centroid3(const double *tri, double *c)
{
    for (int r = 0; r < 3; ++r) c[r] = ((tri[r] + tri[3 + r]) + tri[6 + r]) / 3.0;
}

/* ------------------------------------------------------------------ */
/* visibility (Sec. 2.2: bidirectional rays meet on a facet)           */
/* ------------------------------------------------------------------ */

/* Moller-Trumbore (1997) segment/triangle test.  Segment X(t) = O + t D,
 * t in [0,1].  Returns 2 = hit with margin, 1 = within the margins of an
 * edge / an end point (grazing), 0 = miss.  det == 0 (segment parallel to
 * the plane) is a miss. */
static int mt_segment(const double *O, const double *D, const double *tri,
                      double eps_b, double eps_t)
{
    double e1[3], e2[3], P[3], T[3], Qv[3];
    sub3(tri + 3, tri, e1);
    sub3(tri + 6, tri, e2);
    cross3(D, e2, P);
    const double det = dot3(e1, P);
    if (det == 0.0) return 0;
    const double inv = 1.0 / det;
    sub3(O, tri, T);
    const double u = dot3(T, P) * inv;
    if (u < -eps_b || u > 1.0 + eps_b) return 0;
    cross3(T, e1, Qv);
    const double v = dot3(D, Qv) * inv;
    if (v < -eps_b || u + v > 1.0 + eps_b) return 0;
    const double t = dot3(e2, Qv) * inv;
    if (t < -eps_t || t > 1.0 + eps_t) return 0;
    if (u >= eps_b && v >= eps_b && u + v <= 1.0 - eps_b &&
        t >= eps_t && t <= 1.0 - eps_t)
        return 2;
    return 1;
}

/* Conservative segment-vs-box rejection used only to skip work: a triangle
 * whose box (grown by `pad`) misses the segment's box cannot be hit or
 * grazed by it. */
static int boxes_disjoint(const double *O, const double *Pa, const double *tri,
                          double pad)
{
    for (int r = 0; r < 3; ++r) {
        double smin = O[r] < Pa[r] ? O[r] : Pa[r];
        double smax = O[r] < Pa[r] ? Pa[r] : O[r];
        double tmin = tri[r], tmax = tri[r];
        for (int v = 1; v < 3; ++v) {
            if (tri[3 * v + r] < tmin) tmin = tri[3 * v + r];
            if (tri[3 * v + r] > tmax) tmax = tri[3 * v + r];
        }
        if (tmax + pad < smin || tmin - pad > smax) return 1;
    }
    return 0;
}

/* Where the segment of facet k toward antenna a ends, and the segment
 * itself (D = end - c): the antenna, or (far field) the antenna moved by the
 * facet's offset from its instance origin ref, so that every facet of an
 * instance looks along the same plane-wave direction p_a - ref:
 *   end = p_a + (c - ref),  D = end - c. */
static void segment_to(const double *c, const double *pa, const double *ref, double *D)
{
    double end[3];
    for (int r = 0; r < 3; ++r) end[r] = ref ? pa[r] + (c[r] - ref[r]) : pa[r];
    sub3(end, c, D);
}

/* Facing part of the state of facet k (tri) seen along segment D from its
 * centroid:
 *   BACK     cos(angle between outward normal and D) <= -eps_face on a
 *            one-sided facet, or a zero-area facet (no normal, never lit)
 *   LIT      cos >= eps_face (candidate; occlusion decides)
 *   LIT_REV  a two-sided facet with cos <= -eps_face: lit on its reverse side
 *   *graze   |cos| < eps_face (the facet is then GRAZE unless occluded) */
static int facing_state(const double *tk, const double *D, int two_sided, double eps_face,
                        int *graze)
{
    double e1[3], e2[3], n[3];
    sub3(tk + 3, tk, e1);
    sub3(tk + 6, tk, e2);
    cross3(e1, e2, n);
    const double cosang = dot3(n, D) / (sqrt(dot3(n, n)) * sqrt(dot3(D, D)));
    *graze = 0;
    if (dot3(n, n) == 0.0) return ORC_BACK;
    if (cosang <= -eps_face) return two_sided ? ORC_LIT_REV : ORC_BACK;
    *graze = fabs(cosang) < eps_face;
    return ORC_LIT;
}

/* State of facet k seen from antenna a (BART single bounce, Sec. 2.2):
 *   BACK / LIT / LIT_REV : facing, as above, and no occluder
 *   GRAZE : |cos| < eps_face, or no robust hit but a grazing one
 *   OCCL  : the centroid->end segment robustly hits another facet
 * Brute force over every other facet.  state: A x F bytes.  fref: per-facet
 * instance origins (far-field segments) or NULL; two_sided: per-facet flags
 * or NULL (all one-sided). */
void orc_visibility(const double *tri, int64_t F, const double *ant, int A, const double *fref,
                    const uint8_t *two_sided, double eps_face, double eps_b, double eps_t,
                    uint8_t *state)
{
#pragma omp parallel for schedule(dynamic, 64) collapse(2)
    for (int a = 0; a < A; ++a) {
        for (int64_t k = 0; k < F; ++k) {
            const double *tk = tri + 9 * k;
            double c[3], D[3], end[3];
            centroid3(tk, c);
            segment_to(c, ant + 3 * a, fref ? fref + 3 * k : NULL, D);
            for (int r = 0; r < 3; ++r) end[r] = c[r] + D[r];
            int graze;
            const int face = facing_state(tk, D, two_sided && two_sided[k], eps_face, &graze);
            uint8_t st;
            if (face == ORC_BACK) {
                st = ORC_BACK;
            } else {
                int hit = 0;
                for (int64_t j = 0; j < F && !hit; ++j) {
                    if (j == k) continue;
                    if (boxes_disjoint(c, end, tri + 9 * j, 1e-6)) continue;
                    const int r = mt_segment(c, D, tri + 9 * j, eps_b, eps_t);
                    if (r == 2) hit = 1;
                    else if (r == 1) graze = 1;
                }
                st = hit ? ORC_OCCL : (graze ? ORC_GRAZE : (uint8_t)face);
            }
            state[(int64_t)a * F + k] = st;
        }
    }
}

/* ---- a plain top-down BVH for large scenes (median split on the longest
 * axis of the centroid box, leaves of <= 4 facets, FP64 boxes grown by 1e-6).
 * Box culling only skips work: the decision is the same segment test over
 * every facet whose grown box meets the segment's box, so the states equal
 * the brute-force ones. */
typedef struct {
    double lo[3], hi[3];
    int64_t left, right;     /* children, or -1 for a leaf */
    int64_t first, count;    /* leaf range in the index array */
} orc_node;

typedef struct {
    const double *tri;
    double *cen;
    int64_t *idx;
    orc_node *nodes;
    int64_t n_nodes;
    int axis;
} orc_bvh;

static const double *g_sort_cen;
static int g_sort_axis;
static int cmp_cen(const void *a, const void *b)
{
    const double x = g_sort_cen[3 * *(const int64_t *)a + g_sort_axis];
    const double y = g_sort_cen[3 * *(const int64_t *)b + g_sort_axis];
    if (x < y) return -1;
    if (x > y) return 1;
    return (*(const int64_t *)a < *(const int64_t *)b) ? -1 : 1;
}

static int64_t bvh_build(orc_bvh *b, int64_t first, int64_t count)
{
    const int64_t id = b->n_nodes++;
    orc_node *nd = &b->nodes[id];
    for (int r = 0; r < 3; ++r) {
        nd->lo[r] = 1e300;
        nd->hi[r] = -1e300;
    }
    double clo[3] = {1e300, 1e300, 1e300}, chi[3] = {-1e300, -1e300, -1e300};
    for (int64_t i = first; i < first + count; ++i) {
        const double *t = b->tri + 9 * b->idx[i];
        for (int v = 0; v < 3; ++v)
            for (int r = 0; r < 3; ++r) {
                if (t[3 * v + r] < nd->lo[r]) nd->lo[r] = t[3 * v + r];
                if (t[3 * v + r] > nd->hi[r]) nd->hi[r] = t[3 * v + r];
            }
        for (int r = 0; r < 3; ++r) {
            const double c = b->cen[3 * b->idx[i] + r];
            if (c < clo[r]) clo[r] = c;
            if (c > chi[r]) chi[r] = c;
        }
    }
    for (int r = 0; r < 3; ++r) {
        nd->lo[r] -= 1e-6;
        nd->hi[r] += 1e-6;
    }
    if (count <= 4) {
        nd->left = nd->right = -1;
        nd->first = first;
        nd->count = count;
        return id;
    }
    int axis = 0;
    for (int r = 1; r < 3; ++r)
        if (chi[r] - clo[r] > chi[axis] - clo[axis]) axis = r;
    g_sort_cen = b->cen;
    g_sort_axis = axis;
    qsort(b->idx + first, (size_t)count, sizeof(int64_t), cmp_cen);
    const int64_t half = count / 2;
    const int64_t l = bvh_build(b, first, half);
    const int64_t rr = bvh_build(b, first + half, count - half);
    b->nodes[id].left = l;
    b->nodes[id].right = rr;
    b->nodes[id].first = b->nodes[id].count = 0;
    return id;
}

/* segment box [min(O,Pa), max(O,Pa)] against a node box, then the slab
 * test of the segment in FP64; both conservative (boxes are grown). */
static int seg_meets_box(const double *O, const double *D, const orc_node *nd)
{
    double t0 = 0.0, t1 = 1.0;
    for (int r = 0; r < 3; ++r) {
        if (D[r] == 0.0) {
            if (O[r] < nd->lo[r] || O[r] > nd->hi[r]) return 0;
            continue;
        }
        double a = (nd->lo[r] - O[r]) / D[r], b = (nd->hi[r] - O[r]) / D[r];
        if (a > b) {
            const double tmp = a;
            a = b;
            b = tmp;
        }
        a -= 1e-7 * (fabs(a) + 1.0);      /* slack for the division's rounding */
        b += 1e-7 * (fabs(b) + 1.0);
        if (a > t0) t0 = a;
        if (b < t1) t1 = b;
        if (t0 > t1) return 0;
    }
    return 1;
}

/* Visibility states (A x F) using the BVH above; same definition as
 * orc_visibility. */
void orc_visibility_bvh(const double *tri, int64_t F, const double *ant, int A,
                        const double *fref, const uint8_t *two_sided, double eps_face,
                        double eps_b, double eps_t, uint8_t *state)
{
    orc_bvh b;
    b.tri = tri;
    b.cen = (double *)malloc(sizeof(double) * 3 * (size_t)F);
    b.idx = (int64_t *)malloc(sizeof(int64_t) * (size_t)F);
    b.nodes = (orc_node *)malloc(sizeof(orc_node) * (size_t)(2 * F + 1));
    b.n_nodes = 0;
    for (int64_t k = 0; k < F; ++k) {
        centroid3(tri + 9 * k, b.cen + 3 * k);
        b.idx[k] = k;
    }
    bvh_build(&b, 0, F);
#pragma omp parallel for schedule(dynamic, 256) collapse(2)
    for (int a = 0; a < A; ++a) {
        for (int64_t k = 0; k < F; ++k) {
            const double *tk = tri + 9 * k;
            double c[3], D[3];
            centroid3(tk, c);
            segment_to(c, ant + 3 * a, fref ? fref + 3 * k : NULL, D);
            int graze;
            const int face = facing_state(tk, D, two_sided && two_sided[k], eps_face, &graze);
            uint8_t st;
            if (face == ORC_BACK) {
                st = ORC_BACK;
            } else {
                int hit = 0;
                int64_t stack[128];
                int sp = 0;
                stack[sp++] = 0;
                while (sp > 0 && !hit) {
                    const orc_node *nd = &b.nodes[stack[--sp]];
                    if (!seg_meets_box(c, D, nd)) continue;
                    if (nd->left < 0) {
                        for (int64_t i = nd->first; i < nd->first + nd->count && !hit; ++i) {
                            const int64_t j = b.idx[i];
                            if (j == k) continue;
                            const int r = mt_segment(c, D, tri + 9 * j, eps_b, eps_t);
                            if (r == 2) hit = 1;
                            else if (r == 1) graze = 1;
                        }
                    } else {
                        stack[sp++] = nd->left;
                        stack[sp++] = nd->right;
                    }
                }
                st = hit ? ORC_OCCL : (graze ? ORC_GRAZE : (uint8_t)face);
            }
            state[(int64_t)a * F + k] = st;
        }
    }
    free(b.cen);
    free(b.idx);
    free(b.nodes);
}

/* The same states for selected (antenna, facet) pairs only (pairs: E x 2
 * int64 rows (a, k)), still by brute force over every other facet: used on
 * scenes too large for all pairs. */
void orc_visibility_pairs(const double *tri, int64_t F, const double *ant, const int64_t *pairs,
                          int64_t E, const double *fref, const uint8_t *two_sided,
                          double eps_face, double eps_b, double eps_t, uint8_t *state)
{
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t e = 0; e < E; ++e) {
        const int a = (int)pairs[2 * e];
        const int64_t k = pairs[2 * e + 1];
        const double *tk = tri + 9 * k;
        double c[3], D[3], end[3];
        centroid3(tk, c);
        segment_to(c, ant + 3 * a, fref ? fref + 3 * k : NULL, D);
        for (int r = 0; r < 3; ++r) end[r] = c[r] + D[r];
        int graze;
        const int face = facing_state(tk, D, two_sided && two_sided[k], eps_face, &graze);
        uint8_t st;
        if (face == ORC_BACK) {
            st = ORC_BACK;
        } else {
            int hit = 0;
            for (int64_t j = 0; j < F && !hit; ++j) {
                if (j == k) continue;
                if (boxes_disjoint(c, end, tri + 9 * j, 1e-6)) continue;
                const int r = mt_segment(c, D, tri + 9 * j, eps_b, eps_t);
                if (r == 2) hit = 1;
                else if (r == 1) graze = 1;
            }
            st = hit ? ORC_OCCL : (graze ? ORC_GRAZE : (uint8_t)face);
        }
        state[e] = st;
    }
}

/* ------------------------------------------------------------------ */
/* physical optics facet integral                                      */
/* ------------------------------------------------------------------ */

/* Complete homogeneous symmetric polynomial h_p(x0, x1, x2) = sum over
 * i + j + l = p of x0^i x1^j x2^l (p <= 16). */
static double hsym(int p, const double *x)
{
    double pw[3][17];
    for (int r = 0; r < 3; ++r) {
        pw[r][0] = 1.0;
        for (int e = 1; e <= p; ++e) pw[r][e] = pw[r][e - 1] * x[r];
    }
    double s = 0.0;
    for (int i = 0; i <= p; ++i)
        for (int j = 0; j <= p - i; ++j)
            s += pw[0][i] * pw[1][j] * pw[2][p - i - j];
    return s;
}

/* J(w) = integral over the flat triangle of exp(j w.(r - c)) dA, c the
 * centroid.  Gordon's edge form (divergence theorem in the facet plane):
 *   J = sum_i (-j) e_i.(n x w) / |w_t|^2 * exp(j w.(m_i - c)) * sinc(w.e_i/2)
 * with CCW edges e_i, midpoints m_i, unit normal n, w_t the in-plane part
 * of w.  The edge terms cancel to O(|w_t| d) of their size (d = longest
 * edge), losing ~(|w_t| d)^-2 in relative accuracy, so for |w_t| d < 0.5
 * the power series of the same integral is used instead:
 *   J = 2A sum_{p=0}^{14} j^p h_p(a_0, a_1, a_2) / (p+2)!,  a_i = w.(v_i - c)
 * (|a_i| < 0.5, truncation below 1e-16 relative). */
void orc_facet_integral(const double *tri, const double *w, double *re, double *im)
{
    double c[3], e1[3], e2[3], nn[3], nh[3];
    centroid3(tri, c);
    sub3(tri + 3, tri, e1);
    sub3(tri + 6, tri, e2);
    cross3(e1, e2, nn);
    const double nlen = sqrt(dot3(nn, nn));
    const double area = 0.5 * nlen;
    for (int r = 0; r < 3; ++r) nh[r] = nn[r] / nlen;
    const double wn = dot3(w, nh);
    double wt[3];
    for (int r = 0; r < 3; ++r) wt[r] = w[r] - wn * nh[r];
    const double wt2 = dot3(wt, wt);
    double diam = 0.0;
    for (int i = 0; i < 3; ++i) {
        double e[3];
        sub3(tri + 3 * ((i + 1) % 3), tri + 3 * i, e);
        const double l = sqrt(dot3(e, e));
        if (l > diam) diam = l;
    }
    if (sqrt(wt2) * diam < 0.5) {
        double a[3];
        for (int i = 0; i < 3; ++i) {
            double d[3];
            sub3(tri + 3 * i, c, d);
            a[i] = dot3(w, d);
        }
        double sr = 0.0, si = 0.0, fact = 2.0;        /* (p+2)! */
        for (int p = 0; p <= 14; ++p) {
            const double t = hsym(p, a) / fact;
            switch (p & 3) {                           /* j^p */
            case 0: sr += t; break;
            case 1: si += t; break;
            case 2: sr -= t; break;
            default: si -= t; break;
            }
            fact *= (double)(p + 3);
        }
        *re = 2.0 * area * sr;
        *im = 2.0 * area * si;
        return;
    }
    double nxw[3];
    cross3(nh, w, nxw);
    double sr = 0.0, si = 0.0;
    for (int i = 0; i < 3; ++i) {
        const double *va = tri + 3 * i, *vb = tri + 3 * ((i + 1) % 3);
        double e[3], m[3];
        sub3(vb, va, e);
        for (int r = 0; r < 3; ++r) m[r] = 0.5 * (va[r] + vb[r]) - c[r];
        const double coef = dot3(e, nxw) / wt2;         /* times (-j) */
        const double x = 0.5 * dot3(w, e);
        const double sinc = (x == 0.0) ? 1.0 : sin(x) / x;
        const double ph = dot3(w, m);
        const double cr = cos(ph) * sinc, ci = sin(ph) * sinc;
        /* (-j coef) (cr + j ci) = coef ci - j coef cr */
        sr += coef * ci;
        si -= coef * cr;
    }
    *re = sr;
    *im = si;
}

/* ------------------------------------------------------------------ */
/* far-field RCS of a mesh (plane-wave TX and RX directions)           */
/* ------------------------------------------------------------------ */

/* sigma(f) = |sum_k rho_k (k/sqrt(pi)) o_k J_k(-k(t+r)) exp(-j k (t+r).c_k)|^2
 * over facets whose outward normal faces both unit directions t (toward
 * the transmitter) and r (toward the receiver) -- or, for a two-sided facet
 * (two_sided[k], may be NULL), faces away from both (lit on its reverse);
 * o_k = |n_k.(t+r)|/2 is the scalar co-polarised obliquity (cos(theta)
 * monostatic).  Occlusion is not tested (convex or flat bodies only). */
void orc_rcs_farfield(const double *tri, int64_t F, const float *rho, const uint8_t *two_sided,
                      const double *that, const double *rhat,
                      const double *freqs, int nfreq, double *sigma)
{
#pragma omp parallel for schedule(static)
    for (int fi = 0; fi < nfreq; ++fi) {
        const double k = 2.0 * ORC_PI * freqs[fi] / ORC_C0;
        double b[3] = {that[0] + rhat[0], that[1] + rhat[1], that[2] + rhat[2]};
        double sr = 0.0, si = 0.0;
        for (int64_t f = 0; f < F; ++f) {
            const double *tk = tri + 9 * f;
            double c[3], e1[3], e2[3], nn[3];
            centroid3(tk, c);
            sub3(tk + 3, tk, e1);
            sub3(tk + 6, tk, e2);
            cross3(e1, e2, nn);
            const double nl = sqrt(dot3(nn, nn));
            const double ct = dot3(nn, that), cr = dot3(nn, rhat);
            const int front = ct > 0.0 && cr > 0.0;
            const int rev = two_sided && two_sided[f] && ct < 0.0 && cr < 0.0;
            if (!front && !rev) continue;
            const double o = fabs(0.5 * dot3(nn, b) / nl);
            double w[3] = {-k * b[0], -k * b[1], -k * b[2]};
            double jr, ji;
            orc_facet_integral(tk, w, &jr, &ji);
            const double ph = -k * dot3(b, c);
            const double pr = cos(ph), pi_ = sin(ph);
            const double s = (double)rho[f] * (k / sqrt(ORC_PI)) * o;
            sr += s * (jr * pr - ji * pi_);
            si += s * (jr * pi_ + ji * pr);
        }
        sigma[fi] = sr * sr + si * si;
    }
}

/* ------------------------------------------------------------------ */
/* echo synthesis (Sec. 3.2, Eqs. 7, 9-13)                             */
/* ------------------------------------------------------------------ */

typedef struct {
    double f0, slope, fs, Tc;   /* start frequency, mu, sampling rate, chirp period */
    int M, N, P, Q;
    int intra_chirp_motion;     /* tau evaluated at t_n + t_m (1) or t_n (0) */
    int tdm;                    /* 1: TX p transmits chirp n at (n P + p) T_c */
    int delay_ref;              /* 1: reference-point delay form (Eqs. 11-13 per target) */
    int far_field;              /* 1: plane-wave directions and path from the instance origin */
} orc_radar;

/* One IF sample of channel o = p*Q + q, chirp n, sample m:
 *
 *   x[o][n][m] = sum over facets k lit from TX p AND from RX q of
 *       lambda_m / ((4 pi)^{3/2} R_t R_r)                (Eq. 7 as amplitude)
 *     * rho_k (k_m / sqrt(pi)) o_k J_k(-k_m (t + r))     (PO sigma_f, signed)
 *     * exp{ j 2 pi [ f0 tau + mu t_m tau - mu tau^2 / 2 ] }   (Eq. 13)
 *
 * with f_m = f0 + mu t_m, t_m = m / fs, k_m = 2 pi f_m / c, lambda_m = c / f_m;
 * geometry at the chirp start t_n = n T_c (relative to the frame start):
 * facet vertices translated by v t_n, unit vectors t, r from the facet
 * centroid toward TX / RX, distances R_t, R_r, obliquity
 * o_k = n_k . (t + r) / 2;  tau = (|c(t) - p_tx| + |c(t) - p_rx|) / c at
 * t = t_n + t_m (Eq. 12 with the exact bistatic path of the centroid).
 * The IFFT route of Eqs. 9-11: with stretch processing, sample m sees the
 * instantaneous frequency f_m, so sigma_f at f_m times the dechirp phase is
 * the time-domain product; no separate transform is applied.
 *
 * Time-division MIMO (tdm): the chirp of TX p with index n starts at
 * (n P + p) T_c instead of n T_c; everything else is unchanged.
 *
 * Reference-point form (delay_ref), Eqs. 11-13 taken per target: the
 * target's reference point r_i (its instance origin, fref per facet) moves
 * with the target; with L_k and L_r the TX + RX path lengths of the facet
 * centroid and of the reference point at the chirp start, and L_r(t) that of
 * the reference point at t_n + t_m, the phase is
 *   2 pi [ f_m (L_k - L_r + L_r(t)) / c - mu (L_r(t) / c)^2 / 2 ]
 * i.e. the facet enters through the frequency response relative to the
 * reference point at the chirp's aspect (sigma_f), the delay of Eq. 12, its
 * motion within the chirp and the residual video phase belong to the
 * reference point.
 *
 * Far field (far_field): every facet of an instance is seen along the plane
 * waves of its instance origin r_i, at the origin's ranges: with r0 the
 * origin at the chirp start, t = (p_tx - r0)/R_t, r = (p_rx - r0)/R_r,
 * R_t = |p_tx - r0|, R_r = |p_rx - r0| (amplitude, obliquity and the facet
 * integral use these), and the facet's path is the plane-wave one,
 *   L_k(t) = |p_tx - r(t)| + |p_rx - r(t)| - (t + r).(c_k - r0),
 * the origin moving within the chirp (t = t_n + t_m) and the projection held
 * at the chirp start; tau = L_k / c enters Eq. 13 as above.  A flat plate
 * centred on its origin then gives exactly the radar equation with the
 * far-field PO cross-section 4 pi A^2 / lambda^2 at normal incidence.
 *
 * Two-sided facets (two_sided[k]): the channel sees the facet when both its
 * antennas light the same side (LIT from both, or LIT_REV from both); the
 * obliquity is |n_k . (t + r)| / 2, the normal turned toward the antennas. */
static double path_len(const double *x, const double *ptx, const double *prx)
{
    double ut[3], ur[3];
    sub3(x, ptx, ut);
    sub3(x, prx, ur);
    return sqrt(dot3(ut, ut)) + sqrt(dot3(ur, ur));
}

static void adc_sample(const double *tri0, const double *fvel, const float *rho,
                       const double *fref, const uint8_t *two_sided, const uint8_t *state,
                       int64_t F, const double *tx, const double *rx, const orc_radar *rd, int o,
                       int n, int m, double *out_re, double *out_im)
{
    const int p = o / rd->Q, q = o % rd->Q;
    const double tn = (double)(rd->tdm ? (int64_t)n * rd->P + p : n) * rd->Tc;
    const double tm = (double)m / rd->fs;
    const double fm = rd->f0 + rd->slope * tm;
    const double km = 2.0 * ORC_PI * fm / ORC_C0;
    const double lam = ORC_C0 / fm;
    const double ptx[3] = {tx[3 * p], tx[3 * p + 1], tx[3 * p + 2]};
    const double prx[3] = {rx[3 * q], rx[3 * q + 1], rx[3 * q + 2]};
    const uint8_t *st_t = state + (int64_t)p * F;
    const uint8_t *st_r = state + (int64_t)(rd->P + q) * F;
    const double amp0 = 1.0 / pow(4.0 * ORC_PI, 1.5);
    double sr = 0.0, si = 0.0;
    for (int64_t k = 0; k < F; ++k) {
        const int lit = (st_t[k] == ORC_LIT && st_r[k] == ORC_LIT) ||
                        (st_t[k] == ORC_LIT_REV && st_r[k] == ORC_LIT_REV);
        if (!lit) continue;
        const double *vk = fvel + 3 * k;
        double tri[9];
        for (int i = 0; i < 9; ++i) tri[i] = tri0[9 * k + i] + vk[i % 3] * tn;
        double c[3], e1[3], e2[3], nn[3], dt[3], dr[3], r0[3];
        centroid3(tri, c);
        sub3(tri + 3, tri, e1);
        sub3(tri + 6, tri, e2);
        cross3(e1, e2, nn);
        const double nl = sqrt(dot3(nn, nn));
        if (rd->far_field || rd->delay_ref)
            for (int r = 0; r < 3; ++r) r0[r] = fref[3 * k + r] + vk[r] * tn;
        /* directions and ranges: from the centroid, or (far field) the origin */
        const double *from = rd->far_field ? r0 : c;
        sub3(ptx, from, dt);
        sub3(prx, from, dr);
        const double Rt = sqrt(dot3(dt, dt)), Rr = sqrt(dot3(dr, dr));
        double b[3];
        for (int r = 0; r < 3; ++r) b[r] = dt[r] / Rt + dr[r] / Rr;
        double ok = 0.5 * dot3(nn, b) / nl;
        if (two_sided && two_sided[k]) ok = fabs(ok);
        double w[3] = {-km * b[0], -km * b[1], -km * b[2]};
        double jr, ji;
        orc_facet_integral(tri, w, &jr, &ji);
        const double s = (double)rho[k] * (km / sqrt(ORC_PI)) * ok;
        const double a = lam * amp0 / (Rt * Rr) * s;
        /* round-trip delay at t_n + t_m */
        double phase;
        if (rd->far_field) {
            double rt[3], off[3];
            for (int r = 0; r < 3; ++r) rt[r] = rd->intra_chirp_motion ? r0[r] + vk[r] * tm : r0[r];
            sub3(c, r0, off);
            const double tau = (path_len(rt, ptx, prx) - dot3(b, off)) / ORC_C0;
            phase = 2.0 * ORC_PI *
                (rd->f0 * tau + rd->slope * tm * tau - 0.5 * rd->slope * tau * tau);
        } else if (!rd->delay_ref) {
            double ct[3] = {c[0], c[1], c[2]};
            if (rd->intra_chirp_motion)
                for (int r = 0; r < 3; ++r) ct[r] = c[r] + vk[r] * tm;
            const double tau = path_len(ct, ptx, prx) / ORC_C0;
            phase = 2.0 * ORC_PI *
                (rd->f0 * tau + rd->slope * tm * tau - 0.5 * rd->slope * tau * tau);
        } else {
            double rt[3];
            for (int r = 0; r < 3; ++r) rt[r] = rd->intra_chirp_motion ? r0[r] + vk[r] * tm : r0[r];
            const double Lk = path_len(c, ptx, prx), Lr0 = path_len(r0, ptx, prx);
            const double Lrt = path_len(rt, ptx, prx);
            const double tau_f = (Lk - Lr0 + Lrt) / ORC_C0, tau_r = Lrt / ORC_C0;
            phase = 2.0 * ORC_PI * (fm * tau_f - 0.5 * rd->slope * tau_r * tau_r);
        }
        const double cr = cos(phase), ci = sin(phase);
        sr += a * (jr * cr - ji * ci);
        si += a * (jr * ci + ji * cr);
    }
    *out_re = sr;
    *out_im = si;
}

/* Full ADC cube [O][N][M] (complex128, interleaved). */
void orc_adc_full(const double *tri0, const double *fvel, const float *rho,
                  const double *fref, const uint8_t *two_sided, const uint8_t *state, int64_t F,
                  const double *tx, const double *rx, const orc_radar *rd, double *out)
{
    const int O = rd->P * rd->Q;
#pragma omp parallel for schedule(dynamic, 1) collapse(2)
    for (int o = 0; o < O; ++o)
        for (int n = 0; n < rd->N; ++n)
            for (int m = 0; m < rd->M; ++m) {
                const int64_t idx = ((int64_t)o * rd->N + n) * rd->M + m;
                adc_sample(tri0, fvel, rho, fref, two_sided, state, F, tx, rx, rd, o, n, m,
                           out + 2 * idx, out + 2 * idx + 1);
            }
}

/* Selected entries (o, n, m) of the ADC cube; entries: E x 3 int32. */
void orc_adc_entries(const double *tri0, const double *fvel, const float *rho,
                     const double *fref, const uint8_t *two_sided, const uint8_t *state,
                     int64_t F, const double *tx, const double *rx, const orc_radar *rd,
                     const int32_t *entries, int64_t E, double *out)
{
#pragma omp parallel for schedule(dynamic, 4)
    for (int64_t e = 0; e < E; ++e)
        adc_sample(tri0, fvel, rho, fref, two_sided, state, F, tx, rx, rd, entries[3 * e],
                   entries[3 * e + 1], entries[3 * e + 2], out + 2 * e, out + 2 * e + 1);
}

/* ------------------------------------------------------------------ */
/* double bounce (Sec. 2.2: forward and backward rays connected       */
/* through two facets)                                                 */
/* ------------------------------------------------------------------ */
/*
 * The paper names multi-bounce paths (a forward ray from TX and a backward
 * ray from RX joined on a facet after further reflections) but prints no
 * formula for them.  Reading used here for two facets, geometric optics at
 * the first and physical optics at the second:
 *
 *  - the forward ray from TX p reaches facet a (a lit from TX p, its
 *    single-bounce state LIT or LIT_REV: side s_a = +1 / -1) and reflects
 *    specularly: beyond a, the reflected field is that of the image source
 *    p' = p - 2 ((p - x0_a).n_a / |n_a|^2) n_a (mirror of p in a's plane),
 *    confined to the beam of rays from p' through the triangle a;
 *  - the part of facet b inside that beam, Pi_ab = b clipped by a's front
 *    half-space (s_a n_a.(x - x0_a) >= 0) and the three planes through p'
 *    and a's edges (each keeping a's third vertex), is lit by the image
 *    source; b must face p' (cos >= eps_face, or <= -eps_face on a
 *    two-sided b: side s_b = -1);
 *  - the a -> b leg is the segment from the specular point s (where the
 *    line p' -> c_Pi meets a's plane, c_Pi the mean of Pi's vertices) to
 *    c_Pi; the pair is dropped when that segment hits, or grazes, any facet
 *    other than a and b (the Moller-Trumbore test and margins of the
 *    single-bounce visibility);
 *  - the backward ray from RX q meets b: b's single-bounce state from RX q
 *    is LIT for s_b = +1, LIT_REV for s_b = -1;
 *  - Pi_ab is split into the fan (Pi_0, Pi_i, Pi_i+1); sub-triangles whose
 *    |cross| is at most 1e-6 |n_b| (clip slivers) are dropped; each kept
 *    one is a virtual facet that scatters like a single-bounce facet of the
 *    echo synthesis below, with the transmitter replaced by p' and the
 *    reflectivity by -rho_a rho_b (-1: the reflection coefficient of a
 *    perfectly conducting plane for the scalar, co-polarised field; rho_b
 *    is the PO facet's own, as in the single bounce);
 *  - pairs, clips and visibility are decided on the frame-start geometry,
 *    like the single-bounce states; afterwards a virtual facet moves with b
 *    and p' with a's plane: p'(t) = p'_0 + u t, u = 2 (v_a.n_a / |n_a|^2) n_a.
 *
 * All decisions use one IEEE rounding per operation in the order written
 * (the library built with -ffp-contract=off), so they are reproducible.
 */
#define ORC_DB_MAXV 7
#define ORC_DB_SLIVER 1e-6

/* Sutherland-Hodgman step: the part of the convex polygon (n vertices) with
 * g.(x - base) >= 0.  Returns the new vertex count. */
static int clip_keep(const double *in, int n, const double *g, const double *base, double *out)
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
            const double t = fP / (fP - fQ);
            for (int r = 0; r < 3; ++r) out[3 * k + r] = P[r] + t * (Q[r] - P[r]);
            ++k;
        }
    }
    return k;
}

/* The beam of facet a for a source at p' (point source, dir == NULL) or for
 * plane waves toward the image direction dir (the far-field form): four
 * half-spaces (g, base). */
static void beam_planes(const double *ta, int side_a, const double *src, const double *dir,
                        double *g, double *base)
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
        double m[3], d[3];
        if (dir) {
            double e[3];
            sub3(xj, xi, e);
            cross3(e, dir, m);
            sub3(xk, xi, d);
            for (int r = 0; r < 3; ++r) base[3 * (i + 1) + r] = xi[r];
        } else {
            double u[3], v[3];
            sub3(xi, src, u);
            sub3(xj, src, v);
            cross3(u, v, m);
            sub3(xk, src, d);
            for (int r = 0; r < 3; ++r) base[3 * (i + 1) + r] = src[r];
        }
        const double s = dot3(m, d) < 0.0 ? -1.0 : 1.0;
        for (int r = 0; r < 3; ++r) g[3 * (i + 1) + r] = s * m[r];
    }
}

/* Pi = triangle tb clipped by the four half-spaces; returns its vertex count */
static int beam_clip(const double *tb, const double *g, const double *base, double *poly)
{
    double buf[3 * ORC_DB_MAXV];
    int n = 3;
    for (int i = 0; i < 9; ++i) poly[i] = tb[i];
    for (int h = 0; h < 4 && n >= 3; ++h) {
        n = clip_keep(poly, n, g + 3 * h, base + 3 * h, buf);
        for (int i = 0; i < 3 * n; ++i) poly[i] = buf[i];
    }
    return n;
}

/* Virtual facets of the double-bounce paths of transmitters 0..P-1 (the
 * reading above), in the order (p, a, b, fan index).  tri: F x 9 frame-start
 * world vertices; fvel: F x 3 velocities; rho: F reflectivities; two_sided:
 * F flags or NULL; ant: antennas (TX first); state: single-bounce states
 * (TX rows 0..P-1 used).  Writes up to cap facets: pab (4 int32 each: p, a,
 * b, s_b), vtri (9), src (p'_0, 3), usrc (u, 3), w (-rho_a rho_b); returns
 * the total count (call again with a larger cap when it exceeds cap). */
int64_t orc_bounce2_facets(const double *tri, const double *fvel, const float *rho,
                           const uint8_t *two_sided, int64_t F, const double *ant, int P,
                           const uint8_t *state, double eps_face, double eps_b, double eps_t,
                           int64_t cap, int32_t *pab, double *vtri, double *src, double *usrc,
                           double *w)
{
    int64_t count = 0;
    for (int p = 0; p < P; ++p) {
        const double *pt = ant + 3 * p;
        for (int64_t a = 0; a < F; ++a) {
            const uint8_t st = state[(int64_t)p * F + a];
            if (st != ORC_LIT && st != ORC_LIT_REV) continue;
            const double *ta = tri + 9 * a;
            double e1[3], e2[3], na[3], d[3], img[3], u[3];
            sub3(ta + 3, ta, e1);
            sub3(ta + 6, ta, e2);
            cross3(e1, e2, na);
            const double nn = dot3(na, na);
            sub3(pt, ta, d);
            const double sc = (2.0 * dot3(d, na)) / nn;
            for (int r = 0; r < 3; ++r) img[r] = pt[r] - sc * na[r];
            const double su = (2.0 * dot3(fvel + 3 * a, na)) / nn;
            for (int r = 0; r < 3; ++r) u[r] = su * na[r];
            double g[12], base[12];
            beam_planes(ta, st == ORC_LIT ? 1 : -1, img, NULL, g, base);
            for (int64_t b = 0; b < F; ++b) {
                if (b == a) continue;
                const double *tb = tri + 9 * b;
                double f1[3], f2[3], nb[3], cb[3], D[3];
                sub3(tb + 3, tb, f1);
                sub3(tb + 6, tb, f2);
                cross3(f1, f2, nb);
                const double nbb = dot3(nb, nb);
                if (nbb == 0.0) continue;
                centroid3(tb, cb);
                sub3(img, cb, D);
                const double cosang = dot3(nb, D) / (sqrt(nbb) * sqrt(dot3(D, D)));
                int side_b;
                if (cosang >= eps_face) side_b = 1;
                else if (two_sided && two_sided[b] && cosang <= -eps_face) side_b = -1;
                else continue;
                double poly[3 * ORC_DB_MAXV];
                const int K = beam_clip(tb, g, base, poly);
                if (K < 3) continue;
                const double thr = ORC_DB_SLIVER * sqrt(nbb);
                int keep[ORC_DB_MAXV];
                int nkeep = 0;
                for (int i = 1; i + 1 < K; ++i) {
                    double x1[3], x2[3], cr[3];
                    sub3(poly + 3 * i, poly, x1);
                    sub3(poly + 3 * (i + 1), poly, x2);
                    cross3(x1, x2, cr);
                    keep[i] = sqrt(dot3(cr, cr)) > thr;
                    nkeep += keep[i];
                }
                if (nkeep == 0) continue;
                /* the a -> b leg: specular point s on a's plane -> c_Pi */
                double cp[3] = {0.0, 0.0, 0.0}, sp[3], Dl[3], t1[3], t2[3];
                for (int i = 0; i < K; ++i)
                    for (int r = 0; r < 3; ++r) cp[r] = cp[r] + poly[3 * i + r];
                for (int r = 0; r < 3; ++r) cp[r] = cp[r] / (double)K;
                sub3(ta, img, t1);
                sub3(cp, img, t2);
                const double lam = dot3(na, t1) / dot3(na, t2);
                for (int r = 0; r < 3; ++r) sp[r] = img[r] + lam * t2[r];
                sub3(cp, sp, Dl);
                int blocked = 0;
                for (int64_t j = 0; j < F && !blocked; ++j) {
                    if (j == a || j == b) continue;
                    if (boxes_disjoint(sp, cp, tri + 9 * j, 1e-6)) continue;
                    if (mt_segment(sp, Dl, tri + 9 * j, eps_b, eps_t) != 0) blocked = 1;
                }
                if (blocked) continue;
                for (int i = 1; i + 1 < K; ++i) {
                    if (!keep[i]) continue;
                    if (count < cap) {
                        int32_t *q = pab + 4 * count;
                        q[0] = p;
                        q[1] = (int32_t)a;
                        q[2] = (int32_t)b;
                        q[3] = side_b;
                        double *vt = vtri + 9 * count;
                        for (int r = 0; r < 3; ++r) {
                            vt[r] = poly[r];
                            vt[3 + r] = poly[3 * i + r];
                            vt[6 + r] = poly[3 * (i + 1) + r];
                            src[3 * count + r] = img[r];
                            usrc[3 * count + r] = u[r];
                        }
                        w[count] = -((double)rho[a] * (double)rho[b]);
                    }
                    ++count;
                }
            }
        }
    }
    return count;
}

/* Far-field double-bounce PO cross-section (plane waves, the reading above
 * with the image source at infinity): for unit directions t (toward TX) and
 * r (toward RX), every ordered pair (a, b), a != b, with a facing t (side
 * s_a: n_a.t > 0, or < 0 on a two-sided a), t' = t - 2 (t.n_a) n_a / |n_a|^2
 * the direction toward the image source, b facing t' and r on one side
 * (both cosines > 0, or both < 0 on a two-sided b), Pi_ab = b clipped by
 * a's front half-space and the prism of a along t'; each fan sub-triangle T
 * of Pi_ab adds
 *   -rho_a rho_b (k / sqrt(pi)) o_b J_T(-k (t' + r)) exp(j k L(c_T)),
 *   o_b = |n_b.(t' + r)| / 2 (n_b unit),
 *   L(x) = -(t' + r).x - 2 (t.n_a)(n_a.x0_a) / |n_a|^2,
 * the path of the reflected plane wave relative to the origin (the image
 * wave matches the incident one on a's plane).  sigma = |sum|^2.  No
 * occlusion test (open, convex configurations such as a dihedral). */
void orc_rcs_farfield_bounce2(const double *tri, int64_t F, const float *rho,
                              const uint8_t *two_sided, const double *that, const double *rhat,
                              const double *freqs, int nfreq, double *sigma)
{
    for (int fi = 0; fi < nfreq; ++fi) {
        const double k = 2.0 * ORC_PI * freqs[fi] / ORC_C0;
        double sr = 0.0, si = 0.0;
        for (int64_t a = 0; a < F; ++a) {
            const double *ta = tri + 9 * a;
            double e1[3], e2[3], na[3], tp[3];
            sub3(ta + 3, ta, e1);
            sub3(ta + 6, ta, e2);
            cross3(e1, e2, na);
            const double nn = dot3(na, na);
            if (nn == 0.0) continue;
            const double ct = dot3(na, that);
            int side_a;
            if (ct > 0.0) side_a = 1;
            else if (two_sided && two_sided[a] && ct < 0.0) side_a = -1;
            else continue;
            for (int r = 0; r < 3; ++r) tp[r] = that[r] - (2.0 * ct / nn) * na[r];
            const double shift = -2.0 * ct * dot3(na, ta) / nn;
            double g[12], base[12];
            beam_planes(ta, side_a, NULL, tp, g, base);
            double bv[3] = {tp[0] + rhat[0], tp[1] + rhat[1], tp[2] + rhat[2]};
            for (int64_t b = 0; b < F; ++b) {
                if (b == a) continue;
                const double *tb = tri + 9 * b;
                double f1[3], f2[3], nb[3];
                sub3(tb + 3, tb, f1);
                sub3(tb + 6, tb, f2);
                cross3(f1, f2, nb);
                const double nbl = sqrt(dot3(nb, nb));
                if (nbl == 0.0) continue;
                const double c1 = dot3(nb, tp), c2 = dot3(nb, rhat);
                const int front = c1 > 0.0 && c2 > 0.0;
                const int rev = two_sided && two_sided[b] && c1 < 0.0 && c2 < 0.0;
                if (!front && !rev) continue;
                double poly[3 * ORC_DB_MAXV];
                const int K = beam_clip(tb, g, base, poly);
                const double o = fabs(0.5 * dot3(nb, bv) / nbl);
                const double s = -((double)rho[a] * (double)rho[b]) * (k / sqrt(ORC_PI)) * o;
                for (int i = 1; i + 1 < K; ++i) {
                    double sub[9], cT[3], x1[3], x2[3], cr[3];
                    for (int r = 0; r < 3; ++r) {
                        sub[r] = poly[r];
                        sub[3 + r] = poly[3 * i + r];
                        sub[6 + r] = poly[3 * (i + 1) + r];
                    }
                    sub3(sub + 3, sub, x1);
                    sub3(sub + 6, sub, x2);
                    cross3(x1, x2, cr);
                    if (sqrt(dot3(cr, cr)) <= ORC_DB_SLIVER * nbl) continue;
                    centroid3(sub, cT);
                    double wv[3] = {-k * bv[0], -k * bv[1], -k * bv[2]};
                    double jr, ji;
                    orc_facet_integral(sub, wv, &jr, &ji);
                    const double ph = k * (-dot3(bv, cT) + shift);
                    const double pr = cos(ph), pi_ = sin(ph);
                    sr += s * (jr * pr - ji * pi_);
                    si += s * (jr * pi_ + ji * pr);
                }
            }
        }
        sigma[fi] = sr * sr + si * si;
    }
}

/* Double-bounce part of selected ADC entries (o, n, m): every virtual facet
 * v of TX p = o / Q (orc_bounce2_facets) whose facet b is seen from RX
 * q = o % Q on side s_b scatters as a single-bounce facet of adc_sample
 * (facet delay form) with
 *   vertices vtri_v + v_b t_n, transmitter p'(t_n) = src_v + usrc_v t_n,
 *   reflectivity w_v, obliquity n_v.(t' + r) / 2 (|.| on a two-sided b),
 *   delay at t_n + t_m: (|c(t) - p'(t)| + |c(t) - p_rx|) / c,
 *   c(t) = c_v(t_n) + v_b t_m, p'(t) = p'(t_n) + usrc_v t_m
 * (the motion within the chirp when intra_chirp_motion is set). */
void orc_adc_bounce2_entries(const int32_t *pab, const double *vtri, const double *src,
                             const double *usrc, const double *w, int64_t V,
                             const double *fvel, const uint8_t *two_sided, const uint8_t *state,
                             int64_t F, const double *tx, const double *rx, const orc_radar *rd,
                             const int32_t *entries, int64_t E, double *out)
{
    (void)tx;
#pragma omp parallel for schedule(dynamic, 4)
    for (int64_t e = 0; e < E; ++e) {
        const int o = entries[3 * e], n = entries[3 * e + 1], m = entries[3 * e + 2];
        const int p = o / rd->Q, q = o % rd->Q;
        const double tn = (double)(rd->tdm ? (int64_t)n * rd->P + p : n) * rd->Tc;
        const double tm = (double)m / rd->fs;
        const double fm = rd->f0 + rd->slope * tm;
        const double km = 2.0 * ORC_PI * fm / ORC_C0;
        const double lam = ORC_C0 / fm;
        const double prx[3] = {rx[3 * q], rx[3 * q + 1], rx[3 * q + 2]};
        const uint8_t *st_r = state + (int64_t)(rd->P + q) * F;
        const double amp0 = 1.0 / pow(4.0 * ORC_PI, 1.5);
        double sr = 0.0, si = 0.0;
        for (int64_t v = 0; v < V; ++v) {
            const int32_t *g = pab + 4 * v;
            if (g[0] != p) continue;
            const int64_t b = g[2];
            if (st_r[b] != (g[3] > 0 ? ORC_LIT : ORC_LIT_REV)) continue;
            const double *vb = fvel + 3 * b;
            double tri[9], ptx[3];
            for (int i = 0; i < 9; ++i) tri[i] = vtri[9 * v + i] + vb[i % 3] * tn;
            for (int r = 0; r < 3; ++r) ptx[r] = src[3 * v + r] + usrc[3 * v + r] * tn;
            double c[3], e1[3], e2[3], nn[3], dt[3], dr[3];
            centroid3(tri, c);
            sub3(tri + 3, tri, e1);
            sub3(tri + 6, tri, e2);
            cross3(e1, e2, nn);
            const double nl = sqrt(dot3(nn, nn));
            sub3(ptx, c, dt);
            sub3(prx, c, dr);
            const double Rt = sqrt(dot3(dt, dt)), Rr = sqrt(dot3(dr, dr));
            double bb[3];
            for (int r = 0; r < 3; ++r) bb[r] = dt[r] / Rt + dr[r] / Rr;
            double ok = 0.5 * dot3(nn, bb) / nl;
            if (two_sided && two_sided[b]) ok = fabs(ok);
            double wv[3] = {-km * bb[0], -km * bb[1], -km * bb[2]};
            double jr, ji;
            orc_facet_integral(tri, wv, &jr, &ji);
            const double s = w[v] * (km / sqrt(ORC_PI)) * ok;
            const double amp = lam * amp0 / (Rt * Rr) * s;
            double ct[3] = {c[0], c[1], c[2]}, pt[3] = {ptx[0], ptx[1], ptx[2]};
            if (rd->intra_chirp_motion)
                for (int r = 0; r < 3; ++r) {
                    ct[r] = c[r] + vb[r] * tm;
                    pt[r] = ptx[r] + usrc[3 * v + r] * tm;
                }
            const double tau = path_len(ct, pt, prx) / ORC_C0;
            const double phase = 2.0 * ORC_PI *
                (rd->f0 * tau + rd->slope * tm * tau - 0.5 * rd->slope * tau * tau);
            const double cr = cos(phase), ci = sin(phase);
            sr += amp * (jr * cr - ji * ci);
            si += amp * (jr * ci + ji * cr);
        }
        out[2 * e] = sr;
        out[2 * e + 1] = si;
    }
}
