// Internal declarations shared by the CUDA translation units of libbartsim.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "bartsim.h"

namespace bart {

constexpr double kC0 = 299792458.0;
constexpr double kPi = 3.14159265358979323846;
constexpr int kMaxAnt = BART_MAX_TX + BART_MAX_RX;

// Visibility margins (BART single bounce, Sec. 2.2).  A facet whose normal
// makes |cos| < eps_face with its antenna (kEpsFace unless the radar sets
// grazing_eps), or whose centroid->antenna segment passes within the
// barycentric / parameter margins of another facet without a clear hit, is
// "grazing": excluded and counted.
constexpr double kEpsFace = 1e-6;
constexpr double kEpsB = 1e-9;
constexpr double kEpsT = 1e-9;

// Record classes of the facet integral (see synth.cu).
constexpr int kRecVertex = 0;
constexpr int kRecSeries = 1;
constexpr int kRecEdge = 2;
constexpr double kSeriesKD = 1.0;     // k_max * (u_max - u_min) below this: series
constexpr double kEdgeKd = 0.03;      // k_max * min pair gap below this: edge form
constexpr double kSincSeries = 0.25;  // |k gamma| below this: sinc by its series
constexpr int kSeriesTerms = 15;      // p = 0..14

// Radar constants passed by value to kernels.
struct RadarDev {
    double f0, slope, fs, Tc;
    int M, N, P, Q, O, A;
    int intra;
    int window;
    int tdm;        // time-division MIMO: chirp n of TX p at (n P + p) Tc
    int delay_ref;  // reference-point delay form
    int slots;      // chirp slots per chirp index: P with tdm, else 1
    int far_field;  // plane waves from each instance origin (see bartsim.h)
    double eps_face;  // grazing threshold of |cos| toward an antenna
    double ant[kMaxAnt][3];   // TX 0..P-1, then RX P..P+Q-1
};

// Frame-start facet record in FP32 (80 B, 16-B aligned).
struct __align__(16) FacetRec {
    float c[3];     // centroid
    float area;
    float dv[9];    // vertex offsets from the centroid
    float rho;      // reflectivity
    float n[3];     // unit outward normal
    int inst;       // instance index
    int two_sided;  // 1: lit from either side (BART_MESH_TWO_SIDED)
    float pad;
};
static_assert(sizeof(FacetRec) == 80, "FacetRec layout");

// LBVH node with both child boxes stored in the parent (64 B).  A child
// index >= 0 is an internal node, < 0 is ~facet_id.
struct __align__(16) BvhNode {
    float lmin[3];
    int left;
    float lmax[3];
    int right;
    float rmin[3];
    int pad0;
    float rmax[3];
    int pad1;
};
static_assert(sizeof(BvhNode) == 64, "BvhNode layout");

struct MeshDesc {
    const double *verts;
    const int32_t *tris;
    const float *rho;
    int64_t nf;
    int two_sided;
};

struct InstDev {
    int32_t mesh;
    float rho_scale;
    int64_t off;          // first global facet of this instance
    double pos[3];
    double rot[9];
    double vel[3];
};

// Device status word bits (latched, read by bart_sync).
constexpr int kStatusStackOverflow = 1;
constexpr int kStatusWaitTimeout = 2;   // a bounded device wait expired (see bart_sync)

// ---- scene + BVH (scene_bvh.cu) ----
// tri32: per facet 12 floats -- the world vertices rounded to FP32 and the
// largest |coordinate| among them (for the visibility FP32 pre-test);
// fac_lo: per facet 12 floats, the rounding residues of the FP32 centroid
// and vertex offsets in FacetRec (c - (double)rec.c, dv - (double)rec.dv),
// so that c and dv are available as double-float pairs
// the world-facet kernel (its t0 argument is updated in replayed frame graphs)
const void *build_facets_kernel_fn(int *t0_arg_index, int *n_args);
void launch_build_facets(const MeshDesc *meshes, const InstDev *insts, int n_inst,
                         int64_t F, double t0, double *tri64, float *tri32, double *c64,
                         FacetRec *fac, float *aabb, float *vel32, unsigned int *bounds,
                         double *ref64, float *ref32, float *fac_lo, cudaStream_t s);
void launch_morton(const FacetRec *fac, int64_t F, const unsigned int *bounds,
                   uint32_t *keys, int32_t *vals, cudaStream_t s);
// Stable LSD radix sort of (key, value) pairs on the low `bits` bits.
// Temp buffers sized by radix_sort_temp_words(n).
int64_t radix_sort_temp_words(int64_t n);
void radix_sort_pairs(uint32_t *keys, int32_t *vals, uint32_t *keys_tmp, int32_t *vals_tmp,
                      uint32_t *temp, int64_t n, int bits, cudaStream_t s);
void launch_lbvh_build(const uint32_t *keys, const int32_t *vals, int64_t n,
                       BvhNode *nodes, int32_t *parent, int32_t *leaf_parent,
                       cudaStream_t s);
// Batched scenes (facets [foff[b], foff[b+1]) form scene b, foff on the
// device): Morton codes, a sort by (scene, code), and one hierarchy whose
// scene subtrees are disjoint; root[b] receives scene b's root node (~facet
// for a one-facet scene).  mkeys, skeys: F words of scratch.
void launch_lbvh_batched(const FacetRec *fac, int64_t F, const unsigned int *bounds,
                         const int64_t *foff, int B, uint32_t *keys, int32_t *vals,
                         uint32_t *keys_tmp, int32_t *vals_tmp, uint32_t *temp, uint32_t *mkeys,
                         uint32_t *skeys, BvhNode *nodes, int32_t *parent, int32_t *leaf_parent,
                         int32_t *root, cudaStream_t s);
int lbvh_batched_launches(int B);
void launch_lbvh_refit(const int32_t *vals, const float *aabb, int64_t n, BvhNode *nodes,
                       const int32_t *parent, const int32_t *leaf_parent, int32_t *flags,
                       cudaStream_t s);

// ---- visibility (visibility.cu) ----
// order: facet ids in the sequence the ray threads take them (Morton order), or NULL.
// Batched scenes: foff (B + 1 facet offsets) and root (B scene roots) on the
// device, B > 1; a ray then only meets facets of its own scene.
struct SceneSplit {
    int B = 1;
    const int64_t *foff = nullptr;
    const int32_t *root = nullptr;
};
void launch_visibility(const double *tri64, const float *tri32, const double *c64,
                       const FacetRec *fac, const double *ref64, const BvhNode *nodes,
                       const int32_t *order, int64_t F, const RadarDev &rd,
                       const SceneSplit &sc, uint8_t *state, unsigned long long *n_graze,
                       int *status, cudaStream_t s);
// lists 0..O-1: facets lit from both antennas of each channel; O..O+A-1: facets
// lit from each antenna.  vis_idx is [O+A][F], vis_cnt [O+A].
void launch_compact(const uint8_t *state, int64_t F, const RadarDev &rd,
                    int32_t *blk_cnt, int32_t *vis_idx, int32_t *vis_cnt, cudaStream_t s);
int64_t compact_blk_words(int64_t F, int L);
// per (scene, channel) sub-ranges of the channel lists: vstart[b O + o] is
// the first entry of list o with facet >= foff[b], vcnt its length
void launch_scene_lists(const int32_t *vis_idx, const int32_t *vis_cnt, int64_t F, int O,
                        const int64_t *foff, int B, int32_t *vstart, int32_t *vcnt,
                        cudaStream_t s);

// ---- synthesis (synth.cu) ----
struct SynthArgs {
    const FacetRec *fac;
    const double *tri64;
    const double *c64;
    const double *vel64;     // per instance, 3 doubles
    const float *vel32;      // per instance, 4 floats (xyz, pad)
    const double *ref64;     // per instance, origin at t0 (3 doubles)
    const float *ref32;      // per instance, origin at t0 (4 floats)
    const float *fac_lo;     // per facet 12 floats: residues of FacetRec c[3], dv[9]
    const int32_t *vis_idx;  // [O][F]
    const int32_t *vis_cnt;  // [O + A]
    // virtual channels: VO = scenes x O rows of the output; row v reads
    // vcnt[v] entries of list v % O from entry vstart[v] (vstart NULL: 0)
    int VO;
    const int32_t *vstart;
    const int32_t *vcnt;
    int64_t F;
    const float4 *kin;       // [A][F][9] kinematics Taylor rows (mixed path)
    const double *kquad;     // [A][F][kKinQuadWords] FP64 data of rows without a expansion
    int n0, nc;              // chirp chunk
    void *out;
    int out_c64;
    unsigned long long *counters;   // [0] vertex, [1] series, [2] edge records
    // mixed path work queue (see synth.cu)
    int32_t *item_off;       // [O + 1] first work item of each channel
    int *item_counter;       // next item to hand out
    float2 *partial;         // [items][32 S] unscaled partial sums
    int tiles_per_item;      // 32-record tiles per item (set by the caller)
    int64_t max_items;       // upper bound of the work items (grid sizing)
    int layout_S;            // mixed-kernel samples per lane request (0 default, 8)
    RadarDev rd;
};
// per (antenna, lit facet) Taylor rows of R(t) over the frame (see synth.cu)
constexpr int kKinRowWords = 9;    // float4 per row
constexpr int kKinQuadWords = 5;   // doubles per row: R^2 = q0 + q1 t + q2 t^2 and, in the
                                   // far field, l = l0 + l1 t (path R + l / R)
void launch_kin_coef(const double *c64, const FacetRec *fac, const double *vel64,
                     const double *ref64, int64_t F, const RadarDev &rd, float4 *coef,
                     double *quad, cudaStream_t s);
void launch_synth_mixed(const SynthArgs &a, cudaStream_t s);
// scratch of the mixed path for F facets and a chunk of nc chirps
// scene_F: facets of each scene (n_scene entries); tpi: 32-record tiles per
// work item (0: the default for the largest scene)
int64_t synth_partial_words(const int64_t *scene_F, int n_scene, const RadarDev &rd, int nc,
                            int tpi, int S_req);   // float2 words
int64_t synth_max_items(const int64_t *scene_F, int n_scene, const RadarDev &rd, int nc, int tpi,
                        int S_req);
// samples per lane the mixed kernel uses for M and a layout request
int synth_layout_samples(int M, int S_req);
int synth_tiles_per_item(int64_t F);
void launch_synth_fp64(const SynthArgs &a, cudaStream_t s);
// spectral path (spectral.cu): 1 / (Fourier transform of the spreading
// kernels) at the M samples, host-computed (2 M floats: main grid, then the
// quadratic-phase grids); whether M's shared-memory footprint fits
bool spectral_supported(int M);
void spectral_tables(int M, float *host);
void launch_synth_spectral(const SynthArgs &a, const float *inv_psi, cudaStream_t s);
// chunks per chirp row of the FP64 synthesis; with more than one, SynthArgs
// partial must hold chunks x VO x N x M double2 (the chunks' partial sums)
int synth_fp64_chunks(const RadarDev &rd, int VO, int64_t F);

// ---- adjoint of the FP64 synthesis (adjoint.cu) ----
// gfac: F x 10 (world vertex coordinates at t0, reflectivity) per facet
void launch_adjoint_fp64(const SynthArgs &a, const void *grad, int grad_c64, double *gfac,
                         cudaStream_t s);
void launch_adjoint_mixed(const SynthArgs &a, const void *grad, int grad_c64, double *gfac,
                         cudaStream_t s);
// facet gradients -> instance-major mesh-local vertex gradients (voff: first
// vertex of each instance) and per-facet reflectivity gradients (may be NULL)
void launch_adjoint_scatter(const double *gfac, const FacetRec *fac, const InstDev *insts,
                            const MeshDesc *meshes, const int64_t *voff, int64_t F, double *gverts,
                            int64_t n_vert_words, double *grho, cudaStream_t s);

// ---- additive noise (noise.cu) ----
int64_t noise_scratch_words();   // doubles
void launch_add_noise(void *adc, int dtype, int64_t n, double snr_db, uint64_t seed,
                      unsigned int frame, double *scratch, cudaStream_t s);

// ---- range-Doppler map (rdm.cu) ----
int64_t rdm_workspace_bytes(const RadarDev &rd, int dtype);
// groups: independent cubes of rd.O channels each, back to back (batched
// scenes); rdm receives groups x M x N; ws holds groups x rdm_workspace_bytes
// status: the context's device status word (kStatusWaitTimeout), or NULL
void launch_rdm(const void *adc, int dtype, const RadarDev &rd, int groups, void *ws, float *rdm,
                int *status, cudaStream_t s);
// one block waiting `polls` polls on an mbarrier that nothing completes
// (the bounded-wait expiry path; sets kStatusWaitTimeout in *status)
void launch_wait_selftest(int polls, int *status, cudaStream_t s);

// RDM that also keeps the complex range-Doppler cube Y[o][r][d'] (Doppler
// shifted) in `cube`; X is an O*N*M complex scratch of the same precision.
void launch_rdm_cube(const void *adc, int dtype, const RadarDev &rd, void *X, void *cube,
                     float *rdm, cudaStream_t s);

// Adjoint of the RDM for dL/dRDM = grad_rdm (groups x M x N float32):
// grad_adc (same layout and precision as adc) = d L / d Re(adc) + i d L / d Im(adc).
// X and cube: groups x O x N x M complex scratch each.
void launch_rdm_adjoint(const void *adc, int dtype, const float *grad_rdm, const RadarDev &rd,
                        int groups, void *X, void *cube, void *grad_adc, cudaStream_t s);

// ---- detection: CA-CFAR, angle spectrum, points (detect.cu) ----
struct DetectDev {
    int guard_r, guard_d, hr, hd;  // guard and outer half-sizes
    int n_train;
    double alpha;                  // CA-CFAR threshold factor
    int bins;                      // azimuth grid size
    double lam_c;                  // band-centre wavelength
    double range_scale;            // metres per range bin (Eq. 4)
    double rate_scale;             // m/s per Doppler bin (Eq. 5)
};
struct DetectBufs {
    void *X, *cube;                // O*N*M complex each
    float *rdm;                    // M*N
    void *steer;                   // O*bins complex
    uint8_t *flag;                 // M*N
    int32_t *blk_cnt;              // M*N / rows_per_block
    int32_t *list;                 // M*N cell indices
    int32_t *count;                // 1
};
// bytes of each DetectBufs member for a radar / dtype / grid, 256-B aligned
int64_t detect_workspace_bytes(const RadarDev &rd, int dtype, int bins);
void detect_carve(void *ws, const RadarDev &rd, int dtype, int bins, DetectBufs *b);
// launches the RDM, CFAR, compaction and angle kernels; returns the count
int launch_detect(const void *adc, int dtype, const RadarDev &rd, const DetectDev &dd,
                  const DetectBufs &b, bart_point *points, int max_points, cudaStream_t s);

// Record `msg` as the calling thread's bart_last_error text; returns code.
int set_last_error(int code, const char *msg);

// Size of the static workspace used by bart_form_rdm_static (16 MiB).
constexpr int64_t kRdmStaticWorkspaceBytes = 16ll << 20;
// Device address of that workspace on the current device (looked up on
// every call).  Returns BART_OK or BART_ECUDA with *err set.
int rdm_static_workspace(void **ws, const char **err);

}  // namespace bart
