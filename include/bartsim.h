/*
 * bartsim.h -- C-ABI of the GB300 (sm_103a) BART radar-echo library.
 *
 * The library computes, on one GPU, the data-parallel hot path of the MMW
 * radar simulator of arXiv 2208.10939 (Zong & Zhu):
 *
 *   meshed targets  ->  BART single-bounce visibility  ->  physical-optics
 *   facet scattering per (TX, RX, frequency sample, chirp)  ->  coherent
 *   MIMO FMCW echo synthesis into the ADC cube  ->  windowed range-Doppler
 *   FFT into the range-Doppler map (RDM).
 *
 * Conventions for every entry point:
 *   - Return value: BART_OK (0) or a negative BART_E* status.  The text of
 *     the last error of the calling thread is returned by bart_last_error().
 *     No C++ exception crosses this interface.
 *   - "host" pointers are ordinary CPU memory; "device" pointers are CUDA
 *     global memory of the context's device (e.g. torch tensor data_ptr()).
 *   - Work is enqueued asynchronously on the stream bound with
 *     bart_set_stream (default: the legacy default stream).  Errors that
 *     only the device can detect (a BVH stack overflow) are latched in a
 *     device status word and returned by the next bart_sync().
 *   - The caller owns every pointer it passes; the library copies what it
 *     keeps (meshes, instances, radar) and owns all its scratch memory.
 *   - Geometry is in metres, time in seconds, frequency in hertz.
 *   - A context is not thread-safe: one host thread at a time per context.
 */
#ifndef BARTSIM_H
#define BARTSIM_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* status codes */
#define BART_OK        0
#define BART_EINVAL   (-1)   /* invalid argument or configuration */
#define BART_ENOMEM   (-2)   /* device allocation failed */
#define BART_ECUDA    (-3)   /* CUDA runtime error */
#define BART_ETIMEOUT (-4)   /* bounded device wait expired */
#define BART_ESTATE   (-5)   /* call out of order (e.g. simulate before radar_set) */
#define BART_EDEVICE  (-6)   /* device-side check failed (see bart_last_error) */

/* echo-synthesis precision paths */
#define BART_PATH_FP64  0    /* every quantity in FP64, exact per-sample delay */
#define BART_PATH_MIXED 1    /* FP64 path length + mod-1 reduction, FP32 phasors,
                                compensated (Kahan) accumulation */
#define BART_PATH_SPECTRAL 2 /* the mixed path's records, each chirp row summed by the
                                inverse-FFT route (Sec. 3.2): facet lines spread onto a
                                uniform beat-frequency grid of 2M cells, one inverse FFT
                                per row (a type-1 non-uniform FFT); needs M = 2^a 3^b */

/* complex sample types of an ADC cube (interleaved re, im) */
#define BART_C128 0          /* complex double */
#define BART_C64  1          /* complex float */

/* RDM windows */
#define BART_WINDOW_HANN 0   /* symmetric Hann, w[i] = 0.5 - 0.5 cos(2 pi i/(L-1)) */
#define BART_WINDOW_RECT 1

/* per-(antenna, facet) visibility states returned by bart_get_visibility */
#define BART_VIS_BACK  0     /* facet faces away from the antenna */
#define BART_VIS_LIT   1     /* front facing and unoccluded */
#define BART_VIS_GRAZE 2     /* within the grazing margins: excluded, counted */
#define BART_VIS_OCCL  3     /* centroid->antenna segment hits another facet */
#define BART_VIS_LIT_REV 4   /* two-sided facet lit on its reverse side, unoccluded */

/* mesh flags (bart_mesh_upload) */
#define BART_MESH_TWO_SIDED 1u   /* facets scatter from both sides (open surfaces:
                                    plates, signs); a channel sees such a facet when
                                    its TX and RX light the same side */

#define BART_MAX_TX 16
#define BART_MAX_RX 16

typedef struct bart_ctx bart_ctx;

/* A rigid placement of an uploaded mesh (Sec. 3.1 scene, Eq. 12 motion):
 *   x_world(t) = rot * x_local + pos + vel * t
 * rot is row-major 3x3.  rho_scale multiplies the mesh's facet
 * reflectivities (1 = perfect electric conductor). */
typedef struct bart_instance {
    int32_t mesh_id;
    float   rho_scale;
    double  pos[3];
    double  rot[9];
    double  vel[3];
} bart_instance;

/* FMCW MIMO radar (Sec. 2.1, Eq. 8; Sec. 3.3).  Channel o = p*Q + q pairs
 * TX p with RX q.  The ADC cube is [O][N][M] complex, fast-time sample m
 * contiguous (the paper's O x M x N data matrix, stored sample-major).
 * Sample m of chirp n is taken at t0 + n*Tc + m/fs; its instantaneous
 * transmit frequency is f0 + slope*m/fs.
 * Constraints (else BART_EINVAL): M a multiple of 32 in [32, 1024];
 * 1 <= N <= 32768; 1 <= P <= BART_MAX_TX; 1 <= Q <= BART_MAX_RX;
 * f0, slope, fs, Tc positive and finite; Tc >= M/fs; antenna positions
 * finite; flags 0 or 1; far_field and delay_ref not both set;
 * grazing_eps 0 (default 1e-6) or in (0, 0.1].  bart_form_rdm and
 * bart_detect further need M and N of the form 2^a 3^b (radix-2/3 FFTs;
 * N in [2, 1024]). */
typedef struct bart_radar {
    double  f0;                  /* chirp start frequency, Hz */
    double  slope;               /* mu, Hz/s */
    double  fs;                  /* ADC sampling rate, samples/s */
    double  Tc;                  /* chirp repetition period, s */
    int32_t M, N, P, Q;
    int32_t intra_chirp_motion;  /* 1: delay at t_n + t_m (Eq. 12, continuous t);
                                    0: delay held at the chirp start */
    int32_t window;              /* BART_WINDOW_* for bart_form_rdm */
    double  tx[BART_MAX_TX][3];  /* TX phase centres (first P used) */
    double  rx[BART_MAX_RX][3];  /* RX phase centres (first Q used) */
    int32_t tdm;                 /* 0: all TX chirp together (chirp n at n Tc);
                                    1: time-division MIMO, TX p sends chirp n at
                                    (n P + p) Tc (Doppler period P Tc) */
    int32_t delay_ref;           /* 0: delay of every facet from its own centroid;
                                    1: reference-point form of Eqs. 11-13: the
                                    facet's path length relative to its
                                    instance origin at the chirp start, plus the
                                    origin's path at t_n + t_m; residual video
                                    phase from the origin's delay */
    int32_t far_field;           /* 0: spherical waves from every facet centroid;
                                    1: far field (the Eq. 7 radar equation with
                                    the PO cross-section of the whole target):
                                    every facet of an instance is seen along the
                                    plane waves of the instance origin r, at the
                                    origin's ranges (directions, amplitude,
                                    obliquity, facet integral), its path the
                                    plane-wave one |p_tx - r(t)| + |p_rx - r(t)|
                                    - (t + r).(c_k - r(t_n)), and its visibility
                                    segment runs from the centroid toward
                                    p_a + (c_k - r(t0)) */
    int32_t double_bounce;       /* 0: single bounce only; 1: also the double-bounce
                                    paths of Sec. 2.2 (forward and backward rays
                                    joined through two facets), read as geometric
                                    optics at the first facet a (the field beyond
                                    it that of TX p mirrored in a's plane, within
                                    the beam through a) and physical optics on the
                                    part of the second facet b that the beam
                                    lights; the a -> b leg must be unoccluded and
                                    b seen from RX q; reflectivity -rho_a rho_b.
                                    Decided on the frame-start geometry; always
                                    FP64; one scene per frame, per-facet delay
                                    form (not with far_field or delay_ref), no
                                    adjoint; frames then synchronise the stream
                                    twice (to size the candidates and the
                                    virtual facets) and are not replayed as
                                    graphs.  See bart_get_bounce_facets. */
    double  grazing_eps;         /* facets with |cos| below this toward an antenna
                                    are GRAZE (excluded, counted); 0 = 1e-6 */
} bart_radar;

/* Per-frame counters (filled when a non-NULL pointer is passed; doing so
 * synchronises the stream). */
typedef struct bart_stats {
    int64_t n_facets;       /* facets in the scene */
    int64_t n_terms;        /* echo terms: sum over channels of lit facets x N x M */
    int64_t n_lit_pairs;    /* (facet, channel) pairs lit from TX and RX */
    int64_t n_grazing;      /* (antenna, facet) pairs flagged BART_VIS_GRAZE */
    int64_t n_series;       /* (facet, channel, chirp) records by the series form */
    int64_t n_edge;         /* records by the edge form */
    int64_t n_vertex;       /* records by the vertex form */
    int64_t n_bounce_facets;   /* double-bounce virtual facets (bart_get_bounce_facets) */
    int64_t n_bounce_terms;    /* double-bounce echo terms: (virtual facet, channel,
                                  chirp) records with b seen from the RX, x M */
} bart_stats;

/* Per-stage device times of the last frame, from CUDA events recorded on
 * the context's stream while timing is enabled (bart_set_timing). */
typedef struct bart_timing {
    float   scene_ms;        /* world facets at t0 */
    float   bvh_ms;          /* Morton codes, radix sort, hierarchy, refit */
    float   visibility_ms;   /* visibility states + per-channel lit lists */
    float   kinematics_ms;   /* FP64 Taylor rows of the path lengths (mixed path;
                                on a second stream, overlapping bvh_ms and
                                visibility_ms) */
    float   synthesis_ms;    /* echo-synthesis kernels */
    float   rdm_ms;          /* last bart_form_rdm */
    int32_t synthesis_launches;   /* synthesis kernel launches in the frame */
    int32_t launches;        /* kernels launched by the last simulate + form_rdm */
    float   detect_ms;       /* last bart_detect (RDM, CFAR, angle, points) */
    int32_t detect_launches; /* kernels launched by the last bart_detect */
    float   bounce_discovery_ms;  /* double bounce: virtual-facet count, scan and
                                     fill, with the host read of the count (inside
                                     visibility_ms); 0 without double bounce */
    float   bounce_synthesis_ms;  /* double bounce: the FP64 synthesis of the virtual
                                     facets (inside synthesis_ms on the FP64 and
                                     spectral paths, after it on the mixed path) */
} bart_timing;

/* Text of the calling thread's last error ("" if none).  Valid until the
 * thread's next bart_* call. */
const char *bart_last_error(void);

/* Library version string. */
const char *bart_version(void);

/* Host-side fault injection for tests of the error paths: the nth device
 * allocation the library makes from now on (nth >= 1; counted over every
 * context of the process) fails with BART_ENOMEM before cudaMalloc is
 * called, exactly as an out-of-memory cudaMalloc would surface; later
 * allocations proceed.  nth = 0 disarms it.  Nothing reaches the GPU.
 * Errors: EINVAL (nth < 0). */
int bart_inject_alloc_failure(int32_t nth);

/* Self-test of the bounded device waits (the TMA-fed Doppler pass of
 * bart_form_rdm waits on mbarriers for its tile copies, with a limit): one
 * block waits `polls` polls (1 .. 2^20) on a barrier that nothing
 * completes, so the wait expires by design, and the context's device status
 * records it.  The next bart_sync returns BART_ETIMEOUT, clears the status,
 * and the context stays usable.  Enqueued on the context's stream.
 * Errors: EINVAL (ctx NULL, polls out of range), ECUDA. */
int bart_selftest_wait_timeout(bart_ctx *ctx, int32_t polls);

/* Create a context on CUDA device `device`.  *out receives the handle.
 * Errors: EINVAL (bad device / NULL out), ECUDA. */
int bart_create(bart_ctx **out, int device);

/* Free the context and every device buffer it owns.  NULL is ignored. */
void bart_destroy(bart_ctx *ctx);

/* Enqueue all later work on `stream` (a cudaStream_t, e.g. torch's
 * torch.cuda.current_stream().cuda_stream); 0 = legacy default stream. */
int bart_set_stream(bart_ctx *ctx, void *stream);

/* Upload a triangle mesh (host pointers, copied; the caller may free them
 * on return).  verts: nv x 3 float64; tris: nf x 3 int32 vertex indices,
 * counter-clockwise seen from outside (outward normal (v1-v0)x(v2-v0));
 * rho: nf float32 reflectivities or NULL for all 1; flags: 0 or
 * BART_MESH_TWO_SIDED (Sec. 2.2 visibility, the PO obliquity taken on the
 * side the antennas light).  *mesh_id receives the id used by
 * bart_instance.  Errors: EINVAL (index out of range, nf < 1, unknown flag,
 * a non-finite vertex coordinate or reflectivity), ENOMEM, ECUDA. */
int bart_mesh_upload(bart_ctx *ctx, const double *verts, int64_t nv,
                     const int32_t *tris, int64_t nf, const float *rho,
                     uint32_t flags, int32_t *mesh_id);

/* Replace the vertices (and, if rho is not NULL, the reflectivities) of an
 * uploaded mesh from DEVICE arrays of the uploaded sizes (nv x 3 float64,
 * nf float32), asynchronously on the context's stream.  Topology is kept,
 * so a recorded frame graph stays valid and picks the new values up (the
 * gradient-descent loop of the differentiable echo).  Errors: EINVAL, ECUDA. */
int bart_mesh_update(bart_ctx *ctx, int32_t mesh_id, const double *verts, const float *rho);

/* Remove every uploaded mesh and the scene. */
int bart_mesh_clear(bart_ctx *ctx);

/* Set the scene's instances (host array of n, copied).  Each mesh_id must
 * name an uploaded mesh; positions, velocities, rotations and rho_scale must
 * be finite.  Errors: EINVAL. */
int bart_scene_set(bart_ctx *ctx, const bart_instance *inst, int32_t n);

/* Total facet count of the current scene (host out). */
int bart_scene_facets(bart_ctx *ctx, int64_t *n_facets);

/* The sizes of the buffers the context reads and writes.  The library
 * receives bare addresses, so a caller (the Python binding) checks its
 * buffers against these before each call.  Host-only: nothing is enqueued.
 * Fields are 0 where the state they describe is not set yet. */
typedef struct bart_dims {
    int32_t device;        /* CUDA ordinal of the context */
    int32_t have_radar;    /* 1 after a successful bart_radar_set */
    int32_t n_scenes;      /* S: scenes of the partition (1 without one) */
    int32_t O;             /* channels P*Q */
    int32_t N;             /* chirps */
    int32_t M;             /* samples per chirp */
    int32_t A;             /* antennas P+Q */
    int32_t n_meshes;      /* uploaded meshes */
    int64_t n_facets;      /* facets of the current scene (grad_rho length) */
    int64_t n_inst_verts;  /* vertex count summed over the instances' meshes
                              (grad_verts holds 3 x this many) */
    int64_t vis_antennas;  /* the last frame's visibility states: antennas ... */
    int64_t vis_facets;    /* ... x facets (bart_get_visibility's output) */
} bart_dims;

/* Fill *out (host).  A simulation frame writes S*O*N*M samples; an RDM is
 * S*M*N floats; bart_add_noise and bart_detect take one O*N*M cube.  No
 * counterpart in the paper: bookkeeping of this interface.
 * Errors: EINVAL (NULL argument). */
int bart_get_dims(bart_ctx *ctx, bart_dims *out);

/* Vertex and facet counts of uploaded mesh `mesh_id` (host outs): the sizes
 * bart_mesh_update reads (3 x nv float64, nf float32).  No counterpart in
 * the paper.  Errors: EINVAL (NULL argument, unknown mesh). */
int bart_mesh_dims(bart_ctx *ctx, int32_t mesh_id, int64_t *nv, int64_t *nf);

/* Split the instance table of the last bart_scene_set into independent
 * scenes simulated in one pass (dataset generation: many small scenes per
 * launch).  Instances [first[b], first[b+1]) form scene b, with
 * 0 = first[0] < first[1] < ... < first[n_scenes] = number of instances
 * (host array of n_scenes + 1 int32).  Each scene is simulated as if alone
 * -- its facets are lit, shadowed and summed among its own facets only --
 * and owns one slab of the batched outputs: bart_simulate_frame then writes
 * n_scenes x O x N x M samples ([scene][channel][chirp][sample]), and
 * bart_form_rdm / bart_frame_host read that many and write n_scenes x M x N.
 * Work of all scenes shares each launch: one hierarchy with a subtree per
 * scene, one visibility launch, one synthesis work queue over (scene,
 * channel, chirp group, record chunk) items.  bart_scene_set resets the
 * partition to one scene.  n_scenes x O must not exceed 65535.
 * Errors: EINVAL (bad offsets), ESTATE (no instances). */
int bart_scene_partition(bart_ctx *ctx, const int32_t *first, int32_t n_scenes);

/* Set the radar (host struct, copied and validated: sizes, positive finite
 * f0/slope/fs/Tc with Tc >= M/fs, finite antenna positions, flags 0 or 1,
 * exclusive modes).  Errors: EINVAL. */
int bart_radar_set(bart_ctx *ctx, const bart_radar *radar);

/* Simulate one frame starting at absolute time t0 (Sec. 3.2):
 *   1. world facets at t0 (rigid instance poses),
 *   2. LBVH over the facets and the BART single-bounce visibility of every
 *      facet from every antenna (Sec. 2.2), held for the frame,
 *   3. per (channel, chirp) the physical-optics coefficient of every facet
 *      lit from TX and RX, and the dechirped IF samples (Eqs. 7, 9-13).
 * adc: device pointer to O*N*M complex samples of type `dtype`, written
 * completely.  path: BART_PATH_FP64, BART_PATH_MIXED or BART_PATH_SPECTRAL.
 * stats: optional host pointer (NULL = fully asynchronous).
 * Errors: ESTATE (no radar / scene), EINVAL, ENOMEM, ECUDA. */
int bart_simulate_frame(bart_ctx *ctx, double t0, int32_t path, void *adc,
                        int32_t dtype, bart_stats *stats);

/* Add white complex Gaussian noise to an ADC cube of the current radar
 * shape, in place (Sec. 3.2: noise "with a certain signal-to-noise ratio"):
 *   x[e] += sigma n[e],  sigma^2 = P / 10^(snr_db/10),  P = mean |x|^2 of the cube,
 *   n[e] ~ CN(0, 1) from Philox4x32-10 (Salmon et al., SC 2011) with counter
 *   (e mod 2^32, e div 2^32, frame, 0) and key (seed mod 2^32, seed div 2^32),
 *   mapped to uniforms (w + 1) 2^-32 and through Box-Muller;
 * e is the element index in the [O][N][M] cube.  adc: device pointer of
 * `dtype` (FP64 arithmetic for C128, FP32 for C64).  Deterministic for a
 * given (seed, frame).  Errors: ESTATE, EINVAL, ENOMEM, ECUDA. */
int bart_add_noise(bart_ctx *ctx, void *adc, int32_t dtype, double snr_db, uint64_t seed,
                   uint32_t frame);

/* Adjoint of the plain FP64 echo synthesis (the differentiable echo).  For
 * a real loss L of the ADC cube of the frame at t0, given
 * grad_adc = dL/dRe(adc) + i dL/dIm(adc) (device, the layout
 * bart_simulate_frame writes, dtype C128 or C64), writes
 *   grad_verts: dL/d(mesh-local vertex coordinates), device FP64,
 *       instance-major: instance i's mesh vertices (x, y, z each) start at
 *       3 * (sum of the vertex counts of the meshes of instances 0..i-1);
 *       sum over the instances that share a mesh for that mesh's gradient;
 *   grad_rho: dL/d(mesh reflectivity of each facet), device FP64, one per
 *       scene facet (instance-major), or NULL.
 * The derivative is the exact one of the FP64 synthesis as implemented
 * (every facet-integral form), through the facet integral, the obliquity,
 * the distances and the delay; visibility is recomputed at t0 and held
 * fixed (it is piecewise constant in the vertices).  Instance poses,
 * velocities and rho_scale are constants.  Works with scene partitions.
 * Not available with far_field (EINVAL).
 * Errors: ESTATE, EINVAL, ENOMEM, ECUDA. */
int bart_simulate_adjoint(bart_ctx *ctx, double t0, const void *grad_adc, int32_t dtype,
                          double *grad_verts, double *grad_rho);

/* bart_simulate_adjoint with the per-sample work of vertex-form records in
 * FP32 (Sec. 3.2, Eq. 13 differentiated as above): FP64 fixes each vertex's
 * phase at three samples of a lane of 8, FP32 rotations carry the phasor
 * along the chord of those phases, and the record adjoint is summed in FP32
 * before the FP64 reduction and the FP64 pass through the record
 * construction; series and edge records take the FP64 path.  Same
 * arguments and results as bart_simulate_adjoint, to ~1e-5 of the gradient's
 * norm (the phase's curvature over a lane, ~1e-5 rad on a moving car, and
 * FP32 sums); several times faster.  Errors: ESTATE, EINVAL, ENOMEM, ECUDA. */
int bart_simulate_adjoint_mixed(bart_ctx *ctx, double t0, const void *grad_adc, int32_t dtype,
                                double *grad_verts, double *grad_rho);

/* Frame graphs.  With enable = 1, bart_simulate_frame records its kernel
 * launches (world facets, hierarchy, visibility, lit lists, kinematics,
 * synthesis: some 25-40 launches on two streams) into a CUDA graph the
 * first time it meets a configuration -- meshes, instances, partition,
 * radar, synthesis layout, path, dtype, output pointer and stream -- and
 * replays that graph, one launch, on later calls that differ at most in
 * t0 (the new t0 is written into the recorded world-facet launch).  Any
 * change of the configuration records again.  Calls that request stats,
 * or run with timing enabled, run directly.  enable = 0 (the default)
 * drops the graph.  Errors: EINVAL, ECUDA. */
int bart_set_graph(bart_ctx *ctx, int32_t enable);

/* Work layout of the mixed-path synthesis kernel: samples_per_lane 16 (or
 * 0, the default), 8 (where M allows: M divides 256 or 256 divides M) or 32
 * (M = 256, 512 or 1024);
 * tiles_per_item = 32-record tiles per work item (0 = default, scaled with
 * the largest scene).  The results differ only by FP32 summation order.
 * Errors: EINVAL. */
int bart_set_synth_layout(bart_ctx *ctx, int32_t samples_per_lane, int32_t tiles_per_item);

#define BART_TUNE_MAX 24
/* Autotuner result: every trial's layout and best synthesis time. */
typedef struct bart_tune {
    int32_t n_trials;
    int32_t best_samples_per_lane;
    int32_t best_tiles_per_item;
    float   best_ms;
    int32_t samples_per_lane[BART_TUNE_MAX];
    int32_t tiles_per_item[BART_TUNE_MAX];
    float   synthesis_ms[BART_TUNE_MAX];
} bart_tune;

/* Time the mixed-path synthesis of the current scene at t0 for each
 * candidate layout (samples per lane 16 and, where M allows, 32 and 8; tiles per
 * item 8 ... 512), each run once to warm up and then `reps` times (best
 * time kept, CUDA events around the synthesis launches), and keep the
 * fastest layout for later frames (as bart_set_synth_layout).  adc: device
 * output of the shape bart_simulate_frame writes (overwritten).  Blocks
 * until done.  Errors: EINVAL, ESTATE, ENOMEM, ECUDA. */
int bart_autotune(bart_ctx *ctx, double t0, void *adc, int32_t dtype, int32_t reps,
                  bart_tune *out);

/* Range-Doppler map (Sec. 3.3) of an ADC cube of the current radar shape:
 * window + forward FFT over fast time, window + forward FFT over chirps,
 * |.|^2 summed over the O channels, zero Doppler shifted to bin N/2.
 * adc: device pointer, O*N*M complex of `dtype` (FP64 arithmetic for C128,
 * FP32 for C64).  rdm: device pointer, M x N float32 (range-major).
 * Errors: ESTATE, EINVAL (M or N not of the form 2^a 3^b, N > 1024),
 * ENOMEM, ECUDA. */
int bart_form_rdm(bart_ctx *ctx, const void *adc, int32_t dtype, float *rdm);

/* Adjoint of bart_form_rdm (the RDM step of the differentiable echo): for a
 * real loss L with dL/dRDM = grad_rdm (device, M x N float32 per scene, the
 * RDM layout), writes grad_adc = dL/dRe(adc) + i dL/dIm(adc) (device, the
 * layout and dtype of adc): 2 grad_rdm Y on the range-Doppler cube Y of adc,
 * then the conjugate transposes of the windowed Doppler and range DFTs.
 * adc is the cube the RDM was formed from (the RDM is nonlinear in it).
 * Errors: ESTATE, EINVAL, ENOMEM, ECUDA. */
int bart_rdm_adjoint(bart_ctx *ctx, const void *adc, int32_t dtype, const float *grad_rdm,
                     void *grad_adc);

/* bart_form_rdm without any device allocation, for callers that cannot let
 * a library allocate GPU memory: applications that own all device memory
 * through their own pool allocator or run under a hard memory cap (a
 * foreign cudaMalloc breaks their accounting or fails), and latency-bound
 * loops where cudaMalloc/cudaFree would stall on a device synchronisation.
 * The paper has no counterpart; it is an operational variant of the RDM
 * (Sec. 3.3) computation above and gives the same result.
 *
 * No context is needed: the cube shape is passed explicitly.  adc: device
 * pointer, O*N*M complex samples of `dtype`, [O][N][M]; rdm: device pointer,
 * M x N float32; window: BART_WINDOW_*; stream: a cudaStream_t (0 = legacy
 * default stream) on the current device.  The range-FFT intermediate
 * and the per-channel Doppler power live in a fixed 16 MiB array compiled
 * into the library, which every GPU that loads the library holds until the
 * process exits; cubes needing more (O*N*M > 1398101 complex64 or 699050
 * complex128 samples: 12 bytes, resp. 24, per sample) are rejected with
 * BART_EINVAL.  M and N must be of the form 2^a 3^b (M in [32, 1024], N in
 * [2, 1024]).  Every call looks the array's address up
 * (cudaGetSymbolAddress, which allocates nothing) with the current device,
 * which must be the device of adc and rdm.  Under CUDA's default lazy
 * module loading the array is reserved when this file's module first loads
 * on a device -- the first RDM call or symbol lookup there -- so a process
 * under a hard memory cap should make one warm-up call at initialisation,
 * before it fills the device and before any stream capture.  The array is
 * shared by every call and keeps the last call's contents (each call
 * overwrites the part it reads before reading it, so nothing carries over);
 * calls that overlap on the GPU, from any thread or stream, race on it and
 * must be serialised by the caller.  The call calls no cudaMalloc/cudaFree.
 * Without a context there is no device status word: the Doppler pass's
 * bounded waits for its tile copies (which bart_form_rdm reports through
 * bart_sync as BART_ETIMEOUT) would, if one ever expired, leave the map
 * incomplete without an error code here.
 * Errors: EINVAL, ECUDA. */
int bart_form_rdm_static(const void *adc, int32_t dtype, int32_t O, int32_t N,
                         int32_t M, int32_t window, float *rdm, void *stream);

/* CA-CFAR detector and azimuth estimator settings (Sec. 3.3).  The
 * training cells of a cell under test are those of the rectangle of
 * half-sizes (guard_r + train_r) x (guard_d + train_d) around it that lie
 * outside the guard rectangle of half-sizes guard_r x guard_d; the Doppler
 * axis wraps, range cells whose rectangle leaves [0, M) are not tested.
 * Constraints (else BART_EINVAL): guard_*, train_* >= 0; at least one
 * training cell; guard_r + train_r <= 64 and 2 (guard_r + train_r) < M;
 * guard_d + train_d <= 64 and 2 (guard_d + train_d) < N; 0 < pfa < 1;
 * 2 <= angle_bins <= 4096; reserved == 0. */
typedef struct bart_detect_cfg {
    int32_t guard_r, guard_d;    /* guard half-widths, range / Doppler bins */
    int32_t train_r, train_d;    /* training band widths beyond the guard */
    double  pfa;                 /* design false-alarm probability in exponential
                                    (square-law) noise: threshold factor
                                    alpha = n (pfa^(-1/n) - 1), n training cells */
    int32_t angle_bins;          /* azimuth grid: s_i = sin(az) = -1 + 2 i / angle_bins */
    int32_t reserved;            /* must be 0 */
} bart_detect_cfg;

/* One detected point (56 bytes).  Frame: radar-centred, boresight +Y,
 * azimuth from +Y toward +X. */
typedef struct bart_point {
    double  range;               /* m: c fs r_bin / (2 slope M)              (Eq. 4) */
    double  rate;                /* m/s: lambda_c (d_bin - N/2) / (2 N Tr), Tr = Tc
                                    (P Tc with tdm),
                                    positive receding, lambda_c = c / (f0 + B/2),
                                    B = slope M / fs                         (Eq. 5) */
    double  azimuth;             /* rad: asin(s_i) at the angle-spectrum peak (Eq. 6) */
    double  x, y;                /* m: range sin(azimuth), range cos(azimuth) */
    double  power;               /* RDM value of the cell */
    int32_t r_bin, d_bin;        /* range bin; Doppler bin after the N/2 shift */
} bart_point;

/* Radar point cloud from an ADC cube of the current radar shape (Sec. 3.3,
 * Eqs. 4-6): the RDM of bart_form_rdm; CA-CFAR on it, deciding in FP64
 * (power > alpha * mean of the training cells); for every detection, in
 * row-major (r_bin, d_bin) order, the angle spectrum
 *   S(s_i) = | sum_o Y_o(r, d) exp(+j 2 pi x_o s_i / lambda_c) |^2
 * over the O virtual channels (x_o = tx[p][0] + rx[q][0], o = p Q + q;
 * Y the windowed range-Doppler cube in the FFT's precision), its first
 * maximum giving the azimuth.
 *   adc: device pointer, O*N*M complex of `dtype` (C64: FP32 FFTs and
 *        spectrum; C128: FP64).
 *   rdm: device pointer, M x N float32, receives the RDM; may be NULL.
 *   points: device pointer of max_points bart_point (may be NULL when
 *        max_points is 0); receives the first min(count, max_points) points.
 *   n_points: host pointer or NULL.  When given, the call synchronises the
 *        stream and stores the number of detections (which may exceed
 *        max_points); when NULL the call stays asynchronous.
 * M and N must be of the form 2^a 3^b (N <= 1024) as for bart_form_rdm.
 * Errors: ESTATE, EINVAL, ENOMEM, ECUDA. */
int bart_detect(bart_ctx *ctx, const void *adc, int32_t dtype, const bart_detect_cfg *cfg,
                float *rdm, bart_point *points, int32_t max_points, int32_t *n_points);

/* One whole frame with host buffers: simulate into library-owned device
 * memory, form the RDM and copy it to the host array rdm_host (M x N
 * float32), then synchronise.  Meshes/instances/radar must already be set.
 * stats: optional host pointer. */
int bart_frame_host(bart_ctx *ctx, double t0, int32_t path, float *rdm_host,
                    bart_stats *stats);

/* Copy the frame-start visibility states (BART_VIS_*) of the last
 * simulated frame into the device buffer `state` (A x F uint8, A = P + Q
 * antennas, TX first, then RX), and, when n_grazing is not NULL, store the
 * number of (antenna, facet) pairs flagged BART_VIS_GRAZE there (host
 * pointer; synchronises the stream).  Errors: ESTATE (no frame simulated). */
int bart_get_visibility(bart_ctx *ctx, uint8_t *state, int64_t *n_grazing);

/* One internal node of the bounding-volume hierarchy the visibility rays
 * traverse (Sec. 2.2 ray tracing; a Karras LBVH over the frame-start
 * facets).  left/right >= 0 name internal nodes, a negative child c is the
 * leaf of facet ~c.  Each child's box (FP32, rounded outward from the FP64
 * vertices) is stored in its parent. */
typedef struct bart_bvh_node {
    float   lmin[3];
    int32_t left;
    float   lmax[3];
    int32_t right;
    float   rmin[3];
    int32_t pad0;
    float   rmax[3];
    int32_t pad1;
} bart_bvh_node;

/* Host copy of the last frame's hierarchy, for host-side checks of its
 * invariants (every facet under exactly one leaf, every child's box inside
 * its slot, each scene's subtree holding exactly its own facets).
 * Writes *n_nodes = F - 1 internal nodes (0 when F = 1), *n_facets = F and
 * *n_scenes = S of that frame; with nodes, roots and tri all NULL nothing
 * else is done (a size query).  Otherwise, host buffers: nodes (n_nodes
 * bart_bvh_node, node 0 the root of the whole hierarchy), roots (S int32:
 * the root node of each scene's subtree, ~facet for a one-facet scene) and
 * tri (F x 9 float64: the frame-start world vertices the boxes enclose).
 * Synchronises the stream.  No counterpart in the paper: a diagnostic of
 * this library's own data structure.
 * Errors: EINVAL (NULL size pointers, some but not all buffers NULL),
 * ESTATE (no frame simulated), ECUDA. */
int bart_get_bvh(bart_ctx *ctx, bart_bvh_node *nodes, int32_t *roots, double *tri,
                 int64_t *n_nodes, int64_t *n_facets, int32_t *n_scenes);

/* The virtual facets of the last frame's double-bounce paths (Sec. 2.2;
 * bart_radar.double_bounce): each is one fan piece (Pi_0, Pi_i, Pi_i+1) of
 * the part Pi_ab of facet b lit by TX p's reflection from facet a.  Host
 * buffers, cap entries each: pab (4 int32: p, a, b, side of b lit: +1 the
 * front, -1 the reverse of a two-sided facet), tri (9 doubles: frame-start
 * vertices), src (3: the image source, TX p mirrored in a's plane, at the
 * frame start), usrc (3: its velocity), w (1: -rho_a rho_b).  Order: TX, then
 * a in ascending index, then the order of the BVH traversal (deterministic
 * for a scene).  *n receives the count (all of them; min(cap, n) written).
 * Synchronises the stream.  BART_ESTATE without a frame; the count is 0 when
 * the frame had double bounce off. */
int bart_get_bounce_facets(bart_ctx *ctx, int32_t *pab, double *tri, double *src, double *usrc,
                           double *w, int64_t cap, int64_t *n);

/* Enable (1) or disable (0) recording of per-stage CUDA events.  The events
 * are recorded on the context's stream; enabling adds no synchronisation. */
int bart_set_timing(bart_ctx *ctx, int32_t enable);

/* Per-stage times of the last simulated frame and RDM (host out); waits for
 * the recorded events.  Errors: ESTATE (timing disabled or no frame). */
int bart_get_timing(bart_ctx *ctx, bart_timing *out);

/* Wait for the context's stream; return a latched device-side error
 * (BART_EDEVICE) or a CUDA error, else BART_OK. */
int bart_sync(bart_ctx *ctx);

/* Measured arithmetic-pipe rates of the device (the denominators of the
 * echo-synthesis roofline).  Register-only kernels, eight independent
 * dependency chains per thread, 2048 threads per SM, CUDA-event timed, best
 * of `reps` runs after one warm-up; at whatever clocks the device runs. */
typedef struct bart_peaks {
    double fp32_fma_per_s;     /* scalar FP32 FMAs/s (one FMA-pipe operation each) */
    double fp32x2_fma_per_s;   /* FP32 FMAs/s issued as packed fma.rn.f32x2 (two per instruction) */
    double sincos_per_s;       /* __sincosf pairs/s (MUFU sine + cosine) */
    double fp64_fma_per_s;     /* FP64 FMAs/s */
    int32_t sms;               /* streaming multiprocessors of the device */
    int32_t threads;           /* threads of each launch */
} bart_peaks;

/* Run the peak microbenchmarks on CUDA device `device` (made current),
 * reps in [1, 100].  Allocates and frees a small device buffer; blocks.
 * Errors: EINVAL, ENOMEM, ECUDA. */
int bart_measure_peaks(int32_t device, int32_t reps, bart_peaks *out);

#ifdef __cplusplus
}
#endif

#endif /* BARTSIM_H */
