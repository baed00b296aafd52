// C-ABI of libbartsim (include/bartsim.h): context, uploads and the frame
// orchestration (world facets -> LBVH -> visibility -> kinematics ->
// synthesis -> RDM), all enqueued on the context's stream.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "bart_internal.cuh"
#include "bounce.cuh"
#include "bartsim.h"

using namespace bart;

namespace {

// NVTX ranges for the stages of a call, as the host enqueues them (they show
// the stages in Nsight timelines; header-only, no cost without a tool
// attached): next() closes the open stage and opens another; leaving the
// scope, on any return path, closes the last one
struct Stages {
    bool open = false;
    void next(const char *name)
    {
        if (open) nvtxRangePop();
        nvtxRangePushA(name);
        open = true;
    }
    ~Stages()
    {
        if (open) nvtxRangePop();
    }
};

thread_local std::string g_err;

int fail(int code, const char *fmt, ...) __attribute__((format(printf, 2, 3)));
int fail(int code, const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_err = buf;
    return code;
}

int cuda_fail(cudaError_t e, const char *what)
{
    cudaGetLastError();
    return fail(e == cudaErrorMemoryAllocation ? BART_ENOMEM : BART_ECUDA, "%s: %s", what,
                cudaGetErrorString(e));
}

// Host-side fault injection (bart_inject_alloc_failure): the countdown-th
// device allocation from now fails as if cudaMalloc had run out of memory.
std::atomic<int64_t> g_fail_countdown{0};

bool injected_alloc_failure()
{
    int64_t c = g_fail_countdown.load();
    while (c > 0)
        if (g_fail_countdown.compare_exchange_weak(c, c - 1)) return c == 1;
    return false;
}

template <typename T> struct DevBuf {
    T *p = nullptr;
    size_t cap = 0;
    int ensure(size_t n, const char *what)
    {
        if (n <= cap) return BART_OK;
        release();
        if (n == 0) return BART_OK;
        if (injected_alloc_failure())
            return fail(BART_ENOMEM, "cudaMalloc(%zu bytes) for %s failed: injected failure",
                        n * sizeof(T), what);
        cudaError_t e = cudaMalloc(&p, n * sizeof(T));
        if (e != cudaSuccess) {
            p = nullptr;
            cudaGetLastError();
            return fail(BART_ENOMEM, "cudaMalloc(%zu bytes) for %s failed: %s", n * sizeof(T),
                        what, cudaGetErrorString(e));
        }
        cap = n;
        return BART_OK;
    }
    void release()
    {
        if (p) cudaFree(p);
        p = nullptr;
        cap = 0;
    }
};

struct MeshStore {
    DevBuf<double> verts;
    DevBuf<int32_t> tris;
    DevBuf<float> rho;
    int64_t nv = 0, nf = 0;
    bool has_rho = false;
    uint32_t flags = 0;
};

}  // namespace

namespace bart {
int set_last_error(int code, const char *msg) { return fail(code, "%s", msg); }
}  // namespace bart

struct bart_ctx {
    int device = 0;
    cudaStream_t stream = nullptr;
    std::vector<MeshStore *> pool;     // reused across bart_mesh_clear
    int n_meshes = 0;
    std::vector<bart_instance> insts;
    bart_radar radar{};
    bool have_radar = false;
    bool have_frame = false;
    bool tables_dirty = true;   // mesh / instance tables changed since the last frame
    int64_t frame_F = 0;
    int frame_A = 0;
    int frame_B = 1;            // scenes of the last frame's partition

    DevBuf<MeshDesc> d_meshes;
    DevBuf<InstDev> d_insts;
    DevBuf<double> tri64, c64, vel64;
    DevBuf<float> tri32;
    DevBuf<float> vel32, aabb;
    DevBuf<double> ref64;               // instance origins at t0 (delay reference points)
    DevBuf<float> ref32;
    DevBuf<FacetRec> fac;
    DevBuf<float> fac_lo;
    DevBuf<unsigned int> bounds;
    DevBuf<uint32_t> keys, keys_tmp, sort_temp;
    DevBuf<int32_t> vals, vals_tmp;
    DevBuf<BvhNode> nodes;
    DevBuf<int32_t> parent, leaf_parent, flags;
    DevBuf<uint8_t> state;
    DevBuf<int32_t> blk_cnt, vis_idx, vis_cnt;
    DevBuf<float4> kin;                 // kinematics Taylor rows [A][F][9]
    DevBuf<double> kquad;               // FP64 row data [A][F][kKinQuadWords]
    DevBuf<float2> partial;             // mixed-path per-item partial sums
    DevBuf<int32_t> item_off;
    DevBuf<int> item_counter;
    DevBuf<unsigned long long> counters;   // 0 vertex, 1 series, 2 edge, 3 grazing
    DevBuf<int> status;
    DevBuf<unsigned char> rdm_ws, adc_own;
    DevBuf<double> noise_scratch;
    DevBuf<float> rdm_own;
    DevBuf<float> spec_tab;             // spectral path: 1 / kernel transforms [2][M]
    int spec_M = 0;
    DevBuf<unsigned char> det_ws;       // detection: cube, RDM, steering table, lists
    DevBuf<unsigned char> adj_ws;       // adjoints: RDM cube scratch
    DevBuf<double> gfac;                // synthesis adjoint: per-facet gradients [F][10]
    DevBuf<int64_t> d_voff;             // first mesh vertex of each instance (adjoint output)
    const void *adj_grad = nullptr;     // the pending adjoint call's arguments
    int adj_grad_c64 = 0;
    double *adj_gverts = nullptr, *adj_grho = nullptr;
    int64_t adj_vwords = 0;
    // scene partition (batched dataset frames): instances [scene_first[b],
    // scene_first[b+1]) form scene b; empty = one scene
    std::vector<int32_t> scene_first;
    int n_scenes = 1;
    DevBuf<int64_t> d_foff;             // facet offsets of the scenes [B + 1]
    DevBuf<int32_t> d_root;             // BVH root of each scene [B]
    DevBuf<int32_t> vstart, vcnt;       // per (scene, channel) list ranges [B O]
    // double bounce: pieces per (TX, lit facet) item, their offsets, the scan
    // scratch (its last word the total) and the virtual facets of the frame
    DevBuf<int32_t> db_cnt;
    DevBuf<int32_t> db_roots;           // the candidate traversal's subtree roots
    DevBuf<int64_t> db_off, db_blk;
    DevBuf<BounceFacet> db_vf;
    DevBuf<BounceCand> db_cand;         // candidates (a, b) of every (TX, lit facet a)
    DevBuf<int32_t> db_pcnt;            // virtual facets per candidate
    DevBuf<int64_t> db_poff, db_pblk;   // their offsets and scan scratch
    DevBuf<int64_t> db_txoff;           // first virtual facet of each TX [P + 1]
    DevBuf<unsigned char> db_rows;      // FP32 evaluation: slow-time rows and geometry
    DevBuf<double2> db_part;            // FP32 evaluation: the chunks' partial sums
    int64_t db_n = 0;
    DevBuf<uint32_t> mkeys, skeys;      // batched sort scratch
    int tpi_override = 0;               // synthesis tiles per item (autotuner), 0 = default
    int layout_S = 0;                   // synthesis samples per lane request, 0 = default
    uint64_t version = 1;               // bumped by every change of meshes/scene/radar/layout
    bool graph = false;                 // replay frames as CUDA graphs
    struct FrameGraph {
        cudaGraph_t graph = nullptr;
        cudaGraphExec_t exec = nullptr;
        cudaGraphNode_t t0_node = nullptr;
        cudaKernelNodeParams t0_params{};
        int t0_arg = 0, n_args = 0;
        uint64_t version = 0;
        int path = -1, dtype = -1;
        void *adc = nullptr;
        cudaStream_t stream = nullptr;
        double t0 = 0.0;
        int launches = 0, chunks = 0;
        void release()
        {
            if (exec) cudaGraphExecDestroy(exec);
            if (graph) cudaGraphDestroy(graph);
            exec = nullptr;
            graph = nullptr;
            t0_node = nullptr;
        }
    } fg;

    // stage timing: fixed events + the kinematics and synthesis pairs
    bool timing = false;
    std::vector<cudaEvent_t> ev;        // 0 start, 1 facets, 2 bvh, 3 vis, 4 end, 5/6 rdm,
                                        // 7/8 detect
    std::vector<cudaEvent_t> ev_kin;    // before / after the kinematics rows
    std::vector<cudaEvent_t> ev_syn;    // before / after the synthesis
    std::vector<cudaEvent_t> ev_db;     // double bounce: discovery, synthesis (pairs)
    bool timed_bounce = false;          // the last timed frame recorded ev_db
    cudaStream_t cap_stream = nullptr;  // frame-graph recording stream
    cudaStream_t side = nullptr;        // kinematics rows beside the hierarchy build
    cudaEvent_t fork_ev = nullptr, join_ev = nullptr;
    int chunks = 0;
    int path = 0;
    bool have_rdm_timing = false;
    bool have_detect_timing = false;
    int32_t detect_launches = 0;
    int32_t *count_host = nullptr;      // pinned readback of the detection count
    bool timed_frame = false;           // the last frame recorded its events
    int32_t frame_launches = 0, rdm_launches = 0;

    ~bart_ctx()
    {
        for (cudaEvent_t e : ev) cudaEventDestroy(e);
        for (cudaEvent_t e : ev_kin) cudaEventDestroy(e);
        for (cudaEvent_t e : ev_syn) cudaEventDestroy(e);
        for (cudaEvent_t e : ev_db) cudaEventDestroy(e);
        if (cap_stream) cudaStreamDestroy(cap_stream);
        if (side) cudaStreamDestroy(side);
        if (fork_ev) cudaEventDestroy(fork_ev);
        if (join_ev) cudaEventDestroy(join_ev);
        for (MeshStore *m : pool) {
            m->verts.release();
            m->tris.release();
            m->rho.release();
            delete m;
        }
        d_meshes.release(); d_insts.release(); tri64.release(); tri32.release(); c64.release();
        vel64.release(); vel32.release(); aabb.release(); fac.release(); fac_lo.release();
        bounds.release();
        ref64.release(); ref32.release();
        keys.release(); keys_tmp.release(); sort_temp.release(); vals.release();
        vals_tmp.release(); nodes.release(); parent.release(); leaf_parent.release();
        flags.release(); state.release(); blk_cnt.release(); vis_idx.release();
        vis_cnt.release(); kin.release(); kquad.release(); partial.release(); item_off.release();
        item_counter.release(); counters.release(); status.release();
        rdm_ws.release(); adc_own.release(); rdm_own.release(); noise_scratch.release();
        spec_tab.release();
        fg.release();
        det_ws.release(); adj_ws.release(); gfac.release(); d_voff.release(); d_foff.release(); d_root.release(); vstart.release();
        vcnt.release(); mkeys.release(); skeys.release();
        db_cnt.release(); db_off.release(); db_blk.release(); db_vf.release();
        db_cand.release(); db_pcnt.release(); db_poff.release(); db_pblk.release();
        db_txoff.release(); db_rows.release(); db_part.release(); db_roots.release();
        if (count_host) cudaFreeHost(count_host);
    }
};

#define BART_TRY(expr)                    \
    do {                                  \
        const int _rc = (expr);           \
        if (_rc != BART_OK) return _rc;   \
    } while (0)

#define CUDA_TRY(expr, what)                          \
    do {                                              \
        const cudaError_t _e = (expr);                \
        if (_e != cudaSuccess) return cuda_fail(_e, what); \
    } while (0)

// FFT lengths of the RDM kernels: 2^a 3^b
static bool is_fft_len(int x)
{
    if (x < 1) return false;
    while (x % 2 == 0) x /= 2;
    while (x % 3 == 0) x /= 3;
    return x == 1;
}

static RadarDev make_rd(const bart_radar &r)
{
    RadarDev d;
    std::memset(&d, 0, sizeof d);
    d.f0 = r.f0;
    d.slope = r.slope;
    d.fs = r.fs;
    d.Tc = r.Tc;
    d.M = r.M;
    d.N = r.N;
    d.P = r.P;
    d.Q = r.Q;
    d.O = r.P * r.Q;
    d.A = r.P + r.Q;
    d.intra = r.intra_chirp_motion ? 1 : 0;
    d.window = r.window;
    d.tdm = r.tdm ? 1 : 0;
    d.delay_ref = r.delay_ref ? 1 : 0;
    d.slots = d.tdm ? r.P : 1;
    d.far_field = r.far_field ? 1 : 0;
    d.eps_face = r.grazing_eps > 0.0 ? r.grazing_eps : kEpsFace;
    for (int p = 0; p < r.P; ++p)
        for (int k = 0; k < 3; ++k) d.ant[p][k] = r.tx[p][k];
    for (int q = 0; q < r.Q; ++q)
        for (int k = 0; k < 3; ++k) d.ant[r.P + q][k] = r.rx[q][k];
    return d;
}

static int ensure_events(std::vector<cudaEvent_t> &v, size_t n, bool timing = true)
{
    while (v.size() < n) {
        cudaEvent_t e;
        CUDA_TRY(cudaEventCreateWithFlags(&e, timing ? cudaEventDefault : cudaEventDisableTiming),
                 "cudaEventCreate");
        v.push_back(e);
    }
    return BART_OK;
}

static int set_device(bart_ctx *ctx)
{
    CUDA_TRY(cudaSetDevice(ctx->device), "cudaSetDevice");
    return BART_OK;
}

extern "C" {

const char *bart_last_error(void) { return g_err.c_str(); }

const char *bart_version(void) { return "bartsim 0.2 (sm_103a)"; }

int bart_inject_alloc_failure(int32_t nth)
{
    g_err.clear();
    if (nth < 0) return fail(BART_EINVAL, "bart_inject_alloc_failure: nth=%d", nth);
    g_fail_countdown.store(nth);
    return BART_OK;
}

int bart_selftest_wait_timeout(bart_ctx *ctx, int32_t polls)
{
    g_err.clear();
    if (!ctx) return fail(BART_EINVAL, "bart_selftest_wait_timeout: ctx is NULL");
    if (polls < 1 || polls > (1 << 20))
        return fail(BART_EINVAL, "bart_selftest_wait_timeout: polls=%d outside [1, 2^20]", polls);
    BART_TRY(set_device(ctx));
    launch_wait_selftest(polls, ctx->status.p, ctx->stream);
    CUDA_TRY(cudaGetLastError(), "wait self-test launch");
    return BART_OK;
}

int bart_create(bart_ctx **out, int device)
{
    g_err.clear();
    if (!out) return fail(BART_EINVAL, "bart_create: out is NULL");
    *out = nullptr;
    int n = 0;
    CUDA_TRY(cudaGetDeviceCount(&n), "cudaGetDeviceCount");
    if (device < 0 || device >= n)
        return fail(BART_EINVAL, "bart_create: device %d out of range [0, %d)", device, n);
    CUDA_TRY(cudaSetDevice(device), "cudaSetDevice");
    bart_ctx *c = new (std::nothrow) bart_ctx();
    if (!c) return fail(BART_ENOMEM, "bart_create: host allocation failed");
    c->device = device;
    int rc = c->counters.ensure(5, "counters");
    if (rc == BART_OK) rc = c->status.ensure(1, "status");
    if (rc == BART_OK) rc = c->bounds.ensure(6, "bounds");
    if (rc != BART_OK) {
        delete c;
        return rc;
    }
    cudaError_t e = cudaMemset(c->status.p, 0, sizeof(int));
    if (e != cudaSuccess) {
        delete c;
        return cuda_fail(e, "cudaMemset");
    }
    *out = c;
    return BART_OK;
}

void bart_destroy(bart_ctx *ctx)
{
    if (!ctx) return;
    cudaSetDevice(ctx->device);
    if (ctx->stream) cudaStreamSynchronize(ctx->stream);
    else cudaDeviceSynchronize();
    delete ctx;
}

int bart_set_stream(bart_ctx *ctx, void *stream)
{
    g_err.clear();
    if (!ctx) return fail(BART_EINVAL, "bart_set_stream: ctx is NULL");
    ctx->stream = reinterpret_cast<cudaStream_t>(stream);
    return BART_OK;
}

int bart_mesh_upload(bart_ctx *ctx, const double *verts, int64_t nv, const int32_t *tris,
                     int64_t nf, const float *rho, uint32_t flags, int32_t *mesh_id)
{
    g_err.clear();
    if (!ctx || !verts || !tris || !mesh_id) return fail(BART_EINVAL, "bart_mesh_upload: NULL argument");
    if (flags & ~BART_MESH_TWO_SIDED)
        return fail(BART_EINVAL, "bart_mesh_upload: unknown flags 0x%x", flags);
    if (nv < 3 || nf < 1) return fail(BART_EINVAL, "bart_mesh_upload: nv=%lld nf=%lld", (long long)nv, (long long)nf);
    if (nf > (int64_t)1 << 30) return fail(BART_EINVAL, "bart_mesh_upload: nf too large");
    for (int64_t i = 0; i < 3 * nf; ++i)
        if (tris[i] < 0 || tris[i] >= nv)
            return fail(BART_EINVAL, "bart_mesh_upload: tris[%lld]=%d out of [0,%lld)",
                        (long long)i, tris[i], (long long)nv);
    for (int64_t i = 0; i < 3 * nv; ++i)
        if (!std::isfinite(verts[i]))
            return fail(BART_EINVAL, "bart_mesh_upload: verts[%lld] is not finite", (long long)i);
    if (rho)
        for (int64_t i = 0; i < nf; ++i)
            if (!std::isfinite(rho[i]))
                return fail(BART_EINVAL, "bart_mesh_upload: rho[%lld] is not finite", (long long)i);
    BART_TRY(set_device(ctx));
    if (ctx->n_meshes == (int)ctx->pool.size()) {
        MeshStore *m = new (std::nothrow) MeshStore();
        if (!m) return fail(BART_ENOMEM, "bart_mesh_upload: host allocation failed");
        ctx->pool.push_back(m);
    }
    MeshStore *m = ctx->pool[ctx->n_meshes];
    BART_TRY(m->verts.ensure((size_t)(3 * nv), "mesh vertices"));
    BART_TRY(m->tris.ensure((size_t)(3 * nf), "mesh triangles"));
    BART_TRY(m->rho.ensure((size_t)nf, "mesh reflectivity"));
    CUDA_TRY(cudaMemcpyAsync(m->verts.p, verts, (size_t)(3 * nv) * sizeof(double),
                             cudaMemcpyHostToDevice, ctx->stream), "mesh vertex copy");
    CUDA_TRY(cudaMemcpyAsync(m->tris.p, tris, (size_t)(3 * nf) * sizeof(int32_t),
                             cudaMemcpyHostToDevice, ctx->stream), "mesh index copy");
    if (rho) {
        CUDA_TRY(cudaMemcpyAsync(m->rho.p, rho, (size_t)nf * sizeof(float),
                                 cudaMemcpyHostToDevice, ctx->stream), "mesh rho copy");
    }
    CUDA_TRY(cudaStreamSynchronize(ctx->stream), "cudaStreamSynchronize");
    m->has_rho = rho != nullptr;
    m->flags = flags;
    m->nv = nv;
    m->nf = nf;
    *mesh_id = ctx->n_meshes++;
    ctx->tables_dirty = true;
    ++ctx->version;
    return BART_OK;
}

int bart_mesh_update(bart_ctx *ctx, int32_t mesh_id, const double *verts, const float *rho)
{
    g_err.clear();
    if (!ctx || !verts) return fail(BART_EINVAL, "bart_mesh_update: NULL argument");
    if (mesh_id < 0 || mesh_id >= ctx->n_meshes)
        return fail(BART_EINVAL, "bart_mesh_update: mesh %d (have %d)", mesh_id, ctx->n_meshes);
    BART_TRY(set_device(ctx));
    MeshStore *m = ctx->pool[mesh_id];
    CUDA_TRY(cudaMemcpyAsync(m->verts.p, verts, (size_t)(3 * m->nv) * sizeof(double),
                             cudaMemcpyDeviceToDevice, ctx->stream), "mesh vertex update");
    if (rho) {
        CUDA_TRY(cudaMemcpyAsync(m->rho.p, rho, (size_t)m->nf * sizeof(float),
                                 cudaMemcpyDeviceToDevice, ctx->stream), "mesh rho update");
        if (!m->has_rho) {
            m->has_rho = true;
            ctx->tables_dirty = true;
            ++ctx->version;
        }
    }
    return BART_OK;
}

int bart_mesh_clear(bart_ctx *ctx)
{
    g_err.clear();
    if (!ctx) return fail(BART_EINVAL, "bart_mesh_clear: ctx is NULL");
    ctx->n_meshes = 0;
    ctx->insts.clear();
    ctx->have_frame = false;
    ctx->tables_dirty = true;
    ++ctx->version;
    return BART_OK;
}

int bart_scene_set(bart_ctx *ctx, const bart_instance *inst, int32_t n)
{
    g_err.clear();
    if (!ctx || (n > 0 && !inst)) return fail(BART_EINVAL, "bart_scene_set: NULL argument");
    if (n < 0) return fail(BART_EINVAL, "bart_scene_set: n=%d", n);
    for (int i = 0; i < n; ++i) {
        if (inst[i].mesh_id < 0 || inst[i].mesh_id >= ctx->n_meshes)
            return fail(BART_EINVAL, "bart_scene_set: instance %d names mesh %d (have %d)", i,
                        inst[i].mesh_id, ctx->n_meshes);
        for (int k = 0; k < 3; ++k)
            if (!std::isfinite(inst[i].pos[k]) || !std::isfinite(inst[i].vel[k]))
                return fail(BART_EINVAL, "bart_scene_set: instance %d has a non-finite pose", i);
        for (int k = 0; k < 9; ++k)
            if (!std::isfinite(inst[i].rot[k]))
                return fail(BART_EINVAL, "bart_scene_set: instance %d has a non-finite rotation", i);
        if (!std::isfinite(inst[i].rho_scale))
            return fail(BART_EINVAL, "bart_scene_set: instance %d has a non-finite rho_scale", i);
    }
    ctx->insts.assign(inst, inst + n);
    ctx->scene_first.clear();
    ctx->n_scenes = 1;
    ctx->tables_dirty = true;
    ++ctx->version;
    return BART_OK;
}

int bart_scene_partition(bart_ctx *ctx, const int32_t *first, int32_t n_scenes)
{
    g_err.clear();
    if (!ctx || !first) return fail(BART_EINVAL, "bart_scene_partition: NULL argument");
    const int I = (int)ctx->insts.size();
    if (I == 0) return fail(BART_ESTATE, "bart_scene_partition: no instances set");
    if (n_scenes < 1 || n_scenes > I)
        return fail(BART_EINVAL, "bart_scene_partition: n_scenes=%d with %d instances", n_scenes, I);
    if (first[0] != 0 || first[n_scenes] != I)
        return fail(BART_EINVAL, "bart_scene_partition: offsets must run from 0 to %d", I);
    for (int b = 0; b < n_scenes; ++b)
        if (first[b + 1] <= first[b])
            return fail(BART_EINVAL, "bart_scene_partition: scene %d is empty or offsets decrease", b);
    ctx->scene_first.assign(first, first + n_scenes + 1);
    ctx->n_scenes = n_scenes;
    ctx->tables_dirty = true;
    ++ctx->version;
    return BART_OK;
}

int bart_scene_facets(bart_ctx *ctx, int64_t *n_facets)
{
    g_err.clear();
    if (!ctx || !n_facets) return fail(BART_EINVAL, "bart_scene_facets: NULL argument");
    int64_t F = 0;
    for (const bart_instance &i : ctx->insts) F += ctx->pool[i.mesh_id]->nf;
    *n_facets = F;
    return BART_OK;
}

int bart_get_dims(bart_ctx *ctx, bart_dims *out)
{
    g_err.clear();
    if (!ctx || !out) return fail(BART_EINVAL, "bart_get_dims: NULL argument");
    std::memset(out, 0, sizeof *out);
    out->device = ctx->device;
    out->n_scenes = ctx->n_scenes;
    out->n_meshes = ctx->n_meshes;
    if (ctx->have_radar) {
        out->have_radar = 1;
        out->O = ctx->radar.P * ctx->radar.Q;
        out->N = ctx->radar.N;
        out->M = ctx->radar.M;
        out->A = ctx->radar.P + ctx->radar.Q;
    }
    for (const bart_instance &i : ctx->insts) {
        out->n_facets += ctx->pool[i.mesh_id]->nf;
        out->n_inst_verts += ctx->pool[i.mesh_id]->nv;
    }
    if (ctx->have_frame) {
        out->vis_antennas = ctx->frame_A;
        out->vis_facets = ctx->frame_F;
    }
    return BART_OK;
}

int bart_mesh_dims(bart_ctx *ctx, int32_t mesh_id, int64_t *nv, int64_t *nf)
{
    g_err.clear();
    if (!ctx || !nv || !nf) return fail(BART_EINVAL, "bart_mesh_dims: NULL argument");
    if (mesh_id < 0 || mesh_id >= ctx->n_meshes)
        return fail(BART_EINVAL, "bart_mesh_dims: mesh %d (have %d)", mesh_id, ctx->n_meshes);
    *nv = ctx->pool[mesh_id]->nv;
    *nf = ctx->pool[mesh_id]->nf;
    return BART_OK;
}

int bart_radar_set(bart_ctx *ctx, const bart_radar *r)
{
    g_err.clear();
    if (!ctx || !r) return fail(BART_EINVAL, "bart_radar_set: NULL argument");
    if (r->M < 32 || r->M > 1024 || r->M % 32 != 0)
        return fail(BART_EINVAL, "bart_radar_set: M=%d must be a multiple of 32 in [32,1024]", r->M);
    if (r->N < 1 || r->N > 32768)
        return fail(BART_EINVAL, "bart_radar_set: N=%d out of [1,32768]", r->N);
    if (r->P < 1 || r->P > BART_MAX_TX || r->Q < 1 || r->Q > BART_MAX_RX)
        return fail(BART_EINVAL, "bart_radar_set: P=%d Q=%d out of range", r->P, r->Q);
    if (!(r->f0 > 0) || !(r->slope > 0) || !(r->fs > 0) || !(r->Tc > 0) ||
        !std::isfinite(r->f0) || !std::isfinite(r->slope) || !std::isfinite(r->fs) ||
        !std::isfinite(r->Tc))
        return fail(BART_EINVAL, "bart_radar_set: f0, slope, fs, Tc must be positive and finite");
    for (int a = 0; a < r->P + r->Q; ++a) {
        const double *x = a < r->P ? r->tx[a] : r->rx[a - r->P];
        if (!std::isfinite(x[0]) || !std::isfinite(x[1]) || !std::isfinite(x[2]))
            return fail(BART_EINVAL, "bart_radar_set: %s %d has a non-finite position",
                        a < r->P ? "TX" : "RX", a < r->P ? a : a - r->P);
    }
    if (r->intra_chirp_motion != 0 && r->intra_chirp_motion != 1)
        return fail(BART_EINVAL, "bart_radar_set: intra_chirp_motion=%d (0 or 1)",
                    r->intra_chirp_motion);
    if (r->Tc < (double)r->M / r->fs * (1.0 - 1e-12))
        return fail(BART_EINVAL, "bart_radar_set: Tc=%g shorter than M/fs=%g", r->Tc,
                    (double)r->M / r->fs);
    if (r->window != BART_WINDOW_HANN && r->window != BART_WINDOW_RECT)
        return fail(BART_EINVAL, "bart_radar_set: window=%d", r->window);
    if ((r->tdm != 0 && r->tdm != 1) || (r->delay_ref != 0 && r->delay_ref != 1) ||
        (r->far_field != 0 && r->far_field != 1))
        return fail(BART_EINVAL, "bart_radar_set: tdm=%d delay_ref=%d far_field=%d (0 or 1)",
                    r->tdm, r->delay_ref, r->far_field);
    if (r->far_field && r->delay_ref)
        return fail(BART_EINVAL, "bart_radar_set: far_field and delay_ref are exclusive");
    if (r->double_bounce != 0 && r->double_bounce != 1)
        return fail(BART_EINVAL, "bart_radar_set: double_bounce=%d (0 or 1)", r->double_bounce);
    if (r->double_bounce && (r->far_field || r->delay_ref))
        return fail(BART_EINVAL, "bart_radar_set: double_bounce takes the per-facet delay form "
                    "(far_field and delay_ref off)");
    if (!(r->grazing_eps == 0.0 || (r->grazing_eps > 0.0 && r->grazing_eps <= 0.1)))
        return fail(BART_EINVAL, "bart_radar_set: grazing_eps=%g (0 or in (0, 0.1])",
                    r->grazing_eps);
    ctx->radar = *r;
    ++ctx->version;
    ctx->have_radar = true;
    ctx->have_frame = false;
    return BART_OK;
}

// internal paths: the adjoint of the FP64 synthesis (bart_simulate_adjoint),
// with its vertex-form per-sample work in FP32 (bart_simulate_adjoint_mixed)
constexpr int kPathAdjoint = 100;
constexpr int kPathAdjointMixed = 101;

static int run_frame(bart_ctx *ctx, double t0, int32_t path, void *adc, int32_t dtype,
                     bart_stats *stats)
{
    if (!ctx->have_radar) return fail(BART_ESTATE, "bart_simulate_frame: radar not set");
    if (ctx->insts.empty()) return fail(BART_ESTATE, "bart_simulate_frame: scene has no instances");
    if (path != BART_PATH_FP64 && path != BART_PATH_MIXED && path != BART_PATH_SPECTRAL &&
        path != kPathAdjoint && path != kPathAdjointMixed)
        return fail(BART_EINVAL, "bart_simulate_frame: path=%d", path);
    if (path == BART_PATH_SPECTRAL &&
        (!is_fft_len(ctx->radar.M) || !spectral_supported(ctx->radar.M)))
        return fail(BART_EINVAL, "bart_simulate_frame: the spectral path needs M of the form "
                    "2^a 3^b (M=%d)", ctx->radar.M);
    if (dtype != BART_C64 && dtype != BART_C128)
        return fail(BART_EINVAL, "bart_simulate_frame: dtype=%d", dtype);
    if (!adc) return fail(BART_EINVAL, "bart_simulate_frame: adc is NULL");
    if (!std::isfinite(t0)) return fail(BART_EINVAL, "bart_simulate_frame: t0 not finite");
    BART_TRY(set_device(ctx));
    cudaStream_t s = ctx->stream;
    const RadarDev rd = make_rd(ctx->radar);

    // instance + mesh tables
    const int I = (int)ctx->insts.size();
    std::vector<MeshDesc> md(ctx->n_meshes);
    for (int i = 0; i < ctx->n_meshes; ++i) {
        MeshStore *m = ctx->pool[i];
        md[i] = MeshDesc{m->verts.p, m->tris.p, m->has_rho ? m->rho.p : nullptr, m->nf,
                         (m->flags & BART_MESH_TWO_SIDED) ? 1 : 0};
    }
    std::vector<InstDev> id(I);
    int64_t F = 0;
    for (int i = 0; i < I; ++i) {
        const bart_instance &b = ctx->insts[i];
        InstDev &d = id[i];
        d.mesh = b.mesh_id;
        d.rho_scale = b.rho_scale;
        d.off = F;
        std::memcpy(d.pos, b.pos, sizeof d.pos);
        std::memcpy(d.rot, b.rot, sizeof d.rot);
        std::memcpy(d.vel, b.vel, sizeof d.vel);
        F += ctx->pool[b.mesh_id]->nf;
    }
    if (F > ((int64_t)1 << 31) - 2) return fail(BART_EINVAL, "scene has %lld facets (max 2^31-2)", (long long)F);
    const int A = rd.A, O = rd.O;
    const int B = ctx->n_scenes;
    if ((int64_t)B * O > 65535)
        return fail(BART_EINVAL, "bart_simulate_frame: %d scenes x %d channels exceed 65535", B, O);
    std::vector<int64_t> foff(B + 1), scene_F(B);
    for (int b = 0; b < B; ++b) foff[b] = B > 1 ? id[ctx->scene_first[b]].off : 0;
    foff[B] = F;
    for (int b = 0; b < B; ++b) scene_F[b] = foff[b + 1] - foff[b];

    if (md.size() > ctx->d_meshes.cap || (size_t)I > ctx->d_insts.cap ||
        (size_t)(3 * I) > ctx->vel64.cap)
        ctx->tables_dirty = true;
    BART_TRY(ctx->d_meshes.ensure(md.size(), "mesh table"));
    BART_TRY(ctx->d_insts.ensure(I, "instance table"));
    BART_TRY(ctx->tri64.ensure(9 * F, "facet vertices"));
    BART_TRY(ctx->tri32.ensure(12 * F, "facet vertices (f32)"));
    BART_TRY(ctx->c64.ensure(3 * F, "facet centroids"));
    BART_TRY(ctx->vel64.ensure(3 * I, "instance velocities"));
    BART_TRY(ctx->vel32.ensure(4 * I, "instance velocities (f32)"));
    BART_TRY(ctx->ref64.ensure(3 * I, "instance origins"));
    BART_TRY(ctx->ref32.ensure(4 * I, "instance origins (f32)"));
    BART_TRY(ctx->aabb.ensure(6 * F, "facet boxes"));
    BART_TRY(ctx->fac.ensure(F, "facet records"));
    BART_TRY(ctx->fac_lo.ensure(12 * F, "facet record residues"));
    BART_TRY(ctx->keys.ensure(F, "morton keys"));
    BART_TRY(ctx->keys_tmp.ensure(F, "morton keys"));
    BART_TRY(ctx->vals.ensure(F, "sort values"));
    BART_TRY(ctx->vals_tmp.ensure(F, "sort values"));
    BART_TRY(ctx->sort_temp.ensure(radix_sort_temp_words(F), "sort histogram"));
    BART_TRY(ctx->nodes.ensure(F > 1 ? F - 1 : 1, "bvh nodes"));
    BART_TRY(ctx->parent.ensure(F > 1 ? F - 1 : 1, "bvh parents"));
    BART_TRY(ctx->leaf_parent.ensure(F, "bvh leaf parents"));
    BART_TRY(ctx->flags.ensure(F > 1 ? F - 1 : 1, "bvh refit flags"));
    BART_TRY(ctx->state.ensure((size_t)A * F, "visibility states"));
    BART_TRY(ctx->blk_cnt.ensure(compact_blk_words(F, O + A), "compaction counts"));
    BART_TRY(ctx->vis_idx.ensure((size_t)(O + A) * F, "lit facet lists"));
    BART_TRY(ctx->vis_cnt.ensure(O + A, "lit facet counts"));
    if (path == kPathAdjoint || path == kPathAdjointMixed) {
        BART_TRY(ctx->gfac.ensure((size_t)10 * F, "facet gradients"));
        BART_TRY(ctx->d_voff.ensure((size_t)I, "instance vertex offsets"));
        std::vector<int64_t> voff(I);
        int64_t nvtot = 0;
        for (int i = 0; i < I; ++i) {
            voff[i] = nvtot;
            nvtot += ctx->pool[ctx->insts[i].mesh_id]->nv;
        }
        ctx->adj_vwords = 3 * nvtot;
        CUDA_TRY(cudaMemcpyAsync(ctx->d_voff.p, voff.data(), I * sizeof(int64_t),
                                 cudaMemcpyHostToDevice, s), "vertex offset copy");
    }
    const bool bounce = ctx->radar.double_bounce != 0;
    if (bounce && (B > 1 || path == kPathAdjoint || path == kPathAdjointMixed))
        return fail(BART_EINVAL, "double_bounce: one scene per frame and no adjoint");
    if (bounce) {
        const int64_t items = (int64_t)rd.P * F * bounce_subtrees(rd, F);
        BART_TRY(ctx->db_roots.ensure(8, "double-bounce subtree roots"));
        BART_TRY(ctx->db_cnt.ensure((size_t)items, "double-bounce counts"));
        BART_TRY(ctx->db_off.ensure((size_t)items, "double-bounce offsets"));
        BART_TRY(ctx->db_blk.ensure((size_t)bounce_scan_words(items), "double-bounce scan"));
    }
    if (B > 1) {
        BART_TRY(ctx->d_foff.ensure(B + 1, "scene facet offsets"));
        BART_TRY(ctx->d_root.ensure(B, "scene roots"));
        BART_TRY(ctx->vstart.ensure((size_t)B * O, "scene list starts"));
        BART_TRY(ctx->vcnt.ensure((size_t)B * O, "scene list counts"));
        BART_TRY(ctx->mkeys.ensure(F, "morton keys by facet"));
        BART_TRY(ctx->skeys.ensure(F, "scene keys"));
    }

    if (ctx->tables_dirty) {
        // pageable sources: each copy is staged before the call returns
        CUDA_TRY(cudaMemcpyAsync(ctx->d_meshes.p, md.data(), md.size() * sizeof(MeshDesc),
                                 cudaMemcpyHostToDevice, s), "mesh table copy");
        CUDA_TRY(cudaMemcpyAsync(ctx->d_insts.p, id.data(), (size_t)I * sizeof(InstDev),
                                 cudaMemcpyHostToDevice, s), "instance table copy");
        std::vector<double> v(3 * I);
        for (int i = 0; i < I; ++i)
            for (int k = 0; k < 3; ++k) v[3 * i + k] = ctx->insts[i].vel[k];
        CUDA_TRY(cudaMemcpyAsync(ctx->vel64.p, v.data(), v.size() * sizeof(double),
                                 cudaMemcpyHostToDevice, s), "velocity copy");
        if (B > 1)
            CUDA_TRY(cudaMemcpyAsync(ctx->d_foff.p, foff.data(), (B + 1) * sizeof(int64_t),
                                     cudaMemcpyHostToDevice, s), "scene offset copy");
        ctx->tables_dirty = false;
    }
    // sizes and buffers of the synthesis (before any capture: no allocation
    // may happen while a frame graph is being recorded)
    const int tpi = ctx->tpi_override > 0
                        ? ctx->tpi_override
                        : synth_tiles_per_item(*std::max_element(scene_F.begin(), scene_F.end()));
    int64_t max_items = 0;
    const bool mixed_rows = path == BART_PATH_MIXED || path == BART_PATH_SPECTRAL ||
                            path == kPathAdjointMixed;
    if (path == BART_PATH_SPECTRAL && ctx->spec_M != rd.M) {
        std::vector<float> tab(2 * (size_t)rd.M);
        spectral_tables(rd.M, tab.data());
        BART_TRY(ctx->spec_tab.ensure(tab.size(), "spectral kernel tables"));
        CUDA_TRY(cudaMemcpyAsync(ctx->spec_tab.p, tab.data(), tab.size() * sizeof(float),
                                 cudaMemcpyHostToDevice, s), "spectral table copy");
        CUDA_TRY(cudaStreamSynchronize(s), "cudaStreamSynchronize");
        ctx->spec_M = rd.M;
    }
    if (mixed_rows) {
        // kinematics: Taylor rows of R(t) per antenna and facet (one launch,
        // evaluated per record inside the synthesis)
        BART_TRY(ctx->kin.ensure((size_t)A * F * kKinRowWords, "kinematics rows"));
        BART_TRY(ctx->kquad.ensure((size_t)A * F * kKinQuadWords, "kinematics quadratics"));
        if (path == BART_PATH_MIXED) {
            BART_TRY(ctx->partial.ensure((size_t)synth_partial_words(scene_F.data(), B, rd, rd.N,
                                                                     tpi, ctx->layout_S),
                                         "synthesis partials"));
            max_items = synth_max_items(scene_F.data(), B, rd, rd.N, tpi, ctx->layout_S);
            BART_TRY(ctx->item_off.ensure((size_t)B * O + 1, "synthesis item table"));
            BART_TRY(ctx->item_counter.ensure(1, "synthesis item counter"));
        }
        if (!ctx->side) {
            CUDA_TRY(cudaStreamCreateWithFlags(&ctx->side, cudaStreamNonBlocking),
                     "cudaStreamCreateWithFlags");
            CUDA_TRY(cudaEventCreateWithFlags(&ctx->fork_ev, cudaEventDisableTiming),
                     "cudaEventCreateWithFlags");
            CUDA_TRY(cudaEventCreateWithFlags(&ctx->join_ev, cudaEventDisableTiming),
                     "cudaEventCreateWithFlags");
        }
        if (ctx->timing) {
            BART_TRY(ensure_events(ctx->ev_kin, 2));
            BART_TRY(ensure_events(ctx->ev_syn, 2));
        }
    }
    // the FP64 path splits each row's facet list over several warps when the
    // rows alone would not fill the GPU; their partial sums need scratch
    int fp64_chunks = 1;
    if (path == BART_PATH_FP64) {
        fp64_chunks = synth_fp64_chunks(rd, B * O, F);
        if (fp64_chunks > 1)
            BART_TRY(ctx->partial.ensure((size_t)fp64_chunks * B * O * rd.N * rd.M * 2,
                                         "FP64 synthesis partials"));
    }
    if (ctx->timing) BART_TRY(ensure_events(ctx->ev, 7));
    if (ctx->timing && bounce) BART_TRY(ensure_events(ctx->ev_db, 4));

    // every launch of the frame, on the caller's stream (the mixed path's
    // kinematics rows on a second stream, forked after the world facets and
    // joined before the synthesis): run directly, or recorded into a frame graph
    auto enqueue = [&](double t0v, bool tm, cudaStream_t s) -> int {
        CUDA_TRY(cudaMemsetAsync(ctx->counters.p, 0, 5 * sizeof(unsigned long long), s), "memset");
        if (tm) CUDA_TRY(cudaEventRecord(ctx->ev[0], s), "cudaEventRecord");
        int launches = 0;

        // 1. world facets at t0
        Stages nv;
        nv.next("bart facets");
        launch_build_facets(ctx->d_meshes.p, ctx->d_insts.p, I, F, t0v, ctx->tri64.p, ctx->tri32.p,
                            ctx->c64.p, ctx->fac.p, ctx->aabb.p, ctx->vel32.p, ctx->bounds.p,
                            ctx->ref64.p, ctx->ref32.p, ctx->fac_lo.p, s);
        launches += 1;
        if (tm) CUDA_TRY(cudaEventRecord(ctx->ev[1], s), "cudaEventRecord");
        // the mixed and spectral paths' kinematics rows need only the world
        // facets: they run on a second stream beside the hierarchy build and
        // visibility
        if (mixed_rows) {
            nv.next("bart kinematics rows");
            CUDA_TRY(cudaEventRecord(ctx->fork_ev, s), "cudaEventRecord");
            CUDA_TRY(cudaStreamWaitEvent(ctx->side, ctx->fork_ev, 0), "cudaStreamWaitEvent");
            if (tm) CUDA_TRY(cudaEventRecord(ctx->ev_kin[0], ctx->side), "cudaEventRecord");
            launch_kin_coef(ctx->c64.p, ctx->fac.p, ctx->vel64.p, ctx->ref64.p, F, rd, ctx->kin.p,
                            ctx->kquad.p, ctx->side);
            if (tm) CUDA_TRY(cudaEventRecord(ctx->ev_kin[1], ctx->side), "cudaEventRecord");
            CUDA_TRY(cudaEventRecord(ctx->join_ev, ctx->side), "cudaEventRecord");
        }
        // 2. LBVH (batched scenes: one hierarchy with a subtree per scene)
        SceneSplit split;
        nv.next("bart bvh");
        if (B > 1) {
            launch_lbvh_batched(ctx->fac.p, F, ctx->bounds.p, ctx->d_foff.p, B, ctx->keys.p,
                                ctx->vals.p, ctx->keys_tmp.p, ctx->vals_tmp.p, ctx->sort_temp.p,
                                ctx->mkeys.p, ctx->skeys.p, ctx->nodes.p, ctx->parent.p,
                                ctx->leaf_parent.p, ctx->d_root.p, s);
            launches += lbvh_batched_launches(B);
            split.B = B;
            split.foff = ctx->d_foff.p;
            split.root = ctx->d_root.p;
        } else {
            launch_morton(ctx->fac.p, F, ctx->bounds.p, ctx->keys.p, ctx->vals.p, s);
            radix_sort_pairs(ctx->keys.p, ctx->vals.p, ctx->keys_tmp.p, ctx->vals_tmp.p,
                             ctx->sort_temp.p, F, 30, s);
            launch_lbvh_build(ctx->keys.p, ctx->vals.p, F, ctx->nodes.p, ctx->parent.p,
                              ctx->leaf_parent.p, s);
            launches += 1 + 3 * 4 + (F >= 2 ? 1 : 0);
        }
        launch_lbvh_refit(ctx->vals.p, ctx->aabb.p, F, ctx->nodes.p, ctx->parent.p,
                          ctx->leaf_parent.p, ctx->flags.p, s);
        launches += F >= 2 ? 1 : 0;
        if (tm) CUDA_TRY(cudaEventRecord(ctx->ev[2], s), "cudaEventRecord");
        // 3. visibility + per-channel lit lists (+ their per-scene ranges)
        nv.next("bart visibility");
        launch_visibility(ctx->tri64.p, ctx->tri32.p, ctx->c64.p, ctx->fac.p, ctx->ref64.p,
                          ctx->nodes.p,
                          F >= 2 ? ctx->vals.p : nullptr, F, rd, split, ctx->state.p,
                          ctx->counters.p + 3, ctx->status.p, s);
        launch_compact(ctx->state.p, F, rd, ctx->blk_cnt.p, ctx->vis_idx.p, ctx->vis_cnt.p, s);
        launches += 1 + 3;
        if (B > 1) {
            launch_scene_lists(ctx->vis_idx.p, ctx->vis_cnt.p, F, O, ctx->d_foff.p, B, ctx->vstart.p,
                               ctx->vcnt.p, s);
            launches += 1;
        }
        // 3b. double-bounce virtual facets, in two passes, each a count, a
        // scan, a host read of the total (frame graphs are off with double
        // bounce), an allocation and a fill: the candidates (a, b) of each
        // (TX, lit facet a), then each candidate's virtual facets
        if (bounce) {
            nv.next("bart double bounce");
            const int NS = bounce_subtrees(rd, F);
            const int64_t items = (int64_t)rd.P * F * NS;
            const int64_t tw = bounce_scan_words(items);
            if (tm) CUDA_TRY(cudaEventRecord(ctx->ev_db[0], s), "cudaEventRecord");
            launch_bounce_roots(ctx->nodes.p, F, NS, ctx->db_roots.p, s);
            launch_bounce_candidates(false, ctx->tri64.p, ctx->fac.p, ctx->vel64.p, ctx->nodes.p,
                                     ctx->state.p, ctx->vis_idx.p, ctx->vis_cnt.p, F, rd, NS,
                                     ctx->db_roots.p, ctx->db_cnt.p, nullptr, nullptr,
                                     ctx->status.p, s);
            launch_bounce_scan(ctx->db_cnt.p, items, ctx->db_off.p, ctx->db_blk.p, s);
            int64_t ncand = 0;
            CUDA_TRY(cudaMemcpyAsync(&ncand, ctx->db_blk.p + tw - 1, sizeof ncand,
                                     cudaMemcpyDeviceToHost, s), "double-bounce count copy");
            CUDA_TRY(cudaStreamSynchronize(s), "cudaStreamSynchronize");
            const int64_t pw = bounce_scan_words(ncand);
            BART_TRY(ctx->db_cand.ensure((size_t)std::max<int64_t>(ncand, 1), "double-bounce candidates"));
            BART_TRY(ctx->db_pcnt.ensure((size_t)std::max<int64_t>(ncand, 1), "double-bounce piece counts"));
            BART_TRY(ctx->db_poff.ensure((size_t)std::max<int64_t>(ncand, 1), "double-bounce piece offsets"));
            BART_TRY(ctx->db_pblk.ensure((size_t)pw, "double-bounce scan"));
            BART_TRY(ctx->db_txoff.ensure((size_t)rd.P + 1, "double-bounce TX offsets"));
            if (ncand > 0) {
                launch_bounce_candidates(true, ctx->tri64.p, ctx->fac.p, ctx->vel64.p,
                                         ctx->nodes.p, ctx->state.p, ctx->vis_idx.p,
                                         ctx->vis_cnt.p, F, rd, NS, ctx->db_roots.p, nullptr,
                                         ctx->db_off.p, ctx->db_cand.p, ctx->status.p, s);
                launch_bounce_pairs(false, ctx->tri64.p, ctx->tri32.p, ctx->fac.p, ctx->vel64.p, ctx->nodes.p,
                                    ctx->state.p, ctx->db_cand.p, ncand, F, rd, ctx->db_pcnt.p,
                                    nullptr, nullptr, ctx->status.p, s);
            }
            launch_bounce_scan(ctx->db_pcnt.p, ncand, ctx->db_poff.p, ctx->db_pblk.p, s);
            int64_t total = 0;
            CUDA_TRY(cudaMemcpyAsync(&total, ctx->db_pblk.p + pw - 1, sizeof total,
                                     cudaMemcpyDeviceToHost, s), "double-bounce count copy");
            CUDA_TRY(cudaStreamSynchronize(s), "cudaStreamSynchronize");
            ctx->db_n = total;
            launches += 5 + (ncand > 0 ? 2 : 0) + (ncand > 0 ? 3 : 1);
            if (total > 0) {
                BART_TRY(ctx->db_vf.ensure((size_t)total, "double-bounce virtual facets"));
                launch_bounce_pairs(true, ctx->tri64.p, ctx->tri32.p, ctx->fac.p, ctx->vel64.p, ctx->nodes.p,
                                    ctx->state.p, ctx->db_cand.p, ncand, F, rd, ctx->db_pcnt.p,
                                    ctx->db_poff.p, ctx->db_vf.p, ctx->status.p, s);
                launches += 1;
                if (path != BART_PATH_FP64) {
                    BART_TRY(ctx->db_rows.ensure((size_t)(total * (bounce_row_bytes(rd) +
                                                                   bounce_geo_bytes())),
                                                 "double-bounce rows"));
                    const int nch = bounce_synth_chunks(rd);
                    if (nch > 1)
                        BART_TRY(ctx->db_part.ensure((size_t)nch * O * rd.N * rd.M,
                                                     "double-bounce partial sums"));
                    launch_bounce_rows(ctx->db_vf.p, total, ctx->fac.p, ctx->vel64.p, rd,
                                       ctx->db_rows.p + total * bounce_geo_bytes(),
                                       ctx->db_rows.p, s);
                    launches += 1;
                }
            }
            launch_bounce_tx_offsets(ctx->db_off.p, ctx->db_blk.p + tw - 1, ctx->db_poff.p,
                                     ctx->db_pblk.p + pw - 1, F, rd.P, NS, ctx->db_txoff.p, s);
            launches += 1;
            if (tm) CUDA_TRY(cudaEventRecord(ctx->ev_db[1], s), "cudaEventRecord");
        } else {
            ctx->db_n = 0;
        }
        if (tm) CUDA_TRY(cudaEventRecord(ctx->ev[3], s), "cudaEventRecord");
        // 4. synthesis
        nv.next("bart synthesis");
        SynthArgs a;
        a.fac = ctx->fac.p;
        a.tri64 = ctx->tri64.p;
        a.c64 = ctx->c64.p;
        a.vel64 = ctx->vel64.p;
        a.vel32 = ctx->vel32.p;
        a.ref64 = ctx->ref64.p;
        a.ref32 = ctx->ref32.p;
        a.fac_lo = ctx->fac_lo.p;
        a.vis_idx = ctx->vis_idx.p;
        a.vis_cnt = ctx->vis_cnt.p;
        a.VO = B * O;
        a.vstart = B > 1 ? ctx->vstart.p : nullptr;
        a.vcnt = B > 1 ? ctx->vcnt.p : ctx->vis_cnt.p;
        a.F = F;
        a.kin = nullptr;
        a.kquad = nullptr;
        a.out = adc;
        a.out_c64 = dtype == BART_C64;
        a.counters = ctx->counters.p;
        a.item_off = nullptr;
        a.item_counter = nullptr;
        a.partial = nullptr;
        a.tiles_per_item = tpi;
        a.max_items = 0;
        a.layout_S = ctx->layout_S;
        a.rd = rd;
        if (path == BART_PATH_MIXED) {
            a.partial = ctx->partial.p;
            a.item_off = ctx->item_off.p;
            a.item_counter = ctx->item_counter.p;
            a.max_items = max_items;
            a.kin = ctx->kin.p;
            a.kquad = ctx->kquad.p;
            a.n0 = 0;
            a.nc = rd.N;
            CUDA_TRY(cudaStreamWaitEvent(s, ctx->join_ev, 0), "cudaStreamWaitEvent");
            if (tm) CUDA_TRY(cudaEventRecord(ctx->ev_syn[0], s), "cudaEventRecord");
            launch_synth_mixed(a, s);
            if (tm) CUDA_TRY(cudaEventRecord(ctx->ev_syn[1], s), "cudaEventRecord");
            ctx->chunks = 1;
            launches += 4;
        } else if (path == BART_PATH_SPECTRAL) {
            a.kin = ctx->kin.p;
            a.kquad = ctx->kquad.p;
            a.n0 = 0;
            a.nc = rd.N;
            CUDA_TRY(cudaStreamWaitEvent(s, ctx->join_ev, 0), "cudaStreamWaitEvent");
            if (tm) CUDA_TRY(cudaEventRecord(ctx->ev_syn[0], s), "cudaEventRecord");
            launch_synth_spectral(a, ctx->spec_tab.p, s);
            if (tm) CUDA_TRY(cudaEventRecord(ctx->ev_syn[1], s), "cudaEventRecord");
            ctx->chunks = 1;
            launches += 2;
        } else if (path == kPathAdjoint || path == kPathAdjointMixed) {
            a.n0 = 0;
            a.nc = rd.N;
            if (path == kPathAdjointMixed) {
                a.kin = ctx->kin.p;
                a.kquad = ctx->kquad.p;
                CUDA_TRY(cudaStreamWaitEvent(s, ctx->join_ev, 0), "cudaStreamWaitEvent");
            }
            if (path == kPathAdjoint)
                launch_adjoint_fp64(a, ctx->adj_grad, ctx->adj_grad_c64, ctx->gfac.p, s);
            else
                launch_adjoint_mixed(a, ctx->adj_grad, ctx->adj_grad_c64, ctx->gfac.p, s);
            launch_adjoint_scatter(ctx->gfac.p, ctx->fac.p, ctx->d_insts.p, ctx->d_meshes.p,
                                   ctx->d_voff.p, F, ctx->adj_gverts, ctx->adj_vwords,
                                   ctx->adj_grho, s);
            ctx->chunks = 1;
            launches += 2;
        } else {
            a.n0 = 0;
            a.nc = rd.N;
            a.partial = fp64_chunks > 1 ? ctx->partial.p : nullptr;
            launch_synth_fp64(a, s);
            ctx->chunks = 1;
            launches += fp64_chunks > 1 ? 2 : 1;
        }
        // 5. the double-bounce echo, added into the cube (FP64 on every path)
        if (bounce && ctx->db_n > 0) {
            nv.next("bart double-bounce synthesis");
            if (tm) CUDA_TRY(cudaEventRecord(ctx->ev_db[2], s), "cudaEventRecord");
            launch_bounce_synth(ctx->db_vf.p, ctx->db_txoff.p, ctx->fac.p, ctx->vel64.p, ctx->state.p, F, rd, adc,
                                dtype == BART_C64, path != BART_PATH_FP64,
                                ctx->db_rows.p + ctx->db_n * bounce_geo_bytes(), ctx->db_rows.p,
                                path != BART_PATH_FP64 ? bounce_synth_chunks(rd) : 1,
                                ctx->db_part.p, ctx->counters.p + 4, s);
            if (tm) CUDA_TRY(cudaEventRecord(ctx->ev_db[3], s), "cudaEventRecord");
            launches += (path != BART_PATH_FP64 && bounce_synth_chunks(rd) > 1) ? 2 : 1;
        }
        ctx->timed_bounce = tm && bounce;
        if (tm) CUDA_TRY(cudaEventRecord(ctx->ev[4], s), "cudaEventRecord");
        ctx->path = path;
        ctx->frame_launches = launches;
        ctx->have_rdm_timing = false;
        ctx->have_detect_timing = false;
        ctx->timed_frame = tm;
        return BART_OK;
    };

    const bool use_graph = ctx->graph && !stats && !ctx->timing && path != kPathAdjoint &&
                           path != kPathAdjointMixed && !bounce;
    if (use_graph) {
        bart_ctx::FrameGraph &g = ctx->fg;
        const bool hit = g.exec && g.version == ctx->version && g.path == path &&
                         g.dtype == dtype && g.adc == adc && g.stream == s;
        if (!hit) {
            g.release();
            // record on a private stream (the legacy default stream, torch's
            // usual current stream, cannot be captured); the graph is then
            // launched on the caller's stream, after everything queued there
            if (!ctx->cap_stream)
                CUDA_TRY(cudaStreamCreateWithFlags(&ctx->cap_stream, cudaStreamNonBlocking),
                         "cudaStreamCreate");
            cudaGraph_t graph = nullptr;
            CUDA_TRY(cudaStreamBeginCapture(ctx->cap_stream, cudaStreamCaptureModeRelaxed),
                     "cudaStreamBeginCapture");
            const int rc = enqueue(t0, false, ctx->cap_stream);
            const cudaError_t ce = cudaStreamEndCapture(ctx->cap_stream, &graph);
            if (rc != BART_OK || ce != cudaSuccess) {
                if (graph) cudaGraphDestroy(graph);
                cudaGetLastError();
                return rc != BART_OK ? rc : fail(BART_ECUDA, "frame graph capture: %s",
                                                 cudaGetErrorString(ce));
            }
            g.graph = graph;
            CUDA_TRY(cudaGraphInstantiate(&g.exec, graph, 0), "cudaGraphInstantiate");
            const void *fn = build_facets_kernel_fn(&g.t0_arg, &g.n_args);
            size_t nn = 0;
            CUDA_TRY(cudaGraphGetNodes(graph, nullptr, &nn), "cudaGraphGetNodes");
            std::vector<cudaGraphNode_t> nodes(nn);
            CUDA_TRY(cudaGraphGetNodes(graph, nodes.data(), &nn), "cudaGraphGetNodes");
            for (cudaGraphNode_t n : nodes) {
                cudaGraphNodeType t;
                CUDA_TRY(cudaGraphNodeGetType(n, &t), "cudaGraphNodeGetType");
                if (t != cudaGraphNodeTypeKernel) continue;
                cudaKernelNodeParams kp;
                CUDA_TRY(cudaGraphKernelNodeGetParams(n, &kp), "cudaGraphKernelNodeGetParams");
                if (kp.func == fn) {
                    g.t0_node = n;
                    g.t0_params = kp;
                    break;
                }
            }
            if (!g.t0_node) {
                g.release();
                return fail(BART_ECUDA, "frame graph: world-facet kernel node not found");
            }
            g.version = ctx->version;
            g.path = path;
            g.dtype = dtype;
            g.adc = adc;
            g.stream = s;
            g.t0 = t0;
            g.launches = ctx->frame_launches;
            g.chunks = ctx->chunks;
        } else if (t0 != g.t0) {
            // a new frame time: only the world-facet kernel's t0 argument changes
            void *args[32];
            cudaKernelNodeParams kp = g.t0_params;
            double t0_arg = t0;
            for (int k = 0; k < g.n_args && k < 32; ++k) args[k] = kp.kernelParams[k];
            args[g.t0_arg] = &t0_arg;
            kp.kernelParams = args;
            CUDA_TRY(cudaGraphExecKernelNodeSetParams(g.exec, g.t0_node, &kp),
                     "cudaGraphExecKernelNodeSetParams");
            g.t0 = t0;
        }
        CUDA_TRY(cudaGraphLaunch(g.exec, s), "cudaGraphLaunch");
        ctx->path = path;
        ctx->frame_launches = g.launches;
        ctx->chunks = g.chunks;
        ctx->have_rdm_timing = false;
        ctx->have_detect_timing = false;
        ctx->timed_frame = false;
    } else {
        BART_TRY(enqueue(t0, ctx->timing, s));
    }
    CUDA_TRY(cudaGetLastError(), "kernel launch");
    ctx->have_frame = true;
    ctx->frame_F = F;
    ctx->frame_A = A;
    ctx->frame_B = B;
    if (stats) {
        std::vector<int32_t> cnt(O);
        unsigned long long ctr[5];
        CUDA_TRY(cudaMemcpyAsync(cnt.data(), ctx->vis_cnt.p, O * sizeof(int32_t),
                                 cudaMemcpyDeviceToHost, s), "stats copy");
        CUDA_TRY(cudaMemcpyAsync(ctr, ctx->counters.p, sizeof ctr, cudaMemcpyDeviceToHost, s),
                 "stats copy");
        CUDA_TRY(cudaStreamSynchronize(s), "cudaStreamSynchronize");
        int64_t lit = 0;
        for (int o = 0; o < O; ++o) lit += cnt[o];
        stats->n_facets = F;
        stats->n_lit_pairs = lit;
        stats->n_terms = lit * (int64_t)rd.N * rd.M;
        stats->n_vertex = (int64_t)ctr[0];
        stats->n_series = (int64_t)ctr[1];
        stats->n_edge = (int64_t)ctr[2];
        stats->n_grazing = (int64_t)ctr[3];
        stats->n_bounce_facets = ctx->db_n;
        stats->n_bounce_terms = (int64_t)ctr[4] * rd.M;
    }
    return BART_OK;
}

int bart_simulate_frame(bart_ctx *ctx, double t0, int32_t path, void *adc, int32_t dtype,
                        bart_stats *stats)
{
    g_err.clear();
    if (!ctx) return fail(BART_EINVAL, "bart_simulate_frame: ctx is NULL");
    return run_frame(ctx, t0, path, adc, dtype, stats);
}

static int run_adjoint(bart_ctx *ctx, double t0, const void *grad_adc, int32_t dtype,
                       double *grad_verts, double *grad_rho, int path, const char *name)
{
    g_err.clear();
    if (!ctx || !grad_adc || !grad_verts) return fail(BART_EINVAL, "%s: NULL argument", name);
    if (dtype != BART_C64 && dtype != BART_C128)
        return fail(BART_EINVAL, "%s: dtype=%d", name, dtype);
    if (ctx->have_radar && ctx->radar.far_field)
        return fail(BART_EINVAL, "%s: not available in far-field mode", name);
    ctx->adj_grad = grad_adc;
    ctx->adj_grad_c64 = dtype == BART_C64;
    ctx->adj_gverts = grad_verts;
    ctx->adj_grho = grad_rho;
    // the synthesis output pointer is unused on this path
    const int rc = run_frame(ctx, t0, path, const_cast<void *>(grad_adc), dtype, nullptr);
    ctx->adj_grad = nullptr;
    ctx->adj_gverts = ctx->adj_grho = nullptr;
    return rc;
}

int bart_simulate_adjoint(bart_ctx *ctx, double t0, const void *grad_adc, int32_t dtype,
                          double *grad_verts, double *grad_rho)
{
    return run_adjoint(ctx, t0, grad_adc, dtype, grad_verts, grad_rho, kPathAdjoint,
                       "bart_simulate_adjoint");
}

int bart_simulate_adjoint_mixed(bart_ctx *ctx, double t0, const void *grad_adc, int32_t dtype,
                                double *grad_verts, double *grad_rho)
{
    return run_adjoint(ctx, t0, grad_adc, dtype, grad_verts, grad_rho, kPathAdjointMixed,
                       "bart_simulate_adjoint_mixed");
}

int bart_set_graph(bart_ctx *ctx, int32_t enable)
{
    g_err.clear();
    if (!ctx) return fail(BART_EINVAL, "bart_set_graph: ctx is NULL");
    ctx->graph = enable != 0;
    if (!ctx->graph) {
        BART_TRY(set_device(ctx));
        if (ctx->fg.exec) CUDA_TRY(cudaStreamSynchronize(ctx->fg.stream), "cudaStreamSynchronize");
        ctx->fg.release();
    }
    return BART_OK;
}

int bart_set_synth_layout(bart_ctx *ctx, int32_t samples_per_lane, int32_t tiles_per_item)
{
    g_err.clear();
    if (!ctx) return fail(BART_EINVAL, "bart_set_synth_layout: ctx is NULL");
    if (samples_per_lane != 0 && samples_per_lane != 8 && samples_per_lane != 16 &&
        samples_per_lane != 32)
        return fail(BART_EINVAL, "bart_set_synth_layout: samples_per_lane=%d (0, 8, 16 or 32)",
                    samples_per_lane);
    if (tiles_per_item < 0 || tiles_per_item > 65536)
        return fail(BART_EINVAL, "bart_set_synth_layout: tiles_per_item=%d", tiles_per_item);
    ctx->layout_S = samples_per_lane == 16 ? 0 : samples_per_lane;
    ctx->tpi_override = tiles_per_item;
    ++ctx->version;
    return BART_OK;
}

int bart_autotune(bart_ctx *ctx, double t0, void *adc, int32_t dtype, int32_t reps,
                  bart_tune *out)
{
    g_err.clear();
    if (!ctx || !adc || !out) return fail(BART_EINVAL, "bart_autotune: NULL argument");
    if (!ctx->have_radar) return fail(BART_ESTATE, "bart_autotune: radar not set");
    if (reps < 1 || reps > 100) return fail(BART_EINVAL, "bart_autotune: reps=%d", reps);
    BART_TRY(set_device(ctx));
    const bool timing = ctx->timing, graph = ctx->graph;
    const int S0 = ctx->layout_S, T0 = ctx->tpi_override;
    ctx->timing = true;
    ctx->graph = false;
    std::memset(out, 0, sizeof *out);
    std::vector<int> Ss = {0};
    if (synth_layout_samples(ctx->radar.M, 32) == 32) Ss.push_back(32);
    if (synth_layout_samples(ctx->radar.M, 8) == 8) Ss.push_back(8);
    const int tpis[] = {8, 16, 32, 64, 128, 256, 512};
    int rc = BART_OK;
    float best = 0.f;
    for (int S : Ss) {
        for (int tpi : tpis) {
            if (out->n_trials >= BART_TUNE_MAX) break;
            ctx->layout_S = S;
            ctx->tpi_override = tpi;
            float ms_best = 0.f;
            for (int r = 0; r <= reps && rc == BART_OK; ++r) {   // r = 0 warms up
                rc = run_frame(ctx, t0, BART_PATH_MIXED, adc, dtype, nullptr);
                if (rc != BART_OK) break;
                if (cudaStreamSynchronize(ctx->stream) != cudaSuccess) {
                    cudaGetLastError();
                    rc = fail(BART_ECUDA, "bart_autotune: frame failed");
                    break;
                }
                float ms = 0.f;
                for (int c = 0; c < ctx->chunks; ++c) {
                    float e = 0.f;
                    cudaEventElapsedTime(&e, ctx->ev_syn[2 * c], ctx->ev_syn[2 * c + 1]);
                    ms += e;
                }
                if (r > 0 && (r == 1 || ms < ms_best)) ms_best = ms;
            }
            if (rc != BART_OK) break;
            const int i = out->n_trials++;
            out->samples_per_lane[i] = synth_layout_samples(ctx->radar.M, S);
            out->tiles_per_item[i] = tpi;
            out->synthesis_ms[i] = ms_best;
            if (i == 0 || ms_best < best) {
                best = ms_best;
                out->best_samples_per_lane = out->samples_per_lane[i];
                out->best_tiles_per_item = tpi;
                out->best_ms = ms_best;
            }
        }
        if (rc != BART_OK) break;
    }
    ctx->timing = timing;
    ctx->graph = graph;
    if (rc != BART_OK) {
        ctx->layout_S = S0;
        ctx->tpi_override = T0;
        ++ctx->version;
        return rc;
    }
    ctx->layout_S = out->best_samples_per_lane == 16 ? 0 : out->best_samples_per_lane;
    ctx->tpi_override = out->best_tiles_per_item;
    ++ctx->version;
    return BART_OK;
}

static int run_rdm(bart_ctx *ctx, const void *adc, int32_t dtype, float *rdm)
{
    if (!ctx->have_radar) return fail(BART_ESTATE, "bart_form_rdm: radar not set");
    if (!adc || !rdm) return fail(BART_EINVAL, "bart_form_rdm: NULL buffer");
    if (dtype != BART_C64 && dtype != BART_C128)
        return fail(BART_EINVAL, "bart_form_rdm: dtype=%d", dtype);
    if (!is_fft_len(ctx->radar.M) || !is_fft_len(ctx->radar.N) || ctx->radar.N < 2 ||
        ctx->radar.N > 1024)
        return fail(BART_EINVAL, "bart_form_rdm: the radix-2/3 FFTs need M and N of the form "
                    "2^a 3^b (M=%d, N=%d, 2 <= N <= 1024)", ctx->radar.M, ctx->radar.N);
    BART_TRY(set_device(ctx));
    const RadarDev rd = make_rd(ctx->radar);
    const int groups = ctx->n_scenes;
    if ((int64_t)groups * ctx->radar.P * ctx->radar.Q > 65535)
        return fail(BART_EINVAL, "bart_form_rdm: %d scenes x %d channels exceed 65535", groups,
                    ctx->radar.P * ctx->radar.Q);
    BART_TRY(ctx->rdm_ws.ensure((size_t)rdm_workspace_bytes(rd, dtype) * groups, "rdm workspace"));
    if (ctx->timing) {
        BART_TRY(ensure_events(ctx->ev, 7));
        CUDA_TRY(cudaEventRecord(ctx->ev[5], ctx->stream), "cudaEventRecord");
    }
    Stages nv;
    nv.next("bart rdm");
    launch_rdm(adc, dtype, rd, groups, ctx->rdm_ws.p, rdm, ctx->status.p, ctx->stream);
    CUDA_TRY(cudaGetLastError(), "rdm launch");
    if (ctx->timing) {
        CUDA_TRY(cudaEventRecord(ctx->ev[6], ctx->stream), "cudaEventRecord");
        ctx->have_rdm_timing = true;
    }
    ctx->rdm_launches = 3;
    return BART_OK;
}

int bart_form_rdm(bart_ctx *ctx, const void *adc, int32_t dtype, float *rdm)
{
    g_err.clear();
    if (!ctx) return fail(BART_EINVAL, "bart_form_rdm: ctx is NULL");
    return run_rdm(ctx, adc, dtype, rdm);
}

int bart_add_noise(bart_ctx *ctx, void *adc, int32_t dtype, double snr_db, uint64_t seed,
                   uint32_t frame)
{
    g_err.clear();
    if (!ctx || !adc) return fail(BART_EINVAL, "bart_add_noise: NULL argument");
    if (!ctx->have_radar) return fail(BART_ESTATE, "bart_add_noise: radar not set");
    if (dtype != BART_C64 && dtype != BART_C128)
        return fail(BART_EINVAL, "bart_add_noise: dtype=%d", dtype);
    if (!std::isfinite(snr_db)) return fail(BART_EINVAL, "bart_add_noise: snr_db not finite");
    BART_TRY(set_device(ctx));
    BART_TRY(ctx->noise_scratch.ensure((size_t)noise_scratch_words(), "noise scratch"));
    const int64_t n = (int64_t)ctx->radar.P * ctx->radar.Q * ctx->radar.N * ctx->radar.M;
    launch_add_noise(adc, dtype, n, snr_db, seed, frame, ctx->noise_scratch.p, ctx->stream);
    CUDA_TRY(cudaGetLastError(), "bart_add_noise launch");
    return BART_OK;
}

int bart_detect(bart_ctx *ctx, const void *adc, int32_t dtype, const bart_detect_cfg *cfg,
                float *rdm, bart_point *points, int32_t max_points, int32_t *n_points)
{
    g_err.clear();
    if (!ctx || !adc || !cfg) return fail(BART_EINVAL, "bart_detect: NULL argument");
    if (!ctx->have_radar) return fail(BART_ESTATE, "bart_detect: radar not set");
    if (dtype != BART_C64 && dtype != BART_C128)
        return fail(BART_EINVAL, "bart_detect: dtype=%d", dtype);
    const bart_radar &r = ctx->radar;
    if (!is_fft_len(r.M) || !is_fft_len(r.N) || r.N < 2 || r.N > 1024)
        return fail(BART_EINVAL, "bart_detect: the radix-2/3 FFTs need M and N of the form "
                    "2^a 3^b (M=%d, N=%d, 2 <= N <= 1024)", r.M, r.N);
    const int gr = cfg->guard_r, gd = cfg->guard_d, tr = cfg->train_r, td = cfg->train_d;
    if (gr < 0 || gd < 0 || tr < 0 || td < 0 || gr + tr > 64 || gd + td > 64)
        return fail(BART_EINVAL, "bart_detect: guard/train sizes must be in [0, 64] "
                    "(guard %d,%d train %d,%d)", gr, gd, tr, td);
    const int hr = gr + tr, hd = gd + td;
    if (2 * hr >= r.M || 2 * hd >= r.N)
        return fail(BART_EINVAL, "bart_detect: CFAR window %dx%d does not fit the %dx%d RDM",
                    2 * hr + 1, 2 * hd + 1, r.M, r.N);
    const int64_t n_train = (int64_t)(2 * hr + 1) * (2 * hd + 1) -
                            (int64_t)(2 * gr + 1) * (2 * gd + 1);
    if (n_train < 1) return fail(BART_EINVAL, "bart_detect: no training cells");
    if (!(cfg->pfa > 0.0 && cfg->pfa < 1.0))
        return fail(BART_EINVAL, "bart_detect: pfa=%g outside (0, 1)", cfg->pfa);
    if (cfg->angle_bins < 2 || cfg->angle_bins > 4096 || cfg->reserved != 0)
        return fail(BART_EINVAL, "bart_detect: angle_bins=%d outside [2, 4096] or reserved != 0",
                    cfg->angle_bins);
    if (max_points < 0 || (max_points > 0 && !points))
        return fail(BART_EINVAL, "bart_detect: max_points=%d with points=%p", max_points,
                    (const void *)points);
    BART_TRY(set_device(ctx));
    const RadarDev rd = make_rd(r);
    DetectDev dd;
    dd.guard_r = gr;
    dd.guard_d = gd;
    dd.hr = hr;
    dd.hd = hd;
    dd.n_train = (int)n_train;
    dd.alpha = (double)n_train * (std::pow(cfg->pfa, -1.0 / (double)n_train) - 1.0);
    dd.bins = cfg->angle_bins;
    const double B = r.slope * r.M / r.fs;
    dd.lam_c = kC0 / (r.f0 + 0.5 * B);
    dd.range_scale = kC0 * r.fs / (2.0 * r.slope * r.M);
    // chirp repetition of one channel: Tc, or P Tc with time-division MIMO
    dd.rate_scale = dd.lam_c / (2.0 * r.N * (r.tdm ? r.P : 1) * r.Tc);
    BART_TRY(ctx->det_ws.ensure((size_t)detect_workspace_bytes(rd, dtype, dd.bins),
                                "detection workspace"));
    DetectBufs b;
    detect_carve(ctx->det_ws.p, rd, dtype, dd.bins, &b);
    if (ctx->timing) {
        BART_TRY(ensure_events(ctx->ev, 9));
        CUDA_TRY(cudaEventRecord(ctx->ev[7], ctx->stream), "cudaEventRecord");
    }
    Stages nv;
    nv.next("bart detect");
    ctx->detect_launches = launch_detect(adc, dtype, rd, dd, b, points, max_points, ctx->stream);
    CUDA_TRY(cudaGetLastError(), "bart_detect launch");
    if (rdm)
        CUDA_TRY(cudaMemcpyAsync(rdm, b.rdm, (size_t)r.M * r.N * sizeof(float),
                                 cudaMemcpyDeviceToDevice, ctx->stream), "rdm copy");
    if (ctx->timing) {
        CUDA_TRY(cudaEventRecord(ctx->ev[8], ctx->stream), "cudaEventRecord");
        ctx->have_detect_timing = true;
    }
    if (n_points) {
        if (!ctx->count_host)
            CUDA_TRY(cudaMallocHost(&ctx->count_host, sizeof(int32_t)), "cudaMallocHost");
        CUDA_TRY(cudaMemcpyAsync(ctx->count_host, b.count, sizeof(int32_t),
                                 cudaMemcpyDeviceToHost, ctx->stream), "count copy");
        CUDA_TRY(cudaStreamSynchronize(ctx->stream), "cudaStreamSynchronize");
        *n_points = *ctx->count_host;
    }
    return BART_OK;
}

int bart_rdm_adjoint(bart_ctx *ctx, const void *adc, int32_t dtype, const float *grad_rdm,
                     void *grad_adc)
{
    g_err.clear();
    if (!ctx || !adc || !grad_rdm || !grad_adc)
        return fail(BART_EINVAL, "bart_rdm_adjoint: NULL argument");
    if (!ctx->have_radar) return fail(BART_ESTATE, "bart_rdm_adjoint: radar not set");
    if (dtype != BART_C64 && dtype != BART_C128)
        return fail(BART_EINVAL, "bart_rdm_adjoint: dtype=%d", dtype);
    const bart_radar &r = ctx->radar;
    if (!is_fft_len(r.M) || !is_fft_len(r.N) || r.N < 2 || r.N > 1024)
        return fail(BART_EINVAL, "bart_rdm_adjoint: M and N must be of the form 2^a 3^b "
                    "(M=%d, N=%d, 2 <= N <= 1024)", r.M, r.N);
    const int groups = ctx->n_scenes;
    if ((int64_t)groups * r.P * r.Q > 65535)
        return fail(BART_EINVAL, "bart_rdm_adjoint: %d scenes x %d channels exceed 65535", groups,
                    r.P * r.Q);
    BART_TRY(set_device(ctx));
    const RadarDev rd = make_rd(r);
    const size_t cube = (size_t)groups * rd.O * rd.N * rd.M * (dtype == BART_C64 ? 8 : 16);
    const size_t half = (cube + 255) & ~(size_t)255;
    BART_TRY(ctx->adj_ws.ensure(2 * half, "rdm adjoint workspace"));
    launch_rdm_adjoint(adc, dtype, grad_rdm, rd, groups, ctx->adj_ws.p, ctx->adj_ws.p + half,
                       grad_adc, ctx->stream);
    CUDA_TRY(cudaGetLastError(), "bart_rdm_adjoint launch");
    return BART_OK;
}

int bart_form_rdm_static(const void *adc, int32_t dtype, int32_t O, int32_t N, int32_t M,
                         int32_t window, float *rdm, void *stream)
{
    g_err.clear();
    if (!adc || !rdm) return fail(BART_EINVAL, "bart_form_rdm_static: NULL buffer");
    if (dtype != BART_C64 && dtype != BART_C128)
        return fail(BART_EINVAL, "bart_form_rdm_static: dtype=%d", dtype);
    if (window != BART_WINDOW_HANN && window != BART_WINDOW_RECT)
        return fail(BART_EINVAL, "bart_form_rdm_static: window=%d", window);
    if (O < 1 || !is_fft_len(M) || M < 32 || M > 1024 || !is_fft_len(N) || N < 2 || N > 1024)
        return fail(BART_EINVAL, "bart_form_rdm_static: need O >= 1 and M in [32,1024], "
                    "N in [2,1024], both of the form 2^a 3^b (O=%d N=%d M=%d)", O, N, M);
    RadarDev rd;
    std::memset(&rd, 0, sizeof rd);
    rd.O = O;
    rd.N = N;
    rd.M = M;
    rd.P = O;
    rd.Q = 1;
    rd.window = window;
    const int64_t need = rdm_workspace_bytes(rd, dtype);
    if (need > kRdmStaticWorkspaceBytes)
        return fail(BART_EINVAL, "bart_form_rdm_static: the cube needs %lld bytes of workspace, "
                    "more than the fixed %lld (O*N*M <= %lld complex%s samples)",
                    (long long)need, (long long)kRdmStaticWorkspaceBytes,
                    (long long)(kRdmStaticWorkspaceBytes / (dtype == BART_C64 ? 12 : 24)),
                    dtype == BART_C64 ? "64" : "128");
    void *ws = nullptr;
    const char *err = nullptr;
    const int rc = rdm_static_workspace(&ws, &err);
    if (rc != BART_OK) return fail(rc, "bart_form_rdm_static: %s", err);
    launch_rdm(adc, dtype, rd, 1, ws, rdm, nullptr, reinterpret_cast<cudaStream_t>(stream));
    CUDA_TRY(cudaGetLastError(), "bart_form_rdm_static launch");
    return BART_OK;
}

int bart_frame_host(bart_ctx *ctx, double t0, int32_t path, float *rdm_host, bart_stats *stats)
{
    g_err.clear();
    if (!ctx || !rdm_host) return fail(BART_EINVAL, "bart_frame_host: NULL argument");
    if (!ctx->have_radar) return fail(BART_ESTATE, "bart_frame_host: radar not set");
    const bart_radar &r = ctx->radar;
    const int dtype = path == BART_PATH_FP64 ? BART_C128 : BART_C64;
    const size_t esz = dtype == BART_C64 ? 8 : 16;
    BART_TRY(set_device(ctx));
    const size_t B = (size_t)ctx->n_scenes;
    BART_TRY(ctx->adc_own.ensure(B * r.P * r.Q * r.N * r.M * esz, "frame adc"));
    BART_TRY(ctx->rdm_own.ensure(B * r.M * r.N, "frame rdm"));
    BART_TRY(run_frame(ctx, t0, path, ctx->adc_own.p, dtype, stats));
    BART_TRY(run_rdm(ctx, ctx->adc_own.p, dtype, ctx->rdm_own.p));
    CUDA_TRY(cudaMemcpyAsync(rdm_host, ctx->rdm_own.p, B * r.M * r.N * sizeof(float),
                             cudaMemcpyDeviceToHost, ctx->stream), "rdm copy");
    CUDA_TRY(cudaStreamSynchronize(ctx->stream), "cudaStreamSynchronize");
    return BART_OK;
}

int bart_get_visibility(bart_ctx *ctx, uint8_t *state, int64_t *n_grazing)
{
    g_err.clear();
    if (!ctx || !state) return fail(BART_EINVAL, "bart_get_visibility: NULL argument");
    if (!ctx->have_frame) return fail(BART_ESTATE, "bart_get_visibility: no frame simulated");
    BART_TRY(set_device(ctx));
    CUDA_TRY(cudaMemcpyAsync(state, ctx->state.p, (size_t)ctx->frame_A * ctx->frame_F,
                             cudaMemcpyDeviceToDevice, ctx->stream), "state copy");
    if (n_grazing) {
        unsigned long long g = 0;
        CUDA_TRY(cudaMemcpyAsync(&g, ctx->counters.p + 3, sizeof g, cudaMemcpyDeviceToHost,
                                 ctx->stream), "grazing count copy");
        CUDA_TRY(cudaStreamSynchronize(ctx->stream), "cudaStreamSynchronize");
        *n_grazing = (int64_t)g;
    }
    return BART_OK;
}

int bart_get_bvh(bart_ctx *ctx, bart_bvh_node *nodes, int32_t *roots, double *tri,
                 int64_t *n_nodes, int64_t *n_facets, int32_t *n_scenes)
{
    static_assert(sizeof(bart_bvh_node) == sizeof(bart::BvhNode), "bart_bvh_node layout");
    g_err.clear();
    if (!ctx || !n_nodes || !n_facets || !n_scenes)
        return fail(BART_EINVAL, "bart_get_bvh: NULL argument");
    if (!ctx->have_frame) return fail(BART_ESTATE, "bart_get_bvh: no frame simulated");
    const int64_t F = ctx->frame_F;
    const int B = ctx->frame_B;
    *n_nodes = F > 1 ? F - 1 : 0;
    *n_facets = F;
    *n_scenes = B;
    if (!nodes && !roots && !tri) return BART_OK;
    if (!nodes || !roots || !tri) return fail(BART_EINVAL, "bart_get_bvh: NULL buffer");
    BART_TRY(set_device(ctx));
    if (F > 1)
        CUDA_TRY(cudaMemcpyAsync(nodes, ctx->nodes.p, (size_t)(F - 1) * sizeof(bart::BvhNode),
                                 cudaMemcpyDeviceToHost, ctx->stream), "bvh node copy");
    if (B > 1)
        CUDA_TRY(cudaMemcpyAsync(roots, ctx->d_root.p, (size_t)B * sizeof(int32_t),
                                 cudaMemcpyDeviceToHost, ctx->stream), "bvh root copy");
    else
        roots[0] = F > 1 ? 0 : ~0;
    CUDA_TRY(cudaMemcpyAsync(tri, ctx->tri64.p, (size_t)F * 9 * sizeof(double),
                             cudaMemcpyDeviceToHost, ctx->stream), "facet vertex copy");
    CUDA_TRY(cudaStreamSynchronize(ctx->stream), "cudaStreamSynchronize");
    return BART_OK;
}

int bart_get_bounce_facets(bart_ctx *ctx, int32_t *pab, double *tri, double *src, double *usrc,
                           double *w, int64_t cap, int64_t *n)
{
    g_err.clear();
    if (!ctx || !n) return fail(BART_EINVAL, "bart_get_bounce_facets: NULL argument");
    if (!ctx->have_frame) return fail(BART_ESTATE, "bart_get_bounce_facets: no frame simulated");
    if (cap < 0) return fail(BART_EINVAL, "bart_get_bounce_facets: cap=%lld", (long long)cap);
    *n = ctx->db_n;
    const int64_t k = std::min(cap, ctx->db_n);
    if (k == 0) return BART_OK;
    if (!pab || !tri || !src || !usrc || !w)
        return fail(BART_EINVAL, "bart_get_bounce_facets: NULL output with cap > 0");
    BART_TRY(set_device(ctx));
    std::vector<BounceFacet> h((size_t)k);
    CUDA_TRY(cudaMemcpyAsync(h.data(), ctx->db_vf.p, (size_t)k * sizeof(BounceFacet),
                             cudaMemcpyDeviceToHost, ctx->stream), "virtual facet copy");
    CUDA_TRY(cudaStreamSynchronize(ctx->stream), "cudaStreamSynchronize");
    for (int64_t i = 0; i < k; ++i) {
        const BounceFacet &v = h[(size_t)i];
        pab[4 * i] = v.p;
        pab[4 * i + 1] = v.a;
        pab[4 * i + 2] = v.b;
        pab[4 * i + 3] = v.side;
        for (int r = 0; r < 9; ++r) tri[9 * i + r] = v.tri[r];
        for (int r = 0; r < 3; ++r) {
            src[3 * i + r] = v.src[r];
            usrc[3 * i + r] = v.usrc[r];
        }
        w[i] = v.w;
    }
    return BART_OK;
}

int bart_set_timing(bart_ctx *ctx, int32_t enable)
{
    g_err.clear();
    if (!ctx) return fail(BART_EINVAL, "bart_set_timing: ctx is NULL");
    ctx->timing = enable != 0;
    return BART_OK;
}

static float elapsed(cudaEvent_t a, cudaEvent_t b)
{
    float ms = 0.f;
    cudaEventElapsedTime(&ms, a, b);
    return ms;
}

int bart_get_timing(bart_ctx *ctx, bart_timing *out)
{
    g_err.clear();
    if (!ctx || !out) return fail(BART_EINVAL, "bart_get_timing: NULL argument");
    if (!ctx->timed_frame || !ctx->have_frame || ctx->ev.size() < 7)
        return fail(BART_ESTATE, "bart_get_timing: timing disabled or no frame simulated");
    BART_TRY(set_device(ctx));
    CUDA_TRY(cudaEventSynchronize(ctx->ev[4]), "cudaEventSynchronize");
    std::memset(out, 0, sizeof *out);
    out->scene_ms = elapsed(ctx->ev[0], ctx->ev[1]);
    out->bvh_ms = elapsed(ctx->ev[1], ctx->ev[2]);
    out->visibility_ms = elapsed(ctx->ev[2], ctx->ev[3]);
    if (ctx->path == BART_PATH_MIXED) {
        // the kinematics-row launch, then the synthesis launches
        for (int c = 0; c < ctx->chunks; ++c) {
            out->kinematics_ms += elapsed(ctx->ev_kin[2 * c], ctx->ev_kin[2 * c + 1]);
            out->synthesis_ms += elapsed(ctx->ev_syn[2 * c], ctx->ev_syn[2 * c + 1]);
        }
    } else {
        out->synthesis_ms = elapsed(ctx->ev[3], ctx->ev[4]);
    }
    if (ctx->timed_bounce) {
        out->bounce_discovery_ms = elapsed(ctx->ev_db[0], ctx->ev_db[1]);
        if (ctx->db_n > 0) out->bounce_synthesis_ms = elapsed(ctx->ev_db[2], ctx->ev_db[3]);
    }
    out->synthesis_launches = ctx->chunks;
    out->launches = ctx->frame_launches;
    if (ctx->have_rdm_timing) {
        CUDA_TRY(cudaEventSynchronize(ctx->ev[6]), "cudaEventSynchronize");
        out->rdm_ms = elapsed(ctx->ev[5], ctx->ev[6]);
        out->launches += ctx->rdm_launches;
    }
    if (ctx->have_detect_timing) {
        CUDA_TRY(cudaEventSynchronize(ctx->ev[8]), "cudaEventSynchronize");
        out->detect_ms = elapsed(ctx->ev[7], ctx->ev[8]);
        out->detect_launches = ctx->detect_launches;
    }
    return BART_OK;
}

int bart_sync(bart_ctx *ctx)
{
    g_err.clear();
    if (!ctx) return fail(BART_EINVAL, "bart_sync: ctx is NULL");
    BART_TRY(set_device(ctx));
    CUDA_TRY(cudaStreamSynchronize(ctx->stream), "cudaStreamSynchronize");
    int st = 0;
    CUDA_TRY(cudaMemcpy(&st, ctx->status.p, sizeof st, cudaMemcpyDeviceToHost), "status copy");
    if (st) {
        cudaMemset(ctx->status.p, 0, sizeof st);
        if (st & kStatusWaitTimeout)
            return fail(BART_ETIMEOUT, "a bounded device wait expired (RDM tile copy)");
        if (st & kStatusStackOverflow)
            return fail(BART_EDEVICE, "BVH traversal stack overflow (facets marked grazing)");
        return fail(BART_EDEVICE, "device status 0x%x", st);
    }
    return BART_OK;
}

}  // extern "C"
