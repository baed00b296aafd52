// Declarations of the double-bounce paths (bounce.cu), used by the C ABI.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "bart_internal.cuh"

namespace bart {

// ---- double bounce (bounce.cu) ----
// One virtual facet of a double-bounce path (Sec. 2.2: TX p -> facet a ->
// facet b -> RX): a fan piece of b's part lit by the reflection from a.
struct BounceFacet {
    double tri[9];           // frame-start vertices
    double src[3];           // image source p'_0 (TX p mirrored in a's plane)
    double usrc[3];          // its velocity (a's plane moving)
    double w;                // -rho_a rho_b
    int32_t p, a, b, side;   // TX, first facet, second facet, side of b lit (+1 / -1)
};
static_assert(sizeof(BounceFacet) == 144, "BounceFacet layout");
// A candidate (first facet a, second facet b) of TX p: b in a box that
// meets a's beam and facing TX p's image in a (side of b)
struct BounceCand {
    int32_t a, b, p, side;
};
// words of the scan scratch for n counts (the last one receives the total)
int64_t bounce_scan_words(int64_t n);
// exclusive scan of n int32 counts into off, the total into blk[bounce_scan_words(n) - 1]
void launch_bounce_scan(const int32_t *cnt, int64_t n, int64_t *off, int64_t *blk,
                        cudaStream_t s);
// subtrees NS (1, 2, 4 or 8) the candidate traversal splits the LBVH into,
// and their roots (NS ints)
int bounce_subtrees(const RadarDev &rd, int64_t F);
void launch_bounce_roots(const BvhNode *nodes, int64_t F, int NS, int32_t *roots, cudaStream_t s);
// pass 1 over the (TX p, i-th facet lit from p, subtree) items, P F NS of
// them: the candidates per item into cnt (count), or the candidates at off
// (fill)
void launch_bounce_candidates(bool fill, const double *tri64, const FacetRec *fac,
                              const double *vel64, const BvhNode *nodes, const uint8_t *state,
                              const int32_t *vis_idx, const int32_t *vis_cnt, int64_t F,
                              const RadarDev &rd, int NS, const int32_t *roots, int32_t *cnt,
                              const int64_t *off, BounceCand *cand, int *status, cudaStream_t s);
// pass 2 over the candidates: the virtual facets per candidate into pcnt
// (count: clip, slivers, the a -> b leg), or written at poff (fill)
void launch_bounce_pairs(bool fill, const double *tri64, const float *tri32, const FacetRec *fac,
                         const double *vel64, const BvhNode *nodes, const uint8_t *state,
                         const BounceCand *cand, int64_t ncand, int64_t F, const RadarDev &rd,
                         int32_t *pcnt, const int64_t *poff, BounceFacet *vf, int *status,
                         cudaStream_t s);
// txoff[p] (p <= P): the first virtual facet of TX p (txoff[P] = all of them)
void launch_bounce_tx_offsets(const int64_t *cand_off, const int64_t *ncand, const int64_t *poff,
                              const int64_t *npieces, int64_t F, int P, int NS, int64_t *txoff,
                              cudaStream_t s);
// adds the double-bounce echo of every channel into the cube, the
// per-sample work in FP32 (fp32_eval: records from slow-time rows, FP32
// phasors, the record lists cut into NCH chunks whose partial sums a
// reduction adds in order) or in FP64; records: counter of (virtual facet,
// channel, chirp) records, or NULL
void launch_bounce_synth(const BounceFacet *vf, const int64_t *txoff, const FacetRec *fac,
                         const double *vel64, const uint8_t *state,
                         int64_t F, const RadarDev &rd, void *out, int out_c64,
                         bool fp32_eval, const void *rows, const void *geo, int NCH,
                         double2 *partial, unsigned long long *records, cudaStream_t s);
// chunks per record list of the FP32 evaluation; with more than one,
// launch_bounce_synth needs partial: chunks x O x N x M double2
int bounce_synth_chunks(const RadarDev &rd);
// the FP32 evaluation's per-frame data: slow-time rows of each virtual
// facet's 1 + Q legs (bounce_row_bytes per facet) and its FP32 geometry
// (bounce_geo_bytes per facet)
int64_t bounce_row_bytes(const RadarDev &rd);
int64_t bounce_geo_bytes();
void launch_bounce_rows(const BounceFacet *vf, int64_t V, const FacetRec *fac,
                        const double *vel64, const RadarDev &rd, void *rows, void *geo,
                        cudaStream_t s);

}  // namespace bart
