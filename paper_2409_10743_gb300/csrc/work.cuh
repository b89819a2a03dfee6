// Workspace layout of one clustering call and the launchers of each stage.
#pragma once

#include "abx_internal.cuh"

namespace abx {

// Resolved tuning parameters.
struct Params {
    int leaf_size;   // points per ordinary leaf (1..32)
    int dense;       // dense-cell leaves on/off
    int sub_bits;    // Morton bits per axis below the dense-cell side
    int block;       // threads per block of the traversal kernels
    int dense_min;   // a dense cell needs at least max(minPts, 2, dense_min) points
    int schedule;    // pair traversal: 1 = candidate lists per leaf, then per point; 2 = per point
    int digit_bits;  // radix-sort digit width (RADIX_BITS)
};

// Device buffers of one call; sizes are for n points (L <= n leaves).
struct Work {
    int64_t n;
    int n_sms;
    unsigned *dev_status;            // per-device status word
    State *st;
    unsigned long long *keys[2];     // Morton keys, radix double buffer
    unsigned *vals[2];               // original indices, radix double buffer
    unsigned long long *sort_lb;     // look-back words: [MAX_PASSES][sort_tiles][RADIX], then
                                     // [bucket_tiles][RADIX] of the bucketing pass
    float4 *bpts;                    // [n] points in bucket order (x, y, z, original index); aliases
                                     // nodes, which are written only after the gather has read it
    unsigned long long *scan_lb;     // [scan tiles] look-back words
    float4 *spts;                    // sorted points: x, y, z, original index (as int bits)
    int *dense_root;                 // [n] root of the point's dense cell, or -1
    int *leaf_of;                    // [n] leaf of each sorted point
    int *leaf_first;                 // [n + 1] first sorted point of each leaf
    unsigned char *pdelta;           // [n] split level between sorted points k and k+1
    unsigned char *delta;            // [n] split level between leaves t and t+1
    float4 *nodes;                   // [2 * (2n - 1)] hierarchy records (lo, hi)
    unsigned long long *slot;        // [n] bottom-up meeting slots (global phase)
    int4 *frontier;                  // [n] nodes that finish the build in the global phase
    int4 *cand;                      // [L] candidate leaves of each leaf (aliases frontier, dead after the build)
    int *right_of;                   // [n] right child of each internal node
    int *parent;                     // [n] union-find parents (sorted positions)
    unsigned char *core;             // [n] core flags
    int *bmin;                       // [n] smallest border index per cluster root
    unsigned long long *stats;       // traversal counters (profile mode 2) or null
    // segments (independent point sets); a single clustering call has nseg = 1
    int nseg;
    int *seg_off;                    // [nseg + 1] device offsets (input and sorted order alike)
    SegState *seg;                   // [nseg]
    int *leaf_seg;                   // [n] segment of each leaf
    float *seg_eps_in;               // [nseg] device copy of the caller's eps (batches)
    int *seg_minpts_in;              // [nseg] device copy of the caller's minPts (batches)
    bool any_fof, any_dbscan;        // host: which modes the call's segments use
    size_t sort_tiles, scan_tiles, bucket_tiles;
};

size_t work_bytes(int64_t n, int nseg = 1);
void work_carve(Work &w, void *base, int64_t n, int nseg = 1);

// Segment parameters of a call, as the host gives them.
struct SegHost {
    int nseg;
    const float *eps;      // host [nseg]
    const int32_t *minpts; // host [nseg]
};

// Stages (all asynchronous on `s`).  Segment parameters (eps, minPts,
// offsets) must already be in w.seg / w.seg_off: stage_segments_single puts
// them there for a single clustering call.
void stage_segments_single(const Work &w, float eps, int minpts, cudaStream_t s);
void stage_segments_batch(const Work &w, const float *eps_dev, const int *minpts_dev, int seg_bits, cudaStream_t s);
void stage_bounds_quant(const Work &w, const float *points, const Params &p, cudaStream_t s);
void stage_morton_sort(const Work &w, const float *points, cudaStream_t s);
void stage_gather(const Work &w, const float *points, cudaStream_t s);
void stage_cells_leaves(const Work &w, const Params &p, cudaStream_t s);
void stage_hierarchy(const Work &w, cudaStream_t s);
void stage_cluster(const Work &w, const Params &p, int32_t *labels, cudaStream_t s);

// Parameter resolution (0 fields = defaults) and the autotuner's table.
abx_status resolve_params(const abx_params *in, Params &p);
bool tune_lookup(int64_t n, int32_t minpts, abx_params *out);
bool tune_lookup_batch(int64_t n, bool any_dbscan, abx_params *out);

// The no-allocation entry point's device status word, read and cleared.
abx_status noalloc_take_status(unsigned *out);

// One-time per-device kernel attributes.
void kernels_init_device();
void tree_init_device();
void cluster_init_device();

// Stage timers and launch accounting (profile mode records a CUDA event on the
// launching stream at each stage boundary).
enum Stage {
    ST_BOUNDS = 0, ST_MORTON, ST_BUCKET, ST_SORT, ST_GATHER, ST_CELLS, ST_LEAVES, ST_BUILD,
    ST_CANDS, ST_COUNT, ST_UNION, ST_BORDER, ST_FINALIZE, ST_NUM
};
void prof_begin(cudaStream_t s);
void prof_mark(int stage, cudaStream_t s);
void note_launch(int k = 1);

__host__ __device__ inline int div_up(int64_t a, int64_t b) { return (int)((a + b - 1) / b); }

}  // namespace abx

// The hierarchy handle of the C ABI: the workspace of a build, kept alive.
struct abx_bvh {
    void *ws;
    abx::Work w;
    cudaStream_t stream;
    cudaMemPool_t pool;
};
