/*
 * abx -- BVH-driven density clustering of 3-D particles on one GB300 GPU.
 *
 * DBSCAN with any minPts, and its minPts = 2 friends-of-friends (FoF) case
 * used for halo finding, following "Advances in ArborX to support exascale
 * applications" (arXiv 2409.10743): the definitions of subsection "DBSCAN
 * algorithm", the two-phase Algorithm PDSDbscan, FDBSCAN (fused traversal with
 * union-find, early-terminated core counting, pair traversal) and
 * FDBSCAN-DenseBox (dense grid cells as hierarchy leaves), over a linear BVH
 * built bottom-up from sorted Morton codes with ropes for stackless traversal
 * (subsections "Stackless traversal", "64-bit Morton codes",
 * "Pair traversal").
 *
 * Results are exact and deterministic:
 *   - two points are neighbours iff d2 <= fl(eps*eps), where
 *     d2 = fl(fl(fl(dx*dx) + fl(dy*dy)) + fl(dz*dz)) and dx = fl(xi - xj) etc.:
 *     FP32, round-to-nearest-even, no fused multiply-add, no flush-to-zero;
 *   - |N_eps(x)| counts x itself; x is core iff |N_eps(x)| >= minPts;
 *   - a cluster's id is the smallest original index among its members (core
 *     points and the border points it was given); noise is -1;
 *   - a border point (non-core, with a core neighbour) joins the neighbouring
 *     cluster whose smallest core index is smallest.  (The paper's Algorithm
 *     PDSDbscan lets the first core to arrive claim it; that is
 *     nondeterministic and is replaced by this rule.)
 * Labels are therefore a pure function of (points, eps, minPts): identical
 * across calls, parameter choices, the batched path and the serving path.
 *
 * Conventions for every entry point:
 *   - points are caller-owned float32 [n][3] (x, y, z) rows, contiguous;
 *   - labels are caller-owned int32 [n];
 *   - "device" pointers are CUDA device (or managed) memory of the current
 *     device; "host" pointers are ordinary (preferably pinned) host memory;
 *   - work is enqueued on `stream` (a cudaStream_t; NULL = legacy default
 *     stream) and the call returns without waiting, unless stated otherwise;
 *     the caller keeps inputs alive and unmodified until the stream reaches
 *     the end of the call's work;
 *   - arguments are checked on the host before anything is enqueued;
 *     a bad argument returns ABX_EINVAL and enqueues nothing;
 *   - workspace comes from a library-owned, stream-ordered CUDA memory pool
 *     (one per device), released back to the pool in stream order;
 *   - errors detected on the device (non-finite coordinates, a bounded wait
 *     that ran out) never trap: kernels record them in a per-device status
 *     word that abx_device_status() reads back;
 *   - the library never calls exit(), assert() or __trap().
 * Thread safety: calls on different streams may run concurrently from
 * different host threads.
 */
#ifndef ABX_H
#define ABX_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int32_t abx_status;

#define ABX_OK 0
#define ABX_EINVAL (-1)        /* bad argument; nothing was enqueued */
#define ABX_ENOMEM (-2)        /* device memory pool could not allocate */
#define ABX_ENOMEM_BUDGET (-3) /* serving: request larger than the HBM budget */
#define ABX_ECUDA (-4)         /* a CUDA runtime call failed */
#define ABX_ETIMEOUT (-5)      /* a bounded wait ran out (host wait or device spin) */
#define ABX_ECANCELLED (-6)    /* serving: the server was destroyed first */
#define ABX_EBUSY (-7)         /* serving: no free slot and the queue is full */
#define ABX_ENONFINITE (-8)    /* device: a coordinate was NaN or infinite */
#define ABX_EINTERNAL (-9)     /* device: an internal consistency check failed */

/* Opaque CUDA stream handle (cudaStream_t). */
typedef struct CUstream_st *abx_stream;

/*
 * Tuning parameters.  Every field 0 means "library default".  None of them
 * changes the labels; they only change speed and memory.
 *   leaf_size    points per ordinary hierarchy leaf (1..32, default 4)
 *   dense_cells  1 = FDBSCAN-DenseBox dense-cell leaves on, -1 = off (default on)
 *   sub_bits     Morton bits per axis below the dense-cell side (1..8; -1 = none,
 *                the default)
 *   block        threads per block of the traversal kernels (64..1024, default 256)
 *   dense_min    a cell is dense only with at least max(minPts, 2, dense_min)
 *                points (0..1<<20, default 0)
 *   schedule     how the pair traversal (paper, subsection "Pair traversal") is
 *                scheduled: 1 = two passes, one rope walk per leaf with the
 *                leaf's box collecting candidate leaves, then one thread per
 *                point testing them (the default); 2 = one pass, every point
 *                walks the ropes from its own leaf with its own box
 *   sort_digit_bits  bits per radix-sort digit: 8 (the default, and the only
 *                width built; any other value returns ABX_EINVAL)
 */
typedef struct abx_params {
    int32_t leaf_size;
    int32_t dense_cells;
    int32_t sub_bits;
    int32_t block;
    int32_t dense_min;
    int32_t schedule;
    int32_t sort_digit_bits;
    int32_t reserved[1];
} abx_params;

/* Human-readable name of a status code (static storage). */
const char *abx_status_str(abx_status s);

/*
 * abx_dbscan -- cluster n points (paper, Algorithm PDSDbscan with the FDBSCAN
 * and FDBSCAN-DenseBox kernels).
 *   points  device, float32 [n][3], caller-owned, read only
 *   n       0 <= n <= 2^31 - 1; n = 0 returns ABX_OK and enqueues nothing
 *   eps     finite, >= 0
 *   minpts  >= 1 (minpts <= 2 takes the friends-of-friends path)
 *   labels  device, int32 [n], caller-owned, written
 *   stream  the stream the work is enqueued on
 * Returns ABX_OK once enqueued; ABX_EINVAL, ABX_ENOMEM or ABX_ECUDA otherwise.
 */
abx_status abx_dbscan(const float *points, int64_t n, float eps, int32_t minpts,
                      int32_t *labels, abx_stream stream);

/* abx_dbscan with explicit tuning parameters (params may be NULL). */
abx_status abx_dbscan_ex(const float *points, int64_t n, float eps, int32_t minpts,
                         int32_t *labels, const abx_params *params, abx_stream stream);

/*
 * abx_dbscan_host -- the same clustering from host memory to host memory: the
 * library copies the points in, runs abx_dbscan and copies the labels out,
 * all on `stream`, then waits for the stream.  points_host float32 [n][3] and
 * labels_host int32 [n] are caller-owned host buffers (pinned memory makes the
 * copies asynchronous and faster).  Blocks until the labels are in place.
 */
abx_status abx_dbscan_host(const float *points_host, int64_t n, float eps, int32_t minpts,
                           int32_t *labels_host, abx_stream stream);

/*
 * CUDA graph of one fixed clustering.  abx_graph_create captures every stage
 * of abx_dbscan_ex for these arguments (the same pointers, n, eps, minPts and
 * parameters) into a CUDA graph with a device workspace of its own, so that
 * abx_graph_launch replays the ~29 kernels with one launch: for small inputs
 * the launches, not the kernels, set the time.  The caller may change the
 * CONTENTS of points between replays (a simulation's next time step), not
 * the buffers or n; each replay writes labels for the current contents.
 *   points, n (1 <= n <= 2^31 - 1), eps, minpts, labels, params: as for
 *           abx_dbscan_ex (params NULL = the autotuner's pick or defaults)
 *   out     receives the handle
 * Allocates the workspace (cudaMalloc) and synchronises during creation;
 * ABX_ENOMEM if the workspace does not fit, ABX_ECUDA if capture fails.
 * abx_graph_launch enqueues one replay on `stream` (ABX_EINVAL if the current
 * device is not the one the graph was made on); replays on different streams
 * share the workspace, so keep them in order on one stream.
 * abx_graph_destroy waits for the graph's last replay (not for other work on
 * the device), then frees the graph and its workspace.
 */
typedef struct abx_graph abx_graph;
abx_status abx_graph_create(const float *points, int64_t n, float eps, int32_t minpts, int32_t *labels,
                            const abx_params *params, abx_graph **out);
abx_status abx_graph_launch(abx_graph *graph, abx_stream stream);
abx_status abx_graph_destroy(abx_graph *graph);

/*
 * abx_device_status -- wait for `stream`, then return and clear the current
 * device's status word: ABX_OK, ABX_ENONFINITE (a coordinate was not finite),
 * ABX_ETIMEOUT (a bounded device wait ran out) or ABX_EINTERNAL (a kernel's
 * consistency check failed and it stopped early).  After any of these the
 * labels of the calls since the previous check are unspecified.
 */
abx_status abx_device_status(abx_stream stream);

/*
 * abx_dbscan_batch -- cluster nseg independent point sets in one pass
 * (many sub-volumes at once).  Segment k is points[offsets[k] .. offsets[k+1])
 * of the concatenated array and is clustered with eps[k] and minpts[k] exactly
 * as abx_dbscan would cluster it alone; labels[offsets[k] + i] is a
 * segment-local index (or -1).
 *   points   device, float32 [offsets[nseg]][3]
 *   offsets  host, int64 [nseg + 1], offsets[0] = 0, non-decreasing,
 *            offsets[nseg] <= 2^31 - 1
 *   eps      host, float [nseg], each finite and >= 0
 *   minpts   host, int32 [nseg], each >= 1
 *   labels   device, int32 [offsets[nseg]]
 * The host arrays are read before the call returns.
 */
abx_status abx_dbscan_batch(const float *points, const int64_t *offsets, int32_t nseg,
                            const float *eps, const int32_t *minpts, int32_t *labels,
                            abx_stream stream);

/* abx_dbscan_batch with explicit tuning parameters.  params NULL: the
 * parameters abx_autotune_batch remembered for batches of this class (total
 * points, any DBSCAN segment or none), else the library defaults; the serving
 * loop's batches take this path. */
abx_status abx_dbscan_batch_ex(const float *points, const int64_t *offsets, int32_t nseg,
                               const float *eps, const int32_t *minpts, int32_t *labels,
                               const abx_params *params, abx_stream stream);

/*
 * abx_dbscan_noalloc -- abx_dbscan for callers that cannot allocate device
 * memory (an in-situ hook inside a simulation that has reserved the GPU's
 * memory for itself, or code where allocation calls are not permitted).  The
 * paper has no counterpart: this is a deployment variant of the same
 * clustering, with the same labels.
 *   points, eps, minpts, labels, stream: as for abx_dbscan
 *   n       0 <= n <= 65536; larger inputs return ABX_EINVAL before anything
 *           is enqueued
 * Calls no allocation routine.  The workspace is a fixed array of device
 * memory (12 MiB per device that loads the library, held until
 * the process exits).  The first call on a device looks up that array's
 * address and sets kernel attributes; make that first call before any stream
 * capture.  Every call on a device shares the array: calls whose work
 * overlaps on the GPU race, so serialise them (one stream, one at a time).
 * Device-side errors of this entry point (a non-finite coordinate, a bounded
 * wait that ran out) go to a status word of its own in the same fixed device
 * memory; abx_device_status reads and clears it together with the library's.
 */
abx_status abx_dbscan_noalloc(const float *points, int64_t n, float eps, int32_t minpts,
                              int32_t *labels, abx_stream stream);

/*
 * abx_selftest_wait_timeout -- check that a device wait that can never be
 * satisfied gives up instead of hanging: one thread runs the library's
 * bounded look-back wait (the one the radix sort and the scans use) over a
 * status array in which no predecessor ever publishes, re-reading it at most
 * spin_limit (1 .. 2^24) times, then records a timeout in the device status
 * word and returns.  Enqueued on `stream`; a following abx_device_status
 * returns ABX_ETIMEOUT (and clears it).  No GPU fault, no trap.  The paper
 * has no counterpart: this is failure detection for the library itself.
 */
abx_status abx_selftest_wait_timeout(int32_t spin_limit, abx_stream stream);

/* ---- per-cluster statistics --------------------------------------------------- */

/*
 * abx_cluster_stats -- reduce a labelling (as abx_dbscan writes it) to its
 * clusters, in increasing cluster id: ids[k] (the cluster's id), sizes[k],
 * centres[k] = mean member position (summed in double, rounded to float) and
 * radii[k] = distance from that centre to the farthest member (sqrtf of the
 * largest exact FP32 squared distance) -- the galaxy circles of the paper's
 * HACC section.  Noise (-1) is skipped; labels must lie in [-1, n).
 *   points  device float32 [n][3];  labels device int32 [n]
 *   ids, sizes device int32 [n];  centres device float32 [n][3];  radii device
 *   float32 [n] (capacity n; the first *n_clusters entries are written)
 *   n_clusters  host; the call waits for `stream`
 */
abx_status abx_cluster_stats(const float *points, const int32_t *labels, int64_t n, int32_t *n_clusters,
                             int32_t *ids, int32_t *sizes, float *centres, float *radii, abx_stream stream);

/* ---- autotuning (the paper lists runtime tuning of
 *      occupancy parameters as future work, section "Conclusions") --------- */

/*
 * abx_autotune -- time candidate parameters on this input (leaf size, then
 * traversal block size, then dense cells on/off and the minimum dense-cell
 * size, then the traversal schedule, keeping the best so far; each candidate
 * once to warm up and twice timed with CUDA events on `stream`), remember the
 * fastest for this device and size class (friends-of-friends or DBSCAN,
 * floor(log2 n)), and return it in *best (may be NULL).  Later abx_dbscan
 * calls of that class without explicit parameters use it.  labels (device
 * int32 [n]) receives the labels.  Blocks.
 */
abx_status abx_autotune(const float *points, int64_t n, float eps, int32_t minpts, int32_t *labels,
                        abx_params *best, abx_stream stream);

/*
 * abx_autotune_batch -- the same search on a batch (arguments as for
 * abx_dbscan_batch), remembered for batches of its class (total points, any
 * DBSCAN segment or none) and used by later abx_dbscan_batch calls and by the
 * serving loop.  Blocks.
 */
abx_status abx_autotune_batch(const float *points, const int64_t *offsets, int32_t nseg, const float *eps,
                              const int32_t *minpts, int32_t *labels, abx_params *best, abx_stream stream);

/* The remembered parameters of the size class of (n, minpts) on the current
 * device (ABX_EINVAL if none), and setting them (e.g. from a saved table). */
abx_status abx_tune_get(int64_t n, int32_t minpts, abx_params *out);
abx_status abx_tune_set(int64_t n, int32_t minpts, const abx_params *params);

/* ---- stage timers (tracing) -------------------------------------------------- */

/*
 * abx_profile_enable -- on = 1: every clustering call records a CUDA event on
 * its stream at each stage boundary (bounds, morton, sort, gather, cells,
 * leaves, build, candidates, count, union, border, finalize).  on = 2: the same, and the
 * pair traversal also counts its work (a slower, instrumented kernel; read
 * with abx_profile_traversal).  on = 0: off.  Meant for one call at a time
 * (benchmarks): concurrent profiled calls overwrite each other's events.
 */
abx_status abx_profile_enable(int32_t on);

/* Number of stages and the name of stage i (static storage). */
int32_t abx_profile_stage_count(void);
const char *abx_profile_stage_name(int32_t i);

/*
 * abx_profile_read -- wait for the stream of the most recent profiled call and
 * write the milliseconds each stage took (device time between consecutive
 * stage events) into ms[0 .. n-1].  Stages a call skipped read 0.
 */
abx_status abx_profile_read(float *ms, int32_t n);

/*
 * abx_profile_counters -- facts about the most recent profiled clustering
 * call, written to out[0 .. n-1] in this order: radix passes run, Morton bits
 * per axis, dense cells on (0/1), dense cells found, hierarchy leaves, root
 * node, key width in bits (32 or 64).
 */
abx_status abx_profile_counters(int64_t *out, int32_t n);

/*
 * abx_profile_traversal -- work counters of the pair traversal of the most
 * recent call made in profile mode 2, written to out[0 .. n-1]: node visits,
 * leaf visits, point-pair tests, unions, queries.
 */
abx_status abx_profile_traversal(int64_t *out, int32_t n);

/* Total number of kernels this library has launched in this process. */
unsigned long long abx_launch_count(void);

/* ---- serving: requests arriving over time, continuous batching ------------ */

/*
 * A server owns a scheduler thread and max_slots CUDA streams on one device.
 * Requests (host points in, host labels out) queue in arrival order; whenever
 * a slot is free the scheduler admits requests from the head of the queue
 * into one batch -- as many as fit max_batch_requests, max_batch_points and
 * the HBM budget left by batches still running -- and runs the batch as one
 * abx_dbscan_batch pass on that slot's stream.  Batches admitted while others
 * run overlap on the GPU.  A request's labels are exactly what abx_dbscan
 * returns for it alone.  (Meant for in-situ analysis of many sub-volumes;
 * the paper itself clusters one rank's particles per call.)
 */
typedef struct abx_serve_config {
    uint64_t hbm_budget_bytes;  /* device bytes running batches may hold (0 = 40 GiB) */
    int32_t max_slots;          /* batches on the GPU at once, one stream each (0 = 2, max 16) */
    int32_t max_batch_requests; /* most requests per batch (0 = 512) */
    int64_t max_batch_points;   /* most points per batch (0 = 2^25) */
    int32_t max_queue;          /* queued requests before submit returns ABX_EBUSY (0 = 2^20) */
    int32_t device;             /* CUDA device ordinal */
    int32_t reserved[4];
} abx_serve_config;

typedef struct abx_serve_report {
    uint64_t submitted, completed, failed, cancelled;
    uint64_t batches;            /* batches launched */
    uint64_t queued;             /* requests waiting for admission */
    uint64_t bytes_in_use;       /* device bytes reserved by running batches */
    uint64_t peak_bytes;         /* highest bytes_in_use so far */
    double p50_ms, p99_ms, mean_ms, max_ms;  /* latency: completion - submission */
    double requests_per_s;       /* completed / (last completion - first submission) */
    double mean_batch_requests;  /* requests per batch */
} abx_serve_report;

typedef struct abx_server abx_server;

/* Create a server (cfg may be NULL for defaults).  Host-resident requests'
 * points are copied to the device straight from the caller's memory (or,
 * with ABX_SERVE_STAGING=1, staged through pinned buffers first); their
 * labels come back through pinned buffers, allocated per slot at its first
 * host request for min(max_batch_points, 2^25) labels (with staging, points
 * too) and grown only by a larger batch: max_slots x 4 bytes per point of
 * pinned host memory (16 with staging).  Host-side fault injection for
 * tests: ABX_SERVE_FAULT=hold admits nothing, =alloc fails every batch's
 * device allocation.  (Both read at creation.) */
abx_status abx_serve_create(const abx_serve_config *cfg, abx_server **out);

/*
 * abx_serve_submit -- queue one request.  points: float32 [n][3] and
 * labels: int32 [n], both caller-owned, both host memory or both device
 * memory of the server's device (device-resident requests, the in-situ case,
 * skip the host staging), left untouched by the caller until abx_serve_wait
 * returns for the ticket.  producer: for device requests, the stream whose
 * work writes the points (NULL = legacy default stream); the server reads
 * them only after everything enqueued on it at the time of the call.  Host
 * points must be complete when the call is made.  Returns at once with a ticket;
 * ABX_ENOMEM_BUDGET if the request alone exceeds the budget or the batch
 * size, ABX_EBUSY if the queue is full, ABX_EINVAL for bad arguments.
 */
abx_status abx_serve_submit(abx_server *srv, const float *points, int64_t n, float eps, int32_t minpts,
                            int32_t *labels, abx_stream producer, uint64_t *ticket);

/*
 * abx_serve_wait -- wait up to timeout_ms (< 0: forever) for a request:
 * ABX_ETIMEOUT if it is not done yet (the ticket stays valid), else the
 * request's status (ABX_OK, ABX_ECANCELLED, ABX_ENOMEM, ...), after which the
 * ticket is released.
 */
abx_status abx_serve_wait(abx_server *srv, uint64_t ticket, int32_t timeout_ms);

/* Counters and latency percentiles of the requests completed so far. */
abx_status abx_serve_stats(abx_server *srv, abx_serve_report *out);

/*
 * abx_serve_destroy -- stop the server: queued requests end ABX_ECANCELLED,
 * batches already on the GPU run to completion; then the streams and staging
 * buffers are freed.  Must not run concurrently with other calls on srv.
 */
abx_status abx_serve_destroy(abx_server *srv);

/* ---- the bounding volume hierarchy on its own ------------------------------ */

/* Opaque, library-owned hierarchy over a point set (paper, section "ArborX
 * library": a binary BVH over Morton-sorted points, built bottom-up, with
 * ropes for stackless traversal). */
typedef struct abx_bvh abx_bvh;

/*
 * abx_bvh_build -- build a hierarchy over n points (device float32 [n][3]);
 * the library copies what it needs, so points may be freed once the stream
 * has passed the call.  *out receives the handle; the build is enqueued on
 * `stream` and the handle may be used on that stream right away.
 * params: NULL or tuning parameters as for abx_dbscan_ex (leaf_size and
 * sort_digit_bits apply; dense cells are never built here).
 * 1 <= n <= 2^31 - 1; ABX_EINVAL for bad parameters.
 */
abx_status abx_bvh_build(const float *points, int64_t n, const abx_params *params, abx_bvh **out,
                         abx_stream stream);

/*
 * abx_bvh_count -- early-terminated range counting (paper, subsection "Early
 * termination"): counts[q] = min(cap, number of tree points p with
 * pred(query q, p)), stopping each query's traversal once cap is reached.
 *   queries  device float32 [nq][3];  counts device int32 [nq];  cap >= 1.
 */
abx_status abx_bvh_count(const abx_bvh *bvh, const float *queries, int64_t nq, float eps,
                         int32_t cap, int32_t *counts, abx_stream stream);

/*
 * abx_bvh_first_hit -- early-terminated existence query (paper, subsection
 * "Early termination", with the traversal stopped at the first neighbour):
 * hits[q] = the original index (position in the points given to
 * abx_bvh_build) of a tree point p with pred(query q, p), namely the first
 * one the traversal meets, or -1 if there is none.  Which neighbour is
 * returned depends on the hierarchy; that one exists does not.
 *   queries  device float32 [nq][3];  hits device int32 [nq].
 * ABX_EINVAL for a null handle or pointers, nq < 0, negative or non-finite eps.
 */
abx_status abx_bvh_first_hit(const abx_bvh *bvh, const float *queries, int64_t nq, float eps,
                             int32_t *hits, abx_stream stream);

/*
 * abx_bvh_pair_histogram -- the "find every pair within a radius, apply F"
 * form of pair traversal (paper, subsection "Pair traversal": forces,
 * 2-point correlation counts), with F = count by distance: hist[b] = number of
 * unordered pairs {i, j}, i != j, of the tree's points with
 * fl(r_b^2) < d2 <= fl(r_{b+1}^2), d2 the exact FP32 squared distance of the
 * neighbour test.  Each pair is visited once.
 *   r_edges  host float [nbins + 1], finite, >= 0, strictly increasing
 *   nbins    1..256;  hist  device uint64 [nbins], overwritten
 */
abx_status abx_bvh_pair_histogram(const abx_bvh *bvh, const float *r_edges, int32_t nbins, uint64_t *hist,
                                  abx_stream stream);

/*
 * abx_bvh_pairs -- every unordered pair {i, j} of the hierarchy's points with
 * pred(i, j) for this eps, each exactly once, handed to the caller: the
 * generic "find all pairs within a radius, apply F" form of the paper's pair
 * traversal (subsections "Pair traversal" and "Callbacks"; the library cannot
 * run a caller's function on the device, so the caller applies F to the
 * pairs).  Pairs are written as pairs[2k] < pairs[2k + 1], original indices
 * (positions in the points given to abx_bvh_build), in a fixed order:
 * point by point in the hierarchy's internal order, then in traversal order.
 * Resumable: *cursor (0 to start) is a position in that internal order; each
 * call writes the pairs of as many following points as fit in cap pairs,
 * sets *n_written to their number and advances *cursor; *cursor == n means
 * all pairs were delivered.
 *   eps       finite, >= 0
 *   cursor    host, in/out, 0 <= *cursor <= n
 *   pairs     device int32 [cap][2] (may be NULL when cap = 0)
 *   cap       pairs the buffer holds, >= 0
 *   n_written host, out
 * ABX_ENOMEM (nothing written, cursor unchanged) if the next point alone has
 * more than cap pairs: call again with a larger buffer.  Each call counts the
 * pairs of all remaining points once more, so larger buffers mean fewer
 * passes.  Waits for `stream`.
 */
abx_status abx_bvh_pairs(const abx_bvh *bvh, float eps, int64_t *cursor, int32_t *pairs, int64_t cap,
                         int64_t *n_written, abx_stream stream);

/* Number of points, leaves and levels (depth of the deepest leaf + 1) of a
 * built hierarchy; waits for `stream`. */
abx_status abx_bvh_info(const abx_bvh *bvh, int64_t *n_points, int64_t *n_leaves,
                        int32_t *levels, abx_stream stream);

/* Free a hierarchy (stream-ordered on the stream it was built on). */
abx_status abx_bvh_destroy(abx_bvh *bvh);

#ifdef __cplusplus
}
#endif
#endif /* ABX_H */
