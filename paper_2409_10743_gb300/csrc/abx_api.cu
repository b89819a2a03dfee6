// The C ABI: argument checks, per-device context, workspace, stage sequence.
#include <atomic>
#include <cmath>
#include <cstring>
#include <mutex>
#include <vector>

#include "work.cuh"

namespace abx {

// ---- per-device context --------------------------------------------------------

struct DeviceCtx {
    bool ready = false;
    cudaMemPool_t pool = nullptr;
    unsigned *status = nullptr;
    int n_sms = 0;
};

static std::mutex g_mu;
static DeviceCtx g_ctx[64];

static abx_status device_ctx(DeviceCtx **out)
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64)
        return ABX_ECUDA;
    std::lock_guard<std::mutex> lk(g_mu);
    DeviceCtx &c = g_ctx[dev];
    if (!c.ready) {
        cudaMemPoolProps props;
        memset(&props, 0, sizeof(props));
        props.allocType = cudaMemAllocationTypePinned;
        props.handleTypes = cudaMemHandleTypeNone;
        props.location.type = cudaMemLocationTypeDevice;
        props.location.id = dev;
        if (cudaMemPoolCreate(&c.pool, &props) != cudaSuccess)
            return ABX_ECUDA;
        unsigned long long thresh = ~0ull;  // keep freed blocks for reuse
        cudaMemPoolSetAttribute(c.pool, cudaMemPoolAttrReleaseThreshold, &thresh);
        if (cudaMalloc(&c.status, sizeof(unsigned)) != cudaSuccess)
            return ABX_ECUDA;
        if (cudaMemset(c.status, 0, sizeof(unsigned)) != cudaSuccess)
            return ABX_ECUDA;
        if (cudaDeviceGetAttribute(&c.n_sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
            return ABX_ECUDA;
        kernels_init_device();
        tree_init_device();
        cluster_init_device();
        if (cudaGetLastError() != cudaSuccess)
            return ABX_ECUDA;
        c.ready = true;
    }
    *out = &c;
    return ABX_OK;
}

abx_status bvh_device_ctx(cudaMemPool_t *pool, unsigned **status, int *n_sms)
{
    DeviceCtx *c;
    abx_status rc = device_ctx(&c);
    if (rc == ABX_OK) {
        *pool = c->pool;
        *status = c->status;
        *n_sms = c->n_sms;
    }
    return rc;
}

// ---- stage timers and launch accounting ------------------------------------------

static std::atomic<unsigned long long> g_launches{0};
static std::atomic<int> g_prof_on{0};
static std::mutex g_prof_mu;
static cudaEvent_t g_ev[ST_NUM + 1];
static bool g_ev_ready = false;
static bool g_ev_marked[ST_NUM + 1];
static cudaStream_t g_prof_stream = nullptr;
static State *g_prof_state = nullptr;  // pinned host copy of the last profiled call's state
static unsigned long long *g_stats_dev = nullptr;   // traversal counters (mode 2)
static unsigned long long g_stats_host[8];

// Kernels launched by this host thread (a graph capture counts its own).
static thread_local unsigned long long t_launches = 0;
// Set while this thread captures a graph: no profile events go into it.
static thread_local bool t_capturing = false;

void note_launch(int k)
{
    g_launches.fetch_add((unsigned long long)k, std::memory_order_relaxed);
    t_launches += (unsigned long long)k;
}

void prof_begin(cudaStream_t s)
{
    if (!g_prof_on.load() || t_capturing)
        return;
    std::lock_guard<std::mutex> lk(g_prof_mu);
    if (!g_ev_ready) {
        for (int i = 0; i <= ST_NUM; i++)
            cudaEventCreate(&g_ev[i]);
        g_ev_ready = true;
    }
    for (int i = 0; i <= ST_NUM; i++)
        g_ev_marked[i] = false;
    cudaEventRecord(g_ev[0], s);
    g_ev_marked[0] = true;
    g_prof_stream = s;
}

void prof_mark(int stage, cudaStream_t s)
{
    if (!g_prof_on.load() || t_capturing)
        return;
    std::lock_guard<std::mutex> lk(g_prof_mu);
    if (!g_ev_ready || stage < 0 || stage >= ST_NUM)
        return;
    cudaEventRecord(g_ev[stage + 1], s);
    g_ev_marked[stage + 1] = true;
}

// ---- workspace ------------------------------------------------------------------------

static size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

struct Carver {
    size_t off = 0;
    char *base = nullptr;
    template <class T>
    T *take(size_t count)
    {
        size_t o = off;
        off = align256(off + count * sizeof(T));
        return base ? reinterpret_cast<T *>(base + o) : nullptr;
    }
};

static void carve(Carver &c, Work &w, int64_t n, int nseg)
{
    const size_t N = (size_t)n;
    w.n = n;
    w.nseg = nseg;
    w.seg_off = c.take<int>((size_t)nseg + 1);
    w.seg = c.take<SegState>((size_t)nseg);
    w.seg_eps_in = c.take<float>((size_t)nseg);
    w.seg_minpts_in = c.take<int>((size_t)nseg);
    w.leaf_seg = c.take<int>(N);
    w.sort_tiles = (size_t)div_up(n, SORT_TILE_MIN);
    w.scan_tiles = (size_t)div_up(n, SCAN_TILE);
    w.st = c.take<State>(1);
    w.keys[0] = c.take<unsigned long long>(N);
    w.keys[1] = c.take<unsigned long long>(N);
    w.vals[0] = c.take<unsigned>(N);
    w.vals[1] = c.take<unsigned>(N);
    w.bucket_tiles = (size_t)div_up(n, BUCKET_TILE);
    w.sort_lb = c.take<unsigned long long>(((size_t)MAX_PASSES * w.sort_tiles + w.bucket_tiles) * RADIX);
    w.scan_lb = c.take<unsigned long long>(w.scan_tiles);
    w.spts = c.take<float4>(N);
    w.dense_root = c.take<int>(N);
    w.leaf_of = c.take<int>(N);
    w.leaf_first = c.take<int>(N + 1);
    w.pdelta = c.take<unsigned char>(N);
    w.delta = c.take<unsigned char>(N);
    w.nodes = c.take<float4>(2 * (2 * N - 1));
    w.bpts = w.nodes;  // 2 (2n - 1) >= n records
    w.slot = c.take<unsigned long long>(N);
    w.frontier = c.take<int4>(N);
    w.cand = w.frontier;
    w.right_of = c.take<int>(N);
    w.parent = c.take<int>(N);
    w.core = c.take<unsigned char>(N);
    w.bmin = c.take<int>(N);
}

size_t work_bytes(int64_t n, int nseg)
{
    Carver c;
    Work w;
    carve(c, w, n, nseg);
    return c.off;
}

void work_carve(Work &w, void *base, int64_t n, int nseg)
{
    Carver c;
    c.base = static_cast<char *>(base);
    carve(c, w, n, nseg);
    w.stats = nullptr;
    w.any_fof = w.any_dbscan = false;
}

abx_status resolve_params(const abx_params *in, Params &p)
{
    p.leaf_size = 4;
    p.dense = 1;
    p.sub_bits = 0;
    p.block = 256;
    p.dense_min = 0;
    p.schedule = 1;
    p.digit_bits = 8;
    if (!in)
        return ABX_OK;
    if (in->schedule) {
        if (in->schedule != 1 && in->schedule != 2)
            return ABX_EINVAL;
        p.schedule = in->schedule;
    }
    if (in->sort_digit_bits) {
        if (in->sort_digit_bits != RADIX_BITS)
            return ABX_EINVAL;
        p.digit_bits = in->sort_digit_bits;
    }
    if (in->dense_min) {
        if (in->dense_min < 0 || in->dense_min > (1 << 20))
            return ABX_EINVAL;
        p.dense_min = in->dense_min;
    }
    if (in->leaf_size) {
        if (in->leaf_size < 1 || in->leaf_size > 32)
            return ABX_EINVAL;
        p.leaf_size = in->leaf_size;
    }
    if (in->dense_cells) {
        if (in->dense_cells != 1 && in->dense_cells != -1)
            return ABX_EINVAL;
        p.dense = in->dense_cells == 1;
    }
    if (in->sub_bits) {
        if (in->sub_bits < -1 || in->sub_bits > 8)
            return ABX_EINVAL;
        p.sub_bits = in->sub_bits < 0 ? 0 : in->sub_bits;
    }
    if (in->block) {
        if (in->block < 64 || in->block > 1024 || (in->block & 31))
            return ABX_EINVAL;
        p.block = in->block;
    }
    return ABX_OK;
}

static abx_status cuda_status(cudaError_t e)
{
    if (e == cudaSuccess)
        return ABX_OK;
    return e == cudaErrorMemoryAllocation ? ABX_ENOMEM : ABX_ECUDA;
}

// Enqueue the whole pipeline on `s` over a carved workspace whose segment
// parameters are set up (or about to be, earlier on the same stream).
static void run_stages(Work &w, const float *points, int32_t *labels, const Params &p, cudaStream_t s)
{
    stage_bounds_quant(w, points, p, s);
    stage_morton_sort(w, points, s);
    stage_gather(w, points, s);
    stage_cells_leaves(w, p, s);
    stage_hierarchy(w, s);
    stage_cluster(w, p, labels, s);
    if (g_prof_on.load() && !t_capturing) {
        std::lock_guard<std::mutex> lk(g_prof_mu);
        if (!g_prof_state && cudaMallocHost((void **)&g_prof_state, sizeof(State)) != cudaSuccess) {
            g_prof_state = nullptr;
            cudaGetLastError();
        }
        if (g_prof_state)
            cudaMemcpyAsync(g_prof_state, w.st, sizeof(State), cudaMemcpyDeviceToHost, s);
    }
}

// Self-test of the bounded device waits: the look-back of the radix sort and
// the flag scan, run by one thread for tile `tile` over a status array whose
// words are all unpublished, so the wait can only run out.
__global__ void k_selftest_lookback(const unsigned long long *lb, int tile, int spin_limit, unsigned *dev_status,
                                    unsigned long long *out)
{
    if (blockIdx.x == 0 && threadIdx.x == 0)
        *out = lookback<8>(lb, tile, 1, 0, dev_status, spin_limit);
}

}  // namespace abx

using namespace abx;

extern "C" {

const char *abx_status_str(abx_status s)
{
    switch (s) {
    case ABX_OK: return "ok";
    case ABX_EINVAL: return "invalid argument";
    case ABX_ENOMEM: return "out of device memory";
    case ABX_ENOMEM_BUDGET: return "request exceeds the HBM budget";
    case ABX_ECUDA: return "CUDA error";
    case ABX_ETIMEOUT: return "timed out";
    case ABX_ECANCELLED: return "cancelled";
    case ABX_EBUSY: return "busy";
    case ABX_ENONFINITE: return "non-finite coordinate";
    case ABX_EINTERNAL: return "internal consistency check failed";
    default: return "unknown status";
    }
}

static abx_status check_args(const float *points, int64_t n, float eps, int32_t minpts, const int32_t *labels)
{
    if (n < 0 || n > INT32_MAX || minpts < 1 || !(eps >= 0.0f) || std::isinf(eps))
        return ABX_EINVAL;
    if (n > 0 && (!points || !labels))
        return ABX_EINVAL;
    return ABX_OK;
}

// One clustering; the workspace (work_bytes(n)) is `ws_given` when the caller
// carved it out of a larger block, else it is taken from the pool here.
static abx_status dbscan_run(const float *points, int64_t n, float eps, int32_t minpts, int32_t *labels,
                             const abx_params *params, abx_stream stream, void *ws_given);

abx_status abx_dbscan_ex(const float *points, int64_t n, float eps, int32_t minpts, int32_t *labels,
                         const abx_params *params, abx_stream stream)
{
    return dbscan_run(points, n, eps, minpts, labels, params, stream, nullptr);
}

static abx_status dbscan_run(const float *points, int64_t n, float eps, int32_t minpts, int32_t *labels,
                             const abx_params *params, abx_stream stream, void *ws_given)
{
    abx_status rc = check_args(points, n, eps, minpts, labels);
    if (rc != ABX_OK)
        return rc;
    Params p;
    abx_params tuned;
    if (!params && n > 0 && tune_lookup(n, minpts, &tuned))
        params = &tuned;  // the autotuner's choice for this size class
    if ((rc = resolve_params(params, p)) != ABX_OK)
        return rc;
    if (n == 0)
        return ABX_OK;
    DeviceCtx *ctx;
    if ((rc = device_ctx(&ctx)) != ABX_OK)
        return rc;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    void *ws = ws_given;
    if (!ws && cudaMallocFromPoolAsync(&ws, work_bytes(n), ctx->pool, s) != cudaSuccess) {
        cudaGetLastError();
        return ABX_ENOMEM;
    }
    Work w;
    work_carve(w, ws, n, 1);
    w.n_sms = ctx->n_sms;
    w.dev_status = ctx->status;
    w.any_fof = minpts <= 2;
    w.any_dbscan = !w.any_fof;
    if (g_prof_on.load() == 2) {
        std::lock_guard<std::mutex> lk(g_prof_mu);
        if (!g_stats_dev && cudaMalloc(&g_stats_dev, 8 * sizeof(unsigned long long)) != cudaSuccess) {
            g_stats_dev = nullptr;
            cudaGetLastError();
        }
        if (g_stats_dev) {
            cudaMemsetAsync(g_stats_dev, 0, 8 * sizeof(unsigned long long), s);
            w.stats = g_stats_dev;
        }
    }
    prof_begin(s);
    stage_segments_single(w, eps, minpts, s);
    run_stages(w, points, labels, p, s);
    if (w.stats)
        cudaMemcpyAsync(g_stats_host, g_stats_dev, 8 * sizeof(unsigned long long), cudaMemcpyDeviceToHost, s);
    cudaError_t e = cudaGetLastError();
    if (!ws_given)
        cudaFreeAsync(ws, s);
    return cuda_status(e);
}

abx_status abx_dbscan(const float *points, int64_t n, float eps, int32_t minpts, int32_t *labels,
                      abx_stream stream)
{
    return abx_dbscan_ex(points, n, eps, minpts, labels, nullptr, stream);
}

// ---- the whole clustering of one fixed input as a CUDA graph ----------------------

struct abx_graph {
    int device = -1;
    void *ws = nullptr;           // the graph's own workspace (cudaMalloc)
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    cudaEvent_t last = nullptr;   // recorded after every replay
    unsigned long long launches = 0;  // kernels per replay
};

static void graph_free(abx_graph *g)
{
    if (g->last)
        cudaEventDestroy(g->last);
    if (g->exec)
        cudaGraphExecDestroy(g->exec);
    if (g->graph)
        cudaGraphDestroy(g->graph);
    if (g->ws)
        cudaFree(g->ws);
    delete g;
}

abx_status abx_graph_create(const float *points, int64_t n, float eps, int32_t minpts, int32_t *labels,
                            const abx_params *params, abx_graph **out)
{
    if (!out)
        return ABX_EINVAL;
    *out = nullptr;
    abx_status rc = check_args(points, n, eps, minpts, labels);
    if (rc != ABX_OK || n == 0)
        return n == 0 ? ABX_EINVAL : rc;
    Params p;
    abx_params tuned;
    if (!params && tune_lookup(n, minpts, &tuned))
        params = &tuned;
    if ((rc = resolve_params(params, p)) != ABX_OK)
        return rc;
    DeviceCtx *ctx;
    if ((rc = device_ctx(&ctx)) != ABX_OK)
        return rc;
    abx_graph *g = new abx_graph;
    cudaGetDevice(&g->device);
    if (cudaMalloc(&g->ws, work_bytes(n)) != cudaSuccess) {
        cudaGetLastError();
        g->ws = nullptr;
        graph_free(g);
        return ABX_ENOMEM;
    }
    Work w;
    work_carve(w, g->ws, n, 1);
    w.n_sms = ctx->n_sms;
    w.dev_status = ctx->status;
    w.any_fof = minpts <= 2;
    w.any_dbscan = !w.any_fof;
    cudaStream_t cs;
    if (cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking) != cudaSuccess) {
        cudaGetLastError();
        graph_free(g);
        return ABX_ECUDA;
    }
    const unsigned long long l0 = t_launches;
    cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
        t_capturing = true;
        stage_segments_single(w, eps, minpts, cs);
        run_stages(w, points, labels, p, cs);
        t_capturing = false;
        e = cudaStreamEndCapture(cs, &g->graph);
    }
    g->launches = t_launches - l0;
    if (e == cudaSuccess)
        e = cudaGraphInstantiate(&g->exec, g->graph, 0);
    if (e == cudaSuccess)
        e = cudaEventCreateWithFlags(&g->last, cudaEventDisableTiming);
    cudaStreamDestroy(cs);
    if (e != cudaSuccess) {
        cudaGetLastError();
        graph_free(g);
        return ABX_ECUDA;
    }
    *out = g;
    return ABX_OK;
}

abx_status abx_graph_launch(abx_graph *g, abx_stream stream)
{
    if (!g || !g->exec)
        return ABX_EINVAL;
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev != g->device)
        return ABX_EINVAL;
    if (cudaGraphLaunch(g->exec, reinterpret_cast<cudaStream_t>(stream)) != cudaSuccess ||
        cudaEventRecord(g->last, reinterpret_cast<cudaStream_t>(stream)) != cudaSuccess) {
        cudaGetLastError();
        return ABX_ECUDA;
    }
    note_launch((int)g->launches);
    return ABX_OK;
}

abx_status abx_graph_destroy(abx_graph *g)
{
    if (!g)
        return ABX_EINVAL;
    int cur = -1;
    const int dev = g->device;
    cudaGetDevice(&cur);
    if (cur != dev)
        cudaSetDevice(dev);
    // no replay may still use the workspace: replays are kept in order on one
    // stream, so waiting for the last one's event is enough (other work on
    // the device is not waited for)
    if (g->last)
        cudaEventSynchronize(g->last);
    graph_free(g);
    if (cur >= 0 && cur != dev)
        cudaSetDevice(cur);
    return ABX_OK;
}

abx_status abx_dbscan_host(const float *points_host, int64_t n, float eps, int32_t minpts, int32_t *labels_host,
                           abx_stream stream)
{
    abx_status rc = check_args(points_host, n, eps, minpts, labels_host);
    if (rc != ABX_OK || n == 0)
        return rc;
    DeviceCtx *ctx;
    if ((rc = device_ctx(&ctx)) != ABX_OK)
        return rc;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    // one block of the same size on every call (points, labels, workspace):
    // the pool hands the same memory back instead of growing
    const size_t b_pts = align256((size_t)n * 3 * sizeof(float)), b_lab = align256((size_t)n * sizeof(int32_t));
    char *blk = nullptr;
    if (cudaMallocFromPoolAsync((void **)&blk, b_pts + b_lab + work_bytes(n), ctx->pool, s) != cudaSuccess) {
        cudaGetLastError();
        return ABX_ENOMEM;
    }
    float *dp = reinterpret_cast<float *>(blk);
    int32_t *dl = reinterpret_cast<int32_t *>(blk + b_pts);
    cudaMemcpyAsync(dp, points_host, (size_t)n * 3 * sizeof(float), cudaMemcpyHostToDevice, s);
    rc = dbscan_run(dp, n, eps, minpts, dl, nullptr, stream, blk + b_pts + b_lab);
    if (rc == ABX_OK)
        cudaMemcpyAsync(labels_host, dl, (size_t)n * sizeof(int32_t), cudaMemcpyDeviceToHost, s);
    cudaFreeAsync(blk, s);
    cudaError_t e = cudaStreamSynchronize(s);
    if (rc != ABX_OK)
        return rc;
    return cuda_status(e == cudaSuccess ? cudaGetLastError() : e);
}

abx_status abx_device_status(abx_stream stream)
{
    DeviceCtx *ctx;
    abx_status rc = device_ctx(&ctx);
    if (rc != ABX_OK)
        return rc;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    if (cudaStreamSynchronize(s) != cudaSuccess)
        return ABX_ECUDA;
    unsigned v = 0, v_noalloc = 0;
    if (cudaMemcpy(&v, ctx->status, sizeof(v), cudaMemcpyDeviceToHost) != cudaSuccess)
        return ABX_ECUDA;
    if (v && cudaMemset(ctx->status, 0, sizeof(unsigned)) != cudaSuccess)
        return ABX_ECUDA;
    if (noalloc_take_status(&v_noalloc) != ABX_OK)
        return ABX_ECUDA;
    v |= v_noalloc;
    if (v & DEV_INTERNAL)
        return ABX_EINTERNAL;
    if (v & DEV_TIMEOUT)
        return ABX_ETIMEOUT;
    if (v & DEV_NONFINITE)
        return ABX_ENONFINITE;
    return ABX_OK;
}

abx_status abx_selftest_wait_timeout(int32_t spin_limit, abx_stream stream)
{
    if (spin_limit < 1 || spin_limit > (1 << 24))
        return ABX_EINVAL;
    DeviceCtx *ctx;
    abx_status rc = device_ctx(&ctx);
    if (rc != ABX_OK)
        return rc;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    constexpr int TILES = 4;
    unsigned long long *lb = nullptr;
    if (cudaMallocFromPoolAsync((void **)&lb, (TILES + 1) * sizeof(unsigned long long), ctx->pool, s) !=
        cudaSuccess) {
        cudaGetLastError();
        return ABX_ENOMEM;
    }
    cudaMemsetAsync(lb, 0, (TILES + 1) * sizeof(unsigned long long), s);  // nothing published
    k_selftest_lookback<<<1, 32, 0, s>>>(lb, TILES - 1, spin_limit, ctx->status, lb + TILES);
    note_launch();
    cudaFreeAsync(lb, s);
    return cuda_status(cudaGetLastError());
}

static const char *k_stage_names[ST_NUM] = {"bounds", "morton", "bucket", "sort", "gather", "cells", "leaves",
                                           "build", "candidates", "count", "union", "border", "finalize"};

abx_status abx_profile_enable(int32_t on)
{
    if (on < 0 || on > 2)
        return ABX_EINVAL;
    g_prof_on.store(on);
    return ABX_OK;
}

int32_t abx_profile_stage_count(void) { return ST_NUM; }

const char *abx_profile_stage_name(int32_t i) { return (i >= 0 && i < ST_NUM) ? k_stage_names[i] : ""; }

abx_status abx_profile_read(float *ms, int32_t n)
{
    if (!ms || n < 1)
        return ABX_EINVAL;
    std::lock_guard<std::mutex> lk(g_prof_mu);
    if (!g_ev_ready || !g_ev_marked[0])
        return ABX_EINVAL;
    if (cudaStreamSynchronize(g_prof_stream) != cudaSuccess)
        return ABX_ECUDA;
    int prev = 0;
    for (int i = 0; i < ST_NUM && i < n; i++) {
        ms[i] = 0.0f;
        if (g_ev_marked[i + 1]) {
            float t = 0.0f;
            if (cudaEventElapsedTime(&t, g_ev[prev], g_ev[i + 1]) != cudaSuccess)
                return ABX_ECUDA;
            ms[i] = t;
            prev = i + 1;
        }
    }
    return ABX_OK;
}

unsigned long long abx_launch_count(void) { return g_launches.load(); }

abx_status abx_profile_traversal(int64_t *out, int32_t n)
{
    if (!out || n < 1)
        return ABX_EINVAL;
    std::lock_guard<std::mutex> lk(g_prof_mu);
    if (!g_stats_dev || !g_ev_marked[0])
        return ABX_EINVAL;
    if (cudaStreamSynchronize(g_prof_stream) != cudaSuccess)
        return ABX_ECUDA;
    for (int i = 0; i < n && i < 5; i++)
        out[i] = (int64_t)g_stats_host[i];
    return ABX_OK;
}

abx_status abx_profile_counters(int64_t *out, int32_t n)
{
    if (!out || n < 1)
        return ABX_EINVAL;
    std::lock_guard<std::mutex> lk(g_prof_mu);
    if (!g_prof_state || !g_ev_marked[0])  // the stream itself may be the NULL default stream
        return ABX_EINVAL;
    if (cudaStreamSynchronize(g_prof_stream) != cudaSuccess)
        return ABX_ECUDA;
    const State &st = *g_prof_state;
    int64_t v[7] = {st.n_active, st.bits, st.dense_ok, st.n_cells, st.n_leaves, st.root, st.key32 ? 32 : 64};
    for (int i = 0; i < n && i < 7; i++)
        out[i] = v[i];
    return ABX_OK;
}

abx_status abx_dbscan_batch(const float *points, const int64_t *offsets, int32_t nseg, const float *eps,
                            const int32_t *minpts, int32_t *labels, abx_stream stream)
{
    return abx_dbscan_batch_ex(points, offsets, nseg, eps, minpts, labels, nullptr, stream);
}

abx_status abx_dbscan_batch_ex(const float *points, const int64_t *offsets, int32_t nseg, const float *eps,
                               const int32_t *minpts, int32_t *labels, const abx_params *params, abx_stream stream)
{
    if (nseg < 0 || (nseg > 0 && (!offsets || !eps || !minpts)))
        return ABX_EINVAL;
    if (nseg == 0)
        return ABX_OK;
    if (offsets[0] != 0)
        return ABX_EINVAL;
    for (int32_t k = 0; k < nseg; k++) {
        if (offsets[k + 1] < offsets[k])
            return ABX_EINVAL;
        abx_status rc = check_args(points, offsets[k + 1] - offsets[k], eps[k], minpts[k], labels);
        if (rc != ABX_OK)
            return rc;
    }
    const int64_t n = offsets[nseg];
    if (n > INT32_MAX || nseg > (1 << 24))
        return ABX_EINVAL;
    if (n == 0)
        return ABX_OK;
    bool any_dbscan = false;
    for (int32_t k = 0; k < nseg; k++)
        any_dbscan |= minpts[k] > 2;
    abx_params tuned;
    if (!params && tune_lookup_batch(n, any_dbscan, &tuned))
        params = &tuned;  // the autotuner's choice for batches of this class
    Params p;
    if (resolve_params(params, p) != ABX_OK)
        return ABX_EINVAL;
    if (nseg == 1)
        return abx_dbscan_ex(points, n, eps[0], minpts[0], labels, params, stream);
    DeviceCtx *ctx;
    abx_status rc = device_ctx(&ctx);
    if (rc != ABX_OK)
        return rc;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    void *ws = nullptr;
    if (cudaMallocFromPoolAsync(&ws, work_bytes(n, nseg), ctx->pool, s) != cudaSuccess) {
        cudaGetLastError();
        return ABX_ENOMEM;
    }
    Work w;
    work_carve(w, ws, n, nseg);
    w.n_sms = ctx->n_sms;
    w.dev_status = ctx->status;
    // segment table: int32 offsets, eps, minPts, staged in local (pageable)
    // copies, so the caller's host arrays -- pinned or not -- are read before
    // this call returns (a copy from pageable memory has consumed its source
    // when cudaMemcpyAsync returns)
    std::vector<int> off32((size_t)nseg + 1);
    for (int32_t k = 0; k <= nseg; k++)
        off32[k] = (int)offsets[k];
    std::vector<float> eps_v(eps, eps + nseg);
    std::vector<int> minpts_v(minpts, minpts + nseg);
    for (int32_t k = 0; k < nseg; k++) {
        w.any_fof |= minpts[k] <= 2;
        w.any_dbscan |= minpts[k] > 2;
    }
    cudaMemcpyAsync(w.seg_off, off32.data(), off32.size() * sizeof(int), cudaMemcpyHostToDevice, s);
    cudaMemcpyAsync(w.seg_eps_in, eps_v.data(), (size_t)nseg * sizeof(float), cudaMemcpyHostToDevice, s);
    cudaMemcpyAsync(w.seg_minpts_in, minpts_v.data(), (size_t)nseg * sizeof(int), cudaMemcpyHostToDevice, s);
    int seg_bits = 0;
    while ((1ll << seg_bits) < (long long)nseg)
        seg_bits++;
    prof_begin(s);
    stage_segments_batch(w, w.seg_eps_in, w.seg_minpts_in, seg_bits, s);
    run_stages(w, points, labels, p, s);
    cudaError_t e = cudaGetLastError();
    cudaFreeAsync(ws, s);
    return cuda_status(e);
}

}  // extern "C"
