// Autotuner: pick the tuning parameters (leaf size, traversal block size,
// dense cells on or off and the minimum dense-cell size, how the pair
// traversal is scheduled) by timing candidates on the
// caller's own input, and remember the winner per device for its class:
// single instance or batch, friends-of-friends or DBSCAN, floor(log2 n).
// Clustering calls without explicit parameters use the remembered choice (a
// batch: the batch table, which the serving loop's batches use too).  Labels
// never depend on any of it.  (The paper lists runtime tuning of occupancy
// parameters as future work, section "Conclusions".)
#include <cmath>
#include <functional>
#include <mutex>
#include <vector>

#include "work.cuh"

namespace abx {

struct TuneEntry {
    bool set = false;
    abx_params p{};
};

static std::mutex g_tune_mu;
static TuneEntry g_tune[64][2][2][33];  // [device][batch][DBSCAN][size class]

static int size_class(int64_t n)
{
    int c = 0;
    while (c < 32 && (1ll << (c + 1)) <= n)
        c++;
    return c;
}

static bool current_device(int *dev)
{
    return cudaGetDevice(dev) == cudaSuccess && *dev >= 0 && *dev < 64;
}

static bool lookup(int batch, int64_t n, bool dbscan, abx_params *out)
{
    int dev;
    if (!current_device(&dev))
        return false;
    std::lock_guard<std::mutex> lk(g_tune_mu);
    const TuneEntry &e = g_tune[dev][batch][dbscan][size_class(n)];
    if (e.set)
        *out = e.p;
    return e.set;
}

static void store(int batch, int64_t n, bool dbscan, const abx_params &p)
{
    int dev;
    if (!current_device(&dev))
        return;
    std::lock_guard<std::mutex> lk(g_tune_mu);
    TuneEntry &e = g_tune[dev][batch][dbscan][size_class(n)];
    e.set = true;
    e.p = p;
}

bool tune_lookup(int64_t n, int32_t minpts, abx_params *out) { return lookup(0, n, minpts > 2, out); }
bool tune_lookup_batch(int64_t n, bool any_dbscan, abx_params *out) { return lookup(1, n, any_dbscan, out); }

// One axis at a time, keeping the best so far: each candidate runs once to
// warm up and twice timed with CUDA events on `s`; run(p) enqueues one
// clustering with parameters p.
static abx_status search(const std::function<abx_status(const abx_params &)> &run, cudaStream_t s,
                         abx_params *best)
{
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)
        return ABX_ECUDA;
    auto time_of = [&](const abx_params &p, float *ms) -> abx_status {
        abx_status rc = run(p);  // warm-up
        float bestms = INFINITY;
        for (int r = 0; rc == ABX_OK && r < 2; r++) {
            cudaEventRecord(e0, s);
            rc = run(p);
            cudaEventRecord(e1, s);
            if (cudaEventSynchronize(e1) != cudaSuccess)
                return ABX_ECUDA;
            float t = 0;
            cudaEventElapsedTime(&t, e0, e1);
            bestms = fminf(bestms, t);
        }
        *ms = bestms;
        return rc;
    };
    // each axis: the values tried, applied to a copy of the best so far
    struct Axis {
        int count;
        std::function<void(abx_params &, int)> set;
    };
    const int leafs[] = {2, 4, 8};
    const int blocks[] = {128, 256, 512};
    const int denses[][2] = {{1, 0}, {1, 16}, {-1, 0}};
    const int schedules[] = {1, 2};
    const Axis axes[] = {
        {3, [&](abx_params &p, int k) { p.leaf_size = leafs[k]; }},
        {3, [&](abx_params &p, int k) { p.block = blocks[k]; }},
        {3, [&](abx_params &p, int k) { p.dense_cells = denses[k][0], p.dense_min = denses[k][1]; }},
        {2, [&](abx_params &p, int k) { p.schedule = schedules[k]; }},
    };
    // start from the library defaults, spelled out, so that every field of
    // the pick is explicit even where no candidate beat them
    Params d;
    resolve_params(nullptr, d);
    abx_params cur{};
    cur.leaf_size = d.leaf_size;
    cur.dense_cells = d.dense ? 1 : -1;
    cur.block = d.block;
    cur.dense_min = d.dense_min;
    cur.schedule = d.schedule;
    cur.sort_digit_bits = d.digit_bits;
    float cur_ms = INFINITY;
    abx_status rc = ABX_OK;
    for (const Axis &ax : axes) {
        for (int k = 0; rc == ABX_OK && k < ax.count; k++) {
            abx_params p = cur;
            ax.set(p, k);
            float ms;
            if ((rc = time_of(p, &ms)) != ABX_OK)
                break;
            if (ms < cur_ms) {
                cur_ms = ms;
                cur = p;
            }
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc == ABX_OK)
        *best = cur;
    return rc;
}

}  // namespace abx

using namespace abx;

extern "C" {

abx_status abx_autotune(const float *points, int64_t n, float eps, int32_t minpts, int32_t *labels,
                        abx_params *best, abx_stream stream)
{
    if (n < 1 || n > INT32_MAX || !points || !labels || minpts < 1 || !(eps >= 0.0f) || std::isinf(eps))
        return ABX_EINVAL;
    abx_params cur{};
    abx_status rc = search([&](const abx_params &p) { return abx_dbscan_ex(points, n, eps, minpts, labels, &p, stream); },
                           reinterpret_cast<cudaStream_t>(stream), &cur);
    if (rc != ABX_OK)
        return rc;
    store(0, n, minpts > 2, cur);
    if (best)
        *best = cur;
    return ABX_OK;
}

abx_status abx_autotune_batch(const float *points, const int64_t *offsets, int32_t nseg, const float *eps,
                              const int32_t *minpts, int32_t *labels, abx_params *best, abx_stream stream)
{
    if (nseg < 1 || !offsets || !eps || !minpts || offsets[nseg] < 1)
        return ABX_EINVAL;
    bool any_dbscan = false;
    for (int32_t k = 0; k < nseg; k++)
        any_dbscan |= minpts[k] > 2;
    abx_params cur{};
    abx_status rc = search(
        [&](const abx_params &p) {
            return abx_dbscan_batch_ex(points, offsets, nseg, eps, minpts, labels, &p, stream);
        },
        reinterpret_cast<cudaStream_t>(stream), &cur);
    if (rc != ABX_OK)
        return rc;
    store(1, offsets[nseg], any_dbscan, cur);
    if (best)
        *best = cur;
    return ABX_OK;
}

abx_status abx_tune_get(int64_t n, int32_t minpts, abx_params *out)
{
    if (!out || n < 1 || minpts < 1)
        return ABX_EINVAL;
    return tune_lookup(n, minpts, out) ? ABX_OK : ABX_EINVAL;
}

abx_status abx_tune_set(int64_t n, int32_t minpts, const abx_params *p)
{
    if (!p || n < 1 || minpts < 1)
        return ABX_EINVAL;
    Params check;
    if (resolve_params(p, check) != ABX_OK)
        return ABX_EINVAL;
    store(0, n, minpts > 2, *p);
    return ABX_OK;
}

}  // extern "C"
