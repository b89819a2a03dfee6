// Autotuner: pick the tuning parameters (leaf size, traversal block size,
// dense cells on or off, minimum dense-cell size) by timing candidates on the
// caller's own input, and remember the winner per device for its size class
// (friends-of-friends or DBSCAN, floor(log2 n)).  abx_dbscan without explicit
// parameters uses the remembered choice.  Labels never depend on any of it.
#include <cmath>
#include <mutex>
#include <vector>

#include "work.cuh"

namespace abx {

struct TuneEntry {
    bool set = false;
    abx_params p{};
};

static std::mutex g_tune_mu;
static TuneEntry g_tune[64][2][33];

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

bool tune_lookup(int64_t n, int32_t minpts, abx_params *out)
{
    int dev;
    if (!current_device(&dev))
        return false;
    std::lock_guard<std::mutex> lk(g_tune_mu);
    const TuneEntry &e = g_tune[dev][minpts > 2][size_class(n)];
    if (e.set)
        *out = e.p;
    return e.set;
}

static void tune_store(int64_t n, int32_t minpts, const abx_params &p)
{
    int dev;
    if (!current_device(&dev))
        return;
    std::lock_guard<std::mutex> lk(g_tune_mu);
    TuneEntry &e = g_tune[dev][minpts > 2][size_class(n)];
    e.set = true;
    e.p = p;
}

}  // namespace abx

using namespace abx;

extern "C" {

abx_status abx_autotune(const float *points, int64_t n, float eps, int32_t minpts, int32_t *labels,
                        abx_params *best, abx_stream stream)
{
    if (n < 1 || n > INT32_MAX || !points || !labels || minpts < 1 || !(eps >= 0.0f) || std::isinf(eps))
        return ABX_EINVAL;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)
        return ABX_ECUDA;
    auto time_of = [&](const abx_params &p, float *ms) -> abx_status {
        abx_status rc = abx_dbscan_ex(points, n, eps, minpts, labels, &p, stream);  // warm-up
        float bestms = INFINITY;
        for (int r = 0; rc == ABX_OK && r < 2; r++) {
            cudaEventRecord(e0, s);
            rc = abx_dbscan_ex(points, n, eps, minpts, labels, &p, stream);
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
    abx_params cur{};
    float cur_ms = INFINITY;
    abx_status rc = ABX_OK;
    // one axis at a time, keeping the best so far
    const int leafs[] = {2, 4, 8};
    const int blocks[] = {128, 256, 512};
    const int denses[][2] = {{1, 0}, {1, 16}, {-1, 0}};
    for (int v : leafs) {
        abx_params p = cur;
        p.leaf_size = v;
        float ms;
        if ((rc = time_of(p, &ms)) != ABX_OK)
            break;
        if (ms < cur_ms) {
            cur_ms = ms;
            cur = p;
        }
    }
    for (int k = 0; rc == ABX_OK && k < 3; k++) {
        abx_params p = cur;
        p.block = blocks[k];
        float ms;
        if ((rc = time_of(p, &ms)) != ABX_OK)
            break;
        if (ms < cur_ms) {
            cur_ms = ms;
            cur = p;
        }
    }
    for (int k = 0; rc == ABX_OK && k < 3; k++) {
        abx_params p = cur;
        p.dense_cells = denses[k][0];
        p.dense_min = denses[k][1];
        float ms;
        if ((rc = time_of(p, &ms)) != ABX_OK)
            break;
        if (ms < cur_ms) {
            cur_ms = ms;
            cur = p;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc != ABX_OK)
        return rc;
    tune_store(n, minpts, cur);
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
    tune_store(n, minpts, *p);
    return ABX_OK;
}

}  // extern "C"
