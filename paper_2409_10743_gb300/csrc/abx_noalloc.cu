// Clustering without any device allocation, for callers that cannot allocate.
//
// Some callers may not allocate device memory at all: an in-situ analysis
// hook inside a simulation that has already claimed nearly all of the GPU's
// memory for its own particle arrays and only lends out what it planned for,
// or code that runs where allocation calls are not permitted.  abx_dbscan
// draws its workspace from a pool and would allocate; this entry point runs
// the same stages over a workspace that is a fixed array of device memory,
// reserved once when the library is loaded on a device.
//
// The array is shared by every call on a device and keeps whatever the last
// call left in it; every buffer that must start cleared is cleared by the
// stages themselves.  Calls whose work overlaps on the GPU (different streams,
// or several host threads at once) race on the array, so they must be
// serialised by the caller.
#include <mutex>

#include "work.cuh"

namespace abx {

// Largest input this entry point accepts, and the workspace reserved for it
// (the workspace of 65,536 points is a little over 10 MiB).
constexpr int64_t NOALLOC_MAX_POINTS = 65536;
constexpr size_t NOALLOC_BYTES = (size_t)12 << 20;

static __device__ __align__(256) unsigned char g_noalloc_ws[NOALLOC_BYTES];
static __device__ __align__(256) unsigned g_noalloc_status;

struct NoAllocDevice {
    bool ready = false;
    void *ws = nullptr;
    unsigned *status = nullptr;
    int n_sms = 0;
};

static std::mutex g_noalloc_mu;
static NoAllocDevice g_noalloc_dev[64];

// Per device, once, with that device current: the device addresses of the
// static arrays (in host code their names are only host-side stand-ins) and
// the kernel attributes.  Nothing here allocates.
static abx_status noalloc_setup(NoAllocDevice **out)
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64)
        return ABX_ECUDA;
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    NoAllocDevice &d = g_noalloc_dev[dev];
    if (!d.ready) {
        if (work_bytes(NOALLOC_MAX_POINTS, 1) > NOALLOC_BYTES)
            return ABX_EINTERNAL;
        if (cudaGetSymbolAddress(&d.ws, g_noalloc_ws) != cudaSuccess || !d.ws)
            return ABX_ECUDA;
        if (cudaGetSymbolAddress((void **)&d.status, g_noalloc_status) != cudaSuccess || !d.status)
            return ABX_ECUDA;
        if (cudaDeviceGetAttribute(&d.n_sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
            return ABX_ECUDA;
        kernels_init_device();
        tree_init_device();
        cluster_init_device();
        if (cudaGetLastError() != cudaSuccess)
            return ABX_ECUDA;
        d.ready = true;
    }
    *out = &d;
    return ABX_OK;
}

// The status word of this entry point on the current device, read and
// cleared (0 if the entry point never ran here).  abx_device_status folds it
// into the library's status, after waiting for the caller's stream.
abx_status noalloc_take_status(unsigned *out)
{
    *out = 0;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64)
        return ABX_ECUDA;
    unsigned *status = nullptr;
    {
        std::lock_guard<std::mutex> lk(g_noalloc_mu);
        if (g_noalloc_dev[dev].ready)
            status = g_noalloc_dev[dev].status;
    }
    if (!status)
        return ABX_OK;
    if (cudaMemcpy(out, status, sizeof(unsigned), cudaMemcpyDeviceToHost) != cudaSuccess)
        return ABX_ECUDA;
    if (*out && cudaMemset(status, 0, sizeof(unsigned)) != cudaSuccess)
        return ABX_ECUDA;
    return ABX_OK;
}

}  // namespace abx

using namespace abx;

extern "C" abx_status abx_dbscan_noalloc(const float *points, int64_t n, float eps, int32_t minpts,
                                         int32_t *labels, abx_stream stream)
{
    if (n < 0 || n > NOALLOC_MAX_POINTS || minpts < 1 || !(eps >= 0.0f) || eps == __builtin_inff())
        return ABX_EINVAL;
    if (n == 0)
        return ABX_OK;
    if (!points || !labels)
        return ABX_EINVAL;
    NoAllocDevice *d;
    abx_status rc = noalloc_setup(&d);
    if (rc != ABX_OK)
        return rc;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    Work w;
    work_carve(w, d->ws, n, 1);
    w.n_sms = d->n_sms;
    w.dev_status = d->status;
    w.any_fof = minpts <= 2;
    w.any_dbscan = !w.any_fof;
    Params p;
    resolve_params(nullptr, p);  // the library defaults
    stage_segments_single(w, eps, minpts, s);
    stage_bounds_quant(w, points, p, s);
    stage_morton_sort(w, points, s);
    stage_gather(w, points, s);
    stage_cells_leaves(w, p, s);
    stage_hierarchy(w, s);
    stage_cluster(w, p, labels, s);
    return cudaGetLastError() == cudaSuccess ? ABX_OK : ABX_ECUDA;
}
