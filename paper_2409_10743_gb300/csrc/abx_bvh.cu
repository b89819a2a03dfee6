// The hierarchy as a handle of its own: build once, then run early-terminated
// range queries against it -- counts capped at a value, and the first hit
// (paper, subsections "Callbacks" and "Early termination": a callback's return
// value may stop a query's traversal, e.g. once a count is reached or a
// neighbour is found).
#include <cstring>

#include "work.cuh"

namespace abx {
abx_status bvh_device_ctx(cudaMemPool_t *pool, unsigned **status, int *n_sms);
}

using namespace abx;


namespace abx {

__global__ void k_count_ext(const float *__restrict__ q, int64_t nq, const State *__restrict__ st,
                            const float4 *__restrict__ spts, const float4 *__restrict__ nodes,
                            const int *__restrict__ leaf_first, float e2, int cap, int32_t *counts,
                            unsigned *dev_status)
{
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= nq)
        return;
    const float px = __ldg(q + 3 * k), py = __ldg(q + 3 * k + 1), pz = __ldg(q + 3 * k + 2);
    const int L = st->n_leaves;
    int cnt = 0, node = st->root;
    unsigned steps = 0;
    while (node != SENTINEL && cnt < cap) {
        if ((unsigned)node >= (unsigned)(2 * L - 1) || ++steps > (unsigned)(2 * L)) {
            atomicOr(dev_status, DEV_INTERNAL);
            break;
        }
        const float4 lo = __ldg(nodes + 2 * (size_t)node), hi = __ldg(nodes + 2 * (size_t)node + 1);
        if (box_dist2_rn(px, py, pz, lo, hi) <= e2) {
            if (node < L - 1) {
                node = __float_as_int(lo.w);
                continue;
            }
            const int s = (int)(__float_as_uint(lo.w) & ~DENSE_BIT);
            const int e = leaf_first[node - (L - 1) + 1];
            for (int j = s; j < e && cnt < cap; j++) {
                float4 p = __ldg(spts + j);
                if (dist2_rn(px, py, pz, p.x, p.y, p.z) <= e2)
                    cnt++;
            }
        }
        node = __float_as_int(hi.w);
    }
    counts[k] = cnt;
}

// First hit: the traversal of k_count_ext stopped at the first point within
// eps; hits[k] = that point's original index, -1 if there is none.  Which
// neighbour is found depends on the hierarchy (the first in its pre-order),
// so only "a neighbour, or none" is the contract.
__global__ void k_first_hit(const float *__restrict__ q, int64_t nq, const State *__restrict__ st,
                            const float4 *__restrict__ spts, const float4 *__restrict__ nodes,
                            const int *__restrict__ leaf_first, float e2, int32_t *hits, unsigned *dev_status)
{
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= nq)
        return;
    const float px = __ldg(q + 3 * k), py = __ldg(q + 3 * k + 1), pz = __ldg(q + 3 * k + 2);
    const int L = st->n_leaves;
    int hit = -1, node = st->root;
    unsigned steps = 0;
    while (node != SENTINEL && hit < 0) {
        if ((unsigned)node >= (unsigned)(2 * L - 1) || ++steps > (unsigned)(2 * L)) {
            atomicOr(dev_status, DEV_INTERNAL);
            break;
        }
        const float4 lo = __ldg(nodes + 2 * (size_t)node), hi = __ldg(nodes + 2 * (size_t)node + 1);
        if (box_dist2_rn(px, py, pz, lo, hi) <= e2) {
            if (node < L - 1) {
                node = __float_as_int(lo.w);
                continue;
            }
            const int s = (int)(__float_as_uint(lo.w) & ~DENSE_BIT);
            const int e = leaf_first[node - (L - 1) + 1];
            for (int j = s; j < e; j++) {
                const float4 p = __ldg(spts + j);
                if (dist2_rn(px, py, pz, p.x, p.y, p.z) <= e2) {
                    hit = __float_as_int(p.w);
                    break;
                }
            }
        }
        node = __float_as_int(hi.w);
    }
    hits[k] = hit;
}

// Depth of each leaf: descend from the root; internal node p splits leaves
// [.., p] (left) from [p + 1, ..] (right).
__global__ void k_levels(const State *__restrict__ st, const float4 *__restrict__ nodes,
                         const int *__restrict__ right_of, int *levels)
{
    const int L = st->n_leaves;
    int best = 0;
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < L; t += gridDim.x * blockDim.x) {
        int node = st->root, d = 0;
        while (node < L - 1 && node >= 0 && d <= L) {
            node = t <= node ? __float_as_int(__ldg(nodes + 2 * (size_t)node).w) : right_of[node];
            d++;
        }
        best = max(best, d + 1);
    }
    atomicMax(levels, best);
}

}  // namespace abx

extern "C" {

abx_status abx_bvh_build(const float *points, int64_t n, const abx_params *params, abx_bvh **out,
                         abx_stream stream)
{
    if (!out || !points || n < 1 || n > INT32_MAX)
        return ABX_EINVAL;
    Params p;
    if (resolve_params(params, p) != ABX_OK)
        return ABX_EINVAL;
    p.dense = 0;  // no eps here: the grid only resolves the points
    cudaMemPool_t pool;
    unsigned *status;
    int n_sms;
    abx_status rc = bvh_device_ctx(&pool, &status, &n_sms);
    if (rc != ABX_OK)
        return rc;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    abx_bvh *h = new abx_bvh();
    h->stream = s;
    h->pool = pool;
    if (cudaMallocFromPoolAsync(&h->ws, work_bytes(n), pool, s) != cudaSuccess) {
        cudaGetLastError();
        delete h;
        return ABX_ENOMEM;
    }
    work_carve(h->w, h->ws, n);
    h->w.n_sms = n_sms;
    h->w.dev_status = status;
    h->w.any_fof = true;
    stage_segments_single(h->w, 0.0f, 2, s);
    stage_bounds_quant(h->w, points, p, s);
    stage_morton_sort(h->w, points, s);
    stage_gather(h->w, points, s);
    stage_cells_leaves(h->w, p, s);
    stage_hierarchy(h->w, s);
    if (cudaGetLastError() != cudaSuccess) {
        cudaFreeAsync(h->ws, s);
        delete h;
        return ABX_ECUDA;
    }
    *out = h;
    return ABX_OK;
}

abx_status abx_bvh_count(const abx_bvh *bvh, const float *queries, int64_t nq, float eps, int32_t cap,
                         int32_t *counts, abx_stream stream)
{
    if (!bvh || nq < 0 || nq > INT32_MAX || cap < 1 || !(eps >= 0.0f) || eps == __builtin_inff())
        return ABX_EINVAL;
    if (nq == 0)
        return ABX_OK;
    if (!queries || !counts)
        return ABX_EINVAL;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    const float e2 = eps * eps;
    k_count_ext<<<div_up(nq, 256), 256, 0, s>>>(queries, nq, bvh->w.st, bvh->w.spts, bvh->w.nodes,
                                                bvh->w.leaf_first, e2, cap, counts, bvh->w.dev_status);
    note_launch();
    return cudaGetLastError() == cudaSuccess ? ABX_OK : ABX_ECUDA;
}

abx_status abx_bvh_first_hit(const abx_bvh *bvh, const float *queries, int64_t nq, float eps, int32_t *hits,
                             abx_stream stream)
{
    if (!bvh || nq < 0 || nq > INT32_MAX || !(eps >= 0.0f) || eps == __builtin_inff())
        return ABX_EINVAL;
    if (nq == 0)
        return ABX_OK;
    if (!queries || !hits)
        return ABX_EINVAL;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    const float e2 = eps * eps;
    k_first_hit<<<div_up(nq, 256), 256, 0, s>>>(queries, nq, bvh->w.st, bvh->w.spts, bvh->w.nodes,
                                                bvh->w.leaf_first, e2, hits, bvh->w.dev_status);
    note_launch();
    return cudaGetLastError() == cudaSuccess ? ABX_OK : ABX_ECUDA;
}

abx_status abx_bvh_info(const abx_bvh *bvh, int64_t *n_points, int64_t *n_leaves, int32_t *levels,
                        abx_stream stream)
{
    if (!bvh)
        return ABX_EINVAL;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    int *dlev = nullptr;
    if (cudaMallocFromPoolAsync((void **)&dlev, sizeof(int), bvh->pool, s) != cudaSuccess) {
        cudaGetLastError();
        return ABX_ENOMEM;
    }
    cudaMemsetAsync(dlev, 0, sizeof(int), s);
    k_levels<<<bvh->w.n_sms * 4, 256, 0, s>>>(bvh->w.st, bvh->w.nodes, bvh->w.right_of, dlev);
    int lev = 0, L = 0;
    cudaMemcpyAsync(&lev, dlev, sizeof(int), cudaMemcpyDeviceToHost, s);
    cudaMemcpyAsync(&L, &bvh->w.st->n_leaves, sizeof(int), cudaMemcpyDeviceToHost, s);
    cudaFreeAsync(dlev, s);
    if (cudaStreamSynchronize(s) != cudaSuccess)
        return ABX_ECUDA;
    if (n_points)
        *n_points = bvh->w.n;
    if (n_leaves)
        *n_leaves = L;
    if (levels)
        *levels = lev;
    return ABX_OK;
}

abx_status abx_bvh_destroy(abx_bvh *bvh)
{
    if (!bvh)
        return ABX_EINVAL;
    cudaError_t e = cudaFreeAsync(bvh->ws, bvh->stream);
    delete bvh;
    return e == cudaSuccess ? ABX_OK : ABX_ECUDA;
}

}  // extern "C"
