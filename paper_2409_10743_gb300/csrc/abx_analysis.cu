// Consumers of the clustering and of the hierarchy.
//
// Per-cluster statistics: the paper's HACC section draws each galaxy found by
// DBSCAN as a circle whose radius is the distance of its farthest particle
// from the centre.  abx_cluster_stats reduces labels to, per cluster, its size,
// centre (mean position) and that radius.
//
// Pair-distance histogram: the paper's "Pair traversal" subsection frames the
// traversal as "find every pair within a radius and apply F(i, j)" with
// examples such as forces and the counts of 2-point correlation functions.
// abx_bvh_pair_histogram is that F: every unordered pair is met once (pair
// traversal from the query's own leaf) and counted in its distance bin.
#include <cmath>
#include <vector>

#include "scan.cuh"
#include "work.cuh"

namespace abx {
abx_status bvh_device_ctx(cudaMemPool_t *pool, unsigned **status, int *n_sms);
}

using namespace abx;


namespace abx {

// ---- per-cluster statistics --------------------------------------------------------

__global__ void k_cs_accumulate(const float *__restrict__ pts, const int32_t *__restrict__ labels, int64_t n,
                                int *cnt, double *sum, unsigned *dev_status)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int l = labels[i];
        if (l < 0)
            continue;
        if ((int64_t)l >= n) {
            atomicOr(dev_status, DEV_INTERNAL);
            continue;
        }
        atomicAdd(cnt + l, 1);
        atomicAdd(sum + 3 * (size_t)l, (double)pts[3 * i]);
        atomicAdd(sum + 3 * (size_t)l + 1, (double)pts[3 * i + 1]);
        atomicAdd(sum + 3 * (size_t)l + 2, (double)pts[3 * i + 2]);
    }
}

struct ClusterFlag {
    const int *cnt;
    __device__ bool operator()(int64_t l) const { return cnt[l] > 0; }
};

__global__ void k_cs_centres(const State *st, const int *__restrict__ first, const int *__restrict__ cnt,
                             const double *__restrict__ sum, int32_t *ids, int32_t *sizes, float *centres,
                             unsigned *rad2)
{
    const int K = st->n_cells;  // clusters found by the scan
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < K; k += gridDim.x * blockDim.x) {
        const int l = first[k];
        const int c = cnt[l];
        ids[k] = l;
        sizes[k] = c;
        for (int a = 0; a < 3; a++)
            centres[3 * (size_t)k + a] = (float)(sum[3 * (size_t)l + a] / (double)c);
        rad2[k] = 0u;
    }
}

__global__ void k_cs_radius(const float *__restrict__ pts, const int32_t *__restrict__ labels, int64_t n,
                            const int *__restrict__ slot, const float *__restrict__ centres, unsigned *rad2)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int l = labels[i];
        if (l < 0 || (int64_t)l >= n)
            continue;
        const int k = slot[l];
        const float d2 = dist2_rn(pts[3 * i], pts[3 * i + 1], pts[3 * i + 2], centres[3 * (size_t)k],
                                  centres[3 * (size_t)k + 1], centres[3 * (size_t)k + 2]);
        atomicMax(rad2 + k, __float_as_uint(d2));  // d2 >= 0: integer order = float order
    }
}

__global__ void k_cs_sqrt(const State *st, const unsigned *__restrict__ rad2, float *radii)
{
    const int K = st->n_cells;
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < K; k += gridDim.x * blockDim.x)
        radii[k] = sqrtf(__uint_as_float(rad2[k]));
}

// ---- pair-distance histogram over a hierarchy -------------------------------------

constexpr int MAX_BINS = 256;

struct Edges2 {
    float e2[MAX_BINS + 1];  // fl(r_b * r_b)
    int nbins;
};

__global__ void __launch_bounds__(256) k_pair_hist(int64_t n, const State *__restrict__ st,
                                                   const float4 *__restrict__ spts, const float4 *__restrict__ nodes,
                                                   const int *__restrict__ leaf_of, const int *__restrict__ leaf_first,
                                                   const Edges2 edges, unsigned long long *hist, unsigned *dev_status)
{
    __shared__ unsigned sh[MAX_BINS];
    __shared__ float se2[MAX_BINS + 1];
    const int nb = edges.nbins;
    for (int b = threadIdx.x; b < nb; b += blockDim.x)
        sh[b] = 0;
    for (int b = threadIdx.x; b <= nb; b += blockDim.x)
        se2[b] = edges.e2[b];
    __syncthreads();
    const float emax = se2[nb], emin = se2[0];
    const int L = st->n_leaves;
    const int64_t i64 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i64 < n) {
        const int i = (int)i64;
        const float4 p = spts[i];
        auto bin = [&](float d2) {
            if (d2 <= emin || d2 > emax)
                return;
            int lo = 0, hi = nb - 1;  // the b with e2[b] < d2 <= e2[b + 1]
            while (lo < hi) {
                const int mid = (lo + hi) >> 1;
                if (d2 <= se2[mid + 1])
                    hi = mid;
                else
                    lo = mid + 1;
            }
            atomicAdd(sh + lo, 1u);
        };
        const int my_leaf = L - 1 + leaf_of[i];
        const int e_own = leaf_first[leaf_of[i] + 1];
        for (int j = i + 1; j < e_own; j++) {
            const float4 q = __ldg(spts + j);
            bin(dist2_rn(p.x, p.y, p.z, q.x, q.y, q.z));
        }
        int node = __float_as_int(__ldg(nodes + 2 * (size_t)my_leaf + 1).w);
        unsigned steps = 0;
        while (node != SENTINEL) {
            if ((unsigned)node >= (unsigned)(2 * L - 1) || ++steps > (unsigned)(2 * L)) {
                atomicOr(dev_status, DEV_INTERNAL);
                break;
            }
            const float4 lo = __ldg(nodes + 2 * (size_t)node), hi = __ldg(nodes + 2 * (size_t)node + 1);
            if (box_dist2_rn(p.x, p.y, p.z, lo, hi) <= emax) {
                if (node < L - 1) {
                    node = __float_as_int(lo.w);
                    continue;
                }
                const int s = (int)(__float_as_uint(lo.w) & ~DENSE_BIT);
                const int e = leaf_first[node - (L - 1) + 1];
                for (int j = s; j < e; j++) {
                    const float4 q = __ldg(spts + j);
                    bin(dist2_rn(p.x, p.y, p.z, q.x, q.y, q.z));
                }
            }
            node = __float_as_int(hi.w);
        }
    }
    __syncthreads();
    for (int b = threadIdx.x; b < nb; b += blockDim.x)
        if (sh[b])
            atomicAdd(hist + b, (unsigned long long)sh[b]);
}

}  // namespace abx

extern "C" {

abx_status abx_cluster_stats(const float *points, const int32_t *labels, int64_t n, int32_t *n_clusters,
                             int32_t *ids, int32_t *sizes, float *centres, float *radii, abx_stream stream)
{
    if (!n_clusters || n < 0 || n > INT32_MAX)
        return ABX_EINVAL;
    *n_clusters = 0;
    if (n == 0)
        return ABX_OK;
    if (!points || !labels || !ids || !sizes || !centres || !radii)
        return ABX_EINVAL;
    cudaMemPool_t pool;
    unsigned *status;
    int n_sms;
    abx_status rc = bvh_device_ctx(&pool, &status, &n_sms);
    if (rc != ABX_OK)
        return rc;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    const size_t N = (size_t)n;
    const size_t scan_tiles = (size_t)div_up(n, SCAN_TILE);
    const size_t bytes = sizeof(State) + 256 + N * (sizeof(int) * 2 + sizeof(double) * 3 + sizeof(unsigned)) +
                         (N + 1) * sizeof(int) + scan_tiles * sizeof(unsigned long long) + 6 * 256;
    char *ws = nullptr;
    if (cudaMallocFromPoolAsync((void **)&ws, bytes, pool, s) != cudaSuccess) {
        cudaGetLastError();
        return ABX_ENOMEM;
    }
    size_t off = 0;
    auto take = [&](size_t b) {
        char *p = ws + off;
        off = (off + b + 255) & ~(size_t)255;
        return p;
    };
    State *st = (State *)take(sizeof(State));
    int *cnt = (int *)take(N * sizeof(int));
    double *sum = (double *)take(N * 3 * sizeof(double));
    int *slot = (int *)take(N * sizeof(int));
    int *first = (int *)take((N + 1) * sizeof(int));
    unsigned *rad2 = (unsigned *)take(N * sizeof(unsigned));
    unsigned long long *lb = (unsigned long long *)take(scan_tiles * sizeof(unsigned long long));
    cudaMemsetAsync(st, 0, sizeof(State), s);
    cudaMemsetAsync(cnt, 0, N * sizeof(int), s);
    cudaMemsetAsync(sum, 0, N * 3 * sizeof(double), s);
    cudaMemsetAsync(lb, 0, scan_tiles * sizeof(unsigned long long), s);
    const int g = (int)std::min<int64_t>(div_up(n, 256), (int64_t)n_sms * 8);
    k_cs_accumulate<<<g, 256, 0, s>>>(points, labels, n, cnt, sum, status);
    k_flag_scan<<<(int)scan_tiles, SCAN_THREADS, 0, s>>>(n, FlagItems<ClusterFlag>{{cnt}}, slot, first, &st->n_cells,
                                                         &st->tile_ctr[0], lb, status, st, 0);
    k_cs_centres<<<g, 256, 0, s>>>(st, first, cnt, sum, ids, sizes, centres, rad2);
    k_cs_radius<<<g, 256, 0, s>>>(points, labels, n, slot, centres, rad2);
    k_cs_sqrt<<<g, 256, 0, s>>>(st, rad2, radii);
    note_launch(5);
    int K = 0;
    cudaMemcpyAsync(&K, &st->n_cells, sizeof(int), cudaMemcpyDeviceToHost, s);
    cudaFreeAsync(ws, s);
    if (cudaStreamSynchronize(s) != cudaSuccess)
        return ABX_ECUDA;
    *n_clusters = K;
    return cudaGetLastError() == cudaSuccess ? ABX_OK : ABX_ECUDA;
}

abx_status abx_bvh_pair_histogram(const abx_bvh *bvh, const float *r_edges, int32_t nbins, uint64_t *hist,
                                  abx_stream stream)
{
    if (!bvh || !r_edges || !hist || nbins < 1 || nbins > MAX_BINS)
        return ABX_EINVAL;
    Edges2 e;
    e.nbins = nbins;
    for (int b = 0; b <= nbins; b++) {
        const float r = r_edges[b];
        if (!(r >= 0.0f) || std::isinf(r) || (b > 0 && !(r > r_edges[b - 1])))
            return ABX_EINVAL;
        e.e2[b] = r * r;
    }
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    cudaMemsetAsync(hist, 0, (size_t)nbins * sizeof(uint64_t), s);
    const Work &w = bvh->w;
    k_pair_hist<<<div_up(w.n, 256), 256, 0, s>>>(w.n, w.st, w.spts, w.nodes, w.leaf_of, w.leaf_first, e,
                                                 reinterpret_cast<unsigned long long *>(hist), w.dev_status);
    note_launch();
    return cudaGetLastError() == cudaSuccess ? ABX_OK : ABX_ECUDA;
}

}  // extern "C"
