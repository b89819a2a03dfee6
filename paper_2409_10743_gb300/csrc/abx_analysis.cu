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

// ---- every pair within eps, streamed to the caller ------------------------------------
// The generic form of the paper's pair traversal ("find all pairs within a
// radius, apply F", subsection "Pair traversal"; subsection "Callbacks" for
// the functor interface): the library cannot run a caller's function on the
// device, so it hands the caller the pairs themselves, each unordered pair
// once, in a deterministic order, resumable across calls.

// A hierarchy's grid with the neighbour radius of this call (the build used
// none): e2 and the early-exit margin are recomputed for eps (the margin
// bound of k_quant: eps_eff * inv_step plus the quantisation's rounding).
__global__ void k_pairs_prep(const SegState *__restrict__ seg, float eps, SegState *out)
{
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        SegState g = seg[0];
        g.e2 = __fmul_rn(eps, eps);
        const double eps_eff = fmax(sqrt((double)g.e2), 0x1p-62) * (1.0 + 0x1p-20);
        const double mc = ceil(eps_eff * (double)g.inv_step + ldexp(1.0, g.bits - 20));
        g.margin = (isfinite(mc) && mc < (double)(1 << 22)) ? (int)mc : -1;
        *out = g;
    }
}

// Pair traversal of sorted point i: the points after i in its own leaf, then
// the leaves after it whose boxes the point's box test cannot rule out,
// stopping early once the walk leaves a Morton region that holds every cell a
// neighbour can have.  f(j) for every j with pred(i, j); every unordered pair
// of the hierarchy's points is met from exactly one of its two ends.
template <class F>
__device__ __forceinline__ void pair_walk(int i, const SegState &g, const State *__restrict__ st,
                                          const float4 *__restrict__ spts, const float4 *__restrict__ nodes,
                                          const int *__restrict__ leaf_of, const int *__restrict__ leaf_first,
                                          unsigned *dev_status, F &&f)
{
    const int L = st->n_leaves;
    const float e2 = g.e2;
    const float4 p = spts[i];
    const int me = leaf_of[i];
    const int e_own = leaf_first[me + 1];
    for (int j = i + 1; j < e_own; j++) {
        const float4 q = __ldg(spts + j);
        if (dist2_rn(p.x, p.y, p.z, q.x, q.y, q.z) <= e2)
            f(j, q);
    }
    float4 alo, ahi;
    ld_node(nodes, L - 1 + me, alo, ahi);
    const int H = reach_level(p.x, p.y, p.z, p.x, p.y, p.z, g);
    int M = level_of(ahi);
    int node = region_exit(M, 0, H) ? SENTINEL : __float_as_int(ahi.w);
    unsigned steps = 0;
    while (node != SENTINEL) {
        if ((unsigned)node >= (unsigned)(2 * L - 1) || ++steps > (unsigned)(2 * L)) {
            atomicOr(dev_status, DEV_INTERNAL);
            break;
        }
        float4 lo, hi;
        ld_node(nodes, node, lo, hi);
        if (box_dist2_rn(p.x, p.y, p.z, lo, hi) <= e2) {
            if (node < L - 1) {
                node = __float_as_int(lo.w);
                continue;
            }
            const int s = (int)(__float_as_uint(lo.w) & ~DENSE_BIT);
            const int e = leaf_first[node - (L - 1) + 1];
            for (int j = s; j < e; j++) {
                const float4 q = __ldg(spts + j);
                if (dist2_rn(p.x, p.y, p.z, q.x, q.y, q.z) <= e2)
                    f(j, q);
            }
        }
        const int lv = level_of(hi);
        if (region_exit(lv, M, H))
            break;
        M = max(M, lv);
        node = __float_as_int(hi.w);
    }
}

__global__ void __launch_bounds__(256) k_pairs_count(int64_t from, int64_t n, const SegState *__restrict__ g,
                                                     const State *__restrict__ st, const float4 *__restrict__ spts,
                                                     const float4 *__restrict__ nodes, const int *__restrict__ leaf_of,
                                                     const int *__restrict__ leaf_first, int *cnt,
                                                     unsigned *dev_status)
{
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (from + k >= n)
        return;
    int c = 0;
    pair_walk((int)(from + k), *g, st, spts, nodes, leaf_of, leaf_first, dev_status, [&](int, float4) { c++; });
    cnt[k] = c;
}

// Exclusive prefix sums of cnt[0 .. m) into pre[0 .. m] (pre[m] = the total),
// one pass with a decoupled look-back over tiles of SCAN_TILE counts.
__global__ void __launch_bounds__(SCAN_THREADS) k_pairs_scan(int64_t m, const int *__restrict__ cnt,
                                                             long long *pre, unsigned *tile_ctr,
                                                             unsigned long long *lb, unsigned *dev_status)
{
    __shared__ int s_tile;
    __shared__ unsigned long long s_wsum[SCAN_THREADS / 32];
    __shared__ unsigned long long s_excl;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (tid == 0)
        s_tile = (int)atomicAdd(tile_ctr, 1u);
    __syncthreads();
    const int tile = s_tile;
    const int64_t base = (int64_t)tile * SCAN_TILE + (int64_t)tid * SCAN_ITEMS;
    int v[SCAN_ITEMS];
    unsigned long long mine = 0;
#pragma unroll
    for (int j = 0; j < SCAN_ITEMS; j++) {
        v[j] = base + j < m ? cnt[base + j] : 0;
        mine += (unsigned)v[j];
    }
    unsigned long long x = mine;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const unsigned long long y = __shfl_up_sync(~0u, x, o);
        if (lane >= o)
            x += y;
    }
    if (lane == 31)
        s_wsum[warp] = x;
    __syncthreads();
    unsigned long long wpre = 0, total = 0;
    for (int w = 0; w < SCAN_THREADS / 32; w++) {
        if (w < warp)
            wpre += s_wsum[w];
        total += s_wsum[w];
    }
    if (tid == 0) {
        unsigned long long excl = 0;
        if (tile == 0) {
            lb_store(lb, LB_FLAG_PRE | total);
        } else {
            lb_store(lb + tile, LB_FLAG_AGG | total);
            excl = lookback<16>(lb, tile, 1, 0, dev_status);
            lb_store(lb + tile, LB_FLAG_PRE | (excl + total));
        }
        s_excl = excl;
    }
    __syncthreads();
    unsigned long long run = s_excl + wpre + x - mine;
#pragma unroll
    for (int j = 0; j < SCAN_ITEMS; j++) {
        if (base + j < m)
            pre[base + j] = (long long)run;
        run += (unsigned)v[j];
        if (base + j == m - 1)
            pre[m] = (long long)run;
    }
}

// How many points' pairs fit in cap: the largest k with pre[k] <= cap.
__global__ void k_pairs_limit(int64_t m, const long long *__restrict__ pre, long long cap, long long *res)
{
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        int64_t lo = 0, hi = m;  // pre[0] = 0 <= cap
        while (lo < hi) {
            const int64_t mid = (lo + hi + 1) >> 1;
            if (pre[mid] <= cap)
                lo = mid;
            else
                hi = mid - 1;
        }
        res[0] = lo;
        res[1] = pre[lo];
    }
}

__global__ void __launch_bounds__(256) k_pairs_emit(int64_t from, const long long *__restrict__ res,
                                                    const SegState *__restrict__ g, const State *__restrict__ st,
                                                    const float4 *__restrict__ spts, const float4 *__restrict__ nodes,
                                                    const int *__restrict__ leaf_of, const int *__restrict__ leaf_first,
                                                    const long long *__restrict__ pre, int32_t *out,
                                                    unsigned *dev_status)
{
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= res[0])
        return;
    const int i = (int)(from + k);
    const int oi = __float_as_int(spts[i].w);
    long long w = pre[k];
    pair_walk(i, *g, st, spts, nodes, leaf_of, leaf_first, dev_status, [&](int, float4 q) {
        const int oj = __float_as_int(q.w);
        out[2 * w] = min(oi, oj);
        out[2 * w + 1] = max(oi, oj);
        w++;
    });
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

abx_status abx_bvh_pairs(const abx_bvh *bvh, float eps, int64_t *cursor, int32_t *pairs, int64_t cap,
                         int64_t *n_written, abx_stream stream)
{
    if (!bvh || !cursor || !n_written || cap < 0 || (cap > 0 && !pairs) || !(eps >= 0.0f) ||
        eps == __builtin_inff())
        return ABX_EINVAL;
    const Work &w = bvh->w;
    const int64_t n = w.n;
    if (*cursor < 0 || *cursor > n)
        return ABX_EINVAL;
    *n_written = 0;
    const int64_t from = *cursor, m = n - from;
    if (m == 0)
        return ABX_OK;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    const size_t tiles = (size_t)div_up(m, SCAN_TILE);
    auto al = [](size_t b) { return (b + 255) & ~(size_t)255; };
    const size_t b_seg = al(sizeof(SegState)), b_cnt = al((size_t)m * sizeof(int)),
                 b_pre = al((size_t)(m + 1) * sizeof(long long)), b_lb = al(tiles * sizeof(unsigned long long)),
                 b_misc = al(4 * sizeof(long long));
    char *ws = nullptr;
    if (cudaMallocFromPoolAsync((void **)&ws, b_seg + b_cnt + b_pre + b_lb + b_misc, bvh->pool, s) != cudaSuccess) {
        cudaGetLastError();
        return ABX_ENOMEM;
    }
    SegState *gs = reinterpret_cast<SegState *>(ws);
    int *cnt = reinterpret_cast<int *>(ws + b_seg);
    long long *pre = reinterpret_cast<long long *>(ws + b_seg + b_cnt);
    unsigned long long *lb = reinterpret_cast<unsigned long long *>(ws + b_seg + b_cnt + b_pre);
    long long *res = reinterpret_cast<long long *>(ws + b_seg + b_cnt + b_pre + b_lb);  // [0..1] result, [2] tickets
    cudaMemsetAsync(lb, 0, b_lb + b_misc, s);
    k_pairs_prep<<<1, 32, 0, s>>>(w.seg, eps, gs);
    k_pairs_count<<<div_up(m, 256), 256, 0, s>>>(from, n, gs, w.st, w.spts, w.nodes, w.leaf_of, w.leaf_first, cnt,
                                                 w.dev_status);
    k_pairs_scan<<<(int)tiles, SCAN_THREADS, 0, s>>>(m, cnt, pre, reinterpret_cast<unsigned *>(res + 2), lb,
                                                     w.dev_status);
    k_pairs_limit<<<1, 32, 0, s>>>(m, pre, (long long)cap, res);
    k_pairs_emit<<<div_up(m, 256), 256, 0, s>>>(from, res, gs, w.st, w.spts, w.nodes, w.leaf_of, w.leaf_first, pre,
                                                pairs, w.dev_status);
    note_launch(5);
    long long host[2] = {0, 0}, first_need = 0;
    cudaMemcpyAsync(host, res, 2 * sizeof(long long), cudaMemcpyDeviceToHost, s);
    cudaMemcpyAsync(&first_need, pre + 1, sizeof(long long), cudaMemcpyDeviceToHost, s);
    cudaFreeAsync(ws, s);
    if (cudaStreamSynchronize(s) != cudaSuccess || cudaGetLastError() != cudaSuccess)
        return ABX_ECUDA;
    if (host[0] == 0)
        return first_need > cap ? ABX_ENOMEM : ABX_OK;  // the next point's pairs alone do not fit
    *cursor = from + host[0];
    *n_written = host[1];
    return ABX_OK;
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
