// Fused traversals: core counting, pair traversal with union-find, border
// points and the final labels.
//
// Paper, Algorithm PDSDbscan: if minPts > 2 the core points are found first
// (a counting traversal per point, stopped once the count reaches minPts --
// subsection "Early termination"); then every pair of neighbours is visited
// once and core-core pairs are merged with Union.  Subsection "FDBSCAN": the
// traversal is fused with counting and with union-find (no neighbour lists,
// O(n) memory), and the merging kernel uses pair traversal (subsection "Pair
// traversal"): the thread of point i starts at its own leaf and follows ropes,
// so it only meets leaves after its own and each pair is seen exactly once.
// Here that traversal runs in two passes: once per leaf with the leaf's box
// (k_cand: which leaves after it any of its points can reach), then once per
// point over those candidate leaves only (k_union).
//
// The paper's border step (the first core to arrive claims an unclaimed
// non-core neighbour inside a critical section) is nondeterministic.  It is
// replaced by a separate pass after all unions: each non-core point looks at
// all its core neighbours and joins the cluster whose smallest core index is
// smallest.
#include "work.cuh"

namespace abx {

struct Tree {
    const float4 *__restrict__ nodes;
    const int *__restrict__ leaf_first;
    int L;
};

// A traversal visits every node at most once; a node index outside the
// hierarchy or more steps than nodes means a corrupted tree: the traversal
// stops and records DEV_INTERNAL instead of faulting or spinning.
__device__ __forceinline__ bool node_ok(int node, int L, unsigned &steps, unsigned *dev_status)
{
    if ((unsigned)node >= (unsigned)(2 * L - 1) || ++steps > (unsigned)(2 * L)) {
        atomicOr(dev_status, DEV_INTERNAL);
        return false;
    }
    return true;
}

__device__ __forceinline__ float4 node_lo(const Tree &t, int i) { return __ldg(t.nodes + 2 * (size_t)i); }
__device__ __forceinline__ float4 node_hi(const Tree &t, int i) { return __ldg(t.nodes + 2 * (size_t)i + 1); }

// ---- candidate leaves --------------------------------------------------------------
// The pair traversal of a point starts at its leaf's rope and descends into
// every subtree after its leaf that its own box test cannot rule out.  A node
// whose rounded distance to the LEAF's box exceeds eps is out of reach of
// every point of the leaf (box_box_dist2_rn is a lower bound of the point's
// own box distance), so one traversal per leaf with the leaf's box finds the
// leaves after it that any of its points can reach: its candidate leaves.
// Each point then tests only the points of those leaves (after its own box
// test of each) and visits no node.  Up to CAND_K - 1 candidates are kept (one
// int4 per leaf); when there are more, the last slot holds -(node + 2) for
// the leaf node where the list ran out, and the points walk the ropes from
// there on with their own box tests (which visits that leaf and everything
// after it in pre-order).  -1 ends a list.

constexpr int CAND_K = 4;

template <bool SEG>
__global__ void k_cand(const State *__restrict__ st, const SegState *__restrict__ seg,
                       const int *__restrict__ leaf_seg, const float4 *__restrict__ nodes, int4 *cand,
                       unsigned *dev_status)
{
    const int L = st->n_leaves;
    const int a = blockIdx.x * blockDim.x + threadIdx.x;
    if (a >= L)
        return;
    const Tree T{nodes, nullptr, L};
    const float e2 = seg[SEG ? leaf_seg[a] : 0].e2;
    const float4 alo = node_lo(T, L - 1 + a), ahi = node_hi(T, L - 1 + a);
    int out[CAND_K];
#pragma unroll
    for (int k = 0; k < CAND_K; k++)
        out[k] = SENTINEL;
    int k = 0;
    int node = __float_as_int(ahi.w);
    unsigned steps = 0;
    while (node != SENTINEL) {
        if (!node_ok(node, L, steps, dev_status))
            break;
        const float4 lo = node_lo(T, node), hi = node_hi(T, node);
        if (box_box_dist2_rn(alo, ahi, lo, hi) <= e2) {
            if (node < L - 1) {
                node = __float_as_int(lo.w);
                continue;
            }
            const int v = k == CAND_K - 1 ? -(node + 2) : node - (L - 1);
    #pragma unroll
            for (int q = 0; q < CAND_K; q++)
                if (q == k)
                    out[q] = v;
            if (++k == CAND_K)
                break;
        }
        node = __float_as_int(hi.w);
    }
    cand[a] = make_int4(out[0], out[1], out[2], out[3]);
}

// ---- pair traversal with union-find ------------------------------------------------
// FoF (minPts <= 2): every neighbour pair is merged and both ends become core.
// DBSCAN (minPts > 2): only core threads run, and only core-core pairs merge.

// Traversal statistics (profile mode 2 only, a separate template instance so
// the timed kernel carries no counters): node visits, leaf visits, point
// tests and unions, summed over all threads of the launch.
struct TravStats {
    unsigned long long visits, leaves, tests, unions, queries;
};

template <bool FOF, bool STATS>
__device__ __forceinline__ void union_query(const int i, const float e2, const Tree &T,
                                            const float4 *__restrict__ spts, const int *__restrict__ leaf_of,
                                            const int4 *__restrict__ cand, int *parent, unsigned char *core,
                                            unsigned *dev_status, TravStats *stats)
{
    const int L = T.L;
    const float4 p = spts[i];
    const int *__restrict__ leaf_first = T.leaf_first;
    bool found = false;
    unsigned c_visit = 0, c_leaf = 0, c_test = 0, c_union = 0;

    const int my_leaf = L - 1 + leaf_of[i];
    const unsigned w0 = __float_as_uint(node_lo(T, my_leaf).w);
    if (!(w0 & DENSE_BIT)) {
        const int e = leaf_first[my_leaf - (L - 1) + 1];
        for (int j = i + 1; j < e; j++) {
            float4 q = __ldg(spts + j);
            if (STATS)
                c_test++;
            if ((FOF || core[j]) && dist2_rn(p.x, p.y, p.z, q.x, q.y, q.z) <= e2) {
                uf_unite(parent, spts, i, j);
                if (STATS)
                    c_union++;
                if (FOF) {
                    found = true;
                    core[j] = 1;
                }
            }
        }
    }
    // the points of leaf [s, e): one of the candidate leaves of i's leaf
    auto test_leaf = [&](const unsigned lw, const int e) {
        const int s = (int)(lw & ~DENSE_BIT);
        if (STATS)
            c_leaf++;
        if (lw & DENSE_BIT) {
            // all points of a dense cell are core and already one set:
            // one link is enough, none if i is already in that set
            if (uf_find(parent, i) == uf_find(parent, s)) {
                found = true;
                return;
            }
            for (int j = s; j < e; j++) {
                const float4 q = __ldg(spts + j);
                if (STATS)
                    c_test++;
                if (dist2_rn(p.x, p.y, p.z, q.x, q.y, q.z) <= e2) {
                    uf_unite(parent, spts, i, s);
                    if (STATS)
                        c_union++;
                    found = true;
                    return;
                }
            }
            return;
        }
        for (int j = s; j < e; j++) {
            const float4 q = __ldg(spts + j);
            if (STATS)
                c_test++;
            if ((FOF || core[j]) && dist2_rn(p.x, p.y, p.z, q.x, q.y, q.z) <= e2) {
                uf_unite(parent, spts, i, j);
                if (STATS)
                    c_union++;
                if (FOF) {
                    found = true;
                    core[j] = 1;
                }
            }
        }
    };
    const int me = my_leaf - (L - 1);
    const int4 c4 = cand[me];
    int resume = SENTINEL;
    for (int c = 0; c < CAND_K; c++) {
        const int v = c == 0 ? c4.x : c == 1 ? c4.y : c == 2 ? c4.z : c4.w;
        if (v == SENTINEL)
            break;
        if (v < 0) {
            resume = -v - 2;
            break;
        }
        // the leaf passed the leaf-box test; the point's own box test is
        // tighter and spares the point tests of most far leaves
        const float4 lo = node_lo(T, L - 1 + v), hi = node_hi(T, L - 1 + v);
        if (box_dist2_rn(p.x, p.y, p.z, lo, hi) <= e2)
            test_leaf(__float_as_uint(lo.w), leaf_first[v + 1]);
    }
    // more candidates than the list holds: the plain pair traversal from the
    // leaf where the list ran out
    int node = resume;
    unsigned steps = 0;
    while (node != SENTINEL) {
        if (!node_ok(node, L, steps, dev_status))
            break;
        const float4 lo = node_lo(T, node), hi = node_hi(T, node);
        if (STATS)
            c_visit++;
        if (box_dist2_rn(p.x, p.y, p.z, lo, hi) <= e2) {
            if (node < L - 1) {
                node = __float_as_int(lo.w);
                continue;
            }
            test_leaf(__float_as_uint(lo.w), leaf_first[node - (L - 1) + 1]);
        }
        node = __float_as_int(hi.w);
    }
    if (FOF && found)
        core[i] = 1;
    if (STATS) {
        atomicAdd(&stats->visits, (unsigned long long)c_visit);
        atomicAdd(&stats->leaves, (unsigned long long)c_leaf);
        atomicAdd(&stats->tests, (unsigned long long)c_test);
        atomicAdd(&stats->unions, (unsigned long long)c_union);
        atomicAdd(&stats->queries, 1ull);
    }
}

template <bool FOF, bool STATS>
__global__ void __launch_bounds__(1024, 2) k_union(int64_t n, const State *__restrict__ st, const SegState *__restrict__ seg,
                        const float4 *__restrict__ spts, const float4 *__restrict__ nodes,
                        const int *__restrict__ leaf_of, const int *__restrict__ leaf_first,
                        const int4 *__restrict__ cand, int *parent,
                        unsigned char *core, unsigned *dev_status, TravStats *stats)
{
    const int64_t i64 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i64 >= n)
        return;
    const int i = (int)i64;
    if (!FOF && !core[i])
        return;
    const Tree T{nodes, leaf_first, st->n_leaves};
    union_query<FOF, STATS>(i, seg[0].e2, T, spts, leaf_of, cand, parent, core, dev_status, stats);
}

// Many segments: each query takes its segment's eps and mode from its key.
template <bool STATS>
__global__ void __launch_bounds__(1024, 2) k_union_seg(int64_t n, const State *__restrict__ st, const SegState *__restrict__ seg,
                            const unsigned long long *k0, const unsigned long long *k1,
                            const float4 *__restrict__ spts, const float4 *__restrict__ nodes,
                            const int *__restrict__ leaf_of, const int *__restrict__ leaf_first,
                        const int4 *__restrict__ cand, int *parent,
                            unsigned char *core, unsigned *dev_status, TravStats *stats)
{
    const int64_t i64 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i64 >= n)
        return;
    const int i = (int)i64;
    const SegState &g = seg[seg_of_key(sorted_key(st, k0, k1, i), st->shift)];
    const Tree T{nodes, leaf_first, st->n_leaves};
    if (g.minpts <= 2)
        union_query<true, STATS>(i, g.e2, T, spts, leaf_of, cand, parent, core, dev_status, stats);
    else if (core[i])
        union_query<false, STATS>(i, g.e2, T, spts, leaf_of, cand, parent, core, dev_status, stats);
}

// ---- core counting with early termination (minPts > 2) -------------------------------

template <bool SEG>
__global__ void k_count(int64_t n, const State *__restrict__ st, const SegState *__restrict__ seg,
                        const unsigned long long *k0, const unsigned long long *k1,
                        const float4 *__restrict__ spts, const float4 *__restrict__ nodes,
                        const int *__restrict__ leaf_first, unsigned char *core, unsigned *dev_status)
{
    const int64_t i64 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i64 >= n)
        return;
    const int i = (int)i64;
    if (core[i])
        return;  // member of a dense cell
    int s = 0;
    if (SEG)
        s = seg_of_key(sorted_key(st, k0, k1, i), st->shift);
    const SegState &g = seg[s];
    const int minpts = g.minpts;
    if (SEG && minpts <= 2)
        return;  // a friends-of-friends segment needs no counting
    const float e2 = g.e2;
    const Tree T{nodes, leaf_first, st->n_leaves};
    const int L = T.L;
    const float4 p = spts[i];
    int cnt = 0;
    int node = g.root;
    unsigned steps = 0;
    while (node != SENTINEL) {
        if (!node_ok(node, L, steps, dev_status))
            break;
        const float4 lo = node_lo(T, node), hi = node_hi(T, node);
        if (box_dist2_rn(p.x, p.y, p.z, lo, hi) <= e2) {
            if (node < L - 1) {
                node = __float_as_int(lo.w);
                continue;
            }
            const int s0 = (int)(__float_as_uint(lo.w) & ~DENSE_BIT);
            const int e = leaf_first[node - (L - 1) + 1];
            for (int j = s0; j < e; j++) {
                float4 q = __ldg(spts + j);
                if (dist2_rn(p.x, p.y, p.z, q.x, q.y, q.z) <= e2 && ++cnt >= minpts) {
                    core[i] = 1;
                    return;
                }
            }
        }
        node = __float_as_int(hi.w);
    }
}

// ---- border points (minPts > 2) ----------------------------------------------------------
// For a non-core point b: the root with the smallest priority (= K(C)) among
// the clusters of its core neighbours.  The choice is recorded as parent[b]
// (b is never in a union, so nothing else reads or writes that word) and the
// cluster's smallest border index is kept in bmin[root].

template <bool SEG>
__global__ void k_border(int64_t n, const State *__restrict__ st, const SegState *__restrict__ seg,
                         const unsigned long long *k0, const unsigned long long *k1,
                         const float4 *__restrict__ spts, const float4 *__restrict__ nodes,
                         const int *__restrict__ leaf_first, int *parent, const unsigned char *__restrict__ core,
                         int *bmin, unsigned *dev_status)
{
    const int64_t i64 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i64 >= n)
        return;
    const int i = (int)i64;
    if (core[i])
        return;
    int s = 0;
    if (SEG)
        s = seg_of_key(sorted_key(st, k0, k1, i), st->shift);
    const SegState &g = seg[s];
    if (SEG && g.minpts <= 2)
        return;  // friends-of-friends: no border points
    const float e2 = g.e2;
    const Tree T{nodes, leaf_first, st->n_leaves};
    const int L = T.L;
    const float4 p = spts[i];
    int best_k = 0x7fffffff, best_r = -1;
    int node = g.root;
    unsigned steps = 0;
    while (node != SENTINEL) {
        if (!node_ok(node, L, steps, dev_status))
            break;
        const float4 lo = node_lo(T, node), hi = node_hi(T, node);
        if (box_dist2_rn(p.x, p.y, p.z, lo, hi) <= e2) {
            if (node < L - 1) {
                node = __float_as_int(lo.w);
                continue;
            }
            const unsigned lw = __float_as_uint(lo.w);
            const int s0 = (int)(lw & ~DENSE_BIT);
            const int e = leaf_first[node - (L - 1) + 1];
            for (int j = s0; j < e; j++) {
                if (!core[j])
                    continue;
                float4 q = __ldg(spts + j);
                if (dist2_rn(p.x, p.y, p.z, q.x, q.y, q.z) <= e2) {
                    int r = uf_find(parent, j);
                    int k = orig_of(spts, r);
                    if (k < best_k) {
                        best_k = k;
                        best_r = r;
                    }
                    if (lw & DENSE_BIT)
                        break;  // one cluster per dense cell
                }
            }
        }
        node = __float_as_int(hi.w);
    }
    if (best_r >= 0) {
        parent[i] = best_r;
        atomicMin(bmin + best_r, __float_as_int(p.w));
    }
}

// ---- labels -----------------------------------------------------------------------------------
// Cluster id = the smallest original index among the members: the root's
// (smallest core index) or a smaller border index; scattered to input order,
// relative to the segment's first point.

template <bool SEG>
__global__ void __launch_bounds__(256) k_finalize(int64_t n, const State *__restrict__ st,
                                                  const SegState *__restrict__ seg, const int *__restrict__ off,
                                                  const unsigned long long *k0, const unsigned long long *k1,
                                                  const float4 *__restrict__ spts, int *parent,
                                                  const unsigned char *__restrict__ core,
                                                  const int *__restrict__ bmin, int32_t *labels)
{
    const int64_t i64 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i64 >= n)
        return;
    const int i = (int)i64;
    int s = 0;
    if (SEG)
        s = seg_of_key(sorted_key(st, k0, k1, i), st->shift);
    const bool fof = seg[s].minpts <= 2;
    int lab = -1;
    if (core[i]) {
        int r = uf_find(parent, i);
        lab = orig_of(spts, r);
        if (!fof)
            lab = min(lab, bmin[r]);
    } else if (!fof) {
        int r = parent[i];
        if (r != i)
            lab = min(orig_of(spts, r), bmin[r]);
    }
    // labels were preset to -1: only cluster members are scattered (noise
    // points, most points of a sparse scene, read nothing more)
    if (lab < 0)
        return;
    const int o = __float_as_int(spts[i].w);
    if ((unsigned)o < (unsigned)n)
        labels[o] = SEG ? lab - off[s] : lab;
}

void stage_cluster(const Work &w, const Params &p, int32_t *labels, cudaStream_t s)
{
    const int B = p.block;
    const int g = div_up(w.n, B);
    TravStats *stats = (TravStats *)w.stats;
    cudaMemsetAsync(labels, 0xff, (size_t)w.n * sizeof(int32_t), s);  // noise = -1
    if (w.nseg == 1)
        k_cand<false><<<div_up(w.n, 256), 256, 0, s>>>(w.st, w.seg, w.leaf_seg, w.nodes, w.cand, w.dev_status);
    else
        k_cand<true><<<div_up(w.n, 256), 256, 0, s>>>(w.st, w.seg, w.leaf_seg, w.nodes, w.cand, w.dev_status);
    note_launch();
    prof_mark(ST_CANDS, s);
    if (w.nseg == 1) {
        if (w.any_fof) {
            if (stats)
                k_union<true, true><<<g, B, 0, s>>>(w.n, w.st, w.seg, w.spts, w.nodes, w.leaf_of, w.leaf_first,
                                                    w.cand, w.parent, w.core, w.dev_status, stats);
            else
                k_union<true, false><<<g, B, 0, s>>>(w.n, w.st, w.seg, w.spts, w.nodes, w.leaf_of, w.leaf_first,
                                                     w.cand, w.parent, w.core, w.dev_status, nullptr);
            note_launch();
            prof_mark(ST_UNION, s);
        } else {
            k_count<false><<<g, B, 0, s>>>(w.n, w.st, w.seg, w.keys[0], w.keys[1], w.spts, w.nodes, w.leaf_first,
                                           w.core, w.dev_status);
            note_launch();
            prof_mark(ST_COUNT, s);
            if (stats)
                k_union<false, true><<<g, B, 0, s>>>(w.n, w.st, w.seg, w.spts, w.nodes, w.leaf_of, w.leaf_first,
                                                     w.cand, w.parent, w.core, w.dev_status, stats);
            else
                k_union<false, false><<<g, B, 0, s>>>(w.n, w.st, w.seg, w.spts, w.nodes, w.leaf_of, w.leaf_first,
                                                      w.cand, w.parent, w.core, w.dev_status, nullptr);
            note_launch();
            prof_mark(ST_UNION, s);
            k_border<false><<<g, B, 0, s>>>(w.n, w.st, w.seg, w.keys[0], w.keys[1], w.spts, w.nodes, w.leaf_first,
                                            w.parent, w.core, w.bmin, w.dev_status);
            note_launch();
            prof_mark(ST_BORDER, s);
        }
        k_finalize<false><<<div_up(w.n, 256), 256, 0, s>>>(w.n, w.st, w.seg, w.seg_off, w.keys[0], w.keys[1],
                                                           w.spts, w.parent, w.core, w.bmin, labels);
    } else {
        if (w.any_dbscan) {
            k_count<true><<<g, B, 0, s>>>(w.n, w.st, w.seg, w.keys[0], w.keys[1], w.spts, w.nodes, w.leaf_first,
                                          w.core, w.dev_status);
            note_launch();
            prof_mark(ST_COUNT, s);
        }
        if (stats)
            k_union_seg<true><<<g, B, 0, s>>>(w.n, w.st, w.seg, w.keys[0], w.keys[1], w.spts, w.nodes, w.leaf_of,
                                              w.leaf_first, w.cand, w.parent, w.core, w.dev_status, stats);
        else
            k_union_seg<false><<<g, B, 0, s>>>(w.n, w.st, w.seg, w.keys[0], w.keys[1], w.spts, w.nodes, w.leaf_of,
                                               w.leaf_first, w.cand, w.parent, w.core, w.dev_status, nullptr);
        note_launch();
        prof_mark(ST_UNION, s);
        if (w.any_dbscan) {
            k_border<true><<<g, B, 0, s>>>(w.n, w.st, w.seg, w.keys[0], w.keys[1], w.spts, w.nodes, w.leaf_first,
                                           w.parent, w.core, w.bmin, w.dev_status);
            note_launch();
            prof_mark(ST_BORDER, s);
        }
        k_finalize<true><<<div_up(w.n, 256), 256, 0, s>>>(w.n, w.st, w.seg, w.seg_off, w.keys[0], w.keys[1],
                                                          w.spts, w.parent, w.core, w.bmin, labels);
    }
    note_launch();
    prof_mark(ST_FINALIZE, s);
}

}  // namespace abx
