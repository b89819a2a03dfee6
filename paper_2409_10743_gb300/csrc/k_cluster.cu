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
#include <algorithm>

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

// ---- candidate leaves --------------------------------------------------------------
// The pair traversal of a point starts at its leaf's rope and descends into
// every subtree after its leaf that its own box test cannot rule out.  A node
// whose rounded distance to the LEAF's box exceeds eps is out of reach of
// every point of the leaf (box_box_dist2_rn is a lower bound of the point's
// own box distance), so one traversal per leaf with the leaf's box finds the
// leaves after it that any of its points can reach: its candidate leaves.
// The walk stops early once the subtree it leaves is a Morton region that
// holds every cell a neighbour of the leaf can have (region_exit).
//
// cand[a] = {end of leaf a's points | DENSE_BIT if leaf a is a dense cell,
// c0, c1, c2}: up to three candidate leaves, -1 ending the list.  With four or
// more, c2 = -(node + 2) for the leaf node of the third candidate instead:
// the points walk the ropes from there on with their own box tests (which
// visits that leaf and everything after it in pre-order).

constexpr int CAND_SLOTS = 3;
constexpr int CAND_TICKETS = MAX_PASSES + 3;  // tile_ctr index of the candidate pass's leaf queue
constexpr int CAND_CHUNK = 64;                // leaves a warp takes from the queue at a time
static int g_cand_blocks_per_sm = 4;           // set per process by cluster_init_device

// Persistent: the walks differ in length by an order of magnitude, and a warp
// runs as long as its longest walk, so each lane carries one walk at a time,
// one node visit per step, and a lane whose walk ended takes the next leaf
// from the warp's chunk of the leaf queue (chunks of CAND_CHUNK leaves: one
// global atomic per chunk) -- the warp stays full until the queue runs dry.
template <bool SEG>
__global__ void __launch_bounds__(256, 6) k_cand(State *__restrict__ st, const SegState *__restrict__ seg,
                                              const int *__restrict__ leaf_seg, const float4 *__restrict__ nodes,
                                              const int *__restrict__ leaf_first, int4 *cand, unsigned *dev_status)
{
    const int L = st->n_leaves;
    unsigned *queue = &st->tile_ctr[CAND_TICKETS];
    const int lane = threadIdx.x & 31;
    const unsigned lt = (1u << lane) - 1u;
    // this lane's walk
    int a = 0, node = SENTINEL, M = 0, H = 0, k = 0, own = 0;
    int out0 = SENTINEL, out1 = SENTINEL, out2 = SENTINEL;
    unsigned steps = 0;
    float e2 = 0.0f;
    float4 alo = make_float4(0.0f, 0.0f, 0.0f, 0.0f), ahi = alo;
    bool live = false;
    // the warp's chunk of the queue (the same in every lane)
    int q_next = 0, q_end = 0;
    bool dry = false;
    while (true) {
        // refill once half the warp is idle (so that a leaf's set-up runs with
        // many lanes at once), or when every lane is
        unsigned need = __ballot_sync(~0u, !live);
        if (__popc(need) < 16 && need != ~0u)
            need = 0;
        while (need && !dry) {
            if (q_next >= q_end) {
                unsigned c = 0;
                if (lane == 0)
                    c = atomicAdd(queue, (unsigned)CAND_CHUNK);
                c = __shfl_sync(~0u, c, 0);
                if (c >= (unsigned)L) {
                    dry = true;
                    break;
                }
                q_next = (int)c;
                q_end = (int)min(c + (unsigned)CAND_CHUNK, (unsigned)L);
            }
            const int avail = q_end - q_next;
            const int r = __popc(need & lt);
            if (((need >> lane) & 1u) && r < avail) {
                a = q_next + r;
                const SegState &g = seg[SEG ? leaf_seg[a] : 0];
                e2 = g.e2;
                ld_node(nodes, L - 1 + a, alo, ahi);
                own = leaf_first[a + 1] | (int)(__float_as_uint(alo.w) & DENSE_BIT);
                H = reach_level(alo.x, alo.y, alo.z, ahi.x, ahi.y, ahi.z, g);
                M = level_of(ahi);  // following the leaf's own rope crosses boundary a
                node = region_exit(M, 0, H) ? SENTINEL : __float_as_int(ahi.w);
                k = 0;
                out0 = out1 = out2 = SENTINEL;
                steps = 0;
                live = node != SENTINEL;
                if (!live)
                    cand[a] = make_int4(own, SENTINEL, SENTINEL, SENTINEL);
            }
            q_next += min(__popc(need), avail);
            need = __ballot_sync(~0u, !live);
        }
        if (!__any_sync(~0u, live))
            break;
        if (!live)
            continue;
        // one node visit
        bool fin = false;
        if (!node_ok(node, L, steps, dev_status)) {
            fin = true;
        } else {
            float4 lo, hi;
            ld_node(nodes, node, lo, hi);
            bool descend = false;
            if (box_box_dist2_rn(alo, ahi, lo, hi) <= e2) {
                if (node < L - 1) {
                    node = __float_as_int(lo.w);
                    descend = true;
                } else if (k < CAND_SLOTS) {
                    const int t = node - (L - 1);
                    if (k == 0)
                        out0 = t;
                    else if (k == 1)
                        out1 = t;
                    else
                        out2 = t;
                    k++;
                } else {  // a fourth: resume at the third one's node
                    out2 = -((L - 1 + out2) + 2);
                    fin = true;
                }
            }
            if (!descend && !fin) {
                const int lv = level_of(hi);
                if (region_exit(lv, M, H)) {
                    fin = true;
                } else {
                    M = max(M, lv);
                    node = __float_as_int(hi.w);
                    fin = node == SENTINEL;
                }
            }
        }
        if (fin) {
            cand[a] = make_int4(own, out0, out1, out2);
            live = false;
        }
    }
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

// SCHED 1: the point tests the candidate leaves its leaf collected (k_cand),
// then, if the list overflowed, walks the ropes from the leaf where it ran out.
// SCHED 2: no candidate lists; the point walks the ropes from its own leaf
// with its own box, stopping early like k_cand (region_exit).
// WARP: every lane of the warp calls this (points i of consecutive lanes are
// consecutive), `active` says whether lane i queries, and the pairs inside
// the own leaf (at most span + 1 consecutive points) are tested on the next
// lanes' coordinates, fetched by shuffle with all lanes in step, instead of
// by loads one after another.  Otherwise only querying threads call it.
template <int SCHED, bool FOF, bool STATS, bool WARP>
__device__ __forceinline__ void union_query(const int i, const bool active, const int span, const SegState &g,
                                            const Tree &T,
                                            const float4 *__restrict__ spts, const int *__restrict__ leaf_of,
                                            const int4 *__restrict__ cand, int *parent, unsigned char *core,
                                            unsigned *dev_status, TravStats *stats)
{
    const int L = T.L;
    const float e2 = g.e2;
    const float4 p = spts[i];
    const int *__restrict__ leaf_first = T.leaf_first;
    bool found = false;
    unsigned c_visit = 0, c_leaf = 0, c_test = 0, c_union = 0;

    const int me = leaf_of[i];
    int own_end;  // end of the own leaf's points, DENSE_BIT set for a dense cell
    int4 c4 = make_int4(0, SENTINEL, SENTINEL, SENTINEL);
    int node = SENTINEL, M = 0, H = 255;
    if (SCHED == 1) {
        c4 = cand[me];
        own_end = c4.x;
    } else {
        float4 alo, ahi;
        ld_node(T.nodes, L - 1 + me, alo, ahi);
        own_end = leaf_first[me + 1] | (int)(__float_as_uint(alo.w) & DENSE_BIT);
        H = reach_level(p.x, p.y, p.z, p.x, p.y, p.z, g);
        M = level_of(ahi);
        node = region_exit(M, 0, H) ? SENTINEL : __float_as_int(ahi.w);
    }
    // ri: a member of i's set, its root when last seen.  Sets only grow, so a
    // neighbour whose parent is ri is in i's set already: one load, no finds
    // (on dense data most neighbour pairs are such repeats)
    int ri = i;
    auto link = [&](const int j) {
        if (ld_cg(parent + j) != ri)
            ri = uf_unite(parent, spts, ri, j);
    };
    if (WARP) {
        const int lane = threadIdx.x & 31;
        const int ci = FOF ? 1 : (int)core[i];
        for (int d = 1; d <= span; d++) {
            const float qx = __shfl_down_sync(~0u, p.x, d);
            const float qy = __shfl_down_sync(~0u, p.y, d);
            const float qz = __shfl_down_sync(~0u, p.z, d);
            const int qc = FOF ? 1 : __shfl_down_sync(~0u, ci, d);
            const int j = i + d;
            if (active && j < own_end) {  // (never in a dense cell: DENSE_BIT makes own_end negative)
                float4 q = make_float4(qx, qy, qz, 0.0f);
                bool cj = qc != 0;
                if (lane + d >= 32) {  // the leaf runs on past the warp
                    q = __ldg(spts + j);
                    cj = FOF || core[j];
                }
                if (STATS)
                    c_test++;
                if (cj && dist2_rn(p.x, p.y, p.z, q.x, q.y, q.z) <= e2) {
                    link(j);
                    if (STATS)
                        c_union++;
                    if (FOF) {
                        found = true;
                        core[j] = 1;
                    }
                }
            }
        }
        if (!active)
            return;
    } else if (own_end >= 0) {  // not a dense cell (its points are one set already)
        const int e = own_end;
        for (int j = i + 1; j < e; j++) {
            float4 q = __ldg(spts + j);
            if (STATS)
                c_test++;
            if ((FOF || core[j]) && dist2_rn(p.x, p.y, p.z, q.x, q.y, q.z) <= e2) {
                link(j);
                if (STATS)
                    c_union++;
                if (FOF) {
                    found = true;
                    core[j] = 1;
                }
            }
        }
    }
    // the points of leaf [s, e): a leaf after i's own that may hold neighbours
    auto test_leaf = [&](const unsigned lw, const int e) {
        const int s = (int)(lw & ~DENSE_BIT);
        if (STATS)
            c_leaf++;
        if (lw & DENSE_BIT) {
            // all points of a dense cell are core and already one set:
            // one link is enough, none if i is already in that set
            const int rs = uf_find(parent, s);
            ri = uf_find(parent, ri);
            if (ri == rs) {
                found = true;
                return;
            }
            for (int j = s; j < e; j++) {
                const float4 q = __ldg(spts + j);
                if (STATS)
                    c_test++;
                if (dist2_rn(p.x, p.y, p.z, q.x, q.y, q.z) <= e2) {
                    ri = uf_unite(parent, spts, ri, rs);
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
                link(j);
                if (STATS)
                    c_union++;
                if (FOF) {
                    found = true;
                    core[j] = 1;
                }
            }
        }
    };
    constexpr bool may_exit = SCHED == 2;
    if (SCHED == 1) {
        // The list holds leaves (>= 0) in rope order, then SENTINEL; the
        // third slot may instead hold -(node + 2): more candidates than the
        // list holds, walk on from that node.  Each listed leaf passed the
        // leaf-box test; the point's own box test is tighter and spares the
        // point tests of most far leaves.  The boxes are loaded first, all at
        // once (independent loads), then tested.
        const int v[CAND_SLOTS] = {c4.y, c4.z, c4.w};
        unsigned hit = 0, lw[CAND_SLOTS];
#pragma unroll
        for (int c = 0; c < CAND_SLOTS; c++) {
            lw[c] = 0;
            if (v[c] >= 0) {
                float4 lo, hi;
                ld_node(T.nodes, L - 1 + v[c], lo, hi);
                lw[c] = __float_as_uint(lo.w);
                if (box_dist2_rn(p.x, p.y, p.z, lo, hi) <= e2)
                    hit |= 1u << c;
            }
        }
#pragma unroll
        for (int c = 0; c < CAND_SLOTS; c++)
            if ((hit >> c) & 1u)
                test_leaf(lw[c], leaf_first[v[c] + 1]);
        if (c4.w < SENTINEL)
            node = -c4.w - 2;
    }
    // the plain pair traversal: from i's own leaf (SCHED 2) or from the leaf
    // where the candidate list ran out (SCHED 1, without the early exit: it
    // would need the levels crossed before that leaf, and on dense data, where
    // lists overflow, it rarely fires; measured, it slowed this loop down)
    unsigned steps = 0;
    while (node != SENTINEL) {
        if (!node_ok(node, L, steps, dev_status))
            break;
        float4 lo, hi;
        ld_node(T.nodes, node, lo, hi);
        const int lv = level_of(hi);
        if (STATS)
            c_visit++;
        if (box_dist2_rn(p.x, p.y, p.z, lo, hi) <= e2) {
            if (node < L - 1) {
                node = __float_as_int(lo.w);
                continue;
            }
            test_leaf(__float_as_uint(lo.w), leaf_first[node - (L - 1) + 1]);
        }
        if (may_exit) {
            if (region_exit(lv, M, H))
                break;
            M = max(M, lv);
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

template <int SCHED, bool FOF, bool STATS>
__global__ void __launch_bounds__(1024, 2) k_union(int64_t n, const State *__restrict__ st, const SegState *__restrict__ seg,
                        const unsigned long long *k0, const unsigned long long *k1,
                        const float4 *__restrict__ spts, const float4 *__restrict__ nodes,
                        const int *__restrict__ leaf_of, const int *__restrict__ leaf_first,
                        const int4 *__restrict__ cand, int *parent,
                        unsigned char *core, unsigned *dev_status, TravStats *stats, int span)
{
    const int64_t i64 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const Tree T{nodes, leaf_first, st->n_leaves};
    if (FOF) {  // (measured: the own-leaf loop beats the shuffles when few pairs are neighbours)
        if (i64 < n)
            union_query<SCHED, true, STATS, false>((int)i64, true, 0, seg[0], T, spts, leaf_of, cand, parent, core,
                                                   dev_status, stats);
        return;
    }
    if (i64 - (threadIdx.x & 31) >= n)
        return;  // the whole warp is past the end
    // DBSCAN: every lane takes part in the own-leaf shuffles; lanes past the
    // end and non-core points only lend their coordinates
    const bool in = i64 < n;
    const int i = in ? (int)i64 : (int)n - 1;
    const bool active = in && core[i];
    union_query<SCHED, false, STATS, true>(i, active, span, seg[0], T, spts, leaf_of, cand, parent, core, dev_status,
                                           stats);
}

// Many segments: each query takes its segment's eps and mode from its key.
template <int SCHED, bool STATS>
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
        union_query<SCHED, true, STATS, false>(i, true, 0, g, T, spts, leaf_of, cand, parent, core, dev_status, stats);
    else if (core[i])
        union_query<SCHED, false, STATS, false>(i, true, 0, g, T, spts, leaf_of, cand, parent, core, dev_status,
                                                stats);
}

// ---- core counting with early termination (minPts > 2) -------------------------------

// A walk from the root reaches the query's own leaf (the box of a leaf holds
// its points); after it, the walk may stop at the first subtree it leaves that
// holds the query's leaf and every cell a neighbour can have (region_exit).
// M is the highest split level crossed since that leaf.
struct RootWalkExit {
    int own, H, M;
    bool past;
    __device__ __forceinline__ bool leave(int node, int lv)
    {
        if (node == own)
            past = true;
        if (!past)
            return false;
        if (region_exit(lv, M, H))
            return true;
        M = max(M, lv);
        return false;
    }
};

template <bool SEG>
__global__ void k_count(int64_t n, const State *__restrict__ st, const SegState *__restrict__ seg,
                        const unsigned long long *k0, const unsigned long long *k1,
                        const float4 *__restrict__ spts, const float4 *__restrict__ nodes,
                        const int *__restrict__ leaf_first, const int *__restrict__ leaf_of,
                        const int4 *__restrict__ cand, unsigned char *core, unsigned *dev_status)
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
    const int me = leaf_of[i];
    int cnt = 0;
    if (cand) {
        // Lower bound first: the own leaf's points (i itself among them) and
        // those of the listed candidate leaves (all after the own leaf in
        // pre-order, so none is counted twice).  Enough of them settle most
        // core points in dense data without the walk from the root.
        auto count_leaf = [&](int s0, int e) -> bool {
            for (int j = s0; j < e; j++) {
                const float4 q = __ldg(spts + j);
                if (dist2_rn(p.x, p.y, p.z, q.x, q.y, q.z) <= e2 && ++cnt >= minpts)
                    return true;
            }
            return false;
        };
        auto count_listed = [&](int v) -> bool {
            float4 lo, hi;
            ld_node(nodes, L - 1 + v, lo, hi);
            return box_dist2_rn(p.x, p.y, p.z, lo, hi) <= e2 &&
                   count_leaf((int)(__float_as_uint(lo.w) & ~DENSE_BIT), leaf_first[v + 1]);
        };
        const int4 c4 = cand[me];
        bool core_found = count_leaf(leaf_first[me], c4.x & ~DENSE_BIT);
        const int v[3] = {c4.y, c4.z, c4.w};
        bool ok = true;
#pragma unroll
        for (int c = 0; c < 3; c++) {
            ok = ok && v[c] >= 0;
            if (ok && !core_found)
                core_found = count_listed(v[c]);
        }
        if (core_found) {
            core[i] = 1;
            return;
        }
        cnt = 0;  // the full count walks the whole hierarchy
    }
    RootWalkExit ex{L - 1 + me, reach_level(p.x, p.y, p.z, p.x, p.y, p.z, g), 0, false};
    int node = g.root;
    unsigned steps = 0;
    while (node != SENTINEL) {
        if (!node_ok(node, L, steps, dev_status))
            break;
        float4 lo, hi;
        ld_node(nodes, node, lo, hi);
        const int lv = level_of(hi);
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
        if (ex.leave(node, lv))
            break;
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
                         const int *__restrict__ leaf_first, const int *__restrict__ leaf_of,
                         int *parent, const unsigned char *__restrict__ core,
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
    RootWalkExit ex{L - 1 + leaf_of[i], reach_level(p.x, p.y, p.z, p.x, p.y, p.z, g), 0, false};
    int best_k = 0x7fffffff, best_r = -1;
    int node = g.root;
    unsigned steps = 0;
    while (node != SENTINEL) {
        if (!node_ok(node, L, steps, dev_status))
            break;
        float4 lo, hi;
        ld_node(nodes, node, lo, hi);
        const int lv = level_of(hi);
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
        if (ex.leave(node, lv))
            break;
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

template <int SCHED>
static void launch_union(const Work &w, int g, int B, int span, TravStats *stats, cudaStream_t s)
{
    if (w.nseg > 1) {
        if (stats)
            k_union_seg<SCHED, true><<<g, B, 0, s>>>(w.n, w.st, w.seg, w.keys[0], w.keys[1], w.spts, w.nodes,
                                                     w.leaf_of, w.leaf_first, w.cand, w.parent, w.core,
                                                     w.dev_status, stats);
        else
            k_union_seg<SCHED, false><<<g, B, 0, s>>>(w.n, w.st, w.seg, w.keys[0], w.keys[1], w.spts, w.nodes,
                                                      w.leaf_of, w.leaf_first, w.cand, w.parent, w.core,
                                                      w.dev_status, nullptr);
    } else if (w.any_fof) {
        if (stats)
            k_union<SCHED, true, true><<<g, B, 0, s>>>(w.n, w.st, w.seg, w.keys[0], w.keys[1], w.spts, w.nodes,
                                                       w.leaf_of, w.leaf_first, w.cand, w.parent, w.core,
                                                       w.dev_status, stats, span);
        else
            k_union<SCHED, true, false><<<g, B, 0, s>>>(w.n, w.st, w.seg, w.keys[0], w.keys[1], w.spts, w.nodes,
                                                        w.leaf_of, w.leaf_first, w.cand, w.parent, w.core,
                                                        w.dev_status, nullptr, span);
    } else {
        if (stats)
            k_union<SCHED, false, true><<<g, B, 0, s>>>(w.n, w.st, w.seg, w.keys[0], w.keys[1], w.spts, w.nodes,
                                                        w.leaf_of, w.leaf_first, w.cand, w.parent, w.core,
                                                        w.dev_status, stats, span);
        else
            k_union<SCHED, false, false><<<g, B, 0, s>>>(w.n, w.st, w.seg, w.keys[0], w.keys[1], w.spts, w.nodes,
                                                         w.leaf_of, w.leaf_first, w.cand, w.parent, w.core,
                                                         w.dev_status, nullptr, span);
    }
    note_launch();
}

void stage_cluster(const Work &w, const Params &p, int32_t *labels, cudaStream_t s)
{
    const int B = p.block;
    const int g = div_up(w.n, B);
    const bool seg = w.nseg > 1;
    TravStats *stats = (TravStats *)w.stats;
    cudaMemsetAsync(labels, 0xff, (size_t)w.n * sizeof(int32_t), s);  // noise = -1
    if (p.schedule == 1) {
        const int gc = (int)std::min<int64_t>(div_up(w.n, 256), (int64_t)g_cand_blocks_per_sm * w.n_sms);
        if (seg)
            k_cand<true><<<gc, 256, 0, s>>>(w.st, w.seg, w.leaf_seg, w.nodes, w.leaf_first, w.cand, w.dev_status);
        else
            k_cand<false><<<gc, 256, 0, s>>>(w.st, w.seg, w.leaf_seg, w.nodes, w.leaf_first, w.cand, w.dev_status);
        note_launch();
    }
    prof_mark(ST_CANDS, s);
    if (w.any_dbscan) {
        const int4 *lists = p.schedule == 1 ? w.cand : nullptr;  // k_cand's lists, if it ran
        if (seg)
            k_count<true><<<g, B, 0, s>>>(w.n, w.st, w.seg, w.keys[0], w.keys[1], w.spts, w.nodes, w.leaf_first,
                                          w.leaf_of, lists, w.core, w.dev_status);
        else
            k_count<false><<<g, B, 0, s>>>(w.n, w.st, w.seg, w.keys[0], w.keys[1], w.spts, w.nodes, w.leaf_first,
                                           w.leaf_of, lists, w.core, w.dev_status);
        note_launch();
        prof_mark(ST_COUNT, s);
    }
    if (p.schedule == 1)
        launch_union<1>(w, g, B, p.leaf_size - 1, stats, s);
    else
        launch_union<2>(w, g, B, p.leaf_size - 1, stats, s);
    prof_mark(ST_UNION, s);
    if (w.any_dbscan) {
        if (seg)
            k_border<true><<<g, B, 0, s>>>(w.n, w.st, w.seg, w.keys[0], w.keys[1], w.spts, w.nodes, w.leaf_first,
                                           w.leaf_of, w.parent, w.core, w.bmin, w.dev_status);
        else
            k_border<false><<<g, B, 0, s>>>(w.n, w.st, w.seg, w.keys[0], w.keys[1], w.spts, w.nodes, w.leaf_first,
                                            w.leaf_of, w.parent, w.core, w.bmin, w.dev_status);
        note_launch();
        prof_mark(ST_BORDER, s);
    }
    if (seg)
        k_finalize<true><<<div_up(w.n, 256), 256, 0, s>>>(w.n, w.st, w.seg, w.seg_off, w.keys[0], w.keys[1], w.spts,
                                                          w.parent, w.core, w.bmin, labels);
    else
        k_finalize<false><<<div_up(w.n, 256), 256, 0, s>>>(w.n, w.st, w.seg, w.seg_off, w.keys[0], w.keys[1],
                                                           w.spts, w.parent, w.core, w.bmin, labels);
    note_launch();
    prof_mark(ST_FINALIZE, s);
}

void cluster_init_device()
{
    int b = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_cand<true>, 256, 0) != cudaSuccess || b < 1) {
        cudaGetLastError();
        b = 4;
    }
    g_cand_blocks_per_sm = b;
}

}  // namespace abx
