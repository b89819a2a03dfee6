// Dense cells, hierarchy leaves and the bottom-up LBVH with ropes.
//
// Paper, section "ArborX library": a binary BVH whose leaves wrap the objects
// and whose nodes enclose their children, built from Z-curve sorted objects by
// a single bottom-up pass.  Subsection "Stackless traversal": every node gets
// a rope (escape index), the next node to visit when its box test fails or
// after a leaf; ropes on the right-most path go to a sentinel.  The paper
// builds with Apetrei's bottom-up algorithm and recovers Karras' node order to
// set the ropes.  Here the nodes keep Apetrei's numbering (internal node k
// splits leaves k and k+1) and the ropes come straight from it: the next node
// in pre-order after a subtree whose leaves end at b is the right child of
// internal node b, the highest node whose range starts at b + 1.
//
// Subsection "FDBSCAN-DenseBox": a grid of side eps/sqrt(d) is laid over the
// points; a cell with at least minPts points holds only core points, and the
// hierarchy is built over a mix of those dense cells and the other points.
// Here the cells are runs of equal Morton prefix; a cell is dense when it has
// at least max(minPts, 2) points AND the rounded predicate holds across the
// box of its points (so every pair inside it is a neighbour pair under the
// exact FP32 test, whatever rounding did to the grid).  Dense cells are leaves;
// the other points are grouped into leaves of up to leaf_size consecutive
// points.
#include "work.cuh"
#include "scan.cuh"

namespace abx {

// Leaves are whole subtrees of the point-level radix tree (the tree the
// build would make with one point per leaf): for a point outside dense cells
// its leaf is the highest subtree containing it that holds at most leaf_size
// points and no dense-cell point; a dense cell (itself such a subtree: one
// Morton prefix) is one leaf.  Cutting at arbitrary multiples of leaf_size
// instead lets leaves straddle Z-curve jumps, whose boxes then inflate every
// ancestor box.
//
// The boundary x between sorted points x and x+1 is the split of exactly one
// internal node, whose points run from just after the nearest boundary on the
// left with a higher split level to the nearest boundary on the right with an
// equal or higher one (the build's parent rule: merge across the lower level,
// ties merge left).  x is inside a leaf iff that node holds at most leaf_size
// points and no dense point; so only 2 * leaf_size split levels are read.
// Side effects for dense points: hooked under the cell's root, marked core.
struct LeafFlag {
    const int *dense_root;
    const unsigned char *pdelta;  // split level between sorted points k and k+1
    int *parent;
    unsigned char *core;
    const State *st;
    const unsigned long long *k0, *k1;
    int leaf_size;
    int64_t n;
    __device__ bool operator()(int64_t k64) const
    {
        const int k = (int)k64;
        const bool dok = st->dense_ok;
        if (dok) {
            const int rb = dense_root[k];
            if (rb >= 0) {
                core[k] = 1;
                if (rb != k)
                    parent[k] = rb;
                return k == 0 || dense_root[k - 1] != rb;
            }
            if (k > 0 && dense_root[k - 1] >= 0)
                return true;  // first point after a dense cell
        }
        if (k == 0)
            return true;
        if (st->nseg > 1) {  // leaves never cross segments
            if (seg_of_key(sorted_key(st, k0, k1, k), st->shift) !=
                seg_of_key(sorted_key(st, k0, k1, k - 1), st->shift))
                return true;
        }
        const int x = k - 1, B = leaf_size, last = (int)n - 1;
        const int d = pdelta[x];
        int yr = x + 1;  // nearest boundary on the right with level >= d
        while (yr < last && pdelta[yr] < d) {
            if (++yr - x > B)
                return true;
        }
        int yl = x - 1;  // nearest boundary on the left with level > d
        while (yl >= 0 && pdelta[yl] <= d) {
            if (x - --yl > B)
                return true;
        }
        if (yr - yl > B)  // the node holds points yl + 1 .. yr
            return true;
        if (dok)
            for (int y = yl + 1; y <= yr; y++)
                if (dense_root[y] >= 0)
                    return true;
        return false;
    }

    // The SCAN_ITEMS flags starting at base (a multiple of 16).  For leaf sizes
    // up to 8 and no dense cells or segments the rule needs only the split
    // levels within 8 boundaries of each boundary: they are loaded once into a
    // register window and compared four at a time.
    __device__ unsigned flags(int64_t base64, int64_t n64) const
    {
        const bool simple = leaf_size <= 8 && !st->dense_ok && st->nseg == 1;
        unsigned m = 0;
        if (!simple) {
#pragma unroll 1
            for (int j = 0; j < SCAN_ITEMS; j++)
                if (base64 + j < n64 && (*this)(base64 + j))
                    m |= 1u << j;
            return m;
        }
        const int base = (int)base64, n = (int)n64, B = leaf_size;
        // window byte i = split level of boundary base - 12 + i (255 outside 0 .. n-2)
        unsigned w[10];
#pragma unroll
        for (int k = 0; k < 10; k++) {
            const int y0 = base - 12 + 4 * k;
            if (y0 >= 0 && y0 + 3 <= n - 2) {
                w[k] = *reinterpret_cast<const unsigned *>(pdelta + y0);
            } else {
                unsigned v = 0;
#pragma unroll
                for (int t = 0; t < 4; t++) {
                    const int y = y0 + t;
                    const unsigned b = (y >= 0 && y <= n - 2) ? pdelta[y] : 255u;
                    v |= b << (8 * t);
                }
                w[k] = v;
            }
        }
#pragma unroll
        for (int j = 0; j < SCAN_ITEMS; j++) {
            const int k = base + j;
            if (k >= n)
                break;
            if (k == 0) {
                m |= 1u;
                continue;
            }
            // boundary x = k - 1 sits at window byte j + 11
            const int ox = j + 11;
            const unsigned d = (w[ox / 4] >> (8 * (ox % 4))) & 0xffu;
            const unsigned dd = d * 0x01010101u;
            // right: boundaries x+1 .. x+8 at bytes j+12 .. j+19; nearest with level >= d
            const int orr = j + 12;
            const unsigned r0 = __funnelshift_r(w[orr / 4], w[orr / 4 + 1], 8 * (orr % 4));
            const unsigned r1 = __funnelshift_r(w[orr / 4 + 1], w[orr / 4 + 2], 8 * (orr % 4));
            const unsigned long long mr =
                (unsigned long long)__vcmpgeu4(r0, dd) | ((unsigned long long)__vcmpgeu4(r1, dd) << 32);
            // left: boundaries x-8 .. x-1 at bytes j+3 .. j+10; nearest with level > d
            const int ol = j + 3;
            const unsigned l0 = __funnelshift_r(w[ol / 4], w[ol / 4 + 1], 8 * (ol % 4));
            const unsigned l1 = __funnelshift_r(w[ol / 4 + 1], w[ol / 4 + 2], 8 * (ol % 4));
            const unsigned long long ml =
                (unsigned long long)__vcmpgtu4(l0, dd) | ((unsigned long long)__vcmpgtu4(l1, dd) << 32);
            if (!mr || !ml) {
                m |= 1u << j;  // one side alone holds more than 8 points
                continue;
            }
            const int yr = k + (__ffsll((long long)mr) - 1) / 8;              // x + 1 + byte
            const int yl = k - 9 + (63 - __clzll((long long)ml)) / 8;          // x - 8 + byte
            if (yr - yl > B)
                m |= 1u << j;
        }
        return m;
    }
};

// ---- dense cells (one pass, no scan) ---------------------------------------------
// The thread at the first point of each cell (a run of equal Morton prefix)
// walks the run; a run with at least min_count points whose point box passes
// the rounded predicate is dense: every member gets the member with the
// smallest original index as dense_root (else dense_root stays -1).

__global__ void __launch_bounds__(256) k_dense_cells(int64_t n, State *st, const SegState *__restrict__ seg,
                                                     const unsigned long long *k0, const unsigned long long *k1,
                                                     const float4 *__restrict__ spts, int *dense_root, int dense_min)
{
    if (!st->dense_ok)
        return;
    const int sh = 3 * st->sub, shift = st->shift;
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x) {
        const unsigned long long key = sorted_key(st, k0, k1, k);
        const unsigned long long c = key >> sh;
        if (k > 0 && (sorted_key(st, k0, k1, k - 1) >> sh) == c)
            continue;  // not the first point of its cell
        const SegState &g = seg[seg_of_key(key, shift)];
        if (!g.dense_ok)
            continue;
        const float e2 = g.e2;
        const int min_count = max(max(g.minpts, 2), dense_min);
        int64_t e = k + 1;
        while (e < n && (sorted_key(st, k0, k1, e) >> sh) == c && e - k < min_count)
            e++;
        if (e - k < min_count)
            continue;
        while (e < n && (sorted_key(st, k0, k1, e) >> sh) == c)
            e++;
        float4 p = spts[k];
        float lx = p.x, ly = p.y, lz = p.z, hx = p.x, hy = p.y, hz = p.z;
        int best = __float_as_int(p.w), root = (int)k;
        for (int64_t j = k + 1; j < e; j++) {
            float4 q = spts[j];
            lx = fminf(lx, q.x); ly = fminf(ly, q.y); lz = fminf(lz, q.z);
            hx = fmaxf(hx, q.x); hy = fmaxf(hy, q.y); hz = fmaxf(hz, q.z);
            int o = __float_as_int(q.w);
            if (o < best) {
                best = o;
                root = (int)j;
            }
        }
        // every pair of points in the box passes the rounded predicate
        if (dist2_rn(hx, hy, hz, lx, ly, lz) <= e2) {
            for (int64_t j = k; j < e; j++)
                dense_root[j] = root;
            atomicAdd(&st->n_cells, 1);
        }
    }
}

// ---- leaf records and split levels --------------------------------------------------
// Record i (two float4): internal node i < L-1: (lo, left child), (hi, rope);
// leaf t at i = L-1+t: (lo, first point | DENSE_BIT), (hi, rope).

__global__ void __launch_bounds__(256) k_leaves(const State *st, SegState *seg, const unsigned long long *k0,
                                                const unsigned long long *k1, const unsigned char *__restrict__ pdelta,
                                                const float4 *__restrict__ spts, const int *leaf_first,
                                                const int *dense_root, float4 *nodes, unsigned char *delta,
                                                int *leaf_seg)
{
    const int L = st->n_leaves;
    const int dense_ok = st->dense_ok;
    const int nseg = st->nseg, shift = st->shift;
    const int64_t n = leaf_first[L];
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < L; t += gridDim.x * blockDim.x) {
        int s = leaf_first[t], e = leaf_first[t + 1];
        float4 p = spts[s];
        float lx = p.x, ly = p.y, lz = p.z, hx = p.x, hy = p.y, hz = p.z;
        for (int j = s + 1; j < e; j++) {
            float4 q = spts[j];
            lx = fminf(lx, q.x); ly = fminf(ly, q.y); lz = fminf(lz, q.z);
            hx = fmaxf(hx, q.x); hy = fmaxf(hy, q.y); hz = fmaxf(hz, q.z);
        }
        unsigned w0 = (unsigned)s;
        if (dense_ok && dense_root[s] >= 0)
            w0 |= DENSE_BIT;
        size_t r = 2 * ((size_t)(L - 1) + t);
        nodes[r] = make_float4(lx, ly, lz, __uint_as_float(w0));
        nodes[r + 1] = make_float4(hx, hy, hz, __int_as_float(SENTINEL));
        if (t < L - 1)
            delta[t] = pdelta[e - 1];  // the point-level split level at the leaf boundary
        int sg = 0;
        if (nseg > 1) {
            sg = seg_of_key(sorted_key(st, k0, k1, s), shift);
            const bool first = s == 0 || seg_of_key(sorted_key(st, k0, k1, s - 1), shift) != sg;
            const bool last = e == n || seg_of_key(sorted_key(st, k0, k1, e), shift) != sg;
            if (first && last)
                seg[sg].root = L - 1 + t;  // a segment of a single leaf
        } else if (L == 1) {
            seg[0].root = 0;
        }
        leaf_seg[t] = sg;
    }
}

// ---- bottom-up build -----------------------------------------------------------------
// A node covering leaves [l, r] becomes the left child of internal node r when
// l == 0 or delta[r] < delta[l-1] (r < L-1), else the right child of node l-1.
// Of the two children of a node, the first to arrive parks (its node id and
// its outer bound) in the parent's slot and stops; the second merges the boxes,
// writes the parent and climbs on.
//
// Phase 1 (one block per chunk of BUILD_CHUNK consecutive leaves): parents
// whose split lies inside the chunk meet in shared memory, so most of the tree
// is built without global atomics.  A node whose parent split is outside the
// chunk, or that is still parked when the block ends (its sibling reaches
// outside the chunk), is appended to a frontier list.
// Phase 2 (global): the frontier nodes climb the rest of the way, meeting in
// global slots through acquire-release exchanges.

constexpr unsigned long long SLOT_EMPTY = ~0ull;
constexpr unsigned long long SLOT_DONE = ~1ull;
constexpr int BUILD_CHUNK = 1024;

__device__ __forceinline__ unsigned long long exch_acq_rel(unsigned long long *p, unsigned long long v)
{
    unsigned long long old;
    asm volatile("atom.acq_rel.gpu.global.exch.b64 %0, [%1], %2;" : "=l"(old) : "l"(p), "l"(v) : "memory");
    return old;
}

__device__ __forceinline__ void write_parent(float4 *nodes, int *right_of, int p, const float *b, int lc, int rc,
                                             int r)
{
    // w of hi temporarily holds the range end r (turned into the rope later)
    nodes[2 * (size_t)p] = make_float4(b[0], b[1], b[2], __int_as_float(lc));
    nodes[2 * (size_t)p + 1] = make_float4(b[3], b[4], b[5], __int_as_float(r));
    right_of[p] = rc;
}

// A completed node that covers exactly the leaves of one segment is that
// segment's root (the top of the subtree its full traversals start from).
__device__ __forceinline__ void note_seg_root(SegState *seg, const int *leaf_seg, int nseg, int L, int p, int l,
                                              int r)
{
    if (nseg == 1) {
        if (l == 0 && r == L - 1)
            seg[0].root = p;
        return;
    }
    const int s = leaf_seg[l];
    if ((l == 0 || leaf_seg[l - 1] != s) && (r == L - 1 || leaf_seg[r + 1] != s))
        seg[s].root = p;
}

__device__ __forceinline__ void push_frontier(int4 *frontier, int *count, int node, int l, int r)
{
    int k = atomicAdd(count, 1);
    frontier[k] = make_int4(node, l, r, 0);
}

constexpr size_t BUILD_SMEM = (size_t)(BUILD_CHUNK - 1) * (2 * 6 * sizeof(float) + sizeof(unsigned long long));

__global__ void __launch_bounds__(BUILD_CHUNK) k_build_local(State *st, SegState *seg, const int *leaf_seg,
                                                             const unsigned char *__restrict__ delta,
                                                             float4 *nodes, int *right_of, int4 *frontier,
                                                             int *frontier_count)
{
    const int nseg = st->nseg;
    extern __shared__ __align__(16) unsigned char smem[];
    unsigned long long *stag = reinterpret_cast<unsigned long long *>(smem);
    float *sbox = reinterpret_cast<float *>(stag + (BUILD_CHUNK - 1));  // [slot][side][6]
    const int L = st->n_leaves;
    const int c0 = blockIdx.x * BUILD_CHUNK;
    if (c0 >= L)
        return;
    for (int i = threadIdx.x; i < BUILD_CHUNK - 1; i += blockDim.x)
        stag[i] = SLOT_EMPTY;
    __syncthreads();
    const int t = c0 + threadIdx.x;
    if (t < L) {
        int node = L - 1 + t, l = t, r = t;
        float4 lo = nodes[2 * (size_t)node], hi = nodes[2 * (size_t)node + 1];
        float b[6] = {lo.x, lo.y, lo.z, hi.x, hi.y, hi.z};
        if (L == 1)
            st->root = node;
        while (L > 1) {
            const bool left = (l == 0) || (r != L - 1 && delta[r] < delta[l - 1]);
            const int p = left ? r : l - 1;
            if (p < c0 || p > c0 + BUILD_CHUNK - 2) {
                push_frontier(frontier, frontier_count, node, l, r);
                break;
            }
            const int q = p - c0, side = left ? 0 : 1;
            float *mine = sbox + (q * 2 + side) * 6;
#pragma unroll
            for (int k = 0; k < 6; k++)
                mine[k] = b[k];
            __threadfence_block();
            const unsigned long long tag = ((unsigned long long)(unsigned)node << 32) |
                                           ((unsigned long long)side << 31) | (unsigned)(left ? l : r);
            const unsigned long long other = atomicExch(stag + q, tag);
            if (other == SLOT_EMPTY)
                break;  // parked: the sibling will continue
            stag[q] = SLOT_DONE;
            __threadfence_block();
            const int sib = (int)(other >> 32);
            const int bound = (int)(other & 0x7fffffffu);
            const float *theirs = sbox + (q * 2 + (1 - side)) * 6;
            b[0] = fminf(b[0], theirs[0]); b[1] = fminf(b[1], theirs[1]); b[2] = fminf(b[2], theirs[2]);
            b[3] = fmaxf(b[3], theirs[3]); b[4] = fmaxf(b[4], theirs[4]); b[5] = fmaxf(b[5], theirs[5]);
            if (left)
                r = bound;
            else
                l = bound;
            write_parent(nodes, right_of, p, b, left ? node : sib, left ? sib : node, r);
            note_seg_root(seg, leaf_seg, nseg, L, p, l, r);
            node = p;
            if (l == 0 && r == L - 1) {
                st->root = p;
                break;
            }
        }
    }
    __syncthreads();
    // nodes still parked: their sibling reaches outside the chunk
    for (int q = threadIdx.x; q < BUILD_CHUNK - 1; q += blockDim.x) {
        const unsigned long long tag = stag[q];
        if (tag == SLOT_EMPTY || tag == SLOT_DONE)
            continue;
        const int node = (int)(tag >> 32);
        const int bound = (int)(tag & 0x7fffffffu);
        const int p = c0 + q;
        if ((tag >> 31) & 1u)  // right child [p + 1, bound]
            push_frontier(frontier, frontier_count, node, p + 1, bound);
        else                   // left child [bound, p]
            push_frontier(frontier, frontier_count, node, bound, p);
    }
}

__global__ void __launch_bounds__(256) k_build_global(State *st, SegState *seg, const int *leaf_seg,
                                                      const unsigned char *__restrict__ delta,
                                                      float4 *nodes, unsigned long long *slot, int *right_of,
                                                      const int4 *frontier, const int *frontier_count)
{
    const int L = st->n_leaves;
    const int nseg = st->nseg;
    const int nf = *frontier_count;
    for (int f = blockIdx.x * blockDim.x + threadIdx.x; f < nf; f += gridDim.x * blockDim.x) {
        const int4 it = frontier[f];
        int node = it.x, l = it.y, r = it.z;
        float4 lo = ld_cg4(nodes + 2 * (size_t)node), hi = ld_cg4(nodes + 2 * (size_t)node + 1);
        while (true) {
            const bool left = (l == 0) || (r != L - 1 && delta[r] < delta[l - 1]);
            const int p = left ? r : l - 1;
            const unsigned long long mine = ((unsigned long long)(unsigned)node << 32) | (unsigned)(left ? l : r);
            const unsigned long long other = exch_acq_rel(slot + p, mine);
            if (other == SLOT_EMPTY)
                break;
            const int sib = (int)(other >> 32);
            const int bound = (int)(unsigned)other;
            if (left)
                r = bound;
            else
                l = bound;
            const float4 slo = ld_cg4(nodes + 2 * (size_t)sib), shi = ld_cg4(nodes + 2 * (size_t)sib + 1);
            lo.x = fminf(lo.x, slo.x); lo.y = fminf(lo.y, slo.y); lo.z = fminf(lo.z, slo.z);
            hi.x = fmaxf(hi.x, shi.x); hi.y = fmaxf(hi.y, shi.y); hi.z = fmaxf(hi.z, shi.z);
            const float b[6] = {lo.x, lo.y, lo.z, hi.x, hi.y, hi.z};
            write_parent(nodes, right_of, p, b, left ? node : sib, left ? sib : node, r);
            note_seg_root(seg, leaf_seg, nseg, L, p, l, r);
            node = p;
            if (l == 0 && r == L - 1) {
                st->root = p;
                break;
            }
        }
    }
}

// rope(node covering [.., b]) = right child of internal node b, or the
// sentinel; the split level of leaf boundary b, which following the rope
// crosses (255 with the sentinel), goes into the low bits of hi.x for the
// early exit of the rope walks (with_level).
__global__ void __launch_bounds__(256) k_ropes(const State *st, float4 *nodes, const int *right_of,
                                               const int *leaf_seg, const unsigned char *__restrict__ delta,
                                               unsigned *dev_status)
{
    const int L = st->n_leaves;
    const int nseg = st->nseg;
    const int total = 2 * L - 1;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < total; i += gridDim.x * blockDim.x) {
        float4 hi = nodes[2 * (size_t)i + 1];
        const int b = i < L - 1 ? __float_as_int(hi.w) : i - (L - 1);
        int rope = SENTINEL;
        unsigned lv = 255;
        if ((unsigned)b >= (unsigned)L) {
            atomicOr(dev_status, DEV_INTERNAL);  // node never completed: corrupted build
        } else if (b != L - 1 && (nseg == 1 || leaf_seg[b] == leaf_seg[b + 1])) {
            rope = right_of[b];  // else: last leaf of its segment -> sentinel
            lv = delta[b];
        }
        hi.x = with_level(hi.x, lv);
        hi.w = __int_as_float(rope);
        nodes[2 * (size_t)i + 1] = hi;
    }
}

// ---- launchers -------------------------------------------------------------------------

static int grid_cap(const Work &w, int64_t n, int block, int per_sm = 8)
{
    int64_t g = div_up(n, block);
    int64_t cap = (int64_t)w.n_sms * per_sm;
    if (g > cap)
        g = cap;
    return (int)(g < 1 ? 1 : g);
}

void stage_cells_leaves(const Work &w, const Params &p, cudaStream_t s)
{
    const int scan_tiles = div_up(w.n, SCAN_TILE);
    if (p.dense) {  // (with dense cells off no segment is dense_ok, and nothing reads dense_root)
        cudaMemsetAsync(w.dense_root, 0xff, (size_t)w.n * sizeof(int), s);
        k_dense_cells<<<grid_cap(w, w.n, 256, 16), 256, 0, s>>>(w.n, w.st, w.seg, w.keys[0], w.keys[1], w.spts,
                                                                w.dense_root, p.dense_min);
        note_launch(1);
    }
    prof_mark(ST_CELLS, s);
    cudaMemsetAsync(w.scan_lb, 0, w.scan_tiles * sizeof(unsigned long long), s);
    LeafFlag lf{w.dense_root, w.pdelta, w.parent, w.core, w.st, w.keys[0], w.keys[1], p.leaf_size, w.n};
    k_flag_scan<<<scan_tiles, SCAN_THREADS, 0, s>>>(w.n, lf, w.leaf_of, w.leaf_first, &w.st->n_leaves,
                                                    &w.st->tile_ctr[MAX_PASSES + 1], w.scan_lb, w.dev_status, w.st,
                                                    0);
    k_leaves<<<grid_cap(w, w.n, 256), 256, 0, s>>>(w.st, w.seg, w.keys[0], w.keys[1], w.pdelta, w.spts, w.leaf_first,
                                                   w.dense_root, w.nodes, w.delta, w.leaf_seg);
    note_launch(2);
    prof_mark(ST_LEAVES, s);
}

void stage_hierarchy(const Work &w, cudaStream_t s)
{
    cudaMemsetAsync(w.slot, 0xff, (size_t)w.n * sizeof(unsigned long long), s);
    k_build_local<<<div_up(w.n, BUILD_CHUNK), BUILD_CHUNK, BUILD_SMEM, s>>>(w.st, w.seg, w.leaf_seg, w.delta, w.nodes,
                                                                            w.right_of, w.frontier,
                                                                            &w.st->frontier_count);
    k_build_global<<<grid_cap(w, w.n / 16 + 1, 256), 256, 0, s>>>(w.st, w.seg, w.leaf_seg, w.delta, w.nodes, w.slot,
                                                                  w.right_of, w.frontier, &w.st->frontier_count);
    k_ropes<<<grid_cap(w, 2 * w.n, 256), 256, 0, s>>>(w.st, w.nodes, w.right_of, w.leaf_seg, w.delta,
                                                      w.dev_status);
    note_launch(3);
    prof_mark(ST_BUILD, s);
}

void tree_init_device()
{
    cudaFuncSetAttribute(k_build_local, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)BUILD_SMEM);
}

}  // namespace abx
