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

namespace abx {

__device__ __forceinline__ int final_pass_count(const State *st) { return st->pad[0]; }

__device__ __forceinline__ const unsigned long long *sorted_keys(const State *st, unsigned long long *const k0,
                                                                  unsigned long long *const k1)
{
    return (final_pass_count(st) & 1) ? k1 : k0;
}

// ---- single-pass flag scan (decoupled look-back) --------------------------------
// ids[k] = number of flagged positions <= k, minus one; first[id] = k for each
// flagged k; first[total] = n; *total_out = total.

constexpr unsigned long long SLB_AGG = 1ull << 62;
constexpr unsigned long long SLB_PRE = 2ull << 62;

__device__ __forceinline__ unsigned long long sld(const unsigned long long *p)
{
    unsigned long long v;
    asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void sst(unsigned long long *p, unsigned long long v)
{
    asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

template <class F>
__global__ void __launch_bounds__(SCAN_THREADS) k_flag_scan(int64_t n, F f, int *ids, int *first, int *total_out,
                                                            unsigned *tile_ctr, unsigned long long *lb,
                                                            unsigned *dev_status, const State *st, int need_dense)
{
    if (need_dense && !st->dense_ok)
        return;
    __shared__ int s_tile;
    __shared__ unsigned s_wsum[SCAN_THREADS / 32];
    __shared__ unsigned long long s_excl;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (tid == 0)
        s_tile = (int)atomicAdd(tile_ctr, 1u);
    __syncthreads();
    const int tile = s_tile;
    const int64_t base = (int64_t)tile * SCAN_TILE + (int64_t)tid * SCAN_ITEMS;
    unsigned flags = 0;  // bit j = flag of item j
#pragma unroll
    for (int j = 0; j < SCAN_ITEMS; j++) {
        int64_t pos = base + j;
        if (pos < n && f(pos))
            flags |= 1u << j;
    }
    unsigned c = __popc(flags);
    unsigned x = c;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        unsigned y = __shfl_up_sync(~0u, x, o);
        if (lane >= o)
            x += y;
    }
    if (lane == 31)
        s_wsum[warp] = x;
    __syncthreads();
    unsigned wpre = 0, total = 0;
    for (int w = 0; w < SCAN_THREADS / 32; w++) {
        if (w < warp)
            wpre += s_wsum[w];
        total += s_wsum[w];
    }
    if (tid == 0) {
        unsigned long long excl = 0;
        if (tile == 0) {
            sst(lb, SLB_PRE | total);
        } else {
            sst(lb + tile, SLB_AGG | total);
            for (int t = tile - 1; t >= 0; t--) {
                unsigned long long v;
                int spins = 0;
                while (true) {
                    v = sld(lb + t);
                    if ((v >> 62) != 0)
                        break;
                    if (++spins > SPIN_LIMIT) {
                        atomicOr(dev_status, DEV_TIMEOUT);
                        v = SLB_PRE;
                        break;
                    }
                    if (spins > 64)
                        __nanosleep(64);
                }
                excl += v & ((1ull << 62) - 1);
                if ((v >> 62) == 2)
                    break;
            }
            sst(lb + tile, SLB_PRE | (excl + total));
        }
        s_excl = excl;
    }
    __syncthreads();
    unsigned long long run = s_excl + wpre + x - c;  // flags before this thread's first item
#pragma unroll
    for (int j = 0; j < SCAN_ITEMS; j++) {
        int64_t pos = base + j;
        if (pos < n) {
            if (flags & (1u << j)) {
                first[run] = (int)pos;
                run++;
            }
            ids[pos] = (int)run - 1;
            if (pos == n - 1) {
                first[run] = (int)n;
                *total_out = (int)run;
            }
        }
    }
}

// cell boundary: the Morton prefix above the sub-cell bits changes
struct CellFlag {
    const unsigned long long *k0, *k1;
    const State *st;
    __device__ bool operator()(int64_t k) const
    {
        const unsigned long long *keys = sorted_keys(st, const_cast<unsigned long long *>(k0),
                                                     const_cast<unsigned long long *>(k1));
        if (k == 0)
            return true;
        int sh = 3 * st->sub;
        return (keys[k] >> sh) != (keys[k - 1] >> sh);
    }
};

// leaf boundary: a dense cell starts, the point after a dense cell, or every
// leaf_size points within a run of non-dense points; also applies the dense
// cells to the union-find (every member hooked under the cell's root) and
// marks their points core.
struct LeafFlag {
    const int *cell_id, *cell_root;
    const unsigned char *cell_dense;
    int *parent;
    unsigned char *core;
    const State *st;
    int leaf_size;
    __device__ bool operator()(int64_t k) const
    {
        if (!st->dense_ok)
            return (k % leaf_size) == 0;
        int c = cell_id[k];
        if (cell_dense[c]) {
            core[k] = 1;
            int r = cell_root[c];
            if (r != (int)k)
                parent[k] = r;
            return k == 0 || cell_id[k - 1] != c;
        }
        if (k == 0)
            return true;
        int cp = cell_id[k - 1];
        if (cp != c && cell_dense[cp])
            return true;
        return (k % leaf_size) == 0;
    }
};

// ---- dense cells ------------------------------------------------------------------

__global__ void __launch_bounds__(256) k_dense_cells(int64_t n, const State *st, const int *cell_start,
                                                     const float4 *__restrict__ spts, unsigned char *cell_dense,
                                                     int *cell_root, float e2, int min_count)
{
    if (!st->dense_ok)
        return;
    const int nc = st->n_cells;
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < nc; c += gridDim.x * blockDim.x) {
        int s = cell_start[c], e = cell_start[c + 1];
        unsigned char dense = 0;
        if (e - s >= min_count) {
            float4 p = spts[s];
            float lx = p.x, ly = p.y, lz = p.z, hx = p.x, hy = p.y, hz = p.z;
            int best = __float_as_int(p.w), root = s;
            for (int j = s + 1; j < e; j++) {
                float4 q = spts[j];
                lx = fminf(lx, q.x); ly = fminf(ly, q.y); lz = fminf(lz, q.z);
                hx = fmaxf(hx, q.x); hy = fmaxf(hy, q.y); hz = fmaxf(hz, q.z);
                int o = __float_as_int(q.w);
                if (o < best) {
                    best = o;
                    root = j;
                }
            }
            // every pair of points in the box passes the rounded predicate
            if (dist2_rn(hx, hy, hz, lx, ly, lz) <= e2) {
                dense = 1;
                cell_root[c] = root;
            }
        }
        cell_dense[c] = dense;
    }
}

// ---- leaf records and split levels --------------------------------------------------
// Record i (two float4): internal node i < L-1: (lo, left child), (hi, rope);
// leaf t at i = L-1+t: (lo, first point | DENSE_BIT), (hi, rope).

__device__ __forceinline__ unsigned char split_level(unsigned long long a, unsigned long long b, int t)
{
    unsigned long long x = a ^ b;
    if (x)
        return (unsigned char)(32 + (64 - __clzll((long long)x)));
    return (unsigned char)(32 - __clz(t ^ (t + 1)));
}

__global__ void __launch_bounds__(256) k_leaves(const State *st, const unsigned long long *k0,
                                                const unsigned long long *k1, const float4 *__restrict__ spts,
                                                const int *leaf_first, const int *cell_id,
                                                const unsigned char *cell_dense, float4 *nodes,
                                                unsigned char *delta)
{
    const int L = st->n_leaves;
    const unsigned long long *keys = sorted_keys(st, const_cast<unsigned long long *>(k0),
                                                 const_cast<unsigned long long *>(k1));
    const int dense_ok = st->dense_ok;
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
        if (dense_ok && cell_dense[cell_id[s]])
            w0 |= DENSE_BIT;
        size_t r = 2 * ((size_t)(L - 1) + t);
        nodes[r] = make_float4(lx, ly, lz, __uint_as_float(w0));
        nodes[r + 1] = make_float4(hx, hy, hz, __int_as_float(SENTINEL));
        if (t < L - 1)
            delta[t] = split_level(keys[e - 1], keys[e], t);
    }
}

// ---- bottom-up build (one thread per leaf climbs while it arrives second) -----------
// A node covering leaves [l, r] becomes the left child of internal node r when
// l == 0 or delta[r] < delta[l-1] (r < L-1), else the right child of node l-1.
// The first of two children to arrive parks (its node, its outer bound) in the
// parent's slot and stops; the second merges the boxes and goes on.

constexpr unsigned long long SLOT_EMPTY = ~0ull;

__global__ void __launch_bounds__(256) k_build(State *st, const unsigned char *__restrict__ delta, float4 *nodes,
                                               unsigned long long *slot, int *right_of)
{
    const int L = st->n_leaves;
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < L; t += gridDim.x * blockDim.x) {
        int node = L - 1 + t;
        if (L == 1) {
            st->root = node;
            continue;
        }
        int l = t, r = t;
        float4 lo = nodes[2 * (size_t)node], hi = nodes[2 * (size_t)node + 1];
        while (true) {
            bool left = (l == 0) || (r != L - 1 && delta[r] < delta[l - 1]);
            int p = left ? r : l - 1;
            unsigned long long mine = ((unsigned long long)(unsigned)node << 32) | (unsigned)(left ? l : r);
            __threadfence();
            unsigned long long other = atomicExch(slot + p, mine);
            if (other == SLOT_EMPTY)
                break;
            __threadfence();
            int sib = (int)(other >> 32);
            int bound = (int)(unsigned)other;
            if (left)
                r = bound;
            else
                l = bound;
            float4 slo = ld_cg4(nodes + 2 * (size_t)sib), shi = ld_cg4(nodes + 2 * (size_t)sib + 1);
            lo.x = fminf(lo.x, slo.x); lo.y = fminf(lo.y, slo.y); lo.z = fminf(lo.z, slo.z);
            hi.x = fmaxf(hi.x, shi.x); hi.y = fmaxf(hi.y, shi.y); hi.z = fmaxf(hi.z, shi.z);
            int lc = left ? node : sib, rc = left ? sib : node;
            // w of hi temporarily holds the range end r (turned into the rope later)
            nodes[2 * (size_t)p] = make_float4(lo.x, lo.y, lo.z, __int_as_float(lc));
            nodes[2 * (size_t)p + 1] = make_float4(hi.x, hi.y, hi.z, __int_as_float(r));
            right_of[p] = rc;
            node = p;
            if (l == 0 && r == L - 1) {
                st->root = p;
                break;
            }
        }
    }
}

// rope(node covering [.., b]) = right child of internal node b, or the sentinel
__global__ void __launch_bounds__(256) k_ropes(const State *st, float4 *nodes, const int *right_of,
                                               unsigned *dev_status)
{
    const int L = st->n_leaves;
    const int total = 2 * L - 1;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < total; i += gridDim.x * blockDim.x) {
        int b = i < L - 1 ? __float_as_int(nodes[2 * (size_t)i + 1].w) : i - (L - 1);
        int rope = SENTINEL;
        if ((unsigned)b >= (unsigned)L)
            atomicOr(dev_status, DEV_INTERNAL);  // node never completed: corrupted build
        else if (b != L - 1)
            rope = right_of[b];
        reinterpret_cast<int *>(nodes + 2 * (size_t)i + 1)[3] = rope;
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

void stage_cells_leaves(const Work &w, float eps, int minpts, const Params &p, cudaStream_t s)
{
    const int scan_tiles = div_up(w.n, SCAN_TILE);
    cudaMemsetAsync(w.scan_lb, 0, 2 * w.scan_tiles * sizeof(unsigned long long), s);
    CellFlag cf{w.keys[0], w.keys[1], w.st};
    k_flag_scan<<<scan_tiles, SCAN_THREADS, 0, s>>>(w.n, cf, w.cell_id, w.cell_start, &w.st->n_cells,
                                                    &w.st->tile_ctr[MAX_PASSES], w.scan_lb, w.dev_status, w.st, 1);
    const float e2 = eps * eps;
    const int min_count = minpts < 2 ? 2 : minpts;
    k_dense_cells<<<grid_cap(w, w.n, 256), 256, 0, s>>>(w.n, w.st, w.cell_start, w.spts, w.cell_dense, w.cell_root,
                                                        e2, min_count);
    note_launch(2);
    prof_mark(ST_CELLS, s);
    LeafFlag lf{w.cell_id, w.cell_root, w.cell_dense, w.parent, w.core, w.st, p.leaf_size};
    k_flag_scan<<<scan_tiles, SCAN_THREADS, 0, s>>>(w.n, lf, w.leaf_of, w.leaf_first, &w.st->n_leaves,
                                                    &w.st->tile_ctr[MAX_PASSES + 1], w.scan_lb + w.scan_tiles,
                                                    w.dev_status, w.st, 0);
    k_leaves<<<grid_cap(w, w.n, 256), 256, 0, s>>>(w.st, w.keys[0], w.keys[1], w.spts, w.leaf_first, w.cell_id,
                                                   w.cell_dense, w.nodes, w.delta);
    note_launch(2);
    prof_mark(ST_LEAVES, s);
}

void stage_hierarchy(const Work &w, cudaStream_t s)
{
    cudaMemsetAsync(w.slot, 0xff, (size_t)w.n * sizeof(unsigned long long), s);
    k_build<<<grid_cap(w, w.n, 256), 256, 0, s>>>(w.st, w.delta, w.nodes, w.slot, w.right_of);
    k_ropes<<<grid_cap(w, 2 * w.n, 256), 256, 0, s>>>(w.st, w.nodes, w.right_of, w.dev_status);
    note_launch(2);
    prof_mark(ST_BUILD, s);
}

}  // namespace abx
