// Scene bounds, Morton codes, onesweep LSD radix sort and the sorted gather.
//
// Paper, subsection "64-bit Morton codes": points are ordered along a Z-curve
// before the hierarchy is built; 64-bit codes avoid the massive duplication
// that 32-bit codes (1024 bins per axis) showed on clustered data.  Here each
// axis gets up to 21 bits (63-bit keys).  The quantisation step is tied to
// eps: step = h / 2^sub with h the dense-cell side (about eps/sqrt(3), section
// "FDBSCAN-DenseBox"), so the key's top bits are the dense cell and one sort
// serves both the hierarchy and the cell grid, and the key has only as many
// bits as the extent needs (fewer radix passes).  When the extent spans more
// than 2^(21-sub) cells the step falls back to extent / (2^21 - 1).
// Labels never depend on these choices: they only shape the tree.
#include <algorithm>

#include "work.cuh"

namespace abx {

using u32 = unsigned;
// Below this size the 32-bit key kernels are not launched (their launch costs
// more than the lighter passes save).
constexpr int64_t KEY32_MIN_POINTS = 1 << 16;

// ---- segments and bounds -----------------------------------------------------------

__device__ __forceinline__ void seg_reset(SegState &g, float eps, int minpts)
{
    for (int k = 0; k < 3; k++) {
        g.lo_enc[k] = float_to_ordered(__int_as_float(0x7f800000));          // +inf
        g.hi_enc[k] = float_to_ordered(__int_as_float((int)0xff800000));     // -inf
        g.lo[k] = 0.0f;
    }
    g.inv_step = 0.0f;
    g.e2 = __fmul_rn(eps, eps);
    g.minpts = minpts;
    g.bits = 0;
    g.dense_ok = 0;
    g.root = SENTINEL;
    g.pad = 0;
}

// A single clustering call: one segment covering all n points.
__global__ void k_init_single(State *st, SegState *seg, int *off, int64_t n, float eps, int minpts, int allow32)
{
    if (threadIdx.x == 0) {
        seg_reset(seg[0], eps, minpts);
        off[0] = 0;
        off[1] = (int)n;
        st->nseg = 1;
        st->seg_bits = 0;
        st->allow32 = allow32;
    }
}

// A batch: segment k gets eps[k], minpts[k] (device copies of the host arrays).
__global__ void k_init_batch(State *st, SegState *seg, int nseg, const float *eps, const int *minpts, int seg_bits,
                             int allow32)
{
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < nseg; k += gridDim.x * blockDim.x)
        seg_reset(seg[k], eps[k], minpts[k]);
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        st->nseg = nseg;
        st->seg_bits = seg_bits;
        st->allow32 = allow32;
    }
}

struct MinMax {
    float mn0, mn1, mn2, mx0, mx1, mx2;
    bool bad;
    __device__ void init()
    {
        mn0 = mn1 = mn2 = __int_as_float(0x7f800000);
        mx0 = mx1 = mx2 = __int_as_float((int)0xff800000);
        bad = false;
    }
    __device__ __forceinline__ void upd(int axis, float v)
    {
        bad |= !isfinite(v);
        if (axis == 0) { mn0 = fminf(mn0, v); mx0 = fmaxf(mx0, v); }
        else if (axis == 1) { mn1 = fminf(mn1, v); mx1 = fmaxf(mx1, v); }
        else { mn2 = fminf(mn2, v); mx2 = fmaxf(mx2, v); }
    }
    __device__ __forceinline__ void warp_reduce()
    {
        for (int o = 16; o > 0; o >>= 1) {
            mn0 = fminf(mn0, __shfl_xor_sync(~0u, mn0, o));
            mn1 = fminf(mn1, __shfl_xor_sync(~0u, mn1, o));
            mn2 = fminf(mn2, __shfl_xor_sync(~0u, mn2, o));
            mx0 = fmaxf(mx0, __shfl_xor_sync(~0u, mx0, o));
            mx1 = fmaxf(mx1, __shfl_xor_sync(~0u, mx1, o));
            mx2 = fmaxf(mx2, __shfl_xor_sync(~0u, mx2, o));
        }
    }
    __device__ __forceinline__ void publish(SegState &g) const
    {
        atomicMin(&g.lo_enc[0], float_to_ordered(mn0));
        atomicMin(&g.lo_enc[1], float_to_ordered(mn1));
        atomicMin(&g.lo_enc[2], float_to_ordered(mn2));
        atomicMax(&g.hi_enc[0], float_to_ordered(mx0));
        atomicMax(&g.hi_enc[1], float_to_ordered(mx1));
        atomicMax(&g.hi_enc[2], float_to_ordered(mx2));
    }
};

// One segment: float4 loads over the flat coordinate array, block reduction,
// one atomic per value per block.
__global__ void __launch_bounds__(256) k_bounds(const float *__restrict__ pts, int64_t n, int aligned,
                                                SegState *seg, unsigned *dev_status)
{
    MinMax m;
    m.init();
    const int64_t total = 3 * n;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    int64_t done = 0;
    if (aligned) {
        const float4 *p4 = reinterpret_cast<const float4 *>(pts);
        const int64_t nv = total / 4;
        for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < nv; v += stride) {
            float4 q = __ldg(p4 + v);
            int a = (int)((4 * v) % 3);  // axis of q.x; q.w is on the same axis
            m.upd(a, q.x);
            m.upd(a == 2 ? 0 : a + 1, q.y);
            m.upd(a == 0 ? 2 : a - 1, q.z);
            m.upd(a, q.w);
        }
        done = nv * 4;
    }
    for (int64_t e = done + (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += stride)
        m.upd((int)(e % 3), __ldg(pts + e));

    m.warp_reduce();
    unsigned anybad = __any_sync(~0u, m.bad);
    __shared__ float sm[8][6];
    __shared__ int sbad;
    if (threadIdx.x == 0)
        sbad = 0;
    __syncthreads();
    int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0) {
        sm[w][0] = m.mn0; sm[w][1] = m.mn1; sm[w][2] = m.mn2;
        sm[w][3] = m.mx0; sm[w][4] = m.mx1; sm[w][5] = m.mx2;
        if (anybad)
            sbad = 1;
    }
    __syncthreads();
    if (threadIdx.x < 6) {
        int k = threadIdx.x;
        float v = sm[0][k];
        for (int i = 1; i < (int)(blockDim.x >> 5); i++)
            v = k < 3 ? fminf(v, sm[i][k]) : fmaxf(v, sm[i][k]);
        if (k < 3)
            atomicMin(&seg[0].lo_enc[k], float_to_ordered(v));
        else
            atomicMax(&seg[0].hi_enc[k - 3], float_to_ordered(v));
    }
    if (threadIdx.x == 0 && sbad)
        atomicOr(dev_status, DEV_NONFINITE);
}

// Large single segments: the bounds only place the grid (the Morton kernel
// clamps points outside them and checks every coordinate for finiteness), so
// a strided sample of the points is enough.
__global__ void __launch_bounds__(256) k_bounds_sample(const float *__restrict__ pts, int64_t n, int stride,
                                                       SegState *seg)
{
    MinMax m;
    m.init();
    const int64_t ns = (n + stride - 1) / stride;
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < ns; k += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = k * stride;
        m.upd(0, __ldg(pts + 3 * i));
        m.upd(1, __ldg(pts + 3 * i + 1));
        m.upd(2, __ldg(pts + 3 * i + 2));
    }
    // non-finite samples are ignored here (the Morton kernel flags them)
    m.warp_reduce();
    if ((threadIdx.x & 31) == 0 && m.mn0 <= m.mx0)
        m.publish(seg[0]);
}

// Many segments: one point per lane; a warp whose points share a segment
// reduces first and publishes once, otherwise every lane publishes.
__global__ void __launch_bounds__(256) k_bounds_seg(const float *__restrict__ pts, int64_t n, SegState *seg,
                                                    const int *__restrict__ off, int nseg, unsigned *dev_status)
{
    const int lane = threadIdx.x & 31;
    const int64_t wstride = (int64_t)gridDim.x * blockDim.x;
    bool bad = false;
    for (int64_t base = (int64_t)blockIdx.x * blockDim.x + (threadIdx.x & ~31); base < n; base += wstride) {
        const int64_t i = base + lane;
        const bool valid = i < n;
        MinMax m;
        m.init();
        int s = -1;
        if (valid) {
            s = seg_of_input(off, nseg, i);
            m.upd(0, __ldg(pts + 3 * i));
            m.upd(1, __ldg(pts + 3 * i + 1));
            m.upd(2, __ldg(pts + 3 * i + 2));
            bad |= m.bad;
        }
        const int s0 = __shfl_sync(~0u, s, 0);
        if (__all_sync(~0u, s == s0 || !valid) && s0 >= 0) {
            m.warp_reduce();
            if (lane == 0)
                m.publish(seg[s0]);
        } else if (valid) {
            m.publish(seg[s]);
        }
    }
    if (__any_sync(~0u, bad) && lane == 0)
        atomicOr(dev_status, DEV_NONFINITE);
}

// One thread per segment: choose the quantisation.  With dense cells on, the
// step is the dense-cell side h (slightly below eps/sqrt(3), so a cell's
// diagonal is at most eps) divided by 2^sub, as long as the extent spans few
// enough cells for the per-axis width cap; otherwise extent / (2^cap - 1) and
// no dense cells.  With dense cells off the grid only has to resolve the
// points: about log2(cbrt(n)) + 1 bits per axis (some 8 cells per point), which
// keeps keys short (fewer, lighter radix passes); the tree is as tight.
__global__ void k_quant(State *st, SegState *seg, const int *__restrict__ off, int nseg, int dense_on, int sub_bits)
{
    const int cap = min(21, (64 - st->seg_bits) / 3);
    if (blockIdx.x == 0 && threadIdx.x == 0)
        st->sub = sub_bits;
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < nseg; k += gridDim.x * blockDim.x) {
        SegState &g = seg[k];
        float lo[3], ext = 0.0f;
        for (int a = 0; a < 3; a++) {
            lo[a] = ordered_to_float(g.lo_enc[a]);
            float hi = ordered_to_float(g.hi_enc[a]);
            float e = hi - lo[a];
            if (!(e >= 0.0f) || !isfinite(lo[a]) || !isfinite(hi))
                e = 0.0f;  // empty segment or non-finite input (flagged): any key will do
            if (!isfinite(e))
                e = 3.0e38f;
            ext = fmaxf(ext, e);
            g.lo[a] = isfinite(lo[a]) ? lo[a] : 0.0f;
        }
        const float eps = sqrtf(g.e2);
        const float h = eps * 0.57735026f * 0.999f;
        int bits = cap, dense_ok = 0;
        float inv_step = 0.0f;
        if (!dense_on) {
            const int64_t ns = (int64_t)off[k + 1] - off[k];
            int b = 1;
            while (b < cap && (1ll << (3 * b)) < 8 * ns)
                b++;
            bits = b;
            const float is = ext > 0.0f ? (float)((1 << b) - 1) / ext : 0.0f;
            inv_step = isfinite(is) ? is : 0.0f;
            if (inv_step == 0.0f)
                inv_step = 1e-30f;  // one cell: every key equal
        } else if (h > 1e-30f && isfinite(h) && sub_bits < cap) {
            const float ratio = ext / h;
            if (ratio < (float)((1 << (cap - sub_bits)) - 2)) {
                int bc = 1;
                while ((float)(1 << bc) < ratio + 1.0f)
                    bc++;
                bits = bc + sub_bits;
                inv_step = (float)(1 << sub_bits) / h;
                dense_ok = dense_on;
            }
        }
        if (inv_step == 0.0f) {
            bits = cap;
            float is = ext > 0.0f ? (float)((1 << cap) - 1) / ext : 0.0f;
            inv_step = isfinite(is) ? is : 0.0f;
        }
        if (inv_step == 1e-30f)
            inv_step = 0.0f;
        g.inv_step = inv_step;
        g.bits = bits;
        g.dense_ok = dense_ok;
        atomicMax(&st->max_bits, bits);
        if (dense_ok)
            atomicOr(&st->dense_ok, 1);
        if (k == 0)
            st->bits = bits;
    }
}

// ---- Morton keys + the upfront digit histograms ---------------------------------
// key = segment << shift | Morton code (shift = 3 * the widest per-axis width),
// so segments sort apart and each forms its own subtree.

// Both key widths are launched; the one that does not match the call's key
// width (decided here, on the device) returns at once.
template <bool SEG, typename K>
__global__ void __launch_bounds__(256) k_morton(const float *__restrict__ pts, int64_t n, State *st,
                                                const SegState *__restrict__ seg, const int *__restrict__ off,
                                                K *__restrict__ keys, unsigned *dev_status)
{
    const int nseg = st->nseg;
    const int shift = 3 * st->max_bits;
    const int kbits = st->seg_bits + shift;
    const bool key32 = st->allow32 && kbits <= 32;
    if (key32 != (sizeof(K) == 4))
        return;
    bool bad = false;
    __shared__ unsigned sh[MAX_PASSES * RADIX];
    for (int i = threadIdx.x; i < MAX_PASSES * RADIX; i += blockDim.x)
        sh[i] = 0;
    const int np = (kbits + RADIX_BITS - 1) / RADIX_BITS;
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        st->shift = shift;
        st->n_passes = np;
        st->key32 = key32;
    }
    float lx = seg[0].lo[0], ly = seg[0].lo[1], lz = seg[0].lo[2], is = seg[0].inv_step;
    float qmax = (float)((1u << seg[0].bits) - 1u);
    __syncthreads();
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        unsigned long long top = 0;
        if (SEG) {
            const int s = seg_of_input(off, nseg, i);
            const SegState &g = seg[s];
            lx = g.lo[0]; ly = g.lo[1]; lz = g.lo[2]; is = g.inv_step;
            qmax = (float)((1u << g.bits) - 1u);
            top = (unsigned long long)s << shift;
        }
        float x = __ldg(pts + 3 * i), y = __ldg(pts + 3 * i + 1), z = __ldg(pts + 3 * i + 2);
        bad |= !(isfinite(x) && isfinite(y) && isfinite(z));
        float tx = (x - lx) * is, ty = (y - ly) * is, tz = (z - lz) * is;
        unsigned qx = tx < qmax ? (unsigned)fmaxf(tx, 0.0f) : (unsigned)qmax;
        unsigned qy = ty < qmax ? (unsigned)fmaxf(ty, 0.0f) : (unsigned)qmax;
        unsigned qz = tz < qmax ? (unsigned)fmaxf(tz, 0.0f) : (unsigned)qmax;
        unsigned long long key = top | (spread3(qx) << 2) | (spread3(qy) << 1) | spread3(qz);
        keys[i] = (K)key;
        for (int p = 0; p < np; p++)
            atomicAdd(&sh[p * RADIX + (unsigned)((key >> (RADIX_BITS * p)) & (RADIX - 1))], 1u);
    }
    if (bad)
        atomicOr(dev_status, DEV_NONFINITE);
    __syncthreads();
    for (int i = threadIdx.x; i < np * RADIX; i += blockDim.x)
        if (sh[i])
            atomicAdd(&st->hist[0][0] + i, sh[i]);
}

// One block of RADIX threads: drop passes whose digit is the same for every
// key (a stable pass over a constant digit changes nothing), turn histograms
// into exclusive offsets and number the remaining passes.
__global__ void k_sort_plan(State *st, int64_t n)
{
    __shared__ int active[MAX_PASSES];
    const int d = threadIdx.x;
    const int np = st->n_passes;
    if (d < MAX_PASSES)
        active[d] = d < np;
    __syncthreads();
    for (int p = 0; p < np; p++)
        if ((int64_t)st->hist[p][d] == n)
            active[p] = 0;
    __syncthreads();
    if (d < np) {
        unsigned run = 0;
        for (int k = 0; k < RADIX; k++) {
            unsigned c = st->hist[d][k];
            st->hist[d][k] = run;
            run += c;
        }
    }
    if (d == 0) {
        int ord = 0;
        for (int p = 0; p < MAX_PASSES; p++)
            st->pass_ord[p] = active[p] ? ord++ : -1;
        st->n_active = ord;
    }
}

// ---- onesweep pass ------------------------------------------------------------------
// One tile of sort_tile<K>() keys per block (tile ids handed out in launch order, so
// a tile only ever waits on tiles that are already running).  Each warp ranks
// its keys by digit with __match_any_sync, the tile publishes its digit counts,
// looks back across earlier tiles for its global prefix (decoupled look-back,
// bounded spins) and scatters through shared memory so that keys of one digit
// leave as contiguous runs.

constexpr unsigned long long LB_AGG = LB_FLAG_AGG;
constexpr unsigned long long LB_PRE = LB_FLAG_PRE;

constexpr int SORT_WARPS = SORT_THREADS / 32;
static int g_sort_blocks_per_sm = SORT_MIN_BLOCKS;  // set per process by kernels_init_device
template <typename K>
constexpr size_t onesweep_smem()
{
    return sort_tile<K>() * (sizeof(K) + sizeof(unsigned)) + SORT_WARPS * RADIX * 4 + 2 * RADIX * 4;
}

template <typename K>
__global__ void __launch_bounds__(SORT_THREADS, SORT_MIN_BLOCKS) k_onesweep(int pass, K *k0, K *k1, unsigned *v0, unsigned *v1,
                                                              int64_t n, State *st, unsigned long long *lb_all,
                                                              unsigned *dev_status)
{
    if (st->key32 != (sizeof(K) == 4))
        return;
    const int ord = st->pass_ord[pass];
    if (ord < 0)
        return;
    const K *ksrc = (ord & 1) ? k1 : k0;
    K *kdst = (ord & 1) ? k0 : k1;
    const unsigned *vsrc = (ord & 1) ? v1 : v0;
    unsigned *vdst = (ord & 1) ? v0 : v1;
    const bool first = ord == 0;
    const int shift = pass * RADIX_BITS;
    constexpr int SORT_ITEMS = sort_items<K>();
    constexpr int SORT_TILE = sort_tile<K>();
    const int ntiles = div_up(n, SORT_TILE);
    const unsigned nn = (unsigned)n;
    unsigned long long *lb = lb_all + (size_t)pass * ntiles * RADIX;

    extern __shared__ __align__(16) unsigned char smem[];
    K *s_keys = reinterpret_cast<K *>(smem);
    unsigned *s_vals = reinterpret_cast<unsigned *>(s_keys + SORT_TILE);
    unsigned *s_whist = s_vals + SORT_TILE;      // [warps][RADIX]
    unsigned *s_loc = s_whist + SORT_WARPS * RADIX;  // tile-local digit offsets
    unsigned *s_glob = s_loc + RADIX;            // destination base per digit
    __shared__ int s_tile;
    __shared__ unsigned s_wsum[RADIX / 32];

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    // persistent: each block takes tiles in ticket order until none are left
    // (a tile only waits on tiles whose blocks are already working on them)
    while (true) {
        if (tid == 0)
            s_tile = (int)atomicAdd(&st->tile_ctr[pass], 1u);
        for (int i = tid; i < SORT_WARPS * RADIX; i += SORT_THREADS)
            s_whist[i] = 0;
        __syncthreads();
        const int tile = s_tile;
        if (tile >= ntiles)
            break;
        // positions fit 32 bits: n < 2^31 and a tile ends at most SORT_TILE - 1 past n
        const unsigned base = (unsigned)tile * SORT_TILE + (unsigned)warp * 32 * SORT_ITEMS + lane;

        K key[SORT_ITEMS];
        unsigned val[SORT_ITEMS];
        unsigned rank[SORT_ITEMS];
    #pragma unroll
        for (int k = 0; k < SORT_ITEMS; k++) {
            const unsigned pos = base + k * 32;
            key[k] = pos < nn ? ksrc[pos] : (K)~(K)0;  // pads rank last in digit RADIX-1 and land at >= n
        }
    #pragma unroll
        for (int k = 0; k < SORT_ITEMS; k++) {
            const unsigned pos = base + k * 32;
            val[k] = pos < nn ? (first ? pos : vsrc[pos]) : 0u;
        }
        // stable rank within the warp: lanes with equal digit, in lane order, after
        // the earlier items of this warp.  The lanes sharing a digit are found
        // with one ballot per digit bit (cheaper than a general match).
        unsigned *wh = s_whist + warp * RADIX;
        const unsigned lt_mask = (1u << lane) - 1u;
    #pragma unroll
        for (int k = 0; k < SORT_ITEMS; k++) {
            const unsigned d = (unsigned)(key[k] >> shift) & (RADIX - 1);
            unsigned peers = ~0u;
    #pragma unroll
            for (int b = 0; b < RADIX_BITS; b++) {
                const bool bit = (d >> b) & 1u;
                const unsigned bal = __ballot_sync(~0u, bit);
                peers &= bit ? bal : ~bal;
            }
            const int leader = __ffs(peers) - 1;
            unsigned prev = 0;
            if (lane == leader)
                prev = atomicAdd(wh + d, (unsigned)__popc(peers));
            prev = __shfl_sync(~0u, prev, leader);
            rank[k] = prev + __popc(peers & lt_mask);
        }
        __syncthreads();

        // thread d < RADIX: per-warp exclusive offsets and the tile count of digit d
        unsigned cnt = 0;
        unsigned long long excl = 0;
        if (tid < RADIX) {
            const int d = tid;
    #pragma unroll
            for (int w = 0; w < SORT_WARPS; w++) {
                unsigned c = s_whist[w * RADIX + d];
                s_whist[w * RADIX + d] = cnt;
                cnt += c;
            }
            // publish, then look back
            if (tile == 0) {
                lb_store(lb + d, LB_PRE | cnt);
            } else {
                lb_store(lb + (size_t)tile * RADIX + d, LB_AGG | cnt);
                excl = lookback<8>(lb, tile, RADIX, tid, dev_status);
                lb_store(lb + (size_t)tile * RADIX + d, LB_PRE | (excl + cnt));
            }
        }
        // exclusive scan of cnt over digits (tile-local offsets)
        unsigned x = cnt;
    #pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            unsigned y = __shfl_up_sync(~0u, x, o);
            if (lane >= o)
                x += y;
        }
        if (tid < RADIX && lane == 31)
            s_wsum[warp] = x;
        __syncthreads();
        if (tid < RADIX) {
            unsigned wpre = 0;
            for (int w = 0; w < warp; w++)
                wpre += s_wsum[w];
            const unsigned loc = wpre + x - cnt;
            s_loc[tid] = loc;
            s_glob[tid] = st->hist[pass][tid] + (unsigned)excl - loc;
        }
        __syncthreads();

    #pragma unroll
        for (int k = 0; k < SORT_ITEMS; k++) {
            const unsigned dd = (unsigned)(key[k] >> shift) & (RADIX - 1);
            const unsigned lp = s_loc[dd] + s_whist[warp * RADIX + dd] + rank[k];
            s_keys[lp] = key[k];
            s_vals[lp] = val[k];
        }
        __syncthreads();
    #pragma unroll 4
        for (int i = tid; i < SORT_TILE; i += SORT_THREADS) {
            const K kk = s_keys[i];
            const unsigned dd = (unsigned)(kk >> shift) & (RADIX - 1);
            const unsigned dest = s_glob[dd] + (unsigned)i;
            if (dest < nn) {
                kdst[dest] = kk;
                vdst[dest] = s_vals[i];
            }
        }
        __syncthreads();  // the next tile reuses the shared buffers
    }
}

// ---- gather -----------------------------------------------------------------------
// spts[k] = (x, y, z, original index) of the k-th point in key order; resets
// the union-find, the core flags (all core when the segment's minPts is 1)
// and the border minima.

template <bool SEG>
__global__ void __launch_bounds__(256) k_gather(const float *__restrict__ pts, int64_t n, const State *st,
                                                const SegState *__restrict__ seg, const void *k0,
                                                const void *k1, const unsigned *v0, const unsigned *v1,
                                                float4 *spts, int *parent, unsigned char *core, int *bmin,
                                                unsigned *dev_status)
{
    const int na = st->n_active;
    const unsigned *perm = na == 0 ? nullptr : ((na & 1) ? v1 : v0);
    const int shift = st->shift;
    unsigned char c0 = seg[0].minpts <= 1 ? 1 : 0;
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x) {
        unsigned o = perm ? perm[k] : (unsigned)k;
        if ((int64_t)o >= n) {  // never for a correct sort
            atomicOr(dev_status, DEV_INTERNAL);
            o = (unsigned)k;
        }
        float x = __ldg(pts + 3 * (int64_t)o), y = __ldg(pts + 3 * (int64_t)o + 1), z = __ldg(pts + 3 * (int64_t)o + 2);
        spts[k] = make_float4(x, y, z, __int_as_float((int)o));
        parent[k] = (int)k;
        if (SEG)
            c0 = seg[seg_of_key(sorted_key(st, k0, k1, k), shift)].minpts <= 1 ? 1 : 0;
        core[k] = c0;
        if (bmin)
            bmin[k] = 0x7fffffff;
    }
}

// ---- launchers -------------------------------------------------------------------------

static int grid_for(const Work &w, int64_t n, int block, int per_sm = 8)
{
    int64_t g = div_up(n, block);
    int64_t cap = (int64_t)w.n_sms * per_sm;
    if (g > cap)
        g = cap;
    return (int)(g < 1 ? 1 : g);
}

void stage_segments_single(const Work &w, float eps, int minpts, cudaStream_t s)
{
    cudaMemsetAsync(w.st, 0, sizeof(State), s);
    k_init_single<<<1, 32, 0, s>>>(w.st, w.seg, w.seg_off, w.n, eps, minpts, w.n >= KEY32_MIN_POINTS);
    note_launch();
}

void stage_segments_batch(const Work &w, const float *eps_dev, const int *minpts_dev, int seg_bits, cudaStream_t s)
{
    cudaMemsetAsync(w.st, 0, sizeof(State), s);
    k_init_batch<<<div_up(w.nseg, 128), 128, 0, s>>>(w.st, w.seg, w.nseg, eps_dev, minpts_dev, seg_bits,
                                                      w.n >= KEY32_MIN_POINTS);
    note_launch();
}

void stage_bounds_quant(const Work &w, const float *points, const Params &p, cudaStream_t s)
{
    if (w.nseg == 1) {
        if (w.n >= (1 << 22)) {
            k_bounds_sample<<<grid_for(w, w.n / 32, 256), 256, 0, s>>>(points, w.n, 32, w.seg);
        } else {
            int aligned = (reinterpret_cast<uintptr_t>(points) & 15) == 0;
            k_bounds<<<grid_for(w, (3 * w.n + 3) / 4, 256), 256, 0, s>>>(points, w.n, aligned, w.seg,
                                                                          w.dev_status);
        }
    } else {
        k_bounds_seg<<<grid_for(w, w.n, 256), 256, 0, s>>>(points, w.n, w.seg, w.seg_off, w.nseg, w.dev_status);
    }
    k_quant<<<div_up(w.nseg, 128), 128, 0, s>>>(w.st, w.seg, w.seg_off, w.nseg, p.dense, p.sub_bits);
    note_launch(2);
    prof_mark(ST_BOUNDS, s);
}

void stage_morton_sort(const Work &w, const float *points, cudaStream_t s)
{
    using u64 = unsigned long long;
    u32 *k32[2] = {reinterpret_cast<u32 *>(w.keys[0]), reinterpret_cast<u32 *>(w.keys[1])};
    const bool try32 = w.n >= KEY32_MIN_POINTS;  // must match the allow32 given to the init kernel
    const int g = grid_for(w, w.n, 256);
    if (w.nseg == 1) {
        k_morton<false, u64><<<g, 256, 0, s>>>(points, w.n, w.st, w.seg, w.seg_off, w.keys[0], w.dev_status);
        if (try32)
            k_morton<false, u32><<<g, 256, 0, s>>>(points, w.n, w.st, w.seg, w.seg_off, k32[0], w.dev_status);
    } else {
        k_morton<true, u64><<<g, 256, 0, s>>>(points, w.n, w.st, w.seg, w.seg_off, w.keys[0], w.dev_status);
        if (try32)
            k_morton<true, u32><<<g, 256, 0, s>>>(points, w.n, w.st, w.seg, w.seg_off, k32[0], w.dev_status);
    }
    note_launch(try32 ? 2 : 1);
    prof_mark(ST_MORTON, s);
    k_sort_plan<<<1, RADIX, 0, s>>>(w.st, w.n);
    note_launch();
    cudaMemsetAsync(w.sort_lb, 0, (size_t)MAX_PASSES * w.sort_tiles * RADIX * sizeof(unsigned long long), s);
    const int tiles = (int)std::min<int64_t>(div_up(w.n, SORT_TILE_MIN), (int64_t)g_sort_blocks_per_sm * w.n_sms);
    for (int pass = 0; pass < MAX_PASSES; pass++)
        k_onesweep<u64><<<tiles, SORT_THREADS, onesweep_smem<u64>(), s>>>(pass, w.keys[0], w.keys[1], w.vals[0],
                                                                          w.vals[1], w.n, w.st, w.sort_lb,
                                                                          w.dev_status);
    note_launch(MAX_PASSES);
    if (try32) {
        for (int pass = 0; pass < 4; pass++)
            k_onesweep<u32><<<tiles, SORT_THREADS, onesweep_smem<u32>(), s>>>(pass, k32[0], k32[1], w.vals[0],
                                                                              w.vals[1], w.n, w.st, w.sort_lb,
                                                                              w.dev_status);
        note_launch(4);
    }
    prof_mark(ST_SORT, s);
}

void stage_gather(const Work &w, const float *points, cudaStream_t s)
{
    int *bmin = w.any_dbscan ? w.bmin : nullptr;
    if (w.nseg == 1)
        k_gather<false><<<grid_for(w, w.n, 256, 16), 256, 0, s>>>(points, w.n, w.st, w.seg, w.keys[0], w.keys[1],
                                                                  w.vals[0], w.vals[1], w.spts, w.parent, w.core,
                                                                  bmin, w.dev_status);
    else
        k_gather<true><<<grid_for(w, w.n, 256, 16), 256, 0, s>>>(points, w.n, w.st, w.seg, w.keys[0], w.keys[1],
                                                                 w.vals[0], w.vals[1], w.spts, w.parent, w.core,
                                                                 bmin, w.dev_status);
    note_launch();
    prof_mark(ST_GATHER, s);
}

void kernels_init_device()
{
    int b32 = 0, b64 = 0;
    cudaFuncSetAttribute(k_onesweep<unsigned long long>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)onesweep_smem<unsigned long long>());
    cudaFuncSetAttribute(k_onesweep<u32>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)onesweep_smem<u32>());
    // persistent sort grid: as many blocks as fit on an SM (both key widths
    // share one grid size)
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b64, k_onesweep<unsigned long long>, SORT_THREADS,
                                                      onesweep_smem<unsigned long long>()) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b32, k_onesweep<u32>, SORT_THREADS,
                                                      onesweep_smem<u32>()) != cudaSuccess) {
        cudaGetLastError();
        b32 = b64 = SORT_MIN_BLOCKS;
    }
    g_sort_blocks_per_sm = std::max(1, std::min(b32, b64));
}

}  // namespace abx
