// Sorting the points along the Z-curve: digit histograms, the bucketing pass,
// the onesweep LSD radix passes and the gather into key order.
//
// Paper, subsection "64-bit Morton codes": the points are ordered by their
// Morton codes before the hierarchy is built (section "ArborX library": a
// bottom-up LBVH over Z-sorted objects; the queries are pre-sorted the same
// way so that neighbouring threads traverse nearby).  The sort is a stable
// LSD radix sort of (key, position) pairs.  Every pass is a "onesweep" pass:
// persistent blocks take tiles in ticket order, rank their keys by digit,
// publish per-tile digit counts and find their global offsets with a
// decoupled look-back over earlier tiles (bounded waits), then scatter through
// shared memory so that each digit's run leaves as one contiguous write.  The
// digit histograms of every pass are counted up front in the Morton pass;
// passes whose digit is the same for all keys are skipped on the device.
//
// For inputs larger than L2 the points are first moved into 256 buckets by the
// key's top 8 bits (k_bucket: the same onesweep scheme, reading the input in
// order and carrying the points); the sort then orders positions in that
// bucketed array, and the gather reads it within one or two buckets at a time
// instead of reading the whole input at random.
#include <algorithm>

#include "keys.cuh"

namespace abx {

using u32 = unsigned;
using u64 = unsigned long long;

// ---- digit histograms (and keys, when there is no bucketing pass) --------------
// Both key widths are launched; the one that does not match the call's key
// width (decided here, on the device) returns at once.

template <bool SEG, typename K>
__global__ void __launch_bounds__(256) k_morton(const float *__restrict__ pts, int64_t n, State *st,
                                                const SegState *__restrict__ seg, const int *__restrict__ off,
                                                K *__restrict__ keys, int write_keys, int bucket,
                                                unsigned *dev_status)
{
    const int kbits = key_bits(st);
    const bool key32 = st->allow32 && kbits <= 32;
    if (key32 != (sizeof(K) == 4))
        return;
    bool bad = false;
    __shared__ unsigned sh[(MAX_PASSES + 1) * RADIX];
    for (int i = threadIdx.x; i < (MAX_PASSES + 1) * RADIX; i += blockDim.x)
        sh[i] = 0;
    const int np = (kbits + RADIX_BITS - 1) / RADIX_BITS;
    const int bshift = bucket_shift(st);
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        st->shift = 3 * st->max_bits;
        st->n_passes = np;
        st->key32 = key32;
    }
    const KeyGen<SEG> kg(st, seg, off);
    __syncthreads();
    auto one = [&](int64_t i, float x, float y, float z) {
        const u64 key = kg.template key_of<K>(i, x, y, z, bad);
        if (write_keys)
            keys[i] = (K)key;
        for (int p = 0; p < np; p++)
            atomicAdd(&sh[p * RADIX + (unsigned)((key >> (RADIX_BITS * p)) & (RADIX - 1))], 1u);
        if (bucket)
            atomicAdd(&sh[BUCKET_ROW * RADIX + (unsigned)((key >> bshift) & (RADIX - 1))], 1u);
    };
    // four consecutive points per thread and step, their 48 bytes loaded
    // before any is used (three 16-byte loads when the input is 16-byte
    // aligned): enough bytes in flight per SM to keep HBM busy
    const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x, nthreads = (int64_t)gridDim.x * blockDim.x;
    const int64_t groups = n / 4;
    const bool vec = (reinterpret_cast<uintptr_t>(pts) & 15) == 0;
    for (int64_t q = tid; q < groups; q += nthreads) {
        float c[12];
        if (vec) {
            const float4 *p4 = reinterpret_cast<const float4 *>(pts) + 3 * q;
            const float4 a = __ldg(p4), b = __ldg(p4 + 1), d = __ldg(p4 + 2);
            c[0] = a.x, c[1] = a.y, c[2] = a.z, c[3] = a.w, c[4] = b.x, c[5] = b.y;
            c[6] = b.z, c[7] = b.w, c[8] = d.x, c[9] = d.y, c[10] = d.z, c[11] = d.w;
        } else {
#pragma unroll
            for (int j = 0; j < 12; j++)
                c[j] = __ldg(pts + 12 * q + j);
        }
#pragma unroll
        for (int j = 0; j < 4; j++)
            one(4 * q + j, c[3 * j], c[3 * j + 1], c[3 * j + 2]);
    }
    for (int64_t i = 4 * groups + tid; i < n; i += nthreads)  // the last n % 4 points
        one(i, __ldg(pts + 3 * i), __ldg(pts + 3 * i + 1), __ldg(pts + 3 * i + 2));
    if (bad)
        atomicOr(dev_status, DEV_NONFINITE);
    __syncthreads();
    for (int i = threadIdx.x; i < (MAX_PASSES + 1) * RADIX; i += blockDim.x)
        if (sh[i])
            atomicAdd(&st->hist[0][0] + i, sh[i]);
}

// One block of RADIX threads: drop passes whose digit is the same for every
// key (a stable pass over a constant digit changes nothing), turn histograms
// (and the bucket histogram) into exclusive offsets and number the remaining
// passes.
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
    if (d < np || d == BUCKET_ROW) {
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

// ---- one tile of a counting pass ---------------------------------------------------
constexpr int SORT_WARPS = SORT_THREADS / 32;
static int g_sort_blocks_per_sm = SORT_MIN_BLOCKS;    // set per process by kernels_init_device
static int g_bucket_blocks_per_sm[2] = {SORT_MIN_BLOCKS, 1};  // 32-bit, 64-bit keys (their tiles differ)

struct TileSmem {
    unsigned *whist;  // [SORT_WARPS][RADIX] per-warp digit counts, then per-warp offsets
    unsigned *loc;    // [RADIX] start of each digit's run in the tile
    unsigned *glob;   // [RADIX] output position of the tile's run of each digit, minus its start in the tile
    unsigned *wsum;   // [RADIX / 32]
};

// Ranks the tile's keys by the digit (key >> shift) & (RADIX - 1), stable in
// item order (warp by warp, item by item, lane by lane), and publishes the
// tile's digit counts in its row of the look-back array `lb`.  After the call
// (it ends with a barrier), item k of this thread goes to tile position
//   sm.loc[d] + sm.whist[warp][d] + rank[k].
// Returns the tile's count of digit d = threadIdx.x (threads below RADIX),
// which tile_place needs.
template <typename K, int ITEMS>
__device__ __forceinline__ unsigned tile_rank(const K (&key)[ITEMS], int shift, unsigned (&rank)[ITEMS],
                                              const TileSmem &sm, unsigned long long *lb, int tile)
{
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    // stable rank within the warp: lanes with equal digit, in lane order, after
    // the earlier items of this warp.  The lanes sharing a digit are found
    // with one ballot per digit bit (cheaper than a general match).
    unsigned *wh = sm.whist + warp * RADIX;
    const unsigned lt_mask = (1u << lane) - 1u;
#pragma unroll
    for (int k = 0; k < ITEMS; k++) {
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

    // thread d < RADIX: per-warp exclusive offsets and the tile count of digit
    // d, published at once (inclusive of the tiles before only for tile 0)
    unsigned cnt = 0;
    if (tid < RADIX) {
        const int d = tid;
#pragma unroll
        for (int w = 0; w < SORT_WARPS; w++) {
            unsigned c = sm.whist[w * RADIX + d];
            sm.whist[w * RADIX + d] = cnt;
            cnt += c;
        }
        lb_store(lb + (size_t)tile * RADIX + d, (tile == 0 ? LB_FLAG_PRE : LB_FLAG_AGG) | cnt);
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
        sm.wsum[warp] = x;
    __syncthreads();
    if (tid < RADIX) {
        unsigned wpre = 0;
        for (int w = 0; w < warp; w++)
            wpre += sm.wsum[w];
        sm.loc[tid] = wpre + x - cnt;
    }
    __syncthreads();
    return cnt;
}

// Where the tile's run of each digit goes: sm.glob[d] + (tile position) is
// the output position.  Adds up the counts of the tiles before this one
// (decoupled look-back) and publishes the inclusive counts.  Called once the
// tile's items are in shared memory, so that the wait overlaps that work and
// the items' registers are free; ends with a barrier.
__device__ __forceinline__ void tile_place(unsigned cnt, const TileSmem &sm, unsigned long long *lb, int tile,
                                           const unsigned *digit_base, unsigned *dev_status)
{
    const int tid = threadIdx.x;
    if (tid < RADIX) {
        unsigned long long excl = 0;
        if (tile > 0) {
            excl = lookback<8>(lb, tile, RADIX, tid, dev_status);
            lb_store(lb + (size_t)tile * RADIX + tid, LB_FLAG_PRE | (excl + cnt));
        }
        sm.glob[tid] = digit_base[tid] + (unsigned)excl - sm.loc[tid];
    }
    __syncthreads();
}

template <typename K>
constexpr size_t tile_smem_extra()
{
    return (size_t)SORT_WARPS * RADIX * 4 + 2 * RADIX * 4;
}
template <typename K>
constexpr size_t onesweep_smem()
{
    return sort_tile<K>() * (sizeof(K) + sizeof(unsigned)) + tile_smem_extra<K>();
}
// The bucketing pass keeps each item's point (x, y, z, original index) in
// shared memory beside its key, so the scatter reads nothing from global
// memory; its tiles are half the radix passes' so two blocks fit an SM.
template <typename K>
constexpr size_t bucket_smem()
{
    return BUCKET_TILE * (sizeof(float4) + sizeof(K) + sizeof(unsigned short)) + tile_smem_extra<K>();
}

// ---- bucketing pass ----------------------------------------------------------------
// Stable by the bucket digit, in input order: the keys (recomputed from the
// points) go to kdst and the points, with their original index, to bpts.

template <bool SEG, typename K>
__global__ void __launch_bounds__(SORT_THREADS, 4)
    k_bucket(const float *__restrict__ pts, int64_t n, State *st, const K *__restrict__ ksrc, K *kdst, float4 *bpts,
             unsigned long long *lb, unsigned *dev_status)
{
    if (st->key32 != (sizeof(K) == 4))
        return;
    constexpr int ITEMS = BUCKET_ITEMS;
    constexpr int TILE = BUCKET_TILE;
    const int ntiles = div_up(n, TILE);
    const unsigned nn = (unsigned)n;
    const int shift = bucket_shift(st);

    extern __shared__ __align__(16) unsigned char smem[];
    float4 *s_pts = reinterpret_cast<float4 *>(smem);       // the tile's points, in load order
    K *s_keys = reinterpret_cast<K *>(s_pts + TILE);        // keys, in output order
    unsigned short *s_src = reinterpret_cast<unsigned short *>(s_keys + TILE);  // their load positions
    TileSmem sm;
    sm.whist = reinterpret_cast<unsigned *>(s_src + TILE);
    sm.loc = sm.whist + SORT_WARPS * RADIX;
    sm.glob = sm.loc + RADIX;
    __shared__ unsigned s_wsum[RADIX / 32];
    sm.wsum = s_wsum;
    __shared__ int s_tile;

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    while (true) {
        if (tid == 0)
            s_tile = (int)atomicAdd(&st->tile_ctr[BUCKET_TICKETS], 1u);
        for (int i = tid; i < SORT_WARPS * RADIX; i += SORT_THREADS)
            sm.whist[i] = 0;
        __syncthreads();
        const int tile = s_tile;
        if (tile >= ntiles)
            break;
        const unsigned local = (unsigned)warp * 32 * ITEMS + lane;
        const unsigned base = (unsigned)tile * TILE + local;
        K key[ITEMS];
        unsigned rank[ITEMS];
#pragma unroll
        for (int k = 0; k < ITEMS; k++) {
            const unsigned pos = base + k * 32;
            float4 pt = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
            key[k] = (K)~(K)0;  // pads rank last and land at >= n
            if (pos < nn) {
                key[k] = ksrc[pos];
                pt = make_float4(__ldg(pts + 3 * (size_t)pos), __ldg(pts + 3 * (size_t)pos + 1),
                                 __ldg(pts + 3 * (size_t)pos + 2), __int_as_float((int)pos));
            }
            s_pts[local + k * 32] = pt;
        }
        const unsigned cnt = tile_rank<K, ITEMS>(key, shift, rank, sm, lb, tile);
#pragma unroll
        for (int k = 0; k < ITEMS; k++) {
            const unsigned dd = (unsigned)(key[k] >> shift) & (RADIX - 1);
            const unsigned lp = sm.loc[dd] + sm.whist[warp * RADIX + dd] + rank[k];
            s_keys[lp] = key[k];
            s_src[lp] = (unsigned short)(local + k * 32);
        }
        tile_place(cnt, sm, lb, tile, st->hist[BUCKET_ROW], dev_status);
#pragma unroll 4
        for (int i = tid; i < TILE; i += SORT_THREADS) {
            const K kk = s_keys[i];
            const unsigned dd = (unsigned)(kk >> shift) & (RADIX - 1);
            const unsigned dest = sm.glob[dd] + (unsigned)i;
            if (dest < nn) {
                kdst[dest] = kk;
                bpts[dest] = s_pts[s_src[i]];
            }
        }
        __syncthreads();  // the next tile reuses the shared buffers
    }
}

// ---- onesweep LSD pass -----------------------------------------------------------------

template <typename K>
__global__ void __launch_bounds__(SORT_THREADS, SORT_MIN_BLOCKS)
    k_onesweep(int pass, K *k0, K *k1, unsigned *v0, unsigned *v1, int64_t n, State *st, unsigned long long *lb_all,
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
    constexpr int ITEMS = sort_items<K>();
    constexpr int TILE = sort_tile<K>();
    const int ntiles = div_up(n, TILE);
    const unsigned nn = (unsigned)n;
    unsigned long long *lb = lb_all + (size_t)pass * ntiles * RADIX;

    extern __shared__ __align__(16) unsigned char smem[];
    K *s_keys = reinterpret_cast<K *>(smem);
    unsigned *s_vals = reinterpret_cast<unsigned *>(s_keys + TILE);
    TileSmem sm;
    sm.whist = s_vals + TILE;
    sm.loc = sm.whist + SORT_WARPS * RADIX;
    sm.glob = sm.loc + RADIX;
    __shared__ unsigned s_wsum[RADIX / 32];
    sm.wsum = s_wsum;
    __shared__ int s_tile;

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    // persistent: each block takes tiles in ticket order until none are left
    // (a tile only waits on tiles whose blocks are already working on them)
    while (true) {
        if (tid == 0)
            s_tile = (int)atomicAdd(&st->tile_ctr[pass], 1u);
        for (int i = tid; i < SORT_WARPS * RADIX; i += SORT_THREADS)
            sm.whist[i] = 0;
        __syncthreads();
        const int tile = s_tile;
        if (tile >= ntiles)
            break;
        // positions fit 32 bits: n < 2^31 and a tile ends at most TILE - 1 past n
        const unsigned base = (unsigned)tile * TILE + (unsigned)warp * 32 * ITEMS + lane;
        K key[ITEMS];
        unsigned rank[ITEMS];
#pragma unroll
        for (int k = 0; k < ITEMS; k++) {
            const unsigned pos = base + k * 32;
            key[k] = pos < nn ? ksrc[pos] : (K)~(K)0;  // pads rank last in digit RADIX-1 and land at >= n
        }
        const unsigned cnt = tile_rank<K, ITEMS>(key, shift, rank, sm, lb, tile);
        // the values are read only now, straight into their places: they
        // hold no registers through the ranking
#pragma unroll
        for (int k = 0; k < ITEMS; k++) {
            const unsigned pos = base + k * 32;
            const unsigned dd = (unsigned)(key[k] >> shift) & (RADIX - 1);
            const unsigned lp = sm.loc[dd] + sm.whist[warp * RADIX + dd] + rank[k];
            s_keys[lp] = key[k];
            s_vals[lp] = pos < nn ? (first ? pos : vsrc[pos]) : 0u;
        }
        tile_place(cnt, sm, lb, tile, st->hist[pass], dev_status);
#pragma unroll 4
        for (int i = tid; i < TILE; i += SORT_THREADS) {
            const K kk = s_keys[i];
            const unsigned dd = (unsigned)(kk >> shift) & (RADIX - 1);
            const unsigned dest = sm.glob[dd] + (unsigned)i;
            if (dest < nn) {
                kdst[dest] = kk;
                vdst[dest] = s_vals[i];
            }
        }
        __syncthreads();  // the next tile reuses the shared buffers
    }
}

// ---- gather ---------------------------------------------------------------------------
// spts[k] = (x, y, z, original index) of the k-th point in key order, from the
// bucketed copy (BUCKETED) or the input; pdelta[k] = the split level between
// sorted points k and k + 1 (for the leaves and the hierarchy).  Also resets
// the union-find, the core flags (all core when the segment's minPts is 1)
// and the border minima.

template <bool SEG, bool BUCKETED>
__global__ void __launch_bounds__(256) k_gather(const float *__restrict__ pts, const float4 *__restrict__ bpts,
                                                int64_t n, const State *st, const SegState *__restrict__ seg,
                                                const void *k0, const void *k1, const unsigned *v0,
                                                const unsigned *v1, float4 *spts, unsigned char *pdelta,
                                                int *parent, unsigned char *core, int *bmin, unsigned *dev_status)
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
        if (BUCKETED)
            spts[k] = __ldg(bpts + o);
        else
            spts[k] = make_float4(__ldg(pts + 3 * (int64_t)o), __ldg(pts + 3 * (int64_t)o + 1),
                                  __ldg(pts + 3 * (int64_t)o + 2), __int_as_float((int)o));
        const u64 key = sorted_key(st, k0, k1, k);
        if (k + 1 < n)
            pdelta[k] = split_level(key, sorted_key(st, k0, k1, k + 1), (int)k);
        parent[k] = (int)k;
        if (SEG)
            c0 = seg[seg_of_key(key, shift)].minpts <= 1 ? 1 : 0;
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

template <bool SEG>
static void launch_sort(const Work &w, const float *points, cudaStream_t s)
{
    u32 *k32[2] = {reinterpret_cast<u32 *>(w.keys[0]), reinterpret_cast<u32 *>(w.keys[1])};
    const bool try32 = w.n >= KEY32_MIN_POINTS;  // must match the allow32 given to the init kernel
    const bool bucket = w.n >= BUCKET_MIN_POINTS;
    const int g = grid_for(w, w.n, 256);
    // with a bucketing pass the keys go to the second buffer (input order)
    // and the bucketing pass writes them, in bucket order, to the first
    const int kin = bucket ? 1 : 0;
    k_morton<SEG, u64><<<g, 256, 0, s>>>(points, w.n, w.st, w.seg, w.seg_off, w.keys[kin], 1, bucket, w.dev_status);
    if (try32)
        k_morton<SEG, u32><<<g, 256, 0, s>>>(points, w.n, w.st, w.seg, w.seg_off, k32[kin], 1, bucket,
                                             w.dev_status);
    note_launch(try32 ? 2 : 1);
    prof_mark(ST_MORTON, s);
    k_sort_plan<<<1, RADIX, 0, s>>>(w.st, w.n);
    note_launch();
    cudaMemsetAsync(w.sort_lb, 0,
                    ((size_t)MAX_PASSES * w.sort_tiles + w.bucket_tiles) * RADIX * sizeof(unsigned long long), s);
    if (bucket) {
        // the bucket pass's look-back words lie past every radix pass's rows
        unsigned long long *lb = w.sort_lb + (size_t)MAX_PASSES * w.sort_tiles * RADIX;
        const int64_t ntiles = div_up(w.n, BUCKET_TILE);
        const int t32 = (int)std::min<int64_t>(ntiles, (int64_t)g_bucket_blocks_per_sm[0] * w.n_sms);
        const int t64 = (int)std::min<int64_t>(ntiles, (int64_t)g_bucket_blocks_per_sm[1] * w.n_sms);
        k_bucket<SEG, u64><<<t64, SORT_THREADS, bucket_smem<u64>(), s>>>(points, w.n, w.st, w.keys[1], w.keys[0],
                                                                          w.bpts, lb, w.dev_status);
        k_bucket<SEG, u32><<<t32, SORT_THREADS, bucket_smem<u32>(), s>>>(points, w.n, w.st, k32[1], k32[0], w.bpts,
                                                                          lb, w.dev_status);
        note_launch(2);
    }
    prof_mark(ST_BUCKET, s);  // (with the sort plan and the look-back reset)
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

void stage_morton_sort(const Work &w, const float *points, cudaStream_t s)
{
    if (w.nseg == 1)
        launch_sort<false>(w, points, s);
    else
        launch_sort<true>(w, points, s);
}

void stage_gather(const Work &w, const float *points, cudaStream_t s)
{
    int *bmin = w.any_dbscan ? w.bmin : nullptr;
    const bool bucket = w.n >= BUCKET_MIN_POINTS;
    const int g = grid_for(w, w.n, 256, 16);
#define ABX_GATHER(SEG, BK)                                                                                       \
    k_gather<SEG, BK><<<g, 256, 0, s>>>(points, w.bpts, w.n, w.st, w.seg, w.keys[0], w.keys[1], w.vals[0],         \
                                        w.vals[1], w.spts, w.pdelta, w.parent, w.core, bmin, w.dev_status)
    if (w.nseg == 1) {
        if (bucket)
            ABX_GATHER(false, true);
        else
            ABX_GATHER(false, false);
    } else {
        if (bucket)
            ABX_GATHER(true, true);
        else
            ABX_GATHER(true, false);
    }
#undef ABX_GATHER
    note_launch();
    prof_mark(ST_GATHER, s);
}

void kernels_init_device()
{
    int b32 = 0, b64 = 0, c32 = 0, c64 = 0;
    cudaFuncSetAttribute(k_onesweep<u64>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)onesweep_smem<u64>());
    cudaFuncSetAttribute(k_onesweep<u32>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)onesweep_smem<u32>());
    cudaFuncSetAttribute(k_bucket<false, u64>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bucket_smem<u64>());
    cudaFuncSetAttribute(k_bucket<false, u32>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bucket_smem<u32>());
    cudaFuncSetAttribute(k_bucket<true, u64>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bucket_smem<u64>());
    cudaFuncSetAttribute(k_bucket<true, u32>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bucket_smem<u32>());
    // persistent grids: as many blocks as fit on an SM (both key widths share
    // one grid size)
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b64, k_onesweep<u64>, SORT_THREADS, onesweep_smem<u64>()) !=
            cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b32, k_onesweep<u32>, SORT_THREADS, onesweep_smem<u32>()) !=
            cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&c64, k_bucket<true, u64>, SORT_THREADS, bucket_smem<u64>()) !=
            cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&c32, k_bucket<true, u32>, SORT_THREADS, bucket_smem<u32>()) !=
            cudaSuccess) {
        cudaGetLastError();
        b32 = b64 = c32 = c64 = SORT_MIN_BLOCKS;
    }
    g_sort_blocks_per_sm = std::max(1, std::min(b32, b64));
    g_bucket_blocks_per_sm[0] = std::max(1, c32);
    g_bucket_blocks_per_sm[1] = std::max(1, c64);
}

}  // namespace abx
