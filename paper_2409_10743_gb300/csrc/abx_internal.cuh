// Internal definitions shared by the abx kernels (device + launch helpers).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "../../include/abx.h"

namespace abx {

// ---- device status word bits (OR-ed by kernels, read by abx_device_status) --
enum : unsigned { DEV_NONFINITE = 1u, DEV_TIMEOUT = 2u, DEV_INTERNAL = 4u };

// Bounded spin: iterations before a wait gives up, records DEV_TIMEOUT and
// moves on (the call's output is then unspecified, but the GPU never hangs).
constexpr int SPIN_LIMIT = 1 << 22;

constexpr int SENTINEL = -1;        // rope of the right-most path (paper, fig. f:karras_ropes)
constexpr int RADIX_BITS = 8;
constexpr int RADIX = 1 << RADIX_BITS;
constexpr int MAX_PASSES = 8;       // 64-bit keys, 8 bits per pass
constexpr int SORT_THREADS = 256;
constexpr int SORT_MIN_BLOCKS = 2;  // blocks per SM the sort pass is compiled for
// keys per thread of a sort pass: as many as the registers of 2 blocks per SM
// hold without spilling (key, value and rank per item)
template <typename K>
constexpr int sort_items() { return sizeof(K) == 4 ? 32 : 16; }
template <typename K>
constexpr int sort_tile() { return SORT_THREADS * sort_items<K>(); }
constexpr int SORT_TILE_MIN = SORT_THREADS * 16;  // the smaller tile sizes the look-back buffer
// Below this size the 32-bit key kernels are not launched (their launch costs
// more than the lighter passes save).
constexpr int64_t KEY32_MIN_POINTS = 1 << 16;
// Bucketing pass: above this size the input points no longer fit in L2, and
// gathering them in key order straight from the input is a random 12-byte
// read per point over the whole array.  The points are first moved, with
// their keys, into buckets by the key's top 8 bits (one stable counting pass
// that reads the input in order); the gather after the sort then reads
// within one or two buckets at a time, which L2 holds.
constexpr int64_t BUCKET_MIN_POINTS = 1 << 23;
constexpr int BUCKET_ITEMS = 8;                 // keys per thread of its tiles
constexpr int BUCKET_TILE = SORT_THREADS * BUCKET_ITEMS;
constexpr int BUCKET_ROW = MAX_PASSES;          // its histogram row; its look-back words follow the passes'
constexpr int BUCKET_TICKETS = MAX_PASSES + 2;  // its tile counter (tile_ctr index)
constexpr int SCAN_THREADS = 256;
constexpr int SCAN_ITEMS = 16;
constexpr int SCAN_TILE = SCAN_THREADS * SCAN_ITEMS;
constexpr unsigned DENSE_BIT = 0x80000000u;

// Per-segment device state: one entry per independent point set of a call
// (a single clustering call has one segment; a batch has many).
struct SegState {
    int lo_enc[3], hi_enc[3];   // ordered-int encoded bounds
    float lo[3];                // segment minimum (its grid origin)
    float inv_step;             // Morton quantisation scale
    float e2;                   // fl(eps * eps)
    int minpts;
    int bits;                   // Morton bits per axis used by this segment
    int dense_ok;               // dense cells usable (cell grid = Morton prefix)
    int root;                   // root of the segment's subtree
    int margin;                 // cells a neighbour's quantised coordinate can differ by (-1: unbounded)
};

// Per-call device state (lives in the call's workspace).
struct State {
    int nseg;                   // independent point sets in this call
    int seg_bits;               // bits of the segment id at the top of a key
    int max_bits;               // widest per-axis Morton width over segments
    int shift;                  // key = segment << shift | Morton code
    int sub;                    // Morton bits per axis below the dense-cell side
    int dense_ok;               // some segment uses dense cells
    int n_passes;               // candidate radix passes
    int n_active;               // radix passes run (the rest are constant digits)
    int pass_ord[MAX_PASSES];   // order of pass p among the active ones, -1 = skipped
    unsigned tile_ctr[MAX_PASSES + 4];
    // digit histograms of the radix passes, then exclusive offsets; row
    // BUCKET_ROW: the same for the bucket digit (the key's top 8 bits)
    unsigned hist[MAX_PASSES + 1][RADIX];
    int n_cells;                // dense cells found
    int n_leaves;
    int root;                   // root of the whole hierarchy
    int frontier_count;         // nodes finishing the build in its global phase
    int bits;                   // Morton bits per axis of segment 0 (diagnostics)
    int key32;                  // keys fit 32 bits and are sorted as 32-bit words
    int allow32;                // the call launched the 32-bit key kernels
    int pad[1];
};

// Sorted key k, from whichever buffer the last radix pass wrote, whatever the
// key width of the call.
__device__ __forceinline__ unsigned long long sorted_key(const State *st, const void *k0, const void *k1, int64_t k)
{
    const void *buf = (st->n_active & 1) ? k1 : k0;
    return st->key32 ? (unsigned long long)static_cast<const unsigned *>(buf)[k]
                     : static_cast<const unsigned long long *>(buf)[k];
}

// ---- decoupled look-back ------------------------------------------------------
// Status words: bits 62-63 = 0 (not published), 1 (the tile's own count), 2
// (inclusive prefix through that tile); bits 0-61 = the count.  A tile sums
// its predecessors' words backwards until an inclusive prefix.  The words of
// a window of predecessors are loaded at once (one memory round trip per
// window instead of per tile); a word not yet published is re-read with a
// bounded spin.
constexpr unsigned long long LB_FLAG_AGG = 1ull << 62;
constexpr unsigned long long LB_FLAG_PRE = 2ull << 62;
constexpr unsigned long long LB_COUNT = (1ull << 62) - 1;

__device__ __forceinline__ unsigned long long lb_load(const unsigned long long *p)
{
    unsigned long long v;
    asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void lb_store(unsigned long long *p, unsigned long long v)
{
    asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

// Sum of the counts of tiles [0, tile) in column `slot` of a look-back array
// with `stride` words per tile, LOOKBACK_WINDOW words per round trip.
template <int LOOKBACK_WINDOW>
__device__ __forceinline__ unsigned long long lookback(const unsigned long long *lb, int tile, int stride, int slot,
                                                       unsigned *dev_status, int spin_limit = SPIN_LIMIT)
{
    unsigned long long excl = 0;
    int t = tile - 1;
    int spins = 0;
    while (t >= 0) {
        unsigned long long v[LOOKBACK_WINDOW];
#pragma unroll
        for (int k = 0; k < LOOKBACK_WINDOW; k++)
            v[k] = t - k >= 0 ? lb_load(lb + (size_t)(t - k) * stride + slot) : LB_FLAG_PRE;
        int k = 0;
#pragma unroll
        for (; k < LOOKBACK_WINDOW; k++) {
            const unsigned long long f = v[k] >> 62;
            if (f == 0)
                break;  // tile t - k has not published yet
            excl += v[k] & LB_COUNT;
            if (f == 2)
                return excl;
        }
        t -= k;
        if (k < LOOKBACK_WINDOW) {
            if (++spins > spin_limit) {
                atomicOr(dev_status, DEV_TIMEOUT);
                return excl;
            }
            if (spins > 8)
                __nanosleep(32);
        }
    }
    return excl;
}

// Segment of input index i: the largest s with off[s] <= i (empty segments
// are skipped because their successor has the same offset).
__device__ __forceinline__ int seg_of_input(const int *__restrict__ off, int nseg, int64_t i)
{
    int lo = 0, hi = nseg - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if ((int64_t)__ldg(off + mid) <= i)
            lo = mid;
        else
            hi = mid - 1;
    }
    return lo;
}

// Split level between sorted keys a (position t) and b (position t + 1):
// 33 + the highest bit in which they differ, or, for equal keys, the level of
// the (key, position) tie-break, 32 - clz(t ^ (t + 1)) (below every key bit).
// The hierarchy merges across the lower level first.
__device__ __forceinline__ unsigned char split_level(unsigned long long a, unsigned long long b, int t)
{
    unsigned long long x = a ^ b;
    if (x)
        return (unsigned char)(32 + (64 - __clzll((long long)x)));
    return (unsigned char)(32 - __clz(t ^ (t + 1)));
}

// Segment of a sorted point, read from the top bits of its key.
__device__ __forceinline__ int seg_of_key(unsigned long long key, int shift)
{
    return shift >= 64 ? 0 : (int)(key >> shift);
}

// ---- FP32 exact predicate ---------------------------------------------------
// d2 = fl(fl(fl(dx*dx) + fl(dy*dy)) + fl(dz*dz)), every operation rounded to
// nearest even on its own (the _rn intrinsics are never contracted into FMA).
__device__ __forceinline__ float dist2_rn(float ax, float ay, float az, float bx, float by, float bz)
{
    float dx = __fsub_rn(ax, bx);
    float dy = __fsub_rn(ay, by);
    float dz = __fsub_rn(az, bz);
    float s = __fadd_rn(__fmul_rn(dx, dx), __fmul_rn(dy, dy));
    return __fadd_rn(s, __fmul_rn(dz, dz));
}

// Rounded squared distance from p to the box [lo, hi], same operation order.
// Rounding is monotone and fl(-a) = -fl(a), so for every point q in the box
// this value is <= dist2_rn(p, q): pruning a box when it exceeds e2 never
// drops a neighbour.
__device__ __forceinline__ float box_dist2_rn(float px, float py, float pz, float4 lo, float4 hi)
{
    float dx = fmaxf(0.0f, fmaxf(__fsub_rn(lo.x, px), __fsub_rn(px, hi.x)));
    float dy = fmaxf(0.0f, fmaxf(__fsub_rn(lo.y, py), __fsub_rn(py, hi.y)));
    float dz = fmaxf(0.0f, fmaxf(__fsub_rn(lo.z, pz), __fsub_rn(pz, hi.z)));
    float s = __fadd_rn(__fmul_rn(dx, dx), __fmul_rn(dy, dy));
    return __fadd_rn(s, __fmul_rn(dz, dz));
}

// Rounded distance between two boxes, per axis the gap max(0, lo_b - hi_a,
// lo_a - hi_b).  For p in box a and q in box b, q_x - p_x >= lo_b - hi_a
// exactly, and rounding is monotone, so |fl(p_x - q_x)| >= fl(gap); squares
// and sums keep the order: the value is <= dist2_rn(p, q) for every such
// pair, and pruning at > e2 never drops a neighbour pair.
__device__ __forceinline__ float box_box_dist2_rn(float4 alo, float4 ahi, float4 blo, float4 bhi)
{
    float dx = fmaxf(0.0f, fmaxf(__fsub_rn(blo.x, ahi.x), __fsub_rn(alo.x, bhi.x)));
    float dy = fmaxf(0.0f, fmaxf(__fsub_rn(blo.y, ahi.y), __fsub_rn(alo.y, bhi.y)));
    float dz = fmaxf(0.0f, fmaxf(__fsub_rn(blo.z, ahi.z), __fsub_rn(alo.z, bhi.z)));
    float s = __fadd_rn(__fmul_rn(dx, dx), __fmul_rn(dy, dy));
    return __fadd_rn(s, __fmul_rn(dz, dz));
}

// ---- node records -------------------------------------------------------------
// One hierarchy record is 32 bytes (lo.xyz + left child or first point, hi.xyz
// + rope), fetched with a single 256-bit load: one load instruction per node
// visit instead of two.  Records are read-only in every traversal kernel.
__device__ __forceinline__ void ld_node(const float4 *nodes, int i, float4 &lo, float4 &hi)
{
    asm("ld.global.nc.v8.f32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
        : "=f"(lo.x), "=f"(lo.y), "=f"(lo.z), "=f"(lo.w), "=f"(hi.x), "=f"(hi.y), "=f"(hi.z), "=f"(hi.w)
        : "l"(nodes + 2 * (size_t)i));
}

// ---- early exit of rope walks (Morton regions) -----------------------------------
// A coordinate's grid cell, exactly as the Morton kernel quantises it.
__device__ __forceinline__ unsigned quant_axis(float v, float lo, float inv_step, float qmax)
{
    const float t = __fmul_rn(__fsub_rn(v, lo), inv_step);
    return t < qmax ? (unsigned)fmaxf(t, 0.0f) : (unsigned)qmax;
}

// The quantisation is monotone, and two points that pass the neighbour test
// are at most g.margin cells apart on every axis (the margin bounds eps in
// cells plus the rounding of the quantisation; it is set with the step).  So
// every neighbour of a point of the box [lo, hi] has its cell in
// [q(lo) - margin, q(hi) + margin] per axis.  Returned: the highest bit of the
// interleaved code at which two cells of that grown box can differ (-1: one
// cell; 255: no bound, the walk never stops early).  Bit 3k + 2 - a holds bit
// k of axis a.
__device__ __forceinline__ int reach_level(float lx, float ly, float lz, float hx, float hy, float hz,
                                           const SegState &g)
{
    const int m = g.margin;
    if (m < 0)
        return 255;
    const unsigned qm = (1u << g.bits) - 1u;
    const float qmax = (float)qm;
    const float lo3[3] = {lx, ly, lz}, hi3[3] = {hx, hy, hz};
    int H = -1;
#pragma unroll
    for (int a = 0; a < 3; a++) {
        const unsigned ql = quant_axis(lo3[a], g.lo[a], g.inv_step, qmax);
        const unsigned qh = quant_axis(hi3[a], g.lo[a], g.inv_step, qmax);
        const unsigned gl = ql > (unsigned)m ? ql - (unsigned)m : 0u;
        const unsigned gh = qh + (unsigned)m < qm ? qh + (unsigned)m : qm;
        const unsigned x = gl ^ gh;
        if (x)
            H = max(H, 3 * (31 - __clz(x)) + 2 - a);
    }
    return H;
}

// The split level of the leaf boundary a node's rope crosses travels in the
// lowest 8 bits of the node's hi.x, so a rope walk has it in the record it
// already loaded.  hi.x is rounded UP to the nearest float with those low
// bits: the box grows by less than 256 ulps on that side, which keeps every
// pruning test conservative (a looser box never drops a neighbour).  Near the
// top of the float range the result may be +inf or a NaN; box_dist2_rn and
// box_box_dist2_rn then ignore that side (fmaxf returns its other operand),
// which is conservative too.  Written after the boxes are merged bottom-up.
__device__ __forceinline__ float with_level(float v, unsigned lv)
{
    const unsigned b = __float_as_uint(v);
    if (!(b >> 31)) {  // +0 or positive: larger bit patterns are larger values
        unsigned c = (b & ~0xffu) | lv;
        if (c < b)
            c += 256u;
        return __uint_as_float(c);
    }
    const unsigned m = b & 0x7fffffffu;  // negative: smaller magnitudes are larger values
    unsigned c = (m & ~0xffu) | lv;
    if (c > m) {
        if (m < 256u)
            return __uint_as_float(lv);  // +0 or a positive subnormal, above v
        c -= 256u;
    }
    return __uint_as_float(c | 0x80000000u);
}
__device__ __forceinline__ int level_of(float4 hi) { return (int)(__float_as_uint(hi.x) & 0xffu); }

// Crossing the leaf boundary whose split level is lv (split_level encoding:
// lv > 32 is a key split at bit lv - 33; 255 = the end of the walk) while the
// highest level crossed so far since the walk's own leaf is M: the subtree
// being left is the left child of that boundary's node, it holds the walk's
// own leaf iff lv > M, and then it is exactly the set of keys that share the
// code's bits >= lv - 33.  If the grown box of the query fits in that region
// (lv - 33 > H), no point after it can be a neighbour: stop.
__device__ __forceinline__ bool region_exit(int lv, int M, int H)
{
    return lv != 255 && lv > M && lv > 32 && lv - 33 > H;
}

// ---- ordered float <-> int for atomic min/max ---------------------------------
__device__ __forceinline__ int float_to_ordered(float f)
{
    int i = __float_as_int(f);
    return i >= 0 ? i : i ^ 0x7fffffff;
}
__device__ __forceinline__ float ordered_to_float(int i)
{
    return __int_as_float(i >= 0 ? i : i ^ 0x7fffffff);
}

// ---- relaxed L2 loads for data other threads write during a kernel ----------
__device__ __forceinline__ int ld_cg(const int *p) { return __ldcg(p); }
__device__ __forceinline__ float4 ld_cg4(const float4 *p) { return __ldcg(p); }

// ---- lock-free union-find over sorted positions --------------------------------
// A set's root is its member with the smallest original index (priority =
// original index, kept in float4.w of the sorted points), so after all unions
// the root of a cluster of core points is K(C), its smallest core index.
// Hooking is a CAS on the root's own parent word: parent pointers only ever
// move to members of smaller priority, so stale reads can delay but never
// break a find, and every chain ends at a root.
__device__ __forceinline__ int orig_of(const float4 *pts, int i)
{
    return __float_as_int(__ldg(&pts[i].w));
}

__device__ __forceinline__ int uf_find(int *parent, int x)
{
    while (true) {
        int p = ld_cg(parent + x);
        if (p == x)
            return x;
        int gp = ld_cg(parent + p);
        if (gp == p)
            return p;
        parent[x] = gp;  // path halving (any ancestor is a valid parent)
        x = gp;
    }
}

// Merge the sets of a and b; returns the root that the merged set had when
// the call ended (a member of it ever after: sets only grow).
__device__ __forceinline__ int uf_unite(int *parent, const float4 *pts, int a, int b)
{
    while (true) {
        a = uf_find(parent, a);
        b = uf_find(parent, b);
        if (a == b)
            return a;
        // strict total order (original index, position): chains never cycle
        const int oa = orig_of(pts, a), ob = orig_of(pts, b);
        if (oa > ob || (oa == ob && a > b)) {
            int t = a;
            a = b;
            b = t;
        }
        // hook b (larger priority) under a
        int old = atomicCAS(parent + b, b, a);
        if (old == b)
            return a;
        b = old;
    }
}

// ---- Morton interleave (21 bits per axis -> 63 bits) ------------------------
__device__ __forceinline__ unsigned long long spread3(unsigned v)
{
    unsigned long long x = v & 0x1fffffu;
    x = (x | x << 32) & 0x1f00000000ffffull;
    x = (x | x << 16) & 0x1f0000ff0000ffull;
    x = (x | x << 8) & 0x100f00f00f00f00full;
    x = (x | x << 4) & 0x10c30c30c30c30c3ull;
    x = (x | x << 2) & 0x1249249249249249ull;
    return x;
}

}  // namespace abx
