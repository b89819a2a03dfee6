// Single-pass stream compaction of flagged positions (decoupled look-back).
#pragma once

#include "work.cuh"

namespace abx {

// ---- single-pass flag scan (decoupled look-back) --------------------------------
// ids[k] = number of flagged positions <= k, minus one; first[id] = k for each
// flagged k; first[total] = n; *total_out = total.

// Flag functors give one position's flag; FlagItems turns that into the
// SCAN_ITEMS flags of a thread (functors may instead compute them together).
template <class F>
struct FlagItems : F {
    __device__ unsigned flags(int64_t base, int64_t n) const
    {
        unsigned m = 0;
#pragma unroll
        for (int j = 0; j < SCAN_ITEMS; j++)
            if (base + j < n && (*this)(base + j))
                m |= 1u << j;
        return m;
    }
};

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
    const unsigned flags = f.flags(base, n);  // bit j = flag of item base + j
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
            lb_store(lb, LB_FLAG_PRE | total);
        } else {
            lb_store(lb + tile, LB_FLAG_AGG | total);
            excl = lookback<16>(lb, tile, 1, 0, dev_status);
            lb_store(lb + tile, LB_FLAG_PRE | (excl + total));
        }
        s_excl = excl;
    }
    __syncthreads();
    unsigned long long run = s_excl + wpre + x - c;  // flags before this thread's first item
    if (base + SCAN_ITEMS <= n && (reinterpret_cast<uintptr_t>(ids + base) & 15) == 0) {
        // a whole run of items: the ids leave as SCAN_ITEMS / 4 vector stores
        // (a thread's items are consecutive, so scalar stores would touch a
        // different sector per lane for every item)
        int v[SCAN_ITEMS];
#pragma unroll
        for (int j = 0; j < SCAN_ITEMS; j++) {
            if (flags & (1u << j)) {
                first[run] = (int)(base + j);
                run++;
            }
            v[j] = (int)run - 1;
        }
        int4 *dst = reinterpret_cast<int4 *>(ids + base);
#pragma unroll
        for (int q = 0; q < SCAN_ITEMS / 4; q++)
            dst[q] = make_int4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
        if (base + SCAN_ITEMS == n) {
            first[run] = (int)n;
            *total_out = (int)run;
        }
        return;
    }
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

}  // namespace abx
