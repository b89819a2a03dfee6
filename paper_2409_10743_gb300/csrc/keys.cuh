// Morton keys of the input points (the histogram pass computes and writes
// them).
//
// key = segment << shift | Morton code (shift = 3 * the widest per-axis width),
// so segments sort apart and each forms its own subtree.  Each axis is
// quantised with its segment's step (quant_axis: the same rounded expression
// the early exit of the rope walks relies on) and the three cell indices are
// interleaved, x in bit 3k + 2, y in 3k + 1, z in 3k (paper, subsection
// "64-bit Morton codes").
#pragma once

#include "work.cuh"

namespace abx {

// spread3 for values below 2^10, in 32-bit arithmetic: bit k goes to bit 3k.
__device__ __forceinline__ unsigned spread3_10(unsigned v)
{
    unsigned x = v & 0x3ffu;
    x = (x | x << 16) & 0x030000ffu;
    x = (x | x << 8) & 0x0300f00fu;
    x = (x | x << 4) & 0x030c30c3u;
    x = (x | x << 2) & 0x09249249u;
    return x;
}

template <bool SEG>
struct KeyGen {
    const SegState *seg;
    const int *off;
    int nseg, shift;
    float lx, ly, lz, is, qmax;  // segment 0's grid (the single-segment case)

    __device__ KeyGen(const State *st, const SegState *sg, const int *o)
        : seg(sg), off(o), nseg(st->nseg), shift(3 * st->max_bits)
    {
        lx = sg[0].lo[0];
        ly = sg[0].lo[1];
        lz = sg[0].lo[2];
        is = sg[0].inv_step;
        qmax = (float)((1u << sg[0].bits) - 1u);
    }

    // Key of input point i at (x, y, z) (read by the caller); `bad` is set if
    // a coordinate is not finite.  K = 32-bit keys: at most 10 bits per axis,
    // interleaved in 32-bit arithmetic (the same bits as spread3's).
    template <typename K>
    __device__ __forceinline__ unsigned long long key_of(int64_t i, float x, float y, float z, bool &bad) const
    {
        float x0 = lx, y0 = ly, z0 = lz, s = is, qm = qmax;
        unsigned long long top = 0;
        if (SEG) {
            const int sg = seg_of_input(off, nseg, i);
            const SegState &g = seg[sg];
            x0 = g.lo[0];
            y0 = g.lo[1];
            z0 = g.lo[2];
            s = g.inv_step;
            qm = (float)((1u << g.bits) - 1u);
            top = (unsigned long long)sg << shift;
        }
        bad |= !(isfinite(x) && isfinite(y) && isfinite(z));
        const unsigned qx = quant_axis(x, x0, s, qm);
        const unsigned qy = quant_axis(y, y0, s, qm);
        const unsigned qz = quant_axis(z, z0, s, qm);
        if (sizeof(K) == 4)
            return top | ((spread3_10(qx) << 2) | (spread3_10(qy) << 1) | spread3_10(qz));
        return top | (spread3(qx) << 2) | (spread3(qy) << 1) | spread3(qz);
    }
};

// Width of the key in bits, and the shift that leaves its top RADIX_BITS
// bits: the bucket digit.
__device__ __forceinline__ int key_bits(const State *st) { return st->seg_bits + 3 * st->max_bits; }
__device__ __forceinline__ int bucket_shift(const State *st)
{
    const int kb = key_bits(st);
    return kb > RADIX_BITS ? kb - RADIX_BITS : 0;
}

}  // namespace abx
