// Segments, scene bounds and the Morton quantisation step.
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
    g.margin = -1;
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
        // Cells two neighbours can be apart on one axis.  The test d2 <= e2 bounds
        // each rounded square fl(d_a^2) <= d2 by e2, so |x - y| <= sqrt(e2) (1 + 2^-22)
        // while e2 is a normal number and |x - y| < 2^-62 when it is not (eps_eff
        // below).  In cells that is eps_eff * inv_step, plus the rounding of
        // (x - lo) * inv_step wherever a cell is not clamped (under 2^(bits-22)
        // cells; 2^(bits-20) is used), and the floor adds less than one cell, so
        // the difference of two cells is at most the ceiling of the sum.
        {
            const double eps_eff = fmax(sqrt((double)g.e2), 0x1p-62) * (1.0 + 0x1p-20);
            const double mc = ceil(eps_eff * (double)inv_step + ldexp(1.0, bits - 20));
            g.margin = (isfinite(mc) && mc < (double)(1 << 22)) ? (int)mc : -1;
        }
        g.dense_ok = dense_ok;
        atomicMax(&st->max_bits, bits);
        if (dense_ok)
            atomicOr(&st->dense_ok, 1);
        if (k == 0)
            st->bits = bits;
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

}  // namespace abx
