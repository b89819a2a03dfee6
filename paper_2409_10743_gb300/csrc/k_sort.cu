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
#include "work.cuh"

namespace abx {

// ---- bounds -------------------------------------------------------------------

__global__ void k_init_state(State *st)
{
    if (threadIdx.x < 3) {
        st->lo_enc[threadIdx.x] = float_to_ordered(__int_as_float(0x7f800000));   // +inf
        st->hi_enc[threadIdx.x] = float_to_ordered(__int_as_float((int)0xff800000));  // -inf
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
};

__global__ void __launch_bounds__(256) k_bounds(const float *__restrict__ pts, int64_t n, int aligned,
                                                State *st, unsigned *dev_status)
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

    // block reduction
    for (int o = 16; o > 0; o >>= 1) {
        m.mn0 = fminf(m.mn0, __shfl_xor_sync(~0u, m.mn0, o));
        m.mn1 = fminf(m.mn1, __shfl_xor_sync(~0u, m.mn1, o));
        m.mn2 = fminf(m.mn2, __shfl_xor_sync(~0u, m.mn2, o));
        m.mx0 = fmaxf(m.mx0, __shfl_xor_sync(~0u, m.mx0, o));
        m.mx1 = fmaxf(m.mx1, __shfl_xor_sync(~0u, m.mx1, o));
        m.mx2 = fmaxf(m.mx2, __shfl_xor_sync(~0u, m.mx2, o));
    }
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
            atomicMin(&st->lo_enc[k], float_to_ordered(v));
        else
            atomicMax(&st->hi_enc[k - 3], float_to_ordered(v));
    }
    if (threadIdx.x == 0 && sbad)
        atomicOr(dev_status, DEV_NONFINITE);
}

// One thread: choose the quantisation and the candidate radix passes.
__global__ void k_quant(State *st, float eps, int dense_on, int sub_bits)
{
    float lo[3], ext = 0.0f;
    for (int k = 0; k < 3; k++) {
        lo[k] = ordered_to_float(st->lo_enc[k]);
        float hi = ordered_to_float(st->hi_enc[k]);
        float e = hi - lo[k];
        if (!(e >= 0.0f) || !isfinite(lo[k]) || !isfinite(hi))
            e = 0.0f;  // non-finite input: already flagged; any key will do
        if (!isfinite(e))
            e = 3.0e38f;
        ext = fmaxf(ext, e);
        st->lo[k] = isfinite(lo[k]) ? lo[k] : 0.0f;
    }
    // dense-cell side h slightly below eps/sqrt(3): cell diagonal <= eps
    float h = eps * 0.57735026f * 0.999f;
    int bits = 21, sub = 0, dense_ok = 0;
    float inv_step = 0.0f;
    if (h > 1e-30f && isfinite(h)) {
        float ratio = ext / h;
        if (ratio < (float)((1 << (21 - sub_bits)) - 2)) {
            int bc = 1;
            while ((float)(1 << bc) < ratio + 1.0f)
                bc++;
            sub = sub_bits;
            bits = bc + sub;
            inv_step = (float)(1 << sub) / h;
            dense_ok = dense_on;
        }
    }
    if (inv_step == 0.0f) {
        bits = 21;
        sub = 0;
        float is = ext > 0.0f ? (float)((1 << 21) - 1) / ext : 0.0f;
        inv_step = isfinite(is) ? is : 0.0f;
    }
    st->inv_step = inv_step;
    st->bits = bits;
    st->sub = sub;
    st->dense_ok = dense_ok;
    int np = (3 * bits + RADIX_BITS - 1) / RADIX_BITS;
    st->n_passes = np;
}

// ---- Morton keys + the upfront digit histograms ---------------------------------

__global__ void __launch_bounds__(256) k_morton(const float *__restrict__ pts, int64_t n, State *st,
                                                unsigned long long *__restrict__ keys)
{
    __shared__ unsigned sh[MAX_PASSES * RADIX];
    for (int i = threadIdx.x; i < MAX_PASSES * RADIX; i += blockDim.x)
        sh[i] = 0;
    const float lx = st->lo[0], ly = st->lo[1], lz = st->lo[2];
    const float is = st->inv_step;
    const int np = st->n_passes;
    const float qmax = (float)((1u << st->bits) - 1u);
    __syncthreads();
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        float x = __ldg(pts + 3 * i), y = __ldg(pts + 3 * i + 1), z = __ldg(pts + 3 * i + 2);
        float tx = (x - lx) * is, ty = (y - ly) * is, tz = (z - lz) * is;
        unsigned qx = tx < qmax ? (unsigned)fmaxf(tx, 0.0f) : (unsigned)qmax;
        unsigned qy = ty < qmax ? (unsigned)fmaxf(ty, 0.0f) : (unsigned)qmax;
        unsigned qz = tz < qmax ? (unsigned)fmaxf(tz, 0.0f) : (unsigned)qmax;
        unsigned long long key = (spread3(qx) << 2) | (spread3(qy) << 1) | spread3(qz);
        keys[i] = key;
        for (int p = 0; p < np; p++)
            atomicAdd(&sh[p * RADIX + (unsigned)((key >> (RADIX_BITS * p)) & (RADIX - 1))], 1u);
    }
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
        st->pad[0] = ord;  // number of active passes
    }
}

// ---- onesweep pass ------------------------------------------------------------------
// One tile of SORT_TILE keys per block (tile ids handed out in launch order, so
// a tile only ever waits on tiles that are already running).  Each warp ranks
// its keys by digit with __match_any_sync, the tile publishes its digit counts,
// looks back across earlier tiles for its global prefix (decoupled look-back,
// bounded spins) and scatters through shared memory so that keys of one digit
// leave as contiguous runs.

constexpr unsigned long long LB_AGG = 1ull << 62;
constexpr unsigned long long LB_PRE = 2ull << 62;

__device__ __forceinline__ unsigned long long ld_relaxed_u64(const unsigned long long *p)
{
    unsigned long long v;
    asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_relaxed_u64(unsigned long long *p, unsigned long long v)
{
    asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

// Sum the look-back words of tiles [0, tile) for one slot; bounded.
__device__ unsigned long long lookback_sum(const unsigned long long *lb, int tile, int stride, int slot,
                                           unsigned *dev_status)
{
    unsigned long long excl = 0;
    for (int t = tile - 1; t >= 0; t--) {
        unsigned long long v;
        int spins = 0;
        while (true) {
            v = ld_relaxed_u64(lb + (size_t)t * stride + slot);
            if ((v >> 62) != 0)
                break;
            if (++spins > SPIN_LIMIT) {
                atomicOr(dev_status, DEV_TIMEOUT);
                return excl;
            }
            if (spins > 64)
                __nanosleep(64);
        }
        excl += v & ((1ull << 62) - 1);
        if ((v >> 62) == 2)
            break;
    }
    return excl;
}

constexpr int SORT_WARPS = SORT_THREADS / 32;
constexpr size_t ONESWEEP_SMEM =
    SORT_TILE * sizeof(unsigned long long) + SORT_TILE * sizeof(unsigned) + SORT_WARPS * RADIX * 4 + 2 * RADIX * 4;

__global__ void __launch_bounds__(SORT_THREADS, 2) k_onesweep(int pass, unsigned long long *k0, unsigned long long *k1,
                                                              unsigned *v0, unsigned *v1, int64_t n, State *st,
                                                              unsigned long long *lb_all, unsigned *dev_status)
{
    const int ord = st->pass_ord[pass];
    if (ord < 0)
        return;
    const unsigned long long *ksrc = (ord & 1) ? k1 : k0;
    unsigned long long *kdst = (ord & 1) ? k0 : k1;
    const unsigned *vsrc = (ord & 1) ? v1 : v0;
    unsigned *vdst = (ord & 1) ? v0 : v1;
    const bool first = ord == 0;
    const int shift = pass * RADIX_BITS;
    const int ntiles = div_up(n, SORT_TILE);
    unsigned long long *lb = lb_all + (size_t)pass * ntiles * RADIX;

    extern __shared__ __align__(16) unsigned char smem[];
    unsigned long long *s_keys = reinterpret_cast<unsigned long long *>(smem);
    unsigned *s_vals = reinterpret_cast<unsigned *>(s_keys + SORT_TILE);
    unsigned *s_whist = s_vals + SORT_TILE;      // [warps][RADIX]
    unsigned *s_loc = s_whist + SORT_WARPS * RADIX;  // tile-local digit offsets
    unsigned *s_glob = s_loc + RADIX;            // destination base per digit
    __shared__ int s_tile;
    __shared__ unsigned s_wsum[RADIX / 32];

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    if (tid == 0)
        s_tile = (int)atomicAdd(&st->tile_ctr[pass], 1u);
    for (int i = tid; i < SORT_WARPS * RADIX; i += SORT_THREADS)
        s_whist[i] = 0;
    __syncthreads();
    const int tile = s_tile;
    const int64_t base = (int64_t)tile * SORT_TILE + (int64_t)warp * 32 * SORT_ITEMS + lane;

    unsigned long long key[SORT_ITEMS];
    unsigned val[SORT_ITEMS];
    unsigned rank[SORT_ITEMS];
#pragma unroll
    for (int k = 0; k < SORT_ITEMS; k++) {
        const int64_t pos = base + k * 32;
        key[k] = pos < n ? ksrc[pos] : ~0ull;  // pads rank last in digit RADIX-1 and land at >= n
    }
#pragma unroll
    for (int k = 0; k < SORT_ITEMS; k++) {
        const int64_t pos = base + k * 32;
        val[k] = pos < n ? (first ? (unsigned)pos : vsrc[pos]) : 0u;
    }
    // stable rank within the warp: lanes with equal digit, in lane order, after
    // the earlier items of this warp
    unsigned *wh = s_whist + warp * RADIX;
    const unsigned lt_mask = (1u << lane) - 1u;
#pragma unroll
    for (int k = 0; k < SORT_ITEMS; k++) {
        const unsigned d = (unsigned)(key[k] >> shift) & (RADIX - 1);
        const unsigned peers = __match_any_sync(~0u, d);
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
            st_relaxed_u64(lb + d, LB_PRE | cnt);
        } else {
            st_relaxed_u64(lb + (size_t)tile * RADIX + d, LB_AGG | cnt);
            excl = lookback_sum(lb, tile, RADIX, d, dev_status);
            st_relaxed_u64(lb + (size_t)tile * RADIX + d, LB_PRE | (excl + cnt));
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
        const unsigned long long kk = s_keys[i];
        const unsigned dd = (unsigned)(kk >> shift) & (RADIX - 1);
        const unsigned dest = s_glob[dd] + (unsigned)i;
        if ((int64_t)dest < n) {
            kdst[dest] = kk;
            vdst[dest] = s_vals[i];
        }
    }
}

// ---- gather -----------------------------------------------------------------------
// spts[k] = (x, y, z, original index) of the k-th point in key order; resets
// the union-find and the core flags.

__global__ void __launch_bounds__(256) k_gather(const float *__restrict__ pts, int64_t n, const State *st,
                                                const unsigned *v0, const unsigned *v1, float4 *spts,
                                                int *parent, unsigned char *core, int *bmin, int minpts,
                                                unsigned *dev_status)
{
    const int na = st->pad[0];
    const unsigned *perm = na == 0 ? nullptr : ((na & 1) ? v1 : v0);
    const unsigned char c0 = minpts <= 1 ? 1 : 0;
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x) {
        unsigned o = perm ? perm[k] : (unsigned)k;
        if ((int64_t)o >= n) {  // never for a correct sort
            atomicOr(dev_status, DEV_INTERNAL);
            o = (unsigned)k;
        }
        float x = __ldg(pts + 3 * (int64_t)o), y = __ldg(pts + 3 * (int64_t)o + 1), z = __ldg(pts + 3 * (int64_t)o + 2);
        spts[k] = make_float4(x, y, z, __int_as_float((int)o));
        parent[k] = (int)k;
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

void stage_bounds_quant(const Work &w, const float *points, float eps, const Params &p, cudaStream_t s)
{
    cudaMemsetAsync(w.st, 0, sizeof(State), s);
    k_init_state<<<1, 32, 0, s>>>(w.st);
    int aligned = (reinterpret_cast<uintptr_t>(points) & 15) == 0;
    k_bounds<<<grid_for(w, (3 * w.n + 3) / 4, 256), 256, 0, s>>>(points, w.n, aligned, w.st, w.dev_status);
    k_quant<<<1, 1, 0, s>>>(w.st, eps, p.dense, p.sub_bits);
    note_launch(3);
    prof_mark(ST_BOUNDS, s);
}

void stage_morton_sort(const Work &w, const float *points, cudaStream_t s)
{
    k_morton<<<grid_for(w, w.n, 256), 256, 0, s>>>(points, w.n, w.st, w.keys[0]);
    note_launch();
    prof_mark(ST_MORTON, s);
    k_sort_plan<<<1, RADIX, 0, s>>>(w.st, w.n);
    note_launch();
    cudaMemsetAsync(w.sort_lb, 0, (size_t)MAX_PASSES * w.sort_tiles * RADIX * sizeof(unsigned long long), s);
    const int tiles = div_up(w.n, SORT_TILE);
    for (int pass = 0; pass < MAX_PASSES; pass++)
        k_onesweep<<<tiles, SORT_THREADS, ONESWEEP_SMEM, s>>>(pass, w.keys[0], w.keys[1], w.vals[0], w.vals[1],
                                                              w.n, w.st, w.sort_lb, w.dev_status);
    note_launch(MAX_PASSES);
    prof_mark(ST_SORT, s);
}

void stage_gather(const Work &w, const float *points, int minpts, cudaStream_t s)
{
    k_gather<<<grid_for(w, w.n, 256, 16), 256, 0, s>>>(points, w.n, w.st, w.vals[0], w.vals[1], w.spts, w.parent,
                                                        w.core, minpts > 2 ? w.bmin : nullptr, minpts, w.dev_status);
    note_launch();
    prof_mark(ST_GATHER, s);
}

void kernels_init_device()
{
    cudaFuncSetAttribute(k_onesweep, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)ONESWEEP_SMEM);
}

}  // namespace abx
