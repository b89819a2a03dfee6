/*
 * Oracle: plain CPU DBSCAN (and its minPts = 2 friends-of-friends case).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the independent checker of the GPU
 * library.  Only the test suite, the smoke check and the benchmark's CPU
 * baseline load it; the GPU library never calls it and shares no code with it.
 *
 * What it computes is the plain definition of DBSCAN (paper, section
 * "DBSCAN algorithm", the definitions of the eps-neighbourhood, core, border
 * and noise points), not the paper's fast method: FDBSCAN and
 * FDBSCAN-DenseBox (sections "FDBSCAN", "FDBSCAN-DenseBox") reach exactly this
 * result, only faster.
 *
 *   N_eps(x) = { y in X : pred(x, y) }          x itself included
 *   core(x)  <=> |N_eps(x)| >= minPts
 *   clusters  = connected components of the core points under pred
 *   border b  = non-core point with at least one core neighbour
 *   noise     = every other point, label -1
 *
 * Readings of the paper fixed here:
 *   - pred(p, q): FP32, round-to-nearest-even, no FMA contraction, operations
 *     in this order:  dx = p.x - q.x, dy = ..., dz = ...;
 *     d2 = (dx*dx + dy*dy) + dz*dz;  neighbours iff d2 <= fl(eps*eps).
 *     This file must be compiled with -ffp-contract=off.
 *   - "<=" (the neighbourhood is closed).
 *   - K(C) = the smallest original index of a core point in cluster C.
 *   - a border point joins the cluster with the smallest K among the clusters
 *     of its core neighbours (the paper's first-come critical section in
 *     Algorithm PDSDbscan is nondeterministic; this replaces it).
 *   - the cluster id is the smallest original index over all members of the
 *     cluster, cores and assigned border points; noise is -1.
 *
 * Neighbour enumeration is a uniform grid (cell side H >= the largest
 * per-axis separation pred can accept) with the points sorted by row-major
 * cell key; every point's candidates are the points of the 27 cells around
 * its own.  The union-find is sequential, linking the root with the larger
 * index under the root with the smaller one (Tarjan's disjoint sets, as in
 * Algorithm DSDbscan).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_OK 0
#define ORC_EINVAL (-1)
#define ORC_ENONFINITE (-2)
#define ORC_ENOMEM (-3)

#define CELL_BITS 21
#define CELL_MAX ((int64_t)((1u << CELL_BITS) - 1u))

/* ---- the neighbour predicate (the exactness contract) -------------------- */

static int orc_pred(const float *p, const float *q, float e2)
{
    float dx = p[0] - q[0];
    float dy = p[1] - q[1];
    float dz = p[2] - q[2];
    float d2 = dx * dx + dy * dy;
    d2 = d2 + dz * dz;
    return d2 <= e2;
}

int oracle_pred(const float *p, const float *q, float eps)
{
    float e2 = eps * eps;
    return orc_pred(p, q, e2);
}

/* ---- grid ---------------------------------------------------------------- */

typedef struct {
    uint64_t key; /* cz << 42 | cy << 21 | cx */
    int64_t idx;  /* original index */
} orc_kv;

typedef struct {
    const float *pts;
    int64_t n;
    float e2;
    orc_kv *s; /* points sorted by (cell key, original index) */
} orc_grid;

static uint64_t orc_key(int64_t cx, int64_t cy, int64_t cz)
{
    return ((uint64_t)cz << (2 * CELL_BITS)) | ((uint64_t)cy << CELL_BITS) | (uint64_t)cx;
}

/* Stable LSD radix sort of (key, idx) records by key, 8 bits per pass. */
static void orc_radix_sort(orc_kv *a, orc_kv *tmp, int64_t n)
{
    for (int shift = 0; shift < 64; shift += 8) {
        int64_t count[257];
        memset(count, 0, sizeof(count));
        for (int64_t i = 0; i < n; i++)
            count[((a[i].key >> shift) & 0xFF) + 1]++;
        if (count[1 + ((a[0].key >> shift) & 0xFF)] == n)
            continue; /* every key has the same digit: order unchanged */
        for (int d = 0; d < 256; d++)
            count[d + 1] += count[d];
        for (int64_t i = 0; i < n; i++)
            tmp[count[(a[i].key >> shift) & 0xFF]++] = a[i];
        memcpy(a, tmp, (size_t)n * sizeof(orc_kv));
    }
}

/*
 * Cell side H.  If pred(p, q) holds and fl(eps*eps) is a normal float, then
 * fl(dx*dx) <= fl(eps*eps) gives |dx| <= eps*(1+2^-24)^2 and, the float
 * subtraction being exact or rounded by at most 2^-24, |p.x - q.x| stays
 * below eps*(1 + 2^-10).  For eps < 2^-60 the same bound holds with 2^-60 in
 * place of eps (fl(eps*eps) is then at most 2^-120, still normal).  So with
 * H = max(eps, 2^-60) * (1 + 2^-10) two neighbours are never more than one
 * cell apart on any axis.  A coarser grid is equally correct, so H is also
 * raised until the extent spans at most 2^20 cells per axis (cell keys then
 * fit 21 bits per axis and double-precision cell coordinates are exact to far
 * better than one cell).
 */
static int orc_build_grid(orc_grid *g, const float *pts, int64_t n, float eps)
{
    double lo[3] = {INFINITY, INFINITY, INFINITY};
    double hi[3] = {-INFINITY, -INFINITY, -INFINITY};
    for (int64_t i = 0; i < n; i++)
        for (int k = 0; k < 3; k++) {
            double v = pts[3 * i + k];
            if (v < lo[k])
                lo[k] = v;
            if (v > hi[k])
                hi[k] = v;
        }
    double extent = 0.0;
    for (int k = 0; k < 3; k++)
        if (hi[k] - lo[k] > extent)
            extent = hi[k] - lo[k];

    double H = (double)eps;
    if (H < ldexp(1.0, -60))
        H = ldexp(1.0, -60);
    H *= 1.0 + ldexp(1.0, -10);
    if (extent / H > ldexp(1.0, 20))
        H = extent / ldexp(1.0, 20);

    orc_kv *s = (orc_kv *)malloc((size_t)n * sizeof(orc_kv));
    orc_kv *tmp = (orc_kv *)malloc((size_t)n * sizeof(orc_kv));
    if (!s || !tmp) {
        free(s);
        free(tmp);
        return ORC_ENOMEM;
    }
    for (int64_t i = 0; i < n; i++) {
        int64_t c[3];
        for (int k = 0; k < 3; k++) {
            double q = floor(((double)pts[3 * i + k] - lo[k]) / H);
            if (q < 0.0)
                q = 0.0;
            if (q > (double)(CELL_MAX - 1))
                q = (double)(CELL_MAX - 1);
            c[k] = (int64_t)q;
        }
        s[i].key = orc_key(c[0], c[1], c[2]);
        s[i].idx = i;
    }
    orc_radix_sort(s, tmp, n);
    free(tmp);

    g->pts = pts;
    g->n = n;
    g->e2 = eps * eps;
    g->s = s;
    return ORC_OK;
}

/*
 * Enumerate neighbours.  For every point i (visited in cell order) for which
 * want(i) holds, call visit(i, j) for each j with pred(i, j), i itself
 * included; visit returning nonzero stops the enumeration for this i (early
 * termination, paper section "Early termination").
 *
 * The candidates of a point in cell (cx, cy, cz) are the 9 rows
 * (cy + dy, cz + dz), dy, dz in {-1, 0, 1}, each the key interval
 * [key(cx-1, .), key(cx+1, .)].  Cells are visited in increasing key order and
 * every row interval moves forward monotonically with it, so each row keeps
 * two forward-only cursors into the sorted array.
 */
typedef int (*orc_want_fn)(void *ctx, int64_t i);
typedef int (*orc_visit_fn)(void *ctx, int64_t i, int64_t j);

static void orc_sweep(const orc_grid *g, orc_want_fn want, orc_visit_fn visit, void *ctx)
{
    const orc_kv *s = g->s;
    const int64_t n = g->n;
    int64_t lo[9], hi[9], rlo[9], rhi[9];
    int valid[9];
    for (int r = 0; r < 9; r++) {
        lo[r] = hi[r] = rlo[r] = rhi[r] = 0;
        valid[r] = 0;
    }
    uint64_t cur = ~(uint64_t)0;
    for (int64_t p = 0; p < n; p++) {
        if (s[p].key != cur) {
            cur = s[p].key;
            int64_t cx = (int64_t)(cur & CELL_MAX);
            int64_t cy = (int64_t)((cur >> CELL_BITS) & CELL_MAX);
            int64_t cz = (int64_t)(cur >> (2 * CELL_BITS));
            for (int r = 0; r < 9; r++) {
                int64_t y = cy + (r % 3) - 1;
                int64_t z = cz + (r / 3) - 1;
                valid[r] = (y >= 0 && z >= 0);
                if (!valid[r])
                    continue;
                uint64_t klo = orc_key(cx > 0 ? cx - 1 : 0, y, z);
                uint64_t khi = orc_key(cx + 1, y, z);
                while (lo[r] < n && s[lo[r]].key < klo)
                    lo[r]++;
                if (hi[r] < lo[r])
                    hi[r] = lo[r];
                while (hi[r] < n && s[hi[r]].key <= khi)
                    hi[r]++;
                rlo[r] = lo[r];
                rhi[r] = hi[r];
            }
        }
        int64_t i = s[p].idx;
        if (!want(ctx, i))
            continue;
        const float *pi = g->pts + 3 * i;
        for (int r = 0; r < 9; r++) {
            if (!valid[r])
                continue;
            for (int64_t q = rlo[r]; q < rhi[r]; q++) {
                int64_t j = s[q].idx;
                if (orc_pred(pi, g->pts + 3 * j, g->e2) && visit(ctx, i, j))
                    goto next_point;
            }
        }
    next_point:;
    }
}

/* ---- sequential union-find over original indices ------------------------- */

static int32_t orc_find(int32_t *parent, int32_t x)
{
    int32_t r = x;
    while (parent[r] != r)
        r = parent[r];
    while (parent[x] != r) { /* path compression */
        int32_t nx = parent[x];
        parent[x] = r;
        x = nx;
    }
    return r;
}

static void orc_union(int32_t *parent, int32_t a, int32_t b)
{
    a = orc_find(parent, a);
    b = orc_find(parent, b);
    if (a == b)
        return;
    if (a < b)
        parent[b] = a;
    else
        parent[a] = b;
}

/* ---- the three passes ---------------------------------------------------- */

typedef struct {
    int32_t minpts;
    int32_t *count;  /* |N_eps(i)|, counted up to minPts */
    uint8_t *core;
    int32_t *parent;
    int32_t *border; /* root chosen by a border point, or -1 */
} orc_state;

static int want_all(void *ctx, int64_t i)
{
    (void)ctx;
    (void)i;
    return 1;
}

static int visit_count(void *ctx, int64_t i, int64_t j)
{
    orc_state *st = (orc_state *)ctx;
    (void)j;
    st->count[i]++;
    return st->count[i] >= st->minpts; /* stop once i is known to be core */
}

static int want_core(void *ctx, int64_t i)
{
    return ((orc_state *)ctx)->core[i];
}

static int visit_union(void *ctx, int64_t i, int64_t j)
{
    orc_state *st = (orc_state *)ctx;
    if (j > i && st->core[j])
        orc_union(st->parent, (int32_t)i, (int32_t)j);
    return 0;
}

static int want_noncore(void *ctx, int64_t i)
{
    return !((orc_state *)ctx)->core[i];
}

static int visit_border(void *ctx, int64_t i, int64_t j)
{
    orc_state *st = (orc_state *)ctx;
    if (st->core[j]) {
        /* find() over cores returns K(C): roots are the smallest member. */
        int32_t k = orc_find(st->parent, (int32_t)j);
        if (st->border[i] < 0 || k < st->border[i])
            st->border[i] = k;
    }
    return 0;
}

/*
 * oracle_dbscan: labels[i] = smallest original index in i's cluster, or -1
 * for noise.  points: n x 3 float32, row-major (x, y, z).  Returns ORC_OK or
 * a negative error code; labels is untouched on error.
 */
int oracle_dbscan(const float *points, int64_t n, float eps, int32_t minpts, int32_t *labels)
{
    if (n < 0 || n > INT32_MAX || minpts < 1 || !(eps >= 0.0f) || isinf(eps))
        return ORC_EINVAL;
    if (n == 0)
        return ORC_OK;
    if (!points || !labels)
        return ORC_EINVAL;
    for (int64_t i = 0; i < 3 * n; i++)
        if (!isfinite(points[i]))
            return ORC_ENONFINITE;

    orc_grid g;
    int rc = orc_build_grid(&g, points, n, eps);
    if (rc != ORC_OK)
        return rc;

    orc_state st;
    st.minpts = minpts;
    st.count = (int32_t *)calloc((size_t)n, sizeof(int32_t));
    st.core = (uint8_t *)calloc((size_t)n, 1);
    st.parent = (int32_t *)malloc((size_t)n * sizeof(int32_t));
    st.border = (int32_t *)malloc((size_t)n * sizeof(int32_t));
    if (!st.count || !st.core || !st.parent || !st.border) {
        free(st.count);
        free(st.core);
        free(st.parent);
        free(st.border);
        free(g.s);
        return ORC_ENOMEM;
    }

    /* 1. core points: |N_eps(i)| >= minPts (i counts itself). */
    orc_sweep(&g, want_all, visit_count, &st);
    for (int64_t i = 0; i < n; i++)
        st.core[i] = st.count[i] >= minpts;

    /* 2. clusters: union every pair of neighbouring core points. */
    for (int64_t i = 0; i < n; i++)
        st.parent[i] = (int32_t)i;
    orc_sweep(&g, want_core, visit_union, &st);

    /* 3. border points: the neighbouring cluster with the smallest K. */
    for (int64_t i = 0; i < n; i++)
        st.border[i] = -1;
    orc_sweep(&g, want_noncore, visit_border, &st);

    /* 4. cluster id = min over cores (K, the root) and assigned borders. */
    int32_t *id = st.count; /* reuse: id[root] */
    for (int64_t i = 0; i < n; i++)
        id[i] = INT32_MAX;
    for (int64_t i = 0; i < n; i++)
        if (st.core[i]) {
            int32_t r = orc_find(st.parent, (int32_t)i);
            if ((int32_t)i < id[r])
                id[r] = (int32_t)i;
        }
    for (int64_t i = 0; i < n; i++)
        if (!st.core[i] && st.border[i] >= 0 && (int32_t)i < id[st.border[i]])
            id[st.border[i]] = (int32_t)i;
    for (int64_t i = 0; i < n; i++) {
        if (st.core[i])
            labels[i] = id[orc_find(st.parent, (int32_t)i)];
        else if (st.border[i] >= 0)
            labels[i] = id[st.border[i]];
        else
            labels[i] = -1;
    }

    free(st.count);
    free(st.core);
    free(st.parent);
    free(st.border);
    free(g.s);
    return ORC_OK;
}

/*
 * oracle_core_flags: core[i] = 1 iff |N_eps(i)| >= minPts.  Exposed so the
 * tests can check the core classification on its own.
 */
int oracle_core_flags(const float *points, int64_t n, float eps, int32_t minpts, uint8_t *core)
{
    if (n < 0 || n > INT32_MAX || minpts < 1 || !(eps >= 0.0f) || isinf(eps))
        return ORC_EINVAL;
    if (n == 0)
        return ORC_OK;
    for (int64_t i = 0; i < 3 * n; i++)
        if (!isfinite(points[i]))
            return ORC_ENONFINITE;
    orc_grid g;
    int rc = orc_build_grid(&g, points, n, eps);
    if (rc != ORC_OK)
        return rc;
    orc_state st;
    memset(&st, 0, sizeof(st));
    st.minpts = minpts;
    st.count = (int32_t *)calloc((size_t)n, sizeof(int32_t));
    if (!st.count) {
        free(g.s);
        return ORC_ENOMEM;
    }
    orc_sweep(&g, want_all, visit_count, &st);
    for (int64_t i = 0; i < n; i++)
        core[i] = st.count[i] >= minpts;
    free(st.count);
    free(g.s);
    return ORC_OK;
}

/*
 * oracle_pair_count: the number of unordered pairs {i, j}, i != j, with
 * pred(i, j) -- what the paper's pair traversal visits exactly once each
 * (section "Pair traversal").
 */
int64_t oracle_pair_count(const float *points, int64_t n, float eps);

typedef struct {
    int64_t pairs;
} orc_pairs;

static int visit_pairs(void *ctx, int64_t i, int64_t j)
{
    if (j > i)
        ((orc_pairs *)ctx)->pairs++;
    return 0;
}

int64_t oracle_pair_count(const float *points, int64_t n, float eps)
{
    if (n < 0 || n > INT32_MAX || !(eps >= 0.0f) || isinf(eps))
        return ORC_EINVAL;
    if (n == 0)
        return 0;
    for (int64_t i = 0; i < 3 * n; i++)
        if (!isfinite(points[i]))
            return ORC_ENONFINITE;
    orc_grid g;
    int rc = orc_build_grid(&g, points, n, eps);
    if (rc != ORC_OK)
        return rc;
    orc_pairs c = {0};
    orc_sweep(&g, want_all, visit_pairs, &c);
    free(g.s);
    return c.pairs;
}

/*
 * oracle_pair_list: every unordered pair {i, j}, i < j (original indices),
 * with pred(i, j) -- the pairs the paper's pair traversal hands to its
 * callback F exactly once each (section "Pair traversal").  Writes the first
 * min(total, cap) pairs found to out[2k], out[2k+1] and returns the total.
 */
int64_t oracle_pair_list(const float *points, int64_t n, float eps, int64_t *out, int64_t cap);

typedef struct {
    int64_t pairs, cap;
    int64_t *out;
} orc_pair_list;

static int visit_pair_list(void *ctx, int64_t i, int64_t j)
{
    orc_pair_list *c = (orc_pair_list *)ctx;
    if (j > i) {
        if (c->pairs < c->cap) {
            c->out[2 * c->pairs] = i;
            c->out[2 * c->pairs + 1] = j;
        }
        c->pairs++;
    }
    return 0;
}

int64_t oracle_pair_list(const float *points, int64_t n, float eps, int64_t *out, int64_t cap)
{
    if (n < 0 || n > INT32_MAX || !(eps >= 0.0f) || isinf(eps) || cap < 0 || (cap > 0 && !out))
        return ORC_EINVAL;
    if (n == 0)
        return 0;
    for (int64_t i = 0; i < 3 * n; i++)
        if (!isfinite(points[i]))
            return ORC_ENONFINITE;
    orc_grid g;
    int rc = orc_build_grid(&g, points, n, eps);
    if (rc != ORC_OK)
        return rc;
    orc_pair_list c = {0, cap, out};
    orc_sweep(&g, want_all, visit_pair_list, &c);
    free(g.s);
    return c.pairs;
}

/* ---- consumers of a clustering (plain definitions) ------------------------- */

/*
 * oracle_cluster_stats: per cluster id l (a label value >= 0), in increasing
 * l: size, centre = mean position (summed in double in index order, rounded
 * to float), radius = sqrtf of the largest FP32 squared distance (the
 * predicate's expression) from that centre to a member.  Returns the number
 * of clusters written, or a negative error.  The paper's HACC section draws
 * galaxies as circles of that radius.
 */
int64_t oracle_cluster_stats(const float *points, const int32_t *labels, int64_t n, int32_t *ids, int32_t *sizes,
                             float *centres, float *radii)
{
    if (n < 0)
        return ORC_EINVAL;
    int64_t *cnt = (int64_t *)calloc((size_t)n + 1, sizeof(int64_t));
    double *sum = (double *)calloc(3 * ((size_t)n + 1), sizeof(double));
    float *r2 = (float *)calloc((size_t)n + 1, sizeof(float));
    if (!cnt || !sum || !r2) {
        free(cnt);
        free(sum);
        free(r2);
        return ORC_ENOMEM;
    }
    for (int64_t i = 0; i < n; i++) {
        int32_t l = labels[i];
        if (l < 0)
            continue;
        if (l >= n) {
            free(cnt);
            free(sum);
            free(r2);
            return ORC_EINVAL;
        }
        cnt[l]++;
        for (int k = 0; k < 3; k++)
            sum[3 * l + k] += (double)points[3 * i + k];
    }
    float *cen = (float *)malloc(3 * ((size_t)n + 1) * sizeof(float));
    if (!cen) {
        free(cnt);
        free(sum);
        free(r2);
        return ORC_ENOMEM;
    }
    for (int64_t l = 0; l < n; l++)
        if (cnt[l])
            for (int k = 0; k < 3; k++)
                cen[3 * l + k] = (float)(sum[3 * l + k] / (double)cnt[l]);
    for (int64_t i = 0; i < n; i++) {
        int32_t l = labels[i];
        if (l < 0)
            continue;
        float dx = points[3 * i] - cen[3 * l];
        float dy = points[3 * i + 1] - cen[3 * l + 1];
        float dz = points[3 * i + 2] - cen[3 * l + 2];
        float d2 = dx * dx + dy * dy;
        d2 = d2 + dz * dz;
        if (d2 > r2[l])
            r2[l] = d2;
    }
    int64_t k = 0;
    for (int64_t l = 0; l < n; l++)
        if (cnt[l]) {
            ids[k] = (int32_t)l;
            sizes[k] = (int32_t)cnt[l];
            for (int a = 0; a < 3; a++)
                centres[3 * k + a] = cen[3 * l + a];
            radii[k] = sqrtf(r2[l]);
            k++;
        }
    free(cnt);
    free(sum);
    free(r2);
    free(cen);
    return k;
}

/*
 * oracle_pair_histogram: hist[b] = number of unordered pairs {i, j}, i != j,
 * with fl(r_b^2) < d2 <= fl(r_{b+1}^2), d2 the predicate's FP32 expression
 * (paper, subsection "Pair traversal": apply F to every pair within a radius).
 */
typedef struct {
    const float *pts;
    const float *e2;
    int nbins;
    int64_t *hist;
} orc_hist;

static int visit_hist(void *ctx, int64_t i, int64_t j)
{
    orc_hist *h = (orc_hist *)ctx;
    if (j <= i)
        return 0;
    const float *p = h->pts + 3 * i, *q = h->pts + 3 * j;
    float dx = p[0] - q[0];
    float dy = p[1] - q[1];
    float dz = p[2] - q[2];
    float d2 = dx * dx + dy * dy;
    d2 = d2 + dz * dz;
    for (int b = 0; b < h->nbins; b++)
        if (d2 > h->e2[b] && d2 <= h->e2[b + 1]) {
            h->hist[b]++;
            break;
        }
    return 0;
}

int oracle_pair_histogram(const float *points, int64_t n, const float *r_edges, int32_t nbins, int64_t *hist)
{
    if (n < 0 || nbins < 1 || nbins > 256)
        return ORC_EINVAL;
    float e2[257];
    for (int b = 0; b <= nbins; b++) {
        if (!(r_edges[b] >= 0.0f) || isinf(r_edges[b]) || (b > 0 && !(r_edges[b] > r_edges[b - 1])))
            return ORC_EINVAL;
        e2[b] = r_edges[b] * r_edges[b];
    }
    for (int b = 0; b < nbins; b++)
        hist[b] = 0;
    if (n == 0)
        return ORC_OK;
    orc_grid g;
    int rc = orc_build_grid(&g, points, n, r_edges[nbins]);
    if (rc != ORC_OK)
        return rc;
    orc_hist h = {points, e2, nbins, hist};
    orc_sweep(&g, want_all, visit_hist, &h);
    free(g.s);
    return ORC_OK;
}
