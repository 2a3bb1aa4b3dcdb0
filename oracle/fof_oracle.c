/*
 * Friends-of-Friends CPU ORACLE -- test infrastructure, not the product.
 *
 * Only the test-suite, the smoke check and the benchmark's CPU-baseline leg
 * load this library.  It shares no code, header or constant with the CUDA
 * path; it is a plain, slow, single-threaded restatement of what the group
 * finder must compute.
 *
 * What is computed (paper Sec. 1, footnote on the graph definition):
 * the groups are the connected components of G = (P, E) with
 * E = {{u, v} : dist(u, v) <= l_x}; particles with no neighbour form groups
 * of size one (Sec. 1).  Group labels are the smallest particle index in the
 * group, which is the root that union-by-root produces when every set starts
 * rooted at its own array offset and the larger root is always hooked onto
 * the smaller one (Sec. 2; Sec. 3.1).  Group sizes are stored at the label,
 * like the paper's group_size array indexed by the root (Sec. 3.4.1).
 *
 * Distance arithmetic (the paper does not fix it; the reading used here):
 * per axis d = (double)p_i - (double)p_j, wrapped once into the periodic
 * minimum image by "if d > L/2: d -= L; else if d < -L/2: d += L", then
 * s = (dx*dx + dy*dy) + dz*dz with every operation rounded to nearest in
 * IEEE double and no fused multiply-add, and the pair is linked iff
 * s <= l2 where l2 = l_x * l_x rounded once.  The "at most" wording of the
 * abstract and the <= of the graph definition decide the tie.
 * This file must be compiled with -ffp-contract=off (and no -ffast-math).
 *
 * Entry points (the *_rule variants take the tie rule: strict = 1 links
 * only pairs at distance < l_x, the naive listing's test in Sec. 3.1; the
 * others use <=):
 *   fof_oracle_linked      the predicate itself (for pinning tests)
 *   fof_oracle_linked_many the predicate over arrays of pairs
 *   fof_oracle_groups      cell list + breadth-first search, all particles
 *   fof_oracle_brute       O(N^2) pair loop + serial union-find (tiny N)
 *   fof_oracle_component   breadth-first search of one particle's group
 *   fof_oracle_catalogue   filter of the size array into (label, size)
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------ */
/* the link predicate                                                  */
/* ------------------------------------------------------------------ */

static double wrap_axis(double d, double box)
{
    double half = 0.5 * box;
    if (d > half)
        d = d - box;
    else if (d < -half)
        d = d + box;
    return d;
}

/* strict = 0: linked iff s <= l2 (the graph definition); strict = 1:
 * linked iff s < l2, the "r < l_x" of the paper's naive pair loop (Sec. 3.1),
 * kept to measure the tie rule as a variant. */
static int linked_rule(const float *a, const float *b, double box, double l2, int strict)
{
    double dx = wrap_axis((double)a[0] - (double)b[0], box);
    double dy = wrap_axis((double)a[1] - (double)b[1], box);
    double dz = wrap_axis((double)a[2] - (double)b[2], box);
    double xx = dx * dx;
    double yy = dy * dy;
    double zz = dz * dz;
    double s = xx + yy;
    s = s + zz;
    if (strict)
        return s < l2;
    return s <= l2;
}

static int linked(const float *a, const float *b, double box, double l2)
{
    return linked_rule(a, b, box, l2, 0);
}

int fof_oracle_linked(const float *a, const float *b, double box, double l_x)
{
    double l2 = l_x * l_x;
    return linked(a, b, box, l2);
}

int fof_oracle_linked_rule(const float *a, const float *b, double box, double l_x, int strict)
{
    double l2 = l_x * l_x;
    return linked_rule(a, b, box, l2, strict);
}

/* out[k] = the predicate for the pair (a[k], b[k]), k < m */
void fof_oracle_linked_many(int64_t m, const float *a, const float *b, double box, double l_x,
                            uint8_t *out)
{
    double l2 = l_x * l_x;
    for (int64_t k = 0; k < m; ++k)
        out[k] = (uint8_t)linked(a + 3 * k, b + 3 * k, box, l2);
}

/* ------------------------------------------------------------------ */
/* cell list: particles sorted by the key of a cubic cell of side >= l */
/* ------------------------------------------------------------------ */

typedef struct {
    int64_t n;
    const float *pos;
    double box, l2;
    int strict;          /* tie rule, see linked_rule */
    int64_t nc;          /* cells per axis */
    uint64_t *key;       /* key[k] of the k-th particle in cell order */
    int32_t *idx;        /* idx[k] = particle index */
} grid_t;

typedef struct { uint64_t key; int32_t idx; } kv_t;

static int cmp_kv(const void *pa, const void *pb)
{
    const kv_t *a = (const kv_t *)pa, *b = (const kv_t *)pb;
    if (a->key != b->key)
        return a->key < b->key ? -1 : 1;
    return (a->idx > b->idx) - (a->idx < b->idx);
}

static int64_t cell_of(float x, int64_t nc, double box)
{
    double u = floor((double)x * (double)nc / box);
    int64_t c = (int64_t)u;
    if (c < 0) c = 0;
    if (c >= nc) c = nc - 1;
    return c;
}

static uint64_t pack(int64_t cx, int64_t cy, int64_t cz)
{
    return ((uint64_t)cz << 42) | ((uint64_t)cy << 21) | (uint64_t)cx;
}

/* cell side L/nc is at least l_x (1 + 2^-20); the margin is far above the
 * rounding of the index computation, so any linked pair sits in the same or
 * in periodically adjacent cells. */
static int64_t cells_per_axis(double box, double l_x)
{
    double q = floor(box / (l_x * (1.0 + ldexp(1.0, -20))));
    if (!(q >= 1.0)) q = 1.0;
    if (q > 2097151.0) q = 2097151.0;
    return (int64_t)q;
}

static int grid_build(grid_t *g, int64_t n, const float *pos, double box, double l_x, int strict)
{
    memset(g, 0, sizeof(*g));
    g->n = n; g->pos = pos; g->box = box; g->l2 = l_x * l_x; g->strict = strict;
    g->nc = cells_per_axis(box, l_x);
    if (n == 0)
        return 0;
    kv_t *tmp = (kv_t *)malloc((size_t)n * sizeof(kv_t));
    g->key = (uint64_t *)malloc((size_t)n * sizeof(uint64_t));
    g->idx = (int32_t *)malloc((size_t)n * sizeof(int32_t));
    if (!tmp || !g->key || !g->idx) {
        free(tmp); free(g->key); free(g->idx);
        return -1;
    }
    for (int64_t i = 0; i < n; ++i) {
        const float *p = pos + 3 * i;
        tmp[i].key = pack(cell_of(p[0], g->nc, box), cell_of(p[1], g->nc, box),
                          cell_of(p[2], g->nc, box));
        tmp[i].idx = (int32_t)i;
    }
    qsort(tmp, (size_t)n, sizeof(kv_t), cmp_kv);
    for (int64_t k = 0; k < n; ++k) {
        g->key[k] = tmp[k].key;
        g->idx[k] = tmp[k].idx;
    }
    free(tmp);
    return 0;
}

static void grid_free(grid_t *g)
{
    free(g->key); free(g->idx);
    g->key = NULL; g->idx = NULL;
}

/* first position k with key[k] >= want */
static int64_t lower_bound(const grid_t *g, uint64_t want)
{
    int64_t lo = 0, hi = g->n;
    while (lo < hi) {
        int64_t mid = lo + (hi - lo) / 2;
        if (g->key[mid] < want) lo = mid + 1; else hi = mid;
    }
    return lo;
}

/* the distinct periodic neighbour cells (including the cell itself) */
static int neighbour_keys(const grid_t *g, const float *p, uint64_t out[27])
{
    int64_t nc = g->nc;
    int64_t c[3];
    for (int k = 0; k < 3; ++k) c[k] = cell_of(p[k], nc, g->box);
    int m = 0;
    for (int dz = -1; dz <= 1; ++dz)
        for (int dy = -1; dy <= 1; ++dy)
            for (int dx = -1; dx <= 1; ++dx) {
                int64_t x = ((c[0] + dx) % nc + nc) % nc;
                int64_t y = ((c[1] + dy) % nc + nc) % nc;
                int64_t z = ((c[2] + dz) % nc + nc) % nc;
                uint64_t k = pack(x, y, z);
                int dup = 0;
                for (int q = 0; q < m; ++q)
                    if (out[q] == k) { dup = 1; break; }
                if (!dup) out[m++] = k;
            }
    return m;
}

/* breadth-first search from `start`; marks every reached particle with
 * `label` in mark[] and appends it to queue[] (which must hold n entries).
 * Returns the number of particles reached. */
static int64_t bfs(const grid_t *g, int64_t start, int32_t label,
                   int32_t *mark, int32_t *queue)
{
    int64_t head = 0, tail = 0;
    mark[start] = label;
    queue[tail++] = (int32_t)start;
    uint64_t keys[27];
    while (head < tail) {
        int32_t p = queue[head++];
        const float *pp = g->pos + 3 * (int64_t)p;
        int m = neighbour_keys(g, pp, keys);
        for (int q = 0; q < m; ++q) {
            int64_t k = lower_bound(g, keys[q]);
            for (; k < g->n && g->key[k] == keys[q]; ++k) {
                int32_t j = g->idx[k];
                if (mark[j] == label)
                    continue;
                if (linked_rule(pp, g->pos + 3 * (int64_t)j, g->box, g->l2, g->strict)) {
                    mark[j] = label;
                    queue[tail++] = j;
                }
            }
        }
    }
    return tail;
}

/* ------------------------------------------------------------------ */
/* all groups                                                          */
/* ------------------------------------------------------------------ */

/* ids[i] = smallest index in i's group; sizes[g] = size of the group
 * labelled g, 0 where g is not a label.  Returns 0, or -1 on allocation
 * failure. */
int fof_oracle_groups_rule(int64_t n, const float *pos, double box, double l_x, int strict,
                           int32_t *ids, int32_t *sizes)
{
    if (n == 0)
        return 0;
    grid_t g;
    if (grid_build(&g, n, pos, box, l_x, strict))
        return -1;
    int32_t *queue = (int32_t *)malloc((size_t)n * sizeof(int32_t));
    if (!queue) { grid_free(&g); return -1; }
    for (int64_t i = 0; i < n; ++i) { ids[i] = -1; sizes[i] = 0; }
    /* scanning i upwards, the first unlabelled i is the smallest index of
     * its group: every smaller index was labelled with its own group */
    for (int64_t i = 0; i < n; ++i) {
        if (ids[i] >= 0)
            continue;
        int64_t m = bfs(&g, i, (int32_t)i, ids, queue);
        sizes[i] = (int32_t)m;
    }
    free(queue);
    grid_free(&g);
    return 0;
}

int fof_oracle_groups(int64_t n, const float *pos, double box, double l_x,
                      int32_t *ids, int32_t *sizes)
{
    return fof_oracle_groups_rule(n, pos, box, l_x, 0, ids, sizes);
}

/* ------------------------------------------------------------------ */
/* brute force: the paper's naive all-pairs union-find                 */
/* ------------------------------------------------------------------ */

static int32_t uf_find(int32_t *parent, int32_t x)
{
    while (parent[x] != x)
        x = parent[x];
    return x;
}

/* Every unordered pair i != j is tested; linked pairs merge their roots,
 * the larger root is hooked onto the smaller (Sec. 3.1), so the final root
 * of each set is its smallest index.  ids[i] = that root. */
int fof_oracle_brute_rule(int64_t n, const float *pos, double box, double l_x, int strict,
                          int32_t *ids)
{
    double l2 = l_x * l_x;
    for (int64_t i = 0; i < n; ++i)
        ids[i] = (int32_t)i;
    for (int64_t i = 0; i < n; ++i)
        for (int64_t j = i + 1; j < n; ++j) {
            if (!linked_rule(pos + 3 * i, pos + 3 * j, box, l2, strict))
                continue;
            int32_t ri = uf_find(ids, (int32_t)i);
            int32_t rj = uf_find(ids, (int32_t)j);
            if (ri < rj) ids[rj] = ri;
            else if (rj < ri) ids[ri] = rj;
        }
    for (int64_t i = 0; i < n; ++i)
        ids[i] = uf_find(ids, (int32_t)i);
    return 0;
}

int fof_oracle_brute(int64_t n, const float *pos, double box, double l_x, int32_t *ids)
{
    return fof_oracle_brute_rule(n, pos, box, l_x, 0, ids);
}

/* ------------------------------------------------------------------ */
/* one group                                                           */
/* ------------------------------------------------------------------ */

/* The group containing particle `start`.  members[] receives its indices
 * (capacity n), *count its size and *label its smallest index.
 * Returns 0, or -1 on allocation failure. */
int fof_oracle_component(int64_t n, const float *pos, double box, double l_x,
                         int64_t start, int32_t *members, int64_t *count,
                         int64_t *label)
{
    grid_t g;
    if (grid_build(&g, n, pos, box, l_x, 0))
        return -1;
    int32_t *mark = (int32_t *)malloc((size_t)n * sizeof(int32_t));
    if (!mark) { grid_free(&g); return -1; }
    for (int64_t i = 0; i < n; ++i) mark[i] = -1;
    /* label -2 never equals a "groups mode" label, so no member is skipped */
    int64_t m = bfs(&g, start, -2, mark, members);
    int64_t lo = start;
    for (int64_t k = 0; k < m; ++k)
        if (members[k] < lo) lo = members[k];
    *count = m;
    *label = lo;
    free(mark);
    grid_free(&g);
    return 0;
}

/* ------------------------------------------------------------------ */
/* catalogue                                                           */
/* ------------------------------------------------------------------ */

/* (label, size) for every label g with sizes[g] >= max(min_size, 1), in
 * ascending g.  Writes at most cap pairs to cat[2*k], cat[2*k+1]; returns
 * the number of qualifying groups. */
int64_t fof_oracle_catalogue(int64_t n, const int32_t *sizes, int32_t min_size,
                             int32_t *cat, int64_t cap)
{
    int32_t thr = min_size < 1 ? 1 : min_size;
    int64_t k = 0;
    for (int64_t g = 0; g < n; ++g) {
        if (sizes[g] >= thr) {
            if (k < cap) {
                cat[2 * k] = (int32_t)g;
                cat[2 * k + 1] = sizes[g];
            }
            ++k;
        }
    }
    return k;
}
