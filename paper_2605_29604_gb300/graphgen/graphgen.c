/*
 * graphgen.c -- seeded synthetic graph generators.
 *
 * These build the inputs that both the CUDA path and the CPU oracle consume:
 * undirected, unweighted graphs in int32 CSR form (sorted rows, no duplicate
 * arcs, no self-loops, symmetric), the form the paper's MIS method takes as
 * input (Sec. 4.1.2: all graphs undirected and unweighted).  Nothing here
 * computes any part of the MIS method itself; the file holds random-number
 * streams and graph construction only.
 *
 * Families (stand-ins for the paper's SuiteSparse inputs, Table 1):
 *   - Erdos-Renyi G(n, m): m distinct undirected pairs, uniform.
 *   - R-MAT (Chakrabarti, Zhan, Faloutsos, SDM 2004): recursive quadrant
 *     choice with probabilities (a, b, c, d), no noise.
 *   - W x W 4-neighbour grid plus a chosen number of distinct random
 *     diagonals (i,j)-(i+1,j+1) / (i,j)-(i+1,j-1).
 *   - Random geometric graph in the unit square, radius r, ids in
 *     cell-sorted order.
 *   - Random relabelling of any graph.
 *
 * Random numbers: the splitmix64 generator (Steele, Lea, Flood, "Fast
 * splittable pseudorandom number generators", OOPSLA 2014): a Weyl sequence
 * with increment 0x9E3779B97F4A7C15 fed through a 64-bit finaliser.
 *
 * Host C only; compiled with -ffp-contract=off so that the double-precision
 * geometry gives the same graph on every host.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>

typedef struct {
    int32_t n;
    int64_t arcs;
    int32_t *row_ptr; /* n + 1 */
    int32_t *col_idx; /* arcs */
} gg_graph;

typedef struct {
    uint64_t s;
} gg_rng;

static uint64_t gg_next(gg_rng *r)
{
    uint64_t z = (r->s += 0x9E3779B97F4A7C15ULL);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

/* uniform double in [0, 1) with 53 random bits */
static double gg_unif(gg_rng *r) { return (double)(gg_next(r) >> 11) * 0x1.0p-53; }

/* uniform integer in [0, bound), bound >= 1, by rejection (no modulo bias) */
static uint64_t gg_below(gg_rng *r, uint64_t bound)
{
    uint64_t threshold = (0 - bound) % bound;
    for (;;) {
        uint64_t x = gg_next(r);
        if (x >= threshold) return x % bound;
    }
}

void gg_free(gg_graph *g)
{
    if (!g) return;
    free(g->row_ptr);
    free(g->col_idx);
    free(g);
}

int32_t gg_n(const gg_graph *g) { return g->n; }
int64_t gg_arcs(const gg_graph *g) { return g->arcs; }

void gg_copy(const gg_graph *g, int32_t *row_ptr, int32_t *col_idx)
{
    memcpy(row_ptr, g->row_ptr, sizeof(int32_t) * ((size_t)g->n + 1));
    if (g->arcs) memcpy(col_idx, g->col_idx, sizeof(int32_t) * (size_t)g->arcs);
}

/*
 * Symmetric CSR from an undirected edge list: both directions of every pair,
 * self-loops dropped, duplicates removed, rows sorted ascending.  Two
 * counting-sort passes (by destination, then stably by source) give sorted
 * rows without a comparison sort.  Returns NULL when the arc count does not
 * fit int32 or memory runs out.
 */
gg_graph *gg_from_edges(int32_t n, int64_t ne, const int32_t *eu, const int32_t *ev)
{
    gg_graph *g = (gg_graph *)calloc(1, sizeof(gg_graph));
    int64_t *cnt = (int64_t *)calloc((size_t)n + 1, sizeof(int64_t));
    int64_t *cur = (int64_t *)malloc(sizeof(int64_t) * ((size_t)n + 1));
    if (!g || !cnt || !cur) goto fail;
    g->n = n;
    int64_t total = 0;
    for (int64_t e = 0; e < ne; ++e) {
        int32_t u = eu[e], v = ev[e];
        if (u == v) continue;
        cnt[u]++;
        cnt[v]++;
        total += 2;
    }
    /* pass 1: bucket by destination, storing the source */
    int64_t acc = 0;
    for (int32_t i = 0; i < n; ++i) {
        cur[i] = acc;
        acc += cnt[i];
    }
    cur[n] = acc;
    int32_t *by_dst = (int32_t *)malloc(sizeof(int32_t) * (size_t)(total ? total : 1));
    int32_t *col = (int32_t *)malloc(sizeof(int32_t) * (size_t)(total ? total : 1));
    int64_t *rp = (int64_t *)malloc(sizeof(int64_t) * ((size_t)n + 1));
    if (!by_dst || !col || !rp) {
        free(by_dst);
        free(col);
        free(rp);
        goto fail;
    }
    for (int64_t e = 0; e < ne; ++e) {
        int32_t u = eu[e], v = ev[e];
        if (u == v) continue;
        by_dst[cur[v]++] = u; /* arc u -> v */
        by_dst[cur[u]++] = v; /* arc v -> u */
    }
    /* pass 2: walk destinations in ascending order, append to source rows */
    acc = 0;
    for (int32_t i = 0; i < n; ++i) {
        rp[i] = acc;
        cur[i] = acc;
        acc += cnt[i];
    }
    rp[n] = acc;
    int64_t start = 0;
    for (int32_t d = 0; d < n; ++d) {
        int64_t end = start + cnt[d];
        for (int64_t k = start; k < end; ++k) col[cur[by_dst[k]]++] = d;
        start = end;
    }
    free(by_dst);
    /* dedup in place (rows are sorted) and compact */
    g->row_ptr = (int32_t *)malloc(sizeof(int32_t) * ((size_t)n + 1));
    if (!g->row_ptr) {
        free(col);
        free(rp);
        goto fail;
    }
    int64_t w = 0;
    for (int32_t i = 0; i < n; ++i) {
        int64_t b = rp[i], e = rp[i + 1];
        if (w > INT32_MAX) {
            free(col);
            free(rp);
            goto fail;
        }
        g->row_ptr[i] = (int32_t)w;
        for (int64_t k = b; k < e; ++k) {
            if (k > b && col[k] == col[k - 1]) continue;
            col[w++] = col[k];
        }
    }
    if (w > INT32_MAX) {
        free(col);
        free(rp);
        goto fail;
    }
    g->row_ptr[n] = (int32_t)w;
    g->arcs = w;
    free(rp);
    g->col_idx = (int32_t *)realloc(col, sizeof(int32_t) * (size_t)(w ? w : 1));
    if (!g->col_idx) g->col_idx = col;
    free(cnt);
    free(cur);
    return g;
fail:
    free(cnt);
    free(cur);
    gg_free(g);
    return NULL;
}

/* ---- open-addressing set of 64-bit keys (for distinct-pair sampling) ---- */
typedef struct {
    uint64_t *slot;
    uint64_t mask;
} gg_set;

static int gg_set_init(gg_set *s, int64_t expect)
{
    uint64_t cap = 16;
    while (cap < (uint64_t)expect * 2 + 16) cap <<= 1;
    s->slot = (uint64_t *)malloc(sizeof(uint64_t) * cap);
    if (!s->slot) return -1;
    memset(s->slot, 0xFF, sizeof(uint64_t) * cap); /* empty = all ones */
    s->mask = cap - 1;
    return 0;
}

/* insert; returns 1 when newly added, 0 when present.  key != ~0 */
static int gg_set_add(gg_set *s, uint64_t key)
{
    uint64_t h = key * 0x9E3779B97F4A7C15ULL;
    uint64_t i = (h ^ (h >> 29)) & s->mask;
    for (;;) {
        uint64_t k = s->slot[i];
        if (k == ~0ULL) {
            s->slot[i] = key;
            return 1;
        }
        if (k == key) return 0;
        i = (i + 1) & s->mask;
    }
}

/* Erdos-Renyi G(n, m): m distinct unordered pairs {u, v}, u != v, uniform. */
gg_graph *gg_er_gnm(int32_t n, int64_t m, uint64_t seed)
{
    if (n < 0 || m < 0) return NULL;
    if (n < 2 && m > 0) return NULL;
    if ((double)m > (double)n * (double)(n - 1) / 2.0) return NULL;
    int32_t *eu = (int32_t *)malloc(sizeof(int32_t) * (size_t)(m ? m : 1));
    int32_t *ev = (int32_t *)malloc(sizeof(int32_t) * (size_t)(m ? m : 1));
    gg_set set;
    if (!eu || !ev || gg_set_init(&set, m) != 0) {
        free(eu);
        free(ev);
        return NULL;
    }
    gg_rng r = {seed};
    int64_t got = 0;
    while (got < m) {
        int32_t u = (int32_t)gg_below(&r, (uint64_t)n);
        int32_t v = (int32_t)gg_below(&r, (uint64_t)n);
        if (u == v) continue;
        int32_t lo = u < v ? u : v, hi = u < v ? v : u;
        if (!gg_set_add(&set, ((uint64_t)(uint32_t)lo << 32) | (uint32_t)hi)) continue;
        eu[got] = lo;
        ev[got] = hi;
        ++got;
    }
    free(set.slot);
    gg_graph *g = gg_from_edges(n, m, eu, ev);
    free(eu);
    free(ev);
    return g;
}

/*
 * R-MAT: each of `ne` generated edges descends `scale` levels; at each level
 * one uniform draw picks quadrant (0,0) with prob. a, (0,1) with b, (1,0)
 * with c, (1,1) with d = 1 - a - b - c.  Row bits are set for the lower
 * half, column bits for the right half, most significant bit first.  The
 * result is symmetrised and deduplicated, self-loops dropped (ids are NOT
 * permuted here; see gg_permute).
 */
gg_graph *gg_rmat(int32_t scale, int64_t ne, double a, double b, double c, uint64_t seed)
{
    if (scale < 1 || scale > 30 || ne < 0) return NULL;
    int32_t n = (int32_t)1 << scale;
    int32_t *eu = (int32_t *)malloc(sizeof(int32_t) * (size_t)(ne ? ne : 1));
    int32_t *ev = (int32_t *)malloc(sizeof(int32_t) * (size_t)(ne ? ne : 1));
    if (!eu || !ev) {
        free(eu);
        free(ev);
        return NULL;
    }
    gg_rng r = {seed};
    const double ab = a + b, abc = a + b + c;
    for (int64_t e = 0; e < ne; ++e) {
        uint32_t u = 0, v = 0;
        for (int32_t lvl = scale - 1; lvl >= 0; --lvl) {
            double x = gg_unif(&r);
            if (x < a) {
            } else if (x < ab) {
                v |= 1u << lvl;
            } else if (x < abc) {
                u |= 1u << lvl;
            } else {
                u |= 1u << lvl;
                v |= 1u << lvl;
            }
        }
        eu[e] = (int32_t)u;
        ev[e] = (int32_t)v;
    }
    gg_graph *g = gg_from_edges(n, ne, eu, ev);
    free(eu);
    free(ev);
    return g;
}

/*
 * W x W grid, vertex (i, j) has id i*W + j; every horizontal and vertical
 * neighbour pair is an edge (2 W (W-1) edges).  On top, `ndiag` distinct
 * diagonals drawn uniformly without replacement from the 2 (W-1)^2
 * candidates (i,j)-(i+1,j+1) and (i,j+1)-(i+1,j).
 */
gg_graph *gg_grid_diag(int32_t W, int64_t ndiag, uint64_t seed)
{
    if (W < 1) return NULL;
    int64_t n64 = (int64_t)W * W;
    if (n64 > INT32_MAX) return NULL;
    int64_t cells = (int64_t)(W - 1) * (W - 1);
    if (ndiag < 0 || ndiag > 2 * cells) return NULL;
    int64_t ne = 2 * (int64_t)W * (W - 1) + ndiag;
    int32_t *eu = (int32_t *)malloc(sizeof(int32_t) * (size_t)(ne ? ne : 1));
    int32_t *ev = (int32_t *)malloc(sizeof(int32_t) * (size_t)(ne ? ne : 1));
    uint8_t *taken = (uint8_t *)calloc((size_t)(2 * cells / 8 + 1), 1);
    if (!eu || !ev || !taken) {
        free(eu);
        free(ev);
        free(taken);
        return NULL;
    }
    int64_t k = 0;
    for (int32_t i = 0; i < W; ++i)
        for (int32_t j = 0; j < W; ++j) {
            int32_t id = i * W + j;
            if (j + 1 < W) {
                eu[k] = id;
                ev[k] = id + 1;
                ++k;
            }
            if (i + 1 < W) {
                eu[k] = id;
                ev[k] = id + W;
                ++k;
            }
        }
    gg_rng r = {seed};
    int64_t got = 0;
    while (got < ndiag) {
        uint64_t cand = gg_below(&r, (uint64_t)(2 * cells));
        if (taken[cand >> 3] & (1u << (cand & 7))) continue;
        taken[cand >> 3] |= (uint8_t)(1u << (cand & 7));
        int64_t t = (int64_t)cand / cells, rem = (int64_t)cand % cells;
        int32_t i = (int32_t)(rem / (W - 1)), jj = (int32_t)(rem % (W - 1));
        if (t == 0) {
            eu[k] = i * W + jj;
            ev[k] = (i + 1) * W + jj + 1;
        } else {
            eu[k] = i * W + jj + 1;
            ev[k] = (i + 1) * W + jj;
        }
        ++k;
        ++got;
    }
    free(taken);
    gg_graph *g = gg_from_edges((int32_t)n64, ne, eu, ev);
    free(eu);
    free(ev);
    return g;
}

/*
 * nx x ny x nz box of a 3D lattice, vertex (x, y, z) has id (z ny + y) nx + x
 * (natural order); every pair of distinct vertices whose coordinates differ by
 * at most 1 in each axis is an edge (the 27-point stencil: 26 neighbours
 * inside the box).  Edges are emitted for the 13 offsets that come after
 * (0, 0, 0) in (dz, dy, dx) order.
 */
gg_graph *gg_stencil27(int32_t nx, int32_t ny, int32_t nz)
{
    if (nx < 1 || ny < 1 || nz < 1) return NULL;
    int64_t n64 = (int64_t)nx * ny * nz;
    if (n64 > INT32_MAX) return NULL;
    int64_t ne = 0;
    for (int dz = 0; dz <= 1; ++dz)
        for (int dy = -1; dy <= 1; ++dy)
            for (int dx = -1; dx <= 1; ++dx) {
                if (dz == 0 && (dy < 0 || (dy == 0 && dx <= 0))) continue;
                ne += (int64_t)(nx - (dx ? 1 : 0)) * (ny - (dy ? 1 : 0)) * (nz - dz);
            }
    int32_t *eu = (int32_t *)malloc(sizeof(int32_t) * (size_t)(ne ? ne : 1));
    int32_t *ev = (int32_t *)malloc(sizeof(int32_t) * (size_t)(ne ? ne : 1));
    if (!eu || !ev) {
        free(eu);
        free(ev);
        return NULL;
    }
    int64_t k = 0;
    for (int32_t z = 0; z < nz; ++z)
        for (int32_t y = 0; y < ny; ++y)
            for (int32_t x = 0; x < nx; ++x) {
                const int32_t id = (int32_t)(((int64_t)z * ny + y) * nx + x);
                for (int dz = 0; dz <= 1; ++dz)
                    for (int dy = -1; dy <= 1; ++dy)
                        for (int dx = -1; dx <= 1; ++dx) {
                            if (dz == 0 && (dy < 0 || (dy == 0 && dx <= 0))) continue;
                            const int32_t x2 = x + dx, y2 = y + dy, z2 = z + dz;
                            if (x2 < 0 || x2 >= nx || y2 < 0 || y2 >= ny || z2 >= nz) continue;
                            eu[k] = id;
                            ev[k] = (int32_t)(((int64_t)z2 * ny + y2) * nx + x2);
                            ++k;
                        }
            }
    gg_graph *g = k == ne ? gg_from_edges((int32_t)n64, ne, eu, ev) : NULL;
    free(eu);
    free(ev);
    return g;
}

typedef struct {
    int64_t cell;
    int32_t idx;
} gg_pt;

static int gg_pt_cmp(const void *x, const void *y)
{
    const gg_pt *p = (const gg_pt *)x, *q = (const gg_pt *)y;
    if (p->cell != q->cell) return p->cell < q->cell ? -1 : 1;
    return p->idx < q->idx ? -1 : (p->idx > q->idx);
}

/*
 * Random geometric graph: n points uniform in [0,1)^2, an edge between every
 * pair at Euclidean distance <= r.  Vertex ids follow cell order: the square
 * is cut into k x k cells (k = floor(1/r), so a cell is at least r wide) and
 * points are numbered cell by cell, row-major over cells, ties by draw order.
 */
gg_graph *gg_rgg(int32_t n, double rad, uint64_t seed)
{
    if (n < 0 || !(rad > 0.0)) return NULL;
    double *x = (double *)malloc(sizeof(double) * (size_t)(n ? n : 1));
    double *y = (double *)malloc(sizeof(double) * (size_t)(n ? n : 1));
    gg_pt *pts = (gg_pt *)malloc(sizeof(gg_pt) * (size_t)(n ? n : 1));
    int64_t k = (int64_t)floor(1.0 / rad);
    if (k < 1) k = 1;
    if (k > 46340) k = 46340;
    int64_t *cstart = (int64_t *)calloc((size_t)(k * k + 1), sizeof(int64_t));
    if (!x || !y || !pts || !cstart) {
        free(x);
        free(y);
        free(pts);
        free(cstart);
        return NULL;
    }
    gg_rng r = {seed};
    for (int32_t i = 0; i < n; ++i) {
        x[i] = gg_unif(&r);
        y[i] = gg_unif(&r);
        int64_t cx = (int64_t)(x[i] * (double)k), cy = (int64_t)(y[i] * (double)k);
        if (cx >= k) cx = k - 1;
        if (cy >= k) cy = k - 1;
        pts[i].cell = cy * k + cx;
        pts[i].idx = i;
    }
    qsort(pts, (size_t)n, sizeof(gg_pt), gg_pt_cmp);
    /* relabel: new id i holds point pts[i].idx */
    double *nx = (double *)malloc(sizeof(double) * (size_t)(n ? n : 1));
    double *ny = (double *)malloc(sizeof(double) * (size_t)(n ? n : 1));
    if (!nx || !ny) {
        free(x);
        free(y);
        free(pts);
        free(cstart);
        free(nx);
        free(ny);
        return NULL;
    }
    for (int32_t i = 0; i < n; ++i) {
        nx[i] = x[pts[i].idx];
        ny[i] = y[pts[i].idx];
        cstart[pts[i].cell + 1]++;
    }
    for (int64_t c = 0; c < k * k; ++c) cstart[c + 1] += cstart[c];
    free(x);
    free(y);
    int64_t cap = (int64_t)n * 8 + 16, ne = 0;
    int32_t *eu = (int32_t *)malloc(sizeof(int32_t) * (size_t)cap);
    int32_t *ev = (int32_t *)malloc(sizeof(int32_t) * (size_t)cap);
    const double r2 = rad * rad;
    for (int32_t i = 0; i < n && eu && ev; ++i) {
        int64_t c = pts[i].cell, cx = c % k, cy = c / k;
        for (int64_t dy = -1; dy <= 1; ++dy)
            for (int64_t dx = -1; dx <= 1; ++dx) {
                int64_t ux = cx + dx, uy = cy + dy;
                if (ux < 0 || uy < 0 || ux >= k || uy >= k) continue;
                int64_t cc = uy * k + ux;
                for (int64_t j = cstart[cc]; j < cstart[cc + 1]; ++j) {
                    if (j <= i) continue;
                    double ddx = nx[i] - nx[j], ddy = ny[i] - ny[j];
                    double d2 = ddx * ddx + ddy * ddy;
                    if (d2 > r2) continue;
                    if (ne == cap) {
                        cap *= 2;
                        int32_t *a2 = (int32_t *)realloc(eu, sizeof(int32_t) * (size_t)cap);
                        int32_t *b2 = (int32_t *)realloc(ev, sizeof(int32_t) * (size_t)cap);
                        if (!a2 || !b2) {
                            free(a2 ? a2 : eu);
                            free(b2 ? b2 : ev);
                            eu = ev = NULL;
                            goto out;
                        }
                        eu = a2;
                        ev = b2;
                    }
                    eu[ne] = i;
                    ev[ne] = (int32_t)j;
                    ++ne;
                }
            }
    }
out:;
    gg_graph *g = NULL;
    if (eu && ev) g = gg_from_edges(n, ne, eu, ev);
    free(eu);
    free(ev);
    free(nx);
    free(ny);
    free(pts);
    free(cstart);
    return g;
}

/* Uniform random relabelling (Fisher-Yates): vertex v becomes perm[v]. */
gg_graph *gg_permute(const gg_graph *g, uint64_t seed)
{
    int32_t n = g->n;
    int32_t *perm = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n ? n : 1));
    int64_t ne = g->arcs / 2;
    int32_t *eu = (int32_t *)malloc(sizeof(int32_t) * (size_t)(ne ? ne : 1));
    int32_t *ev = (int32_t *)malloc(sizeof(int32_t) * (size_t)(ne ? ne : 1));
    if (!perm || !eu || !ev) {
        free(perm);
        free(eu);
        free(ev);
        return NULL;
    }
    for (int32_t i = 0; i < n; ++i) perm[i] = i;
    gg_rng r = {seed};
    for (int32_t i = n - 1; i > 0; --i) {
        int32_t j = (int32_t)gg_below(&r, (uint64_t)i + 1);
        int32_t t = perm[i];
        perm[i] = perm[j];
        perm[j] = t;
    }
    int64_t k = 0;
    for (int32_t u = 0; u < n; ++u)
        for (int32_t p = g->row_ptr[u]; p < g->row_ptr[u + 1]; ++p) {
            int32_t v = g->col_idx[p];
            if (u < v) {
                eu[k] = perm[u];
                ev[k] = perm[v];
                ++k;
            }
        }
    gg_graph *out = gg_from_edges(n, k, eu, ev);
    free(perm);
    free(eu);
    free(ev);
    return out;
}

/* One draw of the stream: lets the host derive per-item seeds the same way. */
uint64_t gg_stream(uint64_t seed, uint64_t index)
{
    gg_rng r = {seed + index * 0x9E3779B97F4A7C15ULL};
    return gg_next(&r);
}
