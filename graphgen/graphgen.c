/*
 * Seeded synthetic graph generators (inputs only; no label-propagation or
 * modularity arithmetic lives here).
 *
 * Every generator is deterministic in its seed and independent of the number
 * of OpenMP threads: all randomness is drawn in counter mode from SplitMix64
 * (Steele, Lea & Flood 2014), keyed by the seed and the index of the item
 * being generated.  Output is an undirected graph as a symmetric CSR: every
 * undirected edge {u,v} appears as (u,v) and (v,u), self-loops are dropped,
 * duplicate edges are merged, rows are sorted by neighbour id, and the weight
 * of an edge is a hash of its unordered endpoint pair (so A is symmetric).
 *
 * Classes (stand-ins for the SuiteSparse web / social / collaboration / road
 * graphs of the paper's Table 1):
 *   gg_sbm_planted  planted-partition stochastic block model (p_in, p_out)
 *   gg_sbm_mixing   planted partition given mean degree d and mixing mu
 *   gg_rmat         R-MAT (Chakrabarti, Zhan & Faloutsos 2004) power-law graph
 *   gg_grid_road    2-D grid with deleted edges and short-range shortcuts
 *   gg_kmer_like    union of long random paths plus a few branch edges
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define GG_GAMMA 0x9E3779B97F4A7C15ULL

typedef struct {
    int32_t n;
    int64_t m;
    int32_t *offsets; /* [n+1] */
    int32_t *indices; /* [m] */
    int32_t *weights; /* [m] or NULL (unit) */
} gg_csr;

static uint64_t gg_mix(uint64_t z)
{
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

/* k-th output (k >= 1) of the SplitMix64 stream with state `key`. */
static uint64_t gg_draw(uint64_t key, uint64_t k) { return gg_mix(key + k * GG_GAMMA); }

/* uniform double in [0, 1) with 53 random bits */
static double gg_unit(uint64_t x) { return (double)(x >> 11) * (1.0 / 9007199254740992.0); }

/* Sub-stream keys, so that different uses of one seed never collide. */
static uint64_t gg_key(uint64_t seed, uint64_t purpose) { return gg_draw(gg_mix(seed), purpose); }

void gg_free(gg_csr *g)
{
    if (!g) return;
    free(g->offsets);
    free(g->indices);
    free(g->weights);
    free(g);
}

int32_t gg_n(const gg_csr *g) { return g->n; }
int64_t gg_m(const gg_csr *g) { return g->m; }
int gg_has_weights(const gg_csr *g) { return g->weights != NULL; }

void gg_copy_out(const gg_csr *g, int32_t *offsets, int32_t *indices, int32_t *weights)
{
    memcpy(offsets, g->offsets, sizeof(int32_t) * ((size_t)g->n + 1));
    memcpy(indices, g->indices, sizeof(int32_t) * (size_t)g->m);
    if (weights && g->weights) memcpy(weights, g->weights, sizeof(int32_t) * (size_t)g->m);
}

/* ------------------------------------------------------------------------- */
/* Edge-pair list -> symmetric, de-duplicated CSR                             */
/* ------------------------------------------------------------------------- */

static int cmp_i32(const void *a, const void *b)
{
    int32_t x = *(const int32_t *)a, y = *(const int32_t *)b;
    return (x > y) - (x < y);
}

static void sort_row(int32_t *r, int64_t len)
{
    if (len <= 24) {
        for (int64_t i = 1; i < len; ++i) {
            int32_t x = r[i];
            int64_t j = i - 1;
            while (j >= 0 && r[j] > x) {
                r[j + 1] = r[j];
                --j;
            }
            r[j + 1] = x;
        }
    } else {
        qsort(r, (size_t)len, sizeof(int32_t), cmp_i32);
    }
}

/* weight of the undirected edge {u,v}: uniform in [wmin, wmax] */
static int32_t gg_pair_weight(uint64_t wkey, int32_t u, int32_t v, int32_t wmin, int32_t wmax)
{
    uint32_t a = (uint32_t)(u < v ? u : v), b = (uint32_t)(u < v ? v : u);
    uint64_t h = gg_draw(gg_draw(wkey, (uint64_t)a + 1), (uint64_t)b + 1);
    return wmin + (int32_t)(h % (uint64_t)(wmax - wmin + 1));
}

/* pairs: 2*np int32 (u0,v0,u1,v1,...).  Consumes (frees) pairs.  Weights are
 * implicit (NULL) when wmin == wmax == 1. */
static gg_csr *gg_build(int32_t n, int64_t np, int32_t *pairs, uint64_t wkey, int32_t wmin,
                        int32_t wmax)
{
    gg_csr *g = (gg_csr *)calloc(1, sizeof(gg_csr));
    int64_t *deg = (int64_t *)calloc((size_t)n + 1, sizeof(int64_t));
    int64_t *cur = (int64_t *)malloc(sizeof(int64_t) * ((size_t)n + 1));
    if (!g || !deg || !cur) goto fail;
    g->n = n;

#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < np; ++i) {
        int32_t u = pairs[2 * i], v = pairs[2 * i + 1];
        if (u == v) continue;
#pragma omp atomic
        deg[u]++;
#pragma omp atomic
        deg[v]++;
    }
    int64_t total = 0;
    for (int32_t v = 0; v < n; ++v) {
        cur[v] = total;
        total += deg[v];
    }
    cur[n] = total;
    int64_t *start = (int64_t *)malloc(sizeof(int64_t) * ((size_t)n + 1));
    int32_t *adj = (int32_t *)malloc(sizeof(int32_t) * (size_t)(total > 0 ? total : 1));
    if (!start || !adj) {
        free(start);
        free(adj);
        goto fail;
    }
    memcpy(start, cur, sizeof(int64_t) * ((size_t)n + 1));

#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < np; ++i) {
        int32_t u = pairs[2 * i], v = pairs[2 * i + 1];
        if (u == v) continue;
        int64_t pu, pv;
#pragma omp atomic capture
        pu = cur[u]++;
#pragma omp atomic capture
        pv = cur[v]++;
        adj[pu] = v;
        adj[pv] = u;
    }
    free(pairs);
    pairs = NULL;

    /* sort and de-duplicate every row in place; deg[v] = unique count */
#pragma omp parallel for schedule(dynamic, 1024)
    for (int32_t v = 0; v < n; ++v) {
        int32_t *r = adj + start[v];
        int64_t len = start[v + 1] - start[v];
        sort_row(r, len);
        int64_t k = 0;
        for (int64_t i = 0; i < len; ++i)
            if (k == 0 || r[k - 1] != r[i]) r[k++] = r[i];
        deg[v] = k;
    }
    int64_t m = 0;
    for (int32_t v = 0; v < n; ++v) m += deg[v];
    if (m >= 2147483647LL) {
        free(start);
        free(adj);
        goto fail;
    }
    g->m = m;
    g->offsets = (int32_t *)malloc(sizeof(int32_t) * ((size_t)n + 1));
    g->indices = (int32_t *)malloc(sizeof(int32_t) * (size_t)(m > 0 ? m : 1));
    int weighted = !(wmin == 1 && wmax == 1);
    if (weighted) g->weights = (int32_t *)malloc(sizeof(int32_t) * (size_t)(m > 0 ? m : 1));
    if (!g->offsets || !g->indices || (weighted && !g->weights)) {
        free(start);
        free(adj);
        goto fail;
    }
    int64_t acc = 0;
    for (int32_t v = 0; v < n; ++v) {
        g->offsets[v] = (int32_t)acc;
        acc += deg[v];
    }
    g->offsets[n] = (int32_t)acc;
#pragma omp parallel for schedule(dynamic, 1024)
    for (int32_t v = 0; v < n; ++v) {
        int64_t o = g->offsets[v];
        memcpy(g->indices + o, adj + start[v], sizeof(int32_t) * (size_t)deg[v]);
        if (weighted)
            for (int64_t i = 0; i < deg[v]; ++i)
                g->weights[o + i] = gg_pair_weight(wkey, v, g->indices[o + i], wmin, wmax);
    }
    free(start);
    free(adj);
    free(deg);
    free(cur);
    return g;
fail:
    free(pairs);
    free(deg);
    free(cur);
    gg_free(g);
    return NULL;
}

/* ------------------------------------------------------------------------- */
/* Stochastic block models                                                    */
/* ------------------------------------------------------------------------- */

/* Emit (u, v) for v in [lo, hi) with probability p each, by geometric skips
 * (Batagelj & Brandes 2005).  Returns the count; writes pairs when out != 0. */
static int64_t gg_bernoulli_run(uint64_t key, uint64_t *ctr, int32_t u, int64_t lo, int64_t hi,
                                double p, int32_t *out)
{
    if (p <= 0.0 || lo >= hi) return 0;
    int64_t cnt = 0;
    if (p >= 1.0) {
        for (int64_t v = lo; v < hi; ++v, ++cnt)
            if (out) {
                out[2 * cnt] = u;
                out[2 * cnt + 1] = (int32_t)v;
            }
        return cnt;
    }
    double lq = log1p(-p);
    int64_t v = lo - 1;
    for (;;) {
        double r = gg_unit(gg_draw(key, ++*ctr));
        double skip = floor(log1p(-r) / lq);
        if (skip >= (double)(hi - v)) break;
        v += 1 + (int64_t)skip;
        if (v >= hi) break;
        if (out) {
            out[2 * cnt] = u;
            out[2 * cnt + 1] = (int32_t)v;
        }
        ++cnt;
    }
    return cnt;
}

/* block b holds vertices [b*n/k, (b+1)*n/k) */
static int64_t gg_block_end(int32_t n, int32_t k, int32_t u)
{
    int64_t b = ((int64_t)u * k + k - 1) / n; /* candidate */
    while (b > 0 && (b * n) / k > u) --b;
    while (((b + 1) * n) / k <= u) ++b;
    return ((b + 1) * n) / k;
}

gg_csr *gg_sbm_planted(int32_t n, int32_t k, double p_in, double p_out, uint64_t seed,
                       int32_t wmin, int32_t wmax)
{
    if (n < 0 || k < 1 || k > (n > 0 ? n : 1) || wmin < 1 || wmax < wmin) return NULL;
    uint64_t key = gg_key(seed, 1);
    int64_t *cnt = (int64_t *)calloc((size_t)n + 1, sizeof(int64_t));
    if (!cnt) return NULL;
#pragma omp parallel for schedule(dynamic, 256)
    for (int32_t u = 0; u < n; ++u) {
        uint64_t rk = gg_draw(key, (uint64_t)u + 1), ctr = 0;
        int64_t be = gg_block_end(n, k, u);
        cnt[u] = gg_bernoulli_run(rk, &ctr, u, u + 1, be, p_in, NULL) +
                 gg_bernoulli_run(rk, &ctr, u, be, n, p_out, NULL);
    }
    int64_t total = 0;
    for (int32_t u = 0; u < n; ++u) {
        int64_t c = cnt[u];
        cnt[u] = total;
        total += c;
    }
    int32_t *pairs = (int32_t *)malloc(sizeof(int32_t) * 2 * (size_t)(total > 0 ? total : 1));
    if (!pairs) {
        free(cnt);
        return NULL;
    }
#pragma omp parallel for schedule(dynamic, 256)
    for (int32_t u = 0; u < n; ++u) {
        uint64_t rk = gg_draw(key, (uint64_t)u + 1), ctr = 0;
        int64_t be = gg_block_end(n, k, u);
        int64_t c = gg_bernoulli_run(rk, &ctr, u, u + 1, be, p_in, pairs + 2 * cnt[u]);
        gg_bernoulli_run(rk, &ctr, u, be, n, p_out, pairs + 2 * (cnt[u] + c));
    }
    free(cnt);
    return gg_build(n, total, pairs, gg_key(seed, 2), wmin, wmax);
}

/* planted partition with expected degree d, of which a fraction mu leaves the
 * block: p_in = d(1-mu)/(s-1), p_out = d mu/(n-s), s = n/k */
gg_csr *gg_sbm_mixing(int32_t n, int32_t k, double d, double mu, uint64_t seed, int32_t wmin,
                      int32_t wmax)
{
    if (n < 2 || k < 1 || k > n) return NULL;
    double s = (double)n / k;
    double p_in = s > 1.0 ? d * (1.0 - mu) / (s - 1.0) : 0.0;
    double p_out = (double)n - s > 0.0 ? d * mu / ((double)n - s) : 0.0;
    return gg_sbm_planted(n, k, p_in, p_out, seed, wmin, wmax);
}

/* ------------------------------------------------------------------------- */
/* R-MAT                                                                      */
/* ------------------------------------------------------------------------- */

/* 2^scale vertices, edge_factor * 2^scale generated edges, quadrant
 * probabilities a, b, c (d = 1 - a - b - c), no noise.  Symmetrised, self-loops
 * and duplicates removed.  permute != 0 relabels the vertices by a seeded
 * random permutation (Fisher-Yates). */
gg_csr *gg_rmat(int32_t scale, int32_t edge_factor, double a, double b, double c, uint64_t seed,
                int32_t wmin, int32_t wmax, int permute)
{
    if (scale < 1 || scale > 30 || edge_factor < 1 || wmin < 1 || wmax < wmin) return NULL;
    int32_t n = (int32_t)(1u << scale);
    int64_t ne = (int64_t)edge_factor << scale;
    int32_t *pairs = (int32_t *)malloc(sizeof(int32_t) * 2 * (size_t)ne);
    int32_t *perm = NULL;
    if (!pairs) return NULL;
    uint64_t key = gg_key(seed, 3);
    double ab = a + b, abc = a + b + c;
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < ne; ++i) {
        uint64_t ek = gg_draw(key, (uint64_t)i + 1);
        uint32_t u = 0, v = 0;
        for (int32_t lvl = 0; lvl < scale; ++lvl) {
            double r = gg_unit(gg_draw(ek, (uint64_t)lvl + 1));
            uint32_t bu = r >= ab, bv = (r >= a && r < ab) || r >= abc;
            u = (u << 1) | bu;
            v = (v << 1) | bv;
        }
        pairs[2 * i] = (int32_t)u;
        pairs[2 * i + 1] = (int32_t)v;
    }
    if (permute) {
        perm = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
        if (!perm) {
            free(pairs);
            return NULL;
        }
        for (int32_t i = 0; i < n; ++i) perm[i] = i;
        uint64_t pk = gg_key(seed, 4);
        for (int32_t i = n - 1; i > 0; --i) {
            int32_t j = (int32_t)(gg_draw(pk, (uint64_t)i) % (uint64_t)(i + 1));
            int32_t t = perm[i];
            perm[i] = perm[j];
            perm[j] = t;
        }
#pragma omp parallel for schedule(static)
        for (int64_t i = 0; i < 2 * ne; ++i) pairs[i] = perm[pairs[i]];
        free(perm);
    }
    return gg_build(n, ne, pairs, gg_key(seed, 5), wmin, wmax);
}

/* ------------------------------------------------------------------------- */
/* Road-like grid                                                             */
/* ------------------------------------------------------------------------- */

/* side x side 4-neighbour grid (vertex r*side+c); each grid edge deleted with
 * probability delete_frac; round(shortcut_frac * n) shortcuts from a random
 * vertex to a random vertex within Chebyshev distance `radius` that is not the
 * vertex itself nor a grid neighbour. */
gg_csr *gg_grid_road(int32_t side, double delete_frac, double shortcut_frac, int32_t radius,
                     uint64_t seed, int32_t wmin, int32_t wmax)
{
    if (side < 2 || (int64_t)side * side >= 2147483647LL || radius < 1 || wmin < 1 ||
        wmax < wmin)
        return NULL;
    int32_t n = side * side;
    int64_t ngrid = 2LL * side * (side - 1);
    int64_t nshort = (int64_t)llround(shortcut_frac * (double)n);
    uint64_t dkey = gg_key(seed, 6), skey = gg_key(seed, 7);
    uint64_t thresh = (uint64_t)(delete_frac * 18446744073709551616.0);
    if (delete_frac >= 1.0) thresh = UINT64_MAX;
    int32_t *pairs = (int32_t *)malloc(sizeof(int32_t) * 2 * (size_t)(ngrid + nshort));
    if (!pairs) return NULL;
    /* grid edges: kept ones get their pair, deleted ones a self-loop (dropped later) */
#pragma omp parallel for schedule(static)
    for (int64_t id = 0; id < ngrid; ++id) {
        int32_t u, v;
        int64_t half = (int64_t)side * (side - 1);
        if (id < half) { /* horizontal: (r,c)-(r,c+1) */
            int32_t r = (int32_t)(id / (side - 1)), c = (int32_t)(id % (side - 1));
            u = r * side + c;
            v = u + 1;
        } else { /* vertical: (r,c)-(r+1,c) */
            int64_t j = id - half;
            u = (int32_t)j;
            v = u + side;
        }
        int del = gg_draw(dkey, (uint64_t)id + 1) < thresh;
        pairs[2 * id] = u;
        pairs[2 * id + 1] = del ? u : v;
    }
    int32_t span = 2 * radius + 1;
#pragma omp parallel for schedule(static)
    for (int64_t j = 0; j < nshort; ++j) {
        uint64_t jk = gg_draw(skey, (uint64_t)j + 1);
        int32_t u = 0, v = 0;
        for (uint64_t k = 1;; k += 2) {
            u = (int32_t)(gg_draw(jk, k) % (uint64_t)n);
            uint64_t o = gg_draw(jk, k + 1);
            int32_t dr = (int32_t)(o % (uint64_t)span) - radius;
            int32_t dc = (int32_t)((o >> 32) % (uint64_t)span) - radius;
            int32_t r = u / side + dr, c = u % side + dc;
            if (abs(dr) + abs(dc) <= 1 || r < 0 || r >= side || c < 0 || c >= side) continue;
            v = r * side + c;
            break;
        }
        pairs[2 * (ngrid + j)] = u;
        pairs[2 * (ngrid + j) + 1] = v;
    }
    return gg_build(n, ngrid + nshort, pairs, gg_key(seed, 8), wmin, wmax);
}

/* ------------------------------------------------------------------------- */
/* k-mer-like chains                                                          */
/* ------------------------------------------------------------------------- */

/* A random order of the n vertices cut into paths (a cut after each position
 * with probability 1/mean_path), plus round(branch_frac * n) branch edges from
 * a random vertex to a vertex at most 64 positions away in that order. */
gg_csr *gg_kmer_like(int32_t n, int32_t mean_path, double branch_frac, uint64_t seed)
{
    if (n < 2 || mean_path < 1) return NULL;
    int32_t *perm = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
    int64_t nb = (int64_t)llround(branch_frac * (double)n);
    int32_t *pairs = (int32_t *)malloc(sizeof(int32_t) * 2 * (size_t)((n - 1) + nb));
    if (!perm || !pairs) {
        free(perm);
        free(pairs);
        return NULL;
    }
    for (int32_t i = 0; i < n; ++i) perm[i] = i;
    uint64_t pk = gg_key(seed, 9), ck = gg_key(seed, 10), bk = gg_key(seed, 11);
    for (int32_t i = n - 1; i > 0; --i) {
        int32_t j = (int32_t)(gg_draw(pk, (uint64_t)i) % (uint64_t)(i + 1));
        int32_t t = perm[i];
        perm[i] = perm[j];
        perm[j] = t;
    }
    uint64_t cut = (uint64_t)(18446744073709551616.0 / mean_path);
#pragma omp parallel for schedule(static)
    for (int32_t i = 0; i < n - 1; ++i) {
        int c = gg_draw(ck, (uint64_t)i + 1) < cut;
        pairs[2 * (int64_t)i] = perm[i];
        pairs[2 * (int64_t)i + 1] = c ? perm[i] : perm[i + 1];
    }
#pragma omp parallel for schedule(static)
    for (int64_t j = 0; j < nb; ++j) {
        uint64_t h = gg_draw(bk, (uint64_t)j + 1);
        int32_t i = (int32_t)(h % (uint64_t)n);
        int32_t off = 2 + (int32_t)((h >> 40) % 63);
        int32_t k = i + off < n ? i + off : i - off;
        if (k < 0) k = 0;
        pairs[2 * ((int64_t)(n - 1) + j)] = perm[i];
        pairs[2 * ((int64_t)(n - 1) + j) + 1] = perm[k];
    }
    free(perm);
    return gg_build(n, (n - 1) + nb, pairs, gg_key(seed, 12), 1, 1);
}

int gg_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
