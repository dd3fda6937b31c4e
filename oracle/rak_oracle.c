/*
 * Oracle for RAK label propagation and Newman-Girvan modularity.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is a plain, single-threaded, slow CPU
 * restatement of what the paper's method computes.  Only the test suite, the
 * package smoke check and the CPU-baseline leg of the benchmark may load it.
 * The CUDA library never includes, links or calls anything here, and nothing
 * here is shared with it.
 *
 * Paper: S. Sahu, "Selecting a suitable Parallel Label-propagation based
 * algorithm for Disjoint Community Detection" (arXiv 2301.09125).
 *
 *   RAK (Sec. 3.2): every vertex starts with a unique label; at every step each
 *   vertex adopts the label with the most interconnecting edge weight among its
 *   neighbours.  Ties between maximum-weight labels are broken either by taking
 *   the first of them ("strict") or a random one ("non-strict").  The run has
 *   converged when at least (100 - n)% of the vertices kept their label during
 *   a step, where n is the tolerance.
 *   Asynchronous update (Sec. 3.3, stated for COPRA): a vertex may see labels
 *   its neighbours took earlier in the same iteration.
 *   Modularity (Sec. 1): Newman-Girvan quality of a disjoint partition.
 *
 * Readings where the paper is silent (each one is also listed in the design
 * notes of the repository):
 *   - "first" (strict) = the label whose first occurrence in the vertex's
 *     adjacency list (CSR order) is earliest.
 *   - "random" (non-strict) = among the maximum-weight labels, the one with the
 *     smallest 64-bit counter-based hash of (seed, iteration, vertex, label);
 *     equal hashes fall back to the strict rule.  The hash is SplitMix64's
 *     output function (Steele, Lea & Flood, "Fast splittable pseudorandom
 *     number generators", OOPSLA 2014) applied in counter mode.
 *   - a vertex without edges keeps its label and never counts as changed, but
 *     it is counted in N for the convergence test.
 *   - converged iff changed <= tolerance * N, evaluated in double; the
 *     iteration that meets the test is counted.
 *   - synchronous = every vertex reads the labels of the previous iteration
 *     (double buffer).
 *   - asynchronous = in place, in W waves: wave(v) = v mod W, waves run in
 *     order 0..W-1 and a wave's new labels are stored once the whole wave has
 *     chosen, so a vertex sees this iteration's labels of neighbours in earlier
 *     waves and the previous iteration's labels of the others.  W >= n (the
 *     default, W = 0) puts every vertex in its own wave: plain in-place
 *     updates in ascending vertex order.  W = 1 is the synchronous rule.
 *   - the CSR is taken as given: a stored entry (v,u,w) is A_vu = w, a stored
 *     self-loop counts the vertex's own current label, duplicate entries add.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------------- */
/* SplitMix64 output function (Steele et al. 2014): the 64-bit finaliser     */
/* applied to state + k * golden-gamma.                                       */
/* ------------------------------------------------------------------------- */
#define ORACLE_GOLDEN_GAMMA 0x9E3779B97F4A7C15ULL

uint64_t oracle_mix64(uint64_t z)
{
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

/* Counter-mode draw: the k-th (k >= 1) output of a SplitMix64 stream whose
 * state starts at `key`. */
static uint64_t oracle_draw(uint64_t key, uint64_t k)
{
    return oracle_mix64(key + k * ORACLE_GOLDEN_GAMMA);
}

/* Non-strict tie key of `label` at vertex v in global iteration t.
 * Three nested counter-mode draws: stream(seed) -> t -> v -> label. */
uint64_t oracle_tie_hash(uint64_t seed, int64_t t, int64_t v, int64_t label)
{
    uint64_t k_t = oracle_draw(seed, (uint64_t)t + 1);
    uint64_t k_tv = oracle_draw(k_t, (uint64_t)v + 1);
    return oracle_draw(k_tv, (uint64_t)label + 1);
}

/* ------------------------------------------------------------------------- */
/* One RAK step for one vertex (Sec. 3.2).                                    */
/* ------------------------------------------------------------------------- */

/* Scratch for the insertion-ordered label -> (weight, first position) map. */
typedef struct {
    int32_t *slot_of; /* [n] label -> index into the lists below, -1 if absent */
    int32_t *label;   /* [max_deg] labels in order of first appearance */
    int64_t *weight;  /* [max_deg] summed edge weight per label */
    int32_t *first;   /* [max_deg] first position in the adjacency list */
} oracle_map;

static int oracle_map_init(oracle_map *m, int32_t n, int64_t max_deg)
{
    m->slot_of = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
    m->label = (int32_t *)malloc(sizeof(int32_t) * (size_t)(max_deg > 0 ? max_deg : 1));
    m->weight = (int64_t *)malloc(sizeof(int64_t) * (size_t)(max_deg > 0 ? max_deg : 1));
    m->first = (int32_t *)malloc(sizeof(int32_t) * (size_t)(max_deg > 0 ? max_deg : 1));
    if (!m->slot_of || !m->label || !m->weight || !m->first) return -1;
    for (int32_t i = 0; i < n; ++i) m->slot_of[i] = -1;
    return 0;
}

static void oracle_map_free(oracle_map *m)
{
    free(m->slot_of);
    free(m->label);
    free(m->weight);
    free(m->first);
}

/* The label vertex v adopts when it reads `cur` (Sec. 3.2):
 *   1. sum, per neighbour label, the weights of the edges leading to it;
 *   2. take the largest summed weight;
 *   3. among the labels that reach it, strict picks the first one seen in the
 *      adjacency list, non-strict the one with the smallest tie hash.
 * A vertex without edges keeps cur[v]. */
static int32_t oracle_choose_with(oracle_map *m, int32_t v, const int32_t *offsets,
                                  const int32_t *indices, const int32_t *weights,
                                  const int32_t *cur, int strict, uint64_t seed, int64_t t)
{
    int32_t begin = offsets[v], end = offsets[v + 1];
    if (begin == end) return cur[v];

    /* step 1: accumulate */
    int32_t count = 0;
    for (int32_t e = begin; e < end; ++e) {
        int32_t l = cur[indices[e]];
        int64_t w = weights ? (int64_t)weights[e] : 1;
        int32_t s = m->slot_of[l];
        if (s < 0) {
            s = count++;
            m->slot_of[l] = s;
            m->label[s] = l;
            m->weight[s] = 0;
            m->first[s] = e - begin;
        }
        m->weight[s] += w;
    }

    /* step 2: maximum weight */
    int64_t wmax = m->weight[0];
    for (int32_t s = 1; s < count; ++s)
        if (m->weight[s] > wmax) wmax = m->weight[s];

    /* step 3: tie rule.  Slots are in order of first appearance, so the first
     * maximum-weight slot is the strict choice. */
    int32_t best = -1;
    uint64_t best_hash = 0;
    for (int32_t s = 0; s < count; ++s) {
        if (m->weight[s] != wmax) continue;
        if (strict) {
            best = s;
            break;
        }
        uint64_t h = oracle_tie_hash(seed, t, v, m->label[s]);
        if (best < 0 || h < best_hash) { /* equal hash: keep the earlier slot */
            best = s;
            best_hash = h;
        }
    }
    int32_t chosen = m->label[best];

    for (int32_t s = 0; s < count; ++s) m->slot_of[m->label[s]] = -1;
    return chosen;
}

static int64_t oracle_max_degree(int32_t n, const int32_t *offsets)
{
    int64_t d = 0;
    for (int32_t v = 0; v < n; ++v)
        if (offsets[v + 1] - offsets[v] > d) d = offsets[v + 1] - offsets[v];
    return d;
}

/* The label each vertex in verts[0..count) adopts when reading `cur` in global
 * iteration t.  Used to check single outputs of a sweep at sizes where a whole
 * oracle run would be too slow.  Returns 0, or -1 on allocation failure. */
int oracle_choose_many(int32_t n, const int32_t *offsets, const int32_t *indices,
                       const int32_t *weights, const int32_t *cur, int strict, uint64_t seed,
                       int64_t t, int64_t count, const int32_t *verts, int32_t *out)
{
    oracle_map m;
    if (oracle_map_init(&m, n, oracle_max_degree(n, offsets)) != 0) {
        oracle_map_free(&m);
        return -1;
    }
    for (int64_t i = 0; i < count; ++i)
        out[i] = oracle_choose_with(&m, verts[i], offsets, indices, weights, cur, strict, seed, t);
    oracle_map_free(&m);
    return 0;
}

/* ------------------------------------------------------------------------- */
/* The RAK iteration (Sec. 3.2, with Sec. 3.3's asynchronous update).         */
/* ------------------------------------------------------------------------- */

/* labels: in = initial labels (NULL = unique labels, label[v] = v); out = final.
 * changed_hist[i] receives the number of vertices that changed in iteration i
 * (capacity max_iter, may be NULL).
 * iter_offset shifts the iteration index seen by the tie hash (resume).
 * waves: asynchronous wave count W (0 = every vertex its own wave).
 * Returns 0, or -1 on bad arguments / allocation failure. */
int oracle_rak(int32_t n, const int32_t *offsets, const int32_t *indices,
               const int32_t *weights, double tolerance, int32_t max_iter, int async_mode,
               int strict, uint64_t seed, int32_t iter_offset, const int32_t *init_labels,
               int32_t waves, int32_t *labels, int32_t *out_iterations, int32_t *out_converged,
               int64_t *changed_hist)
{
    if (n < 0 || max_iter < 1 || waves < 0 || !(tolerance >= 0.0 && tolerance <= 1.0)) return -1;
    int32_t w_count = (waves == 0 || waves > n) ? (n > 0 ? n : 1) : waves;
    for (int32_t v = 0; v < n; ++v) labels[v] = init_labels ? init_labels[v] : v;
    *out_iterations = 0;
    *out_converged = 0;

    oracle_map m;
    int32_t *next = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
    if (!next || oracle_map_init(&m, n, oracle_max_degree(n, offsets)) != 0) {
        free(next);
        return -1;
    }

    for (int32_t it = 0; it < max_iter; ++it) {
        int64_t t = (int64_t)it + iter_offset;
        int64_t changed = 0;
        if (async_mode) {
            /* waves in order; a wave chooses from `labels`, which already holds
             * the new labels of the earlier waves, then stores its own */
            for (int32_t k = 0; k < w_count; ++k) {
                for (int32_t v = k; v < n; v += w_count)
                    next[v] = oracle_choose_with(&m, v, offsets, indices, weights, labels, strict,
                                                 seed, t);
                for (int32_t v = k; v < n; v += w_count) {
                    if (next[v] != labels[v]) ++changed;
                    labels[v] = next[v];
                }
            }
        } else {
            /* every vertex reads the previous iteration's labels */
            for (int32_t v = 0; v < n; ++v) {
                next[v] = oracle_choose_with(&m, v, offsets, indices, weights, labels, strict,
                                             seed, t);
                if (next[v] != labels[v]) ++changed;
            }
            memcpy(labels, next, sizeof(int32_t) * (size_t)n);
        }
        if (changed_hist) changed_hist[it] = changed;
        *out_iterations = it + 1;
        if ((double)changed <= tolerance * (double)n) {
            *out_converged = 1;
            break;
        }
    }
    free(next);
    oracle_map_free(&m);
    return 0;
}

/* ------------------------------------------------------------------------- */
/* Modularity (Sec. 1; Newman & Girvan).                                      */
/* ------------------------------------------------------------------------- */

/* Q = (1/2m) sum_{v,u} [A_vu - k_v k_u / 2m] delta(c_v, c_u), where the stored
 * CSR is the matrix A (entry (v,u,w) is A_vu = w), k_v = sum_u A_vu and
 * 2m = sum_v k_v.  Grouping the double sum by community c gives
 * Q = sum_c [ L_c / 2m - (K_c / 2m)^2 ], with L_c the weight of stored entries
 * inside c and K_c the summed k_v of c's vertices.  L = sum_c L_c, K_c and 2m
 * are exact 64-bit integers and S = sum_c K_c^2 an exact 128-bit one; Q is then
 * L/2m - S/(2m)^2 in double.  Labels must lie in [0, n).  A graph without
 * edges has Q = 0.  The three exact integers are also returned (may be NULL). */
double oracle_modularity(int32_t n, const int32_t *offsets, const int32_t *indices,
                         const int32_t *weights, const int32_t *labels, int64_t *out_l,
                         int64_t *out_2m, uint64_t *out_s_hi_lo)
{
    int64_t two_m = 0, l_in = 0;
    int64_t *k_c = (int64_t *)calloc((size_t)(n > 0 ? n : 1), sizeof(int64_t));
    if (!k_c) return 0.0 / 0.0;
    for (int32_t v = 0; v < n; ++v) {
        int64_t k_v = 0;
        for (int32_t e = offsets[v]; e < offsets[v + 1]; ++e) {
            int64_t w = weights ? (int64_t)weights[e] : 1;
            k_v += w;
            if (labels[indices[e]] == labels[v]) l_in += w;
        }
        two_m += k_v;
        k_c[labels[v]] += k_v;
    }
    unsigned __int128 s = 0;
    for (int32_t c = 0; c < n; ++c) s += (unsigned __int128)((uint64_t)k_c[c]) * (uint64_t)k_c[c];
    free(k_c);
    if (out_l) *out_l = l_in;
    if (out_2m) *out_2m = two_m;
    if (out_s_hi_lo) {
        out_s_hi_lo[0] = (uint64_t)(s >> 64);
        out_s_hi_lo[1] = (uint64_t)s;
    }
    if (two_m == 0) return 0.0;
    double dm = (double)two_m;
    return (double)l_in / dm - (double)s / (dm * dm);
}

/*
 * Splitting disconnected communities (the paper does not post-process its
 * communities; it names this split as the step it leaves out, end of
 * Sec. 3.4).  Two vertices stay together when a path of edges whose two ends
 * both carry that community's label joins them.  Breadth-first search from
 * every not yet reached vertex in increasing order: each component is labelled
 * by the vertex its search started from, which is its smallest vertex (a
 * smaller one would have started an earlier search that reached it).
 * out[v] = that vertex; returns the number of components (-1 on bad input).
 */
int64_t oracle_split(int32_t n, const int32_t *offsets, const int32_t *indices,
                     const int32_t *labels, int32_t *out)
{
    if (n < 0) return -1;
    int32_t *queue = (int32_t *)malloc(((size_t)n + 1) * sizeof(int32_t));
    if (!queue) return -1;
    for (int32_t v = 0; v < n; ++v) out[v] = -1;
    int64_t components = 0;
    for (int32_t s = 0; s < n; ++s) {
        if (out[s] >= 0) continue;
        ++components;
        out[s] = s;
        int64_t head = 0, tail = 0;
        queue[tail++] = s;
        while (head < tail) {
            const int32_t v = queue[head++];
            for (int32_t e = offsets[v]; e < offsets[v + 1]; ++e) {
                const int32_t u = indices[e];
                if (labels[u] == labels[v] && out[u] < 0) {
                    out[u] = s;
                    queue[tail++] = u;
                }
            }
        }
    }
    free(queue);
    return components;
}

/* ------------------------------------------------------------------------- */
/* SLPA, the speaker-listener label propagation (Sec. 3.4).                  */
/* ------------------------------------------------------------------------- */
/*
 * Readings where Sec. 3.4 is open:
 *   - the memory holds memory_size labels; slot 0 is the vertex itself and
 *     iteration t (1 <= t < memory_size) fills slot t, so at most
 *     memory_size - 1 iterations run;
 *   - a speaker speaks from the slots its memory held before the iteration
 *     (0 .. t-1), so every listener of one iteration hears the same
 *     memories (synchronous); the slot is drawn by a counter-based SplitMix64
 *     draw of (seed ^ SLPA_SPEAK, t, listener, position of the entry in the
 *     listener's row), mapped to [0, t) by the high 32 bits times t;
 *   - the listener sums the weights of the spoken labels and takes the
 *     heaviest; strict keeps the first such label in row order, non-strict
 *     the one with the smallest RAK tie hash of (seed, t, listener, label);
 *   - a vertex without edges repeats its previous slot;
 *   - converged once at most tolerance * n vertices stored a label that
 *     differs from their previous slot;
 *   - a vertex's community is the label it stored most often, the one first
 *     stored on equal counts.
 */
#define ORACLE_SLPA_SPEAK 0x5350454Bull /* "SPEK": keeps speaker draws apart from tie hashes */

/* memory slot a speaker speaks in iteration t to listener v through the entry
 * at row position pos */
int32_t oracle_slpa_slot(uint64_t seed, int64_t t, int64_t v, int64_t pos)
{
    uint64_t h = oracle_tie_hash(seed ^ ORACLE_SLPA_SPEAK, t, v, pos);
    return (int32_t)(((h >> 32) * (uint64_t)t) >> 32);
}

/* the label listener v stores, given the labels its row's entries speak */
static int32_t oracle_listen(oracle_map *m, int32_t v, int32_t begin, int32_t end,
                             const int32_t *weights, const int32_t *spoken, int strict,
                             uint64_t seed, int64_t t)
{
    int32_t count = 0;
    for (int32_t e = begin; e < end; ++e) {
        int32_t l = spoken[e - begin];
        int64_t w = weights ? (int64_t)weights[e] : 1;
        int32_t s = m->slot_of[l];
        if (s < 0) {
            s = count++;
            m->slot_of[l] = s;
            m->label[s] = l;
            m->weight[s] = 0;
            m->first[s] = e - begin;
        }
        m->weight[s] += w;
    }
    int64_t wmax = m->weight[0];
    for (int32_t s = 1; s < count; ++s)
        if (m->weight[s] > wmax) wmax = m->weight[s];
    int32_t best = -1;
    uint64_t best_hash = 0;
    for (int32_t s = 0; s < count; ++s) {
        if (m->weight[s] != wmax) continue;
        if (strict) {
            best = s;
            break;
        }
        uint64_t h = oracle_tie_hash(seed, t, v, m->label[s]);
        if (best < 0 || h < best_hash) {
            best = s;
            best_hash = h;
        }
    }
    int32_t chosen = m->label[best];
    for (int32_t s = 0; s < count; ++s) m->slot_of[m->label[s]] = -1;
    return chosen;
}

/* SLPA on an n-vertex CSR.  memory (may be NULL): memory_size * n ints, slot
 * t of vertex v at memory[t * n + v], filled for slots 0 .. *iterations.
 * labels: the community of every vertex.  changed_hist (may be NULL,
 * capacity memory_size - 1): vertices whose stored label differs from their
 * previous slot, per iteration.  Returns 0, or -1 on bad input or allocation
 * failure. */
int oracle_slpa(int32_t n, const int32_t *offsets, const int32_t *indices, const int32_t *weights,
                int32_t memory_size, double tolerance, int strict, uint64_t seed,
                int32_t *memory, int32_t *labels, int32_t *iterations, int32_t *converged,
                int64_t *changed_hist)
{
    if (n < 0 || memory_size < 1) return -1;
    int32_t *mem = memory ? memory : (int32_t *)malloc((size_t)memory_size * (n > 0 ? n : 1) *
                                                       sizeof(int32_t));
    int64_t dmax = oracle_max_degree(n, offsets);
    int32_t *spoken = (int32_t *)malloc((size_t)(dmax > 0 ? dmax : 1) * sizeof(int32_t));
    oracle_map m;
    int rc = 0;
    if (!mem || !spoken) {
        rc = -1;
        goto done_alloc;
    }
    if (oracle_map_init(&m, n, dmax) != 0) {
        oracle_map_free(&m);
        rc = -1;
        goto done_alloc;
    }
    for (int32_t v = 0; v < n; ++v) mem[v] = v;
    *iterations = 0;
    *converged = 0;
    for (int32_t t = 1; t < memory_size; ++t) {
        const int32_t *prev = mem + (size_t)(t - 1) * n;
        int32_t *next = mem + (size_t)t * n;
        int64_t changed = 0;
        for (int32_t v = 0; v < n; ++v) {
            int32_t begin = offsets[v], end = offsets[v + 1];
            if (begin == end) {
                next[v] = prev[v];
                continue;
            }
            for (int32_t e = begin; e < end; ++e) {
                int32_t u = indices[e];
                int32_t slot = oracle_slpa_slot(seed, t, v, e - begin);
                spoken[e - begin] = mem[(size_t)slot * n + u];
            }
            next[v] = oracle_listen(&m, v, begin, end, weights, spoken, strict, seed, t);
            if (next[v] != prev[v]) ++changed;
        }
        if (changed_hist) changed_hist[t - 1] = changed;
        *iterations = t;
        if ((double)changed <= tolerance * (double)n) {
            *converged = 1;
            break;
        }
    }
    /* community: the label stored most often, the first stored on equal counts */
    for (int32_t v = 0; v < n; ++v) {
        int32_t best = mem[v], best_count = 0;
        for (int32_t a = 0; a <= *iterations; ++a) {
            int32_t l = mem[(size_t)a * n + v], c = 0, seen_before = 0;
            for (int32_t b = 0; b < a; ++b)
                if (mem[(size_t)b * n + v] == l) seen_before = 1;
            if (seen_before) continue;
            for (int32_t b = a; b <= *iterations; ++b)
                if (mem[(size_t)b * n + v] == l) ++c;
            if (c > best_count) {
                best = l;
                best_count = c;
            }
        }
        labels[v] = best;
    }
    oracle_map_free(&m);
done_alloc:
    free(spoken);
    if (!memory) free(mem);
    return rc;
}

/* ------------------------------------------------------------------------- */
/* COPRA, community overlap propagation (Sec. 3.3).                          */
/* ------------------------------------------------------------------------- */
/*
 * Readings where Sec. 3.3 is open:
 *   - a vertex holds a set of at most max_labels (label, belonging) pairs; the
 *     belongings are integers in units of 2^-16 that sum to exactly
 *     ORACLE_COPRA_ONE = 2^16 (the paper's real coefficients that sum to 1,
 *     in fixed point so that every comparison is exact); the set is stored in
 *     decreasing belonging, equal belongings by first appearance in the scan
 *     that produced it, and its first label is the vertex's best label;
 *   - every vertex starts as its own community: {(v, 2^16)};
 *   - a listener v scans its row in CSR order and, for each neighbour u
 *     (entry weight w), the pairs of u's set in stored order, summing
 *     T(l) += w * b; its own labels are not added (only neighbours', as the
 *     paper does); a label's first appearance is the index of its first
 *     (entry, pair) in that scan;
 *   - the threshold is 1/max_labels of the normalized belonging: label l is
 *     kept iff max_labels * T(l) >= W * 2^16, W the summed weight of the row
 *     (the sum of all T(l));
 *   - no label above the threshold: the best label alone is kept, best =
 *     largest T(l), ties by the RAK rule (strict: first appearance;
 *     non-strict: smallest tie hash of (seed, iteration, v, label), then
 *     first appearance);
 *   - the kept labels are normalized: b(l) = floor(T(l) * 2^16 / T_kept),
 *     and the rounding remainder goes to the best kept label;
 *   - a vertex without edges joins its own community: {(v, 2^16)};
 *   - changed = vertices whose best label differs from the previous
 *     iteration's; converged iff changed <= tolerance * n (the paper's RAK
 *     style test, which it prefers over the original one);
 *   - synchronous and wave-ordered asynchronous updates as for RAK;
 *   - the result is every vertex's best label (disjoint communities).
 */
#define ORACLE_COPRA_ONE 65536u

typedef struct {
    int32_t *slot_of; /* [n] label -> index into the lists below, -1 if absent */
    int32_t *label;   /* [max_deg * L] labels in order of first appearance */
    uint64_t *t;      /* summed w * b */
    int64_t *first;   /* first appearance index */
} oracle_cmap;

/* keep 1 when candidate slot a comes before slot b as the best label */
static int oracle_copra_better(const oracle_cmap *m, int32_t a, int32_t b, int strict,
                               uint64_t seed, int64_t t_iter, int32_t v)
{
    if (m->t[a] != m->t[b]) return m->t[a] > m->t[b];
    if (!strict) {
        uint64_t ha = oracle_tie_hash(seed, t_iter, v, m->label[a]);
        uint64_t hb = oracle_tie_hash(seed, t_iter, v, m->label[b]);
        if (ha != hb) return ha < hb;
    }
    return m->first[a] < m->first[b];
}

/* new set of listener v from the sets `src` of its neighbours (src_l / src_b:
 * n * L entries, b = 0 ends a set); writes L entries at out_l / out_b */
static void oracle_copra_listen(oracle_cmap *m, int32_t v, const int32_t *offsets,
                                const int32_t *indices, const int32_t *weights,
                                const int32_t *const *src_l, const uint32_t *const *src_b,
                                int32_t waves, int32_t k_wave, int32_t L, int strict, uint64_t seed,
                                int64_t t_iter, int32_t *out_l, uint32_t *out_b)
{
    int32_t begin = offsets[v], end = offsets[v + 1];
    for (int32_t s = 0; s < L; ++s) {
        out_l[s] = -1;
        out_b[s] = 0;
    }
    if (begin == end) { /* no labels: the vertex joins its own community */
        out_l[0] = v;
        out_b[0] = ORACLE_COPRA_ONE;
        return;
    }
    int32_t count = 0;
    int64_t k = 0;
    uint64_t W = 0;
    for (int32_t e = begin; e < end; ++e) {
        int32_t u = indices[e];
        uint64_t w = weights ? (uint64_t)weights[e] : 1u;
        W += w;
        int which = (u % waves) < k_wave ? 1 : 0; /* earlier wave: this iteration's set */
        const int32_t *ul = src_l[which] + (size_t)u * L;
        const uint32_t *ub = src_b[which] + (size_t)u * L;
        for (int32_t p = 0; p < L && ub[p] != 0; ++p, ++k) {
            int32_t l = ul[p];
            int32_t s = m->slot_of[l];
            if (s < 0) {
                s = count++;
                m->slot_of[l] = s;
                m->label[s] = l;
                m->t[s] = 0;
                m->first[s] = k;
            }
            m->t[s] += w * (uint64_t)ub[p];
        }
    }
    /* the kept labels: above the threshold, else the best alone */
    int32_t kept[64], nk = 0;
    for (int32_t s = 0; s < count; ++s)
        if ((uint64_t)L * m->t[s] >= W * (uint64_t)ORACLE_COPRA_ONE) kept[nk++] = s;
    if (nk == 0) {
        int32_t best = 0;
        for (int32_t s = 1; s < count; ++s)
            if (oracle_copra_better(m, s, best, strict, seed, t_iter, v)) best = s;
        kept[nk++] = best;
    }
    /* normalize, the remainder to the best kept label */
    uint64_t tk = 0;
    for (int32_t i = 0; i < nk; ++i) tk += m->t[kept[i]];
    uint32_t bsum = 0, bval[64];
    int32_t best_i = 0;
    for (int32_t i = 0; i < nk; ++i) {
        bval[i] = (uint32_t)((m->t[kept[i]] * (uint64_t)ORACLE_COPRA_ONE) / tk);
        bsum += bval[i];
        if (i > 0 && oracle_copra_better(m, kept[i], kept[best_i], strict, seed, t_iter, v))
            best_i = i;
    }
    bval[best_i] += ORACLE_COPRA_ONE - bsum;
    /* store by decreasing belonging, equal belongings by first appearance */
    for (int32_t i = 0; i < nk; ++i) {
        int32_t pick = -1;
        for (int32_t j = 0; j < nk; ++j) {
            if (kept[j] < 0) continue;
            if (pick < 0 || bval[j] > bval[pick] ||
                (bval[j] == bval[pick] && m->first[kept[j]] < m->first[kept[pick]]))
                pick = j;
        }
        out_l[i] = m->label[kept[pick]];
        out_b[i] = bval[pick];
        kept[pick] = -1;
    }
    for (int32_t s = 0; s < count; ++s) m->slot_of[m->label[s]] = -1;
}

/* COPRA on an n-vertex CSR (max_labels 1 .. 64; waves as in oracle_rak, 0 or
 * >= n = the plain in-place ascending order, mode 0 sync).  sets_l / sets_b
 * (n * max_labels each): the final sets, b = 0 after a set's last pair.
 * labels: the best label of every vertex.  changed_hist: capacity max_iter.
 * Returns 0, or -1 on bad input or allocation failure. */
int oracle_copra(int32_t n, const int32_t *offsets, const int32_t *indices, const int32_t *weights,
                 int32_t max_labels, double tolerance, int32_t max_iter, int mode, int32_t waves,
                 int strict, uint64_t seed, int32_t *sets_l, uint32_t *sets_b, int32_t *labels,
                 int32_t *iterations, int32_t *converged, int64_t *changed_hist)
{
    if (n < 0 || max_labels < 1 || max_labels > 64 || max_iter < 1) return -1;
    const int32_t L = max_labels;
    const size_t cells = (size_t)(n > 0 ? n : 1) * (size_t)L;
    int64_t dmax = oracle_max_degree(n, offsets);
    int32_t *buf_l[2] = {(int32_t *)malloc(cells * sizeof(int32_t)),
                         (int32_t *)malloc(cells * sizeof(int32_t))};
    uint32_t *buf_b[2] = {(uint32_t *)malloc(cells * sizeof(uint32_t)),
                          (uint32_t *)malloc(cells * sizeof(uint32_t))};
    oracle_cmap m;
    size_t lists = (size_t)(dmax > 0 ? dmax : 1) * (size_t)L;
    m.slot_of = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
    m.label = (int32_t *)malloc(sizeof(int32_t) * lists);
    m.t = (uint64_t *)malloc(sizeof(uint64_t) * lists);
    m.first = (int64_t *)malloc(sizeof(int64_t) * lists);
    int rc = 0;
    if (!buf_l[0] || !buf_l[1] || !buf_b[0] || !buf_b[1] || !m.slot_of ||
        !m.label || !m.t || !m.first) {
        rc = -1;
        goto done;
    }
    for (int32_t v = 0; v < n; ++v) {
        m.slot_of[v] = -1;
        for (int32_t s = 0; s < L; ++s) {
            buf_l[0][(size_t)v * L + s] = s == 0 ? v : -1;
            buf_b[0][(size_t)v * L + s] = s == 0 ? ORACLE_COPRA_ONE : 0;
        }
    }
    int32_t W = mode == 0 ? 1 : (waves <= 0 || waves > n ? (n > 0 ? n : 1) : waves);
    *iterations = 0;
    *converged = 0;
    int cur = 0;
    for (int32_t it = 0; it < max_iter; ++it) {
        int nxt = cur ^ 1;
        const int32_t *src_l[2] = {buf_l[cur], buf_l[nxt]};
        const uint32_t *src_b[2] = {buf_b[cur], buf_b[nxt]};
        int64_t changed = 0;
        /* wave k reads the new sets of earlier waves, the previous ones otherwise */
        for (int32_t k = 0; k < W; ++k) {
            for (int32_t v = k; v < n; v += W) {
                oracle_copra_listen(&m, v, offsets, indices, weights, src_l, src_b, W, k, L,
                                    strict, seed, it, buf_l[nxt] + (size_t)v * L,
                                    buf_b[nxt] + (size_t)v * L);
                if (buf_l[nxt][(size_t)v * L] != buf_l[cur][(size_t)v * L]) ++changed;
            }
        }
        cur = nxt;
        if (changed_hist) changed_hist[it] = changed;
        *iterations = it + 1;
        if ((double)changed <= tolerance * (double)n) {
            *converged = 1;
            break;
        }
    }
    for (int32_t v = 0; v < n; ++v) {
        labels[v] = buf_l[cur][(size_t)v * L];
        if (sets_l)
            for (int32_t s = 0; s < L; ++s) {
                sets_l[(size_t)v * L + s] = buf_l[cur][(size_t)v * L + s];
                sets_b[(size_t)v * L + s] = buf_b[cur][(size_t)v * L + s];
            }
    }
done:
    free(buf_l[0]);
    free(buf_l[1]);
    free(buf_b[0]);
    free(buf_b[1]);
    free(m.slot_of);
    free(m.label);
    free(m.t);
    free(m.first);
    return rc;
}
