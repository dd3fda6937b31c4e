// One RAK sweep (Sec. 3.2): every vertex of a bucket sums the weights of its
// neighbours' labels and adopts the heaviest one, with the strict ("first in
// adjacency order") or non-strict ("random") tie rule.
//
// Buckets by degree d:
//   small  1..32     k_small : rows of up to 8 entries take one lane each and
//                              count their labels in registers; longer rows are
//                              packed whole into 32-lane chunks, where each
//                              lane sums its label's weight over its row with
//                              shuffles and the per-row argmax is a segmented
//                              redux.sync maximum, so no table is needed.
//   warp   33..128   k_warp  : one warp per vertex, a 256-slot open-addressing
//                              table per warp in shared memory.
//   (cta, cta2 and hub rows up to 4096 entries: once labels settle, a warp per
//    row first tests the majority rule, k_major_rows, and the CTA kernel skips
//    the rows it settled.)
//   cta    129..512  k_cta   : one 128-thread CTA per vertex, 1024-slot table.
//   cta2   513..1024 k_cta   : one 256-thread CTA per vertex, 2048-slot table.
//   hub    1025..4096 k_cta  : one 512-thread CTA per vertex, 8192-slot table.
//   hub    > 4096    k_hub_seg + k_hub_merge : the row is cut into 4096-entry
//                              segments; each segment aggregates its labels in
//                              a shared table and writes them out as records
//                              grouped into label partitions, then one CTA per
//                              partition merges the records of every segment
//                              and the last one of the row picks its label.
// Table rows insert their entries lane by lane with shared-memory atomics (a
// warp-wide __match_any_sync merge of equal labels before insertion cost more
// than the atomics it saved); the one label a warp sees most once labels have
// settled is summed in registers instead (HotLabel).
// A warp or CTA table slot is one 64-bit word, (label + 1) << 32 | summed
// weight: claimed by a 64-bit compare-and-swap, summed by a 32-bit add on its
// low word.  A label's first position (the smallest row position at which it
// occurs) is found only for the labels tied at the maximum, by a second pass
// over the row; the hub segment and partition tables keep (label, summed
// weight, ~first position) records.  Either way the argmax key (weight desc,
// [non-strict key asc,] first position asc) is unique and independent of the
// order in which entries were accumulated.  Weights are summed in int32 (the
// library rejects graphs whose per-vertex weight sum reaches 2^31), so
// results are bit-exact.
#include <algorithm>

#include "lp_device.cuh"
#include "lp_internal.cuh"

namespace lp {
namespace {

struct Vtx {
    int32_t v;    // global vertex
    int32_t g;    // graph
    int32_t vb;   // first global vertex of the graph
    int32_t lv;   // local vertex id
    int32_t d;    // degree
    int32_t own;  // label at the start of the iteration
    int64_t e0;   // global index of the first entry
};

// List item `item` of the launch: its vertex, graph and packed row.
template <bool MULTI>
__device__ __forceinline__ bool load_vtx(const SweepArgs &a, int64_t item, Vtx &x)
{
    const int32_t v = __ldg(a.list + item);
    x.v = v;
    x.g = 0;
    x.vb = 0;
    if (MULTI) {
        x.g = a.vgraph[v];
        if (!a.g_active[x.g]) return false;
        x.vb = a.g_vbase[x.g];
    }
    x.lv = v - x.vb;
    const int64_t rs = __ldg(a.rp + item);
    x.d = (int32_t)(__ldg(a.rp + item + 1) - rs);
    x.e0 = rs;
    x.own = __ldg(a.lab_in + v);
    return true;
}

// The row of a hub task (its packed start and degree are in the task).
template <bool MULTI>
__device__ __forceinline__ bool load_task(const SweepArgs &a, const HubTask &t, Vtx &x)
{
    x.v = t.v;
    x.g = 0;
    x.vb = 0;
    if (MULTI) {
        x.g = a.vgraph[t.v];
        if (!a.g_active[x.g]) return false;
        x.vb = a.g_vbase[x.g];
    }
    x.lv = t.v - x.vb;
    x.d = t.d;
    x.e0 = t.e0;
    x.own = __ldg(a.lab_in + t.v);
    return true;
}

// Next work item of a grid-stride loop, loaded one step ahead so that its
// dependent loads (list entry, row bounds, own label) overlap the current one.
template <bool MULTI>
struct VtxPipe {
    Vtx next;
    bool next_ok = false;
    uint8_t next_maj = 0;  // the majority pre-pass flag (when there is one)
    __device__ __forceinline__ void fetch(const SweepArgs &a, int64_t item)
    {
        next_ok = item < a.len && load_vtx<MULTI>(a, item, next);
        next_maj = next_ok && a.vmaj ? a.vmaj[next.v] : 0;
    }
};

// Whether graph g's vertices try the majority test in this launch: not in
// the first sweep from unique labels (the host clears a.majority: no row
// longer than 8 entries has a majority label then), and only after an
// iteration that changed fewer than 60% of the graph's labels (a synchronous
// run that oscillates changes nearly all of them and no row passes).  On
// R-MAT the test (own label, then the weighted vote's candidate) settles
// nearly every row longer than 32 entries from the second wave of the second
// sweep on.
// Level 1 (20-60% changed: labels still consolidating, many rows fail) tests
// only rows already held in registers, where a failed test costs no memory
// traffic; level 2 (under 20%: nearly every row passes) also runs the
// warp-per-row pre-passes of the CTA kernels' rows and the small kernel's
// packed majority pass.
__device__ __forceinline__ int maj_level(const SweepArgs &a, int32_t g)
{
    if (!a.majority || a.identity) return 0;
    if (!a.changed_prev) return 2;
    const long long c = __ldg(a.changed_prev + g), n = __ldg(a.g_n + g);
    if (5 * c >= 3 * n) return 0;
    return 5 * c < n ? 2 : 1;
}

__device__ __forceinline__ bool try_majority(const SweepArgs &a, int32_t g)
{
    return maj_level(a, g) > 0;
}

// Whether the weighted vote's candidate c (final surplus n, row weight tw) is
// worth a counting pass: a surplus above half the weight already proves the
// majority (the candidate's weight is at least its surplus); a thin surplus
// rarely ends in one, and the row's table gives the exact answer anyway.
__device__ __forceinline__ bool vote_proven(uint32_t n, uint32_t tw)
{
    return 2ull * n > (unsigned long long)tw;
}

__device__ __forceinline__ bool vote_worth_counting(uint32_t n, uint32_t tw)
{
    return 8ull * n >= (unsigned long long)tw;
}

constexpr int32_t ID_MASK = 0x7FFFFFFF;  // packed neighbour id without its wave bit

// Label of the neighbour with packed id `col` (graph's first vertex vb) as
// seen by this launch: a neighbour of an earlier wave (bit 31) is read from
// lab_out, every other one from lab_in.  Neither buffer is written at an
// address this launch reads: lab_in is only written by the next iteration,
// and lab_out entries of earlier waves were written by earlier launches, so
// both go through the read-only path.  When one launch sweeps every wave
// (COH), earlier waves' labels were written by other CTAs of the same launch
// before a grid barrier: they are read from L2 (ld.global.cg), which the
// barrier's fences make coherent, never through a possibly stale L1 line.
template <bool COH = false>
__device__ __forceinline__ int32_t neighbour_label(const SweepArgs &a, int32_t vb, int32_t col)
{
    const int64_t gi = (int64_t)vb + (col & ID_MASK);
    if (COH && col < 0) return __ldcg(a.lab_out + gi);
    return ld_label((col < 0 ? a.lab_out : a.lab_in) + gi);
}


// ----------------------------------------------------------------------------
// Entry quads: a row is read as aligned 16-byte blocks of 4 entries (column
// index and weight), so each lane has four label gathers in flight at once.
// ----------------------------------------------------------------------------
struct Quad {
    int32_t l[4];  // label of each entry, EMPTY outside the row
    int32_t w[4];  // weight, 0 outside the row
};

__device__ __forceinline__ Quad empty_quad()
{
    Quad q;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        q.l[j] = EMPTY;
        q.w[j] = 0;
    }
    return q;
}

// column indices and weights of entries 4*blk .. 4*blk+3 of the arena
__device__ __forceinline__ void load_block(const SweepArgs &a, int64_t blk, int32_t (&u)[4],
                                           int32_t (&w)[4])
{
    const int64_t e0 = blk * 4;
    if (e0 + 3 < a.ne) {
        const int4 I = ld_entries4(a.idx, blk);
        u[0] = I.x;
        u[1] = I.y;
        u[2] = I.z;
        u[3] = I.w;
        if (a.wts) {
            const int4 W = ld_entries4(a.wts, blk);
            w[0] = W.x;
            w[1] = W.y;
            w[2] = W.z;
            w[3] = W.w;
        } else {
            w[0] = w[1] = w[2] = w[3] = 1;
        }
    } else {  // the arena's last, partial block
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const bool ok = e0 + j < a.ne;
            u[j] = ok ? __ldg(a.idx + e0 + j) : 0;
            w[j] = ok ? (a.wts ? __ldg(a.wts + e0 + j) : 1) : 0;
        }
    }
}

// entries 4*blk .. 4*blk+3 of the arena, kept where they lie in [lo, hi)
template <bool COH = false>
__device__ __forceinline__ Quad load_quad(const SweepArgs &a, int64_t blk, int64_t lo, int64_t hi,
                                          int32_t vb)
{
    const int64_t e0 = blk * 4;
    int32_t u[4], w[4];
    load_block(a, blk, u, w);
    Quad q;
    if (a.spoken) {  // SLPA: the labels the entries' speakers spoke
        int32_t sp[4];
        if (e0 + 3 < a.ne) {
            const int4 S = ld_entries4(a.spoken, blk);
            sp[0] = S.x;
            sp[1] = S.y;
            sp[2] = S.z;
            sp[3] = S.w;
        } else {
#pragma unroll
            for (int j = 0; j < 4; ++j) sp[j] = e0 + j < a.ne ? __ldg(a.spoken + e0 + j) : EMPTY;
        }
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const bool in = e0 + j >= lo && e0 + j < hi;
            q.l[j] = in ? sp[j] : EMPTY;
            q.w[j] = in ? w[j] : 0;
        }
        return q;
    }
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const bool in = e0 + j >= lo && e0 + j < hi;
        q.l[j] = in ? neighbour_label<COH>(a, vb, u[j]) : EMPTY;
        q.w[j] = in ? w[j] : 0;
    }
    return q;
}

// Per-warp fast path for a row's dominant label.  Once labels have settled
// most entries of a row carry the same label, and inserting it once per warp
// round would serialise many atomics on one table slot.  The warp picks the
// label of its first entry as its hot label; entries carrying it are summed
// in registers (with their first position) and inserted once at the end.
struct HotLabel {
    int32_t label = EMPTY;       // warp-uniform
    int sum = 0;                 // lane-local
    uint32_t pos = 0xFFFFFFFFu;  // lane-local first position
    __device__ __forceinline__ void pick(const Quad &q)
    {
        if (label != EMPTY) return;
        const unsigned m = __ballot_sync(FULL, q.l[0] != EMPTY);
        if (m) label = __shfl_sync(FULL, q.l[0], __ffs(m) - 1);
    }
    // true if the entry was absorbed
    __device__ __forceinline__ bool take(int32_t l, int w, uint32_t p)
    {
        if (l == EMPTY || l != label) return false;
        sum += w;
        pos = min(pos, p);
        return true;
    }
    // warp totals, valid in every lane
    __device__ __forceinline__ int total() const { return __reduce_add_sync(FULL, sum); }
    __device__ __forceinline__ uint32_t first() const { return __reduce_min_sync(FULL, pos); }
};

// Summed weight of the entries of q carrying label `own`, and of all of them.
__device__ __forceinline__ void own_weight(const Quad &q, int32_t own, uint32_t &ow, uint32_t &tw)
{
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        tw += (uint32_t)q.w[j];
        ow += q.l[j] == own ? (uint32_t)q.w[j] : 0u;
    }
}

// Weighted majority vote (Boyer & Moore's MJRTY with weights): the state is
// a candidate label and its surplus weight.  If some label holds more than
// half of the weight of the entries voted, the final candidate is that label,
// whatever the order in which entries are added and partial states merged.
// A label that holds more than half of a row's weight is the unique maximum
// under either tie rule, so a verified candidate is the row's new label.
struct Vote {
    int32_t c = EMPTY;
    uint32_t n = 0u;
};

__device__ __forceinline__ void vote_add(Vote &v, int32_t l, uint32_t w)
{
    if (l == EMPTY) return;
    if (v.n == 0u) {
        v.c = l;
        v.n = w;
    } else if (v.c == l) {
        v.n += w;
    } else if (v.n >= w) {
        v.n -= w;
    } else {
        v.c = l;
        v.n = w - v.n;
    }
}

__device__ __forceinline__ Vote vote_merge(const Vote &x, const Vote &y)
{
    if (x.n == 0u) return y;
    if (y.n == 0u) return x;
    if (x.c == y.c) return Vote{x.c, x.n + y.n};
    return x.n >= y.n ? Vote{x.c, x.n - y.n} : Vote{y.c, y.n - x.n};
}

// the warp's merged state (lane 0's, broadcast: lanes may merge in different
// orders and disagree when there is no majority)
__device__ __forceinline__ Vote warp_vote_state(Vote v)
{
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) {
        Vote y;
        y.c = __shfl_xor_sync(FULL, v.c, o);
        y.n = __shfl_xor_sync(FULL, v.n, o);
        v = vote_merge(v, y);
    }
    v.c = __shfl_sync(FULL, v.c, 0);
    v.n = __shfl_sync(FULL, v.n, 0);
    return v;
}

// the warp's candidate (EMPTY when nothing is left)
__device__ __forceinline__ int32_t warp_vote(const Vote &v)
{
    const Vote r = warp_vote_state(v);
    return r.n ? r.c : EMPTY;
}

__device__ __forceinline__ void vote_quad(const Quad &q, Vote &v)
{
#pragma unroll
    for (int j = 0; j < 4; ++j) vote_add(v, q.l[j], (uint32_t)q.w[j]);
}

// summed weight of the entries of q carrying label c
__device__ __forceinline__ uint32_t label_weight(const Quad &q, int32_t c)
{
    uint32_t s = 0u;
#pragma unroll
    for (int j = 0; j < 4; ++j) s += q.l[j] == c ? (uint32_t)q.w[j] : 0u;
    return s;
}

// the block's merged vote, valid in every thread (s_v: NT / 32 + 1 entries)
template <int NT>
__device__ __forceinline__ Vote block_vote(const Vote &v, Vote *s_v)
{
    const Vote w = warp_vote_state(v);
    if ((threadIdx.x & 31) == 0) s_v[threadIdx.x >> 5] = w;
    __syncthreads();
    if (threadIdx.x == 0) {
        Vote m;
        for (int k = 0; k < NT / 32; ++k) m = vote_merge(m, s_v[k]);
        s_v[NT / 32] = m;
    }
    __syncthreads();
    const Vote r = s_v[NT / 32];
    __syncthreads();
    return r;
}

// Identity sweep: the labels read are the initial unique labels (label of u
// is u) and no row repeats a neighbour, so a label's summed weight is its one
// edge weight and its first position is that entry's.  The adopted label is
// the argmax of the entries of [lo, hi) (row starting at entry `row`) under
// the same order; this folds the thread's blocks into `best`.
template <int NT>
__device__ __forceinline__ Cand identity_best(const SweepArgs &a, int64_t row, int64_t lo,
                                              int64_t hi, uint64_t ktv, int t)
{
    Cand best{0u, 0u, 0ull, EMPTY};
    const int64_t b_hi = (hi - 1) >> 2;
    for (int64_t blk = (lo >> 2) + t; blk <= b_hi; blk += NT) {
        int32_t u[4], w[4];
        load_block(a, blk, u, w);
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int64_t e = blk * 4 + j;
            if (e < lo || e >= hi || (uint32_t)w[j] < best.sum) continue;
            const int32_t l = u[j] & ID_MASK;  // the initial label of u is u
            const Cand c{(uint32_t)w[j], 0xFFFFFFFFu - (uint32_t)(e - row),
                         a.strict ? 0ull : stream_at(ktv, (uint64_t)l + 1), l};
            if (better(c, best)) best = c;
        }
    }
    return best;
}

// Best candidate of the warp under the total order of `better`, valid in
// every lane; lanes hold their local best (sum 0 = none).
__device__ __forceinline__ Cand warp_argmax(const Cand &c, int strict)
{
    const uint32_t mx = __reduce_max_sync(FULL, c.sum);
    bool cand = c.sum == mx;
    if (!strict) {
        const uint32_t hh = __reduce_min_sync(FULL, cand ? (uint32_t)(c.h >> 32) : 0xFFFFFFFFu);
        cand = cand && (uint32_t)(c.h >> 32) == hh;
        const uint32_t hl = __reduce_min_sync(FULL, cand ? (uint32_t)c.h : 0xFFFFFFFFu);
        cand = cand && (uint32_t)c.h == hl;
    }
    const uint32_t np = __reduce_max_sync(FULL, cand ? c.npos : 0u);
    cand = cand && c.npos == np;
    const int src = __ffs(__ballot_sync(FULL, cand)) - 1;
    Cand r;
    r.sum = mx;
    r.npos = np;
    r.h = __shfl_sync(FULL, c.h, src);
    r.label = __shfl_sync(FULL, c.label, src);
    return r;
}

template <int NT>
__device__ __forceinline__ Cand block_argmax(const Cand &c, int strict, Cand *s_red)
{
    const Cand w = warp_argmax(c, strict);
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    if (lane == 0) s_red[wib] = w;
    __syncthreads();
    Cand r{0u, 0u, 0ull, EMPTY};
    if (wib == 0) {
        if (lane < NT / 32) r = s_red[lane];
        r = warp_argmax(r, strict);
    }
    return r;  // valid in warp 0
}

// ----------------------------------------------------------------------------
// small bucket: several rows per warp chunk
// ----------------------------------------------------------------------------
constexpr int TINY = 8;  // rows of up to TINY entries get one lane each

template <bool MULTI, bool COH = false>
__device__ __forceinline__ void small_sweep(const SweepArgs &a)
{
    const int lane = threadIdx.x & 31;
    const int64_t wid = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    uint32_t my_changed = 0;

    const int rt = a.tile_rows;  // rows per tile: lanes rt..31 hold none
    for (int64_t tile = wid; tile * rt < a.len; tile += nw) {
        const int64_t i = tile * rt + lane;
        Vtx x{0, 0, 0, 0, 0, 0, 0};
        bool ok = false;
        if (lane < rt && i < a.len) ok = load_vtx<MULTI>(a, i, x);
        int d = ok ? x.d : 0;
        const int32_t own = ok ? x.own : 0;

        // Rows of at most TINY entries: one lane per row.  The lane loads the
        // row and forms every entry's label total over the row in registers
        // (O(d^2) compares); the first entry reaching the maximum holds the
        // label with the earliest first position (strict ties).
        const bool tiny = d >= 1 && d <= TINY;
        if (__any_sync(FULL, tiny)) {
            int32_t lab[TINY];
            uint32_t wt[TINY];
#pragma unroll
            for (int j = 0; j < TINY; ++j) {
                lab[j] = EMPTY;
                wt[j] = 0u;
                if (tiny && j < d) {
                    const int64_t e = x.e0 + j;
                    const int32_t u = ld_entry(a.idx + e);
                    wt[j] = a.wts ? (uint32_t)ld_entry(a.wts + e) : 1u;
                    lab[j] = a.spoken ? ld_entry(a.spoken + e)
                             : a.identity ? (u & ID_MASK) : neighbour_label<COH>(a, x.vb, u);
                }
            }
            // entries past the row are EMPTY with weight 0: their totals are 0
            uint32_t bs = 0u;
            int32_t bl = own;
#pragma unroll
            for (int j = 0; j < TINY; ++j) {
                uint32_t t = 0u;
#pragma unroll
                for (int k = 0; k < TINY; ++k) t += lab[k] == lab[j] ? wt[k] : 0u;
                if (t > bs) {
                    bs = t;
                    bl = lab[j];
                }
            }
            if (!a.strict && tiny) {
                // among the labels of maximum total, the least tie key (then
                // the earliest first position)
                uint64_t bh = ~0ull;
#pragma unroll
                for (int j = 0; j < TINY; ++j) {
                    uint32_t t = 0u;
#pragma unroll
                    for (int k = 0; k < TINY; ++k) t += lab[k] == lab[j] ? wt[k] : 0u;
                    if (t == bs) {
                        const uint64_t h = tie_key(a.key_t, x.lv, lab[j]);
                        if (h < bh) {
                            bh = h;
                            bl = lab[j];
                        }
                    }
                }
            }
            const bool ch = tiny && bl != own;
            if (tiny) {
                a.lab_out[x.v] = bl;
                d = 0;  // done: left out of the passes below
            }
            if (MULTI) {
                const unsigned chm = __ballot_sync(FULL, ch);
                if (ch) {
                    const unsigned gg = __match_any_sync(chm, (unsigned)x.g);
                    if (lane == __ffs(gg) - 1) atomicAdd(a.changed + x.g, __popc(gg));
                }
            } else {
                my_changed += __popc(__ballot_sync(FULL, ch));
            }
        }

        if (__any_sync(FULL, d > 0 && maj_level(a, x.g) == 2)) {
            // Majority pass: rows are read as aligned 16-byte blocks, several
            // rows per 32-block chunk; a row whose own label holds more than
            // half of its weight keeps it (the unique maximum) and drops out.
            const int64_t q0 = x.e0 >> 2;
            const int nq = d > 0 ? (int)(((x.e0 + d - 1) >> 2) - q0 + 1) : 0;  // <= 9
            int Q = nq;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int y = __shfl_up_sync(FULL, Q, o);
                if (lane >= o) Q += y;
            }
            const int qexcl = Q - nq;
            const int qtotal = __shfl_sync(FULL, Q, 31);
            unsigned settled = 0u;
            int start = 0, base = 0;
            while (base < qtotal && start < 32) {
                const unsigned fits =
                    __ballot_sync(FULL, (lane >= start && Q - base <= 32) || lane == start);
                const int end = 32 - __clz(fits);
                const int total = __shfl_sync(FULL, Q, end - 1) - base;
                int o = start;
#pragma unroll
                for (int step = 16; step >= 1; step >>= 1) {
                    const int c = o + step;
                    const int ex = __shfl_sync(FULL, qexcl, c & 31);
                    if (c < end && ex - base <= lane) o = c;
                }
                const bool act = lane < total;
                const long long o_e0 = __shfl_sync(FULL, (long long)x.e0, o);
                const int o_d = __shfl_sync(FULL, d, o);
                const int o_vb = MULTI ? __shfl_sync(FULL, x.vb, o) : 0;
                const int32_t o_own = __shfl_sync(FULL, own, o);
                const int o_qex = __shfl_sync(FULL, qexcl, o);
                uint32_t ow = 0, tw = 0;
                if (act) {
                    const int64_t blk = (o_e0 >> 2) + (lane - (o_qex - base));
                    own_weight(load_quad<COH>(a, blk, o_e0, o_e0 + o_d, o_vb), o_own, ow, tw);
                }
                // the row's quads fill lanes [o_qex - base, + its quad count)
                const int o_nq = (int)(((o_e0 + o_d - 1) >> 2) - (o_e0 >> 2) + 1);
                const unsigned og =
                    act ? lane_range(o_qex - base, o_nq) : ~lane_range(0, total);
                const uint32_t OW = __reduce_add_sync(og, ow);
                const uint32_t TW = __reduce_add_sync(og, tw);
                const bool keep = act && lane == __ffs(og) - 1 && 2ull * OW > (unsigned long long)TW;
                settled |= __reduce_or_sync(FULL, keep ? (1u << o) : 0u);
                base += total;
                start = end;
            }
            if ((settled >> lane) & 1u) {
                a.lab_out[x.v] = own;
                d = 0;  // settled: left out of the table-free pass below
            }
        }

        int P = d;  // inclusive prefix of degrees over the tile
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(FULL, P, o);
            if (lane >= o) P += y;
        }
        const int excl = P - d;
        const int total_all = __shfl_sync(FULL, P, 31);

        int start = 0, base = 0;
        while (base < total_all && start < 32) {
            // greedy packing: rows start.. that end within 32 entries of base
            // (row `start` always fits: the bucket holds degrees <= 32)
            const unsigned fits =
                __ballot_sync(FULL, (lane >= start && P - base <= 32) || lane == start);
            const int end = 32 - __clz(fits);
            const int total = __shfl_sync(FULL, P, end - 1) - base;

            // owner of entry `lane`: the last row in [start, end) starting at or before it
            int o = start;
#pragma unroll
            for (int step = 16; step >= 1; step >>= 1) {
                const int c = o + step;
                const int ex = __shfl_sync(FULL, excl, c & 31);
                if (c < end && ex - base <= lane) o = c;
            }
            const bool act = lane < total;
            const int o_excl = __shfl_sync(FULL, excl, o);
            const int o_d = __shfl_sync(FULL, d, o);
            const long long o_e0 = __shfl_sync(FULL, (long long)x.e0, o);
            const int o_vb = MULTI ? __shfl_sync(FULL, x.vb, o) : 0;
            const int o_lv = __shfl_sync(FULL, x.lv, o);
            const int o_v = __shfl_sync(FULL, x.v, o);
            const int32_t o_own = __shfl_sync(FULL, own, o);
            const int pos = lane - (o_excl - base);

            int w = 0;
            int32_t l = EMPTY;
            if (act) {
                const long long e = o_e0 + pos;
                const int32_t u = ld_entry(a.idx + e);
                w = a.wts ? ld_entry(a.wts + e) : 1;
                l = a.spoken ? ld_entry(a.spoken + e)
                             : a.identity ? (u & ID_MASK) : neighbour_label<COH>(a, o_vb, u);
            }
            // the owner's lanes (its whole row: rows fit in the chunk), then the
            // lanes of the owner with an equal label; the lowest lane of a
            // group holds its first position (in an identity sweep every
            // label of a row is distinct)
            const unsigned og = act ? lane_range(o_excl - base, o_d) : ~lane_range(0, total);
            int s = w;
            bool leader = act;
            if (!a.identity) {
                // every lane sums the weights of its row's entries holding its
                // label, reading the k-th entry of its own row from the lane
                // holding it (rows of the chunk in step); the entry at the
                // label's first position leads
                s = 0;
                int first = 32;
                const int seg = o_excl - base;
                const int dmax = __reduce_max_sync(FULL, act ? (unsigned)o_d : 0u);
                for (int k = 0; k < dmax; ++k) {
                    const int src = (seg + k) & 31;
                    const int32_t lk = __shfl_sync(FULL, l, src);
                    const int wk = __shfl_sync(FULL, w, src);
                    const bool same = act && k < o_d && lk == l;
                    s += same ? wk : 0;
                    first = same && k < first ? k : first;
                }
                leader = act && pos == first;
            }
            // segmented argmax over each owner's lanes
            const uint32_t hi = leader ? (uint32_t)s : 0u;
            const uint32_t npos = leader ? 0xFFFFFFFFu - (uint32_t)pos : 0u;
            const uint32_t mhi = __reduce_max_sync(og, hi);
            bool cand = leader && hi == mhi;
            if (!a.strict) {
                const uint64_t h = cand ? tie_key(a.key_t, o_lv, l) : ~0ull;
                const uint32_t hh = __reduce_min_sync(og, cand ? (uint32_t)(h >> 32) : 0xFFFFFFFFu);
                cand = cand && (uint32_t)(h >> 32) == hh;
                const uint32_t hl = __reduce_min_sync(og, cand ? (uint32_t)h : 0xFFFFFFFFu);
                cand = cand && (uint32_t)h == hl;
            }
            const uint32_t mlo = __reduce_max_sync(og, cand ? npos : 0u);
            const bool win = cand && npos == mlo;
            const bool ch = win && l != o_own;
            if (win) a.lab_out[o_v] = l;
            if (MULTI) {
                const int o_g = __shfl_sync(FULL, x.g, o);
                const unsigned chm = __ballot_sync(FULL, ch);
                if (ch) {
                    const unsigned gg = __match_any_sync(chm, (unsigned)o_g);
                    if (lane == __ffs(gg) - 1) atomicAdd(a.changed + o_g, __popc(gg));
                }
            } else {
                my_changed += __popc(__ballot_sync(FULL, ch));
            }
            base += total;
            start = end;
        }
    }
    if (!MULTI && lane == 0 && my_changed) atomicAdd(a.changed, (int)my_changed);
}

template <bool MULTI>
__global__ void __launch_bounds__(256, 6) k_small(SweepArgs a)
{
    if (a.stop && *a.stop) return;  // launched past the end of the run
    small_sweep<MULTI>(a);
}

// Grid-wide barrier of a cooperative launch (every CTA resident).  bar[0]
// counts arrivals over the whole launch (zeroed before it): barrier number
// `epoch` (0, 1, ...) is passed once it has reached (epoch + 1) * expected,
// so an arrival is one atomic and nothing has to be reset in between.  A CTA
// that polls more than BARRIER_SPIN times records *err = 1; every CTA returns
// false once *err is set, so the kernel ends instead of waiting.
constexpr uint32_t BARRIER_SPIN = 1u << 22;

__device__ bool grid_barrier(unsigned *bar, int32_t *err, uint32_t epoch, unsigned expected = 0,
                             uint32_t spin_limit = BARRIER_SPIN)
{
    if (expected == 0) expected = gridDim.x;
    __shared__ int s_ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        const unsigned target = (epoch + 1u) * expected;
        __threadfence();  // this CTA's writes before its arrival
        unsigned seen = atomicAdd(bar, 1u) + 1u;
        volatile unsigned *vbar = bar;
        int ok = 1;
        for (uint32_t spins = 0; seen < target; ++spins) {
            if (spins >= spin_limit) {
                atomicExch(err, 1);
                ok = 0;
                break;
            }
            __nanosleep(32);
            seen = *vbar;
        }
        __threadfence();  // the other CTAs' writes before this CTA's reads
        s_ok = ok && *(volatile int32_t *)err == 0;
    }
    __syncthreads();
    return s_ok != 0;
}

// Self-test of the barrier's time limit: the CTAs wait for one CTA more than
// the grid has, so the wait runs out after spin_limit polls and sets *err.
__global__ void k_barrier_probe(unsigned *bar, int32_t *err, uint32_t spin_limit)
{
    grid_barrier(bar, err, 0u, gridDim.x + 1u, spin_limit);
}

// Every wave of an asynchronous sweep of a single graph whose rows are all in
// the small bucket, in one cooperative launch: the grid sweeps wave k's list,
// then meets at a grid barrier before wave k + 1 (whose rows read wave k's
// labels).  With many short waves this replaces a launch per wave.
__global__ void __launch_bounds__(256, 6) k_small_waves(SweepArgs a, const int32_t *wlist,
                                                        const int64_t *wstart, const int64_t *wcount,
                                                        unsigned *bar, int32_t *err)
{
    if (a.stop && *a.stop) return;  // launched past the end of the run
    for (uint32_t k = 0; k < a.waves; ++k) {
        SweepArgs b = a;
        b.list = wlist + wstart[k];
        b.rp = a.rp + wstart[k];
        b.len = wcount[k];
        b.identity = a.identity && k == 0;  // later waves read this sweep's labels
        small_sweep<false, true>(b);
        if (k + 1 < a.waves && !grid_barrier(bar, err, k)) return;
    }
}

// Every wave of an asynchronous sweep of a single graph whose rows all hold
// at most TINY entries (paths such as the k-mer graphs), in one cooperative
// launch: 32 rows per warp tile, one per lane, counted in registers as the
// small-row kernel counts its rows of at most TINY entries.  Before each grid
// barrier a warp loads its first tile of the next wave (list items, packed
// rows and own labels do not depend on labels of this iteration), so after
// the barrier only the neighbours' labels remain to be read.
struct TinyRow {
    int32_t v, own, d;
    int32_t u[TINY];
    uint32_t w[TINY];
};

__device__ __forceinline__ void tiny_fetch(const SweepArgs &a, const int32_t *list,
                                           const int64_t *rp, int64_t len, int64_t tile,
                                           TinyRow &r)
{
    const int64_t i = tile * 32 + (threadIdx.x & 31);
    r.d = 0;
    r.v = 0;
    r.own = 0;
    if (i < len) {
        r.v = __ldg(list + i);
        const int64_t e0 = __ldg(rp + i);
        r.d = (int32_t)(__ldg(rp + i + 1) - e0);
        r.own = __ldg(a.lab_in + r.v);
#pragma unroll
        for (int j = 0; j < TINY; ++j) {
            const bool in = j < r.d;
            r.u[j] = in ? ld_entry(a.idx + e0 + j) : 0;
            r.w[j] = in ? (a.wts ? (uint32_t)ld_entry(a.wts + e0 + j) : 1u) : 0u;
        }
    }
}

__global__ void __launch_bounds__(256, 2) k_tiny_waves(SweepArgs a, const int32_t *wlist,
                                                       const int64_t *wstart, const int64_t *wcount,
                                                       unsigned *bar, int32_t *err)
{
    if (a.stop && *a.stop) return;  // launched past the end of the run
    const int lane = threadIdx.x & 31;
    const int64_t wid = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    uint32_t my_changed = 0;
    TinyRow r;  // holds this warp's first tile of a wave before the wave starts
    tiny_fetch(a, wlist + wstart[0], a.rp + wstart[0], wcount[0], wid, r);
    for (uint32_t k = 0; k < a.waves; ++k) {
        const int32_t *list = wlist + wstart[k];
        const int64_t *rp = a.rp + wstart[k];
        const int64_t len = wcount[k];
        const bool identity = a.identity && k == 0;  // later waves read this sweep's labels
        for (int64_t tile = wid; tile * 32 < len; tile += nw) {
            if (tile != wid) tiny_fetch(a, list, rp, len, tile, r);  // the first is loaded
            int32_t lab[TINY];
#pragma unroll
            for (int j = 0; j < TINY; ++j)
                lab[j] = j < r.d ? (identity ? (r.u[j] & ID_MASK) : neighbour_label<true>(a, 0, r.u[j]))
                                 : EMPTY;
            // entries past the row are EMPTY with weight 0: their totals are 0
            uint32_t bs = 0u;
            int32_t bl = r.own;
#pragma unroll
            for (int j = 0; j < TINY; ++j) {
                uint32_t t = 0u;
#pragma unroll
                for (int q = 0; q < TINY; ++q) t += lab[q] == lab[j] ? r.w[q] : 0u;
                if (t > bs) {
                    bs = t;
                    bl = lab[j];
                }
            }
            if (!a.strict && r.d > 0) {
                // among the labels of maximum total, the least tie key (then
                // the earliest first position)
                uint64_t bh = ~0ull;
#pragma unroll
                for (int j = 0; j < TINY; ++j) {
                    uint32_t t = 0u;
#pragma unroll
                    for (int q = 0; q < TINY; ++q) t += lab[q] == lab[j] ? r.w[q] : 0u;
                    if (t == bs) {
                        const uint64_t h = tie_key(a.key_t, r.v, lab[j]);
                        if (h < bh) {
                            bh = h;
                            bl = lab[j];
                        }
                    }
                }
            }
            if (r.d > 0) {
                a.lab_out[r.v] = bl;
                if (bl != r.own) ++my_changed;
            }
        }
        if (k + 1 < a.waves) {
            tiny_fetch(a, wlist + wstart[k + 1], a.rp + wstart[k + 1], wcount[k + 1], wid, r);
            if (!grid_barrier(bar, err, k)) return;
        }
    }
    my_changed = __reduce_add_sync(FULL, my_changed);
    if (lane == 0 && my_changed) atomicAdd(a.changed, (int)my_changed);
}

// Insert one quad (entries 4*blk .. 4*blk+3 of a row starting at global
// entry `row`) into a shared table of 2^lg slots: entries of the warp's hot
// label are summed in registers, every other entry is added by its lane.
__device__ __forceinline__ void insert_quad(const Quad &q, int64_t blk, int64_t row,
                                            HotLabel &hot, int32_t *tk, int32_t *ts,
                                            uint32_t *tp, int lg)
{
    hot.pick(q);
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const uint32_t pos = (uint32_t)(blk * 4 + j - row);
        if (!hot.take(q.l[j], q.w[j], pos) && q.l[j] != EMPTY)
            table_add(tk, ts, tp, lg, 1 << lg, q.l[j], q.w[j], pos);
    }
}

// the warp's hot label total, inserted once
__device__ __forceinline__ void insert_hot(const HotLabel &hot, int32_t *tk, int32_t *ts,
                                           uint32_t *tp, int lg)
{
    const int hs = hot.total();
    const uint32_t hp = hot.first();
    if ((threadIdx.x & 31) == 0 && hs > 0) table_add(tk, ts, tp, lg, 1 << lg, hot.label, hs, hp);
}

// ----------------------------------------------------------------------------
// 64-bit tables of the warp and CTA kernels: slot = (label + 1, summed
// weight), one shared atomic per inserted entry.  The strict tie rule needs a
// label's first position only when several labels reach the maximum (rows of
// more than 128 entries rarely tie once a sweep has run); those rows take a
// second pass over their entries that finds the earliest entry whose label
// is at the maximum.
// ----------------------------------------------------------------------------
__device__ __forceinline__ void insert_quad64(const Quad &q, HotLabel &hot, unsigned long long *t,
                                              int lg)
{
    hot.pick(q);
#pragma unroll
    for (int j = 0; j < 4; ++j)
        if (!hot.take(q.l[j], q.w[j], 0u) && q.l[j] != EMPTY)
            table64_add(t, lg, q.l[j], (uint32_t)q.w[j]);
}

__device__ __forceinline__ void insert_hot64(const HotLabel &hot, unsigned long long *t, int lg)
{
    const int hs = hot.total();
    if ((threadIdx.x & 31) == 0 && hs > 0) table64_add(t, lg, hot.label, (uint32_t)hs);
}

// Top of the slots [0, slots) of a 64-bit table, scanned by NT threads
// (index tid), valid in every thread: the maximum, how many labels reach it
// and one of them; with non-strict ties, the least tie key among those labels
// (a second scan), how many share it and one of them.
template <int NT>
__device__ __forceinline__ Top scan64(const unsigned long long *t, int slots, int tid, int strict,
                                      uint64_t ktv, uint64_t *s_k, uint32_t *s_c, int32_t *s_l)
{
    uint32_t ms = 0u, mc = 0u;
    int32_t ml = EMPTY;
    for (int j = tid; j < slots; j += NT) {
        const unsigned long long v = t[j];
        const uint32_t sw = (uint32_t)v;
        if (v != 0ull && sw >= ms) {
            mc = sw > ms ? 1u : mc + 1u;
            ms = sw;
            ml = slot_label(v);
        }
    }
    uint64_t k = ms;
    block_top<NT>(k, mc, ml, s_k, s_c, s_l);
    Top r{(uint32_t)k, mc, ml, 0ull};
    if (!strict && r.sum > 0u) {
        uint64_t hk = 0ull;  // ~tie key: the largest wins
        uint32_t hc = 0u;
        int32_t hl = EMPTY;
        for (int j = tid; j < slots; j += NT) {
            const unsigned long long v = t[j];
            if (v != 0ull && (uint32_t)v == r.sum) {
                const int32_t l = slot_label(v);
                const uint64_t key = ~stream_at(ktv, (uint64_t)l + 1);
                if (hc == 0u || key > hk) {
                    hk = key;
                    hc = 1u;
                    hl = l;
                } else if (key == hk) {
                    ++hc;
                }
            }
        }
        block_top<NT>(hk, hc, hl, s_k, s_c, s_l);
        r.h = ~hk;
        r.cnt = hc;
        r.label = hl;
    }
    return r;
}

template <int NT>
__device__ __forceinline__ void clear64(unsigned long long *t, int slots, int tid)
{
    for (int j = tid; j < slots; j += NT) t[j] = 0ull;
}

// (row position << 32 | label) of the earliest entry of q (entries 4 * blk ..
// of a row starting at `row`) whose label is one of the tied labels of `top`,
// ~0 if none
__device__ __forceinline__ uint64_t tie_quad(const Quad &q, int64_t blk, int64_t row,
                                             const unsigned long long *t, int lg, const Top &top,
                                             int strict, uint64_t ktv)
{
    uint64_t best = ~0ull;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const int32_t l = q.l[j];
        if (l == EMPTY || table64_sum(t, lg, l) != top.sum) continue;
        if (!strict && stream_at(ktv, (uint64_t)l + 1) != top.h) continue;
        const uint64_t c = ((uint64_t)(uint32_t)(blk * 4 + j - row) << 32) | (uint32_t)l;
        best = c < best ? c : best;
    }
    return best;
}

// the same over the entries [lo, hi) of a row, re-read, NT threads (index tid)
template <int NT>
__device__ __forceinline__ uint64_t tie_range(const SweepArgs &a, int64_t row, int64_t lo,
                                              int64_t hi, int32_t vb, int tid,
                                              const unsigned long long *t, int lg, const Top &top,
                                              uint64_t ktv)
{
    uint64_t best = ~0ull;
    for (int64_t blk = (lo >> 2) + tid; blk <= (hi - 1) >> 2; blk += NT) {
        const uint64_t c = tie_quad(load_quad(a, blk, lo, hi, vb), blk, row, t, lg, top, a.strict,
                                    ktv);
        best = c < best ? c : best;
    }
    return best;
}

// Aggregate the entries [lo, hi) of a row into a 64-bit table of 2^lg slots
// (room for every distinct label of the range), NT threads cooperating.
template <int NT>
__device__ __forceinline__ void accumulate_range64(const SweepArgs &a, int64_t lo, int64_t hi,
                                                   int32_t vb, unsigned long long *t, int lg)
{
    const int64_t b_hi = (hi - 1) >> 2;
    HotLabel hot;
    for (int64_t base = lo >> 2; base <= b_hi; base += NT) {
        const int64_t blk = base + threadIdx.x;
        const Quad q = blk <= b_hi ? load_quad(a, blk, lo, hi, vb) : empty_quad();
        insert_quad64(q, hot, t, lg);
    }
    insert_hot64(hot, t, lg);
}

// ----------------------------------------------------------------------------
// warp bucket: one warp per vertex, private shared table
// ----------------------------------------------------------------------------
constexpr int WARP_LG = 8;  // log2(WARP_TABLE)
static_assert((1 << WARP_LG) == WARP_TABLE, "warp table size");

template <bool MULTI>
__global__ void __launch_bounds__(256, 4) k_warp(SweepArgs a)
{
    if (a.stop && *a.stop) return;  // launched past the end of the run
    __shared__ unsigned long long s_tab[8 * WARP_TABLE];
    const int lane = threadIdx.x & 31;
    const int wib = threadIdx.x >> 5;
    unsigned long long *tab = s_tab + wib * WARP_TABLE;
    clear64<32>(tab, WARP_TABLE, lane);
    __syncwarp();

    const int64_t wid = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    uint32_t my_changed = 0;

    VtxPipe<MULTI> pipe;
    pipe.fetch(a, wid);
    for (int64_t item = wid; item < a.len; item += nw) {
        const Vtx x = pipe.next;
        const bool ok = pipe.next_ok;
        pipe.fetch(a, item + nw);
        if (!ok) continue;  // warp-uniform
        const int32_t own = x.own;
        const int64_t lo = x.e0, hi = x.e0 + x.d;
        const int64_t b_hi = (hi - 1) >> 2;
        const uint64_t ktv = stream_at(a.key_t, (uint64_t)x.lv + 1);
        int32_t label;
        if (a.identity) {
            label = warp_argmax(identity_best<32>(a, lo, lo, hi, ktv, lane), a.strict).label;
        } else {
            // a row of at most 32 quads is loaded once, one quad per lane; if
            // the vertex's own label holds more than half of its weight it stays
            const int64_t b0 = lo >> 2;
            const bool one = b_hi - b0 < 32;
            Quad q1 = empty_quad();
            bool settled = false;
            if (one) {
                if (b0 + lane <= b_hi) q1 = load_quad(a, b0 + lane, lo, hi, x.vb);
                if (try_majority(a, x.g)) {
                    // own label first, then the vote's candidate
                    uint32_t ow = 0, tw = 0;
                    own_weight(q1, own, ow, tw);
                    ow = __reduce_add_sync(FULL, ow);
                    tw = __reduce_add_sync(FULL, tw);
                    label = own;
                    settled = 2ull * ow > (unsigned long long)tw;
                    if (!settled) {
                        Vote vt;
                        vote_quad(q1, vt);
                        vt = warp_vote_state(vt);
                        if (vt.n && vt.c != own) {
                            label = vt.c;
                            if (vote_proven(vt.n, tw)) {
                                settled = true;
                            } else if (vote_worth_counting(vt.n, tw)) {
                                const uint32_t cw =
                                    __reduce_add_sync(FULL, label_weight(q1, vt.c));
                                settled = 2ull * cw > (unsigned long long)tw;
                            }
                        }
                    }
                }
            }
            if (!settled) {
                // <= 128 labels in 256 slots: every insert finds its slot
                HotLabel hot;
                for (int64_t base = b0; base <= b_hi; base += 32) {
                    const int64_t blk = base + lane;
                    const Quad q =
                        one ? q1 : (blk <= b_hi ? load_quad(a, blk, lo, hi, x.vb) : empty_quad());
                    insert_quad64(q, hot, tab, WARP_LG);
                }
                insert_hot64(hot, tab, WARP_LG);
                __syncwarp();
                const Top top =
                    scan64<32>(tab, WARP_TABLE, lane, a.strict, ktv, nullptr, nullptr, nullptr);
                label = top.label;
                if (top.cnt > 1u) {  // tied maximum: the earliest entry of a tied label
                    uint64_t t = one ? tie_quad(q1, b0 + lane, lo, tab, WARP_LG, top, a.strict, ktv)
                                     : tie_range<32>(a, lo, lo, hi, x.vb, lane, tab, WARP_LG, top,
                                                     ktv);
                    uint64_t k = ~t;
                    uint32_t c = 0u;
                    int32_t l = EMPTY;
                    warp_top(k, c, l);
                    label = (int32_t)(uint32_t)~k;
                }
                __syncwarp();
                clear64<32>(tab, WARP_TABLE, lane);
                __syncwarp();
            }
        }
        if (lane == 0) {
            a.lab_out[x.v] = label;
            if (label != own) {
                if (MULTI)
                    atomicAdd(a.changed + x.g, 1);
                else
                    ++my_changed;
            }
        }
    }
    if (!MULTI && lane == 0 && my_changed) atomicAdd(a.changed, (int)my_changed);
}

// Scan the table slots [0, slots): local best candidate (strict or non-strict),
// resetting every used slot.  Non-strict scans twice: the block maximum first.
template <int NT>
__device__ __forceinline__ Cand scan_table(int32_t *tk, int32_t *ts, uint32_t *tp, int slots,
                                           int strict, uint64_t ktv, uint32_t *s_u)
{
    Cand best{0u, 0u, 0ull, EMPTY};
    uint32_t mx = 0;
    if (!strict) {
        for (int j = threadIdx.x; j < slots; j += NT)
            if (tk[j] != EMPTY) mx = max(mx, (uint32_t)ts[j]);
        mx = block_max<NT>(mx, s_u);
    }
    for (int j = threadIdx.x; j < slots; j += NT) {
        const int32_t key = tk[j];
        if (key != EMPTY) {
            if (strict) {
                const Cand c{(uint32_t)ts[j], tp[j], 0ull, key};
                if (better(c, best)) best = c;
            } else if ((uint32_t)ts[j] == mx) {
                const Cand c{mx, tp[j], stream_at(ktv, (uint64_t)key + 1), key};
                if (better(c, best)) best = c;
            }
            tk[j] = EMPTY;
            ts[j] = 0;
            tp[j] = 0;
        }
    }
    return best;
}

// Aggregate the entries [lo, hi) of a row starting at global entry `row` into
// the shared table of 2^lg slots (which must have room for every distinct
// label of the range), all NT threads cooperating.
template <int NT>
__device__ __forceinline__ void accumulate_range(const SweepArgs &a, int64_t row, int64_t lo,
                                                 int64_t hi, int32_t vb, int32_t *tk, int32_t *ts,
                                                 uint32_t *tp, int lg)
{
    const int64_t b_hi = (hi - 1) >> 2;
    HotLabel hot;
    for (int64_t base = lo >> 2; base <= b_hi; base += NT) {
        const int64_t blk = base + threadIdx.x;
        const Quad q = blk <= b_hi ? load_quad(a, blk, lo, hi, vb) : empty_quad();
        insert_quad(q, blk, row, hot, tk, ts, tp, lg);
    }
    insert_hot(hot, tk, ts, tp, lg);
}

// Block sums of x and y, valid in every thread (s: 2 * NT / 32 words).
template <int NT>
__device__ __forceinline__ uint2 block_sum2(uint32_t x, uint32_t y, uint32_t *s)
{
    x = __reduce_add_sync(FULL, x);
    y = __reduce_add_sync(FULL, y);
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    if (lane == 0) {
        s[wib] = x;
        s[NT / 32 + wib] = y;
    }
    __syncthreads();
    uint2 r{0u, 0u};
#pragma unroll
    for (int k = 0; k < NT / 32; ++k) {
        r.x += s[k];
        r.y += s[NT / 32 + k];
    }
    __syncthreads();
    return r;
}

// ----------------------------------------------------------------------------
// cta bucket: one CTA per vertex, shared table
// ----------------------------------------------------------------------------
template <int NT, int CAP, bool MULTI>
__global__ void __launch_bounds__(NT, NT >= 512 ? 2 : (1536 / NT < 32 ? 1536 / NT : 32))
    k_cta(SweepArgs a)
{
    if (a.stop && *a.stop) return;  // launched past the end of the run
    extern __shared__ unsigned long long smem64[];
    unsigned long long *tab = smem64;  // CAP 64-bit slots
    __shared__ Cand s_red[NT / 32];
    __shared__ uint64_t s_k[NT / 32 + 1];
    __shared__ uint32_t s_c[NT / 32 + 1];
    __shared__ int32_t s_l[NT / 32 + 1];
    __shared__ uint32_t s_u2[2 * (NT / 32)];
    __shared__ Vote s_vote[NT / 32 + 1];
    constexpr int LG = (CAP == 1024) ? 10 : (CAP == 2048) ? 11 : (CAP == 4096) ? 12 : (CAP == 8192) ? 13 : 14;
    static_assert((1 << LG) == CAP, "table size");
    // quads per thread that hold a row of CAP / 2 entries starting 16-byte aligned
    constexpr int R = CAP / 2 / (4 * NT) > 0 ? CAP / 2 / (4 * NT) : 1;

    clear64<NT>(tab, CAP, threadIdx.x);
    __syncthreads();
    uint32_t my_changed = 0;

    // a single graph whose pre-pass ran in this launch: only the rows it left
    // (listed in cpos) remain
    const bool compact = !MULTI && a.cpos && maj_level(a, 0) > 0;
    const int64_t len = compact ? (int64_t)__ldcg(a.ccount) : a.len;
    auto position = [&](int64_t i) -> int64_t { return compact ? (int64_t)__ldcg(a.cpos + i) : i; };
    VtxPipe<MULTI> pipe;
    if (blockIdx.x < len) pipe.fetch(a, position(blockIdx.x));
    for (int64_t i = blockIdx.x; i < len; i += gridDim.x) {
        const Vtx x = pipe.next;
        const bool ok = pipe.next_ok;
        const uint8_t maj = pipe.next_maj;
        if (i + gridDim.x < len)
            pipe.fetch(a, position(i + gridDim.x));
        else
            pipe.next_ok = false;
        if (!ok) continue;  // block-uniform
        // the pre-pass of this launch tested the row (and wrote its label if
        // it settled)
        const bool pre = compact || (a.vmaj && maj_level(a, x.g) > 0);
        if (!compact && pre && maj) continue;
        // slots in use for this vertex: 2^lg >= 2d (d <= CAP / 2 in this bucket)
        const int lg = min(ilog2_ceil(2u * (uint32_t)x.d), LG);
        const int slots = 1 << lg;
        const uint64_t ktv = stream_at(a.key_t, (uint64_t)x.lv + 1);
        const int64_t end = x.e0 + x.d;
        const int64_t b0 = x.e0 >> 2, b_hi = (end - 1) >> 2;
        int32_t label = x.own;
        if (a.identity) {
            label = block_argmax<NT>(identity_best<NT>(a, x.e0, x.e0, end, ktv, threadIdx.x),
                                     a.strict, s_red)
                        .label;  // valid in warp 0
        } else if (b_hi - b0 < (int64_t)R * NT) {
            // the row in registers, R quads per thread
            Quad q[R];
#pragma unroll
            for (int r = 0; r < R; ++r) {
                const int64_t blk = b0 + r * NT + threadIdx.x;
                q[r] = blk <= b_hi ? load_quad(a, blk, x.e0, end, x.vb) : empty_quad();
            }
            // a label holding more than half of the row's weight is the
            // unique maximum: the own label, else the vote's candidate
            bool settled = false;
            if (!pre && try_majority(a, x.g)) {
                uint32_t ow = 0, tw = 0;
                Vote vt;
#pragma unroll
                for (int r = 0; r < R; ++r) {
                    own_weight(q[r], x.own, ow, tw);
                    vote_quad(q[r], vt);
                }
                const uint2 s2 = block_sum2<NT>(ow, tw, s_u2);
                settled = 2ull * s2.x > (unsigned long long)s2.y;
                if (!settled) {
                    const Vote bv = block_vote<NT>(vt, s_vote);
                    if (bv.n && bv.c != x.own) {
                        if (vote_proven(bv.n, s2.y)) {
                            settled = true;
                            label = bv.c;
                        } else if (vote_worth_counting(bv.n, s2.y)) {
                            uint32_t cw = 0u;
#pragma unroll
                            for (int r = 0; r < R; ++r) cw += label_weight(q[r], bv.c);
                            const uint2 c2 = block_sum2<NT>(cw, 0u, s_u2);
                            if (2ull * c2.x > (unsigned long long)s2.y) {
                                settled = true;
                                label = bv.c;
                            }
                        }
                    }
                }
            }
            if (!settled) {
                HotLabel hot;
#pragma unroll
                for (int r = 0; r < R; ++r) insert_quad64(q[r], hot, tab, lg);
                insert_hot64(hot, tab, lg);
                __syncthreads();
                const Top top = scan64<NT>(tab, slots, threadIdx.x, a.strict, ktv, s_k, s_c, s_l);
                label = top.label;
                if (top.cnt > 1u) {  // tied maximum: the earliest entry of a tied label
                    uint64_t t = ~0ull;
#pragma unroll
                    for (int r = 0; r < R; ++r) {
                        const uint64_t c = tie_quad(q[r], b0 + r * NT + threadIdx.x, x.e0, tab, lg,
                                                    top, a.strict, ktv);
                        t = c < t ? c : t;
                    }
                    uint64_t k = ~t;
                    uint32_t c = 0u;
                    int32_t l = EMPTY;
                    block_top<NT>(k, c, l, s_k, s_c, s_l);
                    label = (int32_t)(uint32_t)~k;
                }
                __syncthreads();
                clear64<NT>(tab, slots, threadIdx.x);
            }
        } else {
            accumulate_range64<NT>(a, x.e0, end, x.vb, tab, lg);
            __syncthreads();
            const Top top = scan64<NT>(tab, slots, threadIdx.x, a.strict, ktv, s_k, s_c, s_l);
            label = top.label;
            if (top.cnt > 1u) {
                uint64_t k = ~tie_range<NT>(a, x.e0, x.e0, end, x.vb, threadIdx.x, tab, lg, top, ktv);
                uint32_t c = 0u;
                int32_t l = EMPTY;
                block_top<NT>(k, c, l, s_k, s_c, s_l);
                label = (int32_t)(uint32_t)~k;
            }
            __syncthreads();
            clear64<NT>(tab, slots, threadIdx.x);
        }
        if (threadIdx.x == 0) {
            a.lab_out[x.v] = label;
            if (label != x.own) {
                if (MULTI)
                    atomicAdd(a.changed + x.g, 1);
                else
                    ++my_changed;
            }
        }
        __syncthreads();
    }
    if (!MULTI && threadIdx.x == 0 && my_changed) atomicAdd(a.changed, (int)my_changed);
}

// ----------------------------------------------------------------------------
// Majority pre-pass for the rows of the CTA kernels (cta, cta2 and hub rows up
// to HUB_ONE_MAX entries): one warp per row counts the weight of the entries
// carrying the row's own label and runs the weighted majority vote.  A label
// holding more than half of the row's weight is the unique maximum: the own
// label if it passes, else the vote's candidate once a second read of the
// row confirms its weight.  The label is written here and the row's flag
// tells the CTA kernel to skip it.  Once labels have settled nearly every
// such row passes, and a warp reads a row with a fraction of the
// instructions a CTA spends on it.
// ----------------------------------------------------------------------------
template <bool MULTI>
__global__ void __launch_bounds__(256) k_major_rows(SweepArgs a)
{
    if (a.stop && *a.stop) return;  // launched past the end of the run
    if (!MULTI && maj_level(a, 0) == 0) return;
    const int lane = threadIdx.x & 31;
    const int64_t wid = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    VtxPipe<MULTI> pipe;
    pipe.fetch(a, wid);
    for (int64_t item = wid; item < a.len; item += nw) {
        const Vtx x = pipe.next;
        const bool ok = pipe.next_ok;
        pipe.fetch(a, item + nw);
        if (!ok) continue;  // warp-uniform
        const int lvl = maj_level(a, x.g);
        if (lvl == 0) continue;
        const int64_t lo = x.e0, hi = x.e0 + x.d;
        const int64_t b_lo = lo >> 2, b_hi = (hi - 1) >> 2;
        uint32_t ow = 0u, tw = 0u;
        Vote vt;
        // the first 32 blocks (128 entries); while labels still consolidate
        // (level 1) a row where neither the own label nor the vote's
        // candidate leads its prefix is left to the CTA kernel unread
        if (b_lo + lane <= b_hi) {
            const Quad q = load_quad(a, b_lo + lane, lo, hi, x.vb);
            own_weight(q, x.own, ow, tw);
            vote_quad(q, vt);
        }
        bool hopeless = false;
        if (lvl == 1 && b_hi - b_lo >= 32) {
            const uint32_t pow_ = __reduce_add_sync(FULL, ow), ptw = __reduce_add_sync(FULL, tw);
            const Vote pv = warp_vote_state(vt);
            hopeless = 2ull * pow_ <= (unsigned long long)ptw && 4ull * pv.n < (unsigned long long)ptw;
        }
        bool settled = false;
        int32_t label = x.own;
        if (!hopeless) {
#pragma unroll 4
            for (int64_t blk = b_lo + 32 + lane; blk <= b_hi; blk += 32) {
                const Quad q = load_quad(a, blk, lo, hi, x.vb);
                own_weight(q, x.own, ow, tw);
                vote_quad(q, vt);
            }
            ow = __reduce_add_sync(FULL, ow);  // row sums < 2^31
            tw = __reduce_add_sync(FULL, tw);
            settled = 2ull * ow > (unsigned long long)tw;
        }
        if (!settled && !hopeless) {
            // the vote's candidate, proven by its surplus or verified by a
            // second read of the row
            vt = warp_vote_state(vt);
            if (vt.n && vt.c != x.own) {
                label = vt.c;
                if (vote_proven(vt.n, tw)) {
                    settled = true;
                } else if (vote_worth_counting(vt.n, tw)) {
                    uint32_t cw = 0u;
#pragma unroll 4
                    for (int64_t blk = (lo >> 2) + lane; blk <= (hi - 1) >> 2; blk += 32)
                        cw += label_weight(load_quad(a, blk, lo, hi, x.vb), vt.c);
                    cw = __reduce_add_sync(FULL, cw);
                    settled = 2ull * cw > (unsigned long long)tw;
                }
            }
        }
        if (lane == 0) {
            a.vmaj[x.v] = settled ? 1 : 0;
            if (!MULTI && !settled && a.cpos) a.cpos[atomicAdd(a.ccount, 1)] = (int32_t)item;
            if (settled) {
                a.lab_out[x.v] = label;
                if (label != x.own) {
                    if (MULTI)
                        atomicAdd(a.changed + x.g, 1);
                    else
                        atomicAdd(a.changed, 1);
                }
            }
        }
    }
}

// the pre-pass over a bucket's list, when the sweep tries the majority test
template <bool MULTI>
int launch_major(const SweepArgs &a, int num_sms, cudaStream_t st)
{
    if (!a.vmaj || !a.majority || a.identity || a.len <= 0) return 0;
    if (!MULTI && a.ccount && cudaMemsetAsync(a.ccount, 0, sizeof(int32_t), st) != cudaSuccess)
        return -1;
    const int64_t blocks = (a.len + 7) / 8;
    k_major_rows<MULTI><<<(int)(blocks < num_sms * 8 ? blocks : num_sms * 8), 256, 0, st>>>(a);
    return 1;
}

// ----------------------------------------------------------------------------
// hub bucket, rows longer than HUB_ONE_MAX: segments, then label partitions
// ----------------------------------------------------------------------------

// Add (l, s, ~first position) to a row's fallback table of 2^glg global slots.
// Returns the slot when this call claimed it, -1 otherwise.
__device__ __forceinline__ int64_t global_add(unsigned long long *gk, uint32_t *gp, int glg,
                                              int32_t l, uint32_t s, uint32_t np)
{
    const uint32_t mask = (1u << glg) - 1u;
    const unsigned long long key = (unsigned long long)((uint32_t)l + 1u) << 32;
    uint32_t h = slot_hash(l, glg);
    for (int i = 0; i <= (int)mask; ++i) {
        const unsigned long long cur = atomicCAS(gk + h, 0ull, key | s);
        if (cur == 0ull) {
            atomicMax(gp + h, np);
            return h;
        }
        if ((cur & 0xFFFFFFFF00000000ull) == key) {
            atomicAdd(gk + h, (unsigned long long)s);  // the sum is the low word
            atomicMax(gp + h, np);
            return -1;
        }
        h = (h + 1) & mask;
    }
    return -1;  // unreachable: the table holds at least 2d slots
}

// Partition of label l among np: the 32-bit finaliser of MurmurHash3
// (Appleby) and a multiply-shift range reduction, independent of slot_hash.
__device__ __forceinline__ uint32_t part_of(int32_t l, uint32_t np)
{
    uint32_t h = (uint32_t)l;
    h ^= h >> 16;
    h *= 0x85EBCA6Bu;
    h ^= h >> 13;
    h *= 0xC2B2AE35u;
    h ^= h >> 16;
    return (uint32_t)(((uint64_t)h * np) >> 32);
}

// In-place exclusive scan of c[0..n) (n <= HUB_PMAX) by NT threads; c[n]
// receives the total.
template <int NT>
__device__ __forceinline__ void block_scan_counts(int32_t *c, int n, int32_t *s_w)
{
    constexpr int PER = (HUB_PMAX + NT - 1) / NT;
    const int t = threadIdx.x, lane = t & 31, w = t >> 5;
    int v[PER];
    int sum = 0;
#pragma unroll
    for (int k = 0; k < PER; ++k) {
        const int q = t * PER + k;
        v[k] = q < n ? c[q] : 0;
        sum += v[k];
    }
    int inc = sum;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(FULL, inc, o);
        if (lane >= o) inc += y;
    }
    if (lane == 31) s_w[w] = inc;
    __syncthreads();
    if (w == 0) {
        const int x = lane < NT / 32 ? s_w[lane] : 0;
        int xi = x;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(FULL, xi, o);
            if (lane >= o) xi += y;
        }
        if (lane < NT / 32) s_w[lane] = xi - x;
        if (lane == 31) s_w[NT / 32] = xi;
    }
    __syncthreads();
    int run = s_w[w] + inc - sum;
#pragma unroll
    for (int k = 0; k < PER; ++k) {
        const int q = t * PER + k;
        if (q < n) c[q] = run;
        run += v[k];
    }
    if (t == 0) c[n] = s_w[NT / 32];
    __syncthreads();
}

// Majority pre-pass over the segments of the long rows: each segment adds its
// row's own-label weight and total weight into the row's counters and stores
// its weighted majority vote, so that the segment and partition passes can
// skip rows where one label holds more than half of the weight (that label is
// then the row's unique maximum).  Counters per long-row task (hmaj, 4
// words): own-label weight, total weight, candidate weight, candidate.
template <bool MULTI>
__global__ void __launch_bounds__(HUB_THREADS) k_hub_major(SweepArgs a)
{
    constexpr int NT = HUB_THREADS;
    if (a.stop && *a.stop) return;  // launched past the end of the run
    __shared__ uint32_t s_sum[2 * (NT / 32)];
    __shared__ Vote s_vote[NT / 32];
    for (int64_t item = blockIdx.x; item < a.hsegs; item += gridDim.x) {
        const int64_t ti = __ldg(a.hseg_task + item);
        const HubTask t = a.htask[ti];
        Vtx x;
        // a pre-pass costs under a tenth of a high-cardinality segment pass
        if (!load_task<MULTI>(a, t, x) || !try_majority(a, x.g)) continue;  // uniform
        const int64_t lo = x.e0 + (int64_t)(item - t.seg0) * HUB_SEG;
        const int64_t hi = min(lo + HUB_SEG, x.e0 + x.d);
        uint32_t ow = 0u, tw = 0u;
        Vote vt;
        for (int64_t blk = (lo >> 2) + threadIdx.x; blk <= (hi - 1) >> 2; blk += NT) {
            const Quad q = load_quad(a, blk, lo, hi, x.vb);
            own_weight(q, x.own, ow, tw);
            vote_quad(q, vt);
        }
        vt = warp_vote_state(vt);
        if ((threadIdx.x & 31) == 0) s_vote[threadIdx.x >> 5] = vt;
        const uint2 s2 = block_sum2<NT>(ow, tw, s_sum);  // its barriers publish s_vote
        if (threadIdx.x == 0) {
            Vote m;
            for (int k = 0; k < NT / 32; ++k) m = vote_merge(m, s_vote[k]);
            a.hvote[item] = make_int2(m.c, (int32_t)m.n);
            atomicAdd(a.hmaj + 4 * ti, s2.x);
            atomicAdd(a.hmaj + 4 * ti + 1, s2.y);
        }
    }
}

// Second pre-pass over the segments of the long rows whose own label failed:
// the row's candidate (its segments' votes merged in segment order, the same
// in every segment) has its weight counted segment by segment.
template <bool MULTI>
__global__ void __launch_bounds__(HUB_THREADS) k_hub_candw(SweepArgs a)
{
    constexpr int NT = HUB_THREADS;
    if (a.stop && *a.stop) return;  // launched past the end of the run
    __shared__ uint32_t s_sum[2 * (NT / 32)];
    __shared__ int32_t s_c;
    for (int64_t item = blockIdx.x; item < a.hsegs; item += gridDim.x) {
        const int64_t ti = __ldg(a.hseg_task + item);
        const HubTask t = a.htask[ti];
        Vtx x;
        if (!load_task<MULTI>(a, t, x) || !try_majority(a, x.g)) continue;  // uniform
        const uint32_t ow = __ldcg(a.hmaj + 4 * ti), tot = __ldcg(a.hmaj + 4 * ti + 1);
        if (2ull * ow > (unsigned long long)tot) continue;  // the own label holds
        if (threadIdx.x == 0) {
            Vote m;
            for (int k = 0; k < t.nseg; ++k) {
                const int2 v = __ldcg(a.hvote + t.seg0 + k);
                m = vote_merge(m, Vote{v.x, (uint32_t)v.y});
            }
            s_c = m.n && m.c != x.own && vote_worth_counting(m.n, tot) ? m.c : EMPTY;
            if (s_c != EMPTY && vote_proven(m.n, tot)) {
                // proven by its surplus: the first segment records it, the
                // others count nothing
                if (item == t.seg0) {
                    a.hmaj[4 * ti + 2] = tot;
                    a.hmaj[4 * ti + 3] = (uint32_t)m.c;
                }
                s_c = EMPTY;
            }
        }
        __syncthreads();
        const int32_t c = s_c;
        __syncthreads();
        if (c == EMPTY) continue;  // uniform
        const int64_t lo = x.e0 + (int64_t)(item - t.seg0) * HUB_SEG;
        const int64_t hi = min(lo + HUB_SEG, x.e0 + x.d);
        uint32_t cw = 0u;
        for (int64_t blk = (lo >> 2) + threadIdx.x; blk <= (hi - 1) >> 2; blk += NT)
            cw += label_weight(load_quad(a, blk, lo, hi, x.vb), c);
        const uint2 s2 = block_sum2<NT>(cw, 0u, s_sum);
        if (threadIdx.x == 0) {
            atomicAdd(a.hmaj + 4 * ti + 2, s2.x);
            if (item == t.seg0) a.hmaj[4 * ti + 3] = (uint32_t)c;
        }
    }
}

// the label of the long row of task ti if one label holds more than half of
// its weight (pre-pass counters), else EMPTY
template <bool MULTI>
__device__ __forceinline__ int32_t hub_settled(const SweepArgs &a, int64_t ti, int32_t g,
                                               int32_t own)
{
    if (!a.hmaj || !try_majority(a, g)) return EMPTY;
    const uint32_t *h = a.hmaj + 4 * ti;
    const uint32_t ow = __ldcg(h), tot = __ldcg(h + 1);
    if (2ull * ow > (unsigned long long)tot) return own;
    if (2ull * __ldcg(h + 2) > (unsigned long long)tot) return (int32_t)__ldcg(h + 3);
    return EMPTY;
}

// Long rows that one label holds by majority take that label here (and
// count as changed if it differs); *open receives the number of the other
// long rows, and the segment and partition passes return at once when there
// is none.  One block.
template <bool MULTI>
__global__ void __launch_bounds__(1024) k_hub_open(SweepArgs a, int32_t *open)
{
    if (a.stop && *a.stop) return;  // launched past the end of the run
    __shared__ int32_t s_n, s_ch;
    if (threadIdx.x == 0) s_n = s_ch = 0;
    __syncthreads();
    int32_t k = 0, ch = 0;
    for (int64_t ti = threadIdx.x; ti < a.hmulti; ti += blockDim.x) {
        const HubTask t = a.htask[ti];
        Vtx x;
        if (!load_task<MULTI>(a, t, x)) continue;
        const int32_t maj = hub_settled<MULTI>(a, ti, x.g, x.own);
        if (maj == EMPTY) {
            ++k;
            continue;
        }
        a.lab_out[x.v] = maj;
        if (maj != x.own) {
            if (MULTI)
                atomicAdd(a.changed + x.g, 1);
            else
                ++ch;
        }
    }
    k = (int32_t)__reduce_add_sync(FULL, (uint32_t)k);
    ch = (int32_t)__reduce_add_sync(FULL, (uint32_t)ch);
    if ((threadIdx.x & 31) == 0) {
        if (k) atomicAdd(&s_n, k);
        if (ch) atomicAdd(&s_ch, ch);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        if (open) *open = s_n;
        if (!MULTI && s_ch) atomicAdd(a.changed, s_ch);
    }
}

// Segment pass: a segment's entries are aggregated in the shared table and
// written out as (label, sum, ~first position) records grouped by partition,
// with the partition offsets.  In an identity sweep the segment's own winner
// is its only record.
template <bool MULTI>
__global__ void __launch_bounds__(HUB_THREADS, 2) k_hub_seg(SweepArgs a)
{
    if (a.stop && *a.stop) return;  // launched past the end of the run
    if (a.hmaj && a.hopen && *a.hopen == 0) return;  // every long row is settled
    constexpr int NT = HUB_THREADS;
    constexpr int LG = 13;
    static_assert((1 << LG) == HUB_TABLE && HUB_TABLE >= 2 * HUB_SEG, "hub table size");
    extern __shared__ int32_t smem[];
    int32_t *tk = smem;
    int32_t *ts = tk + HUB_TABLE;
    uint32_t *tp = reinterpret_cast<uint32_t *>(ts + HUB_TABLE);
    __shared__ Cand s_red[NT / 32];
    __shared__ int32_t s_cnt[HUB_PMAX + 1];
    __shared__ int32_t s_w[NT / 32 + 1];

    for (int j = threadIdx.x; j < HUB_TABLE; j += NT) {
        tk[j] = EMPTY;
        ts[j] = 0;
        tp[j] = 0;
    }
    __syncthreads();
    for (int64_t item = blockIdx.x; item < a.hsegs; item += gridDim.x) {
        const int64_t ti = __ldg(a.hseg_task + item);
        const HubTask t = a.htask[ti];
        Vtx x;
        if (!load_task<MULTI>(a, t, x)) continue;  // block-uniform
        const int seg = (int)(item - t.seg0);
        const int64_t lo = x.e0 + (int64_t)seg * HUB_SEG;
        const int64_t hi = min(lo + HUB_SEG, x.e0 + x.d);
        const int np = t.npart;
        int32_t *out = a.hrec + item * (HUB_REC * HUB_SEG);
        int32_t *poff = a.hpoff + t.poff0 + (int64_t)seg * (np + 1);
        if (hub_settled<MULTI>(a, ti, x.g, x.own) != EMPTY) {  // no records
            for (int q = threadIdx.x; q <= np; q += NT) poff[q] = 0;
            continue;
        }
        if (a.identity) {
            const uint64_t ktv = stream_at(a.key_t, (uint64_t)x.lv + 1);
            const Cand best = block_argmax<NT>(identity_best<NT>(a, x.e0, lo, hi, ktv, threadIdx.x),
                                               a.strict, s_red);
            if (threadIdx.x == 0) {
                s_cnt[0] = best.sum > 0 ? (int)part_of(best.label, (uint32_t)np) : -1;
                out[0] = best.label;
                out[1] = (int)best.sum;
                out[2] = (int)best.npos;
            }
            __syncthreads();
            const int bp = s_cnt[0];
            for (int q = threadIdx.x; q <= np; q += NT) poff[q] = (bp >= 0 && q > bp) ? 1 : 0;
            __syncthreads();
            continue;
        }
        accumulate_range<NT>(a, x.e0, lo, hi, x.vb, tk, ts, tp, LG);
        for (int q = threadIdx.x; q < np; q += NT) s_cnt[q] = 0;
        __syncthreads();
        for (int j = threadIdx.x; j < HUB_TABLE; j += NT)
            if (tk[j] != EMPTY) atomicAdd(&s_cnt[part_of(tk[j], (uint32_t)np)], 1);
        __syncthreads();
        block_scan_counts<NT>(s_cnt, np, s_w);
        for (int q = threadIdx.x; q <= np; q += NT) poff[q] = s_cnt[q];
        __syncthreads();
        for (int j = threadIdx.x; j < HUB_TABLE; j += NT) {
            const int32_t key = tk[j];
            if (key != EMPTY) {
                const int at = atomicAdd(&s_cnt[part_of(key, (uint32_t)np)], 1);
                out[HUB_REC * at] = key;
                out[HUB_REC * at + 1] = ts[j];
                out[HUB_REC * at + 2] = (int)tp[j];
                tk[j] = EMPTY;
                ts[j] = 0;
                tp[j] = 0;
            }
        }
        __syncthreads();
    }
}

// Partition pass: the records of one partition of a row, from every segment,
// are merged in the shared table (a label without room goes to the row's
// fallback table); its best candidate is stored, and the CTA finishing the
// row's last partition picks the best of the partition bests and of the
// fallback slots.
template <bool MULTI>
__global__ void __launch_bounds__(HUB_THREADS, 2) k_hub_merge(SweepArgs a)
{
    if (a.stop && *a.stop) return;  // launched past the end of the run
    if (a.hmaj && a.hopen && *a.hopen == 0) return;  // every long row is settled
    constexpr int NT = HUB_THREADS;
    constexpr int LG = 13;
    constexpr int PROBE = 256;
    extern __shared__ int32_t smem[];
    int32_t *tk = smem;
    int32_t *ts = tk + HUB_TABLE;
    uint32_t *tp = reinterpret_cast<uint32_t *>(ts + HUB_TABLE);
    __shared__ Cand s_red[NT / 32];
    __shared__ uint32_t s_u[NT / 32 + 1];
    __shared__ int s_last;
    __shared__ int32_t s_rb[NT], s_re[NT];
    // partition best of item i: sum, ~first position, label | non-strict key
    uint4 *pbest = reinterpret_cast<uint4 *>(a.hpbest);

    for (int j = threadIdx.x; j < HUB_TABLE; j += NT) {
        tk[j] = EMPTY;
        ts[j] = 0;
        tp[j] = 0;
    }
    __syncthreads();
    uint32_t my_changed = 0;
    for (int64_t item = blockIdx.x; item < a.hparts; item += gridDim.x) {
        const int64_t ti = __ldg(a.hpart_task + item);
        const HubTask t = a.htask[ti];
        Vtx x;
        if (!load_task<MULTI>(a, t, x)) continue;  // block-uniform
        const int p = (int)(item - t.part0);
        const int np = t.npart;
        // a row that one label holds by majority took it in k_hub_open
        if (hub_settled<MULTI>(a, ti, x.g, x.own) != EMPTY) continue;
        const uint64_t ktv = stream_at(a.key_t, (uint64_t)x.lv + 1);
        const int glg = ilog2_ceil(2u * (uint32_t)x.d);
        unsigned long long *gk = a.hkey + t.tab;
        uint32_t *gp = a.hnpos + t.tab;
        int32_t *gu = a.hused + t.tab / 2;
        // this partition's run in every segment: run bounds are staged for up
        // to NT segments at a time, then all threads share each run
        for (int s0 = 0; s0 < t.nseg; s0 += NT) {
            const int ns = min(NT, t.nseg - s0);
            if ((int)threadIdx.x < ns) {
                const int32_t *po = a.hpoff + t.poff0 + (int64_t)(s0 + threadIdx.x) * (np + 1);
                s_rb[threadIdx.x] = __ldg(po + p);
                s_re[threadIdx.x] = __ldg(po + p + 1);
            }
            __syncthreads();
            for (int s = 0; s < ns; ++s) {
                const int32_t *rec = a.hrec + (int64_t)(t.seg0 + s0 + s) * (HUB_REC * HUB_SEG);
                for (int r = s_rb[s] + threadIdx.x; r < s_re[s]; r += NT) {
                    const int4 R = make_int4(__ldg(rec + HUB_REC * r), __ldg(rec + HUB_REC * r + 1),
                                             __ldg(rec + HUB_REC * r + 2), 0);
                    if (!table_add(tk, ts, tp, LG, PROBE, R.x, R.y, 0xFFFFFFFFu - (uint32_t)R.z)) {
                        const int64_t c =
                            global_add(gk, gp, glg, R.x, (uint32_t)R.y, (uint32_t)R.z);
                        if (c >= 0) gu[atomicAdd(a.hnused + ti, 1)] = (int32_t)c;
                    }
                }
            }
            __syncthreads();
        }
        Cand best = block_argmax<NT>(scan_table<NT>(tk, ts, tp, HUB_TABLE, a.strict, ktv, s_u),
                                     a.strict, s_red);
        if (threadIdx.x == 0) {
            pbest[2 * item] = make_uint4(best.sum, best.npos, (uint32_t)best.label, 0u);
            pbest[2 * item + 1] = make_uint4((uint32_t)best.h, (uint32_t)(best.h >> 32), 0u, 0u);
            __threadfence();
            s_last = atomicAdd(a.hdone + ti, 1) == np - 1;
        }
        __syncthreads();
        if (!s_last) continue;

        // the row's last partition: best of the partition bests and fallback slots
        __threadfence();
        const int nused = __ldcg(a.hnused + ti);
        Cand c{0u, 0u, 0ull, EMPTY};
        for (int q = threadIdx.x; q < np; q += NT) {
            const uint4 A = __ldcg(pbest + 2 * (t.part0 + q));
            const uint4 B = __ldcg(pbest + 2 * (t.part0 + q) + 1);
            const Cand y{A.x, A.y, (uint64_t)B.x | ((uint64_t)B.y << 32), (int32_t)A.z};
            if (better(y, c)) c = y;
        }
        for (int u = threadIdx.x; u < nused; u += NT) {
            const int32_t slot = __ldcg(gu + u);
            const unsigned long long kv = __ldcg(gk + slot);
            const int32_t label = (int32_t)((uint32_t)(kv >> 32) - 1u);
            const Cand y{(uint32_t)kv, __ldcg(gp + slot),
                         a.strict ? 0ull : stream_at(ktv, (uint64_t)label + 1), label};
            if (better(y, c)) c = y;
            gk[slot] = 0ull;
            gp[slot] = 0u;
        }
        best = block_argmax<NT>(c, a.strict, s_red);
        if (threadIdx.x == 0) {
            a.lab_out[x.v] = best.label;
            if (best.label != x.own) {
                if (MULTI)
                    atomicAdd(a.changed + x.g, 1);
                else
                    ++my_changed;
            }
            a.hdone[ti] = 0;
            a.hnused[ti] = 0;
        }
        __syncthreads();
    }
    if (!MULTI && threadIdx.x == 0 && my_changed) atomicAdd(a.changed, (int)my_changed);
}

// CTAs of nt threads and smem bytes of dynamic shared memory that fit one SM
// at once (at most 32 CTAs, 2048 threads and 227 KB per SM)
constexpr int resident_ctas(int nt, size_t smem)
{
    const int by_threads = 2048 / nt < 32 ? 2048 / nt : 32;
    const int by_smem = (int)((size_t)232448 / (smem + 1024));
    return by_threads < by_smem ? by_threads : by_smem;
}

template <bool MULTI>
int launch(int bucket, const SweepArgs &a, int num_sms, cudaStream_t st)
{
    constexpr size_t cta_smem = (size_t)CTA_TABLE * 8;
    constexpr size_t cta2_smem = (size_t)CTA2_TABLE * 8;
    constexpr size_t hubcta_smem = (size_t)HUB_TABLE * 8;
    constexpr size_t hub_smem = (size_t)HUB_TABLE * 12;
    if (a.len <= 0) return 0;
    int64_t blocks = 0;
    int n = 1, m = 0;
    switch (bucket) {
    case 0: {
        SweepArgs b = a;
        b.tile_rows = small_tile_rows(a.len, a.small_mean_deg, num_sms);
        blocks = ((a.len + b.tile_rows - 1) / b.tile_rows + 7) / 8;
        k_small<MULTI><<<(int)(blocks < num_sms * 16 ? blocks : num_sms * 16), 256, 0, st>>>(b);
        break;
    }
    case 1:
        blocks = (a.len + 7) / 8;
        k_warp<MULTI><<<(int)(blocks < num_sms * 8 ? blocks : num_sms * 8), 256, 0, st>>>(a);
        break;
    case 2:
        blocks = a.len;
        if ((m = launch_major<MULTI>(a, num_sms, st)) < 0) return -1;
        n += m;
        blocks = std::min<int64_t>(blocks, (int64_t)num_sms * resident_ctas(CTA_THREADS, cta_smem));
        k_cta<CTA_THREADS, CTA_TABLE, MULTI><<<(int)blocks, CTA_THREADS, cta_smem, st>>>(a);
        break;
    case 3:
        blocks = a.len;
        if ((m = launch_major<MULTI>(a, num_sms, st)) < 0) return -1;
        n += m;
        blocks =
            std::min<int64_t>(blocks, (int64_t)num_sms * resident_ctas(CTA2_THREADS, cta2_smem));
        k_cta<CTA2_THREADS, CTA2_TABLE, MULTI><<<(int)blocks, CTA2_THREADS, cta2_smem, st>>>(a);
        break;
    default: {
        n = 0;
        if (a.hmulti > 0) {  // long rows: segments, then label partitions
            const int64_t cap = (int64_t)num_sms * 2;
            SweepArgs h = a;
            if (a.majority && !a.identity && a.hmaj) {
                if (cudaMemsetAsync(a.hmaj, 0, (size_t)a.hmulti * 4 * sizeof(uint32_t), st) !=
                    cudaSuccess)
                    return -1;
                k_hub_major<MULTI>
                    <<<(int)(a.hsegs < cap * 2 ? a.hsegs : cap * 2), HUB_THREADS, 0, st>>>(a);
                k_hub_candw<MULTI>
                    <<<(int)(a.hsegs < cap * 2 ? a.hsegs : cap * 2), HUB_THREADS, 0, st>>>(a);
                n += 2;
                k_hub_open<MULTI><<<1, 1024, 0, st>>>(a, a.hopen);  // writes settled labels
                ++n;
            } else {
                h.hmaj = nullptr;
            }
            k_hub_seg<MULTI><<<(int)(a.hsegs < cap ? a.hsegs : cap), HUB_THREADS, hub_smem, st>>>(h);
            k_hub_merge<MULTI>
                <<<(int)(a.hparts < cap ? a.hparts : cap), HUB_THREADS, hub_smem, st>>>(h);
            n += 2;
        }
        if (a.len > a.hmulti) {  // the other hub rows: one CTA each
            SweepArgs b = a;
            b.list = a.list + a.hmulti;
            b.rp = a.rp + a.hmulti;
            b.len = a.len - a.hmulti;
            blocks = b.len < (int64_t)num_sms * 2 ? b.len : (int64_t)num_sms * 2;
            if ((m = launch_major<MULTI>(b, num_sms, st)) < 0) return -1;
            n += m;
            k_cta<HUB_THREADS, HUB_TABLE, MULTI><<<(int)blocks, HUB_THREADS, hubcta_smem, st>>>(b);
            ++n;
        }
        break;
    }
    }
    return cudaGetLastError() == cudaSuccess ? n : -1;
}

template <bool MULTI>
int prepare()
{
    if (cudaFuncSetAttribute(k_cta<CTA_THREADS, CTA_TABLE, MULTI>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)((size_t)CTA_TABLE * 8)) != cudaSuccess)
        return -1;
    if (cudaFuncSetAttribute(k_cta<CTA2_THREADS, CTA2_TABLE, MULTI>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)((size_t)CTA2_TABLE * 8)) != cudaSuccess)
        return -1;
    if (cudaFuncSetAttribute(k_cta<HUB_THREADS, HUB_TABLE, MULTI>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)((size_t)HUB_TABLE * 8)) != cudaSuccess)
        return -1;
    if (cudaFuncSetAttribute(k_hub_seg<MULTI>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)((size_t)HUB_TABLE * 12)) != cudaSuccess)
        return -1;
    if (cudaFuncSetAttribute(k_hub_merge<MULTI>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)((size_t)HUB_TABLE * 12)) != cudaSuccess)
        return -1;
    return 0;
}

}  // namespace


int sweep_prepare() { return prepare<false>() | prepare<true>(); }

int sweep_launch(int bucket, const SweepArgs &a, bool multi, int num_sms, cudaStream_t st)
{
    return multi ? launch<true>(bucket, a, num_sms, st) : launch<false>(bucket, a, num_sms, st);
}

int barrier_probe_launch(unsigned *bar, int32_t *err, uint32_t spin_limit, cudaStream_t st)
{
    void *args[] = {&bar, &err, &spin_limit};
    if (cudaLaunchCooperativeKernel((const void *)k_barrier_probe, dim3(4), dim3(32), args, 0, st) !=
        cudaSuccess)
        return -1;
    return 1;
}

int small_waves_launch(const SweepArgs &a, const int32_t *wlist, const int64_t *wstart,
                       const int64_t *wcount, int64_t max_len, int32_t max_degree, unsigned *bar,
                       int32_t *err, int num_sms, cudaStream_t st)
{
    // resident CTAs per SM (thread-safe one-time initialisation)
    static const int per_sm = [] {
        int n = 0;
        return cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_small_waves, 256, 0) ==
                       cudaSuccess
                   ? n
                   : 0;
    }();
    static const int per_sm_tiny = [] {
        int n = 0;
        return cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_tiny_waves, 256, 0) ==
                       cudaSuccess
                   ? n
                   : 0;
    }();
    // every row of at most TINY entries: the kernel that loads the next wave's
    // rows before each barrier
    const bool tiny = max_degree <= TINY && !a.spoken;
    const int ps = tiny ? per_sm_tiny : per_sm;
    if (ps <= 0) return -1;
    SweepArgs b = a;
    b.tile_rows = tiny ? 32 : small_tile_rows(max_len, a.small_mean_deg, num_sms);
    const int64_t want = ((max_len + b.tile_rows - 1) / b.tile_rows + 7) / 8;
    const int64_t cap = (int64_t)ps * num_sms;
    const int grid = (int)(want < 1 ? 1 : (want < cap ? want : cap));
    void *args[] = {&b, &wlist, &wstart, &wcount, &bar, &err};
    const void *fn = tiny ? (const void *)k_tiny_waves : (const void *)k_small_waves;
    if (cudaLaunchCooperativeKernel(fn, dim3(grid), dim3(256), args, 0, st) != cudaSuccess)
        return -1;
    return 1;
}

}  // namespace lp
