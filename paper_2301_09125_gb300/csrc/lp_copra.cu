// COPRA, community overlap propagation (Sec. 3.3), for a single graph.
//
// A vertex holds at most L (label, belonging) pairs; belongings are integers
// in units of 2^-16 that sum to exactly COPRA_ONE = 2^16, stored by
// decreasing belonging (equal belongings by first appearance), the first pair
// being the vertex's best label.  In an iteration a listener v sums, over its
// row's entries (u, w) and the pairs (l, b) of u's set, T(l) += w * b (its
// own labels are not added); it keeps the labels with L * T(l) >= W * 2^16
// (W = the row's summed weight), else the best label alone (largest T, ties
// by RAK's strict or non-strict rule on first appearance / tie key), divides
// the kept T by their sum in fixed point (floor, the remainder to the best
// kept label) and stores them sorted.  A vertex without edges is its own
// community.  Asynchronous runs go in waves as RAK's do.
//
// Rows of at most 32 pairs (with L <= 8) take 8 lanes (four rows per warp)
// and a 64-slot table, rows of at most CPW_PAIRS pairs (with L <= 32) one warp
// and a 256-slot table of the warp's own in shared memory; longer rows of at most
// CP_PAIRS pairs take one CTA and a 4096-slot shared table; longer ones one
// CTA each with a region of a global table (a launch of copra_big_ctas()
// CTAs).  Rows that need a CTA are listed once per run, by wave and kind, so
// that a launch visits only its own rows.  In shared memory T(l) is summed
// exactly in two 32-bit words (the carry out of the low word is added to the
// high word), which keeps every shared atomic a native 32-bit one; a
// label's first appearance, row position * 64 + pair index (which orders
// the pairs as the row scan meets them), fits 32 bits there.
#include <type_traits>

#include "lp_device.cuh"
#include "lp_internal.cuh"

namespace lp {
namespace {

constexpr int CP_T = 256;
constexpr int CP_LG = 12;
constexpr int CP_TAB = 1 << CP_LG;    // shared slots per CTA
constexpr int CP_PAIRS = CP_TAB / 2;  // rows of at most this many pairs use shared memory
constexpr int CPW_LG = 8;
constexpr int CPW_TAB = 1 << CPW_LG;    // shared slots per warp
constexpr int CPW_PAIRS = CPW_TAB / 2;  // rows of at most this many pairs take one warp
constexpr int CPW_WARPS = 8;            // warps per block of the warp kernel
constexpr int CPW_MAX_L = 32;           // the warp kernel holds a set in one lane per pair

struct CopraArgs {
    const int32_t *off, *idx, *wts;  // the graph's CSR (wts null = unit weights)
    int32_t n;
    int32_t L;
    const int32_t *cur_l;  // previous iteration's sets (n * L)
    const uint32_t *cur_b;
    int32_t *nxt_l;        // this iteration's sets
    uint32_t *nxt_b;
    uint32_t waves, wave_k;
    uint64_t magic;        // fastmod constant of waves
    int strict;
    uint64_t key_t;        // non-strict key of this iteration
    int32_t *changed;
    // the rows of this wave a CTA kernel takes (list, count; or the count
    // at nrows_dev when set)
    const int32_t *rows;
    int64_t nrows;
    const int32_t *nrows_dev;
    // rows that outgrew the long-row kernel's shared table: count at ovf[0],
    // the rows after it
    int32_t *ovf;
    // long rows: a table of 2^glg_max slots per CTA
    int32_t *gkey;
    unsigned long long *gsum, *gfirst;
    int32_t glg_max;
};

struct CpCand {
    unsigned long long t, h, first;
    int32_t slot;
};

// strictly better as the best label: larger T, then (non-strict) smaller key,
// then earlier first appearance
__device__ __forceinline__ bool cp_better(const CpCand &x, const CpCand &y)
{
    if (x.slot < 0) return false;
    if (y.slot < 0) return true;
    if (x.t != y.t) return x.t > y.t;
    if (x.h != y.h) return x.h < y.h;
    return x.first < y.first;
}

__device__ __forceinline__ CpCand cp_shfl(const CpCand &c, int o)
{
    CpCand r;
    r.t = __shfl_xor_sync(FULL, c.t, o);
    r.h = __shfl_xor_sync(FULL, c.h, o);
    r.first = __shfl_xor_sync(FULL, c.first, o);
    r.slot = __shfl_xor_sync(FULL, c.slot, o);
    return r;
}

__device__ __forceinline__ CpCand cp_warp_best(CpCand c)
{
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) {
        const CpCand y = cp_shfl(c, o);
        if (cp_better(y, c)) c = y;
    }
    return c;
}

__device__ __forceinline__ unsigned long long cp_warp_sum(unsigned long long v)
{
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) v += __shfl_xor_sync(FULL, v, o);
    return v;
}

// floor(t * 2^16 / tk) for 0 <= t <= tk < 2^47 (a belonging in units of
// 2^-16, at most 2^16): a single-precision estimate, off by at most one
// (each rounding of t, tk and their quotient is within 2^-24 relative, so
// the estimate is within 2^16 * 3 * 2^-24 of the quotient), then corrected
// with exact 64-bit integer arithmetic.
__device__ __forceinline__ uint32_t cp_frac(unsigned long long t, unsigned long long tk)
{
    uint32_t q = (uint32_t)(((float)t * 65536.0f) / (float)tk);
    if (q > COPRA_ONE) q = COPRA_ONE;
    long long r = (long long)(t << 16) - (long long)q * (long long)tk;
    while (r < 0) {
        --q;
        r += (long long)tk;
    }
    while (r >= (long long)tk) {
        ++q;
        r -= (long long)tk;
    }
    return q;
}

// Wave of vertex v (0 in synchronous runs).
__device__ __forceinline__ uint32_t cp_wave(const CopraArgs &a, int32_t v)
{
    return a.waves > 1 ? fastmod((uint32_t)v, a.magic, a.waves) : 0u;
}

// Shared table of 2^lg slots: label, T in two 32-bit words, first appearance.
struct CpShared {
    int32_t *key;
    uint32_t *lo, *hi, *first;
    __device__ __forceinline__ unsigned long long t(int j) const
    {
        return ((unsigned long long)hi[j] << 32) | lo[j];
    }
    __device__ __forceinline__ void clear(int j) const
    {
        key[j] = EMPTY;
        lo[j] = 0u;
        hi[j] = 0u;
        first[j] = 0xFFFFFFFFu;
    }
    // add (label l, value val < 2^48, first appearance f < 2^32); the table
    // has room for every label of the row
    // true when this call claimed the label's slot
    __device__ __forceinline__ bool add(int lg, int32_t l, unsigned long long val,
                                        unsigned long long f) const
    {
        const uint32_t mask = (1u << lg) - 1u;
        volatile int32_t *vk = key;
        uint32_t h = slot_hash(l, lg);
        for (uint32_t i = 0; i <= mask; ++i) {
            int32_t cur = vk[h];
            bool claimed = false;
            if (cur == EMPTY) {
                cur = atomicCAS(key + h, EMPTY, l);
                if (cur == EMPTY) {
                    cur = l;
                    claimed = true;
                }
            }
            if (cur == l) {
                const uint32_t vlo = (uint32_t)val, vhi = (uint32_t)(val >> 32);
                const uint32_t old = atomicAdd(lo + h, vlo);
                // the low word wrapped: the carry goes to the high word, so
                // hi * 2^32 + lo is the exact sum of every value added
                const uint32_t up = vhi + (old + vlo < old ? 1u : 0u);
                if (up) atomicAdd(hi + h, up);
                atomicMin(first + h, (uint32_t)f);
                return claimed;
            }
            h = (h + 1) & mask;
        }
        return false;
    }
};

// Global table region of 2^lg slots (native 64-bit atomics).
struct CpGlobal {
    int32_t *key;
    unsigned long long *sum, *first;
    __device__ __forceinline__ unsigned long long t(int64_t j) const { return sum[j]; }
    __device__ __forceinline__ void clear(int64_t j) const
    {
        key[j] = EMPTY;
        sum[j] = 0ull;
        first[j] = ~0ull;
    }
    __device__ __forceinline__ bool add(int lg, int32_t l, unsigned long long val,
                                        unsigned long long f) const
    {
        const uint32_t mask = (1u << lg) - 1u;
        volatile int32_t *vk = key;
        uint32_t h = slot_hash(l, lg);
        for (uint32_t i = 0; i <= mask; ++i) {
            int32_t cur = vk[h];
            bool claimed = false;
            if (cur == EMPTY) {
                cur = atomicCAS(key + h, EMPTY, l);
                if (cur == EMPTY) {
                    cur = l;
                    claimed = true;
                }
            }
            if (cur == l) {
                atomicAdd(sum + h, val);
                atomicMin(first + h, f);
                return claimed;
            }
            h = (h + 1) & mask;
        }
        return false;
    }
};

// f(p, label, belonging) for the pairs of a speaker's set in order, up to its
// first empty pair (sets are prefixes).  Four pairs are loaded at a time, as
// two 16-byte loads when L is a multiple of 4 (a set then starts 16-byte
// aligned), so that a set costs one memory round trip instead of one per
// pair.  The sets read are not written by the launch that reads them.
template <typename F>
__device__ __forceinline__ void cp_each_pair(const int32_t *ul, const uint32_t *ub, uint32_t L,
                                             F &&f)
{
    for (uint32_t p0 = 0; p0 < L; p0 += 4) {
        int32_t l[4];
        uint32_t b[4];
        if ((L & 3u) == 0u) {
            const int4 l4 = __ldg(reinterpret_cast<const int4 *>(ul + p0));
            const uint4 b4 = __ldg(reinterpret_cast<const uint4 *>(ub + p0));
            l[0] = l4.x; l[1] = l4.y; l[2] = l4.z; l[3] = l4.w;
            b[0] = b4.x; b[1] = b4.y; b[2] = b4.z; b[3] = b4.w;
        } else {
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const bool in = p0 + q < L;
                b[q] = in ? __ldg(ub + p0 + q) : 0u;
                l[q] = in ? __ldg(ul + p0 + q) : EMPTY;
            }
        }
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            if (b[q] == 0u) return;
            f(p0 + q, l[q], b[q]);
        }
    }
}

// Best candidate and 64-bit sum over the GS lanes of a group (mask m).
template <int GS>
__device__ __forceinline__ CpCand cp_group_best(CpCand c, unsigned m)
{
#pragma unroll
    for (int o = GS / 2; o >= 1; o >>= 1) {
        CpCand y;
        y.t = __shfl_xor_sync(m, c.t, o);
        y.h = __shfl_xor_sync(m, c.h, o);
        y.first = __shfl_xor_sync(m, c.first, o);
        y.slot = __shfl_xor_sync(m, c.slot, o);
        if (cp_better(y, c)) c = y;
    }
    return c;
}

template <int GS>
__device__ __forceinline__ unsigned long long cp_group_sum(unsigned long long v, unsigned m)
{
#pragma unroll
    for (int o = GS / 2; o >= 1; o >>= 1) v += __shfl_xor_sync(m, v, o);
    return v;
}

// One COPRA step for the rows of wave wave_k with at most 4 GS pairs (rows
// without entries included, L <= GS): a group of GS lanes per vertex (GS =
// 8: four vertices per warp; GS = 32: one), which keeps the kept pairs one
// per lane.  A table of 8 GS slots per group.  The GS = 32 launch takes the
// rows the GS = 8 launch leaves (more than 32 pairs, or L > 8).
template <int GS>
__global__ void __launch_bounds__(CPW_WARPS * 32) k_copra_warp(CopraArgs a)
{
    constexpr int GT = 8 * GS;       // slots per group
    constexpr int GP = 4 * GS;       // pairs per group's row at most
    constexpr int NG = 32 / GS;      // groups per warp
    __shared__ int32_t s_key[CPW_WARPS * CPW_TAB];
    __shared__ uint32_t s_lo[CPW_WARPS * CPW_TAB];
    __shared__ uint32_t s_hi[CPW_WARPS * CPW_TAB];
    __shared__ uint32_t s_first[CPW_WARPS * CPW_TAB];
    static_assert(NG * GT == CPW_TAB, "a warp's groups share its 256 slots");
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const int grp = lane / GS, gl = lane % GS;
    const unsigned gm = GS == 32 ? FULL : (((1u << GS) - 1u) << (grp * GS));
    const int o = wib * CPW_TAB + grp * GT;
    const CpShared tab{s_key + o, s_lo + o, s_hi + o, s_first + o};
    for (int j = gl; j < GT; j += GS) tab.clear(j);
    __syncwarp();

    const uint32_t L = (uint32_t)a.L;
    const int64_t W = a.waves;
    // the wave's vertices (v = wave_k + i W), or the listed rows when a.rows is set
    const int64_t nw = a.rows ? a.nrows
                              : ((int64_t)a.n > (int64_t)a.wave_k
                                     ? ((int64_t)a.n - a.wave_k + W - 1) / W
                                     : 0);
    const int64_t ng = (((int64_t)gridDim.x * blockDim.x) >> 5) * NG;
    uint32_t my_changed = 0;
    for (int64_t i = ((((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5) * NG) + grp; i < nw;
         i += ng) {
        const int32_t v = a.rows ? a.rows[i] : (int32_t)(a.wave_k + i * W);
        const int32_t rs = __ldg(a.off + v), d = __ldg(a.off + v + 1) - rs;
        const int64_t pairs = (int64_t)d * L;
        // group-uniform: the other launch's rows
        if (GS == 32 ? (pairs > CPW_PAIRS || (L <= 8 && pairs <= 32)) : (L > 8 || pairs > GP))
            continue;
        const int32_t prev = a.cur_l[(int64_t)v * L];
        int32_t *out_l = a.nxt_l + (int64_t)v * L;
        uint32_t *out_b = a.nxt_b + (int64_t)v * L;
        if (d == 0) {  // no labels: the vertex is its own community
            for (uint32_t s = gl; s < L; s += GS) {
                out_l[s] = s == 0 ? v : EMPTY;
                out_b[s] = s == 0 ? COPRA_ONE : 0u;
            }
            if (gl == 0 && prev != v) ++my_changed;
            continue;
        }
        const int lg = ilog2_ceil((uint32_t)(2 * pairs));  // 2^lg >= 2 pairs (<= GT)
        const int slots = 1 << lg;
        // T(l) and first appearance over the row's entries and their speakers' pairs
        uint32_t wsum = 0u;
        for (int32_t e = gl; e < d; e += GS) {
            const int32_t u = __ldg(a.idx + rs + e);
            const uint32_t w = a.wts ? (uint32_t)__ldg(a.wts + rs + e) : 1u;
            wsum += w;
            const bool earlier = cp_wave(a, u) < a.wave_k;
            const int32_t *ul = (earlier ? a.nxt_l : a.cur_l) + (int64_t)u * L;
            const uint32_t *ub = (earlier ? a.nxt_b : a.cur_b) + (int64_t)u * L;
            cp_each_pair(ul, ub, L, [&](uint32_t p, int32_t l, uint32_t b) {
                tab.add(lg, l, (unsigned long long)w * b, (uint32_t)e * 64u + p);
            });
        }
        wsum = __reduce_add_sync(gm, wsum);  // < 2^31 (checked at ingest)
        __syncwarp(gm);
        // the labels above the threshold, one per lane from the group's lane 0
        // on, and the best label
        const unsigned long long wt = (unsigned long long)wsum * COPRA_ONE;
        const uint64_t ktv = stream_at(a.key_t, (uint64_t)v + 1);
        CpCand best{0ull, 0ull, 0ull, -1};
        int32_t mine = -1;  // the kept slot this lane holds
        int nk = 0;
        for (int base = 0; base < slots; base += GS) {
            const int j = base + gl;
            bool kept = false;
            if (j < slots) {
                const int32_t l = tab.key[j];
                if (l != EMPTY) {
                    const unsigned long long t = tab.t(j);
                    kept = (unsigned long long)L * t >= wt;
                    const CpCand c{t, a.strict ? 0ull : stream_at(ktv, (uint64_t)l + 1),
                                   (unsigned long long)tab.first[j], j};
                    if (cp_better(c, best)) best = c;
                }
            }
            const unsigned m = (__ballot_sync(gm, kept) & gm) >> (grp * GS);
            const int nm = __popc(m);
            // lane nk + k of the group takes the slot of the k-th kept lane of this round
            const int k = gl - nk;
            const int src = (k >= 0 && k < nm) ? (int)__fns(m, 0, k + 1) : 0;
            const int js = __shfl_sync(gm, j, src, GS);
            if (k >= 0 && k < nm) mine = js;
            nk += nm;  // at most L labels reach the threshold (their T sum to W * 2^16)
        }
        best = cp_group_best<GS>(best, gm);
        if (nk > (int)L) nk = (int)L;  // never (see above); keeps the stores inside the set
        if (nk == 0) {  // none above the threshold: the best label alone
            mine = gl == 0 ? best.slot : -1;
            nk = 1;
        }
        // normalize in fixed point, the remainder to the best label (always kept)
        const bool hold = gl < nk;
        const unsigned long long ti = hold ? tab.t(mine) : 0ull;
        const unsigned long long tk = cp_group_sum<GS>(ti, gm);
        uint32_t bv = hold ? cp_frac(ti, tk) : 0u;
        const uint32_t bsum = __reduce_add_sync(gm, bv);
        if (hold && mine == best.slot) bv += COPRA_ONE - bsum;
        // store by decreasing belonging, equal belongings by first appearance
        const uint32_t fi = hold ? tab.first[mine] : 0xFFFFFFFFu;
        const int32_t li = hold ? tab.key[mine] : EMPTY;
        int rank = 0;
        for (int q = 0; q < nk; ++q) {
            const uint32_t bq = __shfl_sync(gm, bv, q, GS), fq = __shfl_sync(gm, fi, q, GS);
            rank += (bq > bv || (bq == bv && fq < fi)) ? 1 : 0;
        }
        if (hold) {
            out_l[rank] = li;
            out_b[rank] = bv;
            if (rank == 0 && li != prev) ++my_changed;
        }
        for (uint32_t s = (uint32_t)nk + gl; s < L; s += GS) {
            out_l[s] = EMPTY;
            out_b[s] = 0u;
        }
        __syncwarp(gm);
        for (int j = gl; j < slots; j += GS) tab.clear(j);  // leave the table clean
        __syncwarp(gm);
    }
    __syncwarp();
    my_changed = __reduce_add_sync(FULL, my_changed);
    if (lane == 0 && my_changed) atomicAdd(a.changed, (int)my_changed);
}

// Table modes of the CTA kernel: shared with room for every label of the
// row (CP_SHARED), shared with a fixed 2^LG slots that a row may outgrow
// (CP_SPILL: the row is then listed for the global tables), or this CTA's
// region of the global tables (CP_GLOBAL).
constexpr int CP_SHARED = 0, CP_SPILL = 1, CP_GLOBAL = 2;
constexpr int CPL_T = 512;                  // threads of the long-row kernel
constexpr int CPL_LG = 13;
constexpr int CPL_TAB = 1 << CPL_LG;        // its shared slots
constexpr int CPL_FULL = CPL_TAB / 4 * 3;   // claimed slots at which a row moves to the global tables
constexpr int32_t CPL_MAX_D = 1 << 26;      // first appearance e * 64 + p stays below 2^32

// One COPRA step for the listed rows of one wave (a.rows, a.nrows, or
// *a.nrows_dev rows): one CTA of NT threads per vertex.
template <int NT, int LG, int MODE>
__global__ void __launch_bounds__(NT) k_copra_cta(CopraArgs a)
{
    extern __shared__ uint32_t cp_smem[];
    __shared__ CpCand s_red[NT / 32];
    __shared__ unsigned long long s_w[NT / 32];
    __shared__ int32_t s_kept[64];
    __shared__ int s_nk, s_claimed, s_full;
    constexpr int TAB = 1 << LG;
    const int tid = threadIdx.x, lane = tid & 31, wib = tid >> 5;
    using Tab = typename std::conditional<MODE == CP_GLOBAL, CpGlobal, CpShared>::type;
    Tab tab;
    if constexpr (MODE == CP_GLOBAL) {  // this CTA's region (clean at every row's start)
        const int64_t base = (int64_t)blockIdx.x << a.glg_max;
        tab = CpGlobal{a.gkey + base, a.gsum + base, a.gfirst + base};
    } else {
        tab = CpShared{reinterpret_cast<int32_t *>(cp_smem), cp_smem + TAB, cp_smem + 2 * TAB,
                       cp_smem + 3 * TAB};
        for (int j = tid; j < TAB; j += NT) tab.clear(j);
    }
    if (tid == 0) {
        s_claimed = 0;
        s_full = 0;
    }
    __syncthreads();
    const int64_t nrows = a.nrows_dev ? (int64_t)*a.nrows_dev : a.nrows;
    const uint32_t L = (uint32_t)a.L;
    uint32_t my_changed = 0;
    for (int64_t i = blockIdx.x; i < nrows; i += gridDim.x) {
        const int32_t v = a.rows[i];
        const int32_t rs = __ldg(a.off + v), d = __ldg(a.off + v + 1) - rs;
        const int64_t pairs = (int64_t)d * L;
        const int32_t prev = a.cur_l[(int64_t)v * L];
        int32_t *out_l = a.nxt_l + (int64_t)v * L;
        uint32_t *out_b = a.nxt_b + (int64_t)v * L;
        if (d == 0) {  // no labels: the vertex is its own community
            for (uint32_t s = tid; s < L; s += NT) {
                out_l[s] = s == 0 ? v : EMPTY;
                out_b[s] = s == 0 ? COPRA_ONE : 0u;
            }
            if (tid == 0 && prev != v) ++my_changed;
            continue;
        }
        if (MODE == CP_SPILL && d >= CPL_MAX_D) {  // block-uniform
            if (tid == 0) a.ovf[1 + atomicAdd(a.ovf, 1)] = v;
            continue;
        }
        // 2^lg >= 2 pairs slots (<= 2^glg_max), or the whole table in CP_SPILL
        const int lg = MODE == CP_SPILL ? LG : ilog2_ceil((uint32_t)(2 * pairs));
        const int slots = 1 << lg;
        // T(l) and first appearance over the row's entries and their speakers'
        // pairs; each thread sums the runs of its speakers' first (best)
        // labels in registers, so a label most speakers share is added once
        unsigned long long wsum = 0ull;
        int32_t c_l = EMPTY;
        unsigned long long c_v = 0ull, c_f = 0ull;
        auto put = [&](int32_t l, unsigned long long val, unsigned long long f) {
            if (tab.add(lg, l, val, f) && MODE == CP_SPILL) {
                if (atomicAdd(&s_claimed, 1) + 1 >= CPL_FULL) s_full = 1;
            }
        };
        for (int32_t e = tid; e < d; e += NT) {
            if (MODE == CP_SPILL && *(volatile int *)&s_full) break;
            const int32_t u = __ldg(a.idx + rs + e);
            const uint32_t w = a.wts ? (uint32_t)__ldg(a.wts + rs + e) : 1u;
            wsum += w;
            const bool earlier = cp_wave(a, u) < a.wave_k;
            const int32_t *ul = (earlier ? a.nxt_l : a.cur_l) + (int64_t)u * L;
            const uint32_t *ub = (earlier ? a.nxt_b : a.cur_b) + (int64_t)u * L;
            cp_each_pair(ul, ub, L, [&](uint32_t p, int32_t l, uint32_t b) {
                const unsigned long long val = (unsigned long long)w * b;
                const unsigned long long f = (unsigned long long)e * 64ull + p;
                if (p == 0) {
                    if (l == c_l) {
                        c_v += val;  // its first appearance is the cached one (earlier)
                        return;
                    }
                    if (c_l != EMPTY) put(c_l, c_v, c_f);
                    c_l = l;
                    c_v = val;
                    c_f = f;
                    return;
                }
                put(l, val, f);
            });
        }
        if (c_l != EMPTY && !(MODE == CP_SPILL && *(volatile int *)&s_full)) put(c_l, c_v, c_f);
        wsum = cp_warp_sum(wsum);
        if (lane == 0) s_w[wib] = wsum;
        if (tid == 0) s_nk = 0;
        __syncthreads();
        if (MODE == CP_SPILL && s_full) {  // too many labels: the global tables take the row
            if (tid == 0) a.ovf[1 + atomicAdd(a.ovf, 1)] = v;
            for (int j = tid; j < slots; j += NT)
                if (tab.key[j] != EMPTY) tab.clear(j);
            if (tid == 0) {
                s_claimed = 0;
                s_full = 0;
            }
            __syncthreads();
            continue;
        }
        unsigned long long W = 0ull;
#pragma unroll
        for (int k = 0; k < NT / 32; ++k) W += s_w[k];
        // the labels above the threshold and the best label
        const uint64_t ktv = stream_at(a.key_t, (uint64_t)v + 1);
        CpCand best{0ull, 0ull, 0ull, -1};
        for (int j = tid; j < slots; j += NT) {
            const int32_t l = tab.key[j];
            if (l == EMPTY) continue;
            const unsigned long long t = tab.t(j);
            if ((unsigned long long)L * t >= W * (unsigned long long)COPRA_ONE) {
                const int at = atomicAdd(&s_nk, 1);
                if (at < 64) s_kept[at] = j;  // at most L labels pass
            }
            const CpCand c{t, a.strict ? 0ull : stream_at(ktv, (uint64_t)l + 1),
                           (unsigned long long)tab.first[j], j};
            if (cp_better(c, best)) best = c;
        }
        best = cp_warp_best(best);
        if (lane == 0) s_red[wib] = best;
        __syncthreads();
        if (tid == 0) {
            best = s_red[0];
            for (int k = 1; k < NT / 32; ++k)
                if (cp_better(s_red[k], best)) best = s_red[k];
            int nk = s_nk < (int)L ? s_nk : (int)L;  // at most L labels pass
            if (nk == 0) {  // none above the threshold: the best label alone
                s_kept[0] = best.slot;
                nk = 1;
            }
            // normalize in fixed point, the remainder to the best label (always kept)
            unsigned long long tk = 0ull;
            for (int q = 0; q < nk; ++q) tk += tab.t(s_kept[q]);
            uint32_t bv[64];
            uint32_t bsum = 0u;
            for (int q = 0; q < nk; ++q) {
                bv[q] = cp_frac(tab.t(s_kept[q]), tk);
                bsum += bv[q];
            }
            for (int q = 0; q < nk; ++q)
                if (s_kept[q] == best.slot) bv[q] += COPRA_ONE - bsum;
            // store by decreasing belonging, equal belongings by first appearance
            for (int r = 0; r < nk; ++r) {
                int pick = -1;
                for (int q = 0; q < nk; ++q) {
                    if (s_kept[q] < 0) continue;
                    if (pick < 0 || bv[q] > bv[pick] ||
                        (bv[q] == bv[pick] &&
                         (unsigned long long)tab.first[s_kept[q]] <
                             (unsigned long long)tab.first[s_kept[pick]]))
                        pick = q;
                }
                out_l[r] = tab.key[s_kept[pick]];
                out_b[r] = bv[pick];
                s_kept[pick] = -1 - s_kept[pick];  // taken
            }
            for (uint32_t s = nk; s < L; ++s) {
                out_l[s] = EMPTY;
                out_b[s] = 0u;
            }
            if (out_l[0] != prev) ++my_changed;
        }
        __syncthreads();
        for (int j = tid; j < slots; j += NT)  // leave the table clean
            if (tab.key[j] != EMPTY) tab.clear(j);
        if (tid == 0) s_claimed = 0;
        __syncthreads();
    }
    if (tid == 0 && my_changed) atomicAdd(a.changed, (int)my_changed);
}

// every vertex its own community: {(v, 2^16)}
__global__ void k_copra_init(int32_t *l, uint32_t *b, int32_t n, int32_t L)
{
    const int64_t cells = (int64_t)n * L;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < cells;
         i += (int64_t)gridDim.x * blockDim.x) {
        const bool head = i % L == 0;
        l[i] = head ? (int32_t)(i / L) : EMPTY;
        b[i] = head ? COPRA_ONE : 0u;
    }
}

__global__ void k_copra_best(const int32_t *l, int32_t n, int32_t L, int32_t *out)
{
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n;
         v += (int64_t)gridDim.x * blockDim.x)
        out[v] = l[v * L];
}

// Bin of row v among the listed rows: kind * waves + wave (kind 0: a whole
// warp, 1: a CTA with the shared table, 2: the long-row kernel), or -1 for a
// row of the 8-lane kernel, which visits the wave's vertices directly.
__device__ __forceinline__ int64_t cp_bin(const int32_t *off, int32_t v, int32_t L, int32_t waves,
                                          uint64_t magic)
{
    const int64_t pairs = (int64_t)(__ldg(off + v + 1) - __ldg(off + v)) * L;
    if (L <= 8 && pairs <= 32) return -1;
    const uint32_t wave = waves > 1 ? fastmod((uint32_t)v, magic, (uint32_t)waves) : 0u;
    const int kind = (L <= CPW_MAX_L && pairs <= CPW_PAIRS) ? 0 : pairs > CP_PAIRS ? 2 : 1;
    return (int64_t)kind * waves + wave;
}

// count[bin] += rows of each bin (one atomic per bin and warp)
__global__ void __launch_bounds__(256) k_copra_count(const int32_t *off, int32_t n, int32_t L,
                                                     int32_t waves, uint64_t magic, int32_t *count)
{
    const int lane = threadIdx.x & 31;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t base = (int64_t)blockIdx.x * blockDim.x; base < n; base += stride) {
        const int64_t v = base + threadIdx.x;
        const int64_t bin = v < n ? cp_bin(off, (int32_t)v, L, waves, magic) : -1;
        const unsigned peers = __match_any_sync(FULL, (unsigned long long)bin);
        if (bin >= 0 && lane == __ffs(peers) - 1) atomicAdd(count + bin, __popc(peers));
    }
}

// rows[cursor[bin]++] = v for every listed row (cursor: the bins' starts)
__global__ void __launch_bounds__(256) k_copra_scatter(const int32_t *off, int32_t n, int32_t L,
                                                       int32_t waves, uint64_t magic,
                                                       int32_t *cursor, int32_t *rows)
{
    const int lane = threadIdx.x & 31;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t base = (int64_t)blockIdx.x * blockDim.x; base < n; base += stride) {
        const int64_t v = base + threadIdx.x;
        const int64_t bin = v < n ? cp_bin(off, (int32_t)v, L, waves, magic) : -1;
        const unsigned peers = __match_any_sync(FULL, (unsigned long long)bin);
        const int leader = __ffs(peers) - 1;
        int32_t at = 0;
        if (bin >= 0 && lane == leader) at = atomicAdd(cursor + bin, __popc(peers));
        at = __shfl_sync(FULL, at, leader);
        if (bin >= 0) rows[at + __popc(peers & ((1u << lane) - 1u))] = (int32_t)v;
    }
}

int cp_grid(int64_t items) { return (int)(items < 1 ? 1 : (items + 255) / 256 < 8192 ? (items + 255) / 256 : 8192); }

}  // namespace

int copra_init(int32_t *l, uint32_t *b, int32_t n, int32_t L, cudaStream_t st, int64_t *launches)
{
    if (n <= 0) return 0;
    k_copra_init<<<cp_grid((int64_t)n * L), 256, 0, st>>>(l, b, n, L);
    ++*launches;
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

int copra_best(const int32_t *l, int32_t n, int32_t L, int32_t *out, cudaStream_t st,
               int64_t *launches)
{
    if (n <= 0) return 0;
    k_copra_best<<<cp_grid(n), 256, 0, st>>>(l, n, L, out);
    ++*launches;
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

int copra_prepare()
{
    const bool ok =
        cudaFuncSetAttribute(k_copra_cta<CP_T, CP_LG, CP_SHARED>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, CP_TAB * 16) ==
            cudaSuccess &&
        cudaFuncSetAttribute(k_copra_cta<CPL_T, CPL_LG, CP_SPILL>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, CPL_TAB * 16) ==
            cudaSuccess;
    return ok ? 0 : -1;
}

int copra_table_lg(int64_t max_degree, int32_t L)
{
    const int64_t pairs = max_degree * L;
    if (pairs <= CP_PAIRS) return 0;  // every row fits the shared table
    int lg = 0;
    while ((1ll << lg) < 2 * pairs) ++lg;
    return lg;
}

int copra_big_ctas() { return 32; }

int64_t copra_bins(int32_t waves) { return 3 * (int64_t)waves; }

int copra_rows(const int32_t *off, int32_t n, int32_t L, int32_t waves, int32_t *bins,
               int32_t *h_bins, int64_t *h_start, int32_t *rows, cudaStream_t st,
               int64_t *launches)
{
    const int64_t nb = copra_bins(waves);
    const uint64_t magic = fastmod_magic((uint32_t)waves);
    if (cudaMemsetAsync(bins, 0, (size_t)nb * sizeof(int32_t), st) != cudaSuccess) return -1;
    if (n > 0) {
        k_copra_count<<<cp_grid(n), 256, 0, st>>>(off, n, L, waves, magic, bins);
        ++*launches;
    }
    if (cudaMemcpyAsync(h_bins, bins, (size_t)nb * sizeof(int32_t), cudaMemcpyDeviceToHost, st) !=
            cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
        return -1;
    h_start[0] = 0;
    for (int64_t b = 0; b < nb; ++b) h_start[b + 1] = h_start[b] + h_bins[b];
    for (int64_t b = 0; b < nb; ++b) h_bins[b] = (int32_t)h_start[b];
    if (h_start[nb] > 0) {
        if (cudaMemcpyAsync(bins, h_bins, (size_t)nb * sizeof(int32_t), cudaMemcpyHostToDevice,
                            st) != cudaSuccess)
            return -1;
        k_copra_scatter<<<cp_grid(n), 256, 0, st>>>(off, n, L, waves, magic, bins, rows);
        ++*launches;
        // h_bins is read by the copy before it is reused
        if (cudaStreamSynchronize(st) != cudaSuccess) return -1;
    }
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

int copra_step(const CopraStep &s, int num_sms, cudaStream_t st, int64_t *launches)
{
    CopraArgs a{};
    a.off = s.off;
    a.idx = s.idx;
    a.wts = s.wts;
    a.n = s.n;
    a.L = s.L;
    a.cur_l = s.cur_l;
    a.cur_b = s.cur_b;
    a.nxt_l = s.nxt_l;
    a.nxt_b = s.nxt_b;
    a.waves = (uint32_t)s.waves;
    a.wave_k = (uint32_t)s.wave_k;
    a.magic = fastmod_magic((uint32_t)s.waves);
    a.strict = s.strict;
    a.key_t = s.key_t;
    a.changed = s.changed;
    a.gkey = s.gkey;
    a.gsum = s.gsum;
    a.gfirst = s.gfirst;
    a.glg_max = s.glg_max;
    if (s.n <= 0) return 0;
    if (s.L <= 8) {  // rows of at most 32 pairs: four per warp, over the wave's vertices
        const int64_t nw = (s.n - s.wave_k + (int64_t)s.waves - 1) / s.waves;
        int64_t blocks = (nw + 4 * CPW_WARPS - 1) / (4 * CPW_WARPS);
        if (blocks > (int64_t)num_sms * 8) blocks = (int64_t)num_sms * 8;
        if (blocks > 0) {
            k_copra_warp<8><<<(int)blocks, CPW_WARPS * 32, 0, st>>>(a);
            ++*launches;
        }
    }
    if (s.n_warp > 0) {  // the listed rows of up to 128 pairs: one per warp
        a.rows = s.rows_warp;
        a.nrows = s.n_warp;
        int64_t blocks = (s.n_warp + CPW_WARPS - 1) / CPW_WARPS;
        if (blocks > (int64_t)num_sms * 8) blocks = (int64_t)num_sms * 8;
        k_copra_warp<32><<<(int)blocks, CPW_WARPS * 32, 0, st>>>(a);
        ++*launches;
        a.rows = nullptr;
        a.nrows = 0;
    }
    if (s.n_cta > 0) {
        a.rows = s.rows_cta;
        a.nrows = s.n_cta;
        const int64_t grid = s.n_cta < (int64_t)num_sms * 3 ? s.n_cta : (int64_t)num_sms * 3;
        k_copra_cta<CP_T, CP_LG, CP_SHARED><<<(int)grid, CP_T, CP_TAB * 16, st>>>(a);
        ++*launches;
    }
    if (s.n_big > 0) {
        // long rows in shared memory; those with too many labels, then, in the global tables
        if (cudaMemsetAsync(s.ovf, 0, sizeof(int32_t), st) != cudaSuccess) return -1;
        a.rows = s.rows_big;
        a.nrows = s.n_big;
        a.ovf = s.ovf;
        const int64_t grid = s.n_big < num_sms ? s.n_big : num_sms;
        k_copra_cta<CPL_T, CPL_LG, CP_SPILL><<<(int)grid, CPL_T, CPL_TAB * 16, st>>>(a);
        a.rows = s.ovf + 1;
        a.nrows = 0;
        a.nrows_dev = s.ovf;
        const int64_t gg = s.n_big < copra_big_ctas() ? s.n_big : copra_big_ctas();
        k_copra_cta<CP_T, CP_LG, CP_GLOBAL><<<(int)gg, CP_T, 0, st>>>(a);
        *launches += 2;
    }
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

}  // namespace lp
