// Device helpers shared by the sweep kernels: the non-strict tie key, the
// table slot hash, argmax candidates with their total order, warp / block
// reductions of candidates and the open-addressing table insert.
#pragma once

#include <cstdint>

#include "lp_internal.cuh"

namespace lp {
namespace {

// L2 eviction policies (PTX createpolicy): the CSR entries are read once per
// sweep and should not push the label arrays, which every sweep gathers from
// at random, out of L2.
__device__ __forceinline__ uint64_t policy_evict_first()
{
    uint64_t p;
    asm("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
    return p;
}

__device__ __forceinline__ uint64_t policy_evict_last()
{
    uint64_t p;
    asm("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(p));
    return p;
}

// read-only loads with an L2 policy: a 16-byte block of entries, one entry,
// one label
__device__ __forceinline__ int4 ld_entries4(const int32_t *base, int64_t blk)
{
    int4 r;
    asm("ld.global.nc.L1::no_allocate.L2::cache_hint.v4.s32 {%0, %1, %2, %3}, [%4], %5;"
        : "=r"(r.x), "=r"(r.y), "=r"(r.z), "=r"(r.w)
        : "l"(reinterpret_cast<const int4 *>(base) + blk), "l"(policy_evict_first()));
    return r;
}

__device__ __forceinline__ int32_t ld_entry(const int32_t *p)
{
    int32_t r;
    asm("ld.global.nc.L1::no_allocate.L2::cache_hint.s32 %0, [%1], %2;"
        : "=r"(r)
        : "l"(p), "l"(policy_evict_first()));
    return r;
}

__device__ __forceinline__ int32_t ld_label(const int32_t *p)
{
    int32_t r;
    asm("ld.global.nc.L2::cache_hint.s32 %0, [%1], %2;" : "=r"(r) : "l"(p), "l"(policy_evict_last()));
    return r;
}

// Non-strict key of `label` at local vertex lv (see lp.h).
__device__ __forceinline__ uint64_t tie_key(uint64_t key_t, int32_t lv, int32_t label)
{
    return stream_at(stream_at(key_t, (uint64_t)lv + 1), (uint64_t)label + 1);
}

__device__ __forceinline__ uint32_t slot_hash(int32_t label, int lg)
{
    // Fibonacci hashing: the top lg bits of label * 2^32/phi
    return lg == 0 ? 0u : ((uint32_t)label * 0x9E3779B1u) >> (32 - lg);
}

struct Cand {
    uint32_t sum;   // summed weight (0 = no candidate)
    uint32_t npos;  // 0xFFFFFFFF - first position
    uint64_t h;     // non-strict key (0 in strict mode)
    int32_t label;
};

// strictly better: heavier, then smaller non-strict key, then earlier
__device__ __forceinline__ bool better(const Cand &x, const Cand &y)
{
    if (x.sum != y.sum) return x.sum > y.sum;
    if (x.h != y.h) return x.h < y.h;
    return x.npos > y.npos;
}

__device__ __forceinline__ Cand shfl_cand(const Cand &c, int src)
{
    Cand r;
    r.sum = __shfl_sync(FULL, c.sum, src);
    r.npos = __shfl_sync(FULL, c.npos, src);
    r.h = __shfl_sync(FULL, c.h, src);
    r.label = __shfl_sync(FULL, c.label, src);
    return r;
}

__device__ __forceinline__ Cand warp_best(Cand c)
{
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) {
        Cand x;
        x.sum = __shfl_xor_sync(FULL, c.sum, o);
        x.npos = __shfl_xor_sync(FULL, c.npos, o);
        x.h = __shfl_xor_sync(FULL, c.h, o);
        x.label = __shfl_xor_sync(FULL, c.label, o);
        if (better(x, c)) c = x;
    }
    return c;
}

// Lanes [lo, lo + len) of a warp as a mask (0 <= lo, lo + len <= 32).
__device__ __forceinline__ unsigned lane_range(int lo, int len)
{
    return (len >= 32 ? 0xFFFFFFFFu : ((1u << len) - 1u)) << lo;
}

__device__ __forceinline__ int ilog2_ceil(uint32_t x)  // smallest lg with 2^lg >= x
{
    return x <= 1 ? 0 : 32 - __clz(x - 1);
}

template <int NT>
__device__ __forceinline__ Cand block_best(Cand c, Cand *s_red)
{
    c = warp_best(c);
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    if (lane == 0) s_red[wib] = c;
    __syncthreads();
    if (wib == 0) {
        c = lane < NT / 32 ? s_red[lane] : Cand{0u, 0u, 0ull, EMPTY};
        c = warp_best(c);
    }
    return c;  // valid in thread 0
}

template <int NT>
__device__ __forceinline__ uint32_t block_max(uint32_t v, uint32_t *s_u)
{
    v = __reduce_max_sync(FULL, v);
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    if (lane == 0) s_u[wib] = v;
    __syncthreads();
    if (threadIdx.x < 32) {
        v = lane < NT / 32 ? s_u[lane] : 0u;
        v = __reduce_max_sync(FULL, v);
        if (lane == 0) s_u[NT / 32] = v;
    }
    __syncthreads();
    return s_u[NT / 32];
}

// insert (l, s, first position p) into an open-addressing table of mask + 1
// slots, starting at slot h and probing at most `limit` slots; false if that
// window is full of other labels.  The table may be another CTA's shared
// memory in the cluster (generic addresses).
__device__ __forceinline__ bool table_add_at(int32_t *key, int32_t *sum, uint32_t *npos,
                                             uint32_t mask, uint32_t h, int limit, int32_t l,
                                             int s, uint32_t p)
{
    volatile int32_t *vk = key;
    for (int i = 0; i < limit; ++i) {
        int32_t cur = vk[h];
        if (cur == EMPTY) {
            cur = atomicCAS(key + h, EMPTY, l);
            if (cur == EMPTY) cur = l;
        }
        if (cur == l) {
            atomicAdd(sum + h, s);
            atomicMax(npos + h, 0xFFFFFFFFu - p);
            return true;
        }
        h = (h + 1) & mask;
    }
    return false;
}

// the same for a table of 2^lg slots, starting at the label's hash slot
__device__ __forceinline__ bool table_add(int32_t *key, int32_t *sum, uint32_t *npos, int lg,
                                          int limit, int32_t l, int s, uint32_t p)
{
    return table_add_at(key, sum, npos, (1u << lg) - 1u, slot_hash(l, lg), limit, l, s, p);
}

// ----------------------------------------------------------------------------
// Tables of 64-bit slots: (label + 1) << 32 | summed weight, 0 = free.  One
// shared atomic per inserted entry (a claim or an add); the first position of
// a label is not kept: it is recovered for the rows whose maximum is tied
// (tie_position below).
// ----------------------------------------------------------------------------
__device__ __forceinline__ unsigned long long slot_tag(int32_t l)
{
    return (unsigned long long)((uint32_t)l + 1u) << 32;
}

__device__ __forceinline__ int32_t slot_label(unsigned long long v)
{
    return (int32_t)((uint32_t)(v >> 32) - 1u);
}

// add weight s of label l to a table of 2^lg slots that has room for every
// label inserted into it (at most half full).  A slot is claimed with a 64-bit
// CAS (label and first weight at once); later weights of its label are added
// to its low word (the sum) with a native 32-bit atomic, only after the
// claim was seen, so the two atomics never race on a free slot (a failed CAS
// writes nothing).  Sums stay below 2^31 and never carry into the label.
__device__ __forceinline__ void table64_add(unsigned long long *t, int lg, int32_t l, uint32_t s)
{
    const uint32_t mask = (1u << lg) - 1u;
    const unsigned long long tag = slot_tag(l);
    volatile unsigned long long *vt = t;
    uint32_t h = slot_hash(l, lg);
    for (uint32_t i = 0; i <= mask; ++i) {
        unsigned long long cur = vt[h];
        if (cur == 0ull) {
            cur = atomicCAS(t + h, 0ull, tag | s);
            if (cur == 0ull) return;
        }
        if ((cur & 0xFFFFFFFF00000000ull) == tag) {
            atomicAdd(reinterpret_cast<unsigned int *>(t + h), s);  // low word = sum
            return;
        }
        h = (h + 1) & mask;
    }
}

// summed weight of label l in such a table (0 if absent)
__device__ __forceinline__ uint32_t table64_sum(const unsigned long long *t, int lg, int32_t l)
{
    const uint32_t mask = (1u << lg) - 1u;
    const unsigned long long tag = slot_tag(l);
    const volatile unsigned long long *vt = t;
    uint32_t h = slot_hash(l, lg);
    for (uint32_t i = 0; i <= mask; ++i) {
        const unsigned long long cur = vt[h];
        if (cur == 0ull) return 0u;
        if ((cur & 0xFFFFFFFF00000000ull) == tag) return (uint32_t)cur;
        h = (h + 1) & mask;
    }
    return 0u;
}

// The maximum of a table: its weight, how many labels reach it, one of those
// labels, and (non-strict) the least tie key among them with its count.
struct Top {
    uint32_t sum;
    uint32_t cnt;
    int32_t label;
    uint64_t h;  // non-strict: least tie key of the labels at the maximum
};

// Warp-wide combination of per-lane tops, valid in every lane: the largest
// `key` (lanes with key 0 hold nothing), the summed counts of the lanes
// reaching it and the largest label among them.
__device__ __forceinline__ void warp_top(uint64_t &key, uint32_t &cnt, int32_t &label)
{
    uint64_t k = key;
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) {
        const uint64_t y = __shfl_xor_sync(FULL, k, o);
        k = y > k ? y : k;
    }
    const bool at = key == k;
    cnt = __reduce_add_sync(FULL, at ? cnt : 0u);
    label = (int32_t)__reduce_max_sync(FULL, at ? (uint32_t)label + 1u : 0u) - 1;
    key = k;
}

// The same over a block of NT threads (s: NT / 32 + 1 entries of each array),
// valid in every thread.
template <int NT>
__device__ __forceinline__ void block_top(uint64_t &key, uint32_t &cnt, int32_t &label,
                                          uint64_t *s_k, uint32_t *s_c, int32_t *s_l)
{
    warp_top(key, cnt, label);
    if (NT == 32) return;
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    if (lane == 0) {
        s_k[wib] = key;
        s_c[wib] = cnt;
        s_l[wib] = label;
    }
    __syncthreads();
    if (wib == 0) {
        uint64_t k = lane < NT / 32 ? s_k[lane] : 0ull;
        uint32_t c = lane < NT / 32 ? s_c[lane] : 0u;
        int32_t l = lane < NT / 32 ? s_l[lane] : EMPTY;
        warp_top(k, c, l);
        if (lane == 0) {
            s_k[NT / 32] = k;
            s_c[NT / 32] = c;
            s_l[NT / 32] = l;
        }
    }
    __syncthreads();
    key = s_k[NT / 32];
    cnt = s_c[NT / 32];
    label = s_l[NT / 32];
}

// Row of every entry of a chunk of 256 consecutive entries (one warp): rows
// k = 1 .. nr - 1 start at chunk offsets start(k) in (0, 256] (strictly
// increasing: every row has an entry), row 0 holds offset 0.  s_row[e]
// receives the row of offset e: the number of row starts at or before e.
template <typename StartOf>
__device__ __forceinline__ void chunk_rows(StartOf start, int nr, uint16_t *s_row)
{
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int i = 0; i < 8; ++i) s_row[lane + 32 * i] = 0;
    __syncwarp();
    for (int k = 1 + lane; k < nr; k += 32) {
        const int e = start(k);
        if (e < 256) s_row[e] = 1;
    }
    __syncwarp();
    uint16_t m[8];
    int sum = 0;
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        m[i] = s_row[8 * lane + i];
        sum += m[i];
    }
    int inc = sum;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(FULL, inc, o);
        if (lane >= o) inc += y;
    }
    int run = inc - sum;
    __syncwarp();
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        run += m[i];
        s_row[8 * lane + i] = (uint16_t)run;
    }
    __syncwarp();
}

}  // namespace
}  // namespace lp
