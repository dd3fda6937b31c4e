// Modularity (Sec. 1) of every graph of a graph set under a labelling, in
// exact integers.  Per graph g:
//   2m  = sum of all stored weights
//   L   = sum of stored weights whose two ends carry the same label
//   K_c = sum over the vertices v of community c of k_v (k_v = row sum of v)
//   S   = sum_c K_c^2  (128-bit)
//   Q   = L / 2m - S / (2m)^2   (formed in double on the host)
//
// The entry pass streams the packed rows (the sweep's layout: rows in list
// order, contiguous) in chunks of PACK_CHUNK entries, one warp per chunk:
// the warp stages the rows that meet its chunk (their starts, labels and
// graphs) in shared memory, and every lane takes eight consecutive entries,
// gathers their neighbours' labels and sums L and 2m in registers.
// A row's weights within the chunk are summed in shared memory and added to
// K of the row's community: a row split over several chunks adds one part
// from each, which sums to the same K.  Rows of one community in a chunk
// (a converged labelling often has one giant community) are combined before
// the global 64-bit atomics.  The square pass adds K_c^2 into per-graph
// 128-bit accumulators (carry-propagating 64-bit atomics).
#include "lp_device.cuh"
#include "lp_internal.cuh"

namespace lp {
namespace {

// acc layout per graph g: [4g] = L, [4g+1] = 2m, [4g+2] = S high, [4g+3] = S low
__device__ __forceinline__ void add_u128(unsigned long long *hi_lo, unsigned long long hi,
                                         unsigned long long lo)
{
    const unsigned long long old = atomicAdd(hi_lo + 1, lo);
    const unsigned long long carry = (old + lo < old) ? 1ull : 0ull;
    if (hi + carry) atomicAdd(hi_lo, hi + carry);
}

__device__ __forceinline__ unsigned long long warp_sum64(unsigned long long v)
{
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) v += __shfl_xor_sync(FULL, v, o);
    return v;
}

// Running L and 2m contributions of one thread to one graph of a graph set.
struct AccRun {
    int32_t g = -1;
    unsigned long long l = 0, w = 0;
    __device__ __forceinline__ void add(unsigned long long *acc, int32_t gg, unsigned long long lv,
                                        unsigned long long kv)
    {
        if (gg != g) {
            flush(acc);
            g = gg;
        }
        l += lv;
        w += kv;
    }
    __device__ __forceinline__ void flush(unsigned long long *acc)
    {
        if (g >= 0 && w) {
            atomicAdd(acc + 4 * (int64_t)g, l);
            atomicAdd(acc + 4 * (int64_t)g + 1, w);
        }
        l = w = 0;
    }
};

// Sum every thread's (l, w) of a single graph into acc[0..1], one pair of
// global atomics per block (every thread of the block calls this).
__device__ __forceinline__ void block_flush_lw(unsigned long long *acc, unsigned long long l,
                                               unsigned long long w)
{
    __shared__ unsigned long long s_lw[2];
    if (threadIdx.x == 0) s_lw[0] = s_lw[1] = 0;
    __syncthreads();
    l = warp_sum64(l);
    w = warp_sum64(w);
    if ((threadIdx.x & 31) == 0 && w) {
        atomicAdd(s_lw, l);
        atomicAdd(s_lw + 1, w);
    }
    __syncthreads();
    if (threadIdx.x == 0 && s_lw[1]) {
        atomicAdd(acc, s_lw[0]);
        atomicAdd(acc + 1, s_lw[1]);
    }
}

// Sum of a 32-bit value over the lanes of `mask` (values < 2^31), exact in
// 64 bits: the low and high halves are reduced separately.
__device__ __forceinline__ unsigned long long group_sum(unsigned mask, uint32_t v)
{
    const uint32_t lo = __reduce_add_sync(mask, v & 0xFFFFu);
    const uint32_t hi = __reduce_add_sync(mask, v >> 16);
    return ((unsigned long long)hi << 16) + lo;
}

constexpr int MT = 256, MPER = 8;  // threads per block, entries per lane
constexpr int MW = MT / 32;        // warps (chunks) per block
static_assert(32 * MPER == PACK_CHUNK, "one warp per packed chunk");
constexpr int32_t MOD_ID_MASK = 0x7FFFFFFF;  // packed neighbour id without its wave bit
constexpr int64_t SMALL_BLOCKS = 2048;       // blocks of the small-row pass
constexpr int64_t ENTRY_BLOCKS = 2048;       // blocks of the entry pass

// Entry pass, one warp per chunk of PACK_CHUNK entries of the packed rows
// (entries [j_lo, j_lo + PACK_CHUNK), held by the list items r0, holding
// j_lo, to r1, holding the next chunk's first entry or the last item: at
// most PACK_CHUNK + 1 rows).  Warps stage their rows independently.  A block
// takes groups of MW consecutive chunks in a grid-stride loop (a grid of a
// few blocks per SM) and combines L, 2m and the K part of its first row's
// community over all of them, so that these sums, which every block shares
// (a converged labelling often has a giant community), take one global
// atomic per block.
template <bool MULTI>
__global__ void __launch_bounds__(MT, MULTI ? 4 : 5) k_mod_entries(ModArgs a)
{
    constexpr int CH = PACK_CHUNK;
    __shared__ int32_t s_rp_all[MW][CH + 2];   // row starts relative to j_lo
    __shared__ int32_t s_c_all[MW][CH + 1];    // the row's label (local)
    __shared__ uint32_t s_kv_all[MW][CH + 1];  // the row's weight within the chunk
    __shared__ int32_t s_vb_all[MULTI ? MW : 1][MULTI ? CH + 1 : 1];
    __shared__ int32_t s_g_all[MULTI ? MW : 1][MULTI ? CH + 1 : 1];
    __shared__ unsigned long long s_dom;  // K part of the block's first community
    __shared__ int64_t s_dom_slot;
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    int32_t *s_rp = s_rp_all[wib];
    int32_t *s_c = s_c_all[wib];
    uint32_t *s_kv = s_kv_all[wib];
    int32_t *s_vb = s_vb_all[MULTI ? wib : 0];
    int32_t *s_g = s_g_all[MULTI ? wib : 0];
    const int64_t c_lo = a.e_lo / CH;
    const int64_t groups = (a.ncopy - c_lo + MW - 1) / MW;
    if (threadIdx.x == 0) {  // the community of the block's first row
        s_dom = 0ull;
        s_dom_slot = -1;
        const int64_t c0 = c_lo + (int64_t)blockIdx.x * MW;
        if (c0 < a.ncopy) {
            const int32_t v = a.list[a.first_row[c0]];
            s_dom_slot = (MULTI ? (int64_t)a.g_vbase[a.vgraph[v]] : 0) + a.lab[v];
        }
    }
    __syncthreads();
    const int64_t dom = s_dom_slot;
    unsigned long long l = 0, w2 = 0;
    AccRun run;
    for (int64_t grp = blockIdx.x; grp < groups; grp += gridDim.x) {  // block-uniform
    const int64_t chunk = c_lo + grp * MW + wib;
    const bool have = chunk < a.ncopy;  // warp-uniform
    const int64_t j_lo = chunk * CH;
    const int rel0 = lane * MPER;
    const int rel_hi = have ? (int)(min(j_lo + (int64_t)CH, a.ne) - j_lo) : 0;
    // the entries first (they depend on the chunk only) and, for a single
    // graph, their neighbours' labels, so that these loads overlap the
    // staging of the chunk's rows below
    int32_t u[MPER], w[MPER], cu[MPER];
#pragma unroll
    for (int q = 0; q < MPER; ++q) {
        u[q] = 0;
        w[q] = 0;
        cu[q] = EMPTY;
    }
    if (rel0 < rel_hi) {
        const int64_t j0 = j_lo + rel0;
        if (rel0 + MPER <= rel_hi) {  // 32-byte aligned: j_lo and rel0 are multiples of 8
            const int4 *pi = reinterpret_cast<const int4 *>(a.idx + j0);
            const int4 i0 = __ldcs(pi), i1 = __ldcs(pi + 1);
            u[0] = i0.x; u[1] = i0.y; u[2] = i0.z; u[3] = i0.w;
            u[4] = i1.x; u[5] = i1.y; u[6] = i1.z; u[7] = i1.w;
            if (a.wts) {
                const int4 *pw = reinterpret_cast<const int4 *>(a.wts + j0);
                const int4 w0 = __ldcs(pw), w1 = __ldcs(pw + 1);
                w[0] = w0.x; w[1] = w0.y; w[2] = w0.z; w[3] = w0.w;
                w[4] = w1.x; w[5] = w1.y; w[6] = w1.z; w[7] = w1.w;
            } else {
#pragma unroll
                for (int q = 0; q < MPER; ++q) w[q] = 1;
            }
        } else {
#pragma unroll
            for (int q = 0; q < MPER; ++q) {
                const bool in = rel0 + q < rel_hi;
                u[q] = in ? a.idx[j0 + q] : 0;
                w[q] = in ? (a.wts ? a.wts[j0 + q] : 1) : 0;
            }
        }
        // entries of the small rows (summed one row per lane) count as absent
        if (j0 < a.e_lo) {
#pragma unroll
            for (int q = 0; q < MPER; ++q)
                if (j0 + q < a.e_lo) w[q] = 0;
        }
    }
    if (!MULTI) {
#pragma unroll
        for (int q = 0; q < MPER; ++q)
            cu[q] = w[q] ? __ldg(a.lab + (u[q] & MOD_ID_MASK)) : EMPTY;
    }
    int nr = 0;
    if (have) {
        const int64_t r0 = a.first_row[chunk];
        const int64_t r1 = a.first_row[chunk + 1];
        nr = (int)min(r1 - r0 + 1, (int64_t)CH + 1);
        for (int k = lane; k <= nr; k += 32) s_rp[k] = (int32_t)(a.rp[r0 + k] - j_lo);
        for (int k = lane; k < nr; k += 32) {
            const int32_t v = a.list[r0 + k];
            if (MULTI) {
                const int32_t g = a.vgraph[v];
                s_g[k] = g;
                s_vb[k] = a.g_vbase[g];
            }
            s_c[k] = a.lab[v];
            s_kv[k] = 0u;
        }
    }
    __syncwarp();
    if (rel0 < rel_hi) {
        int lo = 0, hi = nr;  // s_rp[lo] <= rel0 < s_rp[hi]
        while (hi - lo > 1) {
            const int mid = (lo + hi) >> 1;
            if (s_rp[mid] <= rel0)
                lo = mid;
            else
                hi = mid;
        }
        // rows of the entries (shared memory)
        int kq[MPER];
        int k = lo;
#pragma unroll
        for (int q = 0; q < MPER; ++q) {
            while (k + 1 < nr && s_rp[k + 1] <= rel0 + q) ++k;
            kq[q] = k;
        }
        if (MULTI) {
#pragma unroll
            for (int q = 0; q < MPER; ++q)
                cu[q] = w[q] ? __ldg(a.lab + (int64_t)s_vb[kq[q]] + (u[q] & MOD_ID_MASK)) : EMPTY;
        }
        int cur = kq[0];
        uint32_t rs = 0u;  // the current row's weight in this lane's entries
#pragma unroll
        for (int q = 0; q < MPER; ++q) {
            if (!w[q]) continue;
            if (kq[q] != cur) {
                if (rs) atomicAdd(&s_kv[cur], rs);
                cur = kq[q];
                rs = 0u;
            }
            rs += (uint32_t)w[q];
            const unsigned long long lw = cu[q] == s_c[kq[q]] ? (unsigned long long)w[q] : 0ull;
            if (MULTI && s_g[kq[q]] != s_g[0]) {
                run.add(a.acc, s_g[kq[q]], lw, (unsigned long long)w[q]);  // rare: a graph boundary
            } else {
                l += lw;  // single graph, or the chunk's first graph
                w2 += (unsigned long long)w[q];
            }
        }
        if (rs) atomicAdd(&s_kv[cur], rs);
    }
    if (MULTI) {  // the chunk's first graph: one pair of atomics per warp
        l = warp_sum64(l);
        w2 = warp_sum64(w2);
        if (have && lane == 0 && w2) {
            atomicAdd(a.acc + 4 * (int64_t)s_g[0], l);
            atomicAdd(a.acc + 4 * (int64_t)s_g[0] + 1, w2);
        }
        l = w2 = 0;
    }
    __syncwarp();  // s_kv of the warp's rows complete

    // K: the rows' parts, combined per community within the warp; the block's
    // first community is combined over the block
    for (int k0 = 0; k0 < nr; k0 += 32) {  // warp-uniform bounds
        const int k = k0 + lane;
        const bool valid = k < nr;
        const int64_t slot = valid ? (MULTI ? (int64_t)s_vb[k] : 0) + s_c[k] : -1;
        const uint32_t kv = valid ? s_kv[k] : 0u;
        const unsigned grp = __match_any_sync(FULL, (unsigned long long)slot);
        const unsigned long long sum = group_sum(grp, kv);
        if (valid && lane == __ffs(grp) - 1 && sum) {
            if (slot == dom)
                atomicAdd(&s_dom, sum);
            else
                atomicAdd(a.kc + slot, sum);
        }
    }
    __syncwarp();  // the next group stages over this one's rows
    }
    if (MULTI)
        run.flush(a.acc);
    else
        block_flush_lw(a.acc, l, w2);  // every thread; its barriers also complete s_dom
    __syncthreads();
    if (threadIdx.x == 0 && s_dom) atomicAdd(a.kc + dom, s_dom);
}

// The rows of the small bucket (the list's first nsmall items, at most 32
// entries each), one row per lane: its weight k_v and the weight of its
// entries whose neighbour carries its label; k_v goes to K of its community,
// combined over the lanes of the same community.  The community of the
// block's first row is summed in shared memory over every row the block
// visits (a converged labelling often has a giant community, whose K would
// otherwise take one global atomic per warp step on a single address).
template <bool MULTI>
__global__ void __launch_bounds__(256) k_mod_small(ModArgs a)
{
    __shared__ unsigned long long s_dom;  // K part of the block's first community
    __shared__ int64_t s_dom_slot;
    const int lane = threadIdx.x & 31;
    const int64_t warps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    if (threadIdx.x == 0) {
        s_dom = 0ull;
        s_dom_slot = -1;
        const int64_t i0 = (int64_t)blockIdx.x * blockDim.x;
        if (i0 < a.nsmall) {
            const int32_t v = a.list[i0];
            s_dom_slot = (MULTI ? (int64_t)a.g_vbase[a.vgraph[v]] : 0) + a.lab[v];
        }
    }
    __syncthreads();
    const int64_t dom = s_dom_slot;
    unsigned long long l = 0, w2 = 0;
    for (int64_t base = (((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5) * 32;
         base < a.nsmall; base += warps * 32) {  // warp-uniform bounds
        const int64_t i = base + lane;
        const bool valid = i < a.nsmall;
        int32_t c = EMPTY, g = 0;
        int64_t vb = 0;
        uint32_t kv = 0u, lv = 0u;
        if (valid) {
            const int32_t v = a.list[i];
            if (MULTI) {
                g = a.vgraph[v];
                vb = a.g_vbase[g];
            }
            c = a.lab[v];
            const int64_t e1 = a.rp[i + 1];
            for (int64_t e = a.rp[i]; e < e1; e += 4) {  // four entries, then four gathers, in flight
                int32_t u[4];
                uint32_t w[4];
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const bool in = e + q < e1;
                    u[q] = in ? a.idx[e + q] & MOD_ID_MASK : 0;
                    w[q] = in ? (a.wts ? (uint32_t)a.wts[e + q] : 1u) : 0u;
                }
                int32_t cu[4];
#pragma unroll
                for (int q = 0; q < 4; ++q) cu[q] = w[q] ? __ldg(a.lab + vb + u[q]) : EMPTY;
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    kv += w[q];
                    if (cu[q] == c) lv += w[q];
                }
            }
        }
        // K: one atomic when the warp's rows share a community (a converged
        // labelling often has a giant one), else one per row
        const int64_t slot = valid ? vb + c : -1;
        const int64_t slot0 = __shfl_sync(FULL, slot, 0);
        if (__all_sync(FULL, !valid || slot == slot0)) {
            const unsigned long long sum = group_sum(FULL, kv);
            if (lane == 0 && sum) {
                if (slot0 == dom)
                    atomicAdd(&s_dom, sum);
                else
                    atomicAdd(a.kc + slot0, sum);
            }
        } else if (valid && kv) {
            atomicAdd(a.kc + slot, (unsigned long long)kv);
        }
        if (MULTI) {  // L and 2m: one pair of atomics when the warp's rows share a graph
            const int32_t g0 = __shfl_sync(FULL, g, 0);
            if (__all_sync(FULL, !valid || g == g0)) {
                const unsigned long long ls = group_sum(FULL, lv), ks = group_sum(FULL, kv);
                if (lane == 0 && ks) {
                    atomicAdd(a.acc + 4 * (int64_t)g0, ls);
                    atomicAdd(a.acc + 4 * (int64_t)g0 + 1, ks);
                }
            } else if (valid && kv) {
                atomicAdd(a.acc + 4 * (int64_t)g, (unsigned long long)lv);
                atomicAdd(a.acc + 4 * (int64_t)g + 1, (unsigned long long)kv);
            }
        } else {
            l += lv;
            w2 += kv;
        }
    }
    if (!MULTI) block_flush_lw(a.acc, l, w2);
    __syncthreads();
    if (threadIdx.x == 0 && s_dom) atomicAdd(a.kc + dom, s_dom);
}

// one graph: 128-bit sums over the warp, then the block, then one add
__device__ __forceinline__ void sumsq_block_add(unsigned long long *s_acc, unsigned long long hi,
                                                unsigned long long lo)
{
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) {
        const unsigned long long olo = __shfl_xor_sync(FULL, lo, o);
        const unsigned long long ohi = __shfl_xor_sync(FULL, hi, o);
        lo += olo;
        hi += ohi + (lo < olo ? 1ull : 0ull);
    }
    __shared__ unsigned long long s_hl[2 * 8];
    const int wib = threadIdx.x >> 5;
    if ((threadIdx.x & 31) == 0) {
        s_hl[2 * wib] = hi;
        s_hl[2 * wib + 1] = lo;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int k = 1; k < (int)(blockDim.x >> 5); ++k) {
            lo += s_hl[2 * k + 1];
            hi += s_hl[2 * k] + (lo < s_hl[2 * k + 1] ? 1ull : 0ull);
        }
        if (hi | lo) add_u128(s_acc, hi, lo);
    }
}

// Square pass: S_g += K_c^2 over runs of SQ_RUN slots per thread (a graph's
// slots are its vertex range, so a run crosses few graph boundaries).
constexpr int SQ_RUN = 16;

template <bool MULTI>
__global__ void __launch_bounds__(256) k_mod_sumsq(ModArgs a, int64_t nslots)
{
    const int64_t first = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) * SQ_RUN;
    if (MULTI && first >= nslots) return;
    const int64_t last = first + SQ_RUN < nslots ? first + SQ_RUN : nslots;
    int32_t g = MULTI ? a.vgraph[first] : 0;
    unsigned long long hi = 0, lo = 0;
    for (int64_t c = first; c < last; ++c) {
        if (MULTI) {
            const int32_t gc = a.vgraph[c];
            if (gc != g) {
                if (hi | lo) add_u128(a.acc + 4 * (int64_t)g + 2, hi, lo);
                hi = lo = 0;
                g = gc;
            }
        }
        const unsigned long long k = a.kc[c];
        const unsigned long long sq_lo = k * k, sq_hi = __umul64hi(k, k);
        lo += sq_lo;
        hi += sq_hi + (lo < sq_lo ? 1ull : 0ull);
    }
    if constexpr (MULTI) {
        if (hi | lo) add_u128(a.acc + 4 * (int64_t)g + 2, hi, lo);
    } else {
        sumsq_block_add(a.acc + 2, hi, lo);
    }
}

}  // namespace

int modularity_launch(const ModArgs &a, int64_t nslots, bool multi, cudaStream_t st,
                      int64_t *launches)
{
    if (a.nsmall > 0) {
        // a grid of a few blocks per SM, so that each block's shared sum of
        // its first community covers many rows
        const int64_t b = (a.nsmall + 255) / 256;
        const unsigned blocks = (unsigned)(b < SMALL_BLOCKS ? b : SMALL_BLOCKS);
        if (multi)
            k_mod_small<true><<<blocks, 256, 0, st>>>(a);
        else
            k_mod_small<false><<<blocks, 256, 0, st>>>(a);
        ++*launches;
    }
    const int64_t chunks = a.ncopy - a.e_lo / PACK_CHUNK;  // from the chunk holding e_lo
    if (a.ne > a.e_lo && chunks > 0) {
        const int64_t groups = (chunks + MW - 1) / MW;
        const unsigned blocks = (unsigned)(groups < ENTRY_BLOCKS ? groups : ENTRY_BLOCKS);
        if (multi)
            k_mod_entries<true><<<blocks, MT, 0, st>>>(a);
        else
            k_mod_entries<false><<<blocks, MT, 0, st>>>(a);
        ++*launches;
    }
    if (nslots > 0) {
        const int64_t threads = (nslots + SQ_RUN - 1) / SQ_RUN;
        const int g = (int)((threads + 255) / 256);
        if (multi)
            k_mod_sumsq<true><<<g, 256, 0, st>>>(a, nslots);
        else
            k_mod_sumsq<false><<<g, 256, 0, st>>>(a, nslots);
        ++*launches;
    }
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

}  // namespace lp
