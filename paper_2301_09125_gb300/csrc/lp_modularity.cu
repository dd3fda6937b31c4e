// Modularity (Sec. 1) of every graph of a graph set under a labelling, in
// exact integers.  Per graph g:
//   2m  = sum of all stored weights
//   L   = sum of stored weights whose two ends carry the same label
//   K_c = sum over the vertices v of community c of k_v (k_v = row sum of v)
//   S   = sum_c K_c^2  (128-bit)
//   Q   = L / 2m - S / (2m)^2   (formed in double on the host)
//
// The entry pass reuses the sweep's degree buckets: tiles of small rows of at
// most 8 entries take one lane per row, other rows of the small bucket
// (<= 32 entries) are read as aligned 16-byte blocks packed several rows to a
// 32-block warp chunk, longer rows get a warp or a CTA of 128, 256 or 512
// threads reading aligned blocks.  Each row adds k_v to K_{c_v}: rows of one
// community in a chunk are summed first, and every thread keeps running sums
// for two communities (one 64-bit atomic when one is evicted).  L and 2m are
// summed in registers and flushed once per block (one graph) or whenever a
// thread's rows move to another graph (graph sets).  The square pass adds
// K_c^2 into per-graph 128-bit accumulators (carry-propagating 64-bit
// atomics).
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

// Running K_c contributions of one thread, cached for two communities:
// consecutive rows of a cached community are summed in a register and added
// with one atomic when the entry is evicted (least recently used).  A
// converged labelling often has one giant community, and atomics on one
// address serialise, so the giant community's slot should stay cached.
struct KcRun {
    int64_t s0 = -1, s1 = -1;
    unsigned long long k0 = 0, k1 = 0;
    __device__ __forceinline__ void add(unsigned long long *kc, int64_t s, unsigned long long k)
    {
        if (s == s0) {
            k0 += k;
            return;
        }
        if (s == s1) {  // becomes the most recent entry
            s1 = s0;
            s0 = s;
            const unsigned long long t = k1;
            k1 = k0;
            k0 = t + k;
            return;
        }
        if (s1 >= 0 && k1) atomicAdd(kc + s1, k1);
        s1 = s0;
        k1 = k0;
        s0 = s;
        k0 = k;
    }
    __device__ __forceinline__ void flush(unsigned long long *kc)
    {
        if (s0 >= 0 && k0) atomicAdd(kc + s0, k0);
        if (s1 >= 0 && k1) atomicAdd(kc + s1, k1);
        k0 = k1 = 0;
    }
};

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

struct MV {  // one vertex as the modularity pass sees it
    int32_t v, g, vb, d;
    int64_t e0;
};

template <bool MULTI>
__device__ __forceinline__ MV load_mv(const ModArgs &a, int32_t v)
{
    MV x;
    x.v = v;
    x.g = MULTI ? a.vgraph[v] : 0;
    x.vb = MULTI ? a.g_vbase[x.g] : 0;
    const int64_t ob = (int64_t)v + x.g;  // graph g's offsets start at vbase_g + g
    const int32_t rs = __ldg(a.off + ob);
    x.d = __ldg(a.off + ob + 1) - rs;
    x.e0 = (MULTI ? a.g_ebase[x.g] : 0) + rs;
    return x;
}

// One 16-byte block of a row's entries: summed weight (k part) and summed
// weight of the entries whose neighbour carries label c (L part).
__device__ __forceinline__ void mod_block(const ModArgs &a, int64_t blk, int64_t lo, int64_t hi,
                                          int32_t vb, int32_t c, uint32_t &kw, uint32_t &lw)
{
    const int64_t e0 = blk * 4;
    int32_t u[4], w[4];
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
    } else {
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            u[j] = e0 + j < a.ne ? __ldg(a.idx + e0 + j) : 0;
            w[j] = e0 + j < a.ne ? (a.wts ? __ldg(a.wts + e0 + j) : 1) : 0;
        }
    }
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        if (e0 + j >= lo && e0 + j < hi) {
            kw += (uint32_t)w[j];
            if (ld_label(a.lab + vb + u[j]) == c) lw += (uint32_t)w[j];
        }
    }
}

constexpr int MOD_TINY = 8;

// tiles whose rows all have degree <= MOD_TINY: one lane per row; other
// tiles: rows as aligned blocks (<= 9 per row), whole rows packed into
// 32-block chunks
template <bool MULTI>
__global__ void __launch_bounds__(256) k_mod_small(ModArgs a)
{
    const int lane = threadIdx.x & 31;
    const int64_t wid = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    unsigned long long l_acc = 0, w_acc = 0;
    KcRun run;
    AccRun graph_run;
    const int rt = a.tile_rows;  // rows per tile: lanes rt..31 hold none
    for (int64_t tile = wid; tile * rt < a.len; tile += nw) {
        const int64_t i = tile * rt + lane;
        const bool have = lane < rt && i < a.len;
        MV x{0, 0, 0, 0, 0};
        if (have) x = load_mv<MULTI>(a, a.list[i]);
        const int32_t cv = have ? __ldg(a.lab + x.v) : 0;
        // a tile of rows of up to MOD_TINY entries: each lane sums its own row
        // (a tile that mixes in longer rows takes the packed pass: a second
        // chain of dependent loads in the same tile costs more than it saves)
        if (__all_sync(FULL, x.d <= MOD_TINY) && x.d >= 1) {
            uint32_t kw = 0, lw = 0;
#pragma unroll
            for (int j = 0; j < MOD_TINY; ++j) {
                if (j < x.d) {
                    const int64_t e = x.e0 + j;
                    const int32_t u = ld_entry(a.idx + e);
                    const uint32_t w = a.wts ? (uint32_t)ld_entry(a.wts + e) : 1u;
                    kw += w;
                    if (ld_label(a.lab + x.vb + u) == cv) lw += w;
                }
            }
            run.add(a.kc, (int64_t)x.vb + cv, kw);
            if (MULTI) {
                graph_run.add(a.acc, x.g, lw, kw);
            } else {
                l_acc += lw;
                w_acc += kw;
            }
            x.d = 0;  // done: left out of the packed pass
        }
        const int64_t q0 = x.e0 >> 2;
        const int nq = x.d > 0 ? (int)(((x.e0 + x.d - 1) >> 2) - q0 + 1) : 0;
        int Q = nq;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(FULL, Q, o);
            if (lane >= o) Q += y;
        }
        const int qexcl = Q - nq;
        const int qtotal = __shfl_sync(FULL, Q, 31);
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
            const int o_d = __shfl_sync(FULL, x.d, o);
            const int o_vb = MULTI ? __shfl_sync(FULL, x.vb, o) : 0;
            const int o_c = __shfl_sync(FULL, cv, o);
            const int o_g = MULTI ? __shfl_sync(FULL, x.g, o) : 0;
            const int o_qex = __shfl_sync(FULL, qexcl, o);
            uint32_t kw = 0, lw = 0;
            if (act)
                mod_block(a, (o_e0 >> 2) + (lane - (o_qex - base)), o_e0, o_e0 + o_d, o_vb, o_c,
                          kw, lw);
            // the row's blocks fill lanes [o_qex - base, + its block count); one
            // row lies wholly in the chunk, so its sums are k_v and L_v (< 2^31)
            const int o_nq = (int)(((o_e0 + o_d - 1) >> 2) - (o_e0 >> 2) + 1);
            const unsigned og = act ? lane_range(o_qex - base, o_nq) : ~lane_range(0, total);
            const uint32_t kv = __reduce_add_sync(og, kw);
            const uint32_t lv = __reduce_add_sync(og, lw);
            const bool row_lead = act && lane == __ffs(og) - 1;
            // rows of one community in the chunk add to K_c together: k_v < 2^31,
            // so the sum is formed from 16-bit halves (each sum < 2^21)
            const int32_t slot = o_vb + o_c;  // < 2^31 (vertex count bound)
            const unsigned sg = __match_any_sync(FULL, row_lead ? (unsigned)slot : 0xFFFFFFFFu);
            const uint32_t k_lo = __reduce_add_sync(sg, row_lead ? kv & 0xFFFFu : 0u);
            const uint32_t k_hi = __reduce_add_sync(sg, row_lead ? kv >> 16 : 0u);
            if (row_lead) {
                if (lane == __ffs(sg) - 1)
                    run.add(a.kc, slot, (unsigned long long)k_lo + ((unsigned long long)k_hi << 16));
                if (MULTI) {
                    graph_run.add(a.acc, o_g, lv, kv);
                } else {
                    l_acc += lv;
                    w_acc += kv;
                }
            }
            base += total;
            start = end;
        }
    }
    run.flush(a.kc);
    if (MULTI)
        graph_run.flush(a.acc);
    else
        block_flush_lw(a.acc, l_acc, w_acc);
}

// rows of degree > 32: NT threads per row, aligned 16-byte blocks
template <int NT, bool MULTI>
__global__ void __launch_bounds__(NT > 256 ? NT : 256) k_mod_rows(ModArgs a)
{
    constexpr int BT = NT > 256 ? NT : 256;  // threads per CTA: BT / NT rows at a time
    __shared__ unsigned long long s_l[BT / 32], s_w[BT / 32];
    constexpr int G = BT / NT;  // rows per CTA at a time
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const int grp = threadIdx.x / NT;
    const int t = threadIdx.x % NT;
    unsigned long long l_tot = 0, w_tot = 0;
    KcRun run;
    AccRun graph_run;
    // every group of the CTA makes the same number of trips (barriers below)
    for (int64_t base = (int64_t)blockIdx.x * G; base < a.len; base += (int64_t)gridDim.x * G) {
        const int64_t item = base + grp;
        const bool have = item < a.len;
        MV x{0, 0, 0, 0, 0};
        int32_t cv = 0;
        if (have) {
            x = load_mv<MULTI>(a, a.list[item]);
            cv = __ldg(a.lab + x.v);
        }
        const int64_t lo = x.e0, hi = x.e0 + x.d, b_hi = (hi - 1) >> 2;
        uint32_t kw = 0, lw = 0;  // row sums < 2^31 (ingest bound)
        if (have)
            for (int64_t blk = (lo >> 2) + t; blk <= b_hi; blk += NT)
                mod_block(a, blk, lo, hi, x.vb, cv, kw, lw);
        unsigned long long kv = __reduce_add_sync(FULL, kw);
        unsigned long long lv = __reduce_add_sync(FULL, lw);
        if (NT > 32) {
            if (lane == 0) {
                s_l[wib] = lv;
                s_w[wib] = kv;
            }
            __syncthreads();
            if (t == 0) {
                const int w0 = wib;  // first warp of this row's group
                for (int k = 1; k < NT / 32; ++k) {
                    lv += s_l[w0 + k];
                    kv += s_w[w0 + k];
                }
            }
            __syncthreads();
        }
        if (t == 0 && have) {
            run.add(a.kc, (int64_t)x.vb + cv, kv);
            if (MULTI) {
                graph_run.add(a.acc, x.g, lv, kv);
            } else {
                l_tot += lv;
                w_tot += kv;
            }
        }
    }
    run.flush(a.kc);
    if (MULTI)
        graph_run.flush(a.acc);
    else
        block_flush_lw(a.acc, l_tot, w_tot);
}

// sum of K_c^2 per graph: each thread squares a run of consecutive slots and
// flushes its 128-bit sum whenever the run crosses into another graph
constexpr int SQ_RUN = 64;

__device__ __forceinline__ void sumsq_block_add(unsigned long long *s_acc, unsigned long long hi,
                                                unsigned long long lo);

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

int grid_cap(int64_t blocks, int cap) { return (int)(blocks < 1 ? 1 : (blocks > cap ? cap : blocks)); }

}  // namespace

int modularity_launch(const ModArgs &base, const int64_t *bucket_begin, const int64_t *bucket_len,
                      int64_t nslots, bool multi, int num_sms, cudaStream_t st, int64_t *launches)
{
    ModArgs a = base;
    if (bucket_len[0] > 0) {
        a.list = base.list + bucket_begin[0];
        a.len = bucket_len[0];
        a.tile_rows = small_tile_rows(a.len, a.small_mean_deg, num_sms);
        const int g = grid_cap(((a.len + a.tile_rows - 1) / a.tile_rows + 7) / 8, num_sms * 16);
        if (multi) k_mod_small<true><<<g, 256, 0, st>>>(a);
        else k_mod_small<false><<<g, 256, 0, st>>>(a);
        ++*launches;
    }
    // one warp per row (warp bucket), 128 / 256 / 512 threads per row (cta,
    // cta2 and hub buckets)
    auto rows = [&](int b, auto kernel, int nt, int bt) {
        if (bucket_len[b] <= 0) return;
        a.list = base.list + bucket_begin[b];
        a.len = bucket_len[b];
        const int64_t per_cta = bt / nt;
        const int g = grid_cap((a.len + per_cta - 1) / per_cta, num_sms * (2048 / bt));
        kernel<<<g, bt, 0, st>>>(a);
        ++*launches;
    };
    if (multi) {
        rows(1, k_mod_rows<32, true>, 32, 256);
        rows(2, k_mod_rows<128, true>, 128, 256);
        rows(3, k_mod_rows<256, true>, 256, 256);
        rows(4, k_mod_rows<512, true>, 512, 512);
    } else {
        rows(1, k_mod_rows<32, false>, 32, 256);
        rows(2, k_mod_rows<128, false>, 128, 256);
        rows(3, k_mod_rows<256, false>, 256, 256);
        rows(4, k_mod_rows<512, false>, 512, 512);
    }
    if (nslots > 0) {
        const int64_t threads = (nslots + SQ_RUN - 1) / SQ_RUN;
        const int g = (int)((threads + 255) / 256);
        if (multi) k_mod_sumsq<true><<<g, 256, 0, st>>>(a, nslots);
        else k_mod_sumsq<false><<<g, 256, 0, st>>>(a, nslots);
        ++*launches;
    }
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

}  // namespace lp
