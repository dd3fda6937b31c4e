// Modularity (Sec. 1) of every graph of a graph set under a labelling, in
// exact integers.  Per graph g:
//   2m  = sum of all stored weights
//   L   = sum of stored weights whose two ends carry the same label
//   K_c = sum over the vertices v of community c of k_v (k_v = row sum of v)
//   S   = sum_c K_c^2  (128-bit)
//   Q   = L / 2m - S / (2m)^2   (formed in double on the host)
//
// The entry pass reuses the sweep's degree buckets: rows of degree <= 32 are
// packed several to a warp chunk, longer rows get a warp or a CTA reading
// aligned 16-byte blocks.  Each row adds k_v to K_{c_v} with one 64-bit
// atomic; L and 2m are summed in registers and flushed once per warp (one
// graph) or per row (graph sets).  The square pass adds K_c^2 into per-graph
// 128-bit accumulators (carry-propagating 64-bit atomics).
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

// Running K_c contribution of one thread: consecutive rows of one community
// are summed in a register and added with one atomic when the community
// changes (a converged labelling often has one community for most rows, and
// atomics on one address serialise).
struct KcRun {
    int64_t slot = -1;
    unsigned long long sum = 0;
    __device__ __forceinline__ void add(unsigned long long *kc, int64_t s, unsigned long long k)
    {
        if (s != slot) {
            flush(kc);
            slot = s;
        }
        sum += k;
    }
    __device__ __forceinline__ void flush(unsigned long long *kc)
    {
        if (slot >= 0 && sum) atomicAdd(kc + slot, sum);
        sum = 0;
    }
};

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

// rows of degree 1..32, packed into 32-entry chunks (as in the small sweep)
template <bool MULTI>
__global__ void __launch_bounds__(256) k_mod_small(ModArgs a)
{
    const int lane = threadIdx.x & 31;
    const int64_t wid = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    unsigned long long l_acc = 0, w_acc = 0;
    KcRun run;
    for (int64_t tile = wid; tile * 32 < a.len; tile += nw) {
        const int64_t i = tile * 32 + lane;
        MV x{0, 0, 0, 0, 0};
        if (i < a.len) x = load_mv<MULTI>(a, a.list[i]);
        const int32_t cv = i < a.len ? __ldg(a.lab + x.v) : 0;
        int P = x.d;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(FULL, P, o);
            if (lane >= o) P += y;
        }
        const int excl = P - x.d;
        const int total_all = __shfl_sync(FULL, P, 31);
        int start = 0, base = 0;
        while (base < total_all && start < 32) {
            const unsigned fits =
                __ballot_sync(FULL, (lane >= start && P - base <= 32) || lane == start);
            const int end = 32 - __clz(fits);
            const int total = __shfl_sync(FULL, P, end - 1) - base;
            int o = start;
#pragma unroll
            for (int step = 16; step >= 1; step >>= 1) {
                const int c = o + step;
                const int ex = __shfl_sync(FULL, excl, c & 31);
                if (c < end && ex - base <= lane) o = c;
            }
            const bool act = lane < total;
            const int o_excl = __shfl_sync(FULL, excl, o);
            const long long o_e0 = __shfl_sync(FULL, (long long)x.e0, o);
            const int o_vb = MULTI ? __shfl_sync(FULL, x.vb, o) : 0;
            const int o_c = __shfl_sync(FULL, cv, o);
            const int o_g = MULTI ? __shfl_sync(FULL, x.g, o) : 0;
            uint32_t w = 0, same = 0;
            if (act) {
                const long long e = o_e0 + lane - (o_excl - base);
                const int32_t u = __ldg(a.idx + e);
                w = a.wts ? (uint32_t)__ldg(a.wts + e) : 1u;
                same = __ldg(a.lab + o_vb + u) == o_c ? w : 0u;
            }
            // one row lies wholly in the chunk: its sums are k_v and L_v (< 2^31)
            const unsigned og = __match_any_sync(FULL, act ? (unsigned)o : 0xFFFFFFFFu);
            const uint32_t kv = __reduce_add_sync(og, w);
            const uint32_t lv = __reduce_add_sync(og, same);
            if (act && lane == __ffs(og) - 1) {
                run.add(a.kc, (int64_t)o_vb + o_c, kv);
                if (MULTI) {
                    atomicAdd(a.acc + 4 * (int64_t)o_g, (unsigned long long)lv);
                    atomicAdd(a.acc + 4 * (int64_t)o_g + 1, (unsigned long long)kv);
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
    if (!MULTI) {
        l_acc = warp_sum64(l_acc);
        w_acc = warp_sum64(w_acc);
        if (lane == 0 && w_acc) {
            atomicAdd(a.acc, l_acc);
            atomicAdd(a.acc + 1, w_acc);
        }
    }
}

// rows of degree > 32: NT threads per row, aligned 16-byte blocks
template <int NT, bool MULTI>
__global__ void __launch_bounds__(256) k_mod_rows(ModArgs a)  // 256 / NT rows per CTA
{
    __shared__ unsigned long long s_l[NT / 32], s_w[NT / 32];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const int64_t grp_id = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / NT;
    const int64_t ngrp = ((int64_t)gridDim.x * blockDim.x) / NT;
    const int t = threadIdx.x % NT;
    unsigned long long l_tot = 0, w_tot = 0;
    KcRun run;
    for (int64_t item = grp_id; item < a.len; item += ngrp) {
        const MV x = load_mv<MULTI>(a, a.list[item]);
        const int32_t cv = __ldg(a.lab + x.v);
        const int64_t lo = x.e0, hi = x.e0 + x.d, b_hi = (hi - 1) >> 2;
        unsigned long long kv = 0, lv = 0;
        for (int64_t blk = (lo >> 2) + t; blk <= b_hi; blk += NT) {
            const int64_t e0 = blk * 4;
            int32_t u[4], w[4];
            if (e0 + 3 < a.ne) {
                const int4 I = __ldg(reinterpret_cast<const int4 *>(a.idx) + blk);
                u[0] = I.x; u[1] = I.y; u[2] = I.z; u[3] = I.w;
                if (a.wts) {
                    const int4 W = __ldg(reinterpret_cast<const int4 *>(a.wts) + blk);
                    w[0] = W.x; w[1] = W.y; w[2] = W.z; w[3] = W.w;
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
                    kv += (unsigned)w[j];
                    if (__ldg(a.lab + x.vb + u[j]) == cv) lv += (unsigned)w[j];
                }
            }
        }
        kv = warp_sum64(kv);
        lv = warp_sum64(lv);
        if (NT > 32) {
            if (lane == 0) {
                s_l[wib] = lv;
                s_w[wib] = kv;
            }
            __syncthreads();
            if (threadIdx.x == 0) {
                for (int k = 1; k < NT / 32; ++k) {
                    lv += s_l[k];
                    kv += s_w[k];
                }
            }
            __syncthreads();
        }
        if (t == 0) {
            run.add(a.kc, (int64_t)x.vb + cv, kv);
            if (MULTI) {
                atomicAdd(a.acc + 4 * (int64_t)x.g, lv);
                atomicAdd(a.acc + 4 * (int64_t)x.g + 1, kv);
            } else {
                l_tot += lv;
                w_tot += kv;
            }
        }
    }
    run.flush(a.kc);
    if (!MULTI && t == 0 && w_tot) {
        atomicAdd(a.acc, l_tot);
        atomicAdd(a.acc + 1, w_tot);
    }
}

// sum of K_c^2 per graph: each thread squares a run of consecutive slots and
// flushes its 128-bit sum whenever the run crosses into another graph
constexpr int SQ_RUN = 64;

template <bool MULTI>
__global__ void __launch_bounds__(256) k_mod_sumsq(ModArgs a, int64_t nslots)
{
    const int64_t first = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) * SQ_RUN;
    if (first >= nslots) return;
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
    if (hi | lo) add_u128(a.acc + 4 * (int64_t)g + 2, hi, lo);
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
        const int g = grid_cap((a.len + 255) / 256, num_sms * 16);
        if (multi) k_mod_small<true><<<g, 256, 0, st>>>(a);
        else k_mod_small<false><<<g, 256, 0, st>>>(a);
        ++*launches;
    }
    if (bucket_len[1] > 0) {
        a.list = base.list + bucket_begin[1];
        a.len = bucket_len[1];
        const int g = grid_cap((a.len + 7) / 8, num_sms * 8);
        if (multi) k_mod_rows<32, true><<<g, 256, 0, st>>>(a);
        else k_mod_rows<32, false><<<g, 256, 0, st>>>(a);
        ++*launches;
    }
    // the cta, cta2 and hub buckets are adjacent
    const int64_t big = bucket_len[2] + bucket_len[3] + bucket_len[4];
    if (big > 0) {
        a.list = base.list + bucket_begin[2];
        a.len = big;
        const int g = grid_cap(big, num_sms * 8);
        if (multi) k_mod_rows<256, true><<<g, 256, 0, st>>>(a);
        else k_mod_rows<256, false><<<g, 256, 0, st>>>(a);
        ++*launches;
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
