// Modularity (Sec. 1) of one graph under a labelling, in exact integers.
//
//   2m  = sum of all stored weights
//   L   = sum of stored weights whose two ends carry the same label
//   K_c = sum over the vertices v of community c of k_v (= row sum of v)
//   S   = sum_c K_c^2  (128-bit)
//   Q   = L / 2m - S / (2m)^2   (formed in double by the caller)
//
// k_mod_entries walks the entries in fixed 256-entry slices per warp (all
// loads coalesced), finds each entry's row by a binary search bounded by the
// slice's first and last row, and merges the weights of one row inside the
// warp (match + redux) before a single 64-bit atomic into K_c.
// k_mod_sumsq squares K_c into per-block 128-bit partial sums.
#include "lp_internal.cuh"

namespace lp {
namespace {

constexpr int SLICE = 256;  // entries per warp slice

// largest v in [lo, hi] with off[v] <= e  (off non-decreasing, off[lo] <= e)
__device__ __forceinline__ int32_t row_of(const int32_t *off, int32_t lo, int32_t hi, int64_t e)
{
    while (lo < hi) {
        const int32_t mid = lo + ((hi - lo + 1) >> 1);
        if ((int64_t)__ldg(off + mid) <= e)
            lo = mid;
        else
            hi = mid - 1;
    }
    return lo;
}

__global__ void __launch_bounds__(256) k_mod_entries(ModArgs a)
{
    const int lane = threadIdx.x & 31;
    const int64_t wid = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    unsigned long long l_in = 0, tw = 0;
    for (int64_t s0 = wid * SLICE; s0 < a.m; s0 += nw * SLICE) {
        const int64_t s1 = s0 + SLICE < a.m ? s0 + SLICE : a.m;
        // rows holding the slice's first and last entries (lane 0 searches)
        int32_t vlo = 0, vhi = 0;
        if (lane == 0) {
            vlo = row_of(a.off, 0, a.n - 1, s0);
            vhi = row_of(a.off, vlo, a.n - 1, s1 - 1);
        }
        vlo = __shfl_sync(FULL, vlo, 0);
        vhi = __shfl_sync(FULL, vhi, 0);
        for (int64_t e0 = s0; e0 < s1; e0 += 32) {
            const int64_t e = e0 + lane;
            const bool act = e < s1;
            int32_t v = -1, cv = 0;
            uint32_t w = 0;
            if (act) {
                v = row_of(a.off, vlo, vhi, e);
                const int32_t u = __ldg(a.idx + e);
                w = a.wts ? (uint32_t)__ldg(a.wts + e) : 1u;
                cv = a.lab[v];
                if (a.lab[u] == cv) l_in += w;
                tw += w;
            }
            // one row's weights in this group sum to < 2^31 (checked at ingest)
            const unsigned grp = __match_any_sync(FULL, v);
            const uint32_t s = __reduce_add_sync(grp, w);
            if (act && lane == __ffs(grp) - 1) atomicAdd(a.kc + cv, (unsigned long long)s);
        }
    }
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) {
        l_in += __shfl_xor_sync(FULL, l_in, o);
        tw += __shfl_xor_sync(FULL, tw, o);
    }
    if (lane == 0 && tw) {
        atomicAdd(a.acc + 0, l_in);
        atomicAdd(a.acc + 1, tw);
    }
}

struct U128 {
    unsigned long long hi, lo;
};

__device__ __forceinline__ U128 add128(U128 x, U128 y)
{
    U128 r;
    r.lo = x.lo + y.lo;
    r.hi = x.hi + y.hi + (r.lo < x.lo ? 1ull : 0ull);
    return r;
}

__global__ void __launch_bounds__(256) k_mod_sumsq(const unsigned long long *kc, int64_t n,
                                                   unsigned long long *partials)
{
    __shared__ U128 s_red[8];
    U128 acc{0ull, 0ull};
    for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < n;
         c += (int64_t)gridDim.x * blockDim.x) {
        const unsigned long long k = kc[c];
        acc = add128(acc, U128{__umul64hi(k, k), k * k});
    }
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) {
        U128 y{__shfl_xor_sync(FULL, acc.hi, o), __shfl_xor_sync(FULL, acc.lo, o)};
        acc = add128(acc, y);
    }
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    if (lane == 0) s_red[wib] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        U128 t{0ull, 0ull};
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t = add128(t, s_red[w]);
        partials[2 * blockIdx.x] = t.hi;
        partials[2 * blockIdx.x + 1] = t.lo;
    }
}

}  // namespace

int modularity_entries(const ModArgs &a, int num_sms, cudaStream_t st, int64_t *launches)
{
    if (a.m == 0 || a.n == 0) return 0;
    const int64_t warps = (a.m + SLICE - 1) / SLICE;
    int64_t blocks = (warps + 7) / 8;
    if (blocks > (int64_t)num_sms * 16) blocks = (int64_t)num_sms * 16;
    k_mod_entries<<<(int)blocks, 256, 0, st>>>(a);
    ++*launches;
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

int modularity_sumsq(const unsigned long long *kc, int64_t n, unsigned long long *partials,
                     int blocks, cudaStream_t st, int64_t *launches)
{
    k_mod_sumsq<<<blocks, 256, 0, st>>>(kc, n, partials);
    ++*launches;
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

}  // namespace lp
