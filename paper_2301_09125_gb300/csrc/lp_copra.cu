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
// One CTA per vertex: the (label, T, first appearance) table lives in shared
// memory for rows of at most CP_PAIRS pairs and in a per-CTA region of global
// memory for longer rows (a second launch with fewer CTAs).  A label's first
// appearance is encoded as row position * 64 + pair index, which orders the
// pairs as the row scan meets them.
#include "lp_device.cuh"
#include "lp_internal.cuh"

namespace lp {
namespace {

constexpr int CP_T = 256;
constexpr int CP_LG = 12;
constexpr int CP_TAB = 1 << CP_LG;    // shared slots per CTA
constexpr int CP_PAIRS = CP_TAB / 2;  // rows of at most this many pairs use shared memory

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

// add (label l, value val, first appearance f) to a table of mask + 1 slots
// (shared or global memory) that has room for every label of the row
__device__ __forceinline__ void cp_insert(int32_t *key, unsigned long long *sum,
                                          unsigned long long *first, int lg, int32_t l,
                                          unsigned long long val, unsigned long long f)
{
    const uint32_t mask = (1u << lg) - 1u;
    volatile int32_t *vk = key;
    uint32_t h = slot_hash(l, lg);
    for (uint32_t i = 0; i <= mask; ++i) {
        int32_t cur = vk[h];
        if (cur == EMPTY) {
            cur = atomicCAS(key + h, EMPTY, l);
            if (cur == EMPTY) cur = l;
        }
        if (cur == l) {
            atomicAdd(sum + h, val);
            atomicMin(first + h, f);
            return;
        }
        h = (h + 1) & mask;
    }
}

__device__ __forceinline__ unsigned long long cp_warp_sum(unsigned long long v)
{
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) v += __shfl_xor_sync(FULL, v, o);
    return v;
}

// One COPRA step for the vertices of wave wave_k whose rows hold more pairs
// than CP_PAIRS (BIG) or at most that many (the others).
template <bool BIG>
__global__ void __launch_bounds__(CP_T) k_copra(CopraArgs a)
{
    extern __shared__ unsigned long long cp_smem[];
    __shared__ CpCand s_red[CP_T / 32];
    __shared__ unsigned long long s_w[CP_T / 32];
    __shared__ int32_t s_kept[64];
    __shared__ int s_nk;
    const int tid = threadIdx.x, lane = tid & 31, wib = tid >> 5;
    int32_t *key;
    unsigned long long *sum, *first;
    if (BIG) {  // this CTA's region of the global tables (clean at every row's start)
        const int64_t base = (int64_t)blockIdx.x << a.glg_max;
        key = a.gkey + base;
        sum = a.gsum + base;
        first = a.gfirst + base;
    } else {
        sum = cp_smem;
        first = sum + CP_TAB;
        key = reinterpret_cast<int32_t *>(first + CP_TAB);
        for (int j = tid; j < CP_TAB; j += CP_T) {
            key[j] = EMPTY;
            sum[j] = 0ull;
            first[j] = ~0ull;
        }
        __syncthreads();
    }
    const uint32_t L = (uint32_t)a.L;
    uint32_t my_changed = 0;
    for (int32_t v = blockIdx.x; v < a.n; v += gridDim.x) {
        if (a.waves > 1 && fastmod((uint32_t)v, a.magic, a.waves) != a.wave_k) continue;
        const int32_t rs = __ldg(a.off + v), d = __ldg(a.off + v + 1) - rs;
        const int64_t pairs = (int64_t)d * L;
        if ((pairs > CP_PAIRS) != BIG) continue;  // block-uniform
        const int32_t prev = a.cur_l[(int64_t)v * L];
        int32_t *out_l = a.nxt_l + (int64_t)v * L;
        uint32_t *out_b = a.nxt_b + (int64_t)v * L;
        if (d == 0) {  // no labels: the vertex is its own community
            for (uint32_t s = tid; s < L; s += CP_T) {
                out_l[s] = s == 0 ? v : EMPTY;
                out_b[s] = s == 0 ? COPRA_ONE : 0u;
            }
            if (tid == 0 && prev != v) ++my_changed;
            continue;
        }
        const int lg = ilog2_ceil((uint32_t)(2 * pairs));  // 2^lg >= 2 pairs (<= 2^glg_max)
        const int slots = 1 << lg;
        // T(l) and first appearance over the row's entries and their speakers' pairs
        unsigned long long wsum = 0ull;
        for (int32_t e = tid; e < d; e += CP_T) {
            const int32_t u = __ldg(a.idx + rs + e);
            const uint32_t w = a.wts ? (uint32_t)__ldg(a.wts + rs + e) : 1u;
            wsum += w;
            const bool earlier = a.waves > 1 && fastmod((uint32_t)u, a.magic, a.waves) < a.wave_k;
            const int32_t *ul = (earlier ? a.nxt_l : a.cur_l) + (int64_t)u * L;
            const uint32_t *ub = (earlier ? a.nxt_b : a.cur_b) + (int64_t)u * L;
            for (uint32_t p = 0; p < L; ++p) {
                const uint32_t b = ub[p];
                if (b == 0u) break;
                cp_insert(key, sum, first, lg, ul[p], (unsigned long long)w * b,
                          (unsigned long long)e * 64ull + p);
            }
        }
        wsum = cp_warp_sum(wsum);
        if (lane == 0) s_w[wib] = wsum;
        if (tid == 0) s_nk = 0;
        __syncthreads();
        unsigned long long W = 0ull;
#pragma unroll
        for (int k = 0; k < CP_T / 32; ++k) W += s_w[k];
        // the labels above the threshold and the best label
        const uint64_t ktv = stream_at(a.key_t, (uint64_t)v + 1);
        CpCand best{0ull, 0ull, 0ull, -1};
        for (int j = tid; j < slots; j += CP_T) {
            const int32_t l = key[j];
            if (l == EMPTY) continue;
            const unsigned long long t = sum[j];
            if ((unsigned long long)L * t >= W * (unsigned long long)COPRA_ONE) {
                const int at = atomicAdd(&s_nk, 1);
                if (at < 64) s_kept[at] = j;  // at most L labels pass
            }
            const CpCand c{t, a.strict ? 0ull : stream_at(ktv, (uint64_t)l + 1), first[j], j};
            if (cp_better(c, best)) best = c;
        }
#pragma unroll
        for (int o = 16; o >= 1; o >>= 1) {
            const CpCand y = cp_shfl(best, o);
            if (cp_better(y, best)) best = y;
        }
        if (lane == 0) s_red[wib] = best;
        __syncthreads();
        if (tid == 0) {
            best = s_red[0];
            for (int k = 1; k < CP_T / 32; ++k)
                if (cp_better(s_red[k], best)) best = s_red[k];
            int nk = s_nk < 64 ? s_nk : 64;
            if (nk == 0) {  // none above the threshold: the best label alone
                s_kept[0] = best.slot;
                nk = 1;
            }
            // normalize in fixed point, the remainder to the best kept label
            unsigned long long tk = 0ull;
            for (int i = 0; i < nk; ++i) tk += sum[s_kept[i]];
            uint32_t bv[64];
            uint32_t bsum = 0u;
            int bi = 0;
            CpCand cb{};
            for (int i = 0; i < nk; ++i) {
                const int j = s_kept[i];
                bv[i] = (uint32_t)((sum[j] * (unsigned long long)COPRA_ONE) / tk);
                bsum += bv[i];
                const CpCand c{sum[j], a.strict ? 0ull : stream_at(ktv, (uint64_t)key[j] + 1),
                               first[j], j};
                if (i == 0 || cp_better(c, cb)) {
                    cb = c;
                    bi = i;
                }
            }
            bv[bi] += COPRA_ONE - bsum;
            // store by decreasing belonging, equal belongings by first appearance
            for (int i = 0; i < nk; ++i) {
                int pick = -1;
                for (int q = 0; q < nk; ++q) {
                    if (s_kept[q] < 0) continue;
                    if (pick < 0 || bv[q] > bv[pick] ||
                        (bv[q] == bv[pick] && first[s_kept[q]] < first[s_kept[pick]]))
                        pick = q;
                }
                out_l[i] = key[s_kept[pick]];
                out_b[i] = bv[pick];
                s_kept[pick] = -1 - s_kept[pick];  // taken
            }
            for (uint32_t s = nk; s < L; ++s) {
                out_l[s] = EMPTY;
                out_b[s] = 0u;
            }
            if (out_l[0] != prev) ++my_changed;
        }
        __syncthreads();
        for (int j = tid; j < slots; j += CP_T) {  // leave the table clean
            if (key[j] != EMPTY) {
                key[j] = EMPTY;
                sum[j] = 0ull;
                first[j] = ~0ull;
            }
        }
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
    const int bytes = CP_TAB * (8 + 8 + 4);
    return cudaFuncSetAttribute(k_copra<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                bytes) == cudaSuccess
               ? 0
               : -1;
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
    const int grid = s.n < num_sms * 2 ? s.n : num_sms * 2;
    k_copra<false><<<grid, CP_T, CP_TAB * (8 + 8 + 4), st>>>(a);
    ++*launches;
    if (s.glg_max > 0) {
        k_copra<true><<<copra_big_ctas(), CP_T, 0, st>>>(a);
        ++*launches;
    }
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

}  // namespace lp
