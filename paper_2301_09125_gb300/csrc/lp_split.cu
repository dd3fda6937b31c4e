// Splitting disconnected communities.  RAK (Sec. 3.2) can leave a community
// whose vertices are not joined by edges inside the community; the paper
// leaves such communities as they are (remark closing Sec. 3.4).  This pass
// splits every community of a labelling into its connected components, where
// only edges between two vertices of the same community count, and labels
// each component by its smallest vertex, so the result is unique.
//
// Lock-free union-find over the vertex ids: the roots of two vertices of one
// community joined by an edge are linked, the larger root under the smaller
// one (atomicCAS), so a component's root is always its smallest vertex.
// Sampling skips most of the work when one component is large (the
// subgraph-sampling idea of Afforest, Sutton, Ben-Nun & Bar-Barak 2018):
// every vertex is first linked to two same-community neighbours, the trees
// are compressed, and the root shared by most of 1024 sampled vertices is
// found; the full pass over the entries then skips the rows whose vertex
// already hangs under that root (an edge from such a row to a vertex outside
// its tree is processed from the other end).  find() halves paths as it walks; parents only ever point
// to smaller ids, so every walk ends.  A link retries only after another
// thread changed the root it tried to link, and gives up after LINK_TRIES
// attempts by raising an error word (never seen; the host reports it).
#include "lp_internal.cuh"

namespace lp {
namespace {

constexpr int LINK_TRIES = 1 << 20;

// parents are read from L2 (ld.global.cg): other SMs relink roots while this
// walk runs, and a stale L1 line would hide their links from the CAS retries
__device__ __forceinline__ int32_t find_root(int32_t *parent, int32_t x)
{
    int32_t p = __ldcg(parent + x);
    while (p != x) {
        const int32_t gp = __ldcg(parent + p);
        // path halving (a benign race: gp is still an ancestor of x), written
        // only when it shortens the path, so walks that end one step below a
        // root add no stores to the lines every walk reads
        if (gp != p) parent[x] = gp;
        x = gp;
        p = __ldcg(parent + x);
    }
    return x;
}

// Join the trees of a and b; returns the root of the joined tree as seen
// (an ancestor of a, a good start for a's next walk).
__device__ __forceinline__ int32_t link(int32_t *parent, int32_t a, int32_t b, int32_t *err)
{
    for (int tries = 0; tries < LINK_TRIES; ++tries) {
        a = find_root(parent, a);
        b = find_root(parent, b);
        if (a == b) return a;
        const int32_t hi = a > b ? a : b, lo = a > b ? b : a;
        // hang root hi under lo, unless hi stopped being a root meanwhile
        if (atomicCAS(parent + hi, hi, lo) == hi) return lo;
    }
    atomicExch(err, 1);
    return a;
}

__global__ void k_split_init(int32_t *parent, int32_t n)
{
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n;
         v += (int64_t)gridDim.x * blockDim.x)
        parent[v] = (int32_t)v;
}

// The most frequent of 1024 evenly spaced vertices' values in vals (labels,
// or roots after compression) and how many of them carry it (one block of
// 1024 threads; vals read from L2).
__device__ void sample_mode(const int32_t *vals, int32_t n, int32_t *mode, int32_t *count)
{
    constexpr int SLOTS = 2048;
    __shared__ int32_t s_key[SLOTS];
    __shared__ int32_t s_cnt[SLOTS];
    __shared__ unsigned long long s_best;
    for (int j = threadIdx.x; j < SLOTS; j += blockDim.x) {
        s_key[j] = EMPTY;
        s_cnt[j] = 0;
    }
    if (threadIdx.x == 0) s_best = 0;
    __syncthreads();
    const int32_t r = __ldcg(vals + (int64_t)threadIdx.x * n / blockDim.x);
    // 1024 keys in 2048 slots: every key finds a slot
    uint32_t h = ((uint32_t)r * 0x9E3779B1u) >> 21;
    int32_t cnt = 0;
    for (int i = 0; i < SLOTS; ++i) {
        const int32_t cur = atomicCAS(&s_key[h], EMPTY, r);
        if (cur == EMPTY || cur == r) {
            cnt = atomicAdd(&s_cnt[h], 1) + 1;
            break;
        }
        h = (h + 1) & (SLOTS - 1);
    }
    // (count, ~value) maximum: the most frequent value, the smallest on ties
    atomicMax(&s_best, ((unsigned long long)(uint32_t)cnt << 32) | (uint32_t)~(uint32_t)r);
    __syncthreads();
    *mode = (int32_t)~(uint32_t)s_best;
    *count = (int32_t)(s_best >> 32);
}

// Sampling pays off only when one community holds a large share of the
// vertices (a giant component can only lie inside one): *use = 1 if the most
// frequent sampled label carries at least an eighth of the samples.
__global__ void __launch_bounds__(1024) k_split_probe(const int32_t *lab, int32_t n,
                                                      int32_t *use)
{
    int32_t mode, count;
    sample_mode(lab, n, &mode, &count);
    if (threadIdx.x == 0) *use = count * 8 >= (int32_t)blockDim.x;
}

// Sampling pass: every vertex linked to its first two same-community
// neighbours (one thread per row).
__global__ void __launch_bounds__(256) k_split_link_two(const int32_t *off, const int32_t *idx,
                                                        const int32_t *lab, int32_t n,
                                                        const int32_t *use, int32_t *parent,
                                                        int32_t *err)
{
    if (!*use) return;
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n;
         v += (int64_t)gridDim.x * blockDim.x) {
        const int32_t rs = __ldg(off + v), re = __ldg(off + v + 1);
        const int32_t c = __ldg(lab + v);
        int linked = 0;
        int32_t rv = (int32_t)v;
        for (int32_t e = rs; e < re && linked < 2; ++e) {
            const int32_t u = __ldg(idx + e);
            if (u != v && __ldg(lab + u) == c) {
                rv = link(parent, rv, u, err);
                ++linked;
            }
        }
    }
}

// every vertex straight under its root
__global__ void k_split_compress(int32_t *parent, int32_t n, const int32_t *use)
{
    if (!*use) return;
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n;
         v += (int64_t)gridDim.x * blockDim.x)
        parent[v] = find_root(parent, (int32_t)v);
}

// One block of 1024 threads: the root most of 1024 evenly spaced vertices
// hang under, if it holds at least an eighth of them (else -1, no skipping).
__global__ void __launch_bounds__(1024) k_split_sample(const int32_t *parent, int32_t n,
                                                       const int32_t *use, int32_t *big)
{
    if (!*use) {
        if (threadIdx.x == 0) *big = -1;
        return;
    }
    int32_t mode, count;
    sample_mode(parent, n, &mode, &count);  // compressed: parents are roots
    if (threadIdx.x == 0) *big = count * 8 >= (int32_t)blockDim.x ? mode : -1;
}

// 2^glg threads per row (1 to 32, from the graph's mean degree): every
// same-community entry of the rows whose vertex is not under the big root
// (both directions, since rows under it are skipped; with no big root, every
// row and each edge from its larger end)
__global__ void __launch_bounds__(256) k_split_link(const int32_t *off, const int32_t *idx,
                                                    const int32_t *lab, int32_t n, int glg,
                                                    const int32_t *big, int32_t *parent,
                                                    int32_t *err)
{
    const int gs = 1 << glg;
    const int t = threadIdx.x & (gs - 1);
    const int64_t grp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> glg;
    const int64_t ng = ((int64_t)gridDim.x * blockDim.x) >> glg;
    const int32_t skip = *big;
    for (int64_t v = grp; v < n; v += ng) {
        const int32_t rs = __ldg(off + v), re = __ldg(off + v + 1);
        if (re == rs) continue;
        // v's root, kept across the row's entries: the walk from it to the
        // current root is short even after its tree was hung elsewhere
        int32_t rv = find_root(parent, (int32_t)v);
        if (rv == skip) continue;  // the same for the whole group
        const int32_t c = __ldg(lab + v);
        for (int32_t e = rs + t; e < re; e += gs) {
            const int32_t u = __ldg(idx + e);
            // with no rows skipped, each edge once (from its larger end)
            if ((skip >= 0 ? u != v : u < v) && __ldg(lab + u) == c)
                rv = link(parent, rv, u, err);
        }
    }
}

// labels = component roots; *count += roots
__global__ void __launch_bounds__(256) k_split_flatten(int32_t *parent, int32_t n, int32_t *lab,
                                                       unsigned long long *count)
{
    unsigned long long roots = 0;
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n;
         v += (int64_t)gridDim.x * blockDim.x) {
        int32_t x = (int32_t)v;
        while (parent[x] != x) x = parent[x];
        lab[v] = x;
        roots += x == (int32_t)v;
    }
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) roots += __shfl_xor_sync(FULL, roots, o);
    if ((threadIdx.x & 31) == 0 && roots) atomicAdd(count, roots);
}

int grid_for(int64_t items, int threads, int cap)
{
    const int64_t b = (items + threads - 1) / threads;
    return (int)(b < 1 ? 1 : (b > cap ? cap : b));
}

}  // namespace

int split_launch(const int32_t *off, const int32_t *idx, int32_t *lab, int32_t n, int64_t m,
                 int32_t *parent, int32_t *err, int32_t *big, unsigned long long *count,
                 int num_sms, cudaStream_t st, int64_t *launches)
{
    if (n <= 0) return 0;
    int32_t *use = big + 1;
    k_split_init<<<grid_for(n, 256, num_sms * 8), 256, 0, st>>>(parent, n);
    k_split_probe<<<1, 1024, 0, st>>>(lab, n, use);
    k_split_link_two<<<grid_for(n, 256, num_sms * 8), 256, 0, st>>>(off, idx, lab, n, use,
                                                                    parent, err);
    k_split_compress<<<grid_for(n, 256, num_sms * 8), 256, 0, st>>>(parent, n, use);
    k_split_sample<<<1, 1024, 0, st>>>(parent, n, use, big);
    // threads per row: the mean degree rounded up to a power of two, <= 32
    int glg = 0;
    while (glg < 5 && ((int64_t)1 << glg) * n < m) ++glg;
    k_split_link<<<grid_for((int64_t)n << glg, 256, num_sms * 8), 256, 0, st>>>(
        off, idx, lab, n, glg, big, parent, err);
    k_split_flatten<<<grid_for(n, 256, num_sms * 8), 256, 0, st>>>(parent, n, lab, count);
    *launches += 7;
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

}  // namespace lp
