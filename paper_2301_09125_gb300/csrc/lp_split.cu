// Splitting disconnected communities.  RAK (Sec. 3.2) can leave a community
// whose vertices are not joined by edges inside the community; the paper
// leaves such communities as they are (remark closing Sec. 3.4).  This pass
// splits every community of a labelling into its connected components, where
// only edges between two vertices of the same community count, and labels
// each component by its smallest vertex, so the result is unique.
//
// Lock-free union-find over the vertex ids: for every stored entry (v, u)
// with u < v and lab[u] == lab[v], the roots of v and u are linked, the larger
// root under the smaller one (atomicCAS), so a component's root is always its
// smallest vertex.  find() halves paths as it walks; parents only ever point
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

// 2^glg threads per row (1 to 32, from the graph's mean degree): entries
// (v, u) with u < v inside v's community
__global__ void __launch_bounds__(256) k_split_link(const int32_t *off, const int32_t *idx,
                                                    const int32_t *lab, int32_t n, int glg,
                                                    int32_t *parent, int32_t *err)
{
    const int gs = 1 << glg;
    const int t = threadIdx.x & (gs - 1);
    const int64_t grp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> glg;
    const int64_t ng = ((int64_t)gridDim.x * blockDim.x) >> glg;
    for (int64_t v = grp; v < n; v += ng) {
        const int32_t rs = __ldg(off + v), re = __ldg(off + v + 1);
        if (re == rs) continue;
        const int32_t c = __ldg(lab + v);
        // v's root, kept across the row's entries: the walk from it to the
        // current root is short even after its tree was hung elsewhere
        int32_t rv = (int32_t)v;
        for (int32_t e = rs + t; e < re; e += gs) {
            const int32_t u = __ldg(idx + e);
            if (u < v && __ldg(lab + u) == c) rv = link(parent, rv, u, err);
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
                 int32_t *parent, int32_t *err, unsigned long long *count, int num_sms,
                 cudaStream_t st, int64_t *launches)
{
    if (n <= 0) return 0;
    k_split_init<<<grid_for(n, 256, num_sms * 8), 256, 0, st>>>(parent, n);
    // threads per row: the mean degree rounded up to a power of two, <= 32
    int glg = 0;
    while (glg < 5 && ((int64_t)1 << glg) * n < m) ++glg;
    k_split_link<<<grid_for((int64_t)n << glg, 256, num_sms * 8), 256, 0, st>>>(
        off, idx, lab, n, glg, parent, err);
    k_split_flatten<<<grid_for(n, 256, num_sms * 8), 256, 0, st>>>(parent, n, lab, count);
    *launches += 3;
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

}  // namespace lp
