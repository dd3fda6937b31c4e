// Graph ingest: CSR validation and degree bucketing of the vertices.
//
// Validation is what keeps every later kernel in bounds: offsets must be a row
// pointer (first 0, non-decreasing, last m), indices must lie in [0, n) and
// weights must be >= 1.  The per-vertex summed weight must stay below 2^31 so
// that the sweep's int32 sums are exact; it is bounded by max degree x max
// weight, and only when that bound fails are the rows summed exactly.
//
// Bucketing sorts the vertices of a graph set into the four degree buckets
// (small / warp / cta / hub) with a stable three-pass count-scan-scatter, so
// the vertices of a bucket stay in ascending id order (coalesced row pointer
// and label accesses in the sweep).
#include "lp_device.cuh"
#include "lp_internal.cuh"

namespace lp {
namespace {

constexpr int BK = 1024;  // threads per bucketing block

// The counting passes (buckets, wave classes, packed row starts) take their
// items in tiles of 1024, each block a run of `per` consecutive tiles, with
// at most TILE_BLOCKS blocks: a few waves of blocks that loop over several
// tiles, rather than one short block per tile (which left these passes
// bound by block scheduling on graphs of millions of vertices).  Per-block
// counts are scanned over the blocks in order, so positions follow the
// items' order as with one block per tile.
constexpr int64_t TILE_BLOCKS = 1024;
// the packing's row-start pass does more per tile (six loads, a block scan,
// three stores): more blocks of fewer tiles each
constexpr int64_t PACK_TILE_BLOCKS = 4096;
struct TileGrid {
    int64_t ntiles, per, nblk;
};
inline TileGrid tile_grid(int64_t items, int64_t max_blocks = TILE_BLOCKS)
{
    TileGrid t;
    t.ntiles = items > 0 ? (items + BK - 1) / BK : 0;
    t.per = t.ntiles > max_blocks ? (t.ntiles + max_blocks - 1) / max_blocks : 1;
    t.nblk = (t.ntiles + t.per - 1) / t.per;
    return t;
}

__device__ __forceinline__ void report(IngestOut *o, int32_t code, int64_t at)
{
    if (atomicCAS(&o->err, 0, code) == 0) o->err_at = (int32_t)(at > 2147483647 ? 2147483647 : at);
}

// The largest of every thread's x into *dst with one global atomic per block
// (a per-warp atomic on one address from every warp of a large grid
// serialises in L2); every thread of the block calls this.
__device__ __forceinline__ void block_max_into(int32_t *dst, int32_t x)
{
    __shared__ int32_t s_max;
    if (threadIdx.x == 0) s_max = 0;
    __syncthreads();
    x = (int32_t)__reduce_max_sync(FULL, (uint32_t)(x > 0 ? x : 0));
    if ((threadIdx.x & 31) == 0 && x) atomicMax(&s_max, x);
    __syncthreads();
    if (threadIdx.x == 0 && s_max) atomicMax(dst, s_max);
}

__global__ void k_val_offsets(const int32_t *off, int32_t n, int64_t m, IngestOut *o)
{
    int32_t local_max = 0;
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v <= n;
         v += (int64_t)gridDim.x * blockDim.x) {
        const int32_t x = off[v];
        if (v == 0 && x != 0) report(o, ING_OFF_FIRST, 0);
        if (v == n && (int64_t)x != m) report(o, ING_OFF_LAST, n);
        if (v < n) {
            const int32_t y = off[v + 1];
            if (y < x)
                report(o, ING_OFF_ORDER, v);
            else
                local_max = max(local_max, y - x);
        }
    }
    block_max_into(&o->max_deg, local_max);
}

__global__ void k_val_entries(const int32_t *idx, const int32_t *wts, int32_t n, int64_t m,
                              IngestOut *o)
{
    int32_t wmax = 0;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < m;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int32_t u = __ldg(idx + e);
        if (u < 0 || u >= n) report(o, ING_INDEX, e);
        if (wts) {
            const int32_t w = __ldg(wts + e);
            if (w < 1)
                report(o, ING_WEIGHT, e);
            else
                wmax = max(wmax, w);
        }
    }
    if (!wts) wmax = m > 0 ? 1 : 0;
    block_max_into(&o->max_w, wmax);
}

__global__ void k_val_wdeg(const int32_t *off, const int32_t *wts, int32_t n, IngestOut *o)
{
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n;
         v += (int64_t)gridDim.x * blockDim.x) {
        int64_t s = 0;
        for (int32_t e = off[v]; e < off[v + 1]; ++e) s += wts ? wts[e] : 1;
        if (s >= 2147483648LL) report(o, ING_WDEG, v);
    }
}

// row starts of a graph set as a bitmap over global entries (rows outside
// [0, ne) are skipped: this may run before the offsets are known valid)
__global__ void k_mark_row_starts(const int32_t *off, int32_t nv, const int32_t *vgraph,
                                  const int64_t *g_ebase, int64_t ne, uint32_t *bits)
{
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < nv;
         v += (int64_t)gridDim.x * blockDim.x) {
        const int32_t g = vgraph ? vgraph[v] : 0;
        const int32_t rs = off[v + g], re = off[v + g + 1];
        if (re > rs && rs >= 0) {
            const int64_t e = (g_ebase ? g_ebase[g] : 0) + rs;
            if (e < ne) atomicOr(bits + (e >> 5), 1u << (e & 31));
        }
    }
}

// One graph's entries in 16-byte blocks: index in [0, n), weight >= 1, and
// (rows marked in bits) strictly increasing indices within each row.
__global__ void k_val_entries4(const int32_t *idx, const int32_t *wts, int32_t n, int64_t m,
                               const uint32_t *bits, IngestOut *o)
{
    int32_t wmax = 0;
    bool unordered = false;
    const int64_t nb = (m + 3) / 4;
    for (int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; b < nb;
         b += (int64_t)gridDim.x * blockDim.x) {
        const int64_t e0 = 4 * b;
        int32_t u[5], w[4];
        if (e0 + 3 < m) {
            const int4 I = __ldcs(reinterpret_cast<const int4 *>(idx) + b);
            u[0] = I.x;
            u[1] = I.y;
            u[2] = I.z;
            u[3] = I.w;
            if (wts) {
                const int4 W = __ldcs(reinterpret_cast<const int4 *>(wts) + b);
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
                u[j] = e0 + j < m ? idx[e0 + j] : 0;
                w[j] = e0 + j < m ? (wts ? wts[e0 + j] : 1) : 1;
            }
        }
        u[4] = e0 + 4 < m ? __ldg(idx + e0 + 4) : 0;
        // positions e0 .. e0 + 3 share one bitmap word; e0 + 4 may start the next
        const uint32_t word = bits[e0 >> 5];
        const uint32_t next = e0 + 4 < m ? bits[(e0 + 4) >> 5] : 0u;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int64_t e = e0 + j;
            if (e >= m) break;
            if (u[j] < 0 || u[j] >= n) report(o, ING_INDEX, e);
            if (w[j] < 1)
                report(o, ING_WEIGHT, e);
            else
                wmax = max(wmax, w[j]);
            const int64_t f = e + 1;
            if (f < m) {
                const bool starts = ((j < 3 ? word : next) >> (f & 31)) & 1u;
                unordered = unordered || (!starts && u[j] >= u[j + 1]);
            }
        }
    }
    if (__any_sync(FULL, unordered) && (threadIdx.x & 31) == 0) atomicExch(&o->repeated, 1);
    block_max_into(&o->max_w, wmax);
}

// entries e, e+1 of one row must satisfy idx[e] < idx[e+1]
__global__ void k_check_row_order(const int32_t *idx, int64_t ne, const uint32_t *bits,
                                  IngestOut *o)
{
    bool bad = false;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e + 1 < ne;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t f = e + 1;
        const bool starts = (bits[f >> 5] >> (f & 31)) & 1u;
        bad = bad || (!starts && __ldg(idx + e) >= __ldg(idx + f));
    }
    if (__any_sync(FULL, bad) && (threadIdx.x & 31) == 0) atomicExch(&o->repeated, 1);
}

__device__ __forceinline__ int bucket_of(int32_t d, const Thresholds &th)
{
    if (d <= 0) return -1;
#pragma unroll
    for (int b = 0; b < NUM_BUCKETS - 1; ++b)
        if (d <= th.max[b]) return b;
    return NUM_BUCKETS - 1;
}

// graph g's row pointer entries start at off[vbase_g + g], so global vertex v
// (of graph g) has its row bounds at off[v + g], off[v + g + 1]
__device__ __forceinline__ int32_t degree_of(const int32_t *off, const int32_t *vgraph, int32_t v)
{
    const int32_t g = vgraph ? vgraph[v] : 0;
    return off[(int64_t)v + g + 1] - off[(int64_t)v + g];
}

// Per block (a run of `per` tiles of BK vertices): its row count (blk) and
// entry count (bent) in every bucket, stored per bucket and block (the class
// scan sums them, so no global atomic is shared by the blocks).  Each thread
// counts in registers; the block adds its warps' sums once at the end.
__global__ void __launch_bounds__(BK) k_bucket_count(const int32_t *off, int32_t nv,
                                                      const int32_t *vgraph, Thresholds th,
                                                      int64_t per, int32_t *blk, int64_t *bent)
{
    __shared__ unsigned long long s_c[BK / 32][NUM_BUCKETS], s_e[BK / 32][NUM_BUCKETS];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    uint32_t cnt[NUM_BUCKETS];
    unsigned long long ent[NUM_BUCKETS];
#pragma unroll
    for (int c = 0; c < NUM_BUCKETS; ++c) {
        cnt[c] = 0u;
        ent[c] = 0ull;
    }
    const int64_t t_lo = (int64_t)blockIdx.x * per;
    for (int64_t t = t_lo; t < t_lo + per; ++t) {
        const int64_t v = t * BK + threadIdx.x;
        if (v >= nv) break;
        const int32_t d = degree_of(off, vgraph, (int32_t)v);
        const int b = bucket_of(d, th);
#pragma unroll
        for (int c = 0; c < NUM_BUCKETS; ++c)
            if (b == c) {
                ++cnt[c];
                ent[c] += (unsigned long long)d;
            }
    }
#pragma unroll
    for (int c = 0; c < NUM_BUCKETS; ++c) {
        const uint32_t wc = __reduce_add_sync(FULL, cnt[c]);
        unsigned long long we = ent[c];
#pragma unroll
        for (int o = 16; o >= 1; o >>= 1) we += __shfl_xor_sync(FULL, we, o);
        if (lane == 0) {
            s_c[wib][c] = wc;
            s_e[wib][c] = we;
        }
    }
    __syncthreads();
    if (threadIdx.x < NUM_BUCKETS) {
        unsigned long long tc = 0ull, te = 0ull;
        for (int w = 0; w < BK / 32; ++w) {
            tc += s_c[w][threadIdx.x];
            te += s_e[w][threadIdx.x];
        }
        const int64_t at = (int64_t)threadIdx.x * gridDim.x + blockIdx.x;
        blk[at] = (int32_t)tc;
        bent[at] = (int64_t)te;
    }
}


// exclusive block scan of one int per thread; returns the prefix, *total the sum
__device__ int64_t block_exclusive_scan(int64_t x, int64_t *s_warp, int64_t *total)
{
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    int64_t incl = x;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int64_t y = __shfl_up_sync(FULL, incl, o);
        if (lane >= o) incl += y;
    }
    if (lane == 31) s_warp[wib] = incl;
    __syncthreads();
    if (wib == 0) {
        int64_t w = lane < (int)(blockDim.x >> 5) ? s_warp[lane] : 0;
        int64_t wi = w;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int64_t y = __shfl_up_sync(FULL, wi, o);
            if (lane >= o) wi += y;
        }
        s_warp[lane] = wi - w;
        if (lane == 31) s_warp[32] = wi;
    }
    __syncthreads();
    const int64_t r = s_warp[wib] + incl - x;
    *total = s_warp[32];
    __syncthreads();
    return r;
}

// Exclusive block scans of K values per thread in one pass: ex[k] the prefix,
// tot[k] the block total of value k (s: shared scratch of 33 rows).
template <int K>
__device__ void block_exclusive_scan_k(const int64_t (&x)[K], int64_t (&ex)[K], int64_t (&tot)[K],
                                       int64_t (*s)[K])
{
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const int nw = (int)(blockDim.x >> 5);
    int64_t inc[K];
#pragma unroll
    for (int k = 0; k < K; ++k) {
        inc[k] = x[k];
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int64_t y = __shfl_up_sync(FULL, inc[k], o);
            if (lane >= o) inc[k] += y;
        }
        if (lane == 31) s[wib][k] = inc[k];
    }
    __syncthreads();
    if (wib == 0) {
#pragma unroll
        for (int k = 0; k < K; ++k) {
            const int64_t w = lane < nw ? s[lane][k] : 0;
            int64_t wi = w;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int64_t y = __shfl_up_sync(FULL, wi, o);
                if (lane >= o) wi += y;
            }
            s[lane][k] = wi - w;
            if (lane == 31) s[32][k] = wi;
        }
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < K; ++k) {
        ex[k] = s[wib][k] + inc[k] - x[k];
        tot[k] = s[32][k];
    }
    __syncthreads();
}

// Counting-sort scans.  Per-block counts are stored class-major: the count
// of class c in block b at hist[c * nblk + b].  One block per class turns its
// counts into exclusive offsets within the class (in place) and records the
// class size; one block then turns the sizes into class starts.
// the entries of bucket blockIdx.x: the sum of its blocks' counts
__global__ void __launch_bounds__(1024) k_bucket_entries(const int64_t *bent, int64_t nblk,
                                                          int64_t *total)
{
    __shared__ int64_t s_warp[33];
    const int64_t *e = bent + (int64_t)blockIdx.x * nblk;
    int64_t part = 0;
    for (int64_t i = threadIdx.x; i < nblk; i += 1024) part += e[i];
    int64_t tot;
    block_exclusive_scan(part, s_warp, &tot);
    if (threadIdx.x == 0) total[blockIdx.x] = tot;
}

__global__ void __launch_bounds__(1024) k_class_scan(int32_t *hist, int64_t nblk,
                                                      int64_t *class_size)
{
    __shared__ int64_t s_warp[33];
    int32_t *h = hist + (int64_t)blockIdx.x * nblk;
    int64_t running = 0;
    for (int64_t i0 = 0; i0 < nblk; i0 += 1024) {
        const int64_t i = i0 + threadIdx.x;
        const int64_t x = i < nblk ? h[i] : 0;
        int64_t tot;
        const int64_t ex = block_exclusive_scan(x, s_warp, &tot);
        if (i < nblk) h[i] = (int32_t)(running + ex);
        running += tot;
    }
    if (threadIdx.x == 0) class_size[blockIdx.x] = running;
}

__global__ void __launch_bounds__(1024) k_class_begin(const int64_t *class_size, int64_t nc,
                                                       int64_t *class_begin)
{
    __shared__ int64_t s_warp[33];
    int64_t running = 0;
    for (int64_t i0 = 0; i0 < nc; i0 += 1024) {
        const int64_t i = i0 + threadIdx.x;
        const int64_t x = i < nc ? class_size[i] : 0;
        int64_t tot;
        const int64_t ex = block_exclusive_scan(x, s_warp, &tot);
        if (i < nc) class_begin[i] = running + ex;
        running += tot;
    }
}

// Every vertex of the block's tiles to its bucket's list, in vertex order:
// bucket start + the block's offset within the bucket + the rows of earlier
// tiles of the block + the rank within the tile (warp after warp, lane after
// lane).
__global__ void __launch_bounds__(BK) k_bucket_scatter(const int32_t *off, int32_t nv,
                                                        const int32_t *vgraph, Thresholds th,
                                                        int64_t per, const int32_t *blk,
                                                        const int64_t *cnt, int32_t *list)
{
    __shared__ int s_pre[NUM_BUCKETS][BK / 32];
    __shared__ int64_t s_base[NUM_BUCKETS];
    __shared__ int s_tile[NUM_BUCKETS];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    if (threadIdx.x < NUM_BUCKETS)
        s_base[threadIdx.x] =
            cnt[NUM_BUCKETS + threadIdx.x] + blk[(int64_t)threadIdx.x * gridDim.x + blockIdx.x];
    const int64_t t_lo = (int64_t)blockIdx.x * per;
    for (int64_t t = t_lo; t < t_lo + per && t * BK < nv; ++t) {  // block-uniform
        const int64_t v = t * BK + threadIdx.x;
        const int b = v < nv ? bucket_of(degree_of(off, vgraph, (int32_t)v), th) : -1;
        int rank = 0;
#pragma unroll
        for (int c = 0; c < NUM_BUCKETS; ++c) {
            const unsigned msk = __ballot_sync(FULL, b == c);
            if (b == c) rank = __popc(msk & ((1u << lane) - 1u));
            if (lane == 0) s_pre[c][wib] = __popc(msk);
        }
        __syncthreads();  // s_pre of every warp (and s_base) written
        if (wib < NUM_BUCKETS) {  // warp c scans bucket c's 32 warp counts
            const int x = s_pre[wib][lane];
            int inc = x;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int y = __shfl_up_sync(FULL, inc, o);
                if (lane >= o) inc += y;
            }
            s_pre[wib][lane] = inc - x;
            if (lane == 31) s_tile[wib] = inc;
        }
        __syncthreads();
        if (b >= 0) list[s_base[b] + s_pre[b][wib] + rank] = (int32_t)v;
        __syncthreads();  // every read of s_pre and s_base done
        if (threadIdx.x < NUM_BUCKETS) s_base[threadIdx.x] += s_tile[threadIdx.x];
    }
}

__global__ void k_iota(int32_t *lab, int32_t nv, const int32_t *vgraph, const int32_t *g_vbase)
{
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < nv;
         v += (int64_t)gridDim.x * blockDim.x)
        lab[v] = (int32_t)v - (vgraph ? g_vbase[vgraph[v]] : 0);
}

__global__ void k_check_labels(const int32_t *lab, int32_t nv, const int32_t *vgraph,
                               const int32_t *g_n, IngestOut *o)
{
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < nv;
         v += (int64_t)gridDim.x * blockDim.x) {
        const int32_t n = g_n[vgraph ? vgraph[v] : 0];
        const int32_t l = lab[v];
        if (l < 0 || l >= n) report(o, ING_LABEL, v);
    }
}

__global__ void k_merge_final(int32_t *lab0, const int32_t *lab1, int32_t nv,
                              const int32_t *vgraph, const int32_t *g_sel)
{
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < nv;
         v += (int64_t)gridDim.x * blockDim.x)
        if (g_sel[vgraph[v]]) lab0[v] = lab1[v];
}

// ---------------------------------------------------------------------------
// hub rows: their order and their tasks, each as a few multi-block passes over
// blocks of HT rows (a block-sum pass, one scan of the block sums, a write
// pass), so that no single block walks the whole hub list
// ---------------------------------------------------------------------------
constexpr int HT = 1024;        // hub rows per block
constexpr int HUB_CLASSES = 32; // degree classes of the hub order: clz(degree)

// Shape of a hub row of d entries: [0] long (more than HUB_ONE_MAX entries),
// [1] short, [2] fallback table slots, [3] segments, [4] partitions, [5]
// partition offsets (the last four 0 for a short row).
__device__ __forceinline__ void hub_shape(int32_t d, int64_t (&x)[6])
{
    const bool big = d > HUB_ONE_MAX;
    int64_t tsz = 0, nseg = 0, npart = 0;
    if (big) {
        tsz = 1;
        while (tsz < 2 * (int64_t)d) tsz <<= 1;
        nseg = ((int64_t)d + HUB_SEG - 1) / HUB_SEG;
        npart = nseg < HUB_PMAX ? nseg : HUB_PMAX;
    }
    x[0] = big;
    x[1] = !big;
    x[2] = tsz;
    x[3] = nseg;
    x[4] = npart;
    x[5] = nseg * (npart + 1);
}

// block sums of the six shape values: bsum[blk * 6 + k]
__global__ void __launch_bounds__(HT) k_hub_task_sums(const int32_t *list, int64_t len,
                                                       const int32_t *off, const int32_t *vgraph,
                                                       int64_t *bsum)
{
    __shared__ int64_t s_scan6[33][6];
    const int64_t i = (int64_t)blockIdx.x * HT + threadIdx.x;
    int64_t x[6] = {0, 0, 0, 0, 0, 0}, ex[6], tot[6];
    if (i < len) hub_shape(degree_of(off, vgraph, list[i]), x);
    block_exclusive_scan_k<6>(x, ex, tot, s_scan6);
    if (threadIdx.x == 0) {
#pragma unroll
        for (int k = 0; k < 6; ++k) bsum[(int64_t)blockIdx.x * 6 + k] = tot[k];
    }
}

// one block: the block sums become exclusive block starts (in place); totals
// as hub_tasks reports them
__global__ void __launch_bounds__(1024) k_hub_task_scan(int64_t *bsum, int64_t nblk,
                                                         int64_t *totals)
{
    __shared__ int64_t s_scan6[33][6];
    int64_t running[6] = {0, 0, 0, 0, 0, 0};
    for (int64_t i0 = 0; i0 < nblk; i0 += 1024) {
        const int64_t i = i0 + threadIdx.x;
        int64_t x[6], ex[6], tot[6];
#pragma unroll
        for (int k = 0; k < 6; ++k) x[k] = i < nblk ? bsum[i * 6 + k] : 0;
        block_exclusive_scan_k<6>(x, ex, tot, s_scan6);
#pragma unroll
        for (int k = 0; k < 6; ++k) {
            if (i < nblk) bsum[i * 6 + k] = running[k] + ex[k];
            running[k] += tot[k];
        }
    }
    if (threadIdx.x == 0) {
        totals[0] = running[0];
        totals[1] = running[2];
        totals[2] = running[3];
        totals[3] = running[4];
        totals[4] = running[5];
    }
}

// the tasks of a block's rows: long rows at their prefix among long rows,
// short rows after every long row at their prefix among short rows
__global__ void __launch_bounds__(HT) k_hub_task_write(const int32_t *list, int64_t len,
                                                        const int32_t *off, const int32_t *vgraph,
                                                        const int64_t *bstart,
                                                        const int64_t *totals, HubTask *tasks)
{
    __shared__ int64_t s_scan6[33][6];
    const int64_t i = (int64_t)blockIdx.x * HT + threadIdx.x;
    int64_t x[6] = {0, 0, 0, 0, 0, 0}, ex[6], tot[6];
    int32_t v = 0, d = 0;
    if (i < len) {
        v = list[i];
        d = degree_of(off, vgraph, v);
        hub_shape(d, x);
    }
    block_exclusive_scan_k<6>(x, ex, tot, s_scan6);
    if (i >= len) return;
    int64_t at[6];
#pragma unroll
    for (int k = 0; k < 6; ++k) at[k] = bstart[(int64_t)blockIdx.x * 6 + k] + ex[k];
    const bool big = x[0] != 0;
    HubTask t;
    t.v = v;
    t.d = d;
    t.nseg = (int32_t)x[3];
    t.npart = (int32_t)x[4];
    t.seg0 = big ? (int32_t)at[3] : 0;
    t.part0 = big ? (int32_t)at[4] : 0;
    t.poff0 = big ? at[5] : 0;
    t.tab = big ? at[2] : 0;
    t.e0 = 0;  // set once the rows are packed (hub_task_starts)
    tasks[big ? at[0] : totals[0] + at[1]] = t;
}

__global__ void k_hub_task_list(const HubTask *tasks, int64_t len, int32_t *list)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < len;
         i += (int64_t)gridDim.x * blockDim.x)
        list[i] = tasks[i].v;
}

// Hub order, counting sort over the classes clz(degree) (degrees >= 1, so
// the longest rows have the smallest class).  Per block of HT rows, the count
// of each class: hist[c * nblk + blk].
__global__ void __launch_bounds__(HT) k_hub_class_count(const int32_t *list, int64_t len,
                                                         const int32_t *off,
                                                         const int32_t *vgraph, int32_t *hist)
{
    __shared__ int32_t s_cnt[HUB_CLASSES];
    if (threadIdx.x < HUB_CLASSES) s_cnt[threadIdx.x] = 0;
    __syncthreads();
    const int64_t i = (int64_t)blockIdx.x * HT + threadIdx.x;
    if (i < len) atomicAdd(&s_cnt[__clz(degree_of(off, vgraph, list[i]))], 1);
    __syncthreads();
    if (threadIdx.x < HUB_CLASSES)
        hist[(int64_t)threadIdx.x * gridDim.x + blockIdx.x] = s_cnt[threadIdx.x];
}

// Each row to class start + its block's offset within the class + its rank
// among the block's rows of the class (warp after warp, lane after lane), so
// the order within a class is the list order.
__global__ void __launch_bounds__(HT) k_hub_class_scatter(const int32_t *list, int64_t len,
                                                           const int32_t *off,
                                                           const int32_t *vgraph,
                                                           const int32_t *hist,
                                                           const int64_t *class_begin,
                                                           int32_t *out)
{
    __shared__ int32_t s_wc[HT / 32][HUB_CLASSES + 1];  // per warp and class: count, then position
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const int64_t i = (int64_t)blockIdx.x * HT + threadIdx.x;
    const bool have = i < len;
    const int32_t v = have ? list[i] : 0;
    const int c = have ? __clz(degree_of(off, vgraph, v)) : HUB_CLASSES;
    const unsigned peers = __match_any_sync(FULL, (unsigned)c);
    const int rank = __popc(peers & ((1u << lane) - 1u));
    s_wc[wib][lane] = 0;
    __syncwarp();
    if (have && rank == 0) s_wc[wib][c] = __popc(peers);
    __syncthreads();
    if (threadIdx.x < HUB_CLASSES) {
        int32_t run = (int32_t)class_begin[threadIdx.x] +
                      hist[(int64_t)threadIdx.x * gridDim.x + blockIdx.x];
        for (int w = 0; w < HT / 32; ++w) {
            const int32_t t = s_wc[w][threadIdx.x];
            s_wc[w][threadIdx.x] = run;
            run += t;
        }
    }
    __syncthreads();
    if (have) out[s_wc[wib][c] + rank] = v;
}

__global__ void k_hub_item_maps(const HubTask *tasks, int64_t nbig, int32_t *seg_task,
                                int32_t *part_task)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nbig;
         i += (int64_t)gridDim.x * blockDim.x) {
        const HubTask t = tasks[i];
        for (int s = 0; s < t.nseg; ++s) seg_task[t.seg0 + s] = (int32_t)i;
        for (int p = 0; p < t.npart; ++p) part_task[t.part0 + p] = (int32_t)i;
    }
}


__global__ void k_hub_task_starts(HubTask *tasks, int64_t n, const int64_t *rp)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        tasks[i].e0 = rp[i];
}

// ---------------------------------------------------------------------------
// packed rows: the rows of a list copied in list order
// ---------------------------------------------------------------------------
constexpr int PK_SCAN = 1024;            // list items per scan tile
static_assert(PK_SCAN == BK, "the packing scans' tiles are the tile grid's");
constexpr int PK_T = 256, PK_PER = 8;    // copy: threads per block, entries per thread
constexpr int PK_OUT = 32 * PK_PER;      // entries per warp chunk
constexpr int PK_WARPS = PK_T / 32;
static_assert(PK_OUT == PACK_CHUNK, "copy chunks are the modularity pass's chunks");

// summed degree of the list items of each block (a run of `per` tiles)
__global__ void __launch_bounds__(PK_SCAN) k_pack_sum(const int32_t *list, int64_t len,
                                                      const int32_t *off, const int32_t *vgraph,
                                                      int64_t per, int64_t *bsum)
{
    __shared__ int64_t s_warp[33];
    int64_t d = 0;
    const int64_t t_lo = (int64_t)blockIdx.x * per;
    for (int64_t t = t_lo; t < t_lo + per; ++t) {
        const int64_t i = t * PK_SCAN + threadIdx.x;
        if (i >= len) break;
        d += degree_of(off, vgraph, list[i]);
    }
    int64_t tot;
    block_exclusive_scan(d, s_warp, &tot);
    if (threadIdx.x == 0) bsum[blockIdx.x] = tot;
}

// rp[i] = block start + prefix of the degrees within the block (tile after
// tile); rp[len] = total; srcw[i] = the row's start in the original CSR | its
// wave class << 48.  Every listed row has at least one entry, so each copy
// block's first entry (a multiple of PK_OUT) lies in exactly one row: that row
// records itself as the block's first row (first_row[ncopy] = the last row).
__global__ void __launch_bounds__(PK_SCAN) k_pack_rp(const int32_t *list, int64_t len,
                                                     const int32_t *off, const int32_t *vgraph,
                                                     const int32_t *g_vbase, const int64_t *g_ebase,
                                                     uint32_t waves, uint64_t magic, int64_t per,
                                                     const int64_t *bstart, int64_t *rp,
                                                     int64_t *srcw, int64_t *first_row,
                                                     int64_t ncopy)
{
    __shared__ int64_t s_warp[33];
    int64_t run = bstart[blockIdx.x];
    const int64_t t_lo = (int64_t)blockIdx.x * per;
    for (int64_t t = t_lo; t < t_lo + per && t * PK_SCAN < len; ++t) {  // block-uniform
        const int64_t i = t * PK_SCAN + threadIdx.x;
        int64_t d = 0, src = 0;
        uint32_t wv = 0;
        if (i < len) {
            const int32_t v = list[i];
            const int32_t g = vgraph ? vgraph[v] : 0;
            const int32_t rs = off[(int64_t)v + g];
            d = off[(int64_t)v + g + 1] - rs;
            src = (g_ebase ? g_ebase[g] : 0) + rs;
            const int32_t lv = v - (vgraph ? g_vbase[g] : 0);
            wv = waves > 1 ? fastmod((uint32_t)lv, magic, waves) : 0u;
        }
        int64_t tot;
        const int64_t ex = block_exclusive_scan(d, s_warp, &tot);
        if (i < len) {
            const int64_t start = run + ex, end = start + d;
            rp[i] = start;
            srcw[i] = src | ((int64_t)wv << 48);
            for (int64_t c = (start + PK_OUT - 1) / PK_OUT; c * PK_OUT < end; ++c) first_row[c] = i;
            if (i == len - 1) {
                rp[len] = end;
                first_row[ncopy] = i;
            }
        }
        run += tot;
    }
}

// Entries [j_lo, j_lo + PK_OUT) of the packed arrays, one warp per chunk: rows
// r0 (holding j_lo) to r1 (holding the next chunk's first entry, or the last
// row), at most PK_OUT + 1 of them.  Their packed and original starts and
// wave classes are staged in the warp's shared memory with the row of every
// entry of the chunk; lane l copies entries l, l + 32, ..., so every load and
// store of the warp covers 32 consecutive entries.
// Order in which the copy visits its chunks: the chunks of bucket b's region
// [c0[b], c0[b + 1]) (its W wave segments one after another, of about q[b]
// chunks each) are taken in turn from every segment, so that the W warps
// copying rows of neighbouring vertices (the same source sectors) run at
// about the same time and the sectors are read from DRAM once.  nreg = 0:
// chunk order.
struct PackOrder {
    int32_t nreg;
    uint32_t waves;
    int64_t c0[NUM_BUCKETS + 1];
    int64_t q[NUM_BUCKETS];
    int64_t slot0[NUM_BUCKETS + 1];
};

__device__ __forceinline__ int64_t pack_chunk_of(const PackOrder &o, int64_t t)
{
    if (o.nreg == 0) return t;
    int b = 0;
    while (b + 1 < o.nreg && t >= o.slot0[b + 1]) ++b;
    if (t >= o.slot0[o.nreg]) return -1;
    const int64_t r = t - o.slot0[b];
    const int64_t c = o.c0[b] + (r % o.waves) * o.q[b] + r / o.waves;
    return c < o.c0[b + 1] ? c : -1;
}

// (row starts are kept relative to the chunk's first entry in 32 bits, so
// that seven blocks fit an SM: a row's start lies at most its length, under
// 2^31, before the chunk; the start after the chunk's last row, which only
// bounds it, is clamped)
__global__ void __launch_bounds__(PK_T, 7) k_pack_rows(const int64_t *rp, const int64_t *srcw,
                                                       const int64_t *first_row, int64_t ncopy,
                                                       const int32_t *idx, const int32_t *wts,
                                                       int64_t ne, uint32_t waves, uint64_t magic,
                                                       PackOrder order, int32_t *pidx,
                                                       int32_t *pwts)
{
    __shared__ int32_t s_rp_all[PK_WARPS][PK_OUT + 2];
    __shared__ int64_t s_src_all[PK_WARPS][PK_OUT + 1];
    __shared__ uint16_t s_row_all[PK_WARPS][PK_OUT];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const int64_t chunk = pack_chunk_of(order, (int64_t)blockIdx.x * PK_WARPS + wib);
    if (chunk < 0 || chunk >= ncopy) return;  // warp-uniform
    int32_t *s_rp = s_rp_all[wib];
    int64_t *s_src = s_src_all[wib];
    uint16_t *s_row = s_row_all[wib];
    const int64_t j_lo = chunk * PK_OUT;
    const int64_t j_hi = min(j_lo + (int64_t)PK_OUT, ne);
    const int64_t r0 = first_row[chunk];
    const int64_t r1 = first_row[chunk + 1];
    const int nr = (int)min(r1 - r0 + 1, (int64_t)PK_OUT + 1);
    for (int k = lane; k <= nr; k += 32)
        s_rp[k] = (int32_t)min(rp[r0 + k] - j_lo, (int64_t)INT32_MAX);
    for (int k = lane; k < nr; k += 32) s_src[k] = srcw[r0 + k];
    __syncwarp();
    chunk_rows([&](int k) { return s_rp[k]; }, nr, s_row);
    int32_t c[PK_PER], w[PK_PER];
#pragma unroll
    for (int q = 0; q < PK_PER; ++q) {  // every load in flight before any use
        const int e = lane + 32 * q;
        const int64_t j = j_lo + e;
        c[q] = w[q] = 0;
        if (j < j_hi) {
            const int k = s_row[e];
            const int64_t src = (s_src[k] & 0xFFFFFFFFFFFFll) + (e - s_rp[k]);
            c[q] = __ldg(idx + src);
            if (wts) w[q] = __ldg(wts + src);
        }
    }
#pragma unroll
    for (int q = 0; q < PK_PER; ++q) {
        const int e = lane + 32 * q;
        const int64_t j = j_lo + e;
        if (j >= j_hi) continue;
        int32_t u = c[q];
        if (waves > 1) {  // the row's wave class, read again from shared memory
            const uint32_t wv = (uint32_t)(s_src[s_row[e]] >> 48);
            if (fastmod((uint32_t)u, magic, waves) < wv) u = (int32_t)((uint32_t)u | 0x80000000u);
        }
        pidx[j] = u;
        if (wts) pwts[j] = w[q];
    }
}

// ---------------------------------------------------------------------------
// wave partition (asynchronous mode)
// ---------------------------------------------------------------------------
constexpr int WV = 1024;  // list entries per block tile
static_assert(WV == BK, "the wave partition's tiles are the tile grid's");

__device__ __forceinline__ int wave_class(const int32_t *list, int64_t i, const int64_t *bb,
                                          const int32_t *vgraph, const int32_t *g_vbase,
                                          uint32_t waves, uint64_t magic)
{
    int b = 0;
#pragma unroll
    for (int c = 1; c < NUM_BUCKETS; ++c)
        if (i >= bb[c]) b = c;
    const int32_t v = list[i];
    const int32_t lv = v - (vgraph ? g_vbase[vgraph[v]] : 0);
    return b * (int)waves + (int)fastmod((uint32_t)lv, magic, waves);
}

struct WaveParams {
    int64_t bb[NUM_BUCKETS];
    uint32_t waves;
    uint64_t magic;
};

// Per block (a run of `per` tiles of WV list items): the count of every
// class, one shared atomic per class present in a warp.
__global__ void __launch_bounds__(WV) k_wave_hist(const int32_t *list, int64_t len, WaveParams p,
                                                   int64_t per, const int32_t *vgraph,
                                                   const int32_t *g_vbase, int32_t *hist)
{
    extern __shared__ int32_t s_cnt[];  // NUM_BUCKETS * waves
    const int lane = threadIdx.x & 31;
    const int nc = NUM_BUCKETS * (int)p.waves;
    for (int c = threadIdx.x; c < nc; c += WV) s_cnt[c] = 0;
    __syncthreads();
    const int64_t t_lo = (int64_t)blockIdx.x * per;
    for (int64_t t = t_lo; t < t_lo + per && t * WV < len; ++t) {  // block-uniform
        const int64_t i = t * WV + threadIdx.x;
        const int c = i < len ? wave_class(list, i, p.bb, vgraph, g_vbase, p.waves, p.magic) : -1;
        const unsigned peers = __match_any_sync(FULL, (unsigned)c);
        if (c >= 0 && lane == __ffs(peers) - 1) atomicAdd(&s_cnt[c], __popc(peers));
    }
    __syncthreads();
    for (int c = threadIdx.x; c < nc; c += WV) hist[(int64_t)c * gridDim.x + blockIdx.x] = s_cnt[c];
}

// Every item of the block's tiles to its class: class start + the block's
// offset within the class + a position taken by its warp's leader for the
// warp's items of the class (in lane order within the warp).
__global__ void __launch_bounds__(WV) k_wave_scatter(const int32_t *list, int64_t len,
                                                      WaveParams p, int64_t per,
                                                      const int32_t *vgraph,
                                                      const int32_t *g_vbase, const int32_t *hist,
                                                      const int64_t *class_begin, int32_t *out)
{
    extern __shared__ int32_t s_cur[];
    const int lane = threadIdx.x & 31;
    const int nc = NUM_BUCKETS * (int)p.waves;
    for (int c = threadIdx.x; c < nc; c += WV)
        s_cur[c] = (int32_t)class_begin[c] + hist[(int64_t)c * gridDim.x + blockIdx.x];
    __syncthreads();
    const int64_t t_lo = (int64_t)blockIdx.x * per;
    for (int64_t t = t_lo; t < t_lo + per && t * WV < len; ++t) {  // block-uniform
        const int64_t i = t * WV + threadIdx.x;
        const int c = i < len ? wave_class(list, i, p.bb, vgraph, g_vbase, p.waves, p.magic) : -1;
        const unsigned peers = __match_any_sync(FULL, (unsigned)c);
        const int leader = __ffs(peers) - 1;
        int base = 0;
        if (c >= 0 && lane == leader) base = atomicAdd(&s_cur[c], __popc(peers));
        base = __shfl_sync(FULL, base, leader);
        if (c >= 0) out[base + __popc(peers & ((1u << lane) - 1u))] = list[i];
    }
}

int grid_for(int64_t items, int threads, int cap)
{
    const int64_t b = (items + threads - 1) / threads;
    return (int)(b < 1 ? 1 : (b > cap ? cap : b));
}

}  // namespace

int ingest_validate(const int32_t *off, const int32_t *idx, const int32_t *wts, int32_t n,
                    int64_t m, IngestOut *d_out, cudaStream_t st, int64_t *launches)
{
    if (cudaMemsetAsync(d_out, 0, sizeof(IngestOut), st) != cudaSuccess) return -1;
    k_val_offsets<<<grid_for((int64_t)n + 1, 256, 4096), 256, 0, st>>>(off, n, m, d_out);
    ++*launches;
    if (m > 0) {
        k_val_entries<<<grid_for(m, 256, 8192), 256, 0, st>>>(idx, wts, n, m, d_out);
        ++*launches;
    }
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

int ingest_validate_ordered(const int32_t *off, const int32_t *idx, const int32_t *wts, int32_t n,
                            int64_t m, uint32_t *bits, IngestOut *d_out, cudaStream_t st,
                            int64_t *launches)
{
    if (cudaMemsetAsync(d_out, 0, sizeof(IngestOut), st) != cudaSuccess) return -1;
    k_val_offsets<<<grid_for((int64_t)n + 1, 256, 4096), 256, 0, st>>>(off, n, m, d_out);
    ++*launches;
    if (m > 0) {
        if (cudaMemsetAsync(bits, 0, (size_t)(m / 32 + 1) * sizeof(uint32_t), st) != cudaSuccess)
            return -1;
        k_mark_row_starts<<<grid_for(n, 256, 8192), 256, 0, st>>>(off, n, nullptr, nullptr, m,
                                                                   bits);
        k_val_entries4<<<grid_for((m + 3) / 4, 256, 8192), 256, 0, st>>>(idx, wts, n, m, bits,
                                                                          d_out);
        *launches += 2;
    }
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

int ingest_row_order(const int32_t *off, const int32_t *idx, int32_t nv, int64_t ne,
                     const int32_t *vgraph, const int64_t *g_ebase, uint32_t *bits,
                     IngestOut *d_out, cudaStream_t st, int64_t *launches)
{
    if (cudaMemsetAsync(&d_out->repeated, 0, sizeof(int32_t), st) != cudaSuccess) return -1;
    if (ne < 2 || nv == 0) return 0;
    if (cudaMemsetAsync(bits, 0, (size_t)(ne / 32 + 1) * sizeof(uint32_t), st) != cudaSuccess)
        return -1;
    k_mark_row_starts<<<grid_for(nv, 256, 8192), 256, 0, st>>>(off, nv, vgraph, g_ebase, ne,
                                                                bits);
    k_check_row_order<<<grid_for(ne, 256, 8192), 256, 0, st>>>(idx, ne, bits, d_out);
    *launches += 2;
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

int ingest_check_wdeg(const int32_t *off, const int32_t *wts, int32_t n, IngestOut *d_out,
                      cudaStream_t st, int64_t *launches)
{
    k_val_wdeg<<<grid_for(n, 256, 4096), 256, 0, st>>>(off, wts, n, d_out);
    ++*launches;
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

// per block and bucket: a row count (int32), then, 8-byte aligned, an entry
// count (int64)
static int64_t bucket_count_words(int64_t nblk) { return (nblk * NUM_BUCKETS + 1) & ~(int64_t)1; }

size_t ingest_bucket_scratch_bytes(int32_t nv_total)
{
    int64_t nblk = tile_grid(nv_total).nblk;
    if (nblk < 1) nblk = 1;
    return (size_t)bucket_count_words(nblk) * sizeof(int32_t) +
           (size_t)nblk * NUM_BUCKETS * sizeof(int64_t);
}

int ingest_bucket(const int32_t *off, int32_t nv, const int32_t *vgraph, const int32_t *,
                  const Thresholds &th, int32_t *list, int32_t *blk, int64_t *d_counts,
                  cudaStream_t st, int64_t *launches)
{
    const TileGrid tg = tile_grid(nv);
    const int64_t nblk = tg.nblk;
    if (cudaMemsetAsync(d_counts, 0, 3 * NUM_BUCKETS * sizeof(int64_t), st) != cudaSuccess)
        return -1;
    if (nblk == 0) return 0;
    int64_t *bent = reinterpret_cast<int64_t *>(blk + bucket_count_words(nblk));
    k_bucket_count<<<(int)nblk, BK, 0, st>>>(off, nv, vgraph, th, tg.per, blk, bent);
    k_bucket_entries<<<NUM_BUCKETS, 1024, 0, st>>>(bent, nblk, d_counts + 2 * NUM_BUCKETS);
    k_class_scan<<<NUM_BUCKETS, 1024, 0, st>>>(blk, nblk, d_counts);
    k_class_begin<<<1, 1024, 0, st>>>(d_counts, NUM_BUCKETS, d_counts + NUM_BUCKETS);
    k_bucket_scatter<<<(int)nblk, BK, 0, st>>>(off, nv, vgraph, th, tg.per, blk, d_counts, list);
    *launches += 5;
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

// class starts (int64, first) and per-block class counts
int64_t wave_hist_ints(int64_t list_len, int waves)
{
    const int64_t nblk = tile_grid(list_len).nblk;
    return ((nblk > 0 ? nblk : 1) + 2) * NUM_BUCKETS * (int64_t)waves;
}

int wave_partition(const int32_t *list, int64_t len, const int64_t *bucket_begin,
                   const int32_t *vgraph, const int32_t *g_vbase, int waves, int32_t *hist,
                   int64_t *d_totals, int32_t *out, cudaStream_t st, int64_t *launches)
{
    const int nc = NUM_BUCKETS * waves;
    if (waves < 1 || waves > WAVE_MAX) return -1;
    if (len == 0) return cudaMemsetAsync(d_totals, 0, (size_t)nc * sizeof(int64_t), st) ==
                          cudaSuccess ? 0 : -1;
    WaveParams p;
    for (int c = 0; c < NUM_BUCKETS; ++c) p.bb[c] = bucket_begin[c];
    p.waves = (uint32_t)waves;
    p.magic = fastmod_magic((uint32_t)waves);
    const TileGrid tg = tile_grid(len);
    const int64_t nblk = tg.nblk;
    const size_t smem = (size_t)nc * sizeof(int32_t);
    int64_t *class_begin = reinterpret_cast<int64_t *>(hist);
    int32_t *counts = hist + 2 * (int64_t)nc;
    k_wave_hist<<<(int)nblk, WV, smem, st>>>(list, len, p, tg.per, vgraph, g_vbase, counts);
    k_class_scan<<<nc, 1024, 0, st>>>(counts, nblk, d_totals);
    k_class_begin<<<1, 1024, 0, st>>>(d_totals, nc, class_begin);
    k_wave_scatter<<<(int)nblk, WV, smem, st>>>(list, len, p, tg.per, vgraph, g_vbase, counts,
                                                class_begin, out);
    *launches += 4;
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

int wave_prepare()
{
    const int bytes = NUM_BUCKETS * WAVE_MAX * (int)sizeof(int32_t);
    if (cudaFuncSetAttribute(k_wave_hist, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes) !=
            cudaSuccess ||
        cudaFuncSetAttribute(k_wave_scatter, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes) !=
            cudaSuccess)
        return -1;
    return 0;
}

int64_t hub_scratch_ints(int64_t len)
{
    const int64_t nblk = len > 0 ? (len + HT - 1) / HT : 1;
    // the order's class counts (int32, HUB_CLASSES per block), class sizes and
    // starts; the tasks' block sums (6 per block) fit in the same words
    return HUB_CLASSES / 2 * nblk + 2 * HUB_CLASSES;
}

int hub_tasks(int32_t *list, int64_t len, const int32_t *off, const int32_t *vgraph,
              HubTask *tasks, int64_t *totals, int64_t *scratch, cudaStream_t st,
              int64_t *launches)
{
    if (len <= 0)
        return cudaMemsetAsync(totals, 0, 5 * sizeof(int64_t), st) == cudaSuccess ? 0 : -1;
    const int64_t nblk = (len + HT - 1) / HT;
    k_hub_task_sums<<<(int)nblk, HT, 0, st>>>(list, len, off, vgraph, scratch);
    k_hub_task_scan<<<1, 1024, 0, st>>>(scratch, nblk, totals);
    k_hub_task_write<<<(int)nblk, HT, 0, st>>>(list, len, off, vgraph, scratch, totals, tasks);
    k_hub_task_list<<<grid_for(len, 256, 1024), 256, 0, st>>>(tasks, len, list);
    *launches += 4;
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

int hub_order(const int32_t *list, int64_t len, const int32_t *off, const int32_t *vgraph,
              int32_t *out, int64_t *scratch, cudaStream_t st, int64_t *launches)
{
    if (len <= 0) return 0;
    const int64_t nblk = (len + HT - 1) / HT;
    int64_t *class_size = scratch, *class_begin = scratch + HUB_CLASSES;
    int32_t *hist = reinterpret_cast<int32_t *>(scratch + 2 * HUB_CLASSES);
    k_hub_class_count<<<(int)nblk, HT, 0, st>>>(list, len, off, vgraph, hist);
    k_class_scan<<<HUB_CLASSES, 1024, 0, st>>>(hist, nblk, class_size);
    k_class_begin<<<1, 1024, 0, st>>>(class_size, HUB_CLASSES, class_begin);
    k_hub_class_scatter<<<(int)nblk, HT, 0, st>>>(list, len, off, vgraph, hist, class_begin,
                                                    out);
    *launches += 4;
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

int hub_task_starts(HubTask *tasks, int64_t n, const int64_t *rp, cudaStream_t st,
                    int64_t *launches)
{
    if (n <= 0) return 0;
    k_hub_task_starts<<<grid_for(n, 256, 1024), 256, 0, st>>>(tasks, n, rp);
    ++*launches;
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

int64_t pack_scratch_ints(int64_t len)
{
    const int64_t nblk = tile_grid(len, PACK_TILE_BLOCKS).nblk;
    return 2 * (nblk > 0 ? nblk : 1) + len;
}

int pack_rows(const int32_t *list, int64_t len, const int32_t *off, const int32_t *idx,
              const int32_t *wts, int64_t ne, const int32_t *vgraph, const int32_t *g_vbase,
              const int64_t *g_ebase, int waves, const int64_t *bucket_entries,
              int64_t *scratch, int64_t *rp, int64_t *first_row, int32_t *pidx, int32_t *pwts,
              cudaStream_t st, int64_t *launches)
{
    if (waves < 1) return -1;
    if (len == 0) return cudaMemsetAsync(rp, 0, sizeof(int64_t), st) == cudaSuccess ? 0 : -1;
    const TileGrid tg = tile_grid(len, PACK_TILE_BLOCKS);
    const int64_t nblk = tg.nblk;
    const int64_t ncopy = (ne + PK_OUT - 1) / PK_OUT;
    int64_t *bsum = scratch, *bstart = scratch + nblk, *srcw = scratch + 2 * nblk;
    const uint64_t magic = fastmod_magic((uint32_t)waves);
    k_pack_sum<<<(int)nblk, PK_SCAN, 0, st>>>(list, len, off, vgraph, tg.per, bsum);
    k_class_begin<<<1, 1024, 0, st>>>(bsum, nblk, bstart);
    k_pack_rp<<<(int)nblk, PK_SCAN, 0, st>>>(list, len, off, vgraph, g_vbase, g_ebase,
                                              (uint32_t)waves, magic, tg.per, bstart, rp, srcw,
                                              first_row, ncopy);
    *launches += 3;
    if (ne > 0) {
        PackOrder order{};
        int64_t slots = ncopy;
        if (waves > 1 && bucket_entries) {
            order.nreg = NUM_BUCKETS;
            order.waves = (uint32_t)waves;
            int64_t e = 0;
            order.slot0[0] = 0;
            for (int b = 0; b < NUM_BUCKETS; ++b) {
                order.c0[b] = e / PK_OUT;
                e += bucket_entries[b];
            }
            order.c0[NUM_BUCKETS] = ncopy;
            for (int b = 0; b < NUM_BUCKETS; ++b) {
                const int64_t nc = order.c0[b + 1] - order.c0[b];
                order.q[b] = (nc + waves - 1) / waves;
                order.slot0[b + 1] = order.slot0[b] + order.q[b] * waves;
            }
            slots = order.slot0[NUM_BUCKETS];
        }
        k_pack_rows<<<(int)((slots + PK_WARPS - 1) / PK_WARPS), PK_T, 0, st>>>(
            rp, srcw, first_row, ncopy, idx, wts, ne, (uint32_t)waves, magic, order, pidx,
            wts ? pwts : nullptr);
        ++*launches;
    }
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

int hub_item_maps(const HubTask *tasks, int64_t nbig, int32_t *seg_task, int32_t *part_task,
                  cudaStream_t st, int64_t *launches)
{
    if (nbig <= 0) return 0;
    k_hub_item_maps<<<grid_for(nbig, 128, 1024), 128, 0, st>>>(tasks, nbig, seg_task, part_task);
    ++*launches;
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

int merge_final_labels(int32_t *lab0, const int32_t *lab1, int32_t nv, const int32_t *vgraph,
                       const int32_t *g_sel, cudaStream_t st, int64_t *launches)
{
    if (nv == 0) return 0;
    k_merge_final<<<grid_for(nv, 256, 8192), 256, 0, st>>>(lab0, lab1, nv, vgraph, g_sel);
    ++*launches;
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

int fill_iota(int32_t *lab, int32_t nv, const int32_t *vgraph, const int32_t *g_vbase,
              cudaStream_t st, int64_t *launches)
{
    if (nv == 0) return 0;
    k_iota<<<grid_for(nv, 256, 8192), 256, 0, st>>>(lab, nv, vgraph, g_vbase);
    ++*launches;
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

int check_labels(const int32_t *lab, int32_t nv, const int32_t *vgraph, const int32_t *,
                 const int32_t *g_n, IngestOut *d_out, cudaStream_t st, int64_t *launches)
{
    if (cudaMemsetAsync(d_out, 0, sizeof(IngestOut), st) != cudaSuccess) return -1;
    if (nv == 0) return 0;
    k_check_labels<<<grid_for(nv, 256, 8192), 256, 0, st>>>(lab, nv, vgraph, g_n, d_out);
    ++*launches;
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

}  // namespace lp
