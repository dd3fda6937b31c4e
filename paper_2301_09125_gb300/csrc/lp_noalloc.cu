// lp_rak_sweep_noalloc: one synchronous RAK sweep that allocates no memory.
//
// Some callers cannot allocate device memory at run time: their GPU memory is
// already fully reserved by another allocator (a framework's caching
// allocator, or a pool sized once at start-up under a fixed budget), so a
// cudaMalloc from a library would fail or would break the budget.  This entry
// point serves them.  The caller passes every input and output buffer; the
// only scratch memory the sweep needs lives in `g_noalloc_scratch`, a
// file-scope __device__ array that every GPU loading this library holds until
// the process exits:
//   - a control block: the changed counter, the validation status, n;
//   - one overflow hash table per CTA (label, summed weight, ~first position)
//     for labels that do not fit the CTA's shared-memory table.
// Its size bounds the graphs it accepts: at most NA_MAX_DEGREE entries per row.
//
// The sweep needs no degree buckets (which would need memory per graph).
// It makes two passes over the vertices, two launches.  First, as many warps
// as fit the GPU take the rows of at most 32 entries, one lane per entry: a
// lane's label total is the sum over the lanes holding the same label
// (__match_any_sync), and the lowest of those lanes is the label's first
// position.  Then NA_CTAS CTAs take the longer rows, each looking at
// NA_THREADS vertices at a time and listing the long ones in shared memory:
// a shared table of 2^ceil(log2(2d)) slots (at most NA_TABLE), probed at most
// NA_PROBE slots from a label's hash; a label whose window is full goes to
// the CTA's overflow table in the static array.
#include <mutex>
#include <string>

#include "lp.h"
#include "lp_device.cuh"
#include "lp_internal.cuh"

namespace lp {
lp_status lp_fail(lp_status s, const std::string &msg);  // lp_api.cu: sets lp_last_error
void lp_add_launches(int64_t n);                         // lp_api.cu: lp_launch_count

namespace {

constexpr int NA_CTAS = 128;          // CTAs of one sweep (one overflow table each)
constexpr int NA_THREADS = 512;
constexpr int NA_TABLE = 8192;        // shared slots per CTA (96 KB)
constexpr int NA_TABLE_LG = 13;
constexpr int NA_PROBE = 32;          // shared probe window before the overflow table
constexpr int NA_MAX_DEGREE = 4096;   // 2 * degree distinct labels fit NA_SLOTS
constexpr int NA_SLOTS = 8192;        // overflow slots per CTA
constexpr int NA_CTRL = 64;           // control words ahead of the tables
constexpr size_t NA_WORDS = NA_CTRL + 3 * (size_t)NA_CTAS * NA_SLOTS;  // 12.6 MB
static_assert(sizeof(IngestOut) <= 16 * sizeof(int32_t), "control block layout");

// Control block (int32 words): [0] changed counter, [16, 32) validation
// status (IngestOut), [32] n.  Then keys, sums, ~positions of the overflow
// tables, NA_CTAS * NA_SLOTS words each.  Every use of an overflow slot
// resets it, so the tables stay clean between calls; the set-up clears them
// once per device.
static __device__ __align__(256) int32_t g_noalloc_scratch[NA_WORDS];

struct NoAllocArgs {
    const int32_t *off, *idx, *wts, *lab_in;
    int32_t *lab_out;
    int32_t n;
    int strict;
    uint64_t key_t;
    int32_t *changed;
    int32_t *ov_key, *ov_sum;
    uint32_t *ov_npos;
};

constexpr int NA_WARP_MAX = 32;  // rows of at most this many entries: one warp each

// Rows of 0 .. 32 entries: one warp each, no table (as many warps as fit
// the GPU: the pass needs no scratch).
__global__ void __launch_bounds__(NA_THREADS) k_noalloc_warp(NoAllocArgs a)
{
    const int lane = threadIdx.x & 31;
    uint32_t my_changed = 0;

    const int64_t wid = ((int64_t)blockIdx.x * NA_THREADS + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * NA_THREADS) >> 5;
    for (int64_t v = wid; v < a.n; v += nw) {
        const int32_t rs = __ldg(a.off + v), d = __ldg(a.off + v + 1) - rs;
        if (d > NA_WARP_MAX) continue;  // warp-uniform
        const int32_t own = __ldg(a.lab_in + v);
        if (d == 0) {  // no neighbours: the label stays (Sec. 3.2 reading c8)
            if (lane == 0) a.lab_out[v] = own;
            continue;
        }
        const bool act = lane < d;
        int32_t l = EMPTY;
        uint32_t w = 0u;
        if (act) {
            const int32_t u = __ldg(a.idx + rs + lane);
            w = a.wts ? (uint32_t)__ldg(a.wts + rs + lane) : 1u;
            l = __ldg(a.lab_in + u);
        }
        const unsigned grp = __match_any_sync(FULL, act ? l : EMPTY);
        const uint32_t sum = __reduce_add_sync(grp, w);  // a row's sum < 2^31
        const bool lead = act && lane == __ffs(grp) - 1;  // the label's first position
        Cand c{0u, 0u, 0ull, EMPTY};
        if (lead) c = Cand{sum, 0xFFFFFFFFu - (uint32_t)lane, 0ull, l};
        if (!a.strict) {
            const uint32_t mx = __reduce_max_sync(FULL, c.sum);
            if (lead && c.sum == mx)
                c.h = stream_at(stream_at(a.key_t, (uint64_t)v + 1), (uint64_t)l + 1);
            else
                c = Cand{0u, 0u, 0ull, EMPTY};
        }
        c = warp_best(c);
        if (lane == 0) {
            a.lab_out[v] = c.label;
            if (c.label != own) ++my_changed;
        }
    }
    my_changed = __reduce_add_sync(FULL, my_changed);
    if (lane == 0 && my_changed) atomicAdd(a.changed, (int)my_changed);
}

// Longer rows: one CTA each, a table of 2^ceil(log2(2d)) slots and the CTA's
// overflow table in the static array (NA_CTAS CTAs).  The CTA looks at
// NA_THREADS vertices at a time, one per thread, and lists the long ones in
// shared memory before taking them one after another.
__global__ void __launch_bounds__(NA_THREADS) k_noalloc_cta(NoAllocArgs a)
{
    extern __shared__ int32_t smem[];
    int32_t *tk = smem;
    int32_t *ts = tk + NA_TABLE;
    uint32_t *tp = reinterpret_cast<uint32_t *>(ts + NA_TABLE);
    __shared__ Cand s_red[NA_THREADS / 32];
    __shared__ uint32_t s_u[NA_THREADS / 32 + 1];
    __shared__ int s_spilled;
    __shared__ int32_t s_long[NA_THREADS];
    __shared__ int s_nlong;
    const int lane = threadIdx.x & 31;
    uint32_t my_changed = 0;
    for (int j = threadIdx.x; j < NA_TABLE; j += NA_THREADS) {
        tk[j] = EMPTY;
        ts[j] = 0;
        tp[j] = 0;
    }
    if (threadIdx.x == 0) s_spilled = 0;
    __syncthreads();
    int32_t *gk = a.ov_key + (int64_t)blockIdx.x * NA_SLOTS;
    int32_t *gs = a.ov_sum + (int64_t)blockIdx.x * NA_SLOTS;
    uint32_t *gp = a.ov_npos + (int64_t)blockIdx.x * NA_SLOTS;
    for (int64_t base = (int64_t)blockIdx.x * NA_THREADS; base < a.n;
         base += (int64_t)gridDim.x * NA_THREADS) {
        if (threadIdx.x == 0) s_nlong = 0;
        __syncthreads();
        {
            const int64_t u = base + threadIdx.x;
            if (u < a.n && __ldg(a.off + u + 1) - __ldg(a.off + u) > NA_WARP_MAX)
                s_long[atomicAdd(&s_nlong, 1)] = (int32_t)u;
        }
        __syncthreads();
        const int nlong = s_nlong;
        for (int q = 0; q < nlong; ++q) {
            const int32_t v = s_long[q];
            const int32_t rs = __ldg(a.off + v), d = __ldg(a.off + v + 1) - rs;
            const int32_t own = __ldg(a.lab_in + v);
            const int glg = ilog2_ceil(2u * (uint32_t)d);  // 2^glg <= NA_SLOTS (degree checked)
            const int lg = glg < NA_TABLE_LG ? glg : NA_TABLE_LG;
            const int probe = NA_PROBE < (1 << lg) ? NA_PROBE : (1 << lg);
            for (int k0 = 0; k0 < d; k0 += NA_THREADS) {
                const int k = k0 + threadIdx.x;
                const bool act = k < d;
                int w = 0;
                int32_t l = EMPTY;
                if (act) {
                    const int32_t u = __ldg(a.idx + rs + k);
                    w = a.wts ? __ldg(a.wts + rs + k) : 1;
                    l = __ldg(a.lab_in + u);
                }
                if (act && !table_add(tk, ts, tp, lg, probe, l, w, k)) {
                    s_spilled = 1;
                    table_add(gk, gs, gp, glg, 1 << glg, l, w, k);
                }
            }
            __syncthreads();
            const int slots = 1 << lg;
            const int gslots = s_spilled ? (1 << glg) : 0;
            Cand best{0u, 0u, 0ull, EMPTY};
            uint32_t mx = 0;
            if (!a.strict) {
                for (int j = threadIdx.x; j < slots + gslots; j += NA_THREADS) {
                    const int32_t key = j < slots ? tk[j] : gk[j - slots];
                    if (key != EMPTY) mx = max(mx, (uint32_t)(j < slots ? ts[j] : gs[j - slots]));
                }
                mx = block_max<NA_THREADS>(mx, s_u);
            }
            const uint64_t ktv = stream_at(a.key_t, (uint64_t)v + 1);
            for (int j = threadIdx.x; j < slots + gslots; j += NA_THREADS) {
                int32_t *K = j < slots ? tk + j : gk + (j - slots);
                int32_t *S = j < slots ? ts + j : gs + (j - slots);
                uint32_t *Q = j < slots ? tp + j : gp + (j - slots);
                const int32_t key = *K;
                if (key != EMPTY) {
                    if (a.strict) {
                        const Cand c{(uint32_t)*S, *Q, 0ull, key};
                        if (better(c, best)) best = c;
                    } else if ((uint32_t)*S == mx) {
                        const Cand c{mx, *Q, stream_at(ktv, (uint64_t)key + 1), key};
                        if (better(c, best)) best = c;
                    }
                    *K = EMPTY;  // every used slot is reset: the tables stay clean
                    *S = 0;
                    *Q = 0;
                }
            }
            best = block_best<NA_THREADS>(best, s_red);
            if (threadIdx.x == 0) {
                a.lab_out[v] = best.label;
                if (best.label != own) ++my_changed;
                s_spilled = 0;
            }
            __syncthreads();
        }
        __syncthreads();  // every thread has read s_nlong before the next chunk resets it
    }
    my_changed = __reduce_add_sync(FULL, my_changed);
    if (lane == 0 && my_changed) atomicAdd(a.changed, (int)my_changed);
}

// Device address of the static array, looked up once per device.
std::mutex g_setup_mu;
int32_t *g_scratch_ptr[64] = {};

}  // namespace
}  // namespace lp

extern "C" lp_status lp_rak_sweep_noalloc(int32_t n, int64_t m, const int32_t *offsets,
                                          const int32_t *indices, const int32_t *weights,
                                          const int32_t *labels_in, int32_t *labels_out,
                                          int32_t strict, uint64_t seed, int32_t iteration,
                                          int64_t *changed, void *cuda_stream)
{
    using namespace lp;
    if (n < 0 || m < 0 || m > 2147483647LL) return lp_fail(LP_EINVAL, "n or m out of range");
    if (!offsets || (m > 0 && !indices) || !labels_in || !labels_out || !changed)
        return lp_fail(LP_EINVAL, "NULL argument");
    if (labels_in == labels_out) return lp_fail(LP_EINVAL, "labels_in and labels_out must differ");
    cudaStream_t st = (cudaStream_t)cuda_stream;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64)
        return lp_fail(LP_ECUDA, "no usable CUDA device");

    // set-up, once per device, with the device current: the device address of
    // the static scratch array (its host-side name is not a device address),
    // the kernel's shared-memory limit, and clean overflow tables
    int32_t *scratch = nullptr;
    {
        std::lock_guard<std::mutex> lock(g_setup_mu);
        if (!g_scratch_ptr[dev]) {
            void *p = nullptr;
            cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
            if (e != cudaSuccess)
                return lp_fail(LP_ECUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
            e = cudaFuncSetAttribute(k_noalloc_cta, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     NA_TABLE * 12);
            const size_t tab = (size_t)NA_CTAS * NA_SLOTS * sizeof(int32_t);
            int32_t *base = static_cast<int32_t *>(p);
            if (e == cudaSuccess) e = cudaMemsetAsync(base, 0, NA_CTRL * sizeof(int32_t), st);
            if (e == cudaSuccess) e = cudaMemsetAsync(base + NA_CTRL, 0xFF, tab, st);
            if (e == cudaSuccess) e = cudaMemsetAsync((char *)(base + NA_CTRL) + tab, 0, 2 * tab, st);
            if (e == cudaSuccess) e = cudaStreamSynchronize(st);
            if (e != cudaSuccess)
                return lp_fail(LP_ECUDA, std::string("no-alloc set-up: ") + cudaGetErrorString(e));
            g_scratch_ptr[dev] = base;
        }
        scratch = g_scratch_ptr[dev];
    }
    IngestOut *d_status = reinterpret_cast<IngestOut *>(scratch + 16);
    int32_t *d_n = scratch + 32;
    int64_t launches = 0;
    IngestOut h{};
    auto read_status = [&](const char *what) -> lp_status {
        cudaError_t e = cudaMemcpyAsync(&h, d_status, sizeof h, cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) return lp_fail(LP_ECUDA, std::string(what) + ": " + cudaGetErrorString(e));
        return LP_OK;
    };

    // the same validation as lp_graph_create, with its status word in the array
    if (ingest_validate(offsets, indices, weights, n, m, d_status, st, &launches) != 0)
        return lp_fail(LP_ECUDA, "validation launch failed");
    lp_status s = read_status("validation");
    if (s != LP_OK) return s;
    if (h.err != ING_OK) return lp_fail(LP_EINVAL, "invalid CSR (same checks as lp_graph_create)");
    if (h.max_deg > NA_MAX_DEGREE)
        return lp_fail(LP_EINVAL, "lp_rak_sweep_noalloc accepts rows of at most 4096 entries");
    if ((int64_t)h.max_deg * h.max_w >= 2147483648LL) {
        if (ingest_check_wdeg(offsets, weights, n, d_status, st, &launches) != 0)
            return lp_fail(LP_ECUDA, "validation launch failed");
        if ((s = read_status("validation")) != LP_OK) return s;
        if (h.err != ING_OK) return lp_fail(LP_EINVAL, "a vertex's summed weight reaches 2^31");
    }
    if (cudaMemcpyAsync(d_n, &n, sizeof n, cudaMemcpyHostToDevice, st) != cudaSuccess ||
        check_labels(labels_in, n, nullptr, nullptr, d_n, d_status, st, &launches) != 0)
        return lp_fail(LP_ECUDA, "label check failed");
    if ((s = read_status("label check")) != LP_OK) return s;
    if (h.err != ING_OK) return lp_fail(LP_EINVAL, "labels_in holds a label outside [0, n)");

    // every call shares the array: the counter must start at zero
    if (cudaMemsetAsync(scratch, 0, sizeof(int32_t), st) != cudaSuccess)
        return lp_fail(LP_ECUDA, "clearing the changed counter failed");
    NoAllocArgs a{};
    a.off = offsets;
    a.idx = indices;
    a.wts = weights;
    a.lab_in = labels_in;
    a.lab_out = labels_out;
    a.n = n;
    a.strict = strict ? 1 : 0;
    a.key_t = stream_at(seed, (uint64_t)(int64_t)iteration + 1);
    a.changed = scratch;
    a.ov_key = scratch + NA_CTRL;
    a.ov_sum = a.ov_key + (size_t)NA_CTAS * NA_SLOTS;
    a.ov_npos = reinterpret_cast<uint32_t *>(a.ov_sum + (size_t)NA_CTAS * NA_SLOTS);
    if (n > 0) {
        int sms = 0;
        if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
            return lp_fail(LP_ECUDA, "no usable CUDA device");
        int64_t wblocks = ((int64_t)n + NA_THREADS / 32 - 1) / (NA_THREADS / 32);  // a warp per vertex
        if (wblocks > (int64_t)sms * 4) wblocks = (int64_t)sms * 4;
        k_noalloc_warp<<<(int)wblocks, NA_THREADS, 0, st>>>(a);
        const int64_t cblocks = ((int64_t)n + NA_THREADS - 1) / NA_THREADS;
        k_noalloc_cta<<<(int)(cblocks < NA_CTAS ? cblocks : NA_CTAS), NA_THREADS, NA_TABLE * 12,
                        st>>>(a);
        launches += 2;
        if (cudaGetLastError() != cudaSuccess) return lp_fail(LP_ECUDA, "sweep launch failed");
    }
    int32_t hc = 0;
    cudaError_t e = cudaMemcpyAsync(&hc, scratch, sizeof hc, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    lp_add_launches(launches);
    if (e != cudaSuccess) return lp_fail(LP_ECUDA, std::string("sweep: ") + cudaGetErrorString(e));
    *changed = hc;
    return LP_OK;
}
