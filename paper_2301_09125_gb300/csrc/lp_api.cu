// C ABI of the library (declared in include/lp.h).
//
// A graph (lp_graph) and a batch (lp_batch) share one device representation,
// GraphSet: an arena of G >= 1 graphs with concatenated CSR arrays, two label
// buffers, degree-bucketed vertex lists and per-iteration changed counters.
// lp_rak_run / lp_batch_run drive the iteration of Sec. 3.2: per iteration one
// launch per non-empty degree bucket, then a read of the changed counters and
// the tolerance test (changed <= tolerance * n, in double) on the host.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <memory>
#include <mutex>
#include <unordered_map>
#include <string>
#include <vector>

#include "lp.h"
#include "lp_internal.cuh"

namespace {

thread_local std::string g_err;
std::atomic<int64_t> g_launches{0};

// Per-kernel sweep statistics (lp_profile_*): while enabled, every sweep
// launch is bracketed by CUDA events on the graph's stream.
const char *const KERNEL_NAMES[lp::NUM_BUCKETS] = {"sweep_small", "sweep_warp", "sweep_cta",
                                                   "sweep_cta2", "sweep_hub"};
struct KernelStat {
    int64_t launches = 0;
    double ms = 0, vertices = 0, entries = 0, bytes = 0;
};
std::mutex g_prof_mu;
std::atomic<bool> g_prof_on{false};
KernelStat g_prof[lp::NUM_BUCKETS];

lp_status fail(lp_status s, const std::string &msg)
{
    g_err = msg;
    return s;
}

std::string cuda_msg(const char *what, cudaError_t e)
{
    return std::string(what) + ": " + cudaGetErrorName(e) + " (" + cudaGetErrorString(e) + ")";
}

#define LP_CU(call)                                                  \
    do {                                                             \
        cudaError_t e_ = (call);                                     \
        if (e_ != cudaSuccess) return fail(LP_ECUDA, cuda_msg(#call, e_)); \
    } while (0)

#define LP_TRY(call)                          \
    do {                                      \
        lp_status s_ = (call);                \
        if (s_ != LP_OK) return s_;           \
    } while (0)

// Adds the kernels launched in a scope to the process-wide counter.
struct Launches {
    int64_t n = 0;
    ~Launches() { g_launches += n; }
};

// Switches to a device for the duration of a call.
struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int dev)
    {
        if (cudaGetDevice(&prev) == cudaSuccess && prev != dev) cudaSetDevice(dev);
    }
    ~DeviceGuard()
    {
        int now = -1;
        if (prev >= 0 && cudaGetDevice(&now) == cudaSuccess && now != prev) cudaSetDevice(prev);
    }
};

// Device memory comes from one stream-ordered pool per device that keeps
// freed blocks for reuse (release threshold = all), so creating and
// destroying graphs in a loop does not pay cudaMalloc / cudaFree each time.
cudaMemPool_t device_pool(int dev)
{
    static std::mutex mu;
    static cudaMemPool_t pools[64] = {};
    std::lock_guard<std::mutex> lock(mu);
    if (dev < 0 || dev >= 64) return nullptr;
    if (!pools[dev]) {
        cudaMemPoolProps props{};
        props.allocType = cudaMemAllocationTypePinned;
        props.handleTypes = cudaMemHandleTypeNone;
        props.location.type = cudaMemLocationTypeDevice;
        props.location.id = dev;
        cudaMemPool_t pool = nullptr;
        if (cudaMemPoolCreate(&pool, &props) != cudaSuccess) {
            cudaGetLastError();
            return nullptr;
        }
        uint64_t keep = UINT64_MAX;
        cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
        pools[dev] = pool;
    }
    return pools[dev];
}

template <typename T>
lp_status dev_alloc(T **p, int64_t count, const char *what, cudaStream_t st, int dev)
{
    *p = nullptr;
    if (count <= 0) count = 1;
    cudaMemPool_t pool = device_pool(dev);
    cudaError_t e = pool ? cudaMallocFromPoolAsync((void **)p, (size_t)count * sizeof(T), pool, st)
                         : cudaMalloc((void **)p, (size_t)count * sizeof(T));
    if (e != cudaSuccess) {
        *p = nullptr;
        cudaGetLastError();
        return fail(e == cudaErrorMemoryAllocation ? LP_ENOMEM : LP_ECUDA,
                    std::string("device allocation of ") + what + " failed: " +
                        cudaGetErrorString(e));
    }
    return LP_OK;
}

// Pinned host blocks of up to PINNED_CACHE_MAX bytes are kept for reuse in
// power-of-two size classes: cudaMallocHost is slow, and cudaFreeHost may
// wait for the whole device, which would stall every other stream of a
// process that creates and destroys graph sets while others run (a server).
constexpr size_t PINNED_CACHE_MAX = (size_t)1 << 20;
constexpr int PINNED_CLASSES = 13;  // 256 B .. 1 MiB
constexpr size_t PINNED_KEEP = 256; // blocks kept per class
struct PinnedCache {
    std::mutex mu;
    std::vector<void *> free_[PINNED_CLASSES];
    std::unordered_map<void *, int> cls;  // live cached-size blocks and their class
};
PinnedCache &pinned_cache()
{
    static PinnedCache *c = new PinnedCache;  // never destroyed: blocks may outlive statics
    return *c;
}
int pinned_class(size_t bytes)
{
    int k = 0;
    while (((size_t)256 << k) < bytes) ++k;
    return k;
}
void *pinned_take(size_t bytes)
{
    if (bytes <= PINNED_CACHE_MAX) {
        const int k = pinned_class(bytes);
        PinnedCache &c = pinned_cache();
        {
            std::lock_guard<std::mutex> lock(c.mu);
            if (!c.free_[k].empty()) {
                void *q = c.free_[k].back();
                c.free_[k].pop_back();
                c.cls[q] = k;
                return q;
            }
        }
        void *q = nullptr;
        if (cudaMallocHost(&q, (size_t)256 << k) != cudaSuccess) {
            cudaGetLastError();
            return nullptr;
        }
        std::lock_guard<std::mutex> lock(c.mu);
        c.cls[q] = k;
        return q;
    }
    void *q = nullptr;
    if (cudaMallocHost(&q, bytes) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return q;
}
void host_free(void *p)
{
    if (!p) return;
    PinnedCache &c = pinned_cache();
    {
        std::lock_guard<std::mutex> lock(c.mu);
        auto it = c.cls.find(p);
        if (it != c.cls.end()) {
            const int k = it->second;
            c.cls.erase(it);
            if (c.free_[k].size() < PINNED_KEEP) {
                c.free_[k].push_back(p);
                return;
            }
        }
    }
    cudaFreeHost(p);
}

template <typename T>
lp_status host_alloc(T **p, int64_t count, const char *what)
{
    *p = nullptr;
    if (count <= 0) count = 1;
    void *q = pinned_take((size_t)count * sizeof(T));
    if (!q) return fail(LP_ENOMEM, std::string("pinned host allocation of ") + what + " failed");
    *p = static_cast<T *>(q);
    return LP_OK;
}

uint64_t next_pow2(uint64_t x)
{
    uint64_t p = 1;
    while (p < x) p <<= 1;
    return p;
}

const char *ingest_what(int32_t code)
{
    switch (code) {
    case lp::ING_OFF_FIRST: return "offsets[0] must be 0";
    case lp::ING_OFF_ORDER: return "offsets must be non-decreasing (first bad vertex)";
    case lp::ING_OFF_LAST: return "offsets[n] must equal m";
    case lp::ING_INDEX: return "column index outside [0, n) (entry)";
    case lp::ING_WEIGHT: return "weight < 1 (entry)";
    case lp::ING_WDEG: return "summed weight of a vertex reaches 2^31 (vertex)";
    case lp::ING_ASYM: return "CSR is not symmetric";
    case lp::ING_LABEL: return "label outside [0, n) (vertex)";
    default: return "invalid input";
    }
}

// Sorted (v, u, summed w) triples of a CSR, duplicates merged.
struct Entry {
    int32_t v, u;
    int64_t w;
};

bool host_symmetric(int32_t n, const int32_t *off, const int32_t *idx, const int32_t *wts)
{
    std::vector<Entry> a, b;
    const int64_t m = off[n];
    a.reserve((size_t)m);
    b.reserve((size_t)m);
    for (int32_t v = 0; v < n; ++v)
        for (int32_t e = off[v]; e < off[v + 1]; ++e) {
            const int64_t w = wts ? wts[e] : 1;
            a.push_back({v, idx[e], w});
            b.push_back({idx[e], v, w});
        }
    auto less = [](const Entry &x, const Entry &y) { return x.v != y.v ? x.v < y.v : x.u < y.u; };
    auto merge = [&](std::vector<Entry> &x) {
        std::sort(x.begin(), x.end(), less);
        size_t k = 0;
        for (size_t i = 0; i < x.size(); ++i) {
            if (k > 0 && x[k - 1].v == x[i].v && x[k - 1].u == x[i].u)
                x[k - 1].w += x[i].w;
            else
                x[k++] = x[i];
        }
        x.resize(k);
    };
    merge(a);
    merge(b);
    if (a.size() != b.size()) return false;
    for (size_t i = 0; i < a.size(); ++i)
        if (a[i].v != b[i].v || a[i].u != b[i].u || a[i].w != b[i].w) return false;
    return true;
}


}  // namespace

// ----------------------------------------------------------------------------
// Device representation shared by graphs and batches
// ----------------------------------------------------------------------------
namespace lp {

struct GraphSet {
    int device = 0;
    int num_sms = 0;
    cudaStream_t st = nullptr;
    int32_t G = 0;
    int32_t nv = 0;  // total vertices
    int64_t ne = 0;  // total entries
    int32_t *off = nullptr, *idx = nullptr, *wts = nullptr;
    bool own_off = true, own_idx = true, own_wts = true;
    int32_t *lab[2] = {nullptr, nullptr};
    int32_t *list = nullptr;
    Thresholds th{};  // bucket bounds (defaults, or the autotuner's choice)
    int64_t bb[NUM_BUCKETS] = {}, bl[NUM_BUCKETS] = {};
    int64_t be[NUM_BUCKETS] = {};  // summed degree of each bucket
    // wave-partitioned bucket lists for asynchronous runs (built per wave count)
    int32_t *wlist = nullptr;
    int64_t *d_wtot = nullptr;
    int32_t wl_waves = 0;
    std::vector<int64_t> wstart, wcount;  // per class b * waves + k
    int32_t max_n = 0;
    bool rows_distinct = false;  // no row repeats a neighbour (identity first sweep)
    // multi-graph bookkeeping (device copies are null for a single graph)
    int32_t *vgraph = nullptr, *g_vbase = nullptr, *g_active = nullptr, *g_n = nullptr;
    int64_t *g_ebase = nullptr;
    std::vector<int32_t> h_n, h_vbase;
    std::vector<int64_t> h_m, h_ebase;
    // iteration state
    int32_t *changed = nullptr, *h_changed = nullptr, *h_active = nullptr;
    int64_t changed_cap = 0;
    std::vector<int> final_buf;
    std::vector<lp_rak_result> results;
    std::vector<int64_t> history;  // graph 0
    // hub tasks of the hub bucket (plain) and of its part in each wave, with
    // their counts of long rows, segments and partitions; segment records,
    // partition offsets and bests (sized for the plain list, which every wave
    // part is a subset of); fallback tables, used lists and per-task counters
    HubTask *htask = nullptr, *htask_w = nullptr;
    int64_t hmulti = 0, hsegs = 0, hparts = 0;
    std::vector<int64_t> hmulti_w, hsegs_w, hparts_w, hsegs_at_w, hparts_at_w;
    int32_t *hseg_task = nullptr, *hpart_task = nullptr;      // plain list
    int32_t *hseg_task_w = nullptr, *hpart_task_w = nullptr;  // wave lists, wave after wave
    int32_t *hrec = nullptr;
    int32_t *hpoff = nullptr;
    uint4 *hpbest = nullptr;
    unsigned long long *hkey = nullptr;
    uint32_t *hnpos = nullptr;
    int32_t *hused = nullptr, *hdone = nullptr, *hnused = nullptr;
    uint32_t *hmaj = nullptr;  // long rows' majority counters (4 per hub task)
    int2 *hvote = nullptr;     // per segment item: its majority vote
    // SLPA (Sec. 3.4): memory slots (slpa_slots x nv, slot t of v at t * nv + v)
    // and the labels spoken to every packed entry in the current iteration
    int32_t *slpa_mem = nullptr, *spoken = nullptr;
    // COPRA (Sec. 3.3): two set buffers (nv x copra_L pairs), which one holds
    // the last run's sets, and the global tables of long rows
    int32_t *cset_l[2] = {nullptr, nullptr};
    uint32_t *cset_b[2] = {nullptr, nullptr};
    int32_t copra_L = 0, copra_cur = 0, copra_cap = 0;
    int32_t *ctab_key = nullptr;
    unsigned long long *ctab_sum = nullptr, *ctab_first = nullptr;
    int32_t ctab_lg = 0;
    // rows that take a CTA, by kind and wave (copra_rows), and the bins' starts
    int32_t *crows = nullptr, *cbins = nullptr, *covf = nullptr;
    int64_t cbins_cap = 0;
    std::vector<int32_t> h_cbins;
    std::vector<int64_t> h_cstart;
    int32_t max_deg = 0;  // longest row (single graphs)
    int32_t slpa_slots = 0, slpa_filled = 0;
    bool slpa_on = false;
    int32_t *cpos = nullptr;   // rows left by a pre-pass (nv) and their count, open long rows
    int32_t *ccount = nullptr;
    // packed rows of the run's list (lp_internal.cuh), built for one wave
    // count at a time (pk_waves, 0 = none yet)
    int64_t *pk_rp = nullptr, *pk_first = nullptr;
    int32_t *pk_idx = nullptr, *pk_wts = nullptr;
    int32_t pk_waves = 0;
    uint8_t *vmaj = nullptr;   // per vertex: settled by the majority pre-pass
    // all-waves launches of many-wave runs over small rows only: wave starts
    // of the small bucket (device) and the grid barrier's words (count,
    // generation, error flag)
    int64_t *d_wstart0 = nullptr;
    int32_t *d_coop = nullptr;
    // modularity and label staging scratch
    unsigned long long *kc = nullptr, *macc = nullptr, *h_macc = nullptr;
    int64_t kc_cap = 0;
    std::vector<double> q_cache;  // per-graph modularity of the current labels
    bool q_valid = false;
    int32_t *g_sel = nullptr;     // per graph: buffer holding its final labels
    int32_t *lab_tmp = nullptr;
    IngestOut *d_ing = nullptr, *h_ing = nullptr;
    int64_t *d_counts = nullptr, *h_counts = nullptr;
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    std::vector<cudaEvent_t> prof_ev;  // start/stop pairs of profiled launches

    ~GraphSet() { release(); }

    void release()
    {
        if (st) cudaStreamSynchronize(st);
        cudaStream_t s0 = st;
        auto f = [s0](void *p) {
            if (p) cudaFreeAsync(p, s0);
        };
        auto fh = [](void *p) {
            if (p) host_free(p);
        };
        if (own_off) f(off);
        if (own_idx) f(idx);
        if (own_wts) f(wts);
        off = idx = wts = nullptr;
        f(lab[0]);
        f(lab[1]);
        f(list);
        f(wlist);
        f(d_wtot);
        f(vgraph);
        f(g_vbase);
        f(g_active);
        f(g_n);
        f(g_ebase);
        f(changed);
        fh(h_changed);
        fh(h_active);
        f(htask);
        f(htask_w);
        f(hkey);
        f(hnpos);
        f(hused);
        f(hnused);
        f(hdone);
        f(hrec);
        f(hpoff);
        f(hpbest);
        f(hmaj);
        f(hvote);
        hvote = nullptr;
        f(cpos);
        f(ccount);
        cpos = ccount = nullptr;
        f(slpa_mem);
        f(spoken);
        slpa_mem = spoken = nullptr;
        for (int b = 0; b < 2; ++b) {
            f(cset_l[b]);
            f(cset_b[b]);
            cset_l[b] = nullptr;
            cset_b[b] = nullptr;
        }
        copra_L = copra_cap = 0;
        f(ctab_key);
        f(ctab_sum);
        f(ctab_first);
        ctab_key = nullptr;
        ctab_sum = ctab_first = nullptr;
        ctab_lg = 0;
        f(crows);
        f(cbins);
        f(covf);
        crows = cbins = covf = nullptr;
        cbins_cap = 0;
        slpa_slots = slpa_filled = 0;
        f(pk_rp);
        f(pk_first);
        f(pk_idx);
        f(pk_wts);
        pk_rp = pk_first = nullptr;
        pk_idx = pk_wts = nullptr;
        pk_waves = 0;
        f(hseg_task);
        f(hpart_task);
        f(hseg_task_w);
        f(hpart_task_w);
        f(d_res);
        f(d_stop);
        f(kc);
        f(macc);
        fh(h_macc);
        f(g_sel);
        f(lab_tmp);
        f(d_ing);
        fh(h_ing);
        f(d_counts);
        fh(h_counts);
        f(vmaj);
        f(d_wstart0);
        f(d_coop);
        if (ev0) cudaEventDestroy(ev0);
        if (ev1) cudaEventDestroy(ev1);
        lab[0] = lab[1] = list = wlist = vgraph = g_vbase = g_active = g_n = nullptr;
        d_wtot = nullptr;
        g_ebase = nullptr;
        changed = h_changed = h_active = nullptr;
        htask = htask_w = nullptr;
        hkey = nullptr;
        hnpos = nullptr;
        hused = hdone = hnused = nullptr;
        hrec = nullptr;
        hpoff = nullptr;
        hpbest = nullptr;
        hmaj = nullptr;
        vmaj = nullptr;
        d_wstart0 = nullptr;
        d_coop = nullptr;
        hseg_task = hpart_task = hseg_task_w = hpart_task_w = nullptr;
        d_res = nullptr;
        d_stop = nullptr;
        kc = macc = h_macc = nullptr;
        g_sel = nullptr;
        lab_tmp = nullptr;
        d_ing = h_ing = nullptr;
        d_counts = h_counts = nullptr;
        ev0 = ev1 = nullptr;
        for (cudaEvent_t e : prof_ev) cudaEventDestroy(e);
        prof_ev.clear();
        if (ev_iter) cudaEventDestroy(ev_iter);
        ev_iter = nullptr;
        drop_graph();
        if (gr_stream) cudaStreamDestroy(gr_stream);
        gr_stream = nullptr;
        if (h_res) host_free(h_res);
        h_res = nullptr;
        if (h_stop) host_free(h_stop);
        h_stop = nullptr;
        h_stop_cap = 0;
        for (cudaEvent_t &e : run_ev) {
            if (e) cudaEventDestroy(e);
            e = nullptr;
        }
        cudaStreamSynchronize(st);
    }

    lp_status begin(void *stream)
    {
        LP_CU(cudaGetDevice(&device));
        LP_CU(cudaDeviceGetAttribute(&num_sms, cudaDevAttrMultiProcessorCount, device));
        st = (cudaStream_t)stream;
        static std::atomic<uint64_t> prepared{0};
        if (device < 64 && !(prepared.load() & (1ull << device))) {
            if (sweep_prepare() != 0 || wave_prepare() != 0 || copra_prepare() != 0)
                return fail(LP_ECUDA, "setting kernel attributes failed");
            prepared |= (1ull << device);
        }
        LP_TRY(dev_alloc(&d_ing, 1, "ingest status", st, device));
        LP_TRY(host_alloc(&h_ing, 1, "ingest status"));
        LP_TRY(dev_alloc(&d_counts, 3 * NUM_BUCKETS, "bucket counts", st, device));
        LP_TRY(host_alloc(&h_counts, 3 * NUM_BUCKETS, "bucket counts"));
        LP_CU(cudaEventCreate(&ev0));
        LP_CU(cudaEventCreate(&ev1));
        return LP_OK;
    }

    lp_status read_ingest(int graph_index)
    {
        LP_CU(cudaMemcpyAsync(h_ing, d_ing, sizeof(IngestOut), cudaMemcpyDeviceToHost, st));
        LP_CU(cudaStreamSynchronize(st));
        if (h_ing->err != ING_OK) {
            char buf[256];
            if (graph_index >= 0)
                snprintf(buf, sizeof buf, "graph %d: %s %d", graph_index, ingest_what(h_ing->err),
                         h_ing->err_at);
            else
                snprintf(buf, sizeof buf, "%s %d", ingest_what(h_ing->err), h_ing->err_at);
            return fail(LP_EINVAL, buf);
        }
        return LP_OK;
    }

    // validate every graph of a batch (device CSR in place): the checks of
    // all graphs are launched before one read-back of their status words (a
    // weight-sum check follows for graphs whose degrees and weights could
    // reach 2^31); errors name the first invalid graph
    lp_status validate_all()
    {
        IngestOut *d_all = nullptr, *h_all = nullptr;
        LP_TRY(dev_alloc(&d_all, G, "validation status", st, device));
        lp_status s = host_alloc(&h_all, G, "validation status");
        Launches L;
        auto launch_and_read = [&](bool wdeg) -> lp_status {
            for (int32_t g = 0; g < G; ++g) {
                const int64_t ob = (int64_t)h_vbase[(size_t)g] + g, e0 = h_ebase[(size_t)g];
                const int32_t *w = wts ? wts + e0 : nullptr;
                int rc = 0;
                if (!wdeg)
                    rc = ingest_validate(off + ob, idx + e0, w, h_n[(size_t)g], h_m[(size_t)g],
                                         d_all + g, st, &L.n);
                else if ((int64_t)h_all[g].max_deg * h_all[g].max_w >= 2147483648LL)
                    rc = ingest_check_wdeg(off + ob, w, h_n[(size_t)g], d_all + g, st, &L.n);
                if (rc != 0) return fail(LP_ECUDA, cuda_msg("validation launch", cudaGetLastError()));
            }
            LP_CU(cudaMemcpyAsync(h_all, d_all, (size_t)G * sizeof(IngestOut),
                                  cudaMemcpyDeviceToHost, st));
            LP_CU(cudaStreamSynchronize(st));
            for (int32_t g = 0; g < G; ++g)
                if (h_all[g].err != ING_OK) {
                    char buf[256];
                    snprintf(buf, sizeof buf, "graph %d: %s %d", g, ingest_what(h_all[g].err),
                             h_all[g].err_at);
                    return fail(LP_EINVAL, buf);
                }
            return LP_OK;
        };
        if (s == LP_OK) s = launch_and_read(false);
        if (s == LP_OK) s = launch_and_read(true);
        cudaFreeAsync(d_all, st);
        if (h_all) host_free(h_all);
        return s;
    }

    // validate a single graph's device CSR and check its row order in one pass
    lp_status validate_single(int32_t n, int64_t m)
    {
        uint32_t *bits = nullptr;
        LP_TRY(dev_alloc(&bits, m / 32 + 1, "row-start bitmap", st, device));
        Launches L;
        const int rc = ingest_validate_ordered(off, idx, wts, n, m, bits, d_ing, st, &L.n);
        cudaFreeAsync(bits, st);
        if (rc != 0) return fail(LP_ECUDA, cuda_msg("validation launch", cudaGetLastError()));
        LP_TRY(read_ingest(-1));
        if ((int64_t)h_ing->max_deg * (int64_t)h_ing->max_w >= 2147483648LL) {
            if (ingest_check_wdeg(off, wts, n, d_ing, st, &L.n) != 0)
                return fail(LP_ECUDA, cuda_msg("weight-sum launch", cudaGetLastError()));
            LP_TRY(read_ingest(-1));
        }
        rows_distinct = h_ing->repeated == 0;
        max_deg = h_ing->max_deg;
        return LP_OK;
    }

    // Every row strictly increasing -> no repeated neighbour: the first sweep
    // from unique labels can take the identity path.
    lp_status check_row_order()
    {
        rows_distinct = false;
        uint32_t *bits = nullptr;
        LP_TRY(dev_alloc(&bits, ne / 32 + 1, "row-start bitmap", st, device));
        LP_CU(cudaMemsetAsync(d_ing, 0, sizeof(IngestOut), st));  // the check's status word
        Launches L;
        const int rc = ingest_row_order(off, idx, nv, ne, vgraph, g_ebase, bits, d_ing, st, &L.n);
        cudaFreeAsync(bits, st);
        if (rc != 0) return fail(LP_ECUDA, cuda_msg("row order check", cudaGetLastError()));
        LP_TRY(read_ingest(-1));
        rows_distinct = h_ing->repeated == 0;
        return LP_OK;
    }

    lp_status bucket()
    {
        Launches L;
        int32_t *blk = nullptr;
        LP_TRY(dev_alloc(&blk, (int64_t)(ingest_bucket_scratch_bytes(nv) / sizeof(int32_t)),
                         "bucket scratch", st, device));
        lp_status s = LP_OK;
        if (dev_alloc(&list, nv, "bucket list", st, device) != LP_OK) {
            cudaFreeAsync(blk, st);
            return LP_ENOMEM;
        }
        if (ingest_bucket(off, nv, vgraph, g_vbase, th, list, blk, d_counts, st, &L.n) != 0)
            s = fail(LP_ECUDA, cuda_msg("bucketing launch", cudaGetLastError()));
        if (s == LP_OK) {
            cudaError_t e = cudaMemcpyAsync(h_counts, d_counts, 3 * NUM_BUCKETS * sizeof(int64_t),
                                            cudaMemcpyDeviceToHost, st);
            if (e == cudaSuccess) e = cudaStreamSynchronize(st);
            if (e != cudaSuccess) s = fail(LP_ECUDA, cuda_msg("bucket counts", e));
        }
        cudaFreeAsync(blk, st);
        if (s != LP_OK) return s;
        for (int c = 0; c < NUM_BUCKETS; ++c) {
            bl[c] = h_counts[c];
            bb[c] = h_counts[NUM_BUCKETS + c];
            be[c] = h_counts[2 * NUM_BUCKETS + c];
        }
        if (!vmaj && bl[2] + bl[3] + bl[HUB_BUCKET] > 0)
            LP_TRY(dev_alloc(&vmaj, nv, "majority flags", st, device));
        if (!ccount) LP_TRY(dev_alloc(&ccount, 2, "pre-pass counters", st, device));
        if (!cpos && G == 1 && bl[2] + bl[3] + bl[HUB_BUCKET] > 0)
            LP_TRY(dev_alloc(&cpos, std::max(bl[2], std::max(bl[3], bl[HUB_BUCKET])),
                             "pre-pass row lists", st, device));
        // hub vertices: longest rows first, so the static CTA assignment of
        // the hub kernels balances
        if (bl[HUB_BUCKET] > 0) {
            int32_t *ordered = nullptr;
            int64_t *hsc = nullptr;
            LP_TRY(dev_alloc(&hsc, hub_scratch_ints(bl[HUB_BUCKET]), "hub scratch", st, device));
            lp_status as = dev_alloc(&ordered, bl[HUB_BUCKET], "hub order", st, device);
            if (as != LP_OK) {
                cudaFreeAsync(hsc, st);
                return as;
            }
            cudaError_t e = cudaSuccess;
            if (hub_order(list + bb[HUB_BUCKET], bl[HUB_BUCKET], off, vgraph, ordered, hsc, st,
                          &L.n) != 0)
                e = cudaGetLastError();
            if (e == cudaSuccess)
                e = cudaMemcpyAsync(list + bb[HUB_BUCKET], ordered, bl[HUB_BUCKET] * sizeof(int32_t),
                                    cudaMemcpyDeviceToDevice, st);
            cudaFreeAsync(ordered, st);
            if (e != cudaSuccess) {
                cudaFreeAsync(hsc, st);
                return fail(LP_ECUDA, cuda_msg("hub order", e));
            }
            // hub tasks, the segment / partition scratch of the long rows and
            // one fallback table per long row (zeroed; every use leaves it zeroed)
            as = dev_alloc(&htask, bl[HUB_BUCKET], "hub tasks", st, device);
            if (as != LP_OK) {
                cudaFreeAsync(hsc, st);
                return as;
            }
            int64_t tot[5] = {0, 0, 0, 0, 0};
            const int rc = hub_tasks(list + bb[HUB_BUCKET], bl[HUB_BUCKET], off, vgraph, htask,
                                     d_counts, hsc, st, &L.n);
            cudaFreeAsync(hsc, st);
            if (rc != 0) return fail(LP_ECUDA, cuda_msg("hub tasks", cudaGetLastError()));
            LP_CU(cudaMemcpyAsync(tot, d_counts, sizeof tot, cudaMemcpyDeviceToHost, st));
            LP_CU(cudaStreamSynchronize(st));
            hmulti = tot[0];
            hsegs = tot[2];
            hparts = tot[3];
            const int64_t slots = tot[1] > 0 ? tot[1] : 1;
            LP_TRY(dev_alloc(&hrec, (tot[2] > 0 ? tot[2] : 1) * (int64_t)HUB_REC * HUB_SEG,
                             "hub records", st, device));
            LP_TRY(dev_alloc(&hpoff, tot[4] > 0 ? tot[4] : 1, "hub partition offsets", st, device));
            LP_TRY(dev_alloc(&hpbest, 2 * (tot[3] > 0 ? tot[3] : 1), "hub partition bests", st,
                             device));
            LP_TRY(dev_alloc(&hseg_task, tot[2], "hub item maps", st, device));
            LP_TRY(dev_alloc(&hpart_task, tot[3], "hub item maps", st, device));
            if (hub_item_maps(htask, hmulti, hseg_task, hpart_task, st, &L.n) != 0)
                return fail(LP_ECUDA, cuda_msg("hub item maps", cudaGetLastError()));
            LP_TRY(dev_alloc(&hkey, slots, "hub tables", st, device));
            LP_TRY(dev_alloc(&hnpos, slots, "hub tables", st, device));
            LP_TRY(dev_alloc(&hused, slots / 2 + 1, "hub used lists", st, device));
            LP_TRY(dev_alloc(&hdone, bl[HUB_BUCKET], "hub counters", st, device));
            LP_TRY(dev_alloc(&hnused, bl[HUB_BUCKET], "hub counters", st, device));
            LP_TRY(dev_alloc(&hmaj, 4 * bl[HUB_BUCKET], "hub majority counters", st, device));
            LP_TRY(dev_alloc(&hvote, tot[2] > 0 ? tot[2] : 1, "hub majority votes", st, device));
            LP_CU(cudaMemsetAsync(hkey, 0, (size_t)slots * sizeof(unsigned long long), st));
            LP_CU(cudaMemsetAsync(hnpos, 0, (size_t)slots * sizeof(uint32_t), st));
            LP_CU(cudaMemsetAsync(hdone, 0, (size_t)bl[HUB_BUCKET] * sizeof(int32_t), st));
            LP_CU(cudaMemsetAsync(hnused, 0, (size_t)bl[HUB_BUCKET] * sizeof(int32_t), st));
        }
        return LP_OK;
    }

    // Sort the vertices into buckets again with other bounds: every list
    // derived from the buckets (hub tasks and scratch, wave lists, captured
    // run graphs) is dropped and rebuilt on demand.
    lp_status rebucket(const Thresholds &t)
    {
        LP_CU(cudaStreamSynchronize(st));
        auto f = [this](void *p) {
            if (p) cudaFreeAsync(p, st);
        };
        f(list);
        f(htask);
        f(htask_w);
        f(hrec);
        f(hpoff);
        f(hpbest);
        f(hmaj);
        f(hvote);
        f(cpos);
        f(hkey);
        f(hnpos);
        f(hused);
        f(hdone);
        f(hnused);
        f(hseg_task);
        f(hpart_task);
        f(hseg_task_w);
        f(hpart_task_w);
        f(wlist);
        list = wlist = nullptr;
        htask = htask_w = nullptr;
        hrec = nullptr;
        hpoff = nullptr;
        hpbest = nullptr;
        hmaj = nullptr;
        hvote = nullptr;
        cpos = nullptr;
        hkey = nullptr;
        hnpos = nullptr;
        hused = hdone = hnused = nullptr;
        hseg_task = hpart_task = hseg_task_w = hpart_task_w = nullptr;
        hmulti = hsegs = hparts = 0;
        wl_waves = 0;
        pk_waves = 0;
        drop_graph();
        gr_last = GraphKey{};
        th = t;
        return bucket();
    }

    // Time `sweeps` iterations (tolerance 0, from unique labels) for a grid
    // of bucket bounds within the kernels' capacities and keep the fastest.
    // Labels, iteration counts and modularity do not depend on the bounds.
    lp_status autotune(const lp_rak_params *p, bool multi, int32_t sweeps, lp_tune_result *out)
    {
        if (!p || !out) return fail(LP_EINVAL, "params or out is NULL");
        if (sweeps < 1 || sweeps > 100) return fail(LP_EINVAL, "sweeps must lie in [1, 100]");
        lp_rak_params q = *p;
        q.tolerance = 0.0;
        q.max_iter = sweeps;
        q.iter_offset = 0;
        q.init_labels = nullptr;
        const Thresholds def{};
        auto timed = [&](const Thresholds &t, float *ms) -> lp_status {
            LP_TRY(rebucket(t));
            LP_TRY(run_host(&q, multi));
            *ms = results[0].gpu_ms;
            return LP_OK;
        };
        const int32_t small_c[] = {8, 16, 24, SMALL_MAX};
        const int32_t warp_c[] = {64, WARP_MAX};
        const int32_t cta_c[] = {256, CTA_MAX};
        Thresholds best = def;
        float best_ms = 0.f;
        LP_TRY(timed(def, &best_ms));
        out->default_ms = best_ms;
        int32_t n = 1;
        for (int32_t a : small_c)
            for (int32_t b : warp_c)
                for (int32_t c : cta_c) {
                    Thresholds t;
                    t.max[0] = a;
                    t.max[1] = b;
                    t.max[2] = c;
                    t.max[3] = CTA2_MAX;
                    bool same = true;
                    for (int k = 0; k < NUM_BUCKETS - 1; ++k) same = same && t.max[k] == def.max[k];
                    if (same) continue;
                    float ms = 0.f;
                    LP_TRY(timed(t, &ms));
                    ++n;
                    if (ms < best_ms) {
                        best_ms = ms;
                        best = t;
                    }
                }
        LP_TRY(rebucket(best));
        out->small_max = best.max[0];
        out->warp_max = best.max[1];
        out->cta_max = best.max[2];
        out->cta2_max = best.max[3];
        out->candidates = n;
        out->best_ms = best_ms;
        return LP_OK;
    }

    // mean degree of the small bucket, rounded up (sizes its kernels' tiles)
    int32_t small_mean_deg() const
    {
        return bl[0] > 0 ? (int32_t)((be[0] + bl[0] - 1) / bl[0]) : 0;
    }

    lp_status alloc_labels()
    {
        LP_TRY(dev_alloc(&lab[0], nv, "labels", st, device));
        LP_TRY(dev_alloc(&lab[1], nv, "labels", st, device));
        Launches L;
        if (fill_iota(lab[0], nv, vgraph, g_vbase, st, &L.n) != 0)
            return fail(LP_ECUDA, cuda_msg("label init", cudaGetLastError()));
        final_buf.assign((size_t)G, 0);
        results.assign((size_t)G, lp_rak_result{0, 0, 0, 0.0f});
        return LP_OK;
    }

    // Partition the bucket lists by wave (local id mod waves), once per wave count.
    lp_status ensure_waves(int32_t waves)
    {
        if (waves == wl_waves) return LP_OK;
        const int64_t len = bb[NUM_BUCKETS - 1] + bl[NUM_BUCKETS - 1];
        if (!wlist) LP_TRY(dev_alloc(&wlist, nv, "wave lists", st, device));
        if (!d_wtot) LP_TRY(dev_alloc(&d_wtot, NUM_BUCKETS * WAVE_MAX, "wave sizes", st, device));
        int32_t *hist = nullptr;
        LP_TRY(dev_alloc(&hist, wave_hist_ints(len, waves), "wave histogram", st, device));
        if (!d_wstart0) LP_TRY(dev_alloc(&d_wstart0, WAVE_MAX, "wave starts", st, device));
        Launches L;
        const int nc = NUM_BUCKETS * waves;
        std::vector<int64_t> tot((size_t)nc);
        cudaError_t e = cudaSuccess;
        if (wave_partition(list, len, bb, vgraph, g_vbase, waves, hist, d_wtot, wlist, st, &L.n) != 0)
            e = cudaGetLastError();
        // the starts of the small bucket's waves: the partition's first class
        // starts (its scratch begins with the class starts)
        if (e == cudaSuccess)
            e = len > 0 ? cudaMemcpyAsync(d_wstart0, hist, (size_t)waves * sizeof(int64_t),
                                          cudaMemcpyDeviceToDevice, st)
                        : cudaMemsetAsync(d_wstart0, 0, (size_t)waves * sizeof(int64_t), st);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(tot.data(), d_wtot, (size_t)nc * sizeof(int64_t),
                                cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        cudaFreeAsync(hist, st);
        if (e != cudaSuccess) return fail(LP_ECUDA, cuda_msg("wave partition", e));
        wstart.assign((size_t)nc, 0);
        wcount = tot;
        int64_t acc = 0;
        for (int c = 0; c < nc; ++c) {
            wstart[(size_t)c] = acc;
            acc += tot[(size_t)c];
        }
        // hub tasks of each wave's part of the hub bucket (contiguous classes)
        hmulti_w.assign((size_t)waves, 0);
        hsegs_w.assign((size_t)waves, 0);
        hparts_w.assign((size_t)waves, 0);
        if (bl[HUB_BUCKET] > 0) {
            if (!htask_w) LP_TRY(dev_alloc(&htask_w, bl[HUB_BUCKET], "hub tasks", st, device));
            const int64_t hub0 = wstart[(size_t)HUB_BUCKET * waves];
            std::vector<int64_t> tots(5 * (size_t)waves, 0);
            int64_t *d_tot = nullptr;
            LP_TRY(dev_alloc(&d_tot, 5 * (int64_t)waves, "hub totals", st, device));
            int64_t most = 1;
            for (int k = 0; k < waves; ++k)
                most = std::max(most, wcount[(size_t)HUB_BUCKET * waves + k]);
            int64_t *hsc = nullptr;
            const lp_status as = dev_alloc(&hsc, hub_scratch_ints(most), "hub scratch", st, device);
            if (as != LP_OK) {
                cudaFreeAsync(d_tot, st);
                return as;
            }
            Launches L2;
            cudaError_t e2 = cudaMemsetAsync(d_tot, 0, tots.size() * sizeof(int64_t), st);
            for (int k = 0; k < waves && e2 == cudaSuccess; ++k) {
                const int64_t c = wcount[(size_t)HUB_BUCKET * waves + k];
                if (c == 0) continue;
                const int64_t st0 = wstart[(size_t)HUB_BUCKET * waves + k];
                if (hub_tasks(wlist + st0, c, off, vgraph, htask_w + (st0 - hub0), d_tot + 5 * k,
                              hsc, st, &L2.n) != 0)
                    e2 = cudaGetLastError();
            }
            cudaFreeAsync(hsc, st);
            if (e2 == cudaSuccess)
                e2 = cudaMemcpyAsync(tots.data(), d_tot, tots.size() * sizeof(int64_t),
                                     cudaMemcpyDeviceToHost, st);
            if (e2 == cudaSuccess) e2 = cudaStreamSynchronize(st);
            cudaFreeAsync(d_tot, st);
            if (e2 != cudaSuccess) return fail(LP_ECUDA, cuda_msg("wave hub tasks", e2));
            hsegs_at_w.assign((size_t)waves, 0);
            hparts_at_w.assign((size_t)waves, 0);
            int64_t seg_at = 0, part_at = 0;
            for (int k = 0; k < waves; ++k) {
                hmulti_w[(size_t)k] = tots[5 * (size_t)k];
                hsegs_w[(size_t)k] = tots[5 * (size_t)k + 2];
                hparts_w[(size_t)k] = tots[5 * (size_t)k + 3];
                hsegs_at_w[(size_t)k] = seg_at;
                hparts_at_w[(size_t)k] = part_at;
                seg_at += hsegs_w[(size_t)k];
                part_at += hparts_w[(size_t)k];
            }
            // the waves' item maps, wave after wave (together the plain list's size)
            if (!hseg_task_w) LP_TRY(dev_alloc(&hseg_task_w, hsegs, "hub item maps", st, device));
            if (!hpart_task_w)
                LP_TRY(dev_alloc(&hpart_task_w, hparts, "hub item maps", st, device));
            for (int k = 0; k < waves; ++k) {
                if (hmulti_w[(size_t)k] == 0) continue;
                const int64_t st0 = wstart[(size_t)HUB_BUCKET * waves + k];
                if (hub_item_maps(htask_w + (st0 - hub0), hmulti_w[(size_t)k],
                                  hseg_task_w + hsegs_at_w[(size_t)k],
                                  hpart_task_w + hparts_at_w[(size_t)k], st, &L2.n) != 0)
                    return fail(LP_ECUDA, cuda_msg("wave hub item maps", cudaGetLastError()));
            }
        }
        wl_waves = waves;
        return LP_OK;
    }

    // Pack the rows of the run's list (the bucket list, or the wave lists of
    // `waves` > 1) in list order, once per wave count; hub tasks learn their
    // packed row starts.  A captured run graph reads the packed arrays, so it
    // is dropped whenever they are rebuilt.
    lp_status ensure_packed(int32_t waves)
    {
        if (waves == pk_waves) return LP_OK;
        drop_graph();
        const int64_t len = bb[HUB_BUCKET] + bl[HUB_BUCKET];
        if (!pk_rp) LP_TRY(dev_alloc(&pk_rp, len + 1, "packed row starts", st, device));
        if (!pk_first)
            LP_TRY(dev_alloc(&pk_first, pack_chunks(ne) + 1, "packed chunk rows", st, device));
        if (!pk_idx) LP_TRY(dev_alloc(&pk_idx, ne, "packed rows", st, device));
        if (wts && !pk_wts) LP_TRY(dev_alloc(&pk_wts, ne, "packed rows", st, device));
        if (((uintptr_t)pk_idx & 15u) || ((uintptr_t)pk_wts & 15u))
            return fail(LP_ECUDA, "device allocation is not 16-byte aligned");
        int64_t *scratch = nullptr;
        LP_TRY(dev_alloc(&scratch, pack_scratch_ints(len), "packing scratch", st, device));
        Launches L;
        int rc = pack_rows(waves > 1 ? wlist : list, len, off, idx, wts, ne, vgraph, g_vbase,
                           g_ebase, waves, be, scratch, pk_rp, pk_first, pk_idx, pk_wts, st, &L.n);
        if (rc == 0 && bl[HUB_BUCKET] > 0) {
            const int64_t hub0 = waves > 1 ? wstart[(size_t)HUB_BUCKET * waves] : bb[HUB_BUCKET];
            rc = hub_task_starts(waves > 1 ? htask_w : htask, bl[HUB_BUCKET], pk_rp + hub0, st,
                                 &L.n);
        }
        cudaFreeAsync(scratch, st);
        if (rc != 0) return fail(LP_ECUDA, cuda_msg("row packing", cudaGetLastError()));
        pk_waves = waves;
        return LP_OK;
    }

    lp_status ensure_changed(int64_t entries)
    {
        if (entries <= changed_cap) return LP_OK;
        if (changed) cudaFreeAsync(changed, st);
        if (h_changed) host_free(h_changed);
        changed = nullptr;
        h_changed = nullptr;
        changed_cap = 0;
        LP_TRY(dev_alloc(&changed, entries, "changed counters", st, device));
        LP_TRY(host_alloc(&h_changed, entries, "changed counters"));
        changed_cap = entries;
        return LP_OK;
    }

    // State of a run in progress (lp_rak_run / lp_batch_run drive it to the
    // end at once; the serving loop advances it one iteration per tick).
    struct RunState {
        lp_rak_params p{};
        bool multi = false;
        int32_t waves = 1;
        int cur = 0;
        int32_t it = 0;  // iterations launched
        int32_t active_left = 0;
        bool prof = false;
        bool coop = false;              // an all-waves launch ran in this run
        std::vector<int> prof_launch;   // bucket of each profiled launch
        std::vector<int64_t> prof_len;  // its vertex count
        std::vector<int32_t> prof_iter; // its iteration (launches past the end are not counted)
        SweepArgs a{};
    } rs;
    cudaEvent_t ev_iter = nullptr;  // end of the last launched iteration

    // a2 and the argument checks of Sec. 3.2's iteration over every graph of the set
    lp_status run_begin(const lp_rak_params *p, bool multi)
    {
        if (!p) return fail(LP_EINVAL, "params is NULL");
        if (!(p->tolerance >= 0.0 && p->tolerance <= 1.0))
            return fail(LP_EINVAL, "tolerance must lie in [0, 1]");
        if (p->max_iter < 1) return fail(LP_EINVAL, "max_iter must be >= 1");
        if (p->mode != LP_SYNC && p->mode != LP_ASYNC)
            return fail(LP_EINVAL, "mode must be LP_SYNC or LP_ASYNC");
        if (p->mode == LP_ASYNC && p->waves < 1) return fail(LP_EINVAL, "waves must be >= 1");
        // Sec. 3.3 asynchronous waves; more waves than vertices change nothing
        int32_t waves = 1;
        if (p->mode == LP_ASYNC) waves = std::min(p->waves, std::max(max_n, 1));
        if (waves > WAVE_MAX)
            return fail(LP_EINVAL, "waves must be <= 4096 unless it is >= the vertex count");
        if (multi && p->init_labels) return fail(LP_EINVAL, "batches start from unique labels");
        LP_TRY(ensure_changed((int64_t)p->max_iter * G));
        if (waves > 1) LP_TRY(ensure_waves(waves));
        LP_TRY(ensure_packed(waves));
        if (!ev_iter) LP_CU(cudaEventCreateWithFlags(&ev_iter, cudaEventDisableTiming));
        Launches L;

        // a2: initial labels (Sec. 3.2: unique labels) or a resumed labelling
        if (p->init_labels) {
            LP_CU(cudaMemcpyAsync(lab[0], p->init_labels, (size_t)nv * sizeof(int32_t),
                                  p->init_labels_on_device ? cudaMemcpyDeviceToDevice
                                                           : cudaMemcpyHostToDevice,
                                  st));
            if (check_labels(lab[0], nv, vgraph, g_vbase, g_n, d_ing, st, &L.n) != 0)
                return fail(LP_ECUDA, cuda_msg("label check", cudaGetLastError()));
            LP_TRY(read_ingest(-1));
        } else if (fill_iota(lab[0], nv, vgraph, g_vbase, st, &L.n) != 0) {
            return fail(LP_ECUDA, cuda_msg("label init", cudaGetLastError()));
        }
        // both buffers hold the initial labels: vertices without edges are never
        // written, and both modes alternate the buffers every iteration
        if (nv > 0)
            LP_CU(cudaMemcpyAsync(lab[1], lab[0], (size_t)nv * sizeof(int32_t),
                                  cudaMemcpyDeviceToDevice, st));
        LP_CU(cudaMemsetAsync(changed, 0, (size_t)p->max_iter * G * sizeof(int32_t), st));
        if (multi) {
            for (int32_t g = 0; g < G; ++g) h_active[g] = 1;
            LP_CU(cudaMemcpyAsync(g_active, h_active, (size_t)G * sizeof(int32_t),
                                  cudaMemcpyHostToDevice, st));
        }
        std::fill(final_buf.begin(), final_buf.end(), 0);
        q_valid = false;
        for (auto &r : results) r = lp_rak_result{0, 0, 0, 0.0f};
        rs.p = *p;
        rs.multi = multi;
        rs.waves = waves;
        rs.cur = 0;
        rs.it = 0;
        rs.active_left = G;
        rs.prof = g_prof_on.load();
        rs.coop = false;
        rs.prof_launch.clear();
        rs.prof_len.clear();
        rs.prof_iter.clear();
        LP_CU(cudaEventRecord(ev0, st));

        SweepArgs &a = rs.a;
        a = SweepArgs{};
        a.rp = pk_rp;
        a.idx = pk_idx;
        a.wts = wts ? pk_wts : nullptr;
        a.ne = ne;
        a.vgraph = vgraph;
        a.g_vbase = g_vbase;
        a.g_ebase = g_ebase;
        a.g_active = g_active;
        a.strict = p->strict ? 1 : 0;
        a.hkey = hkey;
        a.hnpos = hnpos;
        a.hused = hused;
        a.hnused = hnused;
        a.hdone = hdone;
        a.hrec = hrec;
        a.hpoff = hpoff;
        a.hpbest = hpbest;
        a.hmaj = hmaj;
        a.hvote = hvote;
        a.hopen = ccount ? ccount + 1 : nullptr;
        a.cpos = G == 1 ? cpos : nullptr;
        a.ccount = G == 1 ? ccount : nullptr;
        a.vmaj = vmaj;
        a.small_mean_deg = small_mean_deg();
        a.waves = (uint32_t)waves;
        return LP_OK;
    }

    bool run_done() const { return rs.active_left == 0 || rs.it >= rs.p.max_iter; }

    // Launch iteration `it`'s sweeps (a3-a5 for every bucket and wave) on
    // stream s, reading label buffer `cur` and writing cur ^ 1; profiled
    // launches are bracketed by events and listed in rs.prof_launch.
    lp_status launch_sweeps(cudaStream_t s, int32_t it, int cur, bool prof, int64_t *kernels,
                            bool capturing = false)
    {
        const int32_t waves = rs.waves;
        SweepArgs &a = rs.a;
        const int64_t t = (int64_t)it + rs.p.iter_offset;
        // sync reads lab_in only; async reads lab_out for neighbours of
        // earlier waves (written by this iteration's earlier launches)
        a.lab_in = lab[cur];
        a.lab_out = lab[cur ^ 1];
        a.spoken = nullptr;
        if (slpa_on) {  // SLPA: memory slot it is read, slot it + 1 written
            a.lab_in = slpa_mem + (int64_t)it * nv;
            a.lab_out = slpa_mem + (int64_t)(it + 1) * nv;
            a.spoken = spoken;
        }
        a.changed = changed + (int64_t)it * G;
        a.key_t = stream_at(rs.p.seed, (uint64_t)t + 1);
        // the labels read in the first sweep from unique labels never give a
        // row a majority label
        a.majority = rs.p.init_labels || it >= 1;
        a.changed_prev = it > 0 ? changed + (int64_t)(it - 1) * G : nullptr;
        a.g_n = g_n;
        // many waves over small rows only (one graph, not captured): one
        // cooperative launch sweeps every wave with grid barriers between them
        if (!capturing && !rs.multi && waves >= COOP_MIN_WAVES && bl[0] > 0 &&
            bl[1] + bl[2] + bl[3] + bl[HUB_BUCKET] == 0) {
            if (!d_coop) {
                LP_TRY(dev_alloc(&d_coop, 4, "grid barrier", st, device));
                LP_CU(cudaMemsetAsync(d_coop, 0, 4 * sizeof(int32_t), s));
            }
            int64_t max_len = 0;
            for (int k = 0; k < waves; ++k) max_len = std::max(max_len, wcount[(size_t)k]);
            a.identity = rows_distinct && it == 0 && !rs.p.init_labels && !slpa_on;  // wave 0 only
            if (prof) {
                while (prof_ev.size() < 2 * (rs.prof_launch.size() + 1)) {
                    cudaEvent_t e;
                    LP_CU(cudaEventCreate(&e));
                    prof_ev.push_back(e);
                }
                LP_CU(cudaEventRecord(prof_ev[2 * rs.prof_launch.size()], s));
            }
            LP_CU(cudaMemsetAsync(d_coop, 0, 2 * sizeof(int32_t), s));
            a.rp = pk_rp;  // aligned with wlist; the kernel offsets it per wave
            const int nk = small_waves_launch(a, wlist, d_wstart0, d_wtot, max_len, max_deg,
                                              reinterpret_cast<unsigned *>(d_coop), d_coop + 2,
                                              num_sms, s);
            if (nk < 0) return fail(LP_ECUDA, cuda_msg("all-waves launch", cudaGetLastError()));
            *kernels += nk;
            rs.coop = true;
            if (prof) {
                LP_CU(cudaEventRecord(prof_ev[2 * rs.prof_launch.size() + 1], s));
                rs.prof_launch.push_back(0);
                rs.prof_len.push_back(bl[0]);
            }
            return LP_OK;
        }
        for (int launch_i = 0; launch_i < waves * NUM_BUCKETS; ++launch_i) {
            const int k = launch_i / NUM_BUCKETS, b = launch_i % NUM_BUCKETS;
            if (waves == 1) {
                a.list = list + bb[b];
                a.rp = pk_rp + bb[b];
                a.len = bl[b];
                a.htask = htask;
                a.hmulti = hmulti;
                a.hsegs = hsegs;
                a.hparts = hparts;
                a.hseg_task = hseg_task;
                a.hpart_task = hpart_task;
            } else {
                a.list = wlist + wstart[(size_t)b * waves + k];
                a.rp = pk_rp + wstart[(size_t)b * waves + k];
                a.len = wcount[(size_t)b * waves + k];
                if (b == HUB_BUCKET) {
                    a.htask = htask_w + (wstart[(size_t)b * waves + k] - wstart[(size_t)b * waves]);
                    a.hmulti = hmulti_w[(size_t)k];
                    a.hsegs = hsegs_w[(size_t)k];
                    a.hparts = hparts_w[(size_t)k];
                    if (hmulti_w[(size_t)k] > 0) {
                        a.hseg_task = hseg_task_w + hsegs_at_w[(size_t)k];
                        a.hpart_task = hpart_task_w + hparts_at_w[(size_t)k];
                    }
                }
            }
            if (a.len == 0) continue;
            // the first sweep from unique labels reads unique labels only in
            // its first wave (later waves see this sweep's new labels)
            a.identity = rows_distinct && it == 0 && !rs.p.init_labels && k == 0 && !slpa_on;
            if (prof) {
                while (prof_ev.size() < 2 * (rs.prof_launch.size() + 1)) {
                    cudaEvent_t e;
                    LP_CU(cudaEventCreate(&e));
                    prof_ev.push_back(e);
                }
                LP_CU(cudaEventRecord(prof_ev[2 * rs.prof_launch.size()], s));
            }
            const int nk = sweep_launch(b, a, rs.multi, num_sms, s);
            if (nk < 0) return fail(LP_ECUDA, cuda_msg("sweep launch", cudaGetLastError()));
            *kernels += nk;
            if (prof) {
                LP_CU(cudaEventRecord(prof_ev[2 * rs.prof_launch.size() + 1], s));
                rs.prof_launch.push_back(b);
                rs.prof_len.push_back(a.len);
            }
        }
        return LP_OK;
    }

    // launch one iteration and the read of its changed counters; ev_iter
    // marks its end
    lp_status run_launch()
    {
        Launches L;
        const int32_t it = rs.it;
        LP_TRY(launch_sweeps(st, it, rs.cur, rs.prof, &L.n));
        LP_CU(cudaMemcpyAsync(h_changed + (int64_t)it * G, changed + (int64_t)it * G,
                              (size_t)G * sizeof(int32_t), cudaMemcpyDeviceToHost, st));
        LP_CU(cudaEventRecord(ev_iter, st));
        rs.it = it + 1;
        return LP_OK;
    }

    // ------------------------------------------------------------------
    // A whole run as one CUDA graph: iteration i is a conditional (if) node
    // holding its sweeps and the device-side tolerance test, which arms
    // node i + 1 only while some graph goes on.  Built once per parameter
    // set and replayed; used whenever per-launch profiling is off.
    // ------------------------------------------------------------------
    struct GraphKey {
        double tolerance = -1.0;
        int32_t max_iter = 0, mode = -1, strict = -1, iter_offset = 0, waves = 0;
        uint64_t seed = 0;
        bool init = false, multi = false;
        bool operator==(const GraphKey &o) const
        {
            return tolerance == o.tolerance && max_iter == o.max_iter && mode == o.mode &&
                   strict == o.strict && iter_offset == o.iter_offset && waves == o.waves &&
                   seed == o.seed && init == o.init && multi == o.multi;
        }
    };
    GraphKey gr_key{};
    GraphKey gr_last{};  // parameters of the previous run

    GraphKey key_of(const lp_rak_params *p, bool multi) const
    {
        GraphKey k;
        k.tolerance = p->tolerance;
        k.max_iter = p->max_iter;
        k.mode = p->mode;
        k.strict = p->strict ? 1 : 0;
        k.iter_offset = p->iter_offset;
        k.waves = p->mode == LP_ASYNC ? std::min(p->waves, std::max(max_n, 1)) : 1;
        k.seed = p->seed;
        k.init = p->init_labels != nullptr;
        k.multi = multi;
        return k;
    }

    // true when this run repeats the previous run's parameters (or a run
    // graph for them exists)
    bool repeat_key(const lp_rak_params *p, bool multi)
    {
        if (!p) return false;
        const GraphKey k = key_of(p, multi);
        const bool rep = (gr_exec && k == gr_key) || k == gr_last;
        gr_last = k;
        return rep;
    }
    cudaGraph_t gr_graph = nullptr;
    cudaGraphExec_t gr_exec = nullptr;
    cudaStream_t gr_stream = nullptr;  // capture stream
    int64_t gr_kernels_per_iter = 0;
    int32_t *d_res = nullptr, *h_res = nullptr;  // iterations | converged | final | last (x2)

    RunResults run_results() const
    {
        RunResults r;
        r.iterations = d_res;
        r.converged = d_res + G;
        r.final_buf = d_res + 2 * (int64_t)G;
        r.last_changed = reinterpret_cast<long long *>(d_res + 4 * (int64_t)G);
        return r;
    }

    void drop_graph()
    {
        if (gr_exec) cudaGraphExecDestroy(gr_exec);
        if (gr_graph) cudaGraphDestroy(gr_graph);
        gr_exec = nullptr;
        gr_graph = nullptr;
        gr_key = GraphKey{};
    }

    lp_status ensure_graph()
    {
        const GraphKey k = key_of(&rs.p, rs.multi);
        if (gr_exec && k == gr_key) return LP_OK;
        drop_graph();
        if (!gr_stream) LP_CU(cudaStreamCreateWithFlags(&gr_stream, cudaStreamNonBlocking));
        if (!d_res) {
            LP_TRY(dev_alloc(&d_res, 6 * (int64_t)G, "run results", st, device));
            LP_TRY(host_alloc(&h_res, 6 * (int64_t)G, "run results"));
        }
        LP_CU(cudaGraphCreate(&gr_graph, 0));
        const int32_t n_it = rs.p.max_iter;
        std::vector<cudaGraphConditionalHandle> h((size_t)n_it);
        for (int32_t it = 0; it < n_it; ++it)
            LP_CU(cudaGraphConditionalHandleCreate(&h[(size_t)it], gr_graph, it == 0 ? 1u : 0u,
                                                   cudaGraphCondAssignDefault));
        const RunResults res = run_results();
        cudaGraphNode_t prev = nullptr;
        for (int32_t it = 0; it < n_it; ++it) {
            cudaGraphNodeParams cp{};
            cp.type = cudaGraphNodeTypeConditional;
            cp.conditional.handle = h[(size_t)it];
            cp.conditional.type = cudaGraphCondTypeIf;
            cp.conditional.size = 1;
            cudaGraphNode_t node;
            LP_CU(cudaGraphAddNode(&node, gr_graph, prev ? &prev : nullptr, nullptr, prev ? 1 : 0,
                                   &cp));
            cudaGraph_t body = cp.conditional.phGraph_out[0];
            LP_CU(cudaStreamBeginCaptureToGraph(gr_stream, body, nullptr, nullptr, 0,
                                                cudaStreamCaptureModeThreadLocal));
            int64_t nk = 0;
            lp_status ls = launch_sweeps(gr_stream, it, it & 1, false, &nk, true);
            if (ls == LP_OK &&
                converge_launch(changed + (int64_t)it * G, g_n, g_active, G, rs.p.tolerance, it,
                                rs.multi, res, it + 1 < n_it ? h[(size_t)it + 1] : h[0],
                                it + 1 < n_it, nullptr, false, gr_stream) != 0)
                ls = fail(LP_ECUDA, cuda_msg("convergence launch", cudaGetLastError()));
            cudaGraph_t captured = nullptr;
            const cudaError_t ce = cudaStreamEndCapture(gr_stream, &captured);
            if (ls != LP_OK) {
                drop_graph();
                return ls;
            }
            if (ce != cudaSuccess) {
                drop_graph();
                return fail(LP_ECUDA, cuda_msg("run capture", ce));
            }
            gr_kernels_per_iter = nk + 1;
            prev = node;
        }
        const cudaError_t ie = cudaGraphInstantiate(&gr_exec, gr_graph, 0);
        if (ie != cudaSuccess) {
            gr_exec = nullptr;
            drop_graph();
            return fail(LP_ECUDA, cuda_msg("run graph instantiation", ie));
        }
        gr_key = k;
        return LP_OK;
    }

    // Sec. 3.2's iteration over every graph of the set, launched as one graph
    lp_status run_graph(const lp_rak_params *p, bool multi)
    {
        LP_TRY(run_begin(p, multi));
        LP_TRY(ensure_graph());
        const size_t res_bytes = 6 * (size_t)G * sizeof(int32_t);
        LP_CU(cudaMemsetAsync(d_res, 0, res_bytes, st));
        LP_CU(cudaGraphLaunch(gr_exec, st));
        LP_CU(cudaMemcpyAsync(h_res, d_res, res_bytes, cudaMemcpyDeviceToHost, st));
        LP_CU(cudaMemcpyAsync(h_changed, changed, (size_t)rs.p.max_iter * G * sizeof(int32_t),
                              cudaMemcpyDeviceToHost, st));
        LP_CU(cudaEventRecord(ev_iter, st));
        LP_CU(cudaEventSynchronize(ev_iter));
        const long long *last = reinterpret_cast<const long long *>(h_res + 4 * (int64_t)G);
        int32_t ran = 0;
        rs.active_left = 0;
        for (int32_t g = 0; g < G; ++g) {
            lp_rak_result &r = results[(size_t)g];
            r.iterations = h_res[g];
            r.converged = h_res[G + g];
            r.last_changed = last[g];
            final_buf[(size_t)g] = h_res[2 * (int64_t)G + g];
            ran = std::max(ran, r.iterations);
            if (!r.converged) ++rs.active_left;
        }
        rs.it = ran;
        rs.cur = ran & 1;
        g_launches += (int64_t)ran * gr_kernels_per_iter;
        return run_end();
    }

    // a6 after the launched iteration has finished on the device
    lp_status run_finish()
    {
        const int32_t it = rs.it - 1;
        rs.cur ^= 1;
        bool deactivated = false;
        for (int32_t g = 0; g < G; ++g) {
            if (rs.multi && !h_active[g]) continue;
            const int64_t c = h_changed[(int64_t)it * G + g];
            lp_rak_result &r = results[(size_t)g];
            r.iterations = it + 1;
            r.last_changed = c;
            final_buf[(size_t)g] = rs.cur;
            // Sec. 3.2: converged when at most tolerance * n vertices changed
            if ((double)c <= rs.p.tolerance * (double)h_n[(size_t)g]) {
                r.converged = 1;
                if (rs.multi) {
                    h_active[g] = 0;
                    deactivated = true;
                }
                --rs.active_left;
            }
        }
        if (rs.multi && deactivated && rs.active_left > 0)
            LP_CU(cudaMemcpyAsync(g_active, h_active, (size_t)G * sizeof(int32_t),
                                  cudaMemcpyHostToDevice, st));
        return LP_OK;
    }

    lp_status run_end()
    {
        LP_CU(cudaEventRecord(ev1, st));
        LP_CU(cudaEventSynchronize(ev1));
        if (rs.coop) {
            int32_t err = 0;
            LP_CU(cudaMemcpy(&err, d_coop + 2, sizeof(int32_t), cudaMemcpyDeviceToHost));
            if (err) {
                LP_CU(cudaMemset(d_coop, 0, 4 * sizeof(int32_t)));
                return fail(LP_ECUDA, "a grid barrier of the all-waves sweep timed out");
            }
        }
        float ms = 0.f;
        LP_CU(cudaEventElapsedTime(&ms, ev0, ev1));
        for (auto &r : results) r.gpu_ms = ms;
        if (rs.prof && !rs.prof_launch.empty()) {
            std::lock_guard<std::mutex> lock(g_prof_mu);
            for (size_t i = 0; i < rs.prof_launch.size(); ++i) {
                if (i < rs.prof_iter.size() && rs.prof_iter[i] >= rs.it) continue;
                float kms = 0.f;
                LP_CU(cudaEventElapsedTime(&kms, prof_ev[2 * i], prof_ev[2 * i + 1]));
                const int b = rs.prof_launch[i];
                KernelStat &k = g_prof[b];
                k.launches += 1;
                k.ms += kms;
                const double verts = (double)rs.prof_len[i];
                // entries of a wave launch: its share of the bucket's entries
                const double ents = bl[b] ? (double)be[b] * verts / (double)bl[b] : 0.0;
                k.vertices += verts;
                k.entries += ents;
                // algorithmic HBM bytes: row pointer, own label and label write
                // per vertex; column index (and weight) per entry
                k.bytes += 12.0 * verts + (wts ? 8.0 : 4.0) * ents;
            }
        }
        history.assign((size_t)results[0].iterations, 0);
        for (int32_t i = 0; i < results[0].iterations; ++i) history[i] = h_changed[(int64_t)i * G];
        if (rs.multi) LP_TRY(gather_final_labels());
        return LP_OK;
    }

    // whether a run with these parameters sweeps every wave of an iteration in
    // one cooperative launch (a single graph, many waves, small rows only),
    // which a captured run graph cannot hold: the graph would launch every
    // wave on its own (measured 25 % slower on 127 waves of k-mer paths)
    bool all_waves_run(const lp_rak_params *p, bool multi) const
    {
        if (!p || multi || p->mode != LP_ASYNC) return false;
        const int32_t waves = std::min(p->waves, std::max(max_n, 1));
        return waves >= COOP_MIN_WAVES && bl[0] > 0 &&
               bl[1] + bl[2] + bl[3] + bl[HUB_BUCKET] == 0;
    }

    // Sec. 3.2 iteration over every graph of the set, to the end: one graph
    // launch, or (while per-launch profiling is on, or for all-waves runs)
    // launches from the host
    lp_status run(const lp_rak_params *p, bool multi)
    {
        // capturing a run costs about as much as a run of a mid-size graph, so
        // a graph is captured once the same parameters come back
        if (!g_prof_on.load() && !all_waves_run(p, multi) && repeat_key(p, multi))
            return run_graph(p, multi);
        return run_host(p, multi);
    }

    // Sec. 3.2's iteration launched from the host without waiting for each
    // iteration: the tolerance test runs on the device after every iteration
    // and raises a stop flag once the run is over; the host checks the flag
    // of the iteration RUN_LAG (or one, on large graphs) before the one it has
    // just launched, so that iterations launched past the end (at most
    // RUN_LAG) return at once.
    static constexpr int RUN_LAG = 2;
    static constexpr int64_t LAG1_ENTRIES = (int64_t)1 << 25;
    int32_t *d_stop = nullptr, *h_stop = nullptr;
    int32_t h_stop_cap = 0;
    cudaEvent_t run_ev[RUN_LAG + 1] = {};

    lp_status run_host(const lp_rak_params *p, bool multi)
    {
        LP_TRY(run_begin(p, multi));
        if (!d_stop) LP_TRY(dev_alloc(&d_stop, 1, "stop flag", st, device));
        if (h_stop_cap < rs.p.max_iter) {
            if (h_stop) host_free(h_stop);
            h_stop = nullptr;
            h_stop_cap = 0;
            LP_TRY(host_alloc(&h_stop, rs.p.max_iter, "stop flags"));
            h_stop_cap = rs.p.max_iter;
        }
        if (!d_res) {
            LP_TRY(dev_alloc(&d_res, 6 * (int64_t)G, "run results", st, device));
            LP_TRY(host_alloc(&h_res, 6 * (int64_t)G, "run results"));
        }
        for (cudaEvent_t &e : run_ev)
            if (!e) LP_CU(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
        const size_t res_bytes = 6 * (size_t)G * sizeof(int32_t);
        LP_CU(cudaMemsetAsync(d_stop, 0, sizeof(int32_t), st));
        LP_CU(cudaMemsetAsync(d_res, 0, res_bytes, st));
        rs.a.stop = d_stop;
        const RunResults res = run_results();
        for (int32_t it = 0; it < rs.p.max_iter; ++it) {
            Launches L;
            LP_TRY(launch_sweeps(st, it, it & 1, rs.prof, &L.n));
            while (rs.prof_iter.size() < rs.prof_launch.size()) rs.prof_iter.push_back(it);
            if (converge_launch(changed + (int64_t)it * G, g_n, g_active, G, rs.p.tolerance, it,
                                rs.multi, res, 0, false, d_stop, it + 1 == rs.p.max_iter,
                                st) != 0)
                return fail(LP_ECUDA, cuda_msg("convergence launch", cudaGetLastError()));
            ++L.n;
            LP_CU(cudaMemcpyAsync(h_stop + it, d_stop, sizeof(int32_t), cudaMemcpyDeviceToHost,
                                  st));
            LP_CU(cudaEventRecord(run_ev[it % (RUN_LAG + 1)], st));
            // one iteration back when an iteration outlasts the host's
            // launches of the next (a graph of at least LAG1_ENTRIES entries,
            // or one all-waves launch per iteration): one fewer iteration is
            // launched past the end
            const int lag = (rs.coop || ne >= LAG1_ENTRIES) ? 1 : RUN_LAG;
            if (it >= lag) {
                LP_CU(cudaEventSynchronize(run_ev[(it - lag) % (RUN_LAG + 1)]));
                if (h_stop[it - lag]) break;
            }
        }
        LP_CU(cudaMemcpyAsync(h_res, d_res, res_bytes, cudaMemcpyDeviceToHost, st));
        LP_CU(cudaMemcpyAsync(h_changed, changed, (size_t)rs.p.max_iter * G * sizeof(int32_t),
                              cudaMemcpyDeviceToHost, st));
        LP_CU(cudaEventRecord(ev_iter, st));
        LP_CU(cudaEventSynchronize(ev_iter));
        const long long *last = reinterpret_cast<const long long *>(h_res + 4 * (int64_t)G);
        int32_t ran = 0;
        rs.active_left = 0;
        for (int32_t g = 0; g < G; ++g) {
            lp_rak_result &r = results[(size_t)g];
            r.iterations = h_res[g];
            r.converged = h_res[G + g];
            r.last_changed = last[g];
            final_buf[(size_t)g] = h_res[2 * (int64_t)G + g];
            ran = std::max(ran, r.iterations);
            if (!r.converged) ++rs.active_left;
        }
        rs.it = ran;
        rs.cur = ran & 1;
        return run_end();
    }

    // SLPA (Sec. 3.4) on a single graph: iteration t (1 <= t < memory_size)
    // speaks one label per entry from the memories of the previous slots and
    // runs one synchronous RAK sweep over the spoken labels into slot t; the
    // tolerance test counts vertices whose new slot differs from the previous
    // one.  The graph's labels become the communities (the label a memory
    // holds most often).
    lp_status slpa(const lp_slpa_params *p)
    {
        if (!p) return fail(LP_EINVAL, "params is NULL");
        if (p->memory_size < 1 || p->memory_size > SLPA_MAX_MEMORY)
            return fail(LP_EINVAL, "memory_size must lie in [1, 64]");
        if (!(p->tolerance >= 0.0 && p->tolerance <= 1.0))
            return fail(LP_EINVAL, "tolerance must lie in [0, 1]");
        if (G != 1) return fail(LP_EINVAL, "SLPA runs on single graphs");
        const int32_t M = p->memory_size;
        lp_rak_params q{};
        lp_rak_params_default(&q);
        q.mode = LP_SYNC;
        q.strict = p->strict ? 1 : 0;
        q.seed = p->seed;
        q.tolerance = p->tolerance;
        q.max_iter = M > 1 ? M - 1 : 1;
        q.iter_offset = 1;  // the tie key of slot t uses t
        q.init_labels = nullptr;
        if (slpa_slots < M) {
            if (slpa_mem) cudaFreeAsync(slpa_mem, st);
            slpa_mem = nullptr;
            slpa_slots = 0;
            LP_TRY(dev_alloc(&slpa_mem, (int64_t)M * nv, "SLPA memory", st, device));
            slpa_slots = M;
        }
        if (!spoken) LP_TRY(dev_alloc(&spoken, ne, "SLPA spoken labels", st, device));
        LP_TRY(run_begin(&q, false));
        rs.prof = false;
        Launches L;
        if (nv > 0)
            LP_CU(cudaMemcpyAsync(slpa_mem, lab[0], (size_t)nv * sizeof(int32_t),
                                  cudaMemcpyDeviceToDevice, st));  // slot 0: the vertex itself
        int32_t iters = 0, conv = 0;
        int64_t last = 0;
        history.clear();
        slpa_on = true;
        lp_status ls = LP_OK;
        for (int32_t t = 1; t < M && ls == LP_OK; ++t) {
            const int32_t it = t - 1;
            // a vertex without edges repeats its previous slot
            cudaError_t e = cudaMemcpyAsync(slpa_mem + (int64_t)t * nv, slpa_mem + (int64_t)it * nv,
                                            (size_t)nv * sizeof(int32_t), cudaMemcpyDeviceToDevice,
                                            st);
            if (e != cudaSuccess) {
                ls = fail(LP_ECUDA, cuda_msg("SLPA slot copy", e));
                break;
            }
            if (slpa_speak(pk_rp, list, pk_first, ne, pk_idx, slpa_mem, nv, t, p->seed, spoken, st,
                           &L.n) != 0) {
                ls = fail(LP_ECUDA, cuda_msg("SLPA speak launch", cudaGetLastError()));
                break;
            }
            if ((ls = launch_sweeps(st, it, 0, false, &L.n)) != LP_OK) break;
            e = cudaMemcpyAsync(h_changed + it, changed + it, sizeof(int32_t),
                                cudaMemcpyDeviceToHost, st);
            if (e == cudaSuccess) e = cudaStreamSynchronize(st);
            if (e != cudaSuccess) {
                ls = fail(LP_ECUDA, cuda_msg("SLPA changed count", e));
                break;
            }
            iters = t;
            last = h_changed[it];
            history.push_back(last);
            if ((double)last <= p->tolerance * (double)nv) {  // Sec. 3.2's tolerance test
                conv = 1;
                break;
            }
        }
        slpa_on = false;
        LP_TRY(ls);
        slpa_filled = iters + 1;
        if (slpa_community(slpa_mem, nv, iters, lab[0], st, &L.n) != 0)
            return fail(LP_ECUDA, cuda_msg("SLPA community launch", cudaGetLastError()));
        LP_CU(cudaEventRecord(ev1, st));
        LP_CU(cudaEventSynchronize(ev1));
        float ms = 0.f;
        LP_CU(cudaEventElapsedTime(&ms, ev0, ev1));
        std::fill(final_buf.begin(), final_buf.end(), 0);
        q_valid = false;
        results[0] = lp_rak_result{iters, conv, last, ms};
        rs.it = iters;
        rs.active_left = 0;
        return LP_OK;
    }

    // COPRA (Sec. 3.3) on a single graph: every vertex starts as its own
    // community; each iteration (in waves when asynchronous) computes every
    // vertex's set from its neighbours' sets; the tolerance test counts the
    // vertices whose best label changed.  The graph's labels become the best
    // labels.
    lp_status copra(const lp_copra_params *p)
    {
        if (!p) return fail(LP_EINVAL, "params is NULL");
        if (p->max_labels < 1 || p->max_labels > 64)
            return fail(LP_EINVAL, "max_labels must lie in [1, 64]");
        if (!(p->tolerance >= 0.0 && p->tolerance <= 1.0))
            return fail(LP_EINVAL, "tolerance must lie in [0, 1]");
        if (p->max_iter < 1) return fail(LP_EINVAL, "max_iter must be >= 1");
        if (p->mode != LP_SYNC && p->mode != LP_ASYNC)
            return fail(LP_EINVAL, "mode must be LP_SYNC or LP_ASYNC");
        if (p->mode == LP_ASYNC && p->waves < 1) return fail(LP_EINVAL, "waves must be >= 1");
        if (G != 1) return fail(LP_EINVAL, "COPRA runs on single graphs");
        const int32_t L = p->max_labels;
        const int32_t waves = p->mode == LP_ASYNC ? std::min(p->waves, std::max(nv, 1)) : 1;
        const int glg = copra_table_lg(max_deg, L);
        if (glg > 28) return fail(LP_EINVAL, "a row holds too many labels for max_labels");
        if (copra_cap < L) {
            for (int b = 0; b < 2; ++b) {
                if (cset_l[b]) cudaFreeAsync(cset_l[b], st);
                if (cset_b[b]) cudaFreeAsync(cset_b[b], st);
                cset_l[b] = nullptr;
                cset_b[b] = nullptr;
            }
            copra_cap = 0;
            for (int b = 0; b < 2; ++b) {
                LP_TRY(dev_alloc(&cset_l[b], (int64_t)nv * L, "COPRA sets", st, device));
                LP_TRY(dev_alloc(&cset_b[b], (int64_t)nv * L, "COPRA sets", st, device));
            }
            copra_cap = L;
        }
        if (glg > ctab_lg) {
            if (ctab_key) cudaFreeAsync(ctab_key, st);
            if (ctab_sum) cudaFreeAsync(ctab_sum, st);
            if (ctab_first) cudaFreeAsync(ctab_first, st);
            ctab_key = nullptr;
            ctab_sum = ctab_first = nullptr;
            ctab_lg = 0;
            const int64_t slots = (int64_t)copra_big_ctas() << glg;
            LP_TRY(dev_alloc(&ctab_key, slots, "COPRA long-row tables", st, device));
            LP_TRY(dev_alloc(&ctab_sum, slots, "COPRA long-row tables", st, device));
            LP_TRY(dev_alloc(&ctab_first, slots, "COPRA long-row tables", st, device));
            LP_CU(cudaMemsetAsync(ctab_key, 0xFF, (size_t)slots * sizeof(int32_t), st));
            LP_CU(cudaMemsetAsync(ctab_sum, 0, (size_t)slots * sizeof(unsigned long long), st));
            LP_CU(cudaMemsetAsync(ctab_first, 0xFF, (size_t)slots * sizeof(unsigned long long),
                                  st));
            ctab_lg = glg;
        }
        LP_TRY(ensure_changed(p->max_iter));
        // the rows that take a CTA, by kind and wave
        const int64_t nbins = copra_bins(waves);
        if (!crows) LP_TRY(dev_alloc(&crows, std::max(nv, 1), "COPRA row lists", st, device));
        if (!covf) LP_TRY(dev_alloc(&covf, (int64_t)nv + 1, "COPRA row lists", st, device));
        if (cbins_cap < nbins) {
            if (cbins) cudaFreeAsync(cbins, st);
            cbins = nullptr;
            cbins_cap = 0;
            LP_TRY(dev_alloc(&cbins, nbins, "COPRA row lists", st, device));
            cbins_cap = nbins;
        }
        h_cbins.resize((size_t)nbins);
        h_cstart.resize((size_t)nbins + 1);
        Launches L0;
        if (copra_rows(off, nv, L, waves, cbins, h_cbins.data(), h_cstart.data(), crows, st,
                       &L0.n) != 0)
            return fail(LP_ECUDA, cuda_msg("COPRA row lists", cudaGetLastError()));
        LP_CU(cudaMemsetAsync(changed, 0, (size_t)p->max_iter * sizeof(int32_t), st));
        LP_CU(cudaEventRecord(ev0, st));
        if (copra_init(cset_l[0], cset_b[0], nv, L, st, &L0.n) != 0)
            return fail(LP_ECUDA, cuda_msg("COPRA init", cudaGetLastError()));
        int cur = 0;
        int32_t iters = 0, conv = 0;
        int64_t last = 0;
        history.clear();
        for (int32_t it = 0; it < p->max_iter; ++it) {
            CopraStep cs{};
            cs.off = off;
            cs.idx = idx;
            cs.wts = wts;
            cs.n = nv;
            cs.L = L;
            cs.cur_l = cset_l[cur];
            cs.cur_b = cset_b[cur];
            cs.nxt_l = cset_l[cur ^ 1];
            cs.nxt_b = cset_b[cur ^ 1];
            cs.waves = waves;
            cs.strict = p->strict ? 1 : 0;
            cs.key_t = stream_at(p->seed, (uint64_t)it + 1);  // the tie key of iteration it
            cs.changed = changed + it;
            cs.gkey = ctab_key;
            cs.gsum = ctab_sum;
            cs.gfirst = ctab_first;
            cs.glg_max = glg;
            for (int32_t k = 0; k < waves; ++k) {
                cs.wave_k = k;
                auto bin = [&](int kind) { return (size_t)kind * waves + k; };
                cs.rows_warp = crows + h_cstart[bin(0)];
                cs.n_warp = h_cstart[bin(0) + 1] - h_cstart[bin(0)];
                cs.rows_cta = crows + h_cstart[bin(1)];
                cs.n_cta = h_cstart[bin(1) + 1] - h_cstart[bin(1)];
                cs.rows_big = crows + h_cstart[bin(2)];
                cs.n_big = h_cstart[bin(2) + 1] - h_cstart[bin(2)];
                cs.ovf = covf;
                if (copra_step(cs, num_sms, st, &L0.n) != 0)
                    return fail(LP_ECUDA, cuda_msg("COPRA launch", cudaGetLastError()));
            }
            cur ^= 1;
            LP_CU(cudaMemcpyAsync(h_changed + it, changed + it, sizeof(int32_t),
                                  cudaMemcpyDeviceToHost, st));
            LP_CU(cudaStreamSynchronize(st));
            iters = it + 1;
            last = h_changed[it];
            history.push_back(last);
            if ((double)last <= p->tolerance * (double)nv) {  // the RAK-style test
                conv = 1;
                break;
            }
        }
        copra_L = L;
        copra_cur = cur;
        if (copra_best(cset_l[cur], nv, L, lab[0], st, &L0.n) != 0)
            return fail(LP_ECUDA, cuda_msg("COPRA labels", cudaGetLastError()));
        LP_CU(cudaEventRecord(ev1, st));
        LP_CU(cudaEventSynchronize(ev1));
        float ms = 0.f;
        LP_CU(cudaEventElapsedTime(&ms, ev0, ev1));
        std::fill(final_buf.begin(), final_buf.end(), 0);
        q_valid = false;
        results[0] = lp_rak_result{iters, conv, last, ms};
        return LP_OK;
    }

    // Graphs of a batch stop in different iterations, so their final labels
    // sit in either buffer; copy them all into buffer 0.
    lp_status gather_final_labels()
    {
        bool any = false;
        for (int f : final_buf) any = any || f != 0;
        if (!any) return LP_OK;
        if (!g_sel) LP_TRY(dev_alloc(&g_sel, G, "graph buffer selector", st, device));
        std::vector<int32_t> sel(final_buf.begin(), final_buf.end());
        LP_CU(cudaMemcpyAsync(g_sel, sel.data(), (size_t)G * sizeof(int32_t),
                              cudaMemcpyHostToDevice, st));
        Launches L;
        if (merge_final_labels(lab[0], lab[1], nv, vgraph, g_sel, st, &L.n) != 0)
            return fail(LP_ECUDA, cuda_msg("label merge", cudaGetLastError()));
        LP_CU(cudaStreamSynchronize(st));  // sel lives on the host stack
        std::fill(final_buf.begin(), final_buf.end(), 0);
        return LP_OK;
    }

    // Modularity of every graph under `labels` (nv device labels, valid),
    // into q_cache.
    lp_status modularity_all(const int32_t *labels)
    {
        if (nv > kc_cap) {
            if (kc) cudaFreeAsync(kc, st);
            kc = nullptr;
            kc_cap = 0;
            LP_TRY(dev_alloc(&kc, nv, "community weights", st, device));
            kc_cap = nv;
        }
        if (!macc) {
            LP_TRY(dev_alloc(&macc, 4 * (int64_t)G, "modularity accumulators", st, device));
            LP_TRY(host_alloc(&h_macc, 4 * (int64_t)G, "modularity accumulators"));
        }
        Launches L;
        if (nv > 0) LP_CU(cudaMemsetAsync(kc, 0, (size_t)nv * sizeof(unsigned long long), st));
        LP_CU(cudaMemsetAsync(macc, 0, 4 * (size_t)G * sizeof(unsigned long long), st));
        // the entry pass reads the packed rows (those of the last run, or the
        // bucket list's when no run has packed them yet)
        LP_TRY(ensure_packed(pk_waves > 0 ? pk_waves : 1));
        ModArgs ma{};
        ma.rp = pk_rp;
        ma.idx = pk_idx;
        ma.wts = wts ? pk_wts : nullptr;
        ma.lab = labels;
        ma.list = pk_waves > 1 ? wlist : list;
        ma.len = bb[HUB_BUCKET] + bl[HUB_BUCKET];
        ma.ne = ne;
        ma.first_row = pk_first;
        ma.ncopy = pack_chunks(ne);
        ma.nsmall = bl[0];  // the small bucket leads the list (and so the packed rows)
        ma.e_lo = be[0];
        ma.vgraph = vgraph;
        ma.g_vbase = g_vbase;
        ma.kc = kc;
        ma.acc = macc;
        if (modularity_launch(ma, nv, vgraph != nullptr, st, &L.n) != 0)
            return fail(LP_ECUDA, cuda_msg("modularity launch", cudaGetLastError()));
        LP_CU(cudaMemcpyAsync(h_macc, macc, 4 * (size_t)G * sizeof(unsigned long long),
                              cudaMemcpyDeviceToHost, st));
        LP_CU(cudaStreamSynchronize(st));
        q_cache.assign((size_t)G, 0.0);
        for (int32_t g = 0; g < G; ++g) {
            const unsigned long long *acc = h_macc + 4 * (size_t)g;
            const unsigned long long l_in = acc[0], two_m = acc[1];
            const unsigned __int128 s2 = ((unsigned __int128)acc[2] << 64) | acc[3];
            if (two_m == 0) continue;  // no entries: Q = 0
            const double dm = (double)two_m;
            q_cache[(size_t)g] = (double)l_in / dm - (double)s2 / (dm * dm);
        }
        return LP_OK;
    }

    // copy `n` labels of graph g, starting at vertex base vb, to dst
    lp_status copy_labels(int32_t g, int32_t *dst, int32_t on_device)
    {
        const int32_t n = h_n[(size_t)g];
        if (n == 0) return LP_OK;
        LP_CU(cudaMemcpyAsync(dst, lab[final_buf[(size_t)g]] + h_vbase[(size_t)g],
                              (size_t)n * sizeof(int32_t),
                              on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, st));
        LP_CU(cudaStreamSynchronize(st));
        return LP_OK;
    }
};

lp_status lp_fail(lp_status s, const std::string &msg) { return fail(s, msg); }

}  // namespace lp

struct lp_graph;
namespace lp {
// Stepwise iteration of one graph, for the serving loop (lp_serve.cu).
lp_status graph_run_begin(lp_graph *g, const lp_rak_params *p);
bool graph_run_done(lp_graph *g);
lp_status graph_run_launch(lp_graph *g, cudaEvent_t *done_event);
lp_status graph_run_finish(lp_graph *g);
lp_status graph_run_end(lp_graph *g, lp_rak_result *r);
// The same for every graph of a batch at once (converged graphs are left out
// of later iterations on the device; per_graph receives count results).
lp_status batch_run_begin(lp_batch *b, const lp_rak_params *p);
bool batch_run_done(lp_batch *b);
lp_status batch_run_launch(lp_batch *b, cudaEvent_t *done_event);
lp_status batch_run_finish(lp_batch *b);
lp_status batch_run_end(lp_batch *b, lp_rak_result *per_graph);
int32_t batch_run_active(lp_batch *b);  // graphs still iterating

void lp_add_launches(int64_t n) { g_launches += n; }

}  // namespace lp

struct lp_graph {
    lp::GraphSet s;
};

struct lp_batch {
    lp::GraphSet s;
};

namespace lp {
lp_status graph_run_begin(lp_graph *g, const lp_rak_params *p)
{
    DeviceGuard dg(g->s.device);
    return g->s.run_begin(p, false);
}
bool graph_run_done(lp_graph *g) { return g->s.run_done(); }
lp_status graph_run_launch(lp_graph *g, cudaEvent_t *done_event)
{
    DeviceGuard dg(g->s.device);
    LP_TRY(g->s.run_launch());
    *done_event = g->s.ev_iter;
    return LP_OK;
}
lp_status graph_run_finish(lp_graph *g) { return g->s.run_finish(); }
lp_status graph_run_end(lp_graph *g, lp_rak_result *r)
{
    DeviceGuard dg(g->s.device);
    LP_TRY(g->s.run_end());
    *r = g->s.results[0];
    return LP_OK;
}
lp_status batch_run_begin(lp_batch *b, const lp_rak_params *p)
{
    DeviceGuard dg(b->s.device);
    return b->s.run_begin(p, true);
}
bool batch_run_done(lp_batch *b) { return b->s.run_done(); }
int32_t batch_run_active(lp_batch *b) { return b->s.rs.active_left; }
lp_status batch_run_launch(lp_batch *b, cudaEvent_t *done_event)
{
    DeviceGuard dg(b->s.device);
    LP_TRY(b->s.run_launch());
    *done_event = b->s.ev_iter;
    return LP_OK;
}
lp_status batch_run_finish(lp_batch *b)
{
    DeviceGuard dg(b->s.device);
    return b->s.run_finish();
}
lp_status batch_run_end(lp_batch *b, lp_rak_result *per_graph)
{
    DeviceGuard dg(b->s.device);
    LP_TRY(b->s.run_end());
    for (int32_t i = 0; i < b->s.G; ++i) per_graph[i] = b->s.results[(size_t)i];
    return LP_OK;
}
}  // namespace lp

// ----------------------------------------------------------------------------
// Entry points
// ----------------------------------------------------------------------------
extern "C" {

lp_status lp_rak_params_default(lp_rak_params *p)
{
    if (!p) return fail(LP_EINVAL, "params is NULL");
    p->tolerance = 0.05;
    p->max_iter = 20;
    p->mode = LP_SYNC;
    p->strict = 1;
    p->iter_offset = 0;
    p->seed = 0;
    p->init_labels = nullptr;
    p->init_labels_on_device = 0;
    p->waves = 31;
    return LP_OK;
}

lp_status lp_graph_create(int32_t n, int64_t m, const int32_t *offsets, const int32_t *indices,
                          const int32_t *weights, uint32_t flags, void *cuda_stream,
                          lp_graph **out)
{
    if (!out) return fail(LP_EINVAL, "out is NULL");
    *out = nullptr;
    if (n < 0) return fail(LP_EINVAL, "n must be >= 0");
    if (m < 0 || m > 2147483647LL) return fail(LP_EINVAL, "m must lie in [0, 2^31)");
    if (!offsets) return fail(LP_EINVAL, "offsets is NULL");
    if (m > 0 && !indices) return fail(LP_EINVAL, "indices is NULL");
    if ((flags & LP_FLAG_BORROW) && !(flags & LP_FLAG_DEVICE_PTRS))
        return fail(LP_EINVAL, "LP_FLAG_BORROW needs LP_FLAG_DEVICE_PTRS");
    if (flags & ~(uint32_t)(LP_FLAG_DEVICE_PTRS | LP_FLAG_CHECK_SYMMETRIC | LP_FLAG_BORROW))
        return fail(LP_EINVAL, "unknown flag bits");
    std::unique_ptr<lp_graph> g(new (std::nothrow) lp_graph);
    if (!g) return fail(LP_ENOMEM, "host allocation failed");
    lp::GraphSet &s = g->s;
    LP_TRY(s.begin(cuda_stream));
    const bool dev = flags & LP_FLAG_DEVICE_PTRS;
    const cudaMemcpyKind kind = dev ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    s.G = 1;
    s.nv = n;
    s.ne = m;
    s.h_n = {n};
    s.h_m = {m};
    s.h_vbase = {0};
    s.h_ebase = {0};
    s.max_n = n;
    // the sweep reads indices and weights in aligned 16-byte blocks: borrow
    // them only when they start on a 16-byte boundary, otherwise copy
    auto aligned16 = [](const void *p) { return ((uintptr_t)p & 15u) == 0; };
    const bool borrow = (flags & LP_FLAG_BORROW) && aligned16(indices) && aligned16(weights);
    if (borrow) {
        s.off = const_cast<int32_t *>(offsets);
        s.idx = const_cast<int32_t *>(indices);
        s.wts = const_cast<int32_t *>(weights);
        s.own_off = s.own_idx = s.own_wts = false;
    } else {
        LP_TRY(dev_alloc(&s.off, (int64_t)n + 1, "offsets", s.st, s.device));
        LP_TRY(dev_alloc(&s.idx, m, "indices", s.st, s.device));
        LP_CU(cudaMemcpyAsync(s.off, offsets, ((size_t)n + 1) * sizeof(int32_t), kind, s.st));
        if (m > 0) LP_CU(cudaMemcpyAsync(s.idx, indices, (size_t)m * sizeof(int32_t), kind, s.st));
        if (weights) {
            LP_TRY(dev_alloc(&s.wts, m, "weights", s.st, s.device));
            if (m > 0)
                LP_CU(cudaMemcpyAsync(s.wts, weights, (size_t)m * sizeof(int32_t), kind, s.st));
        }
    }
    if (((uintptr_t)s.idx & 15u) || ((uintptr_t)s.wts & 15u))
        return fail(LP_ECUDA, "device allocation is not 16-byte aligned");
    LP_TRY(dev_alloc(&s.g_n, 1, "graph sizes", s.st, s.device));
    LP_CU(cudaMemcpyAsync(s.g_n, &n, sizeof(int32_t), cudaMemcpyHostToDevice, s.st));
    // a1: validation keeps every later kernel in bounds
    LP_TRY(s.validate_single(n, m));
    if (flags & LP_FLAG_CHECK_SYMMETRIC) {
        std::vector<int32_t> ho((size_t)n + 1), hi((size_t)m), hw(weights ? (size_t)m : 0);
        LP_CU(cudaMemcpy(ho.data(), s.off, ho.size() * sizeof(int32_t), cudaMemcpyDeviceToHost));
        if (m > 0)
            LP_CU(cudaMemcpy(hi.data(), s.idx, hi.size() * sizeof(int32_t), cudaMemcpyDeviceToHost));
        if (weights && m > 0)
            LP_CU(cudaMemcpy(hw.data(), s.wts, hw.size() * sizeof(int32_t), cudaMemcpyDeviceToHost));
        if (!host_symmetric(n, ho.data(), hi.data(), weights ? hw.data() : nullptr))
            return fail(LP_EINVAL, "CSR is not symmetric");
    }
    LP_TRY(s.bucket());
    LP_TRY(s.alloc_labels());
    LP_CU(cudaStreamSynchronize(s.st));
    *out = g.release();
    return LP_OK;
}

lp_status lp_graph_autotune(lp_graph *g, const lp_rak_params *p, int32_t sweeps,
                            lp_tune_result *out)
{
    if (!g) return fail(LP_EINVAL, "graph is NULL");
    DeviceGuard dg(g->s.device);
    return g->s.autotune(p, false, sweeps, out);
}

lp_status lp_graph_destroy(lp_graph *g)
{
    if (!g) return LP_OK;
    DeviceGuard dg(g->s.device);
    delete g;
    return LP_OK;
}

lp_status lp_graph_info(const lp_graph *g, int32_t *n, int64_t *m)
{
    if (!g) return fail(LP_EINVAL, "graph is NULL");
    if (n) *n = g->s.nv;
    if (m) *m = g->s.ne;
    return LP_OK;
}

lp_status lp_rak_run(lp_graph *g, const lp_rak_params *p, lp_rak_result *out)
{
    if (!g) return fail(LP_EINVAL, "graph is NULL");
    if (!out) return fail(LP_EINVAL, "result is NULL");
    DeviceGuard dg(g->s.device);
    LP_TRY(g->s.run(p, false));
    *out = g->s.results[0];
    return LP_OK;
}

lp_status lp_copra_params_default(lp_copra_params *p)
{
    if (!p) return fail(LP_EINVAL, "params is NULL");
    p->max_labels = 4;
    p->tolerance = 0.01;
    p->max_iter = 20;
    p->mode = LP_ASYNC;
    p->waves = 31;
    p->strict = 1;
    p->seed = 0;
    return LP_OK;
}

lp_status lp_copra_run(lp_graph *g, const lp_copra_params *p, lp_rak_result *out)
{
    if (!g) return fail(LP_EINVAL, "graph is NULL");
    if (!out) return fail(LP_EINVAL, "result is NULL");
    DeviceGuard dg(g->s.device);
    LP_TRY(g->s.copra(p));
    *out = g->s.results[0];
    return LP_OK;
}

lp_status lp_copra_sets_get(lp_graph *g, int32_t *labels, uint32_t *belongings,
                            int32_t dst_on_device)
{
    if (!g) return fail(LP_EINVAL, "graph is NULL");
    lp::GraphSet &s = g->s;
    if (s.copra_L == 0) return fail(LP_EINVAL, "no COPRA run on this graph");
    if ((!labels || !belongings) && s.nv > 0) return fail(LP_EINVAL, "labels or belongings is NULL");
    if (s.nv == 0) return LP_OK;
    DeviceGuard dg(s.device);
    const size_t cells = (size_t)s.nv * s.copra_L;
    const cudaMemcpyKind kind = dst_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    LP_CU(cudaMemcpyAsync(labels, s.cset_l[s.copra_cur], cells * sizeof(int32_t), kind, s.st));
    LP_CU(cudaMemcpyAsync(belongings, s.cset_b[s.copra_cur], cells * sizeof(uint32_t), kind, s.st));
    LP_CU(cudaStreamSynchronize(s.st));
    return LP_OK;
}

lp_status lp_slpa_params_default(lp_slpa_params *p)
{
    if (!p) return fail(LP_EINVAL, "params is NULL");
    p->memory_size = 20;
    p->tolerance = 0.05;
    p->strict = 1;
    p->seed = 0;
    return LP_OK;
}

lp_status lp_slpa_run(lp_graph *g, const lp_slpa_params *p, lp_rak_result *out)
{
    if (!g) return fail(LP_EINVAL, "graph is NULL");
    if (!out) return fail(LP_EINVAL, "result is NULL");
    DeviceGuard dg(g->s.device);
    LP_TRY(g->s.slpa(p));
    *out = g->s.results[0];
    return LP_OK;
}

lp_status lp_slpa_memory_get(lp_graph *g, int32_t *dst, int32_t slots, int32_t dst_on_device)
{
    if (!g) return fail(LP_EINVAL, "graph is NULL");
    lp::GraphSet &s = g->s;
    if (slots < 0 || slots > s.slpa_filled)
        return fail(LP_EINVAL, "slots must lie in [0, the slots the last SLPA run filled]");
    if (!dst && slots > 0 && s.nv > 0) return fail(LP_EINVAL, "dst is NULL");
    if (slots == 0 || s.nv == 0) return LP_OK;
    DeviceGuard dg(s.device);
    LP_CU(cudaMemcpyAsync(dst, s.slpa_mem, (size_t)slots * s.nv * sizeof(int32_t),
                          dst_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, s.st));
    LP_CU(cudaStreamSynchronize(s.st));
    return LP_OK;
}

lp_status lp_rak_history(const lp_graph *g, int64_t *changed, int32_t capacity, int32_t *count)
{
    if (!g || !count) return fail(LP_EINVAL, "graph or count is NULL");
    if (capacity > 0 && !changed) return fail(LP_EINVAL, "changed is NULL");
    const auto &h = g->s.history;
    *count = (int32_t)h.size();
    for (int32_t i = 0; i < capacity && i < (int32_t)h.size(); ++i) changed[i] = h[(size_t)i];
    return LP_OK;
}

lp_status lp_labels_get(lp_graph *g, int32_t *dst, int32_t dst_on_device)
{
    if (!g) return fail(LP_EINVAL, "graph is NULL");
    if (!dst && g->s.nv > 0) return fail(LP_EINVAL, "dst is NULL");
    DeviceGuard dg(g->s.device);
    return g->s.copy_labels(0, dst, dst_on_device);
}

lp_status lp_modularity(lp_graph *g, const int32_t *labels, int32_t labels_on_device, double *q)
{
    if (!g || !q) return fail(LP_EINVAL, "graph or q is NULL");
    DeviceGuard dg(g->s.device);
    lp::GraphSet &s = g->s;
    const int32_t *lab = s.lab[s.final_buf[0]];
    if (labels) {
        if (!s.lab_tmp) LP_TRY(dev_alloc(&s.lab_tmp, s.nv, "label staging", s.st, s.device));
        if (s.nv > 0)
            LP_CU(cudaMemcpyAsync(s.lab_tmp, labels, (size_t)s.nv * sizeof(int32_t),
                                  labels_on_device ? cudaMemcpyDeviceToDevice
                                                   : cudaMemcpyHostToDevice,
                                  s.st));
        Launches L;
        if (lp::check_labels(s.lab_tmp, s.nv, nullptr, nullptr, s.g_n, s.d_ing, s.st, &L.n) != 0)
            return fail(LP_ECUDA, cuda_msg("label check", cudaGetLastError()));
        LP_TRY(s.read_ingest(-1));
        lab = s.lab_tmp;
    }
    LP_TRY(s.modularity_all(lab));
    s.q_valid = labels == nullptr;
    *q = s.q_cache[0];
    return LP_OK;
}

lp_status lp_batch_create(int32_t count, const lp_graph_desc *graphs, uint32_t flags,
                          void *cuda_stream, lp_batch **out)
{
    if (!out) return fail(LP_EINVAL, "out is NULL");
    *out = nullptr;
    if (count < 1 || !graphs) return fail(LP_EINVAL, "need at least one graph");
    if (flags & ~(uint32_t)LP_FLAG_CHECK_SYMMETRIC)
        return fail(LP_EINVAL, "batches take host CSR; only LP_FLAG_CHECK_SYMMETRIC is allowed");
    int64_t nv = 0, ne = 0, noff = 0;
    bool any_w = false;
    for (int32_t i = 0; i < count; ++i) {
        const lp_graph_desc &d = graphs[i];
        char buf[128];
        snprintf(buf, sizeof buf, "graph %d: bad n, m or NULL arrays", i);
        if (d.n < 0 || d.m < 0 || d.m > 2147483647LL || !d.offsets || (d.m > 0 && !d.indices))
            return fail(LP_EINVAL, buf);
        nv += d.n;
        ne += d.m;
        noff += (int64_t)d.n + 1;
        any_w = any_w || d.weights;
    }
    if (nv + count > 2147483647LL) return fail(LP_EINVAL, "total vertices must stay below 2^31");
    std::unique_ptr<lp_batch> b(new (std::nothrow) lp_batch);
    if (!b) return fail(LP_ENOMEM, "host allocation failed");
    lp::GraphSet &s = b->s;
    LP_TRY(s.begin(cuda_stream));
    s.G = count;
    s.nv = (int32_t)nv;
    s.ne = ne;
    s.h_n.resize((size_t)count);
    s.h_m.resize((size_t)count);
    s.h_vbase.resize((size_t)count);
    s.h_ebase.resize((size_t)count);
    int64_t vb = 0, eb = 0;
    for (int32_t i = 0; i < count; ++i) {
        s.h_n[(size_t)i] = graphs[i].n;
        s.h_m[(size_t)i] = graphs[i].m;
        s.h_vbase[(size_t)i] = (int32_t)vb;
        s.h_ebase[(size_t)i] = eb;
        vb += graphs[i].n;
        eb += graphs[i].m;
        s.max_n = std::max(s.max_n, graphs[i].n);
    }
    LP_TRY(dev_alloc(&s.off, noff, "offsets", s.st, s.device));
    LP_TRY(dev_alloc(&s.idx, ne, "indices", s.st, s.device));
    if (any_w) LP_TRY(dev_alloc(&s.wts, ne, "weights", s.st, s.device));
    std::vector<int32_t> ones;
    for (int32_t i = 0; i < count; ++i) {
        const lp_graph_desc &d = graphs[i];
        const int64_t ob = (int64_t)s.h_vbase[(size_t)i] + i;
        const int64_t e0 = s.h_ebase[(size_t)i];
        LP_CU(cudaMemcpyAsync(s.off + ob, d.offsets, ((size_t)d.n + 1) * sizeof(int32_t),
                              cudaMemcpyHostToDevice, s.st));
        if (d.m > 0)
            LP_CU(cudaMemcpyAsync(s.idx + e0, d.indices, (size_t)d.m * sizeof(int32_t),
                                  cudaMemcpyHostToDevice, s.st));
        if (any_w && d.m > 0) {
            const int32_t *src = d.weights;
            if (!src) {
                if ((int64_t)ones.size() < d.m) ones.assign((size_t)d.m, 1);
                src = ones.data();
            }
            LP_CU(cudaMemcpyAsync(s.wts + e0, src, (size_t)d.m * sizeof(int32_t),
                                  cudaMemcpyHostToDevice, s.st));
        }
        if (flags & LP_FLAG_CHECK_SYMMETRIC) {
            if (!host_symmetric(d.n, d.offsets, d.indices, d.weights)) {
                char buf[96];
                snprintf(buf, sizeof buf, "graph %d: CSR is not symmetric", i);
                return fail(LP_EINVAL, buf);
            }
        }
    }
    LP_TRY(s.validate_all());
    // graph of every global vertex, per-graph bases and sizes
    std::vector<int32_t> vg((size_t)nv);
    for (int32_t i = 0; i < count; ++i)
        std::fill(vg.begin() + s.h_vbase[(size_t)i], vg.begin() + s.h_vbase[(size_t)i] + s.h_n[(size_t)i],
                  i);
    LP_TRY(dev_alloc(&s.vgraph, nv, "vertex graph ids", s.st, s.device));
    LP_TRY(dev_alloc(&s.g_vbase, count, "graph bases", s.st, s.device));
    LP_TRY(dev_alloc(&s.g_ebase, count, "graph bases", s.st, s.device));
    LP_TRY(dev_alloc(&s.g_n, count, "graph sizes", s.st, s.device));
    LP_TRY(dev_alloc(&s.g_active, count, "graph states", s.st, s.device));
    LP_TRY(host_alloc(&s.h_active, count, "graph states"));
    if (nv > 0)
        LP_CU(cudaMemcpyAsync(s.vgraph, vg.data(), vg.size() * sizeof(int32_t),
                              cudaMemcpyHostToDevice, s.st));
    LP_CU(cudaMemcpyAsync(s.g_vbase, s.h_vbase.data(), (size_t)count * sizeof(int32_t),
                          cudaMemcpyHostToDevice, s.st));
    LP_CU(cudaMemcpyAsync(s.g_ebase, s.h_ebase.data(), (size_t)count * sizeof(int64_t),
                          cudaMemcpyHostToDevice, s.st));
    LP_CU(cudaMemcpyAsync(s.g_n, s.h_n.data(), (size_t)count * sizeof(int32_t),
                          cudaMemcpyHostToDevice, s.st));
    LP_CU(cudaStreamSynchronize(s.st));
    LP_TRY(s.check_row_order());
    LP_TRY(s.bucket());
    LP_TRY(s.alloc_labels());
    LP_CU(cudaStreamSynchronize(s.st));
    *out = b.release();
    return LP_OK;
}

lp_status lp_batch_destroy(lp_batch *b)
{
    if (!b) return LP_OK;
    DeviceGuard dg(b->s.device);
    delete b;
    return LP_OK;
}

lp_status lp_batch_run(lp_batch *b, const lp_rak_params *p, lp_rak_result *per_graph)
{
    if (!b) return fail(LP_EINVAL, "batch is NULL");
    DeviceGuard dg(b->s.device);
    LP_TRY(b->s.run(p, true));
    if (per_graph)
        for (int32_t i = 0; i < b->s.G; ++i) per_graph[i] = b->s.results[(size_t)i];
    return LP_OK;
}

namespace {
lp_status set_buckets(lp::GraphSet &s, const int32_t *max_degree)
{
    if (!max_degree) return fail(LP_EINVAL, "max_degree is NULL");
    const int32_t cap[lp::NUM_BUCKETS - 1] = {lp::SMALL_MAX, lp::WARP_MAX, lp::CTA_MAX,
                                               lp::CTA2_MAX};
    lp::Thresholds t;
    int32_t prev = 1;
    for (int k = 0; k < lp::NUM_BUCKETS - 1; ++k) {
        if (max_degree[k] < prev || max_degree[k] > cap[k])
            return fail(LP_EINVAL, "bucket bounds must be non-decreasing, >= 1 and within "
                                   "32 / 128 / 512 / 1024");
        t.max[k] = prev = max_degree[k];
    }
    return s.rebucket(t);
}
}  // namespace

lp_status lp_graph_set_buckets(lp_graph *g, const int32_t *max_degree)
{
    if (!g) return fail(LP_EINVAL, "graph is NULL");
    DeviceGuard dg(g->s.device);
    return set_buckets(g->s, max_degree);
}

lp_status lp_batch_set_buckets(lp_batch *b, const int32_t *max_degree)
{
    if (!b) return fail(LP_EINVAL, "batch is NULL");
    DeviceGuard dg(b->s.device);
    return set_buckets(b->s, max_degree);
}

lp_status lp_batch_autotune(lp_batch *b, const lp_rak_params *p, int32_t sweeps,
                            lp_tune_result *out)
{
    if (!b) return fail(LP_EINVAL, "batch is NULL");
    DeviceGuard dg(b->s.device);
    if (p && p->init_labels) return fail(LP_EINVAL, "batches start from unique labels");
    return b->s.autotune(p, true, sweeps, out);
}

lp_status lp_batch_labels_get(lp_batch *b, int32_t index, int32_t *dst, int32_t dst_on_device)
{
    if (!b) return fail(LP_EINVAL, "batch is NULL");
    if (index < 0 || index >= b->s.G) return fail(LP_EINVAL, "graph index out of range");
    if (!dst && b->s.h_n[(size_t)index] > 0) return fail(LP_EINVAL, "dst is NULL");
    DeviceGuard dg(b->s.device);
    return b->s.copy_labels(index, dst, dst_on_device);
}

lp_status lp_batch_modularity(lp_batch *b, int32_t index, double *q)
{
    if (!b || !q) return fail(LP_EINVAL, "batch or q is NULL");
    if (index < 0 || index >= b->s.G) return fail(LP_EINVAL, "graph index out of range");
    DeviceGuard dg(b->s.device);
    lp::GraphSet &s = b->s;
    if (!s.q_valid) {
        LP_TRY(s.modularity_all(s.lab[0]));  // final labels are gathered in buffer 0
        s.q_valid = true;
    }
    *q = s.q_cache[(size_t)index];
    return LP_OK;
}

lp_status lp_profile_enable(int32_t on)
{
    g_prof_on = on != 0;
    return LP_OK;
}

lp_status lp_profile_reset(void)
{
    std::lock_guard<std::mutex> lock(g_prof_mu);
    for (auto &k : g_prof) k = KernelStat{};
    return LP_OK;
}

lp_status lp_profile_read(lp_kernel_stat *out, int32_t capacity, int32_t *count)
{
    if (!count) return fail(LP_EINVAL, "count is NULL");
    if (capacity > 0 && !out) return fail(LP_EINVAL, "out is NULL");
    std::lock_guard<std::mutex> lock(g_prof_mu);
    *count = lp::NUM_BUCKETS;
    for (int i = 0; i < lp::NUM_BUCKETS && i < capacity; ++i) {
        memset(out[i].name, 0, sizeof out[i].name);
        strncpy(out[i].name, KERNEL_NAMES[i], sizeof out[i].name - 1);
        out[i].launches = g_prof[i].launches;
        out[i].total_ms = g_prof[i].ms;
        out[i].vertices = g_prof[i].vertices;
        out[i].entries = g_prof[i].entries;
        out[i].bytes = g_prof[i].bytes;
    }
    return LP_OK;
}

lp_status lp_split_communities(lp_graph *g, int64_t *communities)
{
    if (!g) return fail(LP_EINVAL, "graph is NULL");
    DeviceGuard dg(g->s.device);
    lp::GraphSet &s = g->s;
    if (communities) *communities = 0;
    if (s.nv == 0) return LP_OK;
    int32_t *lab = s.lab[s.final_buf[0]];
    // scratch: parent array; component count, then error word, sampled root
    // and sampling switch (int32 each)
    int32_t *parent = nullptr;
    unsigned long long *words = nullptr;
    LP_TRY(dev_alloc(&parent, s.nv, "split scratch", s.st, s.device));
    if (dev_alloc(&words, 3, "split scratch", s.st, s.device) != LP_OK) {
        cudaFreeAsync(parent, s.st);
        return LP_ENOMEM;
    }
    unsigned long long h[2] = {0, 0};
    cudaError_t e = cudaMemsetAsync(words, 0, 3 * sizeof(unsigned long long), s.st);
    Launches L;
    if (e == cudaSuccess &&
        lp::split_launch(s.off, s.idx, lab, s.nv, s.ne, parent,
                         reinterpret_cast<int32_t *>(words + 1),
                         reinterpret_cast<int32_t *>(words + 1) + 1,
                         words, s.num_sms, s.st, &L.n) != 0)
        e = cudaGetLastError();
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(h, words, sizeof h, cudaMemcpyDeviceToHost, s.st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s.st);
    cudaFreeAsync(parent, s.st);
    cudaFreeAsync(words, s.st);
    if (e != cudaSuccess) return fail(LP_ECUDA, cuda_msg("community split", e));
    if ((uint32_t)h[1]) return fail(LP_ECUDA, "community split: a union-find link gave up");
    s.q_valid = false;
    if (communities) *communities = (int64_t)h[0];
    return LP_OK;
}

lp_status lp_selftest_barrier_timeout(int32_t *timed_out)
{
    if (!timed_out) return fail(LP_EINVAL, "timed_out is NULL");
    *timed_out = 0;
    int32_t *d = nullptr;  // bar[0], bar[1], err
    if (cudaMalloc(&d, 4 * sizeof(int32_t)) != cudaSuccess)
        return fail(LP_ENOMEM, "barrier self-test: cudaMalloc failed");
    cudaError_t e = cudaMemset(d, 0, 4 * sizeof(int32_t));
    if (e == cudaSuccess &&
        lp::barrier_probe_launch(reinterpret_cast<unsigned *>(d), d + 2, 4096, nullptr) != 1)
        e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    int32_t err = 0;
    if (e == cudaSuccess) e = cudaMemcpy(&err, d + 2, sizeof(int32_t), cudaMemcpyDeviceToHost);
    cudaFree(d);
    if (e != cudaSuccess) return fail(LP_ECUDA, cuda_msg("barrier self-test", e));
    ++g_launches;
    *timed_out = err;
    return LP_OK;
}

const char *lp_last_error(void) { return g_err.c_str(); }

int64_t lp_launch_count(void) { return g_launches.load(); }

}  // extern "C"
