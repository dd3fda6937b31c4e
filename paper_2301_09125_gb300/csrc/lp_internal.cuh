// Internal declarations shared by the library's translation units.
//
// Device layout of a graph set (one graph, or a batch of graphs in one arena):
//   off  int32  per graph n_g + 1 local row offsets, graphs concatenated
//               (graph g's rows start at off[vbase_g + g])
//   idx  int32  local neighbour ids, graphs concatenated (graph g's entries
//               start at ebase_g)
//   wts  int32  weights aligned with idx, or null for unit weights
//   lab  int32  two label buffers of NV entries (vertex v of graph g at
//               vbase_g + v); labels are local vertex ids
//   list int32  global vertex ids sorted into degree buckets
//               [small | warp | cta | cta2 | hub], ascending id inside a bucket
//               except hub, which is sorted by degree, largest first
// Packed rows (what the sweep reads): the rows of the run's list (the bucket
// list, or the wave-partitioned list of an asynchronous run) copied in list
// order, so that the rows of one launch lie next to each other in HBM:
//   rp   int64  [len + 1] start of list item i's row in pidx / pwts
//   pidx int32  neighbour ids (local), bit 31 set when the neighbour's wave
//               comes before the row's vertex's wave (read from this
//               iteration's labels); never set in synchronous runs
//   pwts int32  weights aligned with pidx, or null for unit weights
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace lp {

constexpr unsigned FULL = 0xffffffffu;
constexpr int32_t EMPTY = -1;

// Degree buckets (Sec. 3.2's per-vertex hashtable, mapped to the GPU's
// thread / warp / CTA granularity).
constexpr int SMALL_MAX = 32;   // 1..32: several vertices packed per warp
constexpr int WARP_MAX = 128;   // 33..128: one warp per vertex
constexpr int CTA_MAX = 512;    // 129..512: one 128-thread CTA per vertex
constexpr int CTA2_MAX = 1024;  // 513..1024: one 256-thread CTA per vertex
                                // > 1024: hub
constexpr int NUM_BUCKETS = 5;  // small, warp, cta, cta2, hub
constexpr int HUB_BUCKET = NUM_BUCKETS - 1;

// Largest degree of each bucket but the hub bucket.  The defaults are the
// constants above; a graph set may be re-bucketed with other values (the
// autotuner), each at most its bucket kernel's capacity above and
// non-decreasing.
struct Thresholds {
    int32_t max[NUM_BUCKETS - 1] = {SMALL_MAX, WARP_MAX, CTA_MAX, CTA2_MAX};
};

constexpr int WARP_TABLE = 256;         // slots per warp (>= 2 * WARP_MAX)
constexpr int CTA_THREADS = 128;
constexpr int CTA_TABLE = 1024;         // slots (>= 2 * CTA_MAX)
constexpr int CTA2_THREADS = 256;
constexpr int CTA2_TABLE = 2048;        // slots (>= 2 * CTA2_MAX)
constexpr int HUB_THREADS = 512;
constexpr int HUB_TABLE = 8192;         // shared slots per hub CTA (>= 2 * HUB_ONE_MAX)
constexpr int HUB_ONE_MAX = 4096;       // longest hub row swept by one CTA
constexpr int HUB_SEG = 4096;           // entries per segment of a longer row
constexpr int HUB_REC = 3;              // ints per segment record (label, sum, ~first position)
constexpr int HUB_PMAX = 2048;          // most label partitions of one row

// One hub of a list being swept (the hub bucket, or its part in one wave),
// prepared once per list.  Rows longer than HUB_ONE_MAX come first.  Such a
// row is cut into nseg segments of HUB_SEG entries; each segment aggregates
// its labels in shared memory and writes them out as records grouped into
// npart partitions by label hash, then one CTA per partition merges the
// records of all segments, and the last one to finish picks the row's label.
// A label that finds no room in a partition's shared table goes to the row's
// global fallback table of 2^ceil(log2(2d)) slots starting at slot `tab`
// (used-slot list at tab / 2).
struct HubTask {
    int32_t v;       // global vertex
    int32_t d;       // degree
    int32_t nseg;    // segments (rows longer than HUB_ONE_MAX)
    int32_t npart;   // label partitions
    int32_t seg0;    // first segment item of the row in this list
    int32_t part0;   // first partition item of the row in this list
    int64_t poff0;   // first entry of its partition offsets (nseg x (npart + 1))
    int64_t tab;     // first slot of its fallback table
    int64_t e0;      // first entry of its packed row
};

// Arguments of one sweep kernel launch (one bucket).
struct SweepArgs {
    const int64_t *rp;       // packed row starts, aligned with `list` (rp[i] .. rp[i + 1])
    const int32_t *idx;      // packed neighbour ids (bit 31: earlier wave)
    const int32_t *wts;      // packed weights, null = unit weights
    const int32_t *lab_in;   // labels read (== lab_out in asynchronous mode)
    // SLPA (Sec. 3.4): the label each entry's speaker spoke, aligned with idx
    // (null: an entry's label is its neighbour's current label)
    const int32_t *spoken;
    int32_t *lab_out;        // labels written
    const int32_t *list;     // bucket entries (global vertex ids)
    int64_t len;             // bucket length
    int64_t ne;              // entries in the arena (idx / wts are read in 16-byte blocks)
    // graph set (null for a single graph: every base is 0)
    const int32_t *vgraph;   // graph of each global vertex
    const int32_t *g_vbase;  // first global vertex of each graph
    const int64_t *g_ebase;  // first global entry of each graph
    const int32_t *g_active; // 1 while the graph is still iterating
    int32_t *changed;        // changed counter(s) of this iteration (per graph)
    int strict;              // 1 strict, 0 non-strict
    uint64_t key_t;          // non-strict stream key of this iteration
    // 1 when every label this launch reads is the initial unique label and no
    // row repeats a neighbour: a label's weight is then its one edge weight
    int identity;
    // 1 when a vertex whose own label holds more than half of its row's weight
    // may keep it without a table (that label is then the unique maximum).
    // changed_prev (the previous iteration's changed count per graph, or
    // null) and g_n (vertices per graph) let a kernel try the test only once
    // labels have settled.
    int majority;
    const int32_t *changed_prev;
    const int32_t *g_n;
    // raised by the device-side tolerance test once the run is over: kernels
    // of iterations launched ahead of it return at once (null: not used)
    const int32_t *stop;
    // asynchronous waves (Sec. 3.3): a neighbour of an earlier wave (bit 31 of
    // its packed id) is read from lab_out (this iteration), every other one
    // from lab_in.  waves = 1: sync.
    uint32_t waves;
    // small-row kernel: list entries per warp tile (32, or fewer for short
    // lists of rows long enough to need several chunks; set by the launch
    // from the bucket's mean degree)
    int32_t tile_rows;
    int32_t small_mean_deg;
    // hub launches: the list's tasks (aligned with `list`), how many of them
    // are rows longer than HUB_ONE_MAX, with their segment and partition item
    // counts; segment records (HUB_SEG records of HUB_REC ints per segment
    // item: label, sum, ~first position), partition offsets, partition bests (32 bytes per
    // partition item); fallback tables (slot = (label + 1) << 32 | summed
    // weight, 0 when free, plus ~first position), used-slot lists and
    // per-task counters of finished partitions and used slots (zero between
    // launches)
    const HubTask *htask;
    int64_t hmulti;
    int64_t hsegs;
    int64_t hparts;
    const int32_t *hseg_task;   // task of each segment item
    const int32_t *hpart_task;  // task of each partition item
    int32_t *hrec;
    int32_t *hpoff;
    void *hpbest;
    unsigned long long *hkey;
    uint32_t *hnpos;
    int32_t *hused;
    int32_t *hdone;
    int32_t *hnused;
    // per long-row task: own-label weight, total weight, candidate weight and
    // candidate of the row (the majority test of rows longer than HUB_ONE_MAX,
    // summed over segments); per segment item: its weighted majority vote
    // (candidate, surplus)
    uint32_t *hmaj;
    int2 *hvote;
    int32_t *hopen;   // long rows that no label holds by majority (set before the segment pass)
    // single graphs, majority level 2: the pre-pass lists the positions of the
    // rows it did not settle (cpos, *ccount of them) for the CTA kernel
    int32_t *cpos;
    int32_t *ccount;
    // per vertex: 1 if the majority pre-pass of this launch settled its row
    // (rows of the cta, cta2 and hub buckets; null = no pre-pass)
    uint8_t *vmaj;
};

// Modularity arguments (a whole graph set; graph layout as for SweepArgs).
// The entry pass reads the packed rows in chunks of PACK_CHUNK entries;
// first_row[c] is the list item whose row holds entry c * PACK_CHUNK
// (first_row[ncopy] = the last item).
constexpr int PACK_CHUNK = 256;  // one warp, eight entries per lane
struct ModArgs {
    const int64_t *rp;         // packed row starts, aligned with list (len + 1)
    const int32_t *idx;        // packed neighbour ids (bit 31 ignored)
    const int32_t *wts;        // packed weights, null = unit weights
    const int32_t *lab;        // labels of every vertex (local ids)
    const int32_t *list;       // list items (global vertices), len of them
    int64_t len;
    int64_t ne;                // entries in the arena
    const int64_t *first_row;  // ncopy + 1 entries
    int64_t ncopy;
    // the list's first nsmall items (the small bucket) hold the entries
    // [0, e_lo): their rows are summed one per lane, and the chunk pass
    // counts only entries from e_lo on (chunks from e_lo / PACK_CHUNK)
    int64_t nsmall;
    int64_t e_lo;
    const int32_t *vgraph;     // null for a single graph
    const int32_t *g_vbase;
    unsigned long long *kc;    // [nv] K_c of community c of graph g at vbase_g + c (zeroed)
    unsigned long long *acc;   // [4 G]: L, 2m, S high, S low per graph (zeroed)
};

// Rows per warp tile of the small-row kernels: fewer than 32 while a list
// would fill under 32 warps per SM and its rows are long enough that a tile
// takes several packed chunks one after another (rows of a few entries are
// summed one per lane, where a partly used warp only adds overhead).
inline int32_t small_tile_rows(int64_t len, int32_t mean_deg, int num_sms)
{
    int32_t rt = 32;
    while (rt > 4 && (len + rt - 1) / rt < (int64_t)num_sms * 32 && (int64_t)mean_deg * rt > 64)
        rt >>= 1;
    return rt;
}

// ----------------------------------------------------------------------------
// SplitMix64 output function (Steele, Lea & Flood 2014), used in counter mode
// for the non-strict tie key.
// ----------------------------------------------------------------------------
constexpr uint64_t GOLDEN = 0x9E3779B97F4A7C15ull;

__host__ __device__ __forceinline__ uint64_t splitmix_out(uint64_t z)
{
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

// Remainder by an invariant divisor d (1 <= d < 2^32) without a divide:
// M = floor((2^64 - 1) / d) + 1, a mod d = high64((M * a mod 2^64) * d)
// (Lemire, Kaser & Kurz, "Faster remainder by direct computation", 2019).
__host__ __device__ __forceinline__ uint64_t fastmod_magic(uint32_t d)
{
    return 0xFFFFFFFFFFFFFFFFull / d + 1;
}

__device__ __forceinline__ uint32_t fastmod(uint32_t a, uint64_t magic, uint32_t d)
{
    return (uint32_t)__umul64hi(magic * (uint64_t)a, (uint64_t)d);
}

// k-th output of the stream whose state starts at `key`
__host__ __device__ __forceinline__ uint64_t stream_at(uint64_t key, uint64_t k)
{
    return splitmix_out(key + k * GOLDEN);
}

// ----------------------------------------------------------------------------
// Launchers (lp_sweep.cu, lp_ingest.cu, lp_modularity.cu)
// ----------------------------------------------------------------------------
int sweep_prepare();  // per-device kernel attributes; call with the device current
// launch the sweep kernel(s) of one degree bucket (0 small, 1 warp, 2 cta,
// 3 cta2, 4 hub); returns the number of kernels launched, or -1
int sweep_launch(int bucket, const SweepArgs &a, bool multi, int num_sms, cudaStream_t st);
// Four CTAs wait at a grid barrier for a fifth that never comes: the wait
// gives up after spin_limit polls and sets *err (bar: two zeroed words).
int barrier_probe_launch(unsigned *bar, int32_t *err, uint32_t spin_limit, cudaStream_t st);
// Every wave of an asynchronous single-graph sweep whose rows all lie in the
// small bucket, as one cooperative launch (wave k's list: wlist + wstart[k],
// wcount[k] entries, both device arrays; max_len the longest).  bar: two
// device words, zeroed before every launch (the barriers count arrivals over
// the launch); *err set to 1 if a grid barrier timed out.  Returns the kernel
// count (1) or -1.
// (max_degree: the graph's longest row; rows of at most 8 entries take the
// kernel that loads the next wave's rows before each barrier)
int small_waves_launch(const SweepArgs &a, const int32_t *wlist, const int64_t *wstart,
                       const int64_t *wcount, int64_t max_len, int32_t max_degree, unsigned *bar,
                       int32_t *err, int num_sms, cudaStream_t st);
// Device scratch (int64 words) of hub_order and hub_tasks for a list of len
// rows.
int64_t hub_scratch_ints(int64_t len);
// out = the hub rows of list in decreasing order of floor(log2(degree)),
// stable within a class
int hub_order(const int32_t *list, int64_t len, const int32_t *off, const int32_t *vgraph,
              int32_t *out, int64_t *scratch, cudaStream_t st, int64_t *launches);
// Hub tasks of list[0..len): the rows longer than HUB_ONE_MAX first, then the
// others, each kind in list order; list is rewritten in the same order so that
// tasks[i] belongs to list[i].  totals: [0] rows of the first kind, [1] their
// fallback table slots, [2] segments, [3] partitions, [4] partition offsets.
int hub_tasks(int32_t *list, int64_t len, const int32_t *off, const int32_t *vgraph,
              HubTask *tasks, int64_t *totals, int64_t *scratch, cudaStream_t st,
              int64_t *launches);
// tasks[i].e0 = rp[i] for i < n (the packed row start of task i's row).
int hub_task_starts(HubTask *tasks, int64_t n, const int64_t *rp, cudaStream_t st,
                    int64_t *launches);
// Packed rows of list[0..len) (every listed vertex has at least one entry):
// rp[i] = entries of the rows before item i (rp[len] = their total, the
// arena's entry count), then the rows copied in list order into pidx / pwts
// (pwts skipped when wts is null), with bit 31 of a neighbour id set when
// waves > 1 and the neighbour's wave (local id mod waves) comes before the
// row's; first_row (pack_chunks(ne) + 1 entries) receives the item holding
// each PACK_CHUNK-th entry.  scratch: pack_scratch_ints(len) int64.
// bucket_entries (host, NUM_BUCKETS, or null): the entries of each bucket's
// rows, the list being bucket-major; the copy then takes the wave segments
// of a bucket in turn (results do not depend on it).
int64_t pack_scratch_ints(int64_t len);
inline int64_t pack_chunks(int64_t ne) { return (ne + PACK_CHUNK - 1) / PACK_CHUNK; }
int pack_rows(const int32_t *list, int64_t len, const int32_t *off, const int32_t *idx,
              const int32_t *wts, int64_t ne, const int32_t *vgraph, const int32_t *g_vbase,
              const int64_t *g_ebase, int waves, const int64_t *bucket_entries,
              int64_t *scratch, int64_t *rp, int64_t *first_row, int32_t *pidx, int32_t *pwts,
              cudaStream_t st, int64_t *launches);
// Task index of every segment item and partition item of the first nbig tasks.
int hub_item_maps(const HubTask *tasks, int64_t nbig, int32_t *seg_task, int32_t *part_task,
                  cudaStream_t st, int64_t *launches);

struct IngestOut {
    int32_t err;          // 0 ok, else an error code below
    int32_t err_at;       // offending vertex / entry (first seen)
    int32_t max_w;
    int32_t max_deg;
    int32_t wdeg_overflow;
    int32_t repeated;     // some row does not list its neighbours in strictly increasing order
};
enum IngestErr : int32_t {
    ING_OK = 0,
    ING_OFF_FIRST = 1,
    ING_OFF_ORDER = 2,
    ING_OFF_LAST = 3,
    ING_INDEX = 4,
    ING_WEIGHT = 5,
    ING_WDEG = 6,
    ING_ASYM = 7,
    ING_LABEL = 8,
};

int ingest_validate(const int32_t *off, const int32_t *idx, const int32_t *wts, int32_t n,
                    int64_t m, IngestOut *d_out, cudaStream_t st, int64_t *launches);
// ingest_validate and the row-order check of ingest_row_order in one pass over
// one graph's entries (bits: scratch of m / 32 + 1 words).
int ingest_validate_ordered(const int32_t *off, const int32_t *idx, const int32_t *wts, int32_t n,
                            int64_t m, uint32_t *bits, IngestOut *d_out, cudaStream_t st,
                            int64_t *launches);
// Whether every row lists its neighbours in strictly increasing order (then no
// row repeats a neighbour): d_out->repeated = 0 if so.  Needs a validated CSR
// set and a scratch bitmap of ne / 32 + 1 words; rows of graph g at ebase_g.
int ingest_row_order(const int32_t *off, const int32_t *idx, int32_t nv, int64_t ne,
                     const int32_t *vgraph, const int64_t *g_ebase, uint32_t *bits,
                     IngestOut *d_out, cudaStream_t st, int64_t *launches);
int ingest_check_wdeg(const int32_t *off, const int32_t *wts, int32_t n, IngestOut *d_out,
                      cudaStream_t st, int64_t *launches);
// Bucket every vertex of a graph set.  d_counts[0..B) receives the bucket
// lengths, [B..2B) their starts in `list`, [2B..3B) their summed degrees
// (B = NUM_BUCKETS).
int ingest_bucket(const int32_t *off, int32_t nv_total, const int32_t *vgraph,
                  const int32_t *g_vbase, const Thresholds &th, int32_t *list,
                  int32_t *scratch_blocks, int64_t *d_counts, cudaStream_t st,
                  int64_t *launches);
size_t ingest_bucket_scratch_bytes(int32_t nv_total);
// Wave partition of the bucket lists for asynchronous runs: entries of bucket b
// and wave k (= local vertex id mod waves) are gathered, class by class
// (class = b * waves + k), into `out`; d_totals[class] receives the class sizes.
constexpr int WAVE_MAX = 4096;
// asynchronous runs of at least this many waves over small rows only sweep
// all waves of an iteration in one cooperative launch
constexpr int COOP_MIN_WAVES = 8;
int64_t wave_hist_ints(int64_t list_len, int waves);
int wave_prepare();  // per-device kernel attributes
int wave_partition(const int32_t *list, int64_t list_len, const int64_t *bucket_begin,
                   const int32_t *vgraph, const int32_t *g_vbase, int waves, int32_t *hist,
                   int64_t *d_totals, int32_t *out, cudaStream_t st, int64_t *launches);
// lab0[v] = lab1[v] for the vertices of graphs g with g_sel[g] != 0
int merge_final_labels(int32_t *lab0, const int32_t *lab1, int32_t nv, const int32_t *vgraph,
                       const int32_t *g_sel, cudaStream_t st, int64_t *launches);
int fill_iota(int32_t *lab, int32_t nv, const int32_t *vgraph, const int32_t *g_vbase,
              cudaStream_t st, int64_t *launches);
int check_labels(const int32_t *lab, int32_t nv, const int32_t *vgraph, const int32_t *g_vbase,
                 const int32_t *g_n, IngestOut *d_out, cudaStream_t st, int64_t *launches);

// Per-graph results of a run captured as a CUDA graph (device arrays of G).
struct RunResults {
    int32_t *iterations;
    int32_t *converged;
    int32_t *final_buf;      // label buffer holding the final labels
    long long *last_changed;
};
// The tolerance test of iteration `it` on the device (Sec. 3.2); arms `next`
// (the following iteration's conditional node) if some graph goes on and
// has_next; with `stop`, raises *stop when no graph goes on or `it` is the
// last iteration, and does nothing once *stop is raised.
int converge_launch(const int32_t *changed_it, const int32_t *g_n, int32_t *g_active, int32_t G,
                    double tolerance, int32_t it, bool multi, const RunResults &res,
                    cudaGraphConditionalHandle next, bool has_next, int32_t *stop, bool last,
                    cudaStream_t st);

// SLPA (Sec. 3.4), lp_slpa.cu.  Memory slot t of vertex v at mem[t * n + v].
// SLPA_SPEAK keeps the speakers' slot draws apart from the tie keys (the
// same seed drives both).
constexpr int SLPA_MAX_MEMORY = 64;
constexpr uint64_t SLPA_SPEAK = 0x5350454Bull;
// spoken[e] for every packed entry e of a single graph's rows in iteration t
// (1 <= t < memory_size): the speaker's label in slot draw(seed ^ SLPA_SPEAK,
// t, listener, row position) mod t of its memory.
int slpa_speak(const int64_t *rp, const int32_t *list, const int64_t *first_row, int64_t ne,
               const int32_t *pidx, const int32_t *mem, int32_t n, int32_t t, uint64_t seed,
               int32_t *spoken, cudaStream_t st, int64_t *launches);
// out[v] = the label slots 0 .. last of v's memory hold most often, the first
// stored on equal counts.
int slpa_community(const int32_t *mem, int32_t n, int32_t last, int32_t *out, cudaStream_t st,
                   int64_t *launches);

// COPRA (Sec. 3.3), lp_copra.cu: one iteration (or one wave of it) of a
// single graph.  Sets: L (label, belonging) pairs per vertex, belongings in
// units of 2^-16 summing to COPRA_ONE, belonging 0 after a set's last pair.
constexpr uint32_t COPRA_ONE = 65536u;
struct CopraStep {
    const int32_t *off, *idx, *wts;  // the original CSR
    int32_t n, L;
    const int32_t *cur_l;            // previous iteration's sets
    const uint32_t *cur_b;
    int32_t *nxt_l;                  // this iteration's sets
    uint32_t *nxt_b;
    int32_t waves, wave_k;           // wave_k of waves (1: synchronous)
    int strict;
    uint64_t key_t;                  // non-strict key of the iteration
    int32_t *changed;                // += vertices whose best label changed
    // this wave's listed rows (copra_rows): those of a whole warp, of a CTA
    // with the shared table, and of the long-row kernel
    const int32_t *rows_warp, *rows_cta, *rows_big;
    int64_t n_warp, n_cta, n_big;
    // n + 1 ints of scratch: the long rows that outgrow the shared table
    int32_t *ovf;
    // rows of more than the shared table's pairs: copra_big_ctas() tables of
    // 2^glg_max slots (key -1, sum 0, first ~0 when clean; left clean)
    int32_t *gkey;
    unsigned long long *gsum, *gfirst;
    int32_t glg_max;                 // 0: no such row
};
int copra_prepare();
int copra_init(int32_t *l, uint32_t *b, int32_t n, int32_t L, cudaStream_t st, int64_t *launches);
// out[v] = the best (first) label of v's set
int copra_best(const int32_t *l, int32_t n, int32_t L, int32_t *out, cudaStream_t st,
               int64_t *launches);
// log2 of the slots a row of max_degree entries needs in the global tables
// (0 when every row fits the shared table)
int copra_table_lg(int64_t max_degree, int32_t L);
int copra_big_ctas();
// The rows that the 8-lane kernel does not take (all rows when L > 8, else
// those of more than 32 pairs), grouped by bin = kind * waves + wave (kind 0:
// a whole warp, 1: a CTA with the shared table, 2: the long-row kernel):
// rows[h_start[bin] .. h_start[bin + 1]).  bins: device
// scratch and h_bins host scratch of copra_bins(waves) ints; h_start:
// copra_bins(waves) + 1; rows: n.  Waits for the stream.
int64_t copra_bins(int32_t waves);
int copra_rows(const int32_t *off, int32_t n, int32_t L, int32_t waves, int32_t *bins,
               int32_t *h_bins, int64_t *h_start, int32_t *rows, cudaStream_t st,
               int64_t *launches);
int copra_step(const CopraStep &s, int num_sms, cudaStream_t st, int64_t *launches);

// Split the communities of lab (n vertices, m entries, one graph) into
// connected components in place: lab[v] = smallest vertex of v's component.
// parent: n scratch ints; *err set to 1 if a link gave up; big: two scratch
// ints; *count += components.
int split_launch(const int32_t *off, const int32_t *idx, int32_t *lab, int32_t n, int64_t m,
                 int32_t *parent, int32_t *err, int32_t *big, unsigned long long *count,
                 int num_sms, cudaStream_t st, int64_t *launches);

// Entry and square passes of the modularity of every graph of a set (nslots:
// entries of kc).
int modularity_launch(const ModArgs &a, int64_t nslots, bool multi, cudaStream_t st,
                      int64_t *launches);

}  // namespace lp
