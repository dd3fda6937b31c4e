// SLPA, the speaker-listener label propagation (Sec. 3.4), on the sweep
// kernels of RAK.  Every vertex keeps a memory of memory_size labels (slot 0
// holds the vertex itself); iteration t fills slot t.  In iteration t every
// neighbour u of a listener v speaks one label from the slots its memory held
// before the iteration: slot s = floor(hi32(h) * t / 2^32) with h the
// counter-based SplitMix64 draw of (seed ^ SPEAK, t, v, position of the entry
// in v's row).  The listener stores the heaviest spoken label under RAK's tie
// rules, so a sweep of RAK over the spoken labels (one label per entry,
// written here into `spoken`, aligned with the packed rows) is the listening
// step.  A vertex's community is the label its memory holds most often, the
// one stored first on equal counts.
#include "lp_device.cuh"
#include "lp_internal.cuh"

namespace lp {
namespace {

constexpr int SP_T = 256, SP_PER = 8;  // threads per block, entries per lane
constexpr int SP_WARPS = SP_T / 32;
static_assert(32 * SP_PER == PACK_CHUNK, "one warp per packed chunk");

// Spoken labels of iteration t for the entries of chunk (warp) c of the
// packed rows: rows r0 .. r1 of the chunk are staged (start, listener key).
__global__ void __launch_bounds__(SP_T) k_slpa_speak(const int64_t *rp, const int32_t *list,
                                                     const int64_t *first_row, int64_t ncopy,
                                                     const int32_t *pidx, int64_t ne,
                                                     const int32_t *mem, int64_t n, uint32_t t,
                                                     uint64_t key_t, int32_t *spoken)
{
    __shared__ int64_t s_rp_all[SP_WARPS][PACK_CHUNK + 2];
    __shared__ uint64_t s_key_all[SP_WARPS][PACK_CHUNK + 1];
    __shared__ uint16_t s_row_all[SP_WARPS][PACK_CHUNK];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const int64_t chunk = (int64_t)blockIdx.x * SP_WARPS + wib;
    if (chunk >= ncopy) return;  // warp-uniform
    int64_t *s_rp = s_rp_all[wib];
    uint64_t *s_key = s_key_all[wib];
    uint16_t *s_row = s_row_all[wib];
    const int64_t j_lo = chunk * PACK_CHUNK;
    const int64_t j_hi = min(j_lo + (int64_t)PACK_CHUNK, ne);
    const int64_t r0 = first_row[chunk];
    const int64_t r1 = first_row[chunk + 1];
    const int nr = (int)min(r1 - r0 + 1, (int64_t)PACK_CHUNK + 1);
    for (int k = lane; k <= nr; k += 32) s_rp[k] = rp[r0 + k];
    for (int k = lane; k < nr; k += 32) s_key[k] = stream_at(key_t, (uint64_t)list[r0 + k] + 1);
    __syncwarp();
    chunk_rows([&](int k) { return (int)(s_rp[k] - j_lo); }, nr, s_row);
#pragma unroll
    for (int q = 0; q < SP_PER; ++q) {
        const int e = lane + 32 * q;
        const int64_t j = j_lo + e;
        if (j >= j_hi) continue;
        const int k = s_row[e];
        const uint64_t h = stream_at(s_key[k], (uint64_t)(j - s_rp[k]) + 1);
        const uint64_t slot = ((h >> 32) * (uint64_t)t) >> 32;  // in [0, t)
        const int32_t u = pidx[j] & 0x7FFFFFFF;
        spoken[j] = __ldg(mem + (int64_t)slot * n + u);
    }
}

// community of every vertex: the label its memory slots 0 .. last hold most
// often, the first stored on equal counts (memory_size <= SLPA_MAX_MEMORY)
__global__ void k_slpa_community(const int32_t *mem, int64_t n, int32_t last, int32_t *out)
{
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n;
         v += (int64_t)gridDim.x * blockDim.x) {
        int32_t lab[SLPA_MAX_MEMORY];
        for (int a = 0; a <= last; ++a) lab[a] = mem[(int64_t)a * n + v];
        int32_t best = lab[0], best_count = 0;
        for (int a = 0; a <= last; ++a) {
            bool seen = false;
            for (int b = 0; b < a; ++b) seen = seen || lab[b] == lab[a];
            if (seen) continue;
            int32_t c = 0;
            for (int b = a; b <= last; ++b) c += lab[b] == lab[a];
            if (c > best_count) {
                best = lab[a];
                best_count = c;
            }
        }
        out[v] = best;
    }
}

int grid_of(int64_t items, int threads, int cap)
{
    const int64_t b = (items + threads - 1) / threads;
    return (int)(b < 1 ? 1 : (b > cap ? cap : b));
}

}  // namespace

int slpa_speak(const int64_t *rp, const int32_t *list, const int64_t *first_row, int64_t ne,
               const int32_t *pidx, const int32_t *mem, int32_t n, int32_t t, uint64_t seed,
               int32_t *spoken, cudaStream_t st, int64_t *launches)
{
    if (ne <= 0) return 0;
    const int64_t ncopy = pack_chunks(ne);
    const uint64_t key_t = stream_at(seed ^ SLPA_SPEAK, (uint64_t)t + 1);
    k_slpa_speak<<<(int)((ncopy + SP_WARPS - 1) / SP_WARPS), SP_T, 0, st>>>(
        rp, list, first_row, ncopy, pidx, ne, mem, n, (uint32_t)t, key_t, spoken);
    ++*launches;
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

int slpa_community(const int32_t *mem, int32_t n, int32_t last, int32_t *out, cudaStream_t st,
                   int64_t *launches)
{
    if (n <= 0) return 0;
    if (last < 0 || last >= SLPA_MAX_MEMORY) return -1;
    k_slpa_community<<<grid_of(n, 256, 8192), 256, 0, st>>>(mem, n, last, out);
    ++*launches;
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

}  // namespace lp
