// lp_probe_gather: the memory ceiling of a sweep's data movement, measured on
// the GPU.  Mode 0 streams the column indices and weights of every entry in
// 16-byte blocks (the sweep's HBM traffic); mode 1 also gathers the label of
// every entry's neighbour (the sweep's label gather, which stays in L2 while
// the labels fit there).  No per-row work: a sweep that reads every
// neighbour's label cannot run faster than mode 1 on the same CSR.
#include <string>

#include "lp.h"
#include "lp_device.cuh"
#include "lp_internal.cuh"

namespace lp {
lp_status lp_fail(lp_status s, const std::string &msg);  // lp_api.cu: sets lp_last_error
void lp_add_launches(int64_t n);                         // lp_api.cu: lp_launch_count

namespace {

template <bool GATHER>
__global__ void __launch_bounds__(256) k_probe(const int32_t *idx, const int32_t *wts,
                                               const int32_t *lab, int64_t nblk,
                                               unsigned *sink)
{
    unsigned acc = 0u;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; b < nblk; b += stride) {
        const int4 I = ld_entries4(idx, b);
        const int4 W = wts ? ld_entries4(wts, b) : make_int4(1, 1, 1, 1);
        if (GATHER) {
            const int32_t l0 = ld_label(lab + I.x), l1 = ld_label(lab + I.y);
            const int32_t l2 = ld_label(lab + I.z), l3 = ld_label(lab + I.w);
            acc += (l0 == l1 ? W.x : 0) + (l2 == l3 ? W.y : 0) + (l0 == l2 ? W.z : 0) +
                   (l1 == l3 ? W.w : 0);
            acc ^= (unsigned)(l0 + l3);
        } else {
            acc += (unsigned)(I.x ^ I.y ^ I.z ^ I.w) + (unsigned)(W.x + W.y + W.z + W.w);
        }
    }
    acc = __reduce_add_sync(FULL, acc);
    if ((threadIdx.x & 31) == 0) atomicAdd(sink, acc);  // keeps every load live
}

// sink[1] = 1 if some index of the first nblk blocks lies outside [0, n)
__global__ void __launch_bounds__(256) k_probe_check(const int32_t *idx, int64_t nblk, int32_t n,
                                                     unsigned *sink)
{
    bool bad = false;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; b < nblk; b += stride) {
        const int4 I = reinterpret_cast<const int4 *>(idx)[b];
        bad = bad || (uint32_t)I.x >= (uint32_t)n || (uint32_t)I.y >= (uint32_t)n ||
              (uint32_t)I.z >= (uint32_t)n || (uint32_t)I.w >= (uint32_t)n;
    }
    if (__any_sync(FULL, bad) && (threadIdx.x & 31) == 0) atomicExch(sink + 1, 1u);
}

}  // namespace
}  // namespace lp

extern "C" lp_status lp_probe_gather(int32_t n, int64_t m, const int32_t *indices,
                                     const int32_t *weights, const int32_t *labels,
                                     int32_t mode, int32_t repeats, unsigned *sink,
                                     float *ms_per_pass, void *cuda_stream)
{
    using namespace lp;
    if (n < 1 || m < 4 || !indices || !labels || !sink || !ms_per_pass)
        return lp_fail(LP_EINVAL, "NULL argument, n < 1 or m < 4");
    if (mode != 0 && mode != 1) return lp_fail(LP_EINVAL, "mode must be 0 or 1");
    if (repeats < 1 || repeats > 1000) return lp_fail(LP_EINVAL, "repeats must lie in [1, 1000]");
    if (((uintptr_t)indices & 15u) || ((uintptr_t)weights & 15u))
        return lp_fail(LP_EINVAL, "indices and weights must start on a 16-byte boundary");
    cudaStream_t st = (cudaStream_t)cuda_stream;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return lp_fail(LP_ECUDA, "no usable CUDA device");
    const int64_t nblk = m / 4;  // whole blocks only
    const int grid = sms * 8;
    // the gather reads labels[index]: every index must lie in [0, n)
    unsigned flag = 0u;
    if (cudaMemsetAsync(sink, 0, 2 * sizeof(unsigned), st) != cudaSuccess)
        return lp_fail(LP_ECUDA, "probe set-up failed");
    k_probe_check<<<grid, 256, 0, st>>>(indices, nblk, n, sink);
    if (cudaMemcpyAsync(&flag, sink + 1, sizeof flag, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
        return lp_fail(LP_ECUDA, "probe index check failed");
    if (flag) return lp_fail(LP_EINVAL, "an index lies outside [0, n)");
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
        if (e0) cudaEventDestroy(e0);
        return lp_fail(LP_ECUDA, "event creation failed");
    }
    auto launch = [&]() {
        if (mode == 1)
            k_probe<true><<<grid, 256, 0, st>>>(indices, weights, labels, nblk, sink);
        else
            k_probe<false><<<grid, 256, 0, st>>>(indices, weights, labels, nblk, sink);
    };
    for (int i = 0; i < 3; ++i) launch();  // warm-up
    cudaEventRecord(e0, st);
    for (int i = 0; i < repeats; ++i) launch();
    cudaEventRecord(e1, st);
    cudaError_t e = cudaEventSynchronize(e1);
    float ms = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    lp_add_launches(3 + repeats);
    if (e != cudaSuccess) return lp_fail(LP_ECUDA, std::string("probe: ") + cudaGetErrorString(e));
    *ms_per_pass = ms / (float)repeats;
    return LP_OK;
}
