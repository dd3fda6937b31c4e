// Device-side convergence test (Sec. 3.2).
//
// Runs keep the tolerance test on the device: after each iteration's sweeps,
// k_converge applies it to every graph still iterating and records the
// results.  A run captured as one CUDA graph is a chain of conditional (if)
// nodes, one per iteration, and k_converge arms the next node only if some
// graph goes on; a run driven from the host launches iterations ahead
// without waiting, and k_converge raises a stop flag that makes the kernels
// of iterations launched past the end return at once.  Either way the host
// reads the per-graph results once at the end.
#include "lp_internal.cuh"

namespace lp {
namespace {

// Iteration `it` has ended: for every graph that was still iterating, record
// its results and deactivate it if at most tolerance * n of its vertices
// changed; arm the next iteration if any graph remains active.
__global__ void __launch_bounds__(1024)
    k_converge(const int32_t *changed_it, const int32_t *g_n, int32_t *g_active, int32_t G,
               double tolerance, int32_t it, int32_t multi, RunResults res,
               cudaGraphConditionalHandle next, int32_t has_next, int32_t *stop, int32_t last)
{
    if (stop && *stop) return;  // launched ahead of a run that has ended
    int going = 0;
    for (int32_t g = threadIdx.x; g < G; g += blockDim.x) {
        if (multi && !g_active[g]) continue;
        const int32_t c = changed_it[g];
        res.iterations[g] = it + 1;
        res.last_changed[g] = c;
        res.final_buf[g] = (it + 1) & 1;  // iteration it wrote buffer (it + 1) mod 2
        if ((double)c <= tolerance * (double)g_n[g]) {
            res.converged[g] = 1;
            if (multi) g_active[g] = 0;
        } else {
            going = 1;
        }
    }
    going = __syncthreads_or(going);
    if (threadIdx.x == 0) {
        if (going && has_next) cudaGraphSetConditional(next, 1u);
        if (stop && (!going || last)) *stop = 1;
    }
}

}  // namespace

int converge_launch(const int32_t *changed_it, const int32_t *g_n, int32_t *g_active, int32_t G,
                    double tolerance, int32_t it, bool multi, const RunResults &res,
                    cudaGraphConditionalHandle next, bool has_next, int32_t *stop, bool last,
                    cudaStream_t st)
{
    k_converge<<<1, 1024, 0, st>>>(changed_it, g_n, g_active, G, tolerance, it, multi ? 1 : 0,
                                   res, next, has_next ? 1 : 0, stop, last ? 1 : 0);
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

}  // namespace lp
