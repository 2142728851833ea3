// Control kernels of a CD round run as a CUDA graph (capi.cu): the decision
// at the end of each poll batch that keeps the round's while loop going or
// stops it, and the limits it tests.
#include "csc_internal.cuh"

namespace csc {

namespace {

// End of one poll batch inside the graph of a CD round: advance the launch
// counter by the batch's launches and let the round's while loop go on only
// while no stopping rule holds (see launch_round_step).
__global__ void round_step_kernel(cudaGraphConditionalHandle cond, int *gctr, int batch,
                                  const int *done, const long long *total,
                                  const long long *lim)
{
    const int g = gctr[0] + batch;
    gctr[0] = g;
    const int g_round = gctr[1];
    const bool stop = *(volatile const int *)done != 0 ||
                      *(volatile const long long *)total >= lim[0] ||
                      (lim[1] > 0 && g - g_round >= lim[1]) || g >= lim[2] ||
                      (long long)g + batch > lim[3];
    cudaGraphSetConditional(cond, stop ? 0u : 1u);
}

__global__ void set_limits_kernel(long long *lim, long long a, long long b, long long c,
                                  long long d)
{
    lim[0] = a;
    lim[1] = b;
    lim[2] = c;
    lim[3] = d;
}

}  // namespace

cudaError_t launch_round_step(cudaGraphConditionalHandle cond, int *gctr, int batch,
                              const int *done, const long long *total, const long long *lim,
                              cudaStream_t s)
{
    round_step_kernel<<<1, 1, 0, s>>>(cond, gctr, batch, done, total, lim);
    return cudaGetLastError();
}

cudaError_t launch_set_limits(long long *lim, long long max_updates, long long drift_launches,
                              long long max_g, long long ring, cudaStream_t s)
{
    set_limits_kernel<<<1, 1, 0, s>>>(lim, max_updates, drift_launches, max_g, ring);
    return cudaGetLastError();
}

}  // namespace csc
