// Control kernels of a solve (capi.cu): the state set up at its start and at
// the start of each CD round, and, for a round run as a CUDA graph, the
// decision at the end of each poll batch that keeps the round's while loop
// going or stops it.
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

// Start of a CD round: the done flag cleared, the round's first launch index
// and its stopping rules set (one launch instead of three small ones).
__global__ void round_begin_kernel(int *done, int *gctr, int g_round, long long *lim,
                                   long long a, long long b, long long c, long long d)
{
    *done = 0;
    gctr[1] = g_round;
    lim[0] = a;
    lim[1] = b;
    lim[2] = c;
    lim[3] = d;
}

// Start of a solve: the trace ring and counters zeroed (words [0, nwords)),
// every segment dirty and every resync tile touched, and the start stamped.
__global__ void solve_begin_kernel(unsigned long long *__restrict__ zero, int64_t nwords,
                                   unsigned char *__restrict__ dirty,
                                   unsigned char *__restrict__ touched, int64_t M,
                                   unsigned long long *tstart)
{
    const int64_t i0 = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int64_t step = (int64_t)gridDim.x * blockDim.x;
    if (i0 == 0)
        *tstart = globaltimer_ns();
    for (int64_t i = i0; i < nwords; i += step)
        zero[i] = 0ull;
    for (int64_t i = i0; i < M; i += step) {
        dirty[i] = 1;
        touched[i] = 1;
    }
}

}  // namespace

cudaError_t launch_round_begin(int *done, int *gctr, int g_round, long long *lim,
                               long long max_updates, long long drift_launches, long long max_g,
                               long long ring, cudaStream_t s)
{
    round_begin_kernel<<<1, 1, 0, s>>>(done, gctr, g_round, lim, max_updates, drift_launches,
                                       max_g, ring);
    return cudaGetLastError();
}

cudaError_t launch_solve_begin(unsigned long long *zero, int64_t nwords, unsigned char *dirty,
                               unsigned char *touched, int64_t M, unsigned long long *tstart,
                               cudaStream_t s)
{
    const int64_t n = nwords > M ? nwords : M;
    const int64_t blocks = (n + 255) / 256;
    solve_begin_kernel<<<(unsigned)(blocks < 1024 ? (blocks > 0 ? blocks : 1) : 1024), 256, 0,
                         s>>>(zero, nwords, dirty, touched, M, tstart);
    return cudaGetLastError();
}

cudaError_t launch_round_step(cudaGraphConditionalHandle cond, int *gctr, int batch,
                              const int *done, const long long *total, const long long *lim,
                              cudaStream_t s)
{
    round_step_kernel<<<1, 1, 0, s>>>(cond, gctr, batch, done, total, lim);
    return cudaGetLastError();
}

}  // namespace csc
