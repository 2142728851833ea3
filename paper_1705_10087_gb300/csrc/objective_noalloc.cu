// csc_objective_noalloc: the FP64 objective E(Z) without any device allocation.
//
// csc_objective needs a handle, and a handle allocates its buffers with
// cudaMalloc.  Some callers cannot allocate: a serving loop that admits work
// against a fixed device-memory budget and must not grow it once a request is
// running, or latency-sensitive code that cannot afford the implicit device
// synchronisation cudaMalloc/cudaFree may cause.  This entry point computes
// the same quantity from caller-owned device arrays and keeps its only
// scratch (the per-block partial sums) in a file-scope device array.
//
// That array is g_partials below: 2 * kNoAllocMaxBlocks doubles (1 MiB),
// present on every GPU that loads this library until the process exits.  It
// bounds the signal length to kNoAllocMaxBlocks * kTile = 16,777,216 samples.
// All calls share it: calls whose GPU work overlaps (two streams, two host
// threads without ordering) race on it and must be serialised by the caller.
// Each call overwrites every entry it later reads, so nothing is cleared.
#include <cstring>

#include "csc_internal.cuh"

namespace {

constexpr int kNoAllocMaxBlocks = 1 << 16;

// [0, 2*kNoAllocMaxBlocks): per-block (sum of squared residuals, sum |Z|);
// the extra entry receives E when the caller's output is in host memory.
static __device__ __align__(256) double g_partials[2 * kNoAllocMaxBlocks + 2];

// Device memory of device `dev` (the current one), or managed memory.
bool device_resident(const void *p, int dev)
{
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    if (a.type == cudaMemoryTypeManaged)
        return true;
    return a.type == cudaMemoryTypeDevice && a.device == dev;
}

}  // namespace

// Shared with capi.cu: records the message returned by csc_last_error_string.
int csc_record_error(int code, const char *fmt, ...);

extern "C" int csc_objective_noalloc(const float *D, int K, int P, int L, const float *X,
                                     int64_t T, const float *Z, double lambda, double *E_out,
                                     void *stream)
{
    if (!D || !X || !Z || !E_out)
        return csc_record_error(CSC_EINVAL, "csc_objective_noalloc: null pointer");
    if (K < 1 || K > 256 || P < 1 || L < 1 || L > csc::kMaxL || T < L)
        return csc_record_error(CSC_EINVAL,
                                "csc_objective_noalloc: need 1 <= K <= 256, P >= 1, "
                                "1 <= L <= %d, T >= L",
                                csc::kMaxL);
    if (!(lambda >= 0.0))
        return csc_record_error(CSC_EINVAL, "csc_objective_noalloc: lambda must be >= 0");
    const int64_t nb = (T + csc::kTile - 1) / csc::kTile;
    if (nb > kNoAllocMaxBlocks)
        return csc_record_error(CSC_EINVAL,
                                "csc_objective_noalloc: T = %lld exceeds the static scratch "
                                "limit of %d samples",
                                (long long)T, kNoAllocMaxBlocks * csc::kTile);
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess)
        return csc_record_error(CSC_ECUDA, "csc_objective_noalloc: no usable current device");
    if (!device_resident(D, dev) || !device_resident(X, dev) || !device_resident(Z, dev))
        return csc_record_error(CSC_EINVAL,
                                "csc_objective_noalloc: D, X and Z must be memory of the "
                                "current device (%d)",
                                dev);

    // The host-side name g_partials is not a device address: look the array
    // up on the current device.  This is done on every call (a host-side
    // query), so the address stays right after a context of the device was
    // torn down and created again.
    double *scratch = nullptr;
    {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_partials);
        if (e != cudaSuccess || !p)
            return csc_record_error(CSC_ECUDA,
                                    "csc_objective_noalloc: cudaGetSymbolAddress failed: %s",
                                    cudaGetErrorString(e));
        scratch = static_cast<double *>(p);
    }

    cudaStream_t s = (cudaStream_t)stream;
    const bool out_on_device = device_resident(E_out, dev);
    double *out = out_on_device ? E_out : scratch + 2 * kNoAllocMaxBlocks;
    csc::SigDesc one{};
    one.Z = const_cast<float *>(Z);
    one.X = X;
    one.ld = T - L + 1;
    one.ldx = T;
    one.Tz = T - L + 1;
    one.lam = (float)lambda;
    one.lam_d = lambda;
    e = csc::launch_objective_single(D, one, K, P, L, scratch, out, s);
    if (e != cudaSuccess)
        return csc_record_error(CSC_ECUDA, "csc_objective_noalloc: launch failed: %s",
                                cudaGetErrorString(e));
    if (!out_on_device) {
        e = cudaMemcpyAsync(E_out, out, sizeof(double), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess)
            e = cudaStreamSynchronize(s);
        if (e != cudaSuccess)
            return csc_record_error(CSC_ECUDA, "csc_objective_noalloc: %s",
                                    cudaGetErrorString(e));
    }
    return CSC_OK;
}
