// Host-side helpers shared by the C ABI translation units: pointer-kind
// detection, copies in either direction, growable device buffers and NVTX
// ranges.
#pragma once

#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include <vector>

namespace csc {

// NVTX range over a scope: names an entry point's host span in a profiler's
// timeline (a no-op unless a profiler is attached).
struct TraceRange {
    explicit TraceRange(const char *name) { nvtxRangePushA(name); }
    ~TraceRange() { nvtxRangePop(); }
    TraceRange(const TraceRange &) = delete;
    TraceRange &operator=(const TraceRange &) = delete;
};

// Makes a handle's device current for the scope of an entry point and puts
// the caller's current device back when the scope ends, so that no call of
// this library changes which device is current for the calling thread.
// err holds the result of the switch (checked by the caller).
struct DeviceGuard {
    int prev = -1;
    cudaError_t err = cudaSuccess;
    explicit DeviceGuard(int dev)
    {
        if (cudaGetDevice(&prev) != cudaSuccess) {
            cudaGetLastError();
            prev = -1;
        }
        if (prev != dev)
            err = cudaSetDevice(dev);
    }
    ~DeviceGuard()
    {
        if (err == cudaSuccess && prev >= 0) {
            int cur = -1;
            if (cudaGetDevice(&cur) == cudaSuccess && cur != prev)
                cudaSetDevice(prev);
        }
    }
    DeviceGuard(const DeviceGuard &) = delete;
    DeviceGuard &operator=(const DeviceGuard &) = delete;
};

inline bool is_device_pointer(const void *p)
{
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// Whether p is page-locked host memory: a cudaMemcpyAsync from it returns
// before the copy has read it (from pageable memory it returns after staging).
inline bool is_pinned_host(const void *p)
{
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeHost;
}

inline cudaError_t copy_in(void *dst, const void *src, size_t bytes, cudaStream_t s)
{
    return cudaMemcpyAsync(dst, src, bytes,
                           is_device_pointer(src) ? cudaMemcpyDeviceToDevice
                                                  : cudaMemcpyHostToDevice,
                           s);
}

inline cudaError_t copy_out(void *dst, const void *src, size_t bytes, cudaStream_t s)
{
    return cudaMemcpyAsync(dst, src, bytes,
                           is_device_pointer(dst) ? cudaMemcpyDeviceToDevice
                                                  : cudaMemcpyDeviceToHost,
                           s);
}

template <class T>
cudaError_t grow(T **p, size_t *cap, size_t n)
{
    if (*cap >= n && *p)
        return cudaSuccess;
    if (*p)
        cudaFree(*p);
    *p = nullptr;
    *cap = 0;
    cudaError_t e = cudaMalloc(reinterpret_cast<void **>(p), sizeof(T) * (n ? n : 1));
    if (e == cudaSuccess)
        *cap = n;
    return e;
}

template <class T>
cudaError_t upload(T **p, size_t *cap, const std::vector<T> &v, cudaStream_t s)
{
    cudaError_t e = grow(p, cap, v.size());
    if (e != cudaSuccess)
        return e;
    return cudaMemcpyAsync(*p, v.data(), sizeof(T) * v.size(), cudaMemcpyHostToDevice, s);
}

}  // namespace csc
