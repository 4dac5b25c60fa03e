// ptrkind.cuh -- classification of caller pointers (host code).
//
// The C ABI accepts host or device arrays and detects the kind per pointer.
// Device memory of a device other than the current one is rejected: the
// kernels would dereference it directly, which without peer access is an
// illegal address on the GPU.
#pragma once
#include <cuda_runtime.h>

namespace tw {

enum { PK_HOST = 0, PK_DEV = 1, PK_OTHER = 2 };

// PK_HOST: pageable or pinned host memory (or a pointer CUDA does not know);
// PK_DEV: device memory of the current device, or managed memory;
// PK_OTHER: device memory of another device.
static inline int ptr_kind(const void *p) {
    if (!p) return PK_HOST;
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) { (void)cudaGetLastError(); return PK_HOST; }
    if (a.type == cudaMemoryTypeManaged) return PK_DEV;
    if (a.type != cudaMemoryTypeDevice) return PK_HOST;
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) { (void)cudaGetLastError(); return PK_OTHER; }
    return a.device == dev ? PK_DEV : PK_OTHER;
}

}  // namespace tw
