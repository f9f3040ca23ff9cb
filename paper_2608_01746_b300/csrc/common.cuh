// Shared host/device helpers of the CUDA library: error reporting and complex arithmetic.
#pragma once

#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>
#include <stdint.h>

#include "ptycho_mnf.h"

namespace pm {

// Records a printf-style message as the calling thread's last error and returns `code`.
int fail(int code, const char *fmt, ...);
// Records a CUDA failure ("<what>: <cuda error string>") and returns PTYCHO_ECUDA, or
// PTYCHO_ENOMEM for cudaErrorMemoryAllocation.
int cuda_fail(cudaError_t e, const char *what);
// Every device allocation of the library goes through these two (cudaMalloc; stream-ordered from
// the library's per-device pool, which keeps freed memory for reuse), so that
// ptycho_debug_fail_alloc can make the n-th one report cudaErrorMemoryAllocation.
cudaError_t dev_malloc(void **p, size_t bytes);
cudaError_t dev_malloc_async(void **p, size_t bytes, cudaStream_t st);

// NVTX range for the host-side extent of one stage (visible in Nsight timelines; a no-op
// unless a tool is attached).
struct NvtxRange {
    explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange &) = delete;
    NvtxRange &operator=(const NvtxRange &) = delete;
};

}  // namespace pm

#define PM_CUDA(call)                                                       \
    do {                                                                    \
        cudaError_t pm_e_ = (call);                                         \
        if (pm_e_ != cudaSuccess) return pm::cuda_fail(pm_e_, #call);       \
    } while (0)

#define PM_LAUNCHED(what)                                                   \
    do {                                                                    \
        cudaError_t pm_e_ = cudaGetLastError();                             \
        if (pm_e_ != cudaSuccess) return pm::cuda_fail(pm_e_, what);        \
    } while (0)

// Programmatic dependent launch.  A kernel launched with programmatic stream serialization may
// be scheduled while the previous kernel on its stream is still running: pdl_wait() (first, before
// the kernel touches memory) returns once that kernel has completed and its writes are visible.
// pdl_allow_dependents() lets the next such kernel be scheduled as this one's blocks retire.
// Both are no-ops for kernels launched without the attribute.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_allow_dependents() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
    return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
// conj(a) * b
__device__ __forceinline__ float2 cmulc(float2 a, float2 b) {
    return make_float2(a.x * b.x + a.y * b.y, a.x * b.y - a.y * b.x);
}
__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }

// The same sums as one packed two-lane FP32 instruction each (add / sub .rn.f32x2: per-lane
// IEEE round-to-nearest, the results of cadd / csub bit for bit).
__device__ __forceinline__ float2 cadd_x2(float2 a, float2 b) {
    unsigned long long r;
    asm("add.rn.f32x2 %0, %1, %2;"
        : "=l"(r)
        : "l"(*reinterpret_cast<const unsigned long long *>(&a)), "l"(*reinterpret_cast<const unsigned long long *>(&b)));
    return *reinterpret_cast<const float2 *>(&r);
}
__device__ __forceinline__ float2 csub_x2(float2 a, float2 b) {
    unsigned long long r;
    asm("sub.rn.f32x2 %0, %1, %2;"
        : "=l"(r)
        : "l"(*reinterpret_cast<const unsigned long long *>(&a)), "l"(*reinterpret_cast<const unsigned long long *>(&b)));
    return *reinterpret_cast<const float2 *>(&r);
}
__device__ __forceinline__ float2 cscale(float2 a, float s) { return make_float2(a.x * s, a.y * s); }
__device__ __forceinline__ float cabs2(float2 a) { return a.x * a.x + a.y * a.y; }
