// Thread-local last-error message of the C ABI, and the library's device allocators (with the
// allocation-failure test hook and the per-device pool of the stream-ordered allocations).
#include <atomic>
#include <cstdarg>
#include <cstdint>
#include <cstdio>
#include <mutex>

#include "common.cuh"

namespace {
thread_local char g_last_error[512] = "";
// ptycho_debug_fail_alloc: countdown to the allocation that fails (0 = off)
std::atomic<int> g_fail_alloc{0};

bool injected_alloc_failure() {
    int n = g_fail_alloc.load();
    while (n > 0)
        if (g_fail_alloc.compare_exchange_weak(n, n - 1)) return n == 1;
    return false;
}

// The stream-ordered allocations of the library (reconstruction buffers, fusion scratch) come
// from one pool per device that keeps what is freed for the next allocation (release threshold
// unlimited): a reconstruction created after another was destroyed, or the next scan's fusion,
// reuses the same memory instead of mapping new pages and unmapping them again at the next
// synchronisation.  ptycho_release_memory hands the unused memory back.  A pool is never
// destroyed (a cudaDeviceReset, which would invalidate it, ends the library's use of the device
// as it ends that of every handle).
constexpr int kPoolDevices = 64;
std::mutex g_pool_mu;
cudaMemPool_t g_pool[kPoolDevices] = {};

cudaError_t device_pool(cudaMemPool_t *out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kPoolDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_pool_mu);
    if (!g_pool[dev]) {
        cudaMemPoolProps props = {};
        props.allocType = cudaMemAllocationTypePinned;
        props.handleTypes = cudaMemHandleTypeNone;
        props.location.type = cudaMemLocationTypeDevice;
        props.location.id = dev;
        cudaMemPool_t pool = nullptr;
        if ((e = cudaMemPoolCreate(&pool, &props)) != cudaSuccess) return e;
        uint64_t keep = UINT64_MAX;
        if ((e = cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep)) != cudaSuccess) {
            cudaMemPoolDestroy(pool);
            return e;
        }
        g_pool[dev] = pool;
    }
    *out = g_pool[dev];
    return cudaSuccess;
}
}  // namespace

namespace pm {

int fail(int code, const char *fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_last_error, sizeof g_last_error, fmt, ap);
    va_end(ap);
    return code;
}

int cuda_fail(cudaError_t e, const char *what) {
    const int code = (e == cudaErrorMemoryAllocation) ? PTYCHO_ENOMEM : PTYCHO_ECUDA;
    return fail(code, "%s: %s (%s)", what, cudaGetErrorString(e), cudaGetErrorName(e));
}

cudaError_t dev_malloc(void **p, size_t bytes) {
    *p = nullptr;
    if (injected_alloc_failure()) return cudaErrorMemoryAllocation;
    return cudaMalloc(p, bytes);
}

cudaError_t dev_malloc_async(void **p, size_t bytes, cudaStream_t st) {
    *p = nullptr;
    if (injected_alloc_failure()) return cudaErrorMemoryAllocation;
    cudaMemPool_t pool = nullptr;
    cudaError_t e = device_pool(&pool);
    if (e != cudaSuccess) return e;
    return cudaMallocFromPoolAsync(p, bytes, pool, st);
}

}  // namespace pm

extern "C" const char *ptycho_last_error(void) { return g_last_error; }

extern "C" int ptycho_release_memory(void) {
    std::lock_guard<std::mutex> lock(g_pool_mu);
    int rc = PTYCHO_OK;
    for (int d = 0; d < kPoolDevices; ++d) {
        if (!g_pool[d]) continue;
        // only the unused part goes back: memory that live handles hold stays theirs, and the
        // pools themselves live as long as the process
        cudaError_t e = cudaMemPoolTrimTo(g_pool[d], 0);
        if (e != cudaSuccess && rc == PTYCHO_OK) rc = pm::cuda_fail(e, "ptycho_release_memory");
    }
    return rc;
}

extern "C" int ptycho_debug_fail_alloc(int nth) {
    if (nth < 0) return pm::fail(PTYCHO_EINVAL, "ptycho_debug_fail_alloc: nth = %d < 0", nth);
    g_fail_alloc.store(nth);
    return PTYCHO_OK;
}
