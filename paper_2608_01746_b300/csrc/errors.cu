// Thread-local last-error message of the C ABI, and the library's device allocators (with the
// allocation-failure test hook).
#include <atomic>
#include <cstdarg>
#include <cstdio>

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
    return cudaMallocAsync(p, bytes, st);
}

}  // namespace pm

extern "C" const char *ptycho_last_error(void) { return g_last_error; }

extern "C" int ptycho_debug_fail_alloc(int nth) {
    if (nth < 0) return pm::fail(PTYCHO_EINVAL, "ptycho_debug_fail_alloc: nth = %d < 0", nth);
    g_fail_alloc.store(nth);
    return PTYCHO_OK;
}
