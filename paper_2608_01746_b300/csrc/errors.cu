// Thread-local last-error message of the C ABI.
#include <cstdarg>
#include <cstdio>

#include "common.cuh"

namespace {
thread_local char g_last_error[512] = "";
}

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

}  // namespace pm

extern "C" const char *ptycho_last_error(void) { return g_last_error; }
