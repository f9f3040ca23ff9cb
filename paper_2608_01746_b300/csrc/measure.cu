// Measurement kernels of the library's roofline: the FP32 FMA rate of the device.
//
// The paper states no hardware figures; the FP32 ALU roofline of the exit-wave kernels needs a
// measured denominator.  k_fma_rate runs `iters` rounds of 16 independent FMA chains per thread
// (x <- x * b + c, |b| < 1 keeps every chain bounded), so each SM sub-partition always has an
// independent FMA ready; the caller times the launch with CUDA events on its stream.
#include "common.cuh"
#include "measure.h"

namespace {

constexpr int kChains = 16;
constexpr int kFmaThreads = 256;

__global__ void __launch_bounds__(kFmaThreads) k_fma_rate(float *__restrict__ sink, int iters, float b, float c) {
    float x[kChains];
#pragma unroll
    for (int k = 0; k < kChains; ++k) x[k] = (float)(threadIdx.x + k) * 1e-3f;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int r = 0; r < 8; ++r)
#pragma unroll
            for (int k = 0; k < kChains; ++k) x[k] = fmaf(x[k], b, c);
    }
    float s = 0.f;
#pragma unroll
    for (int k = 0; k < kChains; ++k) s += x[k];
    sink[blockIdx.x * (size_t)blockDim.x + threadIdx.x] = s;
}

}  // namespace

extern "C" int measure_fp32_fma(int blocks, int iters, float *d_sink, double *flops, void *cuda_stream) {
    if (blocks < 1 || iters < 1 || !d_sink || !flops)
        return pm::fail(PTYCHO_EINVAL, "measure_fp32_fma: blocks = %d, iters = %d, sink %p, flops %p", blocks, iters,
                        (void *)d_sink, (void *)flops);
    k_fma_rate<<<blocks, kFmaThreads, 0, (cudaStream_t)cuda_stream>>>(d_sink, iters, 0.9999999f, 1e-7f);
    PM_LAUNCHED("k_fma_rate");
    *flops = 2.0 * kChains * 8.0 * (double)iters * (double)blocks * kFmaThreads;
    return PTYCHO_OK;
}

extern "C" int measure_fma_threads_per_block(void) { return kFmaThreads; }
