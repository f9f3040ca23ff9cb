// Internal interface of the generic tensor-core BF16 GEMM (gemm.cu).
#pragma once

#include <cuda_runtime.h>

namespace pm {

// C[M][N] (FP32, row-major) = A[M][K] B[N][K]^T; A, B BF16 row-major.  M % 128 == 0,
// N % 64 == 0, K % 64 == 0.  *d_status is set to 1 if a bounded device wait gave up.  With a
// workspace (work_floats floats) a GEMM with few output tiles and a long K is split along K into
// slices summed afterwards in slice order.
int gemm_bf16_launch(const void *A, const void *B, float *C, int M, int N, int K, int *d_status, cudaStream_t st,
                     float *work = nullptr, size_t work_floats = 0);

}  // namespace pm
