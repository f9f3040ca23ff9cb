// Internal interface of the generic tensor-core BF16 GEMM (gemm.cu).
#pragma once

#include <cuda_runtime.h>

namespace pm {

// C[M][N] (FP32, row-major) = A[M][K] B[N][K]^T; A, B BF16 row-major.  M % 128 == 0,
// N % 64 == 0, K % 64 == 0.  *d_status is set to 1 if a bounded device wait gave up.
int gemm_bf16_launch(const void *A, const void *B, float *C, int M, int N, int K, int *d_status, cudaStream_t st);

}  // namespace pm
