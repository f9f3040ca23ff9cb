// Generic BF16 GEMM on the fifth-generation tensor cores: C[M][N] (FP32, row-major) =
// A[M][K] B[N][K]^T with A and B BF16 row-major (K contiguous).  The convolution layers of the
// warm-start network (forward, data gradient, weight gradient) are all of this form after
// im2col.  M % 128 == 0, N % 64 == 0, K % 64 == 0 (callers pad with zeros).
//
// One CTA per 128 x 64 tile of C, 128 threads (thread r owns row r of the tile = TMEM lane r).
// K is consumed in chunks of 64 through four shared-memory stages in the no-swizzle core-matrix
// layout, filled with cp.async three chunks ahead of the tensor core.  Every wait is bounded; a
// timeout sets *status.
#include <cuda_bf16.h>

#include <algorithm>
#include <mutex>

#include "common.cuh"
#include "gemm.h"
#include "tcgen05.cuh"
#include "tma.cuh"

namespace {

using namespace pm;

constexpr int kBM = 128, kBN = 64, kBK = 64;
constexpr int kThreads = 128;
constexpr int kStages = 4;                      // chunks in flight
constexpr uint32_t kABytes = kBM * kBK * 2;     // 16 KB
constexpr uint32_t kBBytes = kBN * kBK * 2;     // 8 KB
constexpr uint32_t kStage = kABytes + kBBytes;
constexpr uint32_t kSmem = kStages * kStage + 1024;
constexpr uint32_t kLBO = 128, kSBO = (kBK / 8) * 128;

__device__ __forceinline__ void cp_async16(void *dst, const void *src) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(tc::smem_addr(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
    asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

// This thread's share of chunk kc (A: row m0 + tid, 8 x 16 bytes; B: 4 x 16 bytes) into a stage,
// in the core-matrix layout.
__device__ __forceinline__ void load_chunk(const uint4 *__restrict__ A, const uint4 *__restrict__ B, int m0, int n0,
                                           int k16, int kc, uint8_t *sa, uint8_t *sb) {
    const int tid = threadIdx.x;
    const uint4 *arow = A + (size_t)(m0 + tid) * k16 + kc * 8;
#pragma unroll
    for (int q = 0; q < 8; ++q) cp_async16(sa + ((tid >> 3) * 8 + q) * 128 + (tid & 7) * 16, arow + q);
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const int idx = tid + q * kThreads;     // 0 .. 511: 64 rows x 8 pieces
        const int r = idx >> 3, c = idx & 7;
        cp_async16(sb + ((r >> 3) * 8 + c) * 128 + (r & 7) * 16, B + (size_t)(n0 + r) * k16 + kc * 8 + c);
    }
}

// blockIdx.z selects a slice of K (split-K): chunks [z cps, min((z + 1) cps, K / 64)), written to
// C + z M N (a partial product; the caller sums the slices).  Chunks stream through kStages
// shared-memory stages with cp.async; a stage is refilled once the MMAs that read it have
// committed (their mbarrier), so loads run kStages - 1 chunks ahead of the tensor core.
__global__ void __launch_bounds__(kThreads)
    k_gemm_bf16(const uint4 *__restrict__ A, const uint4 *__restrict__ B, float *__restrict__ C, int M, int N, int K,
                int cps, int *status) {
    extern __shared__ uint8_t smem_raw[];
    uint8_t *sm = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
    __shared__ uint64_t bar[kStages];
    __shared__ uint32_t tmem_slot;
    const int tid = threadIdx.x, warp = tid >> 5;
    const int m0 = blockIdx.x * kBM, n0 = blockIdx.y * kBN;
    if (warp == 0) tc::alloc(&tmem_slot, 64);
    if (tid == 0) {
        for (int q = 0; q < kStages; ++q) tma::mbar_init(&bar[q], 1);
        tma::fence_barrier_init();
    }
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    const uint32_t tmem = tmem_slot;
    const int kc0 = blockIdx.z * cps;
    const int kchunks = min(K / kBK, kc0 + cps) - kc0;
    const int k16 = K / 8;                       // uint4 per row
    C += (size_t)blockIdx.z * M * N;
    uint32_t phase[kStages] = {};
    bool ok = true;
    // prologue: chunks 0 .. kStages - 2 in flight (one commit group each, possibly empty)
#pragma unroll
    for (int q = 0; q < kStages - 1; ++q) {
        if (q < kchunks) load_chunk(A, B, m0, n0, k16, kc0 + q, sm + q * kStage, sm + q * kStage + kABytes);
        cp_async_commit();
    }
    for (int kc = 0; kc < kchunks; ++kc) {
        const int s = kc % kStages;
        uint8_t *sa = sm + s * kStage, *sb = sa + kABytes;
        cp_async_wait<kStages - 2>();            // this thread's copies of chunk kc have landed
        tma::fence_async_smem();
        tc::fence_before();
        __syncthreads();                         // ... and every thread's
        if (tid == 0) {
            tc::fence_after();
            constexpr uint32_t idesc = tc::idesc_bf16_f32(kBM, kBN);
            const uint32_t a0 = tc::smem_addr(sa), b0 = tc::smem_addr(sb);
#pragma unroll
            for (int ks = 0; ks < kBK / 16; ++ks)
                tc::mma_bf16(tmem, tc::smem_desc(a0 + ks * 256, kLBO, kSBO), tc::smem_desc(b0 + ks * 256, kLBO, kSBO),
                             idesc, (uint32_t)((kc | ks) != 0));
            tc::commit(&bar[s]);
        }
        // refill the stage of chunk kc - 1 with chunk kc + kStages - 1 once its MMAs are done
        const int nxt = kc + kStages - 1;
        if (nxt < kchunks) {
            const int sp = nxt % kStages;
            if (kc >= 1) {
                bool w = true;
                if (warp == 0) w = tma::mbar_wait(&bar[sp], phase[sp]);
                ok = __syncthreads_and(w) != 0;
                if (!ok) break;
                phase[sp] ^= 1;
            }
            load_chunk(A, B, m0, n0, k16, kc0 + nxt, sm + sp * kStage, sm + sp * kStage + kABytes);
        }
        cp_async_commit();
    }
    cp_async_wait<0>();
    if (kchunks <= 0) {                          // empty slice: a zero partial
        float *crow = C + (size_t)(m0 + tid) * N + n0;
        for (int q = 0; q < kBN; ++q) crow[q] = 0.f;
    } else if (ok) {
        // the last commit covers every MMA issued before it
        const int s = (kchunks - 1) % kStages;
        bool w = true;
        if (warp == 0) w = tma::mbar_wait(&bar[s], phase[s]);
        ok = __syncthreads_and(w) != 0;
        tc::fence_after();
    }
    if (ok && kchunks > 0) {
        float *crow = C + (size_t)(m0 + tid) * N + n0;
        const uint32_t lane_addr = tmem + ((uint32_t)(32 * warp) << 16);
#pragma unroll
        for (int ch = 0; ch < kBN / 32; ++ch) {
            uint32_t v[32];
            tc::ld_32cols(lane_addr + ch * 32, v);
            tc::wait_ld();
#pragma unroll
            for (int q = 0; q < 8; ++q)
                reinterpret_cast<float4 *>(crow + ch * 32)[q] =
                    make_float4(__uint_as_float(v[4 * q]), __uint_as_float(v[4 * q + 1]), __uint_as_float(v[4 * q + 2]),
                                __uint_as_float(v[4 * q + 3]));
        }
    } else if (!ok) {
        if (tid == 0) atomicExch(status, 1);
        // let MMAs still in flight finish before the columns are released (bounded)
        if (warp == 0)
            for (int q = 0; q < kStages; ++q) tma::mbar_wait(&bar[q], phase[q]);
    }
    tc::fence_before();
    __syncthreads();
    if (warp == 0) {
        tc::fence_after();
        tc::dealloc(tmem, 64);
    }
}

// C[e] = sum over the slices, in slice order (deterministic).
__global__ void k_sum_slices(const float *__restrict__ part, int slices, size_t n, float *__restrict__ C) {
    for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x) {
        float s = 0.f;
        for (int z = 0; z < slices; ++z) s += part[(size_t)z * n + e];
        C[e] = s;
    }
}

// Devices whose kernel attribute (dynamic shared memory above 48 KB) is set; guarded by g_attr_mu
// so that host threads making their first call at the same time do not race.
std::mutex g_attr_mu;
bool g_attr_set[64] = {};

}  // namespace

namespace pm {

int gemm_bf16_launch(const void *A, const void *B, float *C, int M, int N, int K, int *d_status, cudaStream_t st,
                     float *work, size_t work_floats) {
    if (M % kBM || N % kBN || K % kBK || M < 0 || N < 0 || K < 0)
        return fail(PTYCHO_EINVAL, "gemm_bf16: M %% 128, N %% 64, K %% 64 must be 0 (M=%d N=%d K=%d)", M, N, K);
    if (M == 0 || N == 0) return PTYCHO_OK;
    int dev = 0;
    PM_CUDA(cudaGetDevice(&dev));
    {
        std::lock_guard<std::mutex> lk(g_attr_mu);
        if (dev >= 64 || !g_attr_set[dev]) {
            PM_CUDA(cudaFuncSetAttribute(k_gemm_bf16, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmem));
            if (dev < 64) g_attr_set[dev] = true;
        }
    }
    if (K == 0) {
        PM_CUDA(cudaMemsetAsync(C, 0, (size_t)M * N * sizeof(float), st));
        return PTYCHO_OK;
    }
    // split K when the output tiles alone cannot fill the GPU (weight gradients: small M x N,
    // K = every pixel of the batch)
    const int tiles = (M / kBM) * (N / kBN), kch = K / kBK;
    int slices = 1;
    if (work && tiles < 296 && kch >= 8) {
        slices = std::min(std::min((296 + tiles - 1) / tiles, kch / 4), 64);
        while (slices > 1 && (size_t)slices * M * N > work_floats) --slices;
    }
    const int cps = (kch + slices - 1) / slices;
    dim3 grid(M / kBM, N / kBN, slices);
    k_gemm_bf16<<<grid, kThreads, kSmem, st>>>(static_cast<const uint4 *>(A), static_cast<const uint4 *>(B),
                                                slices > 1 ? work : C, M, N, K, cps, d_status);
    PM_LAUNCHED("k_gemm_bf16");
    if (slices > 1) {
        const size_t n = (size_t)M * N;
        k_sum_slices<<<(unsigned)std::min<size_t>((n + 255) / 256, 4096), 256, 0, st>>>(work, slices, n, C);
        PM_LAUNCHED("k_sum_slices");
    }
    return PTYCHO_OK;
}

}  // namespace pm

extern "C" int gemm_bf16(const void *d_A, const void *d_B, float *d_C, int M, int N, int K, int *d_status,
                         void *cuda_stream) {
    if ((M > 0 && N > 0 && K > 0) && (!d_A || !d_B || !d_C || !d_status))
        return pm::fail(PTYCHO_EINVAL, "gemm_bf16: NULL pointer");
    return pm::gemm_bf16_launch(d_A, d_B, d_C, M, N, K, d_status, static_cast<cudaStream_t>(cuda_stream));
}
