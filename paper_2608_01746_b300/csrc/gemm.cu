// Generic BF16 GEMM on the fifth-generation tensor cores: C[M][N] (FP32, row-major) =
// A[M][K] B[N][K]^T with A and B BF16 row-major (K contiguous).  The convolution layers of the
// warm-start network (forward, data gradient, weight gradient) are all of this form after
// im2col.  M % 128 == 0, N % 64 == 0, K % 64 == 0 (callers pad with zeros).
//
// One CTA per 128 x BN tile of C (BN = 256, 192, 128 or 64, chosen from N), 192 threads in three
// roles:
//   warp 0   one lane issues the TMA loads of the 128 x 64 A chunk and the BN x 64 B chunk of
//            every K step into a ring of shared-memory stages (128-byte swizzle, the layout the
//            MMA descriptors read directly); a stage is refilled once the MMAs that read it
//            have completed (its "empty" mbarrier, signalled by tcgen05.commit);
//   warp 1   allocates the BN TMEM accumulator columns; one lane waits for each stage's
//            "full" mbarrier (TMA transaction bytes) and issues the four 128 x BN x 16 MMAs;
//   warps 2-5  (one per 32-lane TMEM quarter) wait for the last commit and store C.
// Every wait is bounded; a timeout sets *status, and the CTA drains the loads and MMAs it
// still has in flight (bounded) before it releases TMEM and exits.
#include <cuda.h>
#include <cuda_bf16.h>

#include <algorithm>
#include <mutex>

#include "common.cuh"
#include "gemm.h"
#include "tcgen05.cuh"
#include "tma.cuh"
#include "tmap.h"

namespace {

using namespace pm;

constexpr int kBM = 128, kBK = 64;
constexpr int kThreads = 192;
constexpr uint32_t kABytes = kBM * kBK * 2;     // 16 KB

template <int BN>
struct Cfg {
    static constexpr int kStages = BN == 256 ? 4 : (BN == 192 ? 5 : (BN == 128 ? 6 : 8));
    static constexpr uint32_t kBBytes = BN * kBK * 2;
    static constexpr uint32_t kStage = kABytes + kBBytes;
    static constexpr uint32_t kSmem = kStages * kStage + 1024;   // + alignment slack
    static constexpr uint32_t kTmemCols = BN == 192 ? 256 : BN;  // a power of two
    static_assert(kSmem <= 227 * 1024, "shared memory");
};

// blockIdx.z selects a slice of K (split-K): chunks [z cps, min((z + 1) cps, K / 64)), written to
// C + z M N (a partial product; the caller sums the slices).
template <int BN>
__global__ void __launch_bounds__(kThreads, 1)
    k_gemm_bf16(const __grid_constant__ CUtensorMap ta, const __grid_constant__ CUtensorMap tb, float *__restrict__ C,
                int M, int N, int K, int cps, int *status) {
    using G = Cfg<BN>;
    constexpr int S = G::kStages;
    extern __shared__ uint8_t smem_raw[];
    uint8_t *sm = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
    __shared__ uint64_t full[S], empty[S], done;
    __shared__ uint32_t tmem_slot;
    __shared__ int s_fail, s_issued, s_consumed;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int m0 = blockIdx.x * kBM, n0 = blockIdx.y * BN;
    const int kc0 = blockIdx.z * cps;
    const int kchunks = min(K / kBK, kc0 + cps) - kc0;
    C += (size_t)blockIdx.z * M * N;
    if (warp == 1) tc::alloc(&tmem_slot, G::kTmemCols);
    if (tid == 0) {
        for (int q = 0; q < S; ++q) {
            tma::mbar_init(&full[q], 1);
            tma::mbar_init(&empty[q], 1);
        }
        tma::mbar_init(&done, 1);
        s_fail = 0;
        s_issued = 0;
        s_consumed = 0;
        tma::fence_barrier_init();
    }
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    const uint32_t tmem = tmem_slot;
    auto stage_a = [&](int s) { return sm + s * G::kStage; };
    if (warp == 0) {
        if (lane == 0) {                                   // TMA producer
            int kc = 0;
            for (; kc < kchunks; ++kc) {
                const int s = kc % S;
                if (kc >= S && !tma::mbar_wait(&empty[s], ((kc / S) - 1) & 1)) {
                    s_fail = 1;
                    break;
                }
                tma::mbar_expect_tx(&full[s], G::kStage);
                tma::load_2d(stage_a(s), &ta, (kc0 + kc) * kBK, m0, &full[s]);
                tma::load_2d(stage_a(s) + kABytes, &tb, (kc0 + kc) * kBK, n0, &full[s]);
            }
            s_issued = kc;
        }
    } else if (warp == 1) {
        if (lane == 0 && kchunks > 0) {                    // MMA issuer
            constexpr uint32_t idesc = tc::idesc_bf16_f32(kBM, BN);
            int kc = 0;
            for (; kc < kchunks; ++kc) {
                const int s = kc % S;
                if (!tma::mbar_wait(&full[s], (kc / S) & 1)) {
                    s_fail = 1;
                    break;
                }
                tc::fence_after();
                const uint32_t a0 = tc::smem_addr(stage_a(s)), b0 = a0 + kABytes;
#pragma unroll
                for (int ks = 0; ks < kBK / 16; ++ks)
                    tc::mma_bf16(tmem, tc::smem_desc_sw128(a0 + ks * 32), tc::smem_desc_sw128(b0 + ks * 32), idesc,
                                 (uint32_t)((kc | ks) != 0));
                tc::commit(&empty[s]);                     // stage s free once these MMAs are done
            }
            s_consumed = kc;
            tc::commit(&done);                             // every MMA issued above
        }
    } else {                                               // epilogue: warps 2..5
        const int q = warp & 3;                            // TMEM lanes 32 q .. 32 q + 31
        float *crow = C + (size_t)(m0 + 32 * q + lane) * N + n0;
        if (kchunks <= 0) {                                // empty slice: a zero partial
            for (int c = 0; c < BN; c += 4) *reinterpret_cast<float4 *>(crow + c) = make_float4(0.f, 0.f, 0.f, 0.f);
        } else {
            bool w = true;
            if (lane == 0) w = tma::mbar_wait(&done, 0);
            w = __shfl_sync(0xffffffffu, (int)w, 0) != 0;
            __syncwarp();
            tc::fence_after();
            if (!w) s_fail = 1;
            else {
                const uint32_t lane_addr = tmem + ((uint32_t)(32 * q) << 16);
#pragma unroll 1
                for (int ch = 0; ch < BN / 32; ++ch) {
                    uint32_t v[32];
                    tc::ld_32cols(lane_addr + ch * 32, v);
                    tc::wait_ld();
#pragma unroll
                    for (int e = 0; e < 8; ++e)
                        reinterpret_cast<float4 *>(crow + ch * 32)[e] =
                            make_float4(__uint_as_float(v[4 * e]), __uint_as_float(v[4 * e + 1]),
                                        __uint_as_float(v[4 * e + 2]), __uint_as_float(v[4 * e + 3]));
                }
            }
        }
    }
    tc::fence_before();
    __syncthreads();
    if (s_fail && tid == 0) {
        atomicExch(status, 1);
        // loads issued but never consumed, then the MMAs (bounded waits)
        for (int kc = s_consumed; kc < s_issued; ++kc) tma::mbar_wait(&full[kc % S], (kc / S) & 1);
        if (kchunks > 0) tma::mbar_wait(&done, 0);
    }
    __syncthreads();
    if (warp == 1) {
        tc::fence_after();
        tc::dealloc(tmem, G::kTmemCols);
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

template <int BN>
int launch_bn(const CUtensorMap &ta, const void *B, float *C, int M, int N, int K, int cps, int slices,
              int *d_status, cudaStream_t st) {
    using G = Cfg<BN>;
    CUtensorMap tb;
    int rc = encode_2d(&tb, const_cast<void *>(B), CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, (uint64_t)K, (uint64_t)N,
                       kBK, BN, CU_TENSOR_MAP_SWIZZLE_128B);
    if (rc) return rc;
    dim3 grid(M / kBM, N / BN, slices);
    k_gemm_bf16<BN><<<grid, kThreads, G::kSmem, st>>>(ta, tb, C, M, N, K, cps, d_status);
    PM_LAUNCHED("k_gemm_bf16");
    return PTYCHO_OK;
}

int gemm_bf16_launch(const void *A, const void *B, float *C, int M, int N, int K, int *d_status, cudaStream_t st,
                     float *work, size_t work_floats) {
    if (M % kBM || N % 64 || K % kBK || M < 0 || N < 0 || K < 0)
        return fail(PTYCHO_EINVAL, "gemm_bf16: M %% 128, N %% 64, K %% 64 must be 0 (M=%d N=%d K=%d)", M, N, K);
    if (M == 0 || N == 0) return PTYCHO_OK;
    if ((reinterpret_cast<uintptr_t>(A) | reinterpret_cast<uintptr_t>(B)) & 15)
        return fail(PTYCHO_EINVAL, "gemm_bf16: A and B must be 16-byte aligned");
    int dev = 0;
    PM_CUDA(cudaGetDevice(&dev));
    {
        std::lock_guard<std::mutex> lk(g_attr_mu);
        if (dev >= 64 || !g_attr_set[dev]) {
            PM_CUDA(cudaFuncSetAttribute(k_gemm_bf16<256>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)Cfg<256>::kSmem));
            PM_CUDA(cudaFuncSetAttribute(k_gemm_bf16<192>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)Cfg<192>::kSmem));
            PM_CUDA(cudaFuncSetAttribute(k_gemm_bf16<128>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)Cfg<128>::kSmem));
            PM_CUDA(cudaFuncSetAttribute(k_gemm_bf16<64>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)Cfg<64>::kSmem));
            if (dev < 64) g_attr_set[dev] = true;
        }
    }
    if (K == 0) {
        PM_CUDA(cudaMemsetAsync(C, 0, (size_t)M * N * sizeof(float), st));
        return PTYCHO_OK;
    }
    // Tile width: the kernels are bound by operand traffic, which per K step is (128 + BN) rows
    // for 128 BN outputs.  With a split-K workspace every width can fill the GPU, so the widest
    // that divides N; otherwise the width with the least (waves of CTAs) x (128 + BN).
    const int kch = K / kBK;
    const bool can_split = work && kch >= 8;
    int BN = 64;
    long best = -1;
    for (int cand : {256, 192, 128, 64}) {
        if (N % cand) continue;
        const long t = (long)(M / kBM) * (N / cand);
        const long cost = can_split ? 0 : ((t + 147) / 148) * (128 + cand);
        if (best < 0 || cost < best) { best = cost; BN = cand; }
    }
    // split K when the output tiles alone cannot fill the GPU (weight gradients: small M x N,
    // K = every pixel of the batch)
    const int tiles = (M / kBM) * (N / BN);
    int slices = 1;
    if (can_split && tiles < 296) {
        slices = std::min(std::min((296 + tiles - 1) / tiles, kch / 4), 64);
        while (slices > 1 && (size_t)slices * M * N > work_floats) --slices;
    }
    const int cps = (kch + slices - 1) / slices;
    CUtensorMap ta;
    int rc = encode_2d(&ta, const_cast<void *>(A), CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, (uint64_t)K, (uint64_t)M, kBK,
                       kBM, CU_TENSOR_MAP_SWIZZLE_128B);
    if (rc) return rc;
    float *dst = slices > 1 ? work : C;
    if (BN == 256) rc = launch_bn<256>(ta, B, dst, M, N, K, cps, slices, d_status, st);
    else if (BN == 192) rc = launch_bn<192>(ta, B, dst, M, N, K, cps, slices, d_status, st);
    else if (BN == 128) rc = launch_bn<128>(ta, B, dst, M, N, K, cps, slices, d_status, st);
    else rc = launch_bn<64>(ta, B, dst, M, N, K, cps, slices, d_status, st);
    if (rc) return rc;
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
