// Multi-Scale Non-Linear Fusion (MNF) of multi-exposure diffraction brackets, §3.4.
//
// Per position j the method builds, for every exposure k, Gaussian pyramids of the radiance
// E_k and of the normalised exposure weight W_k (Eq. 5, Eq. 6), the Laplacian pyramid of E_k
// (Eq. 7), modulates and quantises the details (Eq. 8), collapses each exposure (Eq. 9) and
// sums the collapsed images (Eq. 10).  Because U2 is linear, sum_k R_0^(k) equals one collapse
// of the per-level sums sum_k Ltilde_l^(k) on top of the summed base, so the kernels below
// accumulate over k per level and collapse once:
//
//   reduce0      raw counts -> (E_k, W_k) at level 0 -> G_1[E_k], G_1[W_k]  (shared-memory tile)
//   reduce(l)    G_l -> G_{l+1} for E and W                                   (l = 1 .. L-2)
//   base         R_{L-1} = sum_k base_k(G_{L-1}[E_k], G_{L-1}[W_k])
//   collapse(l)  R_l = U2(R_{l+1}) + sum_k Q_l(G_l[W_k] (G_l[E_k] - U2(G_{l+1}[E_k])))
//                (l = L-2 .. 1 into scratch, l = 0 from the raw counts into the output)
//
// Level-0 planes are never stored: E and W there are pointwise functions of the K raw counts.
// Filters: w_G = [1,4,6,4,1]/16 per axis, D2 keeps even samples, U2 is zero insertion then
// 2 w_G per axis, reflect-101 borders on the grid being filtered.  All arithmetic is FP32.
#include <algorithm>
#include <cmath>
#include <mutex>
#include <vector>

#include "common.cuh"

namespace {

constexpr int kMaxK = 8;
constexpr int kMaxLevels = 11;

struct FuseDev {
    float mu, inv2s2, clip, inv_clip;
    float tscale[kMaxK];        // E_k = I_k * tscale[k]
    float delta[kMaxLevels];    // quantiser step per level (0 = off)
    float inv_delta[kMaxLevels];
    int N, L, base_mode;
};

__device__ __forceinline__ int refl(int i, int n) {
    // reflect-101 for i in [-(n-1), 2n-2]
    return i < 0 ? -i : (i >= n ? 2 * n - 2 - i : i);
}

__device__ __forceinline__ float wg(int a) {
    // w_G = [1, 4, 6, 4, 1] / 16
    return a == 2 ? 0.375f : ((a == 1 || a == 3) ? 0.25f : 0.0625f);
}

// Exposure weights (Eq. 5, normalised over k) and radiance of one level-0 pixel from its K
// raw counts.
template <int K>
__device__ __forceinline__ void level0_counts(const uint16_t (&c)[K], const FuseDev &f, float (&E)[K],
                                              float (&W)[K]) {
    // FP32 with reciprocal multiplications in place of the divisions by the clip level and by
    // the weight sum (each adds at most one rounding to a value the FP64 oracle forms exactly)
    float s = 0.f;
#pragma unroll
    for (int k = 0; k < K; ++k) {
        const float v = (float)c[k];
        E[k] = v * f.tscale[k];
        const float d = fminf(v, f.clip) * f.inv_clip - f.mu;
        W[k] = expf(-d * d * f.inv2s2);
        s += W[k];
    }
    const float inv_s = (s > 0.f) ? 1.0f / s : 0.f;
#pragma unroll
    for (int k = 0; k < K; ++k) W[k] = (s > 0.f) ? W[k] * inv_s : 1.0f / K;
}

template <int K>
__device__ __forceinline__ void level0_pixel(const uint16_t *raw_j, size_t NN, size_t p,
                                             const FuseDev &f, float (&E)[K], float (&W)[K]) {
    uint16_t c[K];
#pragma unroll
    for (int k = 0; k < K; ++k) c[k] = __ldg(raw_j + k * NN + p);
    level0_counts<K>(c, f, E, W);
}

// Delta rint(x / Delta), the ratio formed with the reciprocal of Delta (0 = no quantiser).
__device__ __forceinline__ float quantise(float x, float delta, float inv_delta) {
    return delta > 0.f ? delta * rintf(x * inv_delta) : x;
}

constexpr int kTile = 16;             // outputs per block side of a reduce
constexpr int kIn = 2 * kTile + 3;    // input rows/cols a tile needs
constexpr int kInP = kIn + 1;         // padded pitch

// Level 0 -> level 1 for every exposure: blockIdx.z = position, tile of 16 x 16 outputs.
// Each input pixel's K weights (Eq. 5, normalised) and radiances are computed once into shared
// memory, then every plane is blurred separably (rows, then columns) and decimated.  FULL: a
// whole 16 x 16 tile, whose loop bounds are compile-time constants (the index divisions become
// multiply-shifts); the partial tiles at the edge of an N / 2 not divisible by 16 take the
// general body.  Both compute the same values.
template <int K, bool FULL>
__device__ __forceinline__ void reduce0_body(const uint16_t *__restrict__ raw, float *__restrict__ ge1,
                                             float *__restrict__ gw1, const FuseDev &f, float *sm, int outs_y,
                                             int outs_x) {
    float *s_e = sm;                              // [K][kIn][kInP]
    float *s_w = s_e + K * kIn * kInP;            // [K][kIn][kInP]
    float *h_e = s_w + K * kIn * kInP;            // [K][kIn][kTile]  row-filtered, decimated
    float *h_w = h_e + K * kIn * kTile;
    const int N = f.N, n1 = N >> 1;
    const size_t NN = (size_t)N * N;
    const int j = blockIdx.z;
    const uint16_t *raw_j = raw + (size_t)j * K * NN;
    const int oy0 = blockIdx.y * kTile, ox0 = blockIdx.x * kTile;
    if (FULL) {
        outs_y = kTile;
        outs_x = kTile;
    }
    const int rows = 2 * outs_y + 3, cols = 2 * outs_x + 3;
    const int tid = threadIdx.x;
    if (FULL) {
        // every raw count of this thread's pixels first (all loads in flight together), then
        // the weights and radiances (blockDim.x = 256)
        constexpr int kPix = kIn * kIn, kPer = (kPix + 255) / 256;
        uint16_t c[kPer][K];
#pragma unroll
        for (int i = 0; i < kPer; ++i) {
            const int e = tid + 256 * i;
            if (e < kPix) {
                const int a = e / kIn, b = e % kIn;
                const size_t p = (size_t)refl(2 * oy0 - 2 + a, N) * N + refl(2 * ox0 - 2 + b, N);
#pragma unroll
                for (int k = 0; k < K; ++k) c[i][k] = __ldg(raw_j + k * NN + p);
            }
        }
#pragma unroll
        for (int i = 0; i < kPer; ++i) {
            const int e = tid + 256 * i;
            if (e < kPix) {
                const int a = e / kIn, b = e % kIn;
                float E[K], W[K];
                level0_counts<K>(c[i], f, E, W);
#pragma unroll
                for (int k = 0; k < K; ++k) {
                    s_e[(k * kIn + a) * kInP + b] = E[k];
                    s_w[(k * kIn + a) * kInP + b] = W[k];
                }
            }
        }
    } else {
        for (int e = tid; e < rows * cols; e += blockDim.x) {
            const int a = e / cols, b = e % cols;
            const size_t p = (size_t)refl(2 * oy0 - 2 + a, N) * N + refl(2 * ox0 - 2 + b, N);
            float E[K], W[K];
            level0_pixel<K>(raw_j, NN, p, f, E, W);
#pragma unroll
            for (int k = 0; k < K; ++k) {
                s_e[(k * kIn + a) * kInP + b] = E[k];
                s_w[(k * kIn + a) * kInP + b] = W[k];
            }
        }
    }
    __syncthreads();
    // rows: h[k][a][ox] = sum_b w[b] x[k][a][2 ox + b]
    for (int e = tid; e < K * rows * outs_x; e += blockDim.x) {
        const int ox = e % outs_x, a = (e / outs_x) % rows, k = e / (outs_x * rows);
        const float *re = s_e + (k * kIn + a) * kInP + 2 * ox;
        const float *rw = s_w + (k * kIn + a) * kInP + 2 * ox;
        float ae = 0.f, aw = 0.f;
#pragma unroll
        for (int b = 0; b < 5; ++b) {
            ae += wg(b) * re[b];
            aw += wg(b) * rw[b];
        }
        h_e[(k * kIn + a) * kTile + ox] = ae;
        h_w[(k * kIn + a) * kTile + ox] = aw;
    }
    __syncthreads();
    // columns: out[k][oy][ox] = sum_a w[a] h[k][2 oy + a][ox]
    const size_t n1n1 = (size_t)n1 * n1;
    for (int e = tid; e < K * outs_y * outs_x; e += blockDim.x) {
        const int ox = e % outs_x, oy = (e / outs_x) % outs_y, k = e / (outs_x * outs_y);
        float ae = 0.f, aw = 0.f;
#pragma unroll
        for (int a = 0; a < 5; ++a) {
            ae += wg(a) * h_e[(k * kIn + 2 * oy + a) * kTile + ox];
            aw += wg(a) * h_w[(k * kIn + 2 * oy + a) * kTile + ox];
        }
        const size_t o = ((size_t)j * K + k) * n1n1 + (size_t)(oy0 + oy) * n1 + ox0 + ox;
        ge1[o] = ae;
        gw1[o] = aw;
    }
}

template <int K>
__global__ void __launch_bounds__(256) k_reduce0(const uint16_t *__restrict__ raw,
                                                 float *__restrict__ ge1, float *__restrict__ gw1,
                                                 FuseDev f) {
    extern __shared__ float sm[];
    const int n1 = f.N >> 1;
    const int outs_y = min(kTile, n1 - (int)blockIdx.y * kTile), outs_x = min(kTile, n1 - (int)blockIdx.x * kTile);
    if (outs_y == kTile && outs_x == kTile) reduce0_body<K, true>(raw, ge1, gw1, f, sm, outs_y, outs_x);
    else reduce0_body<K, false>(raw, ge1, gw1, f, sm, outs_y, outs_x);
}

template <int K>
constexpr size_t reduce0_smem() {
    return sizeof(float) * (size_t)K * (2 * kIn * kInP + 2 * kIn * kTile);
}

// Level l -> l+1 (l >= 1) for one plane pair: blockIdx.z = j * K + k.
__global__ void __launch_bounds__(256) k_reduce(const float *__restrict__ ge, const float *__restrict__ gw,
                                                float *__restrict__ ge_next, float *__restrict__ gw_next,
                                                int n) {
    __shared__ float s_e[kIn * kInP];
    __shared__ float s_w[kIn * kInP];
    const int m = n >> 1;
    const size_t plane = blockIdx.z;
    const float *e_in = ge + plane * n * n, *w_in = gw + plane * n * n;
    const int oy0 = blockIdx.y * kTile, ox0 = blockIdx.x * kTile;
    const int outs_y = min(kTile, m - oy0), outs_x = min(kTile, m - ox0);
    const int rows = 2 * outs_y + 3, cols = 2 * outs_x + 3;
    const int tid = threadIdx.x;
    for (int e = tid; e < rows * cols; e += blockDim.x) {
        const int a = e / cols, b = e % cols;
        const size_t p = (size_t)refl(2 * oy0 - 2 + a, n) * n + refl(2 * ox0 - 2 + b, n);
        s_e[a * kInP + b] = __ldg(e_in + p);
        s_w[a * kInP + b] = __ldg(w_in + p);
    }
    __syncthreads();
    const int ty = tid / kTile, tx = tid % kTile;
    if (ty < outs_y && tx < outs_x) {
        float ae = 0.f, aw = 0.f;
#pragma unroll
        for (int a = 0; a < 5; ++a) {
            float re = 0.f, rw = 0.f;
#pragma unroll
            for (int b = 0; b < 5; ++b) {
                re += wg(b) * s_e[(2 * ty + a) * kInP + 2 * tx + b];
                rw += wg(b) * s_w[(2 * ty + a) * kInP + 2 * tx + b];
            }
            ae += wg(a) * re;
            aw += wg(a) * rw;
        }
        const size_t o = plane * m * m + (size_t)(oy0 + ty) * m + ox0 + tx;
        ge_next[o] = ae;
        gw_next[o] = aw;
    }
}

template <int K>
__device__ __forceinline__ float base_value(const float (&E)[K], const float (&W)[K], int mode) {
    float b = 0.f;
#pragma unroll
    for (int k = 0; k < K; ++k) {
        if (mode == PTYCHO_BASE_WEIGHTED) b += W[k] * E[k];
        else b += E[k];
    }
    return mode == PTYCHO_BASE_MEAN ? b / K : b;
}

// Base of the collapse at the coarsest level: from planes (L >= 2) or from raw (L == 1,
// then written straight to the output).  One thread per (j, pixel).
template <int K>
__global__ void k_base(const float *__restrict__ ge, const float *__restrict__ gw,
                       const uint16_t *__restrict__ raw, float *__restrict__ out, int n, int J,
                       FuseDev f) {
    const size_t nn = (size_t)n * n;
    const size_t total = (size_t)J * nn;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total;
         i += (size_t)gridDim.x * blockDim.x) {
        const size_t j = i / nn, p = i % nn;
        float E[K], W[K];
        if (raw) {
            level0_pixel<K>(raw + j * K * nn, nn, p, f, E, W);
        } else {
#pragma unroll
            for (int k = 0; k < K; ++k) {
                E[k] = __ldg(ge + (j * K + k) * nn + p);
                W[k] = __ldg(gw + (j * K + k) * nn + p);
            }
        }
        out[i] = base_value<K>(E, W, f.base_mode);
    }
}

// R_l = U2(R_{l+1}) + sum_k Q_l(G_l[W_k] (G_l[E_k] - U2(G_{l+1}[E_k]))); level 0 reads raw.
// One block per 32 x 32 output tile of one position: the 18 x 18 coarse neighbourhoods of
// R_{l+1} and G_{l+1}[E_k] are staged in shared memory with U2's border extension (coarse
// index -1 -> 1, n -> n - 1) applied while loading.  One thread per 2 x 2 output quad: output
// 2i takes coarse i - 1, i, i + 1 with weights (1/8, 3/4, 1/8) and 2i + 1 takes i, i + 1 with
// (1/2, 1/2) (written as three taps with a zero lead), so the quad's four pixels share one
// 3 x 3 coarse neighbourhood per plane: each coarse row is filtered along x once per column
// parity, then along y once per pixel, in the same order and with the same FMAs as a
// pixel-by-pixel evaluation.
constexpr int kCT = 32;                 // output tile side of the collapse
constexpr int kCC = kCT / 2 + 2;        // coarse rows / columns the tile needs
constexpr int kCP = 48;                 // row pitch: the two quad rows of a warp hit distinct banks

__device__ __forceinline__ int coarse_ext(int i, int n) { return i < 0 ? 1 : min(i, n - 1); }

template <int K>
__global__ void __launch_bounds__(256) k_collapse(const float *__restrict__ ge, const float *__restrict__ gw,
                                                  const uint16_t *__restrict__ raw, const float *__restrict__ ge_next,
                                                  const float *__restrict__ r_next, float *__restrict__ out, int n,
                                                  float delta, float inv_delta, FuseDev f) {
    __shared__ float s_c[K + 1][kCC][kCP];              // [0..K-1] G_{l+1}[E_k], [K] R_{l+1}
    const int m = n >> 1;
    const size_t nn = (size_t)n * n, mm = (size_t)m * m;
    const int j = blockIdx.z;
    const int oy0 = blockIdx.y * kCT, ox0 = blockIdx.x * kCT;
    const int cy0 = oy0 / 2 - 1, cx0 = ox0 / 2 - 1;
    for (int e = threadIdx.x; e < (K + 1) * kCC * kCC; e += blockDim.x) {
        const int pl = e / (kCC * kCC), a = (e / kCC) % kCC, b = e % kCC;
        const size_t src = (size_t)coarse_ext(cy0 + a, m) * m + coarse_ext(cx0 + b, m);
        s_c[pl][a][b] = (pl < K) ? __ldg(ge_next + ((size_t)j * K + pl) * mm + src) : __ldg(r_next + (size_t)j * mm + src);
    }
    __syncthreads();
    const int qy = threadIdx.x / (kCT / 2), qx = threadIdx.x % (kCT / 2);
    const int py0 = oy0 + 2 * qy, px0 = ox0 + 2 * qx;
    if (py0 >= n || px0 >= n) return;
    // coarse neighbourhood of the quad: rows / columns qy .. qy + 2, qx .. qx + 2 of the stage
    // (output 2i has i - 1 at stage index i - cy0 - 1 = qy)
    constexpr float we[3] = {0.125f, 0.75f, 0.125f}, wo[3] = {0.f, 0.5f, 0.5f};
    float up[K + 1][2][2];                              // [plane][dy][dx]
#pragma unroll
    for (int pl = 0; pl <= K; ++pl) {
        float rx[3][2];                                 // coarse row a filtered along x, column parity
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            const float *row = &s_c[pl][qy + a][qx];
            float re = 0.f, ro = 0.f;
#pragma unroll
            for (int b = 0; b < 3; ++b) {
                re += we[b] * row[b];
                ro += wo[b] * row[b];
            }
            rx[a][0] = re;
            rx[a][1] = ro;
        }
#pragma unroll
        for (int dx = 0; dx < 2; ++dx) {
            float ae = 0.f, ao = 0.f;
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                ae += we[a] * rx[a][dx];
                ao += wo[a] * rx[a][dx];
            }
            up[pl][0][dx] = ae;
            up[pl][1][dx] = ao;
        }
    }
#pragma unroll
    for (int dy = 0; dy < 2; ++dy)
#pragma unroll
        for (int dx = 0; dx < 2; ++dx) {
            const int py = py0 + dy, px = px0 + dx;
            if (py >= n || px >= n) continue;
            const size_t p = (size_t)py * n + px;
            float E[K], W[K];
            if (raw) {
                level0_pixel<K>(raw + (size_t)j * K * nn, nn, p, f, E, W);
            } else {
#pragma unroll
                for (int k = 0; k < K; ++k) {
                    E[k] = __ldg(ge + ((size_t)j * K + k) * nn + p);
                    W[k] = __ldg(gw + ((size_t)j * K + k) * nn + p);
                }
            }
            float acc = 0.f;
#pragma unroll
            for (int k = 0; k < K; ++k) acc += quantise(W[k] * (E[k] - up[k][dy][dx]), delta, inv_delta);
            out[(size_t)j * nn + p] = up[K][dy][dx] + acc;
        }
}

unsigned grid_for(size_t total, int threads) {
    size_t b = (total + threads - 1) / threads;
    return (unsigned)std::min<size_t>(std::max<size_t>(b, 1), 148u * 64u);
}

template <int K>
int run_fuse(const uint16_t *d_raw, int J, int N, const FuseDev &f, float *d_fused,
             float *scratch, cudaStream_t st) {
    const int L = f.L;
    if (reduce0_smem<K>() > 48 * 1024)
        PM_CUDA(cudaFuncSetAttribute(k_reduce0<K>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)reduce0_smem<K>()));
    if (L == 1) {
        const size_t total = (size_t)J * N * N;
        k_base<K><<<grid_for(total, 256), 256, 0, st>>>(nullptr, nullptr, d_raw, d_fused, N, J, f);
        PM_LAUNCHED("k_base");
        return PTYCHO_OK;
    }
    // scratch layout per level l >= 1: GE_l [J][K][n_l^2], GW_l [J][K][n_l^2], R_l [J][n_l^2]
    float *ge[kMaxLevels] = {}, *gw[kMaxLevels] = {}, *rr[kMaxLevels] = {};
    float *cur = scratch;
    for (int l = 1; l < L; ++l) {
        const size_t nl2 = (size_t)(N >> l) * (N >> l);
        ge[l] = cur; cur += (size_t)J * K * nl2;
        gw[l] = cur; cur += (size_t)J * K * nl2;
        rr[l] = cur; cur += (size_t)J * nl2;
    }
    {
        const int n1 = N >> 1;
        dim3 grid((n1 + kTile - 1) / kTile, (n1 + kTile - 1) / kTile, J);
        k_reduce0<K><<<grid, 256, reduce0_smem<K>(), st>>>(d_raw, ge[1], gw[1], f);
        PM_LAUNCHED("k_reduce0");
    }
    for (int l = 1; l + 1 < L; ++l) {
        const int n = N >> l, m = n >> 1;
        dim3 grid((m + kTile - 1) / kTile, (m + kTile - 1) / kTile, J * K);
        k_reduce<<<grid, 256, 0, st>>>(ge[l], gw[l], ge[l + 1], gw[l + 1], n);
        PM_LAUNCHED("k_reduce");
    }
    {
        const int n = N >> (L - 1);
        const size_t total = (size_t)J * n * n;
        k_base<K><<<grid_for(total, 256), 256, 0, st>>>(ge[L - 1], gw[L - 1], nullptr, rr[L - 1], n, J, f);
        PM_LAUNCHED("k_base");
    }
    for (int l = L - 2; l >= 0; --l) {
        const int n = N >> l;
        dim3 grid((n + kCT - 1) / kCT, (n + kCT - 1) / kCT, J);
        if (l == 0) {
            k_collapse<K><<<grid, 256, 0, st>>>(nullptr, nullptr, d_raw, ge[1], rr[1], d_fused, n, f.delta[0],
                                                f.inv_delta[0], f);
        } else {
            k_collapse<K><<<grid, 256, 0, st>>>(ge[l], gw[l], nullptr, ge[l + 1], rr[l + 1], rr[l], n, f.delta[l],
                                                f.inv_delta[l], f);
        }
        PM_LAUNCHED("k_collapse");
    }
    return PTYCHO_OK;
}

size_t scratch_floats_per_position(int K, int N, int L) {
    size_t s = 0;
    for (int l = 1; l < L; ++l) s += (size_t)(2 * K + 1) * (N >> l) * (N >> l);
    return s;
}

bool is_pow2(int n) { return n > 0 && (n & (n - 1)) == 0; }

}  // namespace

namespace pm {

int validate_fuse(const uint16_t *d_raw, int J, int K, int N, const float *h_t,
                  const fuse_params *p, float *d_fused, FuseDev *out) {
    if (!p) return fail(PTYCHO_EINVAL, "fuse_stack: params is NULL");
    if (J < 0) return fail(PTYCHO_EINVAL, "fuse_stack: J = %d < 0", J);
    if (K < 1 || K > kMaxK) return fail(PTYCHO_EINVAL, "fuse_stack: K = %d not in [1, %d]", K, kMaxK);
    if (!is_pow2(N) || N < 8 || N > 1024)
        return fail(PTYCHO_EINVAL, "fuse_stack: N = %d is not a power of two in [8, 1024]", N);
    if (p->levels < 1 || p->levels > kMaxLevels || (N >> (p->levels - 1)) < 4)
        return fail(PTYCHO_EINVAL, "fuse_stack: levels = %d needs N / 2^(L-1) >= 4 (N = %d)", p->levels, N);
    if (!(p->sigma > 0.f) || !std::isfinite(p->sigma) || !std::isfinite(p->mu))
        return fail(PTYCHO_EINVAL, "fuse_stack: sigma must be finite and > 0, mu finite");
    if (!(p->clip > 0.f) || !std::isfinite(p->clip)) return fail(PTYCHO_EINVAL, "fuse_stack: clip must be finite and > 0");
    if (!(p->delta0 >= 0.f) || !std::isfinite(p->delta0) || !(p->delta_ratio > 0.f) || !std::isfinite(p->delta_ratio))
        return fail(PTYCHO_EINVAL, "fuse_stack: delta0 >= 0 and delta_ratio > 0 required");
    if (p->base_mode < PTYCHO_BASE_MEAN || p->base_mode > PTYCHO_BASE_WEIGHTED)
        return fail(PTYCHO_EINVAL, "fuse_stack: unknown base_mode %d", p->base_mode);
    if (p->domain != PTYCHO_DOMAIN_RADIANCE && p->domain != PTYCHO_DOMAIN_RAW)
        return fail(PTYCHO_EINVAL, "fuse_stack: unknown domain %d", p->domain);
    if (!h_t) return fail(PTYCHO_EINVAL, "fuse_stack: exposure times pointer is NULL");
    float tmax = 0.f;
    for (int k = 0; k < K; ++k) {
        if (!(h_t[k] > 0.f) || !std::isfinite(h_t[k]))
            return fail(PTYCHO_EINVAL, "fuse_stack: t[%d] = %g must be finite and > 0", k, (double)h_t[k]);
        tmax = std::max(tmax, h_t[k]);
    }
    if (J > 0 && (!d_raw || !d_fused)) return fail(PTYCHO_EINVAL, "fuse_stack: NULL raw or output pointer");
    FuseDev f{};
    f.mu = p->mu;
    f.inv2s2 = (float)(1.0 / (2.0 * (double)p->sigma * (double)p->sigma));
    f.clip = p->clip;
    f.inv_clip = (float)(1.0 / (double)p->clip);
    for (int k = 0; k < K; ++k)
        f.tscale[k] = (p->domain == PTYCHO_DOMAIN_RAW) ? 1.0f : (float)((double)tmax / (double)h_t[k]);
    for (int l = 0; l < kMaxLevels; ++l)
        f.delta[l] = (float)((double)p->delta0 * std::pow((double)p->delta_ratio, (double)l));
    for (int l = 0; l < kMaxLevels; ++l) f.inv_delta[l] = f.delta[l] > 0.f ? (float)(1.0 / (double)f.delta[l]) : 0.f;
    f.N = N;
    f.L = p->levels;
    f.base_mode = p->base_mode;
    *out = f;
    return PTYCHO_OK;
}

int fuse_dispatch(const uint16_t *d_raw, int J, int K, int N, const FuseDev &f, float *d_fused,
                  float *scratch, cudaStream_t st) {
    switch (K) {
        case 1: return run_fuse<1>(d_raw, J, N, f, d_fused, scratch, st);
        case 2: return run_fuse<2>(d_raw, J, N, f, d_fused, scratch, st);
        case 3: return run_fuse<3>(d_raw, J, N, f, d_fused, scratch, st);
        case 4: return run_fuse<4>(d_raw, J, N, f, d_fused, scratch, st);
        case 5: return run_fuse<5>(d_raw, J, N, f, d_fused, scratch, st);
        case 6: return run_fuse<6>(d_raw, J, N, f, d_fused, scratch, st);
        case 7: return run_fuse<7>(d_raw, J, N, f, d_fused, scratch, st);
        default: return run_fuse<8>(d_raw, J, N, f, d_fused, scratch, st);
    }
}

}  // namespace pm

extern "C" int fuse_stack(const uint16_t *d_raw, int J, int K, int N, const float *h_t,
                          const fuse_params *p, float *d_fused, void *cuda_stream) {
    pm::NvtxRange range("fuse_stack");
    FuseDev f;
    int rc = pm::validate_fuse(d_raw, J, K, N, h_t, p, d_fused, &f);
    if (rc != PTYCHO_OK || J == 0) return rc;
    cudaStream_t st = (cudaStream_t)cuda_stream;
    const size_t per_pos = scratch_floats_per_position(K, N, f.L);
    // Positions are independent: process them in chunks whose scratch stays below 2 GiB.
    const size_t cap_floats = ((size_t)2 << 30) / sizeof(float);
    int chunk = J;
    if (per_pos > 0) chunk = (int)std::max<size_t>(1, std::min<size_t>((size_t)J, cap_floats / per_pos));
    chunk = std::min(chunk, 65535 / K);           // grid.z of the reduce kernels is J * K
    float *scratch = nullptr;
    if (per_pos > 0) PM_CUDA(pm::dev_malloc_async((void **)&scratch, per_pos * chunk * sizeof(float), st));
    const size_t NN = (size_t)N * N;
    for (int j0 = 0; j0 < J && rc == PTYCHO_OK; j0 += chunk) {
        const int jn = std::min(chunk, J - j0);
        rc = pm::fuse_dispatch(d_raw + (size_t)j0 * K * NN, jn, K, N, f, d_fused + (size_t)j0 * NN, scratch, st);
    }
    if (scratch) {
        cudaError_t e = cudaFreeAsync(scratch, st);
        if (rc == PTYCHO_OK && e != cudaSuccess) return pm::cuda_fail(e, "cudaFreeAsync");
    }
    return rc;
}

// ---------------------------------------------------------------------------------------
// Fusion from a host-resident stack: the copies of chunks of positions run on a copy stream of
// the library (one per device, created on first use) and the fusion of each chunk on the
// caller's stream as soon as that chunk has landed, so the copy of chunk c + 1 overlaps the
// fusion of chunk c.  The copy stream first waits for the caller's stream (d_raw may still be in
// use by earlier work), and the caller's stream waits for every copy before it fuses.
namespace {

std::mutex g_copy_mu;
cudaStream_t g_copy_stream[64] = {};

int copy_stream(cudaStream_t *out) {
    int dev = 0;
    PM_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64) return pm::fail(PTYCHO_EINVAL, "fuse_stack_host: device %d out of range", dev);
    std::lock_guard<std::mutex> lk(g_copy_mu);
    if (!g_copy_stream[dev]) PM_CUDA(cudaStreamCreateWithFlags(&g_copy_stream[dev], cudaStreamNonBlocking));
    *out = g_copy_stream[dev];
    return PTYCHO_OK;
}

}  // namespace

extern "C" int fuse_stack_host(const uint16_t *h_raw, uint16_t *d_raw, int J, int K, int N, const float *h_t,
                               const fuse_params *p, float *d_fused, int chunk_positions, void *cuda_stream) {
    pm::NvtxRange range("fuse_stack_host");
    FuseDev f;
    int rc = pm::validate_fuse(d_raw, J, K, N, h_t, p, d_fused, &f);
    if (rc != PTYCHO_OK || J == 0) return rc;
    if (!h_raw) return pm::fail(PTYCHO_EINVAL, "fuse_stack_host: host raw pointer is NULL");
    if (chunk_positions < 0) return pm::fail(PTYCHO_EINVAL, "fuse_stack_host: chunk_positions %d < 0", chunk_positions);
    cudaStream_t st = (cudaStream_t)cuda_stream, cs = nullptr;
    if ((rc = copy_stream(&cs))) return rc;
    const size_t per_pos = scratch_floats_per_position(K, N, f.L);
    const size_t cap_floats = ((size_t)2 << 30) / sizeof(float);
    int chunk = chunk_positions > 0 ? chunk_positions : (J + 7) / 8;          // default: 8 chunks
    if (per_pos > 0) chunk = (int)std::min<size_t>((size_t)chunk, std::max<size_t>(1, cap_floats / per_pos));
    chunk = std::max(1, std::min(std::min(chunk, J), 65535 / K));
    const int nchunks = (J + chunk - 1) / chunk;
    const size_t NN = (size_t)N * N, pos_elems = (size_t)K * NN;
    std::vector<cudaEvent_t> ev(nchunks + 1, nullptr);
    auto cleanup = [&]() {
        for (cudaEvent_t e : ev)
            if (e) cudaEventDestroy(e);                        // released once complete
    };
    for (auto &e : ev) {
        const cudaError_t err = cudaEventCreateWithFlags(&e, cudaEventDisableTiming);
        if (err != cudaSuccess) { e = nullptr; cleanup(); return pm::cuda_fail(err, "cudaEventCreate"); }
    }
    cudaError_t err = cudaEventRecord(ev[nchunks], st);
    if (err == cudaSuccess) err = cudaStreamWaitEvent(cs, ev[nchunks], 0);
    for (int c = 0; c < nchunks && err == cudaSuccess; ++c) {
        const int j0 = c * chunk, jn = std::min(chunk, J - j0);
        err = cudaMemcpyAsync(d_raw + (size_t)j0 * pos_elems, h_raw + (size_t)j0 * pos_elems,
                              (size_t)jn * pos_elems * sizeof(uint16_t), cudaMemcpyHostToDevice, cs);
        if (err == cudaSuccess) err = cudaEventRecord(ev[c], cs);
    }
    if (err != cudaSuccess) { cleanup(); return pm::cuda_fail(err, "fuse_stack_host: copies"); }
    float *scratch = nullptr;
    if (per_pos > 0) {
        err = pm::dev_malloc_async((void **)&scratch, per_pos * chunk * sizeof(float), st);
        if (err != cudaSuccess) {
            for (int c = 0; c < nchunks; ++c) cudaStreamWaitEvent(st, ev[c], 0);   // d_raw stays ordered
            cleanup();
            return pm::cuda_fail(err, "fuse_stack_host: scratch");
        }
    }
    for (int c = 0; c < nchunks && rc == PTYCHO_OK; ++c) {
        const int j0 = c * chunk, jn = std::min(chunk, J - j0);
        err = cudaStreamWaitEvent(st, ev[c], 0);
        if (err != cudaSuccess) { rc = pm::cuda_fail(err, "cudaStreamWaitEvent"); break; }
        rc = pm::fuse_dispatch(d_raw + (size_t)j0 * pos_elems, jn, K, N, f, d_fused + (size_t)j0 * NN, scratch, st);
    }
    if (rc != PTYCHO_OK)
        for (int c = 0; c < nchunks; ++c) cudaStreamWaitEvent(st, ev[c], 0);       // later work after every copy
    if (scratch) {
        err = cudaFreeAsync(scratch, st);
        if (rc == PTYCHO_OK && err != cudaSuccess) rc = pm::cuda_fail(err, "cudaFreeAsync");
    }
    cleanup();
    return rc;
}

// ---------------------------------------------------------------------------------------
// Allocation-free variant of fuse_stack.
//
// Some callers cannot call cudaMalloc or any other device allocator: for example code that
// runs while another framework's caching allocator has reserved nearly all device memory, or
// a latency-critical loop in which an allocation (which can synchronise the device) is not
// acceptable.  fuse_stack_noalloc runs the same kernels with its scratch in a fixed,
// file-scope device array instead of stream-ordered allocations.
//
// The array below is part of the library image: every GPU that loads the library holds it
// until the process exits.  Its host-side name is only a stand-in for the symbol, so the
// device address is looked up with cudaGetSymbolAddress with the device current.  A call on a
// stream that is not being captured looks it up again (the address belongs to the device's
// current context, which cudaDeviceReset replaces); a call on a capturing stream uses the
// address the device's last uncaptured call found, so the first call on a device should
// happen before any stream capture, and none should be captured across a cudaDeviceReset.
// All calls share the array and it keeps the previous call's contents (every element a call
// reads is written by that call first, so nothing needs clearing); calls whose work overlaps
// on the GPU race on it.
namespace {
constexpr size_t kNoAllocScratchBytes = (size_t)16 << 20;   // 16 MiB
constexpr int kMaxDevices = 64;
}  // namespace

static __device__ __align__(256) float g_fuse_scratch[kNoAllocScratchBytes / sizeof(float)];

static int noalloc_scratch(float **out, cudaStream_t st) {
    static std::mutex mu;
    static float *by_device[kMaxDevices] = {};
    int dev = 0;
    PM_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kMaxDevices) return pm::fail(PTYCHO_EINVAL, "fuse_stack_noalloc: device %d unsupported", dev);
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    PM_CUDA(cudaStreamIsCapturing(st, &cap));
    std::lock_guard<std::mutex> lock(mu);
    if (cap == cudaStreamCaptureStatusNone) {
        void *p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_fuse_scratch);
        if (e != cudaSuccess) return pm::cuda_fail(e, "cudaGetSymbolAddress(fusion scratch)");
        by_device[dev] = (float *)p;
    } else if (!by_device[dev]) {
        return pm::fail(PTYCHO_EINVAL, "fuse_stack_noalloc: the first call on device %d is being captured; "
                                       "make one uncaptured call on the device first", dev);
    }
    *out = by_device[dev];
    return PTYCHO_OK;
}

extern "C" int fuse_stack_noalloc(const uint16_t *d_raw, int J, int K, int N, const float *h_t,
                                  const fuse_params *p, float *d_fused, void *cuda_stream) {
    FuseDev f;
    int rc = pm::validate_fuse(d_raw, J, K, N, h_t, p, d_fused, &f);
    if (rc != PTYCHO_OK) return rc;
    const size_t per_pos = scratch_floats_per_position(K, N, f.L);
    const size_t cap = kNoAllocScratchBytes / sizeof(float);
    if (per_pos > cap)
        return pm::fail(PTYCHO_EINVAL,
                        "fuse_stack_noalloc: one position needs %zu bytes of scratch (N = %d, K = %d, L = %d), "
                        "more than the %zu-byte static buffer",
                        per_pos * sizeof(float), N, K, f.L, kNoAllocScratchBytes);
    if (J == 0) return PTYCHO_OK;
    float *scratch = nullptr;
    cudaStream_t st = (cudaStream_t)cuda_stream;
    if (per_pos > 0 && (rc = noalloc_scratch(&scratch, st))) return rc;
    int chunk = per_pos > 0 ? (int)std::min<size_t>((size_t)J, cap / per_pos) : J;
    chunk = std::max(1, std::min(chunk, 65535 / K));
    const size_t NN = (size_t)N * N;
    for (int j0 = 0; j0 < J && rc == PTYCHO_OK; j0 += chunk) {
        const int jn = std::min(chunk, J - j0);
        rc = pm::fuse_dispatch(d_raw + (size_t)j0 * K * NN, jn, K, N, f, d_fused + (size_t)j0 * NN, scratch, st);
    }
    return rc;
}

// ---------------------------------------------------------------------------------------
// Standard Linear Integration (the linear HDR comparator of §1 and §2.2): per pixel,
// t_max * sum_{k: I_k < clip} I_k / sum_{k: I_k < clip} t_k; a pixel saturated in every
// exposure takes the shortest exposure's clipped rate.  One thread per (position, pixel).
namespace {

struct SliDev {
    float t[kMaxK];
    float tmax, clip;
    int kmin;
};

__global__ void k_sli(const uint16_t *__restrict__ raw, float *__restrict__ out, int K, size_t NN, size_t total,
                      SliDev s) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x) {
        const size_t j = i / NN, p = i % NN;
        const uint16_t *rj = raw + j * K * NN + p;
        float num = 0.f, den = 0.f;
        for (int k = 0; k < K; ++k) {
            const float v = (float)__ldg(rj + k * NN);
            if (v < s.clip) {
                num += v;
                den += s.t[k];
            }
        }
        out[i] = den > 0.f ? s.tmax * (num / den) : s.tmax * ((float)__ldg(rj + s.kmin * NN) / s.t[s.kmin]);
    }
}

}  // namespace

extern "C" int fuse_sli(const uint16_t *d_raw, int J, int K, int N, const float *h_t, float clip, float *d_out,
                        void *cuda_stream) {
    if (J < 0) return pm::fail(PTYCHO_EINVAL, "fuse_sli: J = %d < 0", J);
    if (K < 1 || K > kMaxK) return pm::fail(PTYCHO_EINVAL, "fuse_sli: K = %d not in [1, %d]", K, kMaxK);
    if (N < 1 || N > 4096) return pm::fail(PTYCHO_EINVAL, "fuse_sli: N = %d not in [1, 4096]", N);
    if (!(clip > 0.f) || !std::isfinite(clip)) return pm::fail(PTYCHO_EINVAL, "fuse_sli: clip must be finite and > 0");
    if (!h_t) return pm::fail(PTYCHO_EINVAL, "fuse_sli: exposure times pointer is NULL");
    SliDev s{};
    s.tmax = 0.f;
    s.kmin = 0;
    for (int k = 0; k < K; ++k) {
        if (!(h_t[k] > 0.f) || !std::isfinite(h_t[k]))
            return pm::fail(PTYCHO_EINVAL, "fuse_sli: t[%d] = %g must be finite and > 0", k, (double)h_t[k]);
        s.t[k] = h_t[k];
        s.tmax = std::max(s.tmax, h_t[k]);
        if (h_t[k] < h_t[s.kmin]) s.kmin = k;
    }
    s.clip = clip;
    if (J == 0) return PTYCHO_OK;
    if (!d_raw || !d_out) return pm::fail(PTYCHO_EINVAL, "fuse_sli: NULL raw or output pointer");
    const size_t NN = (size_t)N * N, total = (size_t)J * NN;
    k_sli<<<grid_for(total, 256), 256, 0, (cudaStream_t)cuda_stream>>>(d_raw, d_out, K, NN, total, s);
    PM_LAUNCHED("k_sli");
    return PTYCHO_OK;
}
