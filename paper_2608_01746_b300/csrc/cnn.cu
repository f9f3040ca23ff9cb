// Learned warm start: a convolutional encoder-decoder trained and run with the project's own
// kernels.  Storage is BF16 (weights as used by the GEMMs, activations, gradients entering a
// GEMM); every contraction accumulates in FP32 on the tensor cores (gemm.cu); master weights,
// Adam moments, biases and the loss are FP32.
//
// A 3 x 3 convolution layer is three GEMMs after im2col (P = batch x output pixels, K = 9 Cin):
//   forward       Z[P][Cout]  = col[P][K] . W[Cout][K]^T           (+ bias, ReLU -> BF16)
//   data grad     s1 / up: dX[P][Cin] = col(dZ)[P][9 Cout] . Wflip[Cin][9 Cout]^T, the
//                 stride-1 convolution of dZ with the flipped kernel (then the 2 x 2 sum for up);
//                 s2: dcol[P][K] = dZ[P][Cout] . W^T[K][Cout]^T, then col2im (a gather)
//   weight grad   dW[Cout][K] = dZ^T[Cout][P] . col^T[K][P]^T
// with every dimension zero-padded to the GEMM tile multiples.  Modes: s1 (stride 1), s2
// (stride 2), up (nearest 2x up-sampling, then stride 1); zero padding of one pixel.
#include <cuda_bf16.h>

#include <cmath>
#include <algorithm>
#include <cstring>
#include <new>
#include <random>
#include <vector>

#include "common.cuh"
#include "gemm.h"
#include "warm_start.h"

namespace {

using bf16 = __nv_bfloat16;
constexpr int kT = 256;

int rup(int x, int m) { return (x + m - 1) / m * m; }

unsigned nblk(size_t n) { return (unsigned)std::min<size_t>((n + kT - 1) / kT, (size_t)1 << 20); }

// ---------------------------------------------------------------------------------------------
// im2col: element (p, k), p = (b, i, j) output pixel, k = c * 9 + u * 3 + v, of the conv input
// x_in[b][c][s i + u - 1][s j + v - 1] (zero outside; for "up", x_in = nearest up-sampling).
// Index arithmetic is 32-bit (every buffer holds fewer than 2^31 elements).
// Input element read by im2col entry (b, c, i, j, u, v) for layer mode MODE (zero outside).
template <int MODE>
__device__ __forceinline__ bf16 conv_tap(const bf16 *__restrict__ x, int cin, int hin, int b, int c, int i, int j,
                                         int u, int v) {
    int yi, xi;
    if (MODE == WS_MODE_S2) {
        yi = 2 * i + u - 1;
        xi = 2 * j + v - 1;
    } else if (MODE == WS_MODE_UP) {
        const int yu = i + u - 1, xu = j + v - 1;
        if (yu < 0 || xu < 0 || yu >= 2 * hin || xu >= 2 * hin) return __float2bfloat16_rn(0.f);
        yi = yu >> 1;
        xi = xu >> 1;
    } else {
        yi = i + u - 1;
        xi = j + v - 1;
    }
    if (yi < 0 || xi < 0 || yi >= hin || xi >= hin) return __float2bfloat16_rn(0.f);
    return x[(((unsigned)b * cin + c) * hin + yi) * hin + xi];
}

// Each thread writes 8 consecutive elements of one output row (one 16-byte store).  Row layout
// out[p][k] (Pp x Kp), groups along k = c * 9 + u * 3 + v: the lanes of a warp take one k group
// of 32 consecutive pixels (each load instruction reads consecutive input pixels of one channel
// tap) and consecutive warps the next k groups of the same pixels.  Transposed out[k][p]
// (Kp x Pp), groups along p = (b, i, j): the lanes take consecutive pixel groups of one k (a warp
// writes 512 contiguous bytes).  Pp % 128 == 0 and Kp % 64 == 0, so no group straddles a row;
// the indices of a group's first element are decomposed once and then stepped.  The values are
// exact copies of the (BF16) input, zero outside the image and in the padding.
template <int MODE, bool TRANSPOSED>
__global__ void k_im2col(const bf16 *__restrict__ x, int cin, int hin, int hout, int P, int K, int Pp, int Kp,
                         bf16 *__restrict__ out) {
    const unsigned ninner = TRANSPOSED ? (unsigned)Pp : (unsigned)Kp, groups = ninner / 8u;
    const unsigned n = (TRANSPOSED ? (unsigned)Kp : (unsigned)Pp) * groups, hw = (unsigned)(hout * hout);
    for (unsigned g = blockIdx.x * blockDim.x + threadIdx.x; g < n; g += gridDim.x * blockDim.x) {
        unsigned outer, i0;
        if (TRANSPOSED) {
            outer = g / groups;
            i0 = (g - outer * groups) * 8u;
        } else {                                               // warp = (32-pixel block, k group)
            const unsigned w = g >> 5, pblk = w / groups;
            outer = pblk * 32u + (g & 31u);
            i0 = (w - pblk * groups) * 8u;
        }
        const unsigned p0 = TRANSPOSED ? i0 : outer, k0 = TRANSPOSED ? outer : i0;
        int b = (int)(p0 / hw);
        const unsigned q = p0 - (unsigned)b * hw;
        int i = (int)(q / (unsigned)hout), j = (int)(q - (unsigned)i * hout);
        int c = (int)(k0 / 9u), r = (int)(k0 - 9u * c);
        __align__(16) bf16 v[8];
#pragma unroll
        for (int e = 0; e < 8; ++e) {
            const int p = (int)p0 + (TRANSPOSED ? e : 0), k = (int)k0 + (TRANSPOSED ? 0 : e);
            const int u = (r >= 3) + (r >= 6), w = r - 3 * u;
            v[e] = (p < P && k < K) ? conv_tap<MODE>(x, cin, hin, b, c, i, j, u, w) : __float2bfloat16_rn(0.f);
            if (TRANSPOSED) {                                  // next pixel
                if (++j == hout) {
                    j = 0;
                    if (++i == hout) { i = 0; ++b; }
                }
            } else if (++r == 9) {                             // next tap
                r = 0;
                ++c;
            }
        }
        *reinterpret_cast<uint4 *>(out + (size_t)outer * ninner + i0) = *reinterpret_cast<const uint4 *>(v);
    }
}

unsigned im2col_grid(int Pp, int Kp) {
    const size_t groups = (size_t)Pp * Kp / 8;
    return (unsigned)std::min<size_t>((groups + kT - 1) / kT, (size_t)148 * 16);
}

template <bool TRANSPOSED>
int launch_im2col(const bf16 *x, int cin, int hin, int mode, int hout, int P, int K, int Pp, int Kp, bf16 *out,
                  cudaStream_t st) {
    const unsigned grid = im2col_grid(Pp, Kp);
    if (mode == WS_MODE_S2) k_im2col<WS_MODE_S2, TRANSPOSED><<<grid, kT, 0, st>>>(x, cin, hin, hout, P, K, Pp, Kp, out);
    else if (mode == WS_MODE_UP)
        k_im2col<WS_MODE_UP, TRANSPOSED><<<grid, kT, 0, st>>>(x, cin, hin, hout, P, K, Pp, Kp, out);
    else k_im2col<WS_MODE_S1, TRANSPOSED><<<grid, kT, 0, st>>>(x, cin, hin, hout, P, K, Pp, Kp, out);
    PM_LAUNCHED("k_im2col");
    return PTYCHO_OK;
}

// col2im (adjoint of im2col) as a gather: dx[b][c][y][x] = sum of dcol[p][k] over the (p, k)
// whose im2col element reads x[b][c][y][x].
__global__ void k_col2im(const float *__restrict__ dcol, int Kp, int B, int cin, int hin, int mode, int hout,
                         float *__restrict__ dx) {
    const unsigned n = (unsigned)B * cin * hin * hin;
    for (unsigned e = blockIdx.x * blockDim.x + threadIdx.x; e < n; e += gridDim.x * blockDim.x) {
        const unsigned hh = (unsigned)hin * hin;
        const unsigned bc = e / hh, yx = e - bc * hh;
        const int y = (int)(yx / (unsigned)hin), x = (int)(yx - (unsigned)y * hin);
        const unsigned b = bc / (unsigned)cin, c = bc - b * cin;
        const size_t pb = (size_t)b * hout * hout;
        float acc = 0.f;
        for (int u = 0; u < 3; ++u)
            for (int v = 0; v < 3; ++v) {
                const int k = (int)c * 9 + u * 3 + v;
                if (mode == WS_MODE_S2) {
                    const int ti = y - u + 1, tj = x - v + 1;
                    if (ti < 0 || tj < 0 || (ti & 1) || (tj & 1)) continue;
                    const int i = ti >> 1, j = tj >> 1;
                    if (i >= hout || j >= hout) continue;
                    acc += dcol[(pb + (size_t)i * hout + j) * Kp + k];
                } else if (mode == WS_MODE_UP) {
                    for (int sy = 0; sy < 2; ++sy)
                        for (int sx = 0; sx < 2; ++sx) {
                            const int i = 2 * y + sy - u + 1, j = 2 * x + sx - v + 1;
                            if (i < 0 || j < 0 || i >= hout || j >= hout) continue;
                            acc += dcol[(pb + (size_t)i * hout + j) * Kp + k];
                        }
                } else {
                    const int i = y - u + 1, j = x - v + 1;
                    if (i < 0 || j < 0 || i >= hout || j >= hout) continue;
                    acc += dcol[(pb + (size_t)i * hout + j) * Kp + k];
                }
            }
        dx[e] = acc;
    }
}

// Data gradient of a stride-1 or up-sampling layer as a stride-1 convolution of dZ with the
// flipped, channel-transposed kernel, at the layer's output resolution:
//   dx_c[b][c][y][x] = sum_{o, u', v'} dZ[b][o][y + u' - 1][x + v' - 1] W[o][c][2 - u'][2 - v']
// (dx_c = dx for s1; for "up" it is the gradient of the up-sampled input, and dx is its 2 x 2
// sum).  Operand col[p][k'] (Pp x K2p), p = (b, y, x) at hout, k' = o * 9 + u' * 3 + v', read
// from dz[p][o] (Pp x Coutp, BF16): exact copies, zero outside the image and in the padding.
__global__ void k_im2col_dz(const bf16 *__restrict__ dz, int Coutp, int cout, int hout, int P, int Pp, int K2p,
                            bf16 *__restrict__ out) {
    const unsigned groups = (unsigned)K2p / 8u, n = (unsigned)Pp * groups, hw = (unsigned)(hout * hout);
    const int K2 = 9 * cout;
    for (unsigned g = blockIdx.x * blockDim.x + threadIdx.x; g < n; g += gridDim.x * blockDim.x) {
        const unsigned p = g / groups, k0 = (g - p * groups) * 8u;
        const unsigned b = p / hw, q = p - b * hw, i = q / (unsigned)hout, j = q - i * (unsigned)hout;
        __align__(16) bf16 v[8];
#pragma unroll
        for (int e = 0; e < 8; ++e) {
            const int k = (int)k0 + e;
            bf16 val = __float2bfloat16_rn(0.f);
            if ((int)p < P && k < K2) {
                const int o = k / 9, r = k - 9 * o, u = r / 3, w = r - 3 * u;
                const int y = (int)i + u - 1, x = (int)j + w - 1;
                if (y >= 0 && x >= 0 && y < hout && x < hout)
                    val = dz[((size_t)b * hw + (unsigned)y * hout + (unsigned)x) * Coutp + o];
            }
            v[e] = val;
        }
        *reinterpret_cast<uint4 *>(out + (size_t)p * K2p + k0) = *reinterpret_cast<const uint4 *>(v);
    }
}

// dx[b][c][y][x] (FP32, NCHW, at hin) from the rows C[p][c] (Cinp columns) of the convolution
// above: s1 copies; up sums the 2 x 2 block (2y + sy, 2x + sx) in the order (0,0) (0,1) (1,0) (1,1).
// Block = 32 output pixels x 32 channels through a shared-memory tile: C is read along c and dx
// written along the pixels (both coalesced).  Grid (ceil(B hin^2 / 32), Cinp / 32).
__global__ void k_dx_from_rows(const float *__restrict__ C, int Cinp, int B, int cin, int hin, int mode, int hout,
                               float *__restrict__ dx) {
    __shared__ float t[32][33];                            // [pixel][channel]
    const unsigned hh = (unsigned)(hin * hin), npix = (unsigned)B * hh;
    const unsigned q0 = blockIdx.x * 32u, c0 = blockIdx.y * 32u;
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
    for (int r = ty; r < 32; r += kT / 32) {
        const unsigned e = q0 + r;
        float acc = 0.f;
        if (e < npix) {
            const unsigned b = e / hh, yx = e - b * hh, y = yx / (unsigned)hin, x = yx - y * hin;
            const float *row = C + ((size_t)b * hout * hout) * Cinp + c0 + tx;
            if (mode == WS_MODE_UP) {
                acc = row[((2 * y) * hout + 2 * x) * (size_t)Cinp];
                acc += row[((2 * y) * hout + 2 * x + 1) * (size_t)Cinp];
                acc += row[((2 * y + 1) * hout + 2 * x) * (size_t)Cinp];
                acc += row[((2 * y + 1) * hout + 2 * x + 1) * (size_t)Cinp];
            } else {
                acc = row[(y * hout + x) * (size_t)Cinp];
            }
        }
        t[r][tx] = acc;
    }
    __syncthreads();
    for (int r = ty; r < 32; r += kT / 32) {
        const unsigned c = c0 + r, e = q0 + tx;
        if (c < (unsigned)cin && e < npix) {
            const unsigned b = e / hh, yx = e - b * hh;
            dx[((size_t)b * cin + c) * hh + yx] = t[tx][r];
        }
    }
}

// Z[p][o] + bias -> ReLU -> BF16 activation y[b][o][i][j]; the last layer stores FP32.  Block =
// 32 pixels x 32 channels through a shared-memory tile (C read along o, y written along the
// pixels).  Grid (ceil(B hout^2 / 32), Coutp / 32).
__global__ void k_fwd_epilogue(const float *__restrict__ C, int Coutp, const float *__restrict__ bias, int B, int cout,
                               int hout, int relu, bf16 *__restrict__ y, float *__restrict__ yf) {
    __shared__ float t[32][33];                            // [pixel][channel]
    const unsigned hw = (unsigned)(hout * hout), P = (unsigned)B * hw;
    const unsigned p0 = blockIdx.x * 32u, o0 = blockIdx.y * 32u;
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
    for (int r = ty; r < 32; r += kT / 32) {
        const unsigned p = p0 + r;
        t[r][tx] = p < P ? C[(size_t)p * Coutp + o0 + tx] : 0.f;
    }
    __syncthreads();
    for (int r = ty; r < 32; r += kT / 32) {
        const unsigned o = o0 + r, p = p0 + tx;
        if (o < (unsigned)cout && p < P) {
            float z = t[tx][r] + bias[o];
            if (relu) z = fmaxf(z, 0.f);
            const unsigned b = p / hw, q = p - b * hw;
            const size_t e = ((size_t)b * cout + o) * hw + q;
            if (yf) yf[e] = z;
            else y[e] = __float2bfloat16_rn(z);
        }
    }
}

// dZ = dL/dy * relu'(y) in the two GEMM layouts, zero-padded: dz[p][o] (Pp x Coutp) and
// dzt[o][p] (Coutp128 x Pp).  Block = 32 channels x 32 pixels: g and y are read along the
// pixels and dzt written along them; dz is written along the channels from a shared-memory
// tile.  Grid (Pp / 32, Coutp128 / 32).
__global__ void k_bwd_dz(const float *__restrict__ g, const bf16 *__restrict__ y, int relu, int B, int cout, int hout,
                         int Pp, int Coutp, int Coutp128, bf16 *__restrict__ dz, bf16 *__restrict__ dzt) {
    __shared__ bf16 t[32][34];                             // [channel][pixel]
    const unsigned hw = (unsigned)(hout * hout), P = (unsigned)B * hw;
    const unsigned p0 = blockIdx.x * 32u, o0 = blockIdx.y * 32u;
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
    for (int r = ty; r < 32; r += kT / 32) {
        const unsigned o = o0 + r, p = p0 + tx;
        float d = 0.f;
        if (p < P && o < (unsigned)cout) {
            const unsigned b = p / hw, q = p - b * hw;
            const size_t idx = ((size_t)b * cout + o) * hw + q;
            d = g[idx];
            if (relu && !(__bfloat162float(y[idx]) > 0.f)) d = 0.f;
        }
        const bf16 h = __float2bfloat16_rn(d);
        dzt[(size_t)o * Pp + p] = h;
        t[r][tx] = h;
    }
    __syncthreads();
    for (int r = ty; r < 32; r += kT / 32) {
        const unsigned p = p0 + r, o = o0 + tx;
        if (o < (unsigned)Coutp) dz[(size_t)p * Coutp + o] = t[tx][r];
    }
}

// db[o] = sum over the batch and pixels of dL/dy * relu'(y), in two fixed-order passes: block
// (o, slice) sums its slice of the B * hout^2 pixels (per-thread FP32 sums, then a tree) into
// part[o * slices + slice]; k_bias_sum adds the slices in order.  32-bit indices (every
// activation holds fewer than 2^31 elements).
constexpr int kBiasSlices = 32;

__global__ void k_bias_grad(const float *__restrict__ g, const bf16 *__restrict__ y, int relu, int B, int cout,
                            int hout, int slices, float *__restrict__ part) {
    __shared__ float s[kT];
    const int o = blockIdx.x, sl = blockIdx.y;
    const unsigned hw = (unsigned)hout * hout, n = (unsigned)B * hw;
    const unsigned chunk = (n + slices - 1) / slices, e0 = sl * chunk, e1 = min(n, e0 + chunk);
    float acc = 0.f;
    for (unsigned e = e0 + threadIdx.x; e < e1; e += blockDim.x) {
        const unsigned b = e / hw, q = e - b * hw;
        const unsigned idx = (b * cout + o) * hw + q;
        float d = g[idx];
        if (relu && !(__bfloat162float(y[idx]) > 0.f)) d = 0.f;
        acc += d;
    }
    s[threadIdx.x] = acc;
    __syncthreads();
    for (int w = kT / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) s[threadIdx.x] += s[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) part[o * slices + sl] = s[0];
}

__global__ void k_bias_sum(const float *__restrict__ part, int cout, int slices, float *__restrict__ db) {
    const int o = blockIdx.x * blockDim.x + threadIdx.x;
    if (o >= cout) return;
    float a = 0.f;
    for (int sl = 0; sl < slices; ++sl) a += part[o * slices + sl];
    db[o] = a;
}

// The flipped, channel-transposed BF16 kernel of the data-gradient convolution:
// wf[c][o * 9 + u' * 3 + v'] = w[o][c * 9 + (2 - u') * 3 + (2 - v')]  (Cinp x K2p, zero padded).
__global__ void k_weights_flip(const float *__restrict__ w, int cout, int cin, int Cinp, int K2p,
                               bf16 *__restrict__ wf) {
    const size_t n = (size_t)Cinp * K2p;
    for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x) {
        const int c = (int)(e / K2p), k = (int)(e % K2p);
        float val = 0.f;
        if (c < cin && k < 9 * cout) {
            const int o = k / 9, r = k - 9 * o, u = r / 3, v = r - 3 * u;
            val = w[(size_t)o * (9 * cin) + c * 9 + (2 - u) * 3 + (2 - v)];
        }
        wf[e] = __float2bfloat16_rn(val);
    }
}

// BF16 copies of the FP32 master weights w[o][k]: wb[o][k] (Coutp x Kp) and wt[k][o] (Kp x Coutp).
__global__ void k_weights_bf16(const float *__restrict__ w, int cout, int K, int Coutp, int Kp, bf16 *__restrict__ wb,
                               bf16 *__restrict__ wt) {
    const size_t n = (size_t)Coutp * Kp;
    for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x) {
        const int o = (int)(e / Kp), k = (int)(e % Kp);
        const bf16 h = __float2bfloat16_rn((o < cout && k < K) ? w[(size_t)o * K + k] : 0.f);
        wb[e] = h;
        wt[(size_t)k * Coutp + o] = h;
    }
}

__global__ void k_copy_wgrad(const float *__restrict__ dW, int Kp, int cout, int K, float *__restrict__ gw) {
    const size_t n = (size_t)cout * K;
    for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x)
        gw[e] = dW[(e / K) * Kp + e % K];
}

// Mean squared error: per-block FP64 partial sums of (y - t)^2 and dL/dy = 2 (y - t) / n.
__global__ void k_mse(const float *__restrict__ y, const float *__restrict__ t, size_t n, float *__restrict__ dy,
                      double *__restrict__ part) {
    __shared__ double s[kT];
    double acc = 0.0;
    const float sc = 2.0f / (float)n;
    for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x) {
        const float d = y[e] - t[e];
        acc += (double)d * d;
        dy[e] = sc * d;
    }
    s[threadIdx.x] = acc;
    __syncthreads();
    for (int w = kT / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) s[threadIdx.x] += s[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) part[blockIdx.x] = s[0];
}

__global__ void k_adam(float *__restrict__ w, const float *__restrict__ g, float *__restrict__ m,
                       float *__restrict__ v, size_t n, float lr, float b1, float b2, float eps, float bc1, float bc2) {
    for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x) {
        const float gg = g[e];
        const float mm = b1 * m[e] + (1.f - b1) * gg;
        const float vv = b2 * v[e] + (1.f - b2) * gg * gg;
        m[e] = mm;
        v[e] = vv;
        w[e] -= lr * (mm / bc1) / (sqrtf(vv / bc2) + eps);
    }
}

// ---------------------------------------------------------------------------------------------
// Warm-start data transforms.
__global__ void k_preprocess(const float *__restrict__ f, int J, int N, bf16 *__restrict__ x) {
    const int h = N / 2;
    const size_t n = (size_t)J * h * h;
    for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x) {
        const int c = (int)(e % h), r = (int)((e / h) % h);
        const size_t j = e / ((size_t)h * h);
        const float *fj = f + j * N * N;
        const float s = fmaxf(fj[(2 * r) * N + 2 * c], 0.f) + fmaxf(fj[(2 * r) * N + 2 * c + 1], 0.f) +
                        fmaxf(fj[(2 * r + 1) * N + 2 * c], 0.f) + fmaxf(fj[(2 * r + 1) * N + 2 * c + 1], 0.f);
        x[e] = __float2bfloat16_rn(log1pf(s) * 0.1f);
    }
}

__global__ void k_targets(const float2 *__restrict__ obj, int M, const int2 *__restrict__ pos, int J, int N,
                          float *__restrict__ t) {
    const int n = N / 4;
    const size_t cnt = (size_t)J * n * n;
    for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < cnt; e += (size_t)gridDim.x * blockDim.x) {
        const int c = (int)(e % n), r = (int)((e / n) % n);
        const size_t j = e / ((size_t)n * n);
        const int2 pj = pos[j];
        float re = 0.f, im = 0.f;
        for (int a = 0; a < 4; ++a)
            for (int b = 0; b < 4; ++b) {
                const float2 o = obj[(size_t)(pj.x + 4 * r + a) * M + pj.y + 4 * c + b];
                re += o.x;
                im += o.y;
            }
        t[(j * 2 + 0) * n * n + (size_t)r * n + c] = re * (1.f / 16.f);
        t[(j * 2 + 1) * n * n + (size_t)r * n + c] = im * (1.f / 16.f);
    }
}

// Coarse weights: the 4 x 4 mean of |P|^2.
__global__ void k_coarse_weights(const float2 *__restrict__ probe, int N, float *__restrict__ w) {
    const int n = N / 4;
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n * n; e += gridDim.x * blockDim.x) {
        const int r = e / n, c = e % n;
        float s = 0.f;
        for (int a = 0; a < 4; ++a)
            for (int b = 0; b < 4; ++b) {
                const float2 p = probe[(4 * r + a) * N + 4 * c + b];
                s += p.x * p.x + p.y * p.y;
            }
        w[e] = s * (1.f / 16.f);
    }
}

// Owner-computes accumulation on the coarse grid: coarse pixel (R, C) sums the weighted
// predictions of every position whose coarse patch covers it (no atomics, fixed order).
__global__ void k_stitch_coarse(const float *__restrict__ pred, const int2 *__restrict__ pos, int J, int n,
                                const float *__restrict__ wgt, int Mc, float2 *__restrict__ num,
                                float *__restrict__ den) {
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < Mc * Mc; e += gridDim.x * blockDim.x) {
        const int R = e / Mc, C = e % Mc;
        float2 a = make_float2(0.f, 0.f);
        float d = 0.f;
        for (int j = 0; j < J; ++j) {
            const int2 pj = pos[j];
            const int r = R - pj.x / 4, c = C - pj.y / 4;
            if (r < 0 || c < 0 || r >= n || c >= n) continue;
            const float w = wgt[r * n + c];
            a.x += w * pred[((size_t)j * 2 + 0) * n * n + r * n + c];
            a.y += w * pred[((size_t)j * 2 + 1) * n * n + r * n + c];
            d += w;
        }
        num[e] = a;
        den[e] = d;
    }
}

__global__ void k_max_reduce(const float *__restrict__ v, int n, float *__restrict__ out) {
    __shared__ float s[kT];
    float m = 0.f;
    for (int e = threadIdx.x; e < n; e += blockDim.x) m = fmaxf(m, v[e]);
    s[threadIdx.x] = m;
    __syncthreads();
    for (int w = kT / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) s[threadIdx.x] = fmaxf(s[threadIdx.x], s[threadIdx.x + w]);
        __syncthreads();
    }
    if (threadIdx.x == 0) *out = s[0];
}

__device__ __forceinline__ float2 coarse_at(const float2 *num, const float *den, float thr, int Mc, int r, int c) {
    const float d = den[r * Mc + c];
    if (!(d >= thr)) return make_float2(1.f, 0.f);
    const float2 a = num[r * Mc + c];
    return make_float2(a.x / d, a.y / d);
}

// Bilinear up-sampling by 4: fine pixel f at coarse coordinate (f - 1.5) / 4, clamped.
__global__ void k_stitch_upsample(const float2 *__restrict__ num, const float *__restrict__ den,
                                  const float *__restrict__ dmax, int Mc, int M, float2 *__restrict__ obj) {
    const float thr = 1e-3f * dmax[0];
    const size_t n = (size_t)M * M;
    for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x) {
        const int y = (int)(e / M), x = (int)(e % M);
        const float cy = fminf(fmaxf((y - 1.5f) * 0.25f, 0.f), (float)(Mc - 1));
        const float cx = fminf(fmaxf((x - 1.5f) * 0.25f, 0.f), (float)(Mc - 1));
        const int y0 = min((int)floorf(cy), Mc - 2), x0 = min((int)floorf(cx), Mc - 2);
        const float ty = cy - y0, tx = cx - x0;
        const float2 a = coarse_at(num, den, thr, Mc, y0, x0), b = coarse_at(num, den, thr, Mc, y0, x0 + 1);
        const float2 c = coarse_at(num, den, thr, Mc, y0 + 1, x0), d = coarse_at(num, den, thr, Mc, y0 + 1, x0 + 1);
        const float2 top = make_float2(a.x * (1 - tx) + b.x * tx, a.y * (1 - tx) + b.y * tx);
        const float2 bot = make_float2(c.x * (1 - tx) + d.x * tx, c.y * (1 - tx) + d.y * tx);
        obj[e] = make_float2(top.x * (1 - ty) + bot.x * ty, top.y * (1 - ty) + bot.y * ty);
    }
}

}  // namespace

// ---------------------------------------------------------------------------------------------
struct wsnet_ctx {
    struct Layer {
        int cin = 0, cout = 0, mode = 0, relu = 0, hin = 0, hout = 0;
        int K = 0, Kp = 0, Coutp = 0, Coutp128 = 0;
        float *w = nullptr, *b = nullptr, *mw = nullptr, *vw = nullptr, *mb = nullptr, *vb = nullptr;
        float *gw = nullptr, *gb = nullptr;
        bf16 *wb = nullptr, *wt = nullptr, *y = nullptr;
        int Cinp = 0, K2p = 0;                 // data-gradient convolution (s1, up): Cinp x K2p kernel
        bf16 *wf = nullptr;
    };
    std::vector<Layer> L;
    int in_side = 0, max_batch = 0, out_channels = 0, out_side = 0;
    cudaStream_t st = nullptr;
    bf16 *col = nullptr;
    float *cbuf = nullptr, *pred = nullptr, *g0 = nullptr, *g1 = nullptr, *dpred = nullptr;
    float *work = nullptr;                     // split-K partial products of the weight gradients
    float *bpart = nullptr;                    // bias-gradient slice sums [cout][slices]
    size_t work_floats = 0;
    bf16 *dz = nullptr, *dzt = nullptr;
    double *part = nullptr;
    int *status = nullptr;
    long long step = 0;
    bool wdirty = true;
    std::vector<void *> allocs;
};

namespace {

template <typename T>
int nalloc(wsnet_ctx *n, T **p, size_t count) {
    *p = nullptr;
    cudaError_t e = pm::dev_malloc((void **)p, std::max<size_t>(count, 1) * sizeof(T));
    if (e != cudaSuccess) return pm::cuda_fail(e, "wsnet: cudaMalloc");
    n->allocs.push_back(*p);
    return PTYCHO_OK;
}

void free_net(wsnet_ctx *n) {
    if (!n) return;
    if (n->st) cudaStreamSynchronize(n->st);
    for (void *p : n->allocs) cudaFree(p);
    delete n;
}

int refresh_weights(wsnet_ctx *n) {
    if (!n->wdirty) return PTYCHO_OK;
    for (auto &l : n->L) {
        k_weights_bf16<<<nblk((size_t)l.Coutp * l.Kp), kT, 0, n->st>>>(l.w, l.cout, l.K, l.Coutp, l.Kp, l.wb, l.wt);
        PM_LAUNCHED("k_weights_bf16");
        if (l.wf) {
            k_weights_flip<<<nblk((size_t)l.Cinp * l.K2p), kT, 0, n->st>>>(l.w, l.cout, l.cin, l.Cinp, l.K2p, l.wf);
            PM_LAUNCHED("k_weights_flip");
        }
    }
    n->wdirty = false;
    return PTYCHO_OK;
}

int forward(wsnet_ctx *n, const bf16 *x, int B, float *out) {
    int rc = refresh_weights(n);
    if (rc) return rc;
    const bf16 *in = x;
    for (size_t li = 0; li < n->L.size(); ++li) {
        auto &l = n->L[li];
        const int P = B * l.hout * l.hout, Pp = rup(P, 128);
        if ((rc = launch_im2col<false>(in, l.cin, l.hin, l.mode, l.hout, P, l.K, Pp, l.Kp, n->col, n->st))) return rc;
        if ((rc = pm::gemm_bf16_launch(n->col, l.wb, n->cbuf, Pp, l.Coutp, l.Kp, n->status, n->st))) return rc;
        const bool last = li + 1 == n->L.size();
        k_fwd_epilogue<<<dim3((unsigned)((P + 31) / 32), (unsigned)(l.Coutp / 32)), kT, 0, n->st>>>(
            n->cbuf, l.Coutp, l.b, B, l.cout, l.hout, l.relu, l.y, last ? out : nullptr);
        PM_LAUNCHED("k_fwd_epilogue");
        in = l.y;
    }
    return PTYCHO_OK;
}

// Forward, loss against t, gradients of every layer into gw / gb.
int backward(wsnet_ctx *n, const bf16 *x, const float *t, int B, double *h_loss) {
    int rc = forward(n, x, B, n->pred);
    if (rc) return rc;
    const size_t nout = (size_t)B * n->out_channels * n->out_side * n->out_side;
    const unsigned nb = std::min<unsigned>(nblk(nout), 1024);
    k_mse<<<nb, kT, 0, n->st>>>(n->pred, t, nout, n->dpred, n->part);
    PM_LAUNCHED("k_mse");
    const float *g = n->dpred;
    for (int li = (int)n->L.size() - 1; li >= 0; --li) {
        auto &l = n->L[li];
        const int P = B * l.hout * l.hout, Pp = rup(P, 128);
        const bf16 *in = li == 0 ? x : n->L[li - 1].y;
        k_bwd_dz<<<dim3((unsigned)(Pp / 32), (unsigned)(l.Coutp128 / 32)), kT, 0, n->st>>>(
            g, l.y, l.relu, B, l.cout, l.hout, Pp, l.Coutp, l.Coutp128, n->dz, n->dzt);
        PM_LAUNCHED("k_bwd_dz");
        {
            const int slices = std::max(1, std::min(kBiasSlices, B * l.hout * l.hout / (4 * kT)));
            k_bias_grad<<<dim3(l.cout, slices), kT, 0, n->st>>>(g, l.y, l.relu, B, l.cout, l.hout, slices, n->bpart);
            PM_LAUNCHED("k_bias_grad");
            k_bias_sum<<<(l.cout + kT - 1) / kT, kT, 0, n->st>>>(n->bpart, l.cout, slices, l.gb);
            PM_LAUNCHED("k_bias_sum");
        }
        // weight gradient: dW[Coutp128][Kp] = dzt[Coutp128][Pp] . colT[Kp][Pp]^T
        if ((rc = launch_im2col<true>(in, l.cin, l.hin, l.mode, l.hout, P, l.K, Pp, l.Kp, n->col, n->st))) return rc;
        if ((rc = pm::gemm_bf16_launch(n->dzt, n->col, n->cbuf, l.Coutp128, l.Kp, Pp, n->status, n->st, n->work,
                                       n->work_floats)))
            return rc;
        k_copy_wgrad<<<nblk((size_t)l.cout * l.K), kT, 0, n->st>>>(n->cbuf, l.Kp, l.cout, l.K, l.gw);
        PM_LAUNCHED("k_copy_wgrad");
        if (li == 0) break;                      // no gradient for the network input
        float *gx = (g == n->g0) ? n->g1 : n->g0;
        if (l.wf) {
            // s1 / up: dx by the flipped-kernel convolution of dZ (rows C[Pp][Cinp]), then the
            // 2 x 2 sum for up
            k_im2col_dz<<<im2col_grid(Pp, l.K2p), kT, 0, n->st>>>(n->dz, l.Coutp, l.cout, l.hout, P, Pp, l.K2p,
                                                                  n->col);
            PM_LAUNCHED("k_im2col_dz");
            if ((rc = pm::gemm_bf16_launch(n->col, l.wf, n->cbuf, Pp, l.Cinp, l.K2p, n->status, n->st))) return rc;
            k_dx_from_rows<<<dim3((unsigned)((B * l.hin * l.hin + 31) / 32), (unsigned)(l.Cinp / 32)), kT, 0,
                             n->st>>>(n->cbuf, l.Cinp, B, l.cin, l.hin, l.mode, l.hout, gx);
            PM_LAUNCHED("k_dx_from_rows");
        } else {
            // s2: dcol[Pp][Kp] = dz[Pp][Coutp] . wt[Kp][Coutp]^T, then col2im
            if ((rc = pm::gemm_bf16_launch(n->dz, l.wt, n->cbuf, Pp, l.Kp, l.Coutp, n->status, n->st))) return rc;
            k_col2im<<<nblk((size_t)B * l.cin * l.hin * l.hin), kT, 0, n->st>>>(n->cbuf, l.Kp, B, l.cin, l.hin,
                                                                                l.mode, l.hout, gx);
            PM_LAUNCHED("k_col2im");
        }
        g = gx;
    }
    if (h_loss) {
        std::vector<double> part(nb);
        PM_CUDA(cudaMemcpyAsync(part.data(), n->part, nb * sizeof(double), cudaMemcpyDeviceToHost, n->st));
        int status = 0;
        PM_CUDA(cudaMemcpyAsync(&status, n->status, sizeof(int), cudaMemcpyDeviceToHost, n->st));
        PM_CUDA(cudaStreamSynchronize(n->st));
        if (status) return pm::fail(PTYCHO_ETIMEDOUT, "wsnet: a bounded device wait gave up");
        double s = 0.0;
        for (double v : part) s += v;
        *h_loss = s / (double)nout;
        if (!std::isfinite(*h_loss)) return pm::fail(PTYCHO_ENONFINITE, "wsnet: loss is not finite");
    }
    return PTYCHO_OK;
}

int adam(wsnet_ctx *n, float lr) {
    ++n->step;
    const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
    const float bc1 = (float)(1.0 - std::pow(0.9, (double)n->step));
    const float bc2 = (float)(1.0 - std::pow(0.999, (double)n->step));
    for (auto &l : n->L) {
        const size_t nw = (size_t)l.cout * l.K;
        k_adam<<<nblk(nw), kT, 0, n->st>>>(l.w, l.gw, l.mw, l.vw, nw, lr, b1, b2, eps, bc1, bc2);
        PM_LAUNCHED("k_adam");
        k_adam<<<nblk(l.cout), kT, 0, n->st>>>(l.b, l.gb, l.mb, l.vb, (size_t)l.cout, lr, b1, b2, eps, bc1, bc2);
        PM_LAUNCHED("k_adam");
    }
    n->wdirty = true;
    return PTYCHO_OK;
}

bool check_batch(const wsnet_ctx *n, int B, const char *what) {
    if (B < 1 || B > n->max_batch) {
        pm::fail(PTYCHO_EINVAL, "%s: batch %d not in [1, %d]", what, B, n->max_batch);
        return false;
    }
    return true;
}

}  // namespace

extern "C" int wsnet_create(wsnet *out, const int *cin, const int *cout, const int *mode, int nlayers, int in_side,
                            int max_batch, unsigned long long seed, void *cuda_stream) {
    if (!out) return pm::fail(PTYCHO_EINVAL, "wsnet_create: out is NULL");
    *out = nullptr;
    if (!cin || !cout || !mode || nlayers < 1 || nlayers > 64)
        return pm::fail(PTYCHO_EINVAL, "wsnet_create: need 1..64 layers");
    if (in_side < 1 || in_side > 4096 || max_batch < 1 || max_batch > 4096)
        return pm::fail(PTYCHO_EINVAL, "wsnet_create: in_side %d / max_batch %d out of range", in_side, max_batch);
    int side = in_side;
    for (int i = 0; i < nlayers; ++i) {
        if (cin[i] < 1 || cout[i] < 1 || cin[i] > 4096 || cout[i] > 4096 || (i > 0 && cin[i] != cout[i - 1]))
            return pm::fail(PTYCHO_EINVAL, "wsnet_create: layer %d channels %d -> %d inconsistent", i, cin[i], cout[i]);
        if (mode[i] != WS_MODE_S1 && mode[i] != WS_MODE_S2 && mode[i] != WS_MODE_UP)
            return pm::fail(PTYCHO_EINVAL, "wsnet_create: layer %d mode %d unknown", i, mode[i]);
        if (mode[i] == WS_MODE_S2 && (side & 1))
            return pm::fail(PTYCHO_EINVAL, "wsnet_create: layer %d halves an odd side %d", i, side);
        side = mode[i] == WS_MODE_S2 ? side / 2 : (mode[i] == WS_MODE_UP ? side * 2 : side);
        if (side > 4096) return pm::fail(PTYCHO_EINVAL, "wsnet_create: side grows beyond 4096");
    }
    wsnet_ctx *n = new (std::nothrow) wsnet_ctx();
    if (!n) return pm::fail(PTYCHO_ENOMEM, "wsnet_create: host allocation failed");
    n->st = (cudaStream_t)cuda_stream;
    n->in_side = in_side;
    n->max_batch = max_batch;
    auto bail = [&](int r) { free_net(n); return r; };
    int rc;
    size_t max_col = 0, max_c = 0, max_dz = 0, max_act = (size_t)max_batch * cin[0] * in_side * in_side;
    size_t max_w = 0;
    side = in_side;
    std::mt19937_64 rng(seed);
    for (int i = 0; i < nlayers; ++i) {
        wsnet_ctx::Layer l;
        l.cin = cin[i];
        l.cout = cout[i];
        l.mode = mode[i];
        l.relu = i + 1 < nlayers;
        l.hin = side;
        l.hout = mode[i] == WS_MODE_S2 ? side / 2 : (mode[i] == WS_MODE_UP ? side * 2 : side);
        side = l.hout;
        l.K = l.cin * 9;
        l.Kp = rup(l.K, 64);
        l.Coutp = rup(l.cout, 64);
        l.Coutp128 = rup(l.cout, 128);
        const size_t Pp = (size_t)rup(max_batch * l.hout * l.hout, 128);
        const bool flipped = i > 0 && l.mode != WS_MODE_S2;      // data gradient by convolution of dZ
        if (flipped) {
            l.Cinp = rup(l.cin, 64);
            l.K2p = rup(9 * l.cout, 64);
            max_col = std::max(max_col, Pp * l.K2p);
        }
        max_col = std::max(max_col, Pp * l.Kp);
        max_c = std::max(std::max(max_c, Pp * (size_t)l.Coutp), std::max(Pp * (size_t)l.Kp, (size_t)l.Coutp128 * l.Kp));
        max_dz = std::max(max_dz, Pp * l.Coutp128);
        max_w = std::max(max_w, (size_t)l.Coutp128 * l.Kp);
        max_act = std::max(max_act, (size_t)max_batch * l.cout * l.hout * l.hout);
        const size_t nw = (size_t)l.cout * l.K;
        if ((rc = nalloc(n, &l.w, nw)) || (rc = nalloc(n, &l.b, l.cout)) || (rc = nalloc(n, &l.mw, nw)) ||
            (rc = nalloc(n, &l.vw, nw)) || (rc = nalloc(n, &l.mb, l.cout)) || (rc = nalloc(n, &l.vb, l.cout)) ||
            (rc = nalloc(n, &l.gw, nw)) || (rc = nalloc(n, &l.gb, l.cout)) ||
            (rc = nalloc(n, &l.wb, (size_t)l.Coutp * l.Kp)) || (rc = nalloc(n, &l.wt, (size_t)l.Kp * l.Coutp)) ||
            (rc = nalloc(n, &l.y, (size_t)max_batch * l.cout * l.hout * l.hout)) ||
            (flipped && (rc = nalloc(n, &l.wf, (size_t)l.Cinp * l.K2p))))
            return bail(rc);
        // He-normal initial weights (std sqrt(2 / fan_in)), zero biases and moments
        std::normal_distribution<float> nd(0.f, std::sqrt(2.f / (float)l.K));
        std::vector<float> hw(nw);
        for (auto &v : hw) v = nd(rng);
        cudaError_t e;
        if ((e = cudaMemcpy(l.w, hw.data(), nw * sizeof(float), cudaMemcpyHostToDevice)) ||
            (e = cudaMemset(l.b, 0, l.cout * sizeof(float))) || (e = cudaMemset(l.mw, 0, nw * sizeof(float))) ||
            (e = cudaMemset(l.vw, 0, nw * sizeof(float))) || (e = cudaMemset(l.mb, 0, l.cout * sizeof(float))) ||
            (e = cudaMemset(l.vb, 0, l.cout * sizeof(float))))
            return bail(pm::cuda_fail(e, "wsnet_create: initial weights"));
        n->L.push_back(l);
    }
    n->out_channels = cout[nlayers - 1];
    n->out_side = side;
    const size_t nout = (size_t)max_batch * n->out_channels * side * side;
    // the layout kernels index with 32-bit arithmetic
    if (std::max(std::max(max_col, max_c), std::max(max_dz, std::max(max_act, nout))) >= ((size_t)1 << 31))
        return bail(pm::fail(PTYCHO_EINVAL, "wsnet_create: a layer buffer would hold 2^31 or more elements"));
    if ((rc = nalloc(n, &n->col, max_col)) || (rc = nalloc(n, &n->cbuf, max_c)) || (rc = nalloc(n, &n->dz, max_dz)) ||
        (rc = nalloc(n, &n->dzt, max_dz)) || (rc = nalloc(n, &n->g0, max_act)) || (rc = nalloc(n, &n->g1, max_act)) ||
        (rc = nalloc(n, &n->pred, nout)) || (rc = nalloc(n, &n->dpred, nout)) || (rc = nalloc(n, &n->part, 1024)) ||
        (rc = nalloc(n, &n->status, 1)))
        return bail(rc);
    n->work_floats = 64 * max_w;
    if ((rc = nalloc(n, &n->work, n->work_floats))) return bail(rc);
    int max_cout = 0;
    for (int i = 0; i < nlayers; ++i) max_cout = std::max(max_cout, cout[i]);
    if ((rc = nalloc(n, &n->bpart, (size_t)max_cout * kBiasSlices))) return bail(rc);
    cudaError_t e;
    if ((e = cudaMemset(n->status, 0, sizeof(int)))) return bail(pm::cuda_fail(e, "wsnet_create: status"));
    *out = n;
    return PTYCHO_OK;
}

extern "C" int wsnet_set_params(wsnet n, int layer, const float *h_w, const float *h_b) {
    if (!n || !h_w || !h_b || layer < 0 || layer >= (int)n->L.size())
        return pm::fail(PTYCHO_EINVAL, "wsnet_set_params: bad network, layer or pointer");
    auto &l = n->L[layer];
    PM_CUDA(cudaMemcpyAsync(l.w, h_w, (size_t)l.cout * l.K * sizeof(float), cudaMemcpyHostToDevice, n->st));
    PM_CUDA(cudaMemcpyAsync(l.b, h_b, (size_t)l.cout * sizeof(float), cudaMemcpyHostToDevice, n->st));
    PM_CUDA(cudaStreamSynchronize(n->st));
    n->wdirty = true;
    return PTYCHO_OK;
}

static int get_pair(wsnet n, int layer, float *h_a, float *h_b, bool grads, const char *what) {
    if (!n || !h_a || !h_b || layer < 0 || layer >= (int)n->L.size())
        return pm::fail(PTYCHO_EINVAL, "%s: bad network, layer or pointer", what);
    auto &l = n->L[layer];
    PM_CUDA(cudaMemcpyAsync(h_a, grads ? l.gw : l.w, (size_t)l.cout * l.K * sizeof(float), cudaMemcpyDeviceToHost,
                            n->st));
    PM_CUDA(cudaMemcpyAsync(h_b, grads ? l.gb : l.b, (size_t)l.cout * sizeof(float), cudaMemcpyDeviceToHost, n->st));
    PM_CUDA(cudaStreamSynchronize(n->st));
    return PTYCHO_OK;
}

extern "C" int wsnet_get_params(wsnet n, int layer, float *h_w, float *h_b) {
    return get_pair(n, layer, h_w, h_b, false, "wsnet_get_params");
}

extern "C" int wsnet_get_grads(wsnet n, int layer, float *h_dw, float *h_db) {
    return get_pair(n, layer, h_dw, h_db, true, "wsnet_get_grads");
}

extern "C" int wsnet_forward(wsnet n, const void *d_x, int B, float *d_y) {
    if (!n || !d_x || !d_y) return pm::fail(PTYCHO_EINVAL, "wsnet_forward: NULL argument");
    if (!check_batch(n, B, "wsnet_forward")) return PTYCHO_EINVAL;
    return forward(n, static_cast<const bf16 *>(d_x), B, d_y);
}

extern "C" int wsnet_backward(wsnet n, const void *d_x, const float *d_t, int B, double *h_loss) {
    if (!n || !d_x || !d_t) return pm::fail(PTYCHO_EINVAL, "wsnet_backward: NULL argument");
    if (!check_batch(n, B, "wsnet_backward")) return PTYCHO_EINVAL;
    return backward(n, static_cast<const bf16 *>(d_x), d_t, B, h_loss);
}

extern "C" int wsnet_adam(wsnet n, float lr) {
    if (!n || !(lr >= 0.f) || !std::isfinite(lr)) return pm::fail(PTYCHO_EINVAL, "wsnet_adam: bad network or rate");
    return adam(n, lr);
}

extern "C" int wsnet_train_step(wsnet n, const void *d_x, const float *d_t, int B, float lr, double *h_loss) {
    int rc = wsnet_backward(n, d_x, d_t, B, h_loss);
    if (rc) return rc;
    return wsnet_adam(n, lr);
}

extern "C" void wsnet_destroy(wsnet n) { free_net(n); }

extern "C" int ws_preprocess(const float *d_fused, int J, int N, void *d_x, void *cuda_stream) {
    if (J < 0 || N < 2 || (N & 1)) return pm::fail(PTYCHO_EINVAL, "ws_preprocess: J = %d, N = %d", J, N);
    if (J == 0) return PTYCHO_OK;
    if (!d_fused || !d_x) return pm::fail(PTYCHO_EINVAL, "ws_preprocess: NULL pointer");
    k_preprocess<<<nblk((size_t)J * (N / 2) * (N / 2)), kT, 0, (cudaStream_t)cuda_stream>>>(d_fused, J, N,
                                                                                           static_cast<bf16 *>(d_x));
    PM_LAUNCHED("k_preprocess");
    return PTYCHO_OK;
}

extern "C" int ws_targets(const void *d_obj, int M, const int32_t *d_pos, int J, int N, float *d_t, void *cuda_stream) {
    if (J < 0 || N < 4 || (N & 3) || M < N) return pm::fail(PTYCHO_EINVAL, "ws_targets: M = %d, N = %d", M, N);
    if (J == 0) return PTYCHO_OK;
    if (!d_obj || !d_pos || !d_t) return pm::fail(PTYCHO_EINVAL, "ws_targets: NULL pointer");
    k_targets<<<nblk((size_t)J * (N / 4) * (N / 4)), kT, 0, (cudaStream_t)cuda_stream>>>(
        static_cast<const float2 *>(d_obj), M, reinterpret_cast<const int2 *>(d_pos), J, N, d_t);
    PM_LAUNCHED("k_targets");
    return PTYCHO_OK;
}

extern "C" int ws_stitch(const float *d_pred, const int32_t *d_pos, int J, const void *d_probe, int N, int M,
                         void *d_obj, void *cuda_stream) {
    if (J < 1 || N < 8 || (N & 3) || M < N || (M & 3))
        return pm::fail(PTYCHO_EINVAL, "ws_stitch: J = %d, N = %d, M = %d", J, N, M);
    if (!d_pred || !d_pos || !d_probe || !d_obj) return pm::fail(PTYCHO_EINVAL, "ws_stitch: NULL pointer");
    cudaStream_t st = (cudaStream_t)cuda_stream;
    const int n = N / 4, Mc = M / 4;
    // one scratch block: num (float2, Mc^2) | den (Mc^2) | wgt (n^2) | dmax (1)
    void *blk = nullptr;
    const size_t MMc = (size_t)Mc * Mc;
    PM_CUDA(pm::dev_malloc_async(&blk, MMc * sizeof(float2) + (MMc + (size_t)n * n + 1) * sizeof(float), st));
    float2 *num = static_cast<float2 *>(blk);
    float *den = reinterpret_cast<float *>(num + MMc);
    float *wgt = den + MMc;
    float *dmax = wgt + (size_t)n * n;
    k_coarse_weights<<<nblk((size_t)n * n), kT, 0, st>>>(static_cast<const float2 *>(d_probe), N, wgt);
    k_stitch_coarse<<<nblk((size_t)Mc * Mc), kT, 0, st>>>(d_pred, reinterpret_cast<const int2 *>(d_pos), J, n, wgt,
                                                         Mc, num, den);
    k_max_reduce<<<1, kT, 0, st>>>(den, Mc * Mc, dmax);
    k_stitch_upsample<<<nblk((size_t)M * M), kT, 0, st>>>(num, den, dmax, Mc, M, static_cast<float2 *>(d_obj));
    cudaError_t e = cudaGetLastError();
    cudaFreeAsync(blk, st);
    if (e != cudaSuccess) return pm::cuda_fail(e, "ws_stitch");
    return PTYCHO_OK;
}
