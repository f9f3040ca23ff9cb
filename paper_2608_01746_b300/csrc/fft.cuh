// Register/shared-memory radix FFT for N = R * R points (R = 4, 8, 16) executed by a group of
// R threads.  Thread t of a group holds the elements x[t + R m], m = 0 .. R-1, in registers
// and, after the transform, X[t + R m] (natural order in both directions).
//
// Decomposition (n = n2 + R n1, k = k1 + R k2, W_N = exp(sign 2 pi i / N)):
//   X[k1 + R k2] = sum_n2 W_R^(n2 k2) [ W_N^(n2 k1) sum_n1 x[n2 + R n1] W_R^(n1 k1) ]
// Thread t = n2 does the inner R-point DFT in registers and the twiddle, the group exchanges
// through a padded R x (R+1) shared-memory buffer (conflict-free for both the write and the
// transposed read), then thread t = k1 does the outer R-point DFT in registers.
#pragma once

#include "common.cuh"

namespace pm {

// cos(2 pi k / 16), sin(2 pi k / 16) for k = 0 .. 7
__device__ __forceinline__ float cos16(int k) {
    switch (k) {
        case 0: return 1.0f;
        case 1: return 0.92387953251128674f;
        case 2: return 0.70710678118654752f;
        case 3: return 0.38268343236508977f;
        case 4: return 0.0f;
        case 5: return -0.38268343236508977f;
        case 6: return -0.70710678118654752f;
        default: return -0.92387953251128674f;
    }
}
__device__ __forceinline__ float sin16(int k) {
    switch (k) {
        case 0: return 0.0f;
        case 1: return 0.38268343236508977f;
        case 2: return 0.70710678118654752f;
        case 3: return 0.92387953251128674f;
        case 4: return 1.0f;
        case 5: return 0.92387953251128674f;
        case 6: return 0.70710678118654752f;
        default: return 0.38268343236508977f;
    }
}

// v * exp(SIGN * 2 pi i k16 / 16) for a compile-time-foldable k16 in [0, 8).
template <int SIGN>
__device__ __forceinline__ float2 rot16(float2 v, int k16) {
    if (k16 == 0) return v;
    if (k16 == 4) return SIGN < 0 ? make_float2(v.y, -v.x) : make_float2(-v.y, v.x);
    const float c = cos16(k16), s = SIGN * sin16(k16);
    return make_float2(v.x * c - v.y * s, v.x * s + v.y * c);
}

// Bit reversal of i in [0, R), written out so that unrolled indices fold to constants.
template <int R>
__device__ __forceinline__ int bitrev(int i) {
    if constexpr (R == 2) return i;
    else if constexpr (R == 4) return ((i & 1) << 1) | ((i & 2) >> 1);
    else if constexpr (R == 8) return ((i & 1) << 2) | (i & 2) | ((i & 4) >> 2);
    else return ((i & 1) << 3) | ((i & 2) << 1) | ((i & 4) >> 1) | ((i & 8) >> 3);
}

// Radix-2 decimation-in-time butterflies of span LEN, then the next stage.
template <int R, int SIGN, int LEN>
__device__ __forceinline__ void dit_stage(float2 (&y)[R]) {
#pragma unroll
    for (int i = 0; i < R; i += LEN) {
#pragma unroll
        for (int k = 0; k < LEN / 2; ++k) {
            const float2 a = y[i + k];
            const float2 b = rot16<SIGN>(y[i + k + LEN / 2], k * (16 / LEN));
            y[i + k] = cadd_x2(a, b);
            y[i + k + LEN / 2] = csub_x2(a, b);
        }
    }
    if constexpr (LEN < R) dit_stage<R, SIGN, LEN * 2>(y);
}

// In-register R-point DFT (R in {2, 4, 8, 16}): d[k] <- sum_n d[n] exp(SIGN 2 pi i n k / R).
template <int R, int SIGN>
__device__ __forceinline__ void dft_reg(float2 (&d)[R]) {
    float2 y[R];
#pragma unroll
    for (int i = 0; i < R; ++i) y[i] = d[bitrev<R>(i)];
    dit_stage<R, SIGN, 2>(y);
#pragma unroll
    for (int i = 0; i < R; ++i) d[i] = y[i];
}

// Group FFT of N = R*R points (see the file comment).  `xb` is the group's R*(R+1) float2
// exchange buffer, `tw` the table W_N^(a b) (forward sign) indexed [a * R + b] (symmetric),
// `t` the thread's rank in the group.  The caller's group is a warp-aligned run of R lanes;
// `__syncwarp` orders the exchange.
template <int R, int SIGN>
__device__ __forceinline__ void fft_group(float2 (&d)[R], float2 *xb, const float2 *tw, int t) {
    dft_reg<R, SIGN>(d);
#pragma unroll
    for (int k1 = 1; k1 < R; ++k1) {
        float2 w = tw[k1 * R + t];
        if (SIGN > 0) w.y = -w.y;
        d[k1] = cmul(d[k1], w);
    }
    __syncwarp();
#pragma unroll
    for (int k1 = 0; k1 < R; ++k1) xb[k1 * (R + 1) + t] = d[k1];
    __syncwarp();
#pragma unroll
    for (int n2 = 0; n2 < R; ++n2) d[n2] = xb[t * (R + 1) + n2];
    dft_reg<R, SIGN>(d);
}

}  // namespace pm

namespace pm {

// Same transform as fft_group, with an unpadded R*R exchange buffer laid out with an XOR
// swizzle (element (k1, n2) at k1 * R + (n2 ^ k1)): conflict-free for the write and the
// transposed read without padding.  `tw_reg[k1]` holds W_N^(t k1) (forward sign) for this
// thread's t, so the twiddles cost no shared-memory traffic.
template <int R, int SIGN>
__device__ __forceinline__ void fft_group_x(float2 (&d)[R], float2 *xb, const float2 (&tw_reg)[R], int t) {
    dft_reg<R, SIGN>(d);
#pragma unroll
    for (int k1 = 1; k1 < R; ++k1) {
        float2 w = tw_reg[k1];
        if (SIGN > 0) w.y = -w.y;
        d[k1] = cmul(d[k1], w);
    }
    __syncwarp();
#pragma unroll
    for (int k1 = 0; k1 < R; ++k1) xb[k1 * R + (t ^ k1)] = d[k1];
    __syncwarp();
#pragma unroll
    for (int n2 = 0; n2 < R; ++n2) d[n2] = xb[t * R + (n2 ^ t)];
    dft_reg<R, SIGN>(d);
}

}  // namespace pm

namespace pm {

// fft_group_x with the twiddles read from a shared-memory table tw[k1 * R + t] = W_N^(t k1)
// (forward sign; consecutive t are consecutive words, so the reads are conflict-free).
template <int R, int SIGN>
__device__ __forceinline__ void fft_group_xs(float2 (&d)[R], float2 *xb, const float2 *tw, int t) {
    dft_reg<R, SIGN>(d);
#pragma unroll
    for (int k1 = 1; k1 < R; ++k1) {
        float2 w = tw[k1 * R + t];
        if (SIGN > 0) w.y = -w.y;
        d[k1] = cmul(d[k1], w);
    }
    __syncwarp();
#pragma unroll
    for (int k1 = 0; k1 < R; ++k1) xb[k1 * R + (t ^ k1)] = d[k1];
    __syncwarp();
#pragma unroll
    for (int n2 = 0; n2 < R; ++n2) d[n2] = xb[t * R + (n2 ^ t)];
    dft_reg<R, SIGN>(d);
}

}  // namespace pm

namespace pm {

constexpr int kTw128Pitch = 9;                       // twiddle table of the N = 128 transforms
constexpr int kTw128Size = 16 * kTw128Pitch;

// N = 128 = 8 x 16 by a group of 8 threads holding 16 elements each.  tw[k1 * 9 + n] = W_128^(n k1)
// (forward sign), k1 < 16, n < 8: rows of 9, so that the 8 threads of a group reading
// W_128^(k1 n) for their own k1 = 2t + i (fft128_rev_to_nat) hit distinct banks, as do those
// reading one row (fft128_nat_to_rev).  The exchange buffer is [8][18] float2 per group (rows 18 apart;
// with groups 145 float2 apart, both exchange patterns of two groups sharing a half-warp hit
// distinct banks).
//
// fft128_nat_to_rev: thread t holds x[t + 8 m] (natural order).  With n = n2 + 8 n1 and
// k = k1 + 16 k2:
//   X[k1 + 16 k2] = sum_n2 W_8^(n2 k2) [ W_128^(n2 k1) sum_n1 x[n2 + 8 n1] W_16^(n1 k1) ]
// thread t = n2 does the 16-point DFT and the twiddle, the group exchanges, then thread t takes
// k1 = 2t and 2t + 1 and does two 8-point DFTs: afterwards d[8 i + k2] = X[2t + i + 16 k2].
template <int SIGN>
__device__ __forceinline__ void fft128_nat_to_rev(float2 (&d)[16], float2 *xb, const float2 *tw, int t) {
    dft_reg<16, SIGN>(d);
#pragma unroll
    for (int k1 = 1; k1 < 16; ++k1) {
        float2 w = tw[k1 * kTw128Pitch + t];
        if (SIGN > 0) w.y = -w.y;
        d[k1] = cmul(d[k1], w);
    }
    __syncwarp();
#pragma unroll
    for (int k1 = 0; k1 < 16; ++k1) xb[t * 18 + k1] = d[k1];
    __syncwarp();
#pragma unroll
    for (int i = 0; i < 2; ++i) {
        float2 e[8];
#pragma unroll
        for (int n2 = 0; n2 < 8; ++n2) e[n2] = xb[n2 * 18 + 2 * t + i];
        dft_reg<8, SIGN>(e);
#pragma unroll
        for (int k2 = 0; k2 < 8; ++k2) d[8 * i + k2] = e[k2];
    }
}

// The mirror split: d[8 i + k2] = X[2t + i + 16 k2] in, x[t + 8 m] out.  With k = k1 + 16 k2,
// n = n1 + 8 n2:
//   x[n1 + 8 n2] = sum_k1 W_16^(k1 n2) [ W_128^(k1 n1) sum_k2 X[k1 + 16 k2] W_8^(k2 n1) ]
// (exponent signs SIGN): two 8-point DFTs over k2 (k1 = 2t, 2t + 1), the twiddle, the exchange,
// then thread t = n1 does the 16-point DFT over k1.
template <int SIGN>
__device__ __forceinline__ void fft128_rev_to_nat(float2 (&d)[16], float2 *xb, const float2 *tw, int t) {
#pragma unroll
    for (int i = 0; i < 2; ++i) {
        float2 e[8];
#pragma unroll
        for (int k2 = 0; k2 < 8; ++k2) e[k2] = d[8 * i + k2];
        dft_reg<8, SIGN>(e);
        const int k1 = 2 * t + i;
#pragma unroll
        for (int n1 = 0; n1 < 8; ++n1) {
            float2 w = tw[k1 * kTw128Pitch + n1];
            if (SIGN > 0) w.y = -w.y;
            d[8 * i + n1] = cmul(e[n1], w);
        }
    }
    __syncwarp();
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int n1 = 0; n1 < 8; ++n1) xb[n1 * 18 + 2 * t + i] = d[8 * i + n1];
    __syncwarp();
#pragma unroll
    for (int k1 = 0; k1 < 16; ++k1) d[k1] = xb[t * 18 + k1];
    dft_reg<16, SIGN>(d);
}

// Position of element e of thread t after fft128_nat_to_rev: 2t + e / 8 + 16 (e % 8).
__device__ __forceinline__ int rev128(int t, int e) { return 2 * t + (e >> 3) + 16 * (e & 7); }

}  // namespace pm
