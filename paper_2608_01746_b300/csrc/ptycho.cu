// Iterative ptychographic reconstruction on one GPU (§3.3 forward model, Eqs. 2-3).
//
// One iteration (full-batch alternating projections):
//   exit waves     per position j (persistent grids):
//                  psi = P * O_j  ->  row FFTs  ->  column FFTs, modulus replacement against
//                  A_j and Fourier error, inverse column FFTs  ->  inverse row FFTs  ->  psi_j'
//                  k_exit_wave<R> (N = 16, 64): one CTA per position, the whole N x N tile
//                  in shared memory.  k_exit_wave128 (N = 128): one CTA per position, groups of
//                  8 threads with 16 elements each, the tile in shared memory.
//                  k_exit_wave_tma (N = 256): the 512 KB tile does not fit one SM, so each
//                  CTA streams it through a private slot in global memory (L2) with TMA bulk
//                  tensor copies, rows and columns in batches of 16 or 32 (fft.cuh radix-16
//                  group transforms in registers and shared memory).
//   k_object_gather  owner-computes object update: each 8 x 32 object tile sums
//                  conj(P) psi_j' and |P|^2 over the positions whose patch covers it, in
//                  ascending j (deterministic, no atomics).
//   k_apply        O = num / (den + alpha_O max den) on pixels inside some scan patch.
//   k_probe_partial / k_probe_reduce / k_apply
//                  P = sum_j conj(O_j) psi_j' / (sum_j |O_j|^2 + alpha_P max), with the new
//                  object, as fixed-order partial sums over position chunks.
//   k_error_reduce   per-iteration Fourier error in FP64, fixed order (ePIE by colour; the
//                    alternating projections form it in block 0 of the object step's k_apply).
#include <algorithm>
#include <climits>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include <cuda.h>

#include "common.cuh"
#include "dftgemm.h"
#include "fft.cuh"
#include "tma.cuh"
#include "tcgen05.cuh"
#include "tmap.h"


namespace {

constexpr int kThreads = 256;
constexpr int kTW = 32;          // tile width (columns) of the object gather and probe sums
constexpr int kListChunk = 512;  // tile-list entries staged per chunk in the object gather
constexpr int kTR = 8;           // tile height (rows): one register per row and lane

enum { ST_EXIT = 0, ST_OBJECT = 1, ST_PROBE = 2, ST_ERROR = 3, ST_COUNT = 4 };

// What an exit-wave kernel launch does per unit of work.
//   XM_FULL  unit = position j: psi_j' = F^-1[A_j F(P O_j) / |F(P O_j)|] (one probe mode)
//   XM_FWD   unit = (j, m): Psi_jm = F(P_m O_j), unitary, into psi[j][m] (row-major, DC at 0)
//   XM_INV   unit = (j, m): psi[j][m] <- F^-1 psi[j][m] (after the mode-summed modulus step)
//   XM_LIST  as XM_FULL for the positions list[0 .. count) only (ePIE colours)
enum { XM_FULL = 0, XM_FWD = 1, XM_INV = 2, XM_LIST = 3 };

struct ExitArgs {
    // XM_FULL only: when `table` is set, the launch serves several datasets of the same N: unit
    // iu belongs to the dataset d with ustart[d] <= iu < ustart[d + 1] and uses table[d].
    const ExitArgs *table;
    const int *ustart;
    int ntable;
    const float2 *obj;
    const float2 *probe;     // [Q][N][N]
    const float *amp;        // [J][N][N] column-major per position: amp[j][kx][ky]
    const int2 *pos;         // (y, x)
    float2 *psi;             // [J][Q][N][N] row-major
    double *err;             // [J] Fourier error per position (XM_FULL)
    const int *list;         // XM_FULL: if not NULL, process positions list[0 .. count)
    int count;
    int M, J, Q;
};

// Shared memory of the small-tile exit-wave kernel: twiddles, the FFT groups' exchange
// buffers, and the whole N x N tile (pitch N + 1).
template <int R>
constexpr size_t exit_smem_bytes() {
    constexpr int N = R * R;
    constexpr int G = kThreads / R;
    return sizeof(float2) * ((size_t)N + (size_t)G * R * (R + 1) + (size_t)N * (N + 1));
}

// Per-unit body of the N <= 64 exit wave, run by NT threads (rank tid) that synchronise with
// sync(): the whole N x N tile in shared memory: row FFTs, column FFTs (with the modulus
// replacement between the forward and inverse column transforms in XM_FULL), inverse row FFTs.
// c: the unit's dataset arguments; u: the unit (position j, or j Q + m); tw: [N] twiddles;
// xb_all: [NT / R][R][R + 1] exchange buffers; rows: [N][N + 1]; s_red: [NT / 32].
template <int R, int XM, int NT, typename Sync>
__device__ __forceinline__ void exit_small_unit(const ExitArgs &c, int u, const float2 *tw, float2 *xb_all,
                                                float2 *rows, double *s_red, int tid, int Q, Sync sync) {
    constexpr int N = R * R;
    constexpr int G = NT / R;                // FFT groups
    constexpr int TP = N + 1;                // padded row pitch
    constexpr bool kFull = (XM == XM_FULL || XM == XM_LIST);
    const int t = tid % R, g = tid / R;
    float2 *xb = xb_all + g * R * (R + 1);
    // Row / column of group g within each pass of G: at N = 64 the two groups of a half-warp
    // take rows (columns) 8 apart, whose 8-byte accesses with the row pitch of 65 then fall on
    // distinct banks (consecutive rows would overlap on 14 of their 16 banks).
    const int gp = (R == 8) ? (((g >> 1) & 7) | ((g & 1) << 3) | (g & ~15)) : g;
    const float invN = 1.0f / (float)N;
    const int M = c.M;
    const int j = kFull ? u : u / Q;
    const int mode = kFull ? 0 : u % Q;
    float2 *psi_u = c.psi + (size_t)u * N * N;          // u = j (one mode) or j Q + m
    if constexpr (XM != XM_INV) {
        // (1) psi = P_m * O_j, forward row FFTs in place
        const int2 pj = c.pos[j];
        for (int r0 = 0; r0 < N; r0 += G) {
            const int r = r0 + gp;
            if (r < N) {                                 // warp-uniform (see fft.cuh)
                float2 d[R];
                const float2 *orow = c.obj + (size_t)(pj.x + r) * M + pj.y;
                const float2 *prow = c.probe + (size_t)mode * N * N + (size_t)r * N;
#pragma unroll
                for (int m = 0; m < R; ++m) d[m] = cmul(__ldg(prow + t + R * m), __ldg(orow + t + R * m));
                pm::fft_group<R, -1>(d, xb, tw, t);
#pragma unroll
                for (int m = 0; m < R; ++m) rows[r * TP + t + R * m] = d[m];
            }
        }
    } else {
        for (int i = tid; i < N * N; i += NT) rows[(i / N) * TP + i % N] = psi_u[i];
    }
    sync();
    // (2) column FFTs: forward (+ modulus + inverse in XM_FULL) or inverse (XM_INV)
    float err = 0.f;
    const float *amp_j = c.amp + (size_t)j * N * N;
    for (int c0 = 0; c0 < N; c0 += G) {
        const int col = c0 + gp;
        if (col < N) {
            float2 d[R];
#pragma unroll
            for (int m = 0; m < R; ++m) d[m] = rows[(t + R * m) * TP + col];
            if constexpr (XM == XM_INV) {
                pm::fft_group<R, +1>(d, xb, tw, t);
            } else {
                pm::fft_group<R, -1>(d, xb, tw, t);
                if constexpr (!kFull) {                 // spectra for the modes' common modulus
#pragma unroll
                    for (int m = 0; m < R; ++m) d[m] = cscale(d[m], invN);
                }
            }
            if constexpr (kFull) {
                // d = N Psi (the forward transform unscaled): |Psi| = |d| / N, and the
                // projection A Psi / |Psi| = A d / |d| does not depend on the scale
#pragma unroll
                for (int m = 0; m < R; ++m) {
                    const float2 X = d[m];
                    const float A = __ldg(amp_j + (size_t)col * N + t + R * m);
                    const float mag2 = cabs2(X);
                    if (mag2 > 0.f) {
                        const float inv = rsqrtf(mag2);
                        const float dm = mag2 * inv * invN - A;
                        err += dm * dm;
                        d[m] = cscale(X, A * inv);
                    } else {
                        err += A * A;
                        d[m] = make_float2(A, 0.f);
                    }
                }
                pm::fft_group<R, +1>(d, xb, tw, t);
            }
#pragma unroll
            for (int m = 0; m < R; ++m) rows[(t + R * m) * TP + col] = d[m];
        }
    }
    sync();
    if constexpr (XM == XM_FWD) {
        for (int i = tid; i < N * N; i += NT) psi_u[i] = rows[(i / N) * TP + i % N];
    } else {
        // (3) inverse row FFTs, psi' written row-major
        for (int r0 = 0; r0 < N; r0 += G) {
            const int r = r0 + gp;
            if (r < N) {
                float2 d[R];
#pragma unroll
                for (int m = 0; m < R; ++m) d[m] = rows[r * TP + t + R * m];
                pm::fft_group<R, +1>(d, xb, tw, t);
#pragma unroll
                for (int m = 0; m < R; ++m) psi_u[(size_t)r * N + t + R * m] = cscale(d[m], invN);
            }
        }
    }
    if constexpr (kFull) {
        // Fourier error of position j (FP64 sum over the NT threads)
        double e = (double)err;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) e += __shfl_xor_sync(0xffffffffu, e, o);
        if ((tid & 31) == 0) s_red[tid >> 5] = e;
        sync();
        if (tid == 0) {
            double sum = 0.0;
            for (int w = 0; w < NT / 32; ++w) sum += s_red[w];
            c.err[j] = sum;
        }
    }
    sync();          // the next unit's first pass overwrites the tile
}

// The N x N twiddle table W_N^(a b) (forward sign) indexed [a * R + b], N = R * R.
template <int R>
__device__ __forceinline__ void fill_twiddles(float2 *tw, int tid, int nt) {
    constexpr int N = R * R;
    for (int i = tid; i < N; i += nt) {
        const int ab = (i / R) * (i % R);
        double sn, cs;
        sincospi(-2.0 * (double)ab / (double)N, &sn, &cs);
        tw[i] = make_float2((float)cs, (float)sn);
    }
}

// Dataset of unit iu of a multi-dataset launch: the d with ustart[d] <= iu < ustart[d + 1].
__device__ __forceinline__ int table_lookup(const int *ustart, int ntable, int iu) {
    int lo = 0, hi = ntable - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (__ldg(ustart + mid) <= iu) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// N <= 64: one CTA per unit at a time (persistent grid).
template <int R, int XM>
__global__ void __launch_bounds__(kThreads) k_exit_wave(ExitArgs a) {
    constexpr int N = R * R;
    constexpr int G = kThreads / R;          // FFT groups per CTA
    extern __shared__ float2 smem[];
    float2 *tw = smem;                       // [N] W_N^(a b), forward sign
    float2 *xb_all = tw + N;                 // [G][R][R+1]
    float2 *rows = xb_all + G * R * (R + 1); // [N][N+1]
    __shared__ double s_red[kThreads / 32];
    const int tid = threadIdx.x;
    fill_twiddles<R>(tw, tid, kThreads);
    __syncthreads();
    constexpr bool kFull = (XM == XM_FULL || XM == XM_LIST);
    const int units = (XM == XM_LIST) ? a.count : (kFull ? a.J : a.J * a.Q);
    for (int iu = blockIdx.x; iu < units; iu += gridDim.x) {
        int u = (XM == XM_LIST) ? a.list[iu] : iu;
        ExitArgs c = a;
        if (XM == XM_FULL && a.table) {
            const int d = table_lookup(a.ustart, a.ntable, iu);
            c = a.table[d];
            u = iu - __ldg(a.ustart + d);
        }
        exit_small_unit<R, XM, kThreads>(c, u, tw, xb_all, rows, s_red, tid, a.Q, [] { __syncthreads(); });
    }
}

// N = 128 = 8 x 16 (one probe mode; XM_FULL, XM_LIST; dataset tables as k_exit_wave): groups
// of 8 threads, 16 elements each.  Forward transforms leave digit-reversed order
// (fft128_nat_to_rev), inverse transforms consume it (fft128_rev_to_nat), so the tile holds the
// row spectrum at its true frequencies and each column is forward-transformed, projected and
// inverse-transformed in registers.
constexpr int kThreads128 = 512;         // 64 groups of 8 threads: 64 rows / columns per pass

constexpr int kXB128 = 145;              // exchange buffer per group: [8][18] float2 + 1 (bank offset)

constexpr size_t exit128_smem_bytes() {
    constexpr int N = 128, G = kThreads128 / 8;
    return sizeof(float2) * ((size_t)pm::kTw128Size + (size_t)G * kXB128 + (size_t)N * (N + 1));
}

// Per-unit body of the N = 128 exit wave (position j of dataset c), kThreads128 threads.
// tw: [16][kTw128Pitch] W_128^(k1 n); xb_all: [G][kXB128]; rows: [N][N + 1]; s_red: [16].
__device__ __forceinline__ void exit128_unit(const ExitArgs &c, int j, const float2 *tw, float2 *xb_all,
                                             float2 *rows, double *s_red) {
    constexpr int N = 128, R1 = 8, E = 16;
    constexpr int G = kThreads128 / R1;
    constexpr int TP = N + 1;
    const int tid = threadIdx.x;
    const int t = tid % R1, g = tid / R1;
    float2 *xb = xb_all + g * kXB128;
    const float invN = 1.0f / (float)N;
    const int M = c.M;
    float2 *psi_j = c.psi + (size_t)j * N * N;
    const int2 pj = c.pos[j];
    // (1) psi = P O_j, forward row FFTs; stored at the true frequency kx
    for (int r0 = 0; r0 < N; r0 += G) {
        const int r = r0 + g;
        float2 d[E];
        const float2 *orow = c.obj + (size_t)(pj.x + r) * M + pj.y;
        const float2 *prow = c.probe + (size_t)r * N;
#pragma unroll
        for (int m = 0; m < E; ++m) d[m] = cmul(__ldg(prow + t + R1 * m), __ldg(orow + t + R1 * m));
        pm::fft128_nat_to_rev<-1>(d, xb, tw, t);
#pragma unroll
        for (int e = 0; e < E; ++e) rows[r * TP + pm::rev128(t, e)] = d[e];
    }
    __syncthreads();
    // (2) columns: forward, modulus (ky = rev128(t, e)), inverse back to natural rows
    float err = 0.f;
    const float *amp_j = c.amp + (size_t)j * N * N;
    // the 4 groups of a warp take columns 8 apart: with the row pitch of 129 float2 their
    // column reads and writes fall in distinct banks (2 t + 16 q words)
    const int col_off = 8 * (g & 3) + ((g >> 2) & 7) + 32 * (g >> 5);
    for (int c0 = 0; c0 < N; c0 += G) {
        const int col = c0 + col_off;
        float2 d[E];
#pragma unroll
        for (int m = 0; m < E; ++m) d[m] = rows[(t + R1 * m) * TP + col];
        pm::fft128_nat_to_rev<-1>(d, xb, tw, t);
        // d = N Psi (the forward transform unscaled); the projection A d / |d| is scale-free
#pragma unroll
        for (int e = 0; e < E; ++e) {
            const float2 X = d[e];
            const float A = __ldg(amp_j + (size_t)col * N + pm::rev128(t, e));
            const float mag2 = cabs2(X);
            if (mag2 > 0.f) {
                const float inv = rsqrtf(mag2);
                const float dm = mag2 * inv * invN - A;
                err += dm * dm;
                d[e] = cscale(X, A * inv);
            } else {
                err += A * A;
                d[e] = make_float2(A, 0.f);
            }
        }
        pm::fft128_rev_to_nat<+1>(d, xb, tw, t);
#pragma unroll
        for (int m = 0; m < E; ++m) rows[(t + R1 * m) * TP + col] = d[m];
    }
    __syncthreads();
    // (3) inverse row FFTs from the true frequencies, psi' written row-major
    for (int r0 = 0; r0 < N; r0 += G) {
        const int r = r0 + g;
        float2 d[E];
#pragma unroll
        for (int e = 0; e < E; ++e) d[e] = rows[r * TP + pm::rev128(t, e)];
        pm::fft128_rev_to_nat<+1>(d, xb, tw, t);
#pragma unroll
        for (int m = 0; m < E; ++m) psi_j[(size_t)r * N + t + R1 * m] = cscale(d[m], invN);
    }
    // Fourier error of position j (FP64 block sum)
    double e64 = (double)err;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) e64 += __shfl_xor_sync(0xffffffffu, e64, o);
    if ((tid & 31) == 0) s_red[tid >> 5] = e64;
    __syncthreads();
    if (tid == 0) {
        double sum = 0.0;
        for (int w = 0; w < kThreads128 / 32; ++w) sum += s_red[w];
        c.err[j] = sum;
    }
    __syncthreads();
}

// tw[k1 * kTw128Pitch + n] = W_128^(k1 n) (forward sign)
__device__ __forceinline__ void fill_twiddles128(float2 *tw, int tid, int nt) {
    for (int i = tid; i < pm::kTw128Size; i += nt) {
        double sn, cs;
        sincospi(-2.0 * (double)((i / pm::kTw128Pitch) * (i % pm::kTw128Pitch)) / 128.0, &sn, &cs);
        tw[i] = make_float2((float)cs, (float)sn);
    }
}

template <int XM>
__global__ void __launch_bounds__(kThreads128) k_exit_wave128(ExitArgs a) {
    constexpr int N = 128;
    constexpr int G = kThreads128 / 8;
    extern __shared__ float2 smem[];
    float2 *tw = smem;                       // [16][kTw128Pitch] W_128^(k1 n), forward sign
    float2 *xb_all = tw + pm::kTw128Size;    // [G][kXB128]
    float2 *rows = xb_all + G * kXB128;      // [N][N+1]
    __shared__ double s_red[kThreads128 / 32];
    fill_twiddles128(tw, threadIdx.x, kThreads128);
    __syncthreads();
    const int units = (XM == XM_LIST) ? a.count : a.J;
    for (int iu = blockIdx.x; iu < units; iu += gridDim.x) {
        int j = (XM == XM_LIST) ? a.list[iu] : iu;
        ExitArgs c = a;
        if (XM == XM_FULL && a.table) {
            const int d = table_lookup(a.ustart, a.ntable, iu);
            c = a.table[d];
            j = iu - __ldg(a.ustart + d);
        }
        exit128_unit(c, j, tw, xb_all, rows, s_red);
    }
}

// Mixed-state modulus constraint, one block per position: S = sum_m |Psi_m|^2,
// error (sqrt(S) - A)^2, Psi_m <- Psi_m A / sqrt(S) (where S = 0: Psi_0 = A, other modes 0).
// psi: [J][Q][N][N] spectra (row-major, DC at 0); amp_nat: [J][N][N] row-major amplitudes.
// Q is a template parameter so that a pixel's Q loads are issued together and its values stay
// in registers between the sum and the scaling (one read and one write of each spectrum);
// 512-thread blocks, two per SM (64 registers), keep the last wave of positions short.
constexpr int kModThreads = 512;

template <int Q>
__global__ void __launch_bounds__(kModThreads, 2) k_modulus_modes(float2 *__restrict__ psi,
                                                               const float *__restrict__ amp_nat,
                                                               double *__restrict__ err, int N) {
    __shared__ double s_red[kModThreads / 32];
    const int j = blockIdx.x;
    const size_t NN = (size_t)N * N;
    float2 *pj = psi + (size_t)j * Q * NN;
    double acc = 0.0;
#pragma unroll 1
    for (size_t q = threadIdx.x; q < NN; q += kModThreads) {
        float2 v[Q];
#pragma unroll
        for (int m = 0; m < Q; ++m) v[m] = pj[m * NN + q];
        const float A = __ldg(amp_nat + (size_t)j * NN + q);
        float S = 0.f;
#pragma unroll
        for (int m = 0; m < Q; ++m) S += cabs2(v[m]);
        if (S > 0.f) {
            const float inv = rsqrtf(S);
            const float dm = S * inv - A;
            acc += (double)(dm * dm);
            const float sc = A * inv;
#pragma unroll
            for (int m = 0; m < Q; ++m) pj[m * NN + q] = cscale(v[m], sc);
        } else {
            acc += (double)A * (double)A;
            pj[q] = make_float2(A, 0.f);
#pragma unroll
            for (int m = 1; m < Q; ++m) pj[m * NN + q] = make_float2(0.f, 0.f);
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) s_red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double r = 0.0;
        for (int w = 0; w < kModThreads / 32; ++w) r += s_red[w];
        err[j] = r;
    }
}

int launch_modulus_modes(float2 *psi, const float *amp_nat, double *err, int J, int N, int Q, cudaStream_t st) {
    switch (Q) {
        case 2: k_modulus_modes<2><<<J, kModThreads, 0, st>>>(psi, amp_nat, err, N); break;
        case 3: k_modulus_modes<3><<<J, kModThreads, 0, st>>>(psi, amp_nat, err, N); break;
        case 4: k_modulus_modes<4><<<J, kModThreads, 0, st>>>(psi, amp_nat, err, N); break;
        case 5: k_modulus_modes<5><<<J, kModThreads, 0, st>>>(psi, amp_nat, err, N); break;
        case 6: k_modulus_modes<6><<<J, kModThreads, 0, st>>>(psi, amp_nat, err, N); break;
        case 7: k_modulus_modes<7><<<J, kModThreads, 0, st>>>(psi, amp_nat, err, N); break;
        case 8: k_modulus_modes<8><<<J, kModThreads, 0, st>>>(psi, amp_nat, err, N); break;
        default: return pm::fail(PTYCHO_EINVAL, "k_modulus_modes: Q = %d not in [2, 8]", Q);
    }
    PM_LAUNCHED("k_modulus_modes");
    return PTYCHO_OK;
}

// The mode-summed modulus constraint of the N = 256 mixed-state path without rewriting the
// spectra: per pixel the scale F = A / sqrt(S), S = sum_m |Psi_m|^2, which the inverse TMA
// kernel applies to each spectrum as it loads it (the same product the rewrite would store);
// where S = 0 the spectra are written here (Psi_0 = A, the other modes 0) and F = 1.  One
// block per (32-column strip, position): warp w takes rows w, w + 8, ..., lane = column; the
// strip's scales are transposed in shared memory into the amplitude order (column kx, then
// rows t + 16 k2 at t * 16 + k2) and written as 32 contiguous 1 KB columns.  The Fourier
// error of each strip goes to err[j * 8 + strip] (FP64, fixed order).
constexpr int kScaleCols = 32;

template <int Q>
__global__ void __launch_bounds__(kThreads) k_mode_scale(float2 *__restrict__ psi, const float *__restrict__ amp_nat,
                                                         float *__restrict__ fscale, double *__restrict__ err) {
    constexpr int N = 256;
    __shared__ float sF[kScaleCols][N + 1];
    __shared__ double s_red[kThreads / 32];
    const int strip = blockIdx.x, j = blockIdx.y;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const size_t NN = (size_t)N * N;
    float2 *pj = psi + (size_t)j * Q * NN;
    const int kx = strip * kScaleCols + lane;
    double acc = 0.0;
#pragma unroll 1
    for (int ky = warp; ky < N; ky += kThreads / 32) {
        const size_t q = (size_t)ky * N + kx;
        float2 v[Q];
#pragma unroll
        for (int m = 0; m < Q; ++m) v[m] = pj[m * NN + q];
        const float A = __ldg(amp_nat + (size_t)j * NN + q);
        float S = 0.f;
#pragma unroll
        for (int m = 0; m < Q; ++m) S += cabs2(v[m]);
        float F = 1.0f;
        if (S > 0.f) {
            const float inv = rsqrtf(S);
            const float dm = S * inv - A;
            acc += (double)(dm * dm);
            F = A * inv;
        } else {
            acc += (double)A * (double)A;
            pj[q] = make_float2(A, 0.f);
#pragma unroll
            for (int m = 1; m < Q; ++m) pj[m * NN + q] = make_float2(0.f, 0.f);
        }
        sF[lane][(ky & 15) * 16 + (ky >> 4)] = F;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (lane == 0) s_red[warp] = acc;
    __syncthreads();
    float *fj = fscale + (size_t)j * NN + (size_t)strip * kScaleCols * N;
    for (int i = threadIdx.x; i < kScaleCols * N; i += kThreads) fj[i] = sF[i / N][i % N];
    if (threadIdx.x == 0) {
        double r = 0.0;
        for (int w = 0; w < kThreads / 32; ++w) r += s_red[w];
        err[(size_t)j * (N / kScaleCols) + strip] = r;
    }
}

int launch_mode_scale(float2 *psi, const float *amp_nat, float *fscale, double *err, int J, int Q, cudaStream_t st) {
    const dim3 grid(256 / kScaleCols, J);
    switch (Q) {
        case 2: k_mode_scale<2><<<grid, kThreads, 0, st>>>(psi, amp_nat, fscale, err); break;
        case 3: k_mode_scale<3><<<grid, kThreads, 0, st>>>(psi, amp_nat, fscale, err); break;
        case 4: k_mode_scale<4><<<grid, kThreads, 0, st>>>(psi, amp_nat, fscale, err); break;
        case 5: k_mode_scale<5><<<grid, kThreads, 0, st>>>(psi, amp_nat, fscale, err); break;
        case 6: k_mode_scale<6><<<grid, kThreads, 0, st>>>(psi, amp_nat, fscale, err); break;
        case 7: k_mode_scale<7><<<grid, kThreads, 0, st>>>(psi, amp_nat, fscale, err); break;
        case 8: k_mode_scale<8><<<grid, kThreads, 0, st>>>(psi, amp_nat, fscale, err); break;
        default: return pm::fail(PTYCHO_EINVAL, "k_mode_scale: Q = %d not in [2, 8]", Q);
    }
    PM_LAUNCHED("k_mode_scale");
    return PTYCHO_OK;
}

#include "exit_tma.cuh"

// ---------------------------------------------------------------------------------------
// One persistent launch for the exit waves of many datasets of every probe size (batches of
// uneven scans).  A unit is (kind, dataset, first position, count): kind 256 and 128 take the
// whole 512-thread CTA for one position (the bodies of k_exit_wave_tma<32> and k_exit_wave128);
// kinds 64 and 16 run up to four positions at once, one per 128-thread quarter of the CTA
// (k_exit_wave's body with a named barrier per quarter).  Units are ordered by cost (256, 128,
// 64, 16) and dealt to the CTAs round-robin, one CTA per SM.  Per-position arithmetic is that of
// the per-size kernels, so the results are bit-identical to them.
constexpr int kAllThreads = 512;
constexpr int kQuarter = kAllThreads / 4;
template <int R>
__host__ __device__ constexpr size_t quarter_bytes() {
    constexpr int N = R * R, G = kQuarter / R;
    return sizeof(float2) * ((size_t)G * R * (R + 1) + (size_t)N * (N + 1));
}
__host__ __device__ constexpr size_t cmax(size_t a, size_t b) { return a > b ? a : b; }
constexpr size_t kAllScratch =
    cmax(3 * tma_buf_bytes<32>(),
         cmax(sizeof(float2) * ((size_t)(kThreads128 / 8) * kXB128 + 128 * 129), 4 * quarter_bytes<8>()));
constexpr size_t kAllTw = sizeof(float2) * (256 + pm::kTw128Size + 64 + 16);
constexpr size_t all_smem_bytes() { return 1024 + kAllScratch + kAllTw; }

// Out-of-line unit bodies of the one launch (N <= 128), so that the inlined N = 256 body keeps
// its registers.
__device__ __noinline__ void all_unit128(const ExitArgs &c, int j, const float2 *tw, unsigned char *base, double *s_red) {
    exit128_unit(c, j, tw, (float2 *)base, (float2 *)base + (kThreads128 / 8) * kXB128, s_red);
}
template <int R>
__device__ __noinline__ void all_unit_small(const ExitArgs &c, int u, const float2 *tw, unsigned char *base,
                                            double *s_red, int q, int qt) {
    constexpr int G = kQuarter / R;
    float2 *xb = (float2 *)(base + q * quarter_bytes<R>());
    auto sync = [q] { asm volatile("bar.sync %0, %1;" ::"r"(1 + q), "r"(kQuarter) : "memory"); };
    exit_small_unit<R, XM_FULL, kQuarter>(c, u, tw, xb, xb + G * R * (R + 1), s_red + 4 * q, qt, 1, sync);
}

__global__ void __launch_bounds__(kAllThreads, 1)
k_exit_wave_all(const int4 *__restrict__ units, int nunits, const ExitArgs *__restrict__ etab,
                const TmaArgs *__restrict__ ttab, const TmaMaps *__restrict__ mtab, int *status) {
    extern __shared__ unsigned char smem_raw[];
    unsigned char *base = (unsigned char *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    float2 *tw256 = (float2 *)(base + kAllScratch);
    float2 *tw128 = tw256 + 256, *tw64 = tw128 + pm::kTw128Size, *tw16 = tw64 + 64;
    __shared__ uint64_t s_bar[4];
    __shared__ double s_red[96];                  // the N = 256 unit: warp sums [2][32], batch sums [8]
    __shared__ uint32_t s_pending;
    const int tid = threadIdx.x;
    TmaPipe p;
    fill_twiddles128(tw128, tid, kAllThreads);
    fill_twiddles<8>(tw64, tid, kAllThreads);
    fill_twiddles<4>(tw16, tid, kAllThreads);
    tma_pipe_init(p, base, tw256, s_bar, &s_pending, s_red, blockIdx.x * 256);   // ends with a barrier
    for (int iu = blockIdx.x; iu < nunits && !p.failed; iu += gridDim.x) {
        const int4 un = units[iu];                       // (kind, dataset, first position, count)
        if (un.x == 256) {
            tma_apply(p, tma_unit<32, XM_FULL>(p, ttab[un.y], mtab[un.y], un.z));
        } else if (un.x == 128) {
            all_unit128(etab[un.y], un.z, tw128, base, s_red);
        } else {
            const int q = tid / kQuarter, qt = tid % kQuarter;
            if (q < un.w) {
                if (un.x == 64) all_unit_small<8>(etab[un.y], un.z + q, tw64, base, s_red, q, qt);
                else all_unit_small<4>(etab[un.y], un.z + q, tw16, base, s_red, q, qt);
            }
            __syncthreads();
        }
    }
    tma_pipe_finish(p, status);
}

// Each warp parks its kTR x 32 register tile in shared memory; after one barrier, thread
// (r, c) sums the 8 warps' values for pixel (r, c) in warp order (deterministic).
struct WarpTiles {
    float2 num[kThreads / 32][kTR][kTW];
    float den[kThreads / 32][kTR][kTW];
    unsigned hit[kThreads / 32][kTW];
};

__device__ __forceinline__ void combine_warps(const float2 (&acc)[kTR], const float (&dn)[kTR], unsigned hit,
                                              WarpTiles &wt, float2 &num, float &den, bool &covered) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int r = 0; r < kTR; ++r) {
        wt.num[warp][r][lane] = acc[r];
        wt.den[warp][r][lane] = dn[r];
    }
    wt.hit[warp][lane] = hit;
    __syncthreads();
    num = make_float2(0.f, 0.f);
    den = 0.f;
    covered = false;
    if (threadIdx.x < kTR * kTW) {
        const int r = threadIdx.x / kTW, c = threadIdx.x % kTW;
#pragma unroll
        for (int w = 0; w < kThreads / 32; ++w) {
            num = cadd(num, wt.num[w][r][c]);
            den += wt.den[w][r][c];
            covered |= ((wt.hit[w][c] >> r) & 1u) != 0u;
        }
    }
}

// Position lists of the object tiles: tile t's list holds (j, y, x, 0) for every position j
// whose N x N patch touches the tile, in ascending j, at tlist[tstart[t] ..).  One warp per
// tile walks the positions 32 at a time and packs the hits in order (ballot + prefix count).
// The host sized each list with the same test; an entry past the list's end is dropped.
__global__ void __launch_bounds__(kThreads) k_tile_lists(const int2 *__restrict__ pos, int J, int N, int ntx,
                                                         int ntiles, const int *__restrict__ tstart,
                                                         int4 *__restrict__ tlist) {
    const int t = (int)((blockIdx.x * (size_t)blockDim.x + threadIdx.x) >> 5);
    const int lane = threadIdx.x & 31;
    if (t >= ntiles) return;                                   // whole warps
    const int ty = t / ntx, tx = t % ntx;
    const int base = tstart[t], cap = tstart[t + 1] - base;
    int k = 0;
    for (int j0 = 0; j0 < J; j0 += 32) {
        const int j = j0 + lane;
        int2 p = make_int2(0, 0);
        bool hit = false;
        if (j < J) {
            p = pos[j];
            hit = p.x / kTR <= ty && ty <= (p.x + N - 1) / kTR && p.y / kTW <= tx && tx <= (p.y + N - 1) / kTW;
        }
        const unsigned m = __ballot_sync(0xffffffffu, hit);
        const int slot = k + __popc(m & ((1u << lane) - 1u));
        if (hit && slot < cap) tlist[base + slot] = make_int4(j, p.x, p.y, 0);
        k += __popc(m);
    }
}

// Owner-computes object numerator and denominator, one kTR x 32 object tile per block.
// Warp w takes every 8th position of the tile's (ascending) list; lane = tile column, and
// each lane keeps its column's kTR pixels in registers.
template <int QC>   // QC = 1: one probe mode (compile-time); 0: Q modes at run time
__global__ void __launch_bounds__(kThreads, QC == 1 ? 3 : 2) k_object_gather(
    const float2 *__restrict__ psi, const float2 *__restrict__ probe, const int2 *__restrict__ pos,
    const int4 *__restrict__ tlist, const int *__restrict__ torder, const int2 *__restrict__ trange,
    float2 *__restrict__ num, float *__restrict__ den, float *__restrict__ tile_max, int M, int N, int ntx, int Q) {
    __shared__ WarpTiles wt;
    __shared__ float s_max[kThreads / 32];
    __shared__ int3 s_list[kListChunk];
    pdl_allow_dependents();
    pdl_wait();                                       // the exit waves are complete
    const int tile = torder[blockIdx.x];              // longest position lists first
    const int ty0 = (tile / ntx) * kTR, tx0 = (tile % ntx) * kTW;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    float2 acc[kTR];
    float dn[kTR];
#pragma unroll
    for (int r = 0; r < kTR; ++r) { acc[r] = make_float2(0.f, 0.f); dn[r] = 0.f; }
    unsigned hit = 0u;
    const size_t NN = (size_t)N * N;
    const int nq = QC ? QC : Q;                       // probe modes (one for coherent data)
    // The tile's list is staged in shared memory in chunks (no entry prefetch in registers),
    // and both operands share the in-plane offsets, so one 32-bit offset per row is live while
    // the 16 loads are in flight: no spills at three blocks per SM.
    const int2 lr = trange[blockIdx.x];               // the tile's list [l0, l1), in block order
    const int l0 = lr.x, l1 = lr.y;
    for (int c0 = l0; c0 < l1; c0 += kListChunk) {
        const int cn = min(kListChunk, l1 - c0);
        __syncthreads();                              // the previous chunk is consumed
        for (int i = threadIdx.x; i < cn; i += kThreads) {
            const int4 v = tlist[c0 + i];
            s_list[i] = make_int3(v.x, v.y, v.z);     // (j, y, x)
        }
        __syncthreads();
        for (int i = warp; i < cn; i += kThreads / 32) {  // warp w: every 8th entry, ascending
            const int j = s_list[i].x, py = s_list[i].y, px = s_list[i].z;
            const int lx = tx0 + lane - px;
            const int lxc = min(max(lx, 0), N - 1);
            const int ly0 = ty0 - py;
            for (int m = 0; m < nq; ++m) {
                const float2 *psi_j = psi + ((size_t)j * nq + m) * NN;
                const float2 *probe_m = probe + (size_t)m * NN;
                // all loads first, from clamped (always valid) offsets, so they are in flight
                // together; pixels outside the patch are masked out afterwards
                float2 pv[kTR], vv[kTR];
#pragma unroll
                for (int r = 0; r < kTR; ++r) {
                    const int off = min(max(ly0 + r, 0), N - 1) * N + lxc;
                    pv[r] = __ldg(probe_m + off);
                    vv[r] = __ldg(psi_j + off);
                }
                if (lx >= 0 && lx < N) {
#pragma unroll
                    for (int r = 0; r < kTR; ++r) {
                        if ((unsigned)(ly0 + r) < (unsigned)N) {
                            acc[r] = cadd(acc[r], cmulc(pv[r], vv[r]));
                            dn[r] += cabs2(pv[r]);
                            hit |= 1u << r;
                        }
                    }
                }
            }
        }
    }
    float2 tnum;
    float tden;
    bool covered;
    combine_warps(acc, dn, hit, wt, tnum, tden, covered);
    float mx = 0.f;
    if (threadIdx.x < kTR * kTW) {
        const int r = threadIdx.x / kTW, c = threadIdx.x % kTW;
        const int py = ty0 + r, px = tx0 + c;
        if (py < M && px < M) {
            num[(size_t)py * M + px] = tnum;
            den[(size_t)py * M + px] = covered ? tden : -1.0f;       // -1: outside every patch
            mx = tden;
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if (lane == 0) s_max[warp] = mx;
    __syncthreads();
    if (threadIdx.x == 0) {
        float m = 0.f;
        for (int w = 0; w < kThreads / 32; ++w) m = fmaxf(m, s_max[w]);
        tile_max[tile] = m;
    }
}

// ePIE by colour, object step for the positions list[0 .. n) of one colour (disjoint patches,
// so the scatter needs no atomics): one block per position j, from psi_j' (exit-wave kernel):
//   Delta = psi_j' - P O_j;  O_j += alpha conj(P) Delta / max |P|^2
//   part[u] = conj(O_j) Delta / max |O_j|^2   (O_j before the step; the probe step's summand)
__global__ void __launch_bounds__(kThreads) k_epie_object(float2 *__restrict__ obj, const float2 *__restrict__ probe,
                                                          const float2 *__restrict__ psi, const int2 *__restrict__ pos,
                                                          const int *__restrict__ list, float2 *__restrict__ part,
                                                          int M, int N, float alpha) {
    __shared__ float s_mp[kThreads / 32], s_mo[kThreads / 32];
    const int u = blockIdx.x, j = list[u];
    const int2 pj = pos[j];
    const int NN = N * N, lgN = __ffs(N) - 1;          // N is a power of two (16, 64, 128, 256)
    float mp = 0.f, mo = 0.f;
    for (int q = threadIdx.x; q < NN; q += blockDim.x) {
        mp = fmaxf(mp, cabs2(probe[q]));
        mo = fmaxf(mo, cabs2(obj[(size_t)(pj.x + (q >> lgN)) * M + pj.y + (q & (N - 1))]));
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        mp = fmaxf(mp, __shfl_xor_sync(0xffffffffu, mp, o));
        mo = fmaxf(mo, __shfl_xor_sync(0xffffffffu, mo, o));
    }
    if ((threadIdx.x & 31) == 0) { s_mp[threadIdx.x >> 5] = mp; s_mo[threadIdx.x >> 5] = mo; }
    __syncthreads();
    mp = 0.f;
    mo = 0.f;
    for (int w = 0; w < kThreads / 32; ++w) { mp = fmaxf(mp, s_mp[w]); mo = fmaxf(mo, s_mo[w]); }
    const float so = mp > 0.f ? alpha / mp : 0.f;
    const float sp = mo > 0.f ? 1.0f / mo : 0.f;
    const float2 *psi_j = psi + (size_t)j * NN;
    for (int q = threadIdx.x; q < NN; q += blockDim.x) {
        float2 *op = obj + (size_t)(pj.x + (q >> lgN)) * M + pj.y + (q & (N - 1));
        const float2 p = probe[q];
        const float2 o = *op;
        const float2 d = csub(psi_j[q], cmul(p, o));
        *op = cadd(o, cscale(cmulc(p, d), so));
        part[(size_t)u * NN + q] = cscale(cmulc(o, d), sp);
    }
}

// ePIE by colour, probe step: P += (beta / n) sum_{u < n} part[u] (fixed order).
__global__ void __launch_bounds__(kThreads) k_epie_probe(float2 *__restrict__ probe, const float2 *__restrict__ part,
                                                         int n, size_t NN, float scale) {
    for (size_t q = blockIdx.x * (size_t)blockDim.x + threadIdx.x; q < NN; q += (size_t)gridDim.x * blockDim.x) {
        float2 acc = make_float2(0.f, 0.f);
        for (int u = 0; u < n; ++u) acc = cadd(acc, part[(size_t)u * NN + q]);
        probe[q] = cadd(probe[q], cscale(acc, scale));
    }
}

__device__ float block_max(const float *v, int n) {
    __shared__ float s[kThreads / 32];
    float m = 0.f;
    for (int i = threadIdx.x; i < n; i += blockDim.x) m = fmaxf(m, v[i]);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) s[threadIdx.x >> 5] = m;
    __syncthreads();
    float r = 0.f;
    for (int w = 0; w < (int)(blockDim.x / 32); ++w) r = fmaxf(r, s[w]);
    return r;
}

// Fourier error of an iteration: sum_j err[j] * inv_norm, by one block of kThreads threads
// (thread t sums err[t], err[t + kThreads], ...; then a fixed tree over the threads).
__device__ void error_sum_block(const double *__restrict__ err, int J, const double *__restrict__ inv_norm,
                                double *__restrict__ out) {
    __shared__ double s[kThreads];
    double a = 0.0;
    for (int i = threadIdx.x; i < J; i += kThreads) a += err[i];
    s[threadIdx.x] = a;
    __syncthreads();
    for (int w = kThreads / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) s[threadIdx.x] += s[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) *out = s[0] * inv_norm[0];
}

// x = num / (den + alpha max den) where den >= 0 (the pixel lies in some patch; -1 marks
// pixels outside every patch) and den + alpha max den > 0; elsewhere x keeps its value.
// With err_out, block 0 also forms the iteration's Fourier error from the per-position errors
// of the exit waves (which precede this kernel on the stream), saving a launch of its own.
__global__ void __launch_bounds__(kThreads) k_apply(float2 *__restrict__ x, const float2 *__restrict__ num,
                                                    const float *__restrict__ den, const float *__restrict__ partial_max,
                                                    int nmax, size_t n, float alpha, const double *__restrict__ err,
                                                    int J, const double *__restrict__ inv_norm,
                                                    double *__restrict__ err_out) {
    pdl_allow_dependents();
    pdl_wait();                                       // the numerators and denominators are complete
    const float reg = alpha * block_max(partial_max, nmax);
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const float d = den[i];
        if (d >= 0.f && d + reg > 0.f) {
            const float s = 1.0f / (d + reg);
            x[i] = cscale(num[i], s);
        }
    }
    if (err_out && blockIdx.x == 0) error_sum_block(err, J, inv_norm, err_out);
}

// Probe partial sums: block (kTR x 32 probe tile, chunk of positions) -> partial[chunk][q].
// Warp w takes every 8th position of the chunk; lane = tile column, kTR rows in registers.
template <int QC>   // QC = 1: one probe mode (compile-time); 0: Q modes at run time
__global__ void __launch_bounds__(kThreads, QC == 1 ? 3 : 2) k_probe_partial(
    const float2 *__restrict__ psi, const float2 *__restrict__ obj, const int2 *__restrict__ pos,
    float2 *__restrict__ pnum, float *__restrict__ pden, int M, int N, int J, int per_chunk, int Q) {
    __shared__ WarpTiles wt;
    pdl_allow_dependents();
    pdl_wait();                                       // the new object is complete
    const int nqx = (N + kTW - 1) / kTW;
    const int qt = blockIdx.x, chunk = blockIdx.y;
    const int qy0 = (qt / nqx) * kTR, qx0 = (qt % nqx) * kTW;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int qx = qx0 + lane;
    float2 acc[kTR];
    float dn[kTR];
#pragma unroll
    for (int r = 0; r < kTR; ++r) { acc[r] = make_float2(0.f, 0.f); dn[r] = 0.f; }
    const int j0 = chunk * per_chunk, j1 = min(J, j0 + per_chunk);
    const size_t NN = (size_t)N * N;
    int2 pn = (j0 + warp < j1) ? pos[j0 + warp] : make_int2(0, 0);
    for (int j = j0 + warp; j < j1; j += kThreads / 32) {
        const int2 pj = pn;
        if (j + kThreads / 32 < j1) pn = pos[j + kThreads / 32];
        const float2 *psi_j = psi + (QC ? (size_t)j * NN : ((size_t)j * Q + blockIdx.z) * NN);
        const int qxc = min(qx, N - 1);
        float2 ov[kTR], vv[kTR];
#pragma unroll
        for (int r = 0; r < kTR; ++r) {                  // loads first (clamped, always valid)
            const int qyc = min(qy0 + r, N - 1);
            ov[r] = __ldg(obj + (size_t)(pj.x + qyc) * M + pj.y + qxc);
            vv[r] = __ldg(psi_j + (size_t)qyc * N + qxc);
        }
        if (qx < N) {
#pragma unroll
            for (int r = 0; r < kTR; ++r) {
                if (qy0 + r < N) {
                    acc[r] = cadd(acc[r], cmulc(ov[r], vv[r]));
                    dn[r] += cabs2(ov[r]);
                }
            }
        }
    }
    float2 tnum;
    float tden;
    bool covered;
    combine_warps(acc, dn, 0u, wt, tnum, tden, covered);
    if (threadIdx.x < kTR * kTW) {
        const int r = threadIdx.x / kTW, c = threadIdx.x % kTW;
        const int y = qy0 + r, x = qx0 + c;
        if (y < N && x < N) {
            const size_t o = (QC ? (size_t)chunk * NN : ((size_t)chunk * Q + blockIdx.z) * NN) + (size_t)y * N + x;
            pnum[o] = tnum;
            pden[o] = tden;
        }
    }
}

// Fixed-order sum of the chunk partials; per-block max of the denominator.
__global__ void __launch_bounds__(kThreads) k_probe_reduce(const float2 *__restrict__ pnum,
                                                           const float *__restrict__ pden, float2 *__restrict__ num,
                                                           float *__restrict__ den, float *__restrict__ bmax, int NN,
                                                           int nchunk) {
    __shared__ float s[kThreads / 32];
    pdl_allow_dependents();
    pdl_wait();                                       // the partial sums are complete
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    float d = 0.f;
    if (i < NN) {
        float2 a = make_float2(0.f, 0.f);
        for (int c = 0; c < nchunk; ++c) {
            a = cadd(a, pnum[(size_t)c * NN + i]);
            d += pden[(size_t)c * NN + i];
        }
        num[i] = a;
        den[i] = d;
    }
    float m = d;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) s[threadIdx.x >> 5] = m;
    __syncthreads();
    if (threadIdx.x == 0) {
        float r = 0.f;
        for (int w = 0; w < kThreads / 32; ++w) r = fmaxf(r, s[w]);
        bmax[blockIdx.x] = r;
    }
}

// Per-iteration error: sum_j err[j] (fixed order) * inv_norm.
__global__ void __launch_bounds__(kThreads) k_error_reduce(const double *__restrict__ err, int J,
                                                           const double *__restrict__ inv_norm,
                                                           double *__restrict__ out) {
    error_sum_block(err, J, inv_norm, out);
}

// A = sqrt(max(I, 0)) with DC moved from the centre to index 0, stored per position column by
// column (amp[j][kx][...]) and, for the mixed-state path, also row-major (amp_nat[j][ky][kx]).  Within a column the order is ky (R = 0) or, for the N = 256
// kernel (R = 16), the order its FFT groups consume: thread t's targets ky = t + 16 k2 are
// contiguous (index t * 16 + k2).  Also the sum of A^2 per position.
__global__ void __launch_bounds__(kThreads) k_amplitudes(const float *__restrict__ fused, float *__restrict__ amp,
                                                         float *__restrict__ amp_nat, double *__restrict__ a2, int N,
                                                         int R) {
    __shared__ double s[kThreads / 32];
    const int j = blockIdx.x;
    const size_t NN = (size_t)N * N;
    const int h = N / 2, lgN = __ffs(N) - 1;          // N is a power of two; R is 0 or 16
    double acc = 0.0;
    for (int i = threadIdx.x; i < N * N; i += blockDim.x) {
        const int kx = i >> lgN, w = i & (N - 1);    // destination column kx, slot w
        const int ky = R ? (w >> 4) + 16 * (w & 15) : w;
        const int sy = (ky + h) & (N - 1), sx = (kx + h) & (N - 1);
        const float v = sqrtf(fmaxf(fused[(size_t)j * NN + (size_t)sy * N + sx], 0.f));
        amp[(size_t)j * NN + i] = v;
        if (amp_nat) amp_nat[(size_t)j * NN + (size_t)ky * N + kx] = v;   // row-major [ky][kx]
        acc += (double)v * (double)v;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) s[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double r = 0.0;
        for (int w = 0; w < kThreads / 32; ++w) r += s[w];
        a2[j] = r;
    }
}

__global__ void k_inv_norm(const double *__restrict__ a2, int J, double *__restrict__ inv_norm) {
    __shared__ double s[kThreads];
    double a = 0.0;
    for (int i = threadIdx.x; i < J; i += blockDim.x) a += a2[i];
    s[threadIdx.x] = a;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) s[threadIdx.x] += s[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) inv_norm[0] = s[0] > 0.0 ? 1.0 / s[0] : 0.0;
}

}  // namespace

struct ptycho_ctx {
    int M = 0, N = 0, J = 0, R = 0, Q = 1;
    int algorithm = PTYCHO_ALG_AP;
    float epie_alpha = 1.f, epie_beta = 1.f;
    std::vector<int> colour_start, colour_of;             // ePIE: colour c = list[start[c] .. start[c+1])
    int *d_colour_list = nullptr;
    float2 *d_epie_part = nullptr;
    const int *cur_list = nullptr;                        // exit-wave launches: unit list or NULL
    int cur_count = 0;
    float alpha_O = 0.f, alpha_P = 0.f;
    int probe_update_start = 0;
    long long iter = 0;
    cudaStream_t st = nullptr;
    int2 *d_pos = nullptr;
    float2 *d_obj = nullptr, *d_probe = nullptr, *d_psi = nullptr, *d_slot = nullptr;
    float2 *d_num_o = nullptr, *d_num_p = nullptr, *d_pnum = nullptr;
    float *d_amp_nat = nullptr;                           // row-major amplitudes (Q > 1)
    float *d_fscale = nullptr;     // mode-summed modulus scales (Q > 1, N = 256), amplitude order
    int n_err = 0;                 // per-position error slots summed into the Fourier error
    float *d_amp = nullptr, *d_den_o = nullptr, *d_den_p = nullptr, *d_pden = nullptr;
    float *d_tile_max = nullptr, *d_pmax = nullptr;
    double *d_err_pos = nullptr, *d_a2 = nullptr, *d_inv_norm = nullptr, *d_err = nullptr;
    int err_cap = 0;
    // Error slot of batch iterations: allocated once at init and never replaced, so a captured
    // batch graph may keep its address while ptycho_iterate grows d_err.
    double *d_err_batch = nullptr;
    int *d_tstart = nullptr;
    int *d_torder = nullptr;                              // per gather block: its tile (longest lists first)
    int2 *d_trange = nullptr;                             // per gather block: its tile's list range
    int4 *d_tlist = nullptr;                              // tile lists: (j, y, x, 0)
    int ntx = 0, ntiles = 0;
    int *d_status = nullptr;
    int *d_tail_sync = nullptr;                           // N = 256 tail split: hand-off counters
    double *d_tail_err = nullptr;                         // ... and per-batch error sums [grid / 2][16]
    int inject_wait = 0;                                  // test hook, see ptycho_debug_wait_timeout (0, 1, 2)
    int exit_kernels = 1;                                 // kernels of the last full-batch exit pass
    TmaMaps tm;
    bool exit_tma = false;
    bool fft_gemm = false;                                // split-BF16 tensor-core DFTs (N = 64, 128, 256)
    const uint4 *gmat = nullptr;                          // N = 256 tensor-core form: the split DFT matrix
    int gemm_sms = 0;
    int tma_batch = 32;
    int grid_exit = 0, nchunk = 0, per_chunk = 0, nqt = 0, nred = 0;
    size_t exit_smem = 0;
    // timing
    bool timing = false;
    double stage_ms[ST_COUNT] = {};
    long long stage_launches[ST_COUNT] = {};
    std::vector<cudaEvent_t> ev;
    // stage events of the current ptycho_iterate call: stage s of iteration i ran between events
    // mark[2 (i ST_COUNT + s)] and mark[... + 1] (-1: not run); ev_used events are recorded,
    // the last of them with no launch after it while ev_fresh (the next stage starts there)
    std::vector<int> mark;
    size_t ev_used = 0;
    bool ev_fresh = false;
    // the object and probe update kernels of ptycho_iterate are launched with programmatic
    // stream serialization (not while the stream is being captured, nor from a batch)
    bool pdl = false;
};

namespace {

template <typename T>
int dalloc(T **p, size_t count) {
    *p = nullptr;
    if (count == 0) count = 1;
    cudaError_t e = pm::dev_malloc((void **)p, count * sizeof(T));
    if (e != cudaSuccess) return pm::cuda_fail(e, "cudaMalloc");
    return PTYCHO_OK;
}

// Buffers of a handle: stream-ordered on the handle's stream, from the library's pool (freed
// memory is kept there for the next handle).  Another stream may use them once the handle's
// stream has passed the allocation (ptycho_init and the re-allocations below synchronise it).
template <typename T>
int halloc(ptycho_ctx *h, T **p, size_t count) {
    *p = nullptr;
    if (count == 0) count = 1;
    cudaError_t e = pm::dev_malloc_async((void **)p, count * sizeof(T), h->st);
    if (e != cudaSuccess) return pm::cuda_fail(e, "device allocation");
    return PTYCHO_OK;
}

template <typename T>
int hfree(ptycho_ctx *h, T **p) {
    cudaError_t e = *p ? cudaFreeAsync(*p, h->st) : cudaSuccess;
    *p = nullptr;
    return e == cudaSuccess ? PTYCHO_OK : pm::cuda_fail(e, "cudaFreeAsync");
}

void free_ctx(ptycho_ctx *h) {
    if (!h) return;
    cudaStreamSynchronize(h->st);                       // the default stream too (documented wait)
    void *ptrs[] = {h->d_pos, h->d_obj, h->d_probe, h->d_psi, h->d_slot, h->d_num_o, h->d_num_p, h->d_pnum,
                    h->d_amp, h->d_amp_nat, h->d_fscale, h->d_den_o, h->d_den_p, h->d_pden, h->d_tile_max, h->d_pmax, h->d_err_pos,
                    h->d_a2, h->d_inv_norm, h->d_err, h->d_err_batch, h->d_tstart, h->d_tlist, h->d_status, h->d_torder, h->d_trange,
                    h->d_tail_sync, h->d_tail_err,
                    h->d_colour_list, h->d_epie_part};
    for (void *p : ptrs)
        if (p && cudaFreeAsync(p, h->st) != cudaSuccess) {
            (void)cudaGetLastError();                    // e.g. the stream was destroyed first:
            cudaFree(p);                                 // free after a device synchronisation
        }
    for (cudaEvent_t e : h->ev) cudaEventDestroy(e);
    delete h;
}

using pm::encode_2d;

template <int B, int XM, bool TC = false>
int setup_tma_kernel(ptycho_ctx *h, int *per_sm) {
    const size_t smem = tma_kernel_smem<B, TC>();
    PM_CUDA(cudaFuncSetAttribute(k_exit_wave_tma<B, XM, TC>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    if constexpr (XM == XM_FULL)
        PM_CUDA(cudaFuncSetAttribute(k_exit_wave_tma<B, XM, TC, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)smem));
    PM_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(per_sm, k_exit_wave_tma<B, XM, TC>, B * 16, smem));
    if (*per_sm < 1) return pm::fail(PTYCHO_ECUDA, "TMA exit-wave kernel cannot be resident");
    h->exit_smem = smem;
    return PTYCHO_OK;
}

// Batch size of the N = 256 kernel (rows per stage): 16, two 256-thread CTAs per SM (measured
// at lab scale: 1.083 ms per launch; 32, one 512-thread CTA per SM whose 148 live slots the L2
// keeps, moves 1.23 instead of 1.84 MB of DRAM traffic per position but takes 1.106 ms), unless
// PTYCHO_TMA_BATCH = 32.  The mixed-state forward/inverse kernels use 16.
int tma_batch_choice(int Q) {
    const char *env = std::getenv("PTYCHO_TMA_BATCH");
    if (Q == 1 && env && std::atoi(env) == 32) return 32;
    return 16;
}

int setup_exit_tma(ptycho_ctx *h) {
    int dev = 0, sms = 0, per_sm = 0, rc;
    PM_CUDA(cudaGetDevice(&dev));
    PM_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    h->tma_batch = tma_batch_choice(h->Q);
    if (h->Q > 1) {
        int p2 = 0;
        if ((rc = setup_tma_kernel<16, XM_FWD>(h, &per_sm))) return rc;
        if ((rc = setup_tma_kernel<16, XM_INV>(h, &p2))) return rc;
        per_sm = std::min(per_sm, p2);
    } else if (h->algorithm == PTYCHO_ALG_EPIE_COLOUR) {
        h->tma_batch = 32;
        if ((rc = setup_tma_kernel<32, XM_LIST>(h, &per_sm))) return rc;
    } else if (h->fft_gemm) {
        // tensor-core form: 16-row stages, one CTA per SM (the DFT matrix and operand need room)
        h->tma_batch = 16;
        const void *gm = nullptr;
        if ((rc = pm::dft64_matrix(&gm))) return rc;
        h->gmat = static_cast<const uint4 *>(gm);
        if ((rc = setup_tma_kernel<16, XM_FULL, true>(h, &per_sm))) return rc;
    } else if (h->tma_batch == 32) {
        if ((rc = setup_tma_kernel<32, XM_FULL>(h, &per_sm))) return rc;
    } else {
        if ((rc = setup_tma_kernel<16, XM_FULL>(h, &per_sm))) return rc;
    }
    h->exit_tma = true;
    h->grid_exit = std::max(1, std::min(h->J * h->Q, sms * per_sm));
    return PTYCHO_OK;
}

// Tensor maps of the TMA kernel; called once the buffers exist.
// Tensor maps of the N = 256 kernel with B rows per stage over the given probe, psi and slot
// buffers (slots: `slots` column-major 256 x 256 tiles).
int encode_tma_maps(TmaMaps *tm, float2 *probe, float2 *psi, float2 *slot, int Q, int J, int slots, int B) {
    const uint64_t N = 256;
    const CUtensorMapDataType c64 = CU_TENSOR_MAP_DATA_TYPE_FLOAT64;    // one complex64 = 8 bytes
    const uint64_t psi_rows = N * (uint64_t)Q * (uint64_t)J;
    const uint32_t b = (uint32_t)B;
    int rc;
    if ((rc = encode_2d(&tm->prow, probe, c64, 8, N, N * Q, 256, b, CU_TENSOR_MAP_SWIZZLE_NONE))) return rc;
    if ((rc = encode_2d(&tm->slot_r, slot, c64, 8, N, N * slots, 16, 256, CU_TENSOR_MAP_SWIZZLE_128B))) return rc;
    if ((rc = encode_2d(&tm->slot_c, slot, c64, 8, N, N * slots, 256, b, CU_TENSOR_MAP_SWIZZLE_NONE))) return rc;
    if ((rc = encode_2d(&tm->psi_c, psi, c64, 8, N, psi_rows, 16, 256, CU_TENSOR_MAP_SWIZZLE_128B))) return rc;
    if ((rc = encode_2d(&tm->psi_r, psi, c64, 8, N, psi_rows, 256, b, CU_TENSOR_MAP_SWIZZLE_NONE))) return rc;
    return encode_2d(&tm->psi_w, psi, c64, 8, N, psi_rows, 256, 16, CU_TENSOR_MAP_SWIZZLE_NONE);
}

// Slots of the N = 256 kernel: one per CTA (a split tail reuses the slots of the first launch).
int exit_slots(int grid) { return grid; }

int encode_exit_tma(ptycho_ctx *h) {
    return encode_tma_maps(&h->tm, h->d_probe, h->d_psi, h->d_slot, h->Q, h->J, exit_slots(h->grid_exit),
                           h->tma_batch);
}

int alloc_tail(ptycho_ctx *h) {
    int rc = hfree(h, &h->d_tail_sync);
    if (!rc) rc = hfree(h, &h->d_tail_err);
    const int cap = std::max(1, h->grid_exit / 2);
    if (!rc) rc = halloc(h, &h->d_tail_sync, (size_t)cap);
    if (!rc) rc = halloc(h, &h->d_tail_err, (size_t)cap * 16);
    return rc;
}

TmaArgs tma_args(ptycho_ctx *h) {
    TmaArgs a;
    a.obj = h->d_obj;
    a.amp = h->d_amp;
    a.pos = h->d_pos;
    a.err = h->d_err_pos;
    a.status = h->d_status;
    a.list = h->cur_list;
    a.count = h->cur_count;
    a.M = h->M;
    a.J = h->J;
    a.Q = h->Q;
    a.inject_wait = h->inject_wait;
    a.gmat = h->gmat;
    a.split = 1;
    a.tail_base = h->J;
    a.tail_sync = h->d_tail_sync;
    a.tail_err = h->d_tail_err;
    a.fscale = h->d_fscale;
    return a;
}

// Split factor of the last, partial round of a full-batch launch over J positions on `grid`
// persistent CTAs: the T = J mod grid leftover positions are each shared by S CTAs (a power of
// two with S T <= grid and at least two batches per part), so the round takes ~1/S of a
// position's time instead of one.  1 = no split (no leftover, fewer positions than CTAs, a
// stream being captured, or the test hook).
int tail_split(const ptycho_ctx *h, int nb) {
    const int G = h->grid_exit, J = h->J;
    if (h->inject_wait == 1 || J <= G || J % G == 0 || !h->d_tail_sync) return 1;
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(h->st, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone) return 1;
    const int T = J % G;
    int S = 1;
    while (2 * S * T <= G && 2 * S <= nb / 2) S *= 2;
    return S;
}

// Full-batch launch: the whole rounds, then (split tail) the leftover units over S CTAs each in
// a second, cooperative launch, so that every part of a tail unit is resident; if the driver
// refuses the cooperative launch, one unsplit launch takes the tail instead.
template <int B, bool TC>
int launch_full_split(ptycho_ctx *h, TmaArgs a) {
    const int S = tail_split(h, 256 / B);
    h->exit_kernels = S > 1 ? 2 : 1;
    if (S > 1) {
        const int G = h->grid_exit, T = h->J % G;
        a.split = S;
        a.tail_base = h->J - T;
        k_exit_wave_tma<B, XM_FULL, TC><<<G, B * 16, h->exit_smem, h->st>>>(a, h->tm);
        PM_LAUNCHED("k_exit_wave_tma");
        PM_CUDA(cudaMemsetAsync(h->d_tail_sync, 0, (size_t)T * sizeof(int), h->st));
        void *args[] = {(void *)&a, (void *)&h->tm};
        const cudaError_t e = cudaLaunchCooperativeKernel((const void *)k_exit_wave_tma<B, XM_FULL, TC, true>,
                                                          dim3(S * T), dim3(B * 16), args, h->exit_smem, h->st);
        if (e == cudaSuccess) return PTYCHO_OK;
        (void)cudaGetLastError();                          // not launched: the tail unsplit,
        a.split = 1;                                       // one CTA per leftover unit
        k_exit_wave_tma<B, XM_FULL, TC, true><<<T, B * 16, h->exit_smem, h->st>>>(a, h->tm);
        return PTYCHO_OK;
    }
    k_exit_wave_tma<B, XM_FULL, TC><<<h->grid_exit, B * 16, h->exit_smem, h->st>>>(a, h->tm);
    return PTYCHO_OK;
}

int launch_exit_tma(ptycho_ctx *h, int xm) {
    const TmaArgs a = tma_args(h);
    if (xm == XM_FWD) k_exit_wave_tma<16, XM_FWD><<<h->grid_exit, 16 * 16, h->exit_smem, h->st>>>(a, h->tm);
    else if (xm == XM_INV) k_exit_wave_tma<16, XM_INV><<<h->grid_exit, 16 * 16, h->exit_smem, h->st>>>(a, h->tm);
    else if (xm == XM_LIST) k_exit_wave_tma<32, XM_LIST><<<h->grid_exit, 32 * 16, h->exit_smem, h->st>>>(a, h->tm);
    else {
        int rc;
        if (h->fft_gemm) rc = launch_full_split<16, true>(h, a);
        else if (h->tma_batch == 32) rc = launch_full_split<32, false>(h, a);
        else rc = launch_full_split<16, false>(h, a);
        if (rc) return rc;
    }
    PM_LAUNCHED("k_exit_wave_tma");
    return PTYCHO_OK;
}

template <int R, int XM>
int setup_small_kernel(ptycho_ctx *h, int *per_sm) {
    const size_t smem = exit_smem_bytes<R>();
    PM_CUDA(cudaFuncSetAttribute(k_exit_wave<R, XM>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    PM_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(per_sm, k_exit_wave<R, XM>, kThreads, smem));
    if (*per_sm < 1) return pm::fail(PTYCHO_ECUDA, "exit-wave kernel cannot be resident (smem %zu)", smem);
    h->exit_smem = smem;
    return PTYCHO_OK;
}

template <int R>
int setup_exit_kernel(ptycho_ctx *h) {
    int dev = 0, sms = 0, per_sm = 0, p2 = 0, rc;
    PM_CUDA(cudaGetDevice(&dev));
    PM_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    if (h->Q > 1) {
        if ((rc = setup_small_kernel<R, XM_FWD>(h, &per_sm))) return rc;
        if ((rc = setup_small_kernel<R, XM_INV>(h, &p2))) return rc;
        per_sm = std::min(per_sm, p2);
    } else if (h->algorithm == PTYCHO_ALG_EPIE_COLOUR) {
        if ((rc = setup_small_kernel<R, XM_LIST>(h, &per_sm))) return rc;
    } else if ((rc = setup_small_kernel<R, XM_FULL>(h, &per_sm))) {
        return rc;
    }
    h->exit_tma = false;
    h->grid_exit = std::max(1, std::min(h->J * h->Q, sms * per_sm));
    return PTYCHO_OK;
}

template <int R>
int launch_exit(ptycho_ctx *h, int xm) {
    ExitArgs a{};
    a.obj = h->d_obj;
    a.probe = h->d_probe;
    a.amp = h->d_amp;
    a.pos = h->d_pos;
    a.psi = h->d_psi;
    a.err = h->d_err_pos;
    a.list = h->cur_list;
    a.count = h->cur_count;
    a.M = h->M;
    a.J = h->J;
    a.Q = h->Q;
    if (xm == XM_FWD) k_exit_wave<R, XM_FWD><<<h->grid_exit, kThreads, h->exit_smem, h->st>>>(a);
    else if (xm == XM_INV) k_exit_wave<R, XM_INV><<<h->grid_exit, kThreads, h->exit_smem, h->st>>>(a);
    else if (xm == XM_LIST) k_exit_wave<R, XM_LIST><<<h->grid_exit, kThreads, h->exit_smem, h->st>>>(a);
    else k_exit_wave<R, XM_FULL><<<h->grid_exit, kThreads, h->exit_smem, h->st>>>(a);
    PM_LAUNCHED("k_exit_wave");
    return PTYCHO_OK;
}

int setup_exit128(ptycho_ctx *h) {
    int dev = 0, sms = 0, per_sm = 0;
    PM_CUDA(cudaGetDevice(&dev));
    PM_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const size_t smem = exit128_smem_bytes();
    if (h->algorithm == PTYCHO_ALG_EPIE_COLOUR) {
        PM_CUDA(cudaFuncSetAttribute(k_exit_wave128<XM_LIST>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        PM_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_exit_wave128<XM_LIST>, kThreads128, smem));
    } else {
        PM_CUDA(cudaFuncSetAttribute(k_exit_wave128<XM_FULL>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        PM_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_exit_wave128<XM_FULL>, kThreads128, smem));
    }
    if (per_sm < 1) return pm::fail(PTYCHO_ECUDA, "N = 128 exit-wave kernel cannot be resident (smem %zu)", smem);
    h->exit_smem = smem;
    h->exit_tma = false;
    h->grid_exit = std::max(1, std::min(h->J, sms * per_sm));
    return PTYCHO_OK;
}

int launch_exit128(ptycho_ctx *h, int xm) {
    ExitArgs a{};
    a.obj = h->d_obj;
    a.probe = h->d_probe;
    a.amp = h->d_amp;
    a.pos = h->d_pos;
    a.psi = h->d_psi;
    a.err = h->d_err_pos;
    a.list = h->cur_list;
    a.count = h->cur_count;
    a.M = h->M;
    a.J = h->J;
    a.Q = 1;
    if (xm == XM_LIST) k_exit_wave128<XM_LIST><<<h->grid_exit, kThreads128, h->exit_smem, h->st>>>(a);
    else k_exit_wave128<XM_FULL><<<h->grid_exit, kThreads128, h->exit_smem, h->st>>>(a);
    PM_LAUNCHED("k_exit_wave128");
    return PTYCHO_OK;
}

int setup_exit(ptycho_ctx *h) {
    switch (h->R) {
        case 128: return setup_exit128(h);
        case 4: return setup_exit_kernel<4>(h);
        case 8: return setup_exit_kernel<8>(h);
        default: return setup_exit_tma(h);
    }
}

int launch_exit_pass(ptycho_ctx *h, int xm) {
    if (h->fft_gemm && h->N != 256) {
        pm::Dft64Exit e{h->d_obj, h->d_probe, h->d_amp, h->d_pos, h->d_psi, h->d_err_pos, h->d_status, h->M, h->J};
        if (h->N == 128) return pm::dft128_exit_launch(e, h->gemm_sms, h->st);
        return pm::dft64_exit_launch(e, h->gemm_sms, h->st);
    }
    switch (h->R) {
        case 128: return launch_exit128(h, xm);
        case 4: return launch_exit<4>(h, xm);
        case 8: return launch_exit<8>(h, xm);
        default: return launch_exit_tma(h, xm);
    }
}

// Exit waves of one iteration: the fused kernel (one mode), or forward FFTs of every
// (position, mode), the mode-summed modulus constraint, inverse FFTs (mixed state).
// Returns the number of kernel launches through *launches.
int launch_exit_any(ptycho_ctx *h, int *launches) {
    int rc;
    if (h->Q == 1) {
        h->exit_kernels = 1;
        rc = launch_exit_pass(h, XM_FULL);
        *launches = h->exit_kernels;                      // 2 when the last round was split
        return rc;
    }
    *launches = 3;
    if ((rc = launch_exit_pass(h, XM_FWD))) return rc;
    if (h->d_fscale) rc = launch_mode_scale(h->d_psi, h->d_amp_nat, h->d_fscale, h->d_err_pos, h->J, h->Q, h->st);
    else rc = launch_modulus_modes(h->d_psi, h->d_amp_nat, h->d_err_pos, h->J, h->N, h->Q, h->st);
    if (rc) return rc;
    return launch_exit_pass(h, XM_INV);
}

// Stage s of an iteration: an NVTX range around its launches, and CUDA events when timing.
const char *const kStageNames[ST_COUNT] = {"ptycho: exit waves", "ptycho: object update", "ptycho: probe update",
                                           "ptycho: error"};

// Stage s of the iteration whose marks start at `base` (= i ST_COUNT): a stage that follows
// another with no launch in between starts at that stage's end event, so the timed stages of a
// call cost one recorded event each plus one (each recorded event costs the stream a short
// serialisation).
int stage_begin(ptycho_ctx *h, int s, size_t base) {
    nvtxRangePushA(kStageNames[s]);
    if (!h->timing) return PTYCHO_OK;
    if (!h->ev_fresh) {
        if (h->ev_used >= h->ev.size()) return pm::fail(PTYCHO_ECUDA, "stage timing: out of events");
        PM_CUDA(cudaEventRecord(h->ev[h->ev_used++], h->st));
    }
    h->mark[2 * (base + s)] = (int)h->ev_used - 1;
    h->ev_fresh = false;
    return PTYCHO_OK;
}

int stage_end(ptycho_ctx *h, int s, size_t base, int launches) {
    nvtxRangePop();
    if (!h->timing) return PTYCHO_OK;
    if (h->ev_used >= h->ev.size()) return pm::fail(PTYCHO_ECUDA, "stage timing: out of events");
    PM_CUDA(cudaEventRecord(h->ev[h->ev_used], h->st));
    h->mark[2 * (base + s) + 1] = (int)h->ev_used++;
    h->ev_fresh = true;
    h->stage_launches[s] += launches;
    return PTYCHO_OK;
}

// Launch of an update kernel on the handle's stream; with h->pdl, as a programmatic dependent of
// the kernel before it (the kernel calls pdl_wait before it touches memory).
template <typename... KArgs, typename... Args>
int launch_update(ptycho_ctx *h, void (*kernel)(KArgs...), dim3 grid, const char *what, Args... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = dim3(kThreads);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = h->st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = h->pdl ? 1 : 0;
    const cudaError_t e = cudaLaunchKernelEx(&cfg, kernel, args...);
    if (e != cudaSuccess) return pm::cuda_fail(e, what);
    return PTYCHO_OK;
}

// ePIE by colour: colours in ascending order; per colour the fused exit-wave kernel on the
// colour's positions, the object step (disjoint patches, no atomics) and the averaged probe
// step.  The whole colour loop is timed as stage 0.
int iterate_one_epie(ptycho_ctx *h, double *err_dst, size_t ev_base, bool update_probe) {
    int rc;
    if ((rc = stage_begin(h, ST_EXIT, ev_base))) return rc;
    const size_t NN = (size_t)h->N * h->N;
    const int ncol = (int)h->colour_start.size() - 1;
    int launches = 0;
    for (int c = 0; c < ncol; ++c) {
        const int b = h->colour_start[c], n = h->colour_start[c + 1] - b;
        h->cur_list = h->d_colour_list + b;
        h->cur_count = n;
        rc = launch_exit_pass(h, XM_LIST);
        h->cur_list = nullptr;
        h->cur_count = 0;
        if (rc) return rc;
        k_epie_object<<<n, kThreads, 0, h->st>>>(h->d_obj, h->d_probe, h->d_psi, h->d_pos, h->d_colour_list + b,
                                                 h->d_epie_part, h->M, h->N, h->epie_alpha);
        PM_LAUNCHED("k_epie_object");
        launches += 2;
        if (update_probe) {
            const unsigned gp = (unsigned)std::min<size_t>((NN + kThreads - 1) / kThreads, 148 * 4);
            k_epie_probe<<<gp, kThreads, 0, h->st>>>(h->d_probe, h->d_epie_part, n, NN, h->epie_beta / n);
            PM_LAUNCHED("k_epie_probe");
            ++launches;
        }
    }
    if ((rc = stage_end(h, ST_EXIT, ev_base, launches))) return rc;
    for (int st = ST_OBJECT; st <= ST_PROBE; ++st) {
        if ((rc = stage_begin(h, st, ev_base))) return rc;
        if ((rc = stage_end(h, st, ev_base, 0))) return rc;
    }
    if ((rc = stage_begin(h, ST_ERROR, ev_base))) return rc;
    k_error_reduce<<<1, kThreads, 0, h->st>>>(h->d_err_pos, h->J, h->d_inv_norm, err_dst);
    PM_LAUNCHED("k_error_reduce");
    return stage_end(h, ST_ERROR, ev_base, 1);
}

// err_dst: device slot of this iteration's Fourier error.  exit_done: the exit waves of this
// iteration were already computed by a multi-dataset launch.
int iterate_one(ptycho_ctx *h, double *err_dst, size_t ev_base, bool update_probe, bool exit_done = false) {
    if (h->algorithm == PTYCHO_ALG_EPIE_COLOUR) return iterate_one_epie(h, err_dst, ev_base, update_probe);
    int rc;
    // exit waves
    if (!exit_done) {
        if ((rc = stage_begin(h, ST_EXIT, ev_base))) return rc;
        int exit_launches = 1;
        if ((rc = launch_exit_any(h, &exit_launches))) return rc;
        if ((rc = stage_end(h, ST_EXIT, ev_base, exit_launches))) return rc;
    }
    // object
    if ((rc = stage_begin(h, ST_OBJECT, ev_base))) return rc;
    if ((rc = launch_update(h, h->Q == 1 ? k_object_gather<1> : k_object_gather<0>, dim3(h->ntiles),
                            "k_object_gather", (const float2 *)h->d_psi, (const float2 *)h->d_probe,
                            (const int2 *)h->d_pos, (const int4 *)h->d_tlist, (const int *)h->d_torder,
                            (const int2 *)h->d_trange, h->d_num_o, h->d_den_o, h->d_tile_max, h->M, h->N, h->ntx,
                            h->Q)))
        return rc;
    const size_t MM = (size_t)h->M * h->M;
    const unsigned gapply = (unsigned)std::min<size_t>((MM + kThreads - 1) / kThreads, 148 * 8);
    if ((rc = launch_update(h, k_apply, dim3(gapply), "k_apply(object)", h->d_obj, (const float2 *)h->d_num_o,
                            (const float *)h->d_den_o, (const float *)h->d_tile_max, h->ntiles, MM, h->alpha_O,
                            (const double *)h->d_err_pos, h->n_err, (const double *)h->d_inv_norm, err_dst)))
        return rc;
    if ((rc = stage_end(h, ST_OBJECT, ev_base, 2))) return rc;
    // probe
    if ((rc = stage_begin(h, ST_PROBE, ev_base))) return rc;
    if (update_probe) {
        const int NN = h->N * h->N * h->Q;                // all probe modes
        if ((rc = launch_update(h, h->Q == 1 ? k_probe_partial<1> : k_probe_partial<0>,
                                dim3(h->nqt, h->nchunk, h->Q == 1 ? 1 : h->Q), "k_probe_partial",
                                (const float2 *)h->d_psi, (const float2 *)h->d_obj, (const int2 *)h->d_pos, h->d_pnum,
                                h->d_pden, h->M, h->N, h->J, h->per_chunk, h->Q)))
            return rc;
        if ((rc = launch_update(h, k_probe_reduce, dim3(h->nred), "k_probe_reduce", (const float2 *)h->d_pnum,
                                (const float *)h->d_pden, h->d_num_p, h->d_den_p, h->d_pmax, NN, h->nchunk)))
            return rc;
        const unsigned gp = (unsigned)std::min<int>((NN + kThreads - 1) / kThreads, 148 * 4);
        if ((rc = launch_update(h, k_apply, dim3(gp), "k_apply(probe)", h->d_probe, (const float2 *)h->d_num_p,
                                (const float *)h->d_den_p, (const float *)h->d_pmax, h->nred, (size_t)NN, h->alpha_P,
                                (const double *)nullptr, 0, (const double *)nullptr, (double *)nullptr)))
            return rc;
    }
    if ((rc = stage_end(h, ST_PROBE, ev_base, update_probe ? 3 : 0))) return rc;
    // the error is formed by block 0 of the object step's k_apply: no stage of its own
    return PTYCHO_OK;
}

int copy_in_complex(float2 *dst, const void *src, size_t count, bool on_device, cudaStream_t st) {
    PM_CUDA(cudaMemcpyAsync(dst, src, count * sizeof(float2),
                            on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, st));
    return PTYCHO_OK;
}

}  // namespace

extern "C" int ptycho_init(ptycho_handle *out, const ptycho_desc *d) {
    if (!out) return pm::fail(PTYCHO_EINVAL, "ptycho_init: out is NULL");
    *out = nullptr;
    pm::NvtxRange range("ptycho_init");
    if (!d) return pm::fail(PTYCHO_EINVAL, "ptycho_init: desc is NULL");
    int R = 0;
    if (d->N == 16) R = 4;
    else if (d->N == 64) R = 8;
    else if (d->N == 128) R = 128;                   // 8 x 16: k_exit_wave128
    else if (d->N == 256) R = 16;
    else return pm::fail(PTYCHO_EINVAL, "ptycho_init: N = %d unsupported (16, 64, 128 or 256)", d->N);
    if (d->J < 1) return pm::fail(PTYCHO_EINVAL, "ptycho_init: J = %d < 1", d->J);
    if (d->M < d->N || d->M > 32768) return pm::fail(PTYCHO_EINVAL, "ptycho_init: M = %d must be in [N, 32768]", d->M);
    if (!d->h_pos || !d->d_fused || !d->obj0 || !d->probe0)
        return pm::fail(PTYCHO_EINVAL, "ptycho_init: NULL position, fused, object or probe pointer");
    if (!(d->alpha_O >= 0.f) || !(d->alpha_P >= 0.f) || !std::isfinite(d->alpha_O) || !std::isfinite(d->alpha_P))
        return pm::fail(PTYCHO_EINVAL, "ptycho_init: regularisers must be finite and >= 0");
    if (d->probe_update_start < 0) return pm::fail(PTYCHO_EINVAL, "ptycho_init: probe_update_start < 0");
    if (d->modes < 1 || d->modes > 8) return pm::fail(PTYCHO_EINVAL, "ptycho_init: modes = %d not in [1, 8]", d->modes);
    if (d->algorithm != PTYCHO_ALG_AP && d->algorithm != PTYCHO_ALG_EPIE_COLOUR)
        return pm::fail(PTYCHO_EINVAL, "ptycho_init: unknown algorithm %d", d->algorithm);
    if (d->N == 128 && d->modes != 1)
        return pm::fail(PTYCHO_EINVAL, "ptycho_init: N = 128 supports one probe mode");
    if (d->algorithm == PTYCHO_ALG_EPIE_COLOUR && d->modes != 1)
        return pm::fail(PTYCHO_EINVAL, "ptycho_init: ePIE by colour supports one probe mode");
    if (d->algorithm == PTYCHO_ALG_EPIE_COLOUR &&
        (!std::isfinite(d->epie_alpha) || !std::isfinite(d->epie_beta) || !(d->epie_alpha > 0.f) || !(d->epie_beta >= 0.f)))
        return pm::fail(PTYCHO_EINVAL, "ptycho_init: ePIE step sizes must be finite, alpha > 0, beta >= 0");
    if (d->fft_path != PTYCHO_FFT_RADIX_FP32 && d->fft_path != PTYCHO_FFT_DFTGEMM_BF16X3)
        return pm::fail(PTYCHO_EINVAL, "ptycho_init: unknown fft_path %d", d->fft_path);
    if (d->fft_path == PTYCHO_FFT_DFTGEMM_BF16X3 &&
        ((d->N != 64 && d->N != 128 && d->N != 256) || d->modes != 1 || d->algorithm != PTYCHO_ALG_AP))
        return pm::fail(PTYCHO_EINVAL,
                        "ptycho_init: the DFT-GEMM path needs N = 64, 128 or 256, one mode and algorithm AP");
    const int M = d->M, N = d->N, J = d->J, Q = d->modes;
    for (int j = 0; j < J; ++j) {
        const int y = d->h_pos[2 * j], x = d->h_pos[2 * j + 1];
        if (y < 0 || x < 0 || y > M - N || x > M - N)
            return pm::fail(PTYCHO_EINVAL, "ptycho_init: position %d = (%d, %d) outside [0, %d]", j, y, x, M - N);
    }
    ptycho_ctx *h = new (std::nothrow) ptycho_ctx();
    if (!h) return pm::fail(PTYCHO_ENOMEM, "ptycho_init: host allocation failed");
    h->M = M; h->N = N; h->J = J; h->R = R; h->Q = Q;
    h->algorithm = d->algorithm;
    h->epie_alpha = d->epie_alpha;
    h->epie_beta = d->epie_beta;
    h->fft_gemm = d->fft_path == PTYCHO_FFT_DFTGEMM_BF16X3;
    std::vector<int> colour_list;
    int max_colour_size = 0;
    if (h->algorithm == PTYCHO_ALG_EPIE_COLOUR) {
        // greedy colouring in position order: smallest colour unused by an earlier overlapping position
        h->colour_of.assign(J, -1);
        int ncol = 0;
        std::vector<char> taken;
        for (int j = 0; j < J; ++j) {
            taken.assign(ncol + 1, 0);
            const int yj = d->h_pos[2 * j], xj = d->h_pos[2 * j + 1];
            for (int i = 0; i < j; ++i)
                if (std::abs(d->h_pos[2 * i] - yj) < N && std::abs(d->h_pos[2 * i + 1] - xj) < N)
                    taken[h->colour_of[i]] = 1;
            int c = 0;
            while (taken[c]) ++c;
            h->colour_of[j] = c;
            ncol = std::max(ncol, c + 1);
        }
        h->colour_start.assign(ncol + 1, 0);
        for (int j = 0; j < J; ++j) ++h->colour_start[h->colour_of[j] + 1];
        for (int c = 0; c < ncol; ++c) {
            max_colour_size = std::max(max_colour_size, h->colour_start[c + 1]);
            h->colour_start[c + 1] += h->colour_start[c];
        }
        colour_list.resize(J);
        std::vector<int> fill(h->colour_start.begin(), h->colour_start.end() - 1);
        for (int j = 0; j < J; ++j) colour_list[fill[h->colour_of[j]]++] = j;
    }
    h->alpha_O = d->alpha_O; h->alpha_P = d->alpha_P;
    h->probe_update_start = d->probe_update_start;
    h->st = (cudaStream_t)d->cuda_stream;
    int rc = PTYCHO_OK;
    const size_t NN = (size_t)N * N, MM = (size_t)M * M;
    // object tiles and their position lists (ascending j)
    h->ntx = (M + kTW - 1) / kTW;
    const int nty = (M + kTR - 1) / kTR;
    h->ntiles = h->ntx * nty;
    // list lengths on the host (each patch adds one to a rectangle of tiles: a 2-D difference
    // array and its prefix sums), the lists themselves on the device (k_tile_lists)
    std::vector<int> tstart(h->ntiles + 1, 0), torder(h->ntiles);
    std::vector<long long> count(h->ntiles, 0);
    {
        const int ntx = h->ntx;
        std::vector<long long> diff((size_t)(nty + 1) * (ntx + 1), 0);
        for (int j = 0; j < J; ++j) {
            const int y = d->h_pos[2 * j], x = d->h_pos[2 * j + 1];
            const int ty0 = y / kTR, ty1 = (y + N - 1) / kTR, tx0 = x / kTW, tx1 = (x + N - 1) / kTW;
            diff[(size_t)ty0 * (ntx + 1) + tx0] += 1;
            diff[(size_t)ty0 * (ntx + 1) + tx1 + 1] -= 1;
            diff[(size_t)(ty1 + 1) * (ntx + 1) + tx0] -= 1;
            diff[(size_t)(ty1 + 1) * (ntx + 1) + tx1 + 1] += 1;
        }
        for (int ty = 0; ty < nty; ++ty)
            for (int tx = 0; tx < ntx; ++tx) {
                long long c = diff[(size_t)ty * (ntx + 1) + tx];
                if (ty > 0) c += count[(size_t)(ty - 1) * ntx + tx];
                if (tx > 0) c += count[(size_t)ty * ntx + tx - 1];
                if (ty > 0 && tx > 0) c -= count[(size_t)(ty - 1) * ntx + tx - 1];
                count[(size_t)ty * ntx + tx] = c;
            }
        long long total = 0;
        for (int t = 0; t < h->ntiles; ++t) {
            total += count[t];
            if (total > INT_MAX) {
                delete h;
                return pm::fail(PTYCHO_EINVAL, "ptycho_init: more than 2^31 tile-list entries");
            }
            tstart[t + 1] = (int)total;
        }
        for (int t = 0; t < h->ntiles; ++t) torder[t] = t;
        std::stable_sort(torder.begin(), torder.end(), [&](int a, int b) { return count[a] > count[b]; });
    }
    // probe partial-sum layout
    h->nqt = ((N + kTW - 1) / kTW) * ((N + kTR - 1) / kTR);
    h->per_chunk = 128;                                  // 16 positions per warp
    h->nchunk = (J + h->per_chunk - 1) / h->per_chunk;
    h->nred = (int)((NN * Q + kThreads - 1) / kThreads);

    rc = setup_exit(h);
    if (!rc && h->fft_gemm) rc = pm::dft64_prepare(&h->gemm_sms);
    if (!rc) rc = halloc(h, &h->d_pos, J);
    if (!rc) rc = halloc(h, &h->d_obj, MM);
    if (!rc) rc = halloc(h, &h->d_probe, NN * Q);
    if (!rc) rc = halloc(h, &h->d_psi, (size_t)J * Q * NN);
    if (!rc && h->exit_tma) rc = halloc(h, &h->d_slot, (size_t)exit_slots(h->grid_exit) * NN);
    if (!rc && h->exit_tma) rc = alloc_tail(h);
    if (!rc) rc = halloc(h, &h->d_status, 1);
    if (!rc) rc = halloc(h, &h->d_num_o, MM);
    if (!rc) rc = halloc(h, &h->d_den_o, MM);
    if (!rc) rc = halloc(h, &h->d_tile_max, h->ntiles);
    if (!rc) rc = halloc(h, &h->d_num_p, NN * Q);
    if (!rc) rc = halloc(h, &h->d_den_p, NN * Q);
    if (!rc) rc = halloc(h, &h->d_pnum, (size_t)h->nchunk * Q * NN);
    if (!rc) rc = halloc(h, &h->d_pden, (size_t)h->nchunk * Q * NN);
    if (!rc) rc = halloc(h, &h->d_pmax, h->nred);
    if (!rc) rc = halloc(h, &h->d_amp, (size_t)J * NN);
    if (!rc && Q > 1) rc = halloc(h, &h->d_amp_nat, (size_t)J * NN);
    if (!rc && Q > 1 && h->exit_tma) rc = halloc(h, &h->d_fscale, (size_t)J * NN);
    h->n_err = (Q > 1 && h->exit_tma) ? J * (256 / kScaleCols) : J;   // mixed N = 256: per strip
    if (!rc) rc = halloc(h, &h->d_err_pos, (size_t)h->n_err);
    if (!rc) rc = halloc(h, &h->d_a2, J);
    if (!rc) rc = halloc(h, &h->d_inv_norm, 1);
    if (!rc) rc = halloc(h, &h->d_err_batch, 1);
    if (!rc) rc = halloc(h, &h->d_tstart, h->ntiles + 1);
    if (!rc) rc = halloc(h, &h->d_tlist, (size_t)tstart[h->ntiles]);
    if (!rc) rc = halloc(h, &h->d_torder, (size_t)h->ntiles);
    if (!rc) rc = halloc(h, &h->d_trange, (size_t)h->ntiles);
    if (!rc && h->algorithm == PTYCHO_ALG_EPIE_COLOUR) rc = halloc(h, &h->d_colour_list, (size_t)J);
    if (!rc && h->algorithm == PTYCHO_ALG_EPIE_COLOUR) rc = halloc(h, &h->d_epie_part, (size_t)max_colour_size * NN);
    if (!rc && h->exit_tma) rc = encode_exit_tma(h);
    if (rc) { free_ctx(h); return rc; }
    auto fail_cuda = [&](cudaError_t e, const char *what) {
        int r = pm::cuda_fail(e, what);
        free_ctx(h);
        return r;
    };
    cudaError_t e;
    std::vector<int2> pos2(J);
    for (int j = 0; j < J; ++j) pos2[j] = make_int2(d->h_pos[2 * j], d->h_pos[2 * j + 1]);
    if ((e = cudaMemcpyAsync(h->d_pos, pos2.data(), J * sizeof(int2), cudaMemcpyHostToDevice, h->st)))
        return fail_cuda(e, "copy positions");
    if ((e = cudaMemcpyAsync(h->d_tstart, tstart.data(), tstart.size() * sizeof(int), cudaMemcpyHostToDevice, h->st)))
        return fail_cuda(e, "copy tile starts");
    std::vector<int2> trange(h->ntiles);
    for (int i = 0; i < h->ntiles; ++i) trange[i] = make_int2(tstart[torder[i]], tstart[torder[i] + 1]);
    if ((e = cudaMemcpyAsync(h->d_torder, torder.data(), torder.size() * sizeof(int), cudaMemcpyHostToDevice, h->st)))
        return fail_cuda(e, "copy tile order");
    if ((e = cudaMemcpyAsync(h->d_trange, trange.data(), trange.size() * sizeof(int2), cudaMemcpyHostToDevice, h->st)))
        return fail_cuda(e, "copy tile ranges");
    if (h->d_colour_list &&
        (e = cudaMemcpyAsync(h->d_colour_list, colour_list.data(), J * sizeof(int), cudaMemcpyHostToDevice, h->st)))
        return fail_cuda(e, "copy colour lists");
    k_tile_lists<<<(unsigned)(((size_t)h->ntiles * 32 + kThreads - 1) / kThreads), kThreads, 0, h->st>>>(
        h->d_pos, J, N, h->ntx, h->ntiles, h->d_tstart, h->d_tlist);
    if ((e = cudaGetLastError())) return fail_cuda(e, "k_tile_lists");
    if ((rc = copy_in_complex(h->d_obj, d->obj0, MM, d->init_on_device != 0, h->st))) { free_ctx(h); return rc; }
    if ((rc = copy_in_complex(h->d_probe, d->probe0, NN * Q, d->init_on_device != 0, h->st))) { free_ctx(h); return rc; }
    if ((e = cudaMemsetAsync(h->d_status, 0, sizeof(int), h->st))) return fail_cuda(e, "clear status");
    k_amplitudes<<<J, kThreads, 0, h->st>>>(d->d_fused, h->d_amp, h->d_amp_nat, h->d_a2, N, h->exit_tma ? 16 : 0);
    if ((e = cudaGetLastError())) return fail_cuda(e, "k_amplitudes");
    k_inv_norm<<<1, kThreads, 0, h->st>>>(h->d_a2, J, h->d_inv_norm);
    if ((e = cudaGetLastError())) return fail_cuda(e, "k_inv_norm");
    if ((e = cudaStreamSynchronize(h->st))) return fail_cuda(e, "ptycho_init synchronise");
    *out = h;
    return PTYCHO_OK;
}

extern "C" int ptycho_iterate(ptycho_handle h, int n_iter, double *h_err) {
    pm::NvtxRange range("ptycho_iterate");
    if (!h) return pm::fail(PTYCHO_EINVAL, "ptycho_iterate: NULL handle");
    if (n_iter < 0) return pm::fail(PTYCHO_EINVAL, "ptycho_iterate: n_iter = %d < 0", n_iter);
    if (n_iter == 0) return PTYCHO_OK;
    if (n_iter > h->err_cap) {
        int rc = hfree(h, &h->d_err);
        if (!rc) rc = halloc(h, &h->d_err, (size_t)n_iter);
        if (rc) { h->err_cap = 0; return rc; }
        h->err_cap = n_iter;
    }
    if (h->timing) {
        const size_t need = (size_t)n_iter * ST_COUNT + 1;      // at most one per stage, plus one
        while (h->ev.size() < need) {
            cudaEvent_t ev;
            PM_CUDA(cudaEventCreate(&ev));
            h->ev.push_back(ev);
        }
        h->mark.assign((size_t)n_iter * ST_COUNT * 2, -1);
        h->ev_used = 0;
        h->ev_fresh = false;
    }
    {
        cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
        PM_CUDA(cudaStreamIsCapturing(h->st, &cap));
        struct PdlScope {
            ptycho_ctx *h;
            ~PdlScope() { h->pdl = false; }
        } scope{h};
        h->pdl = cap == cudaStreamCaptureStatusNone;
        for (int i = 0; i < n_iter; ++i) {
            const bool upd = h->iter >= h->probe_update_start;
            int rc = iterate_one(h, h->d_err + i, (size_t)i * ST_COUNT, upd);
            if (rc) return rc;
            ++h->iter;
        }
    }
    if (h->timing && h->ev_used > 0) {
        PM_CUDA(cudaEventSynchronize(h->ev[h->ev_used - 1]));
        for (size_t m = 0; m < (size_t)n_iter * ST_COUNT; ++m) {
            if (h->mark[2 * m] < 0) continue;
            float ms = 0.f;
            PM_CUDA(cudaEventElapsedTime(&ms, h->ev[h->mark[2 * m]], h->ev[h->mark[2 * m + 1]]));
            h->stage_ms[m % ST_COUNT] += ms;
        }
    }
    if (h_err) {
        int status = 0;
        PM_CUDA(cudaMemcpyAsync(h_err, h->d_err, (size_t)n_iter * sizeof(double), cudaMemcpyDeviceToHost, h->st));
        PM_CUDA(cudaMemcpyAsync(&status, h->d_status, sizeof(int), cudaMemcpyDeviceToHost, h->st));
        PM_CUDA(cudaStreamSynchronize(h->st));
        if (status) return pm::fail(PTYCHO_ETIMEDOUT, "ptycho_iterate: a bounded device wait gave up");
        for (int i = 0; i < n_iter; ++i)
            if (!std::isfinite(h_err[i]))
                return pm::fail(PTYCHO_ENONFINITE, "ptycho_iterate: error of iteration %d is not finite", i);
    }
    return PTYCHO_OK;
}

static int get_complex(ptycho_handle h, const float2 *src, size_t count, void *dst, int dst_on_device) {
    if (!h || !dst) return pm::fail(PTYCHO_EINVAL, "get: NULL handle or destination");
    PM_CUDA(cudaMemcpyAsync(dst, src, count * sizeof(float2),
                            dst_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, h->st));
    if (!dst_on_device) PM_CUDA(cudaStreamSynchronize(h->st));
    return PTYCHO_OK;
}

extern "C" int ptycho_get_object(ptycho_handle h, void *dst, int dst_on_device) {
    if (!h) return pm::fail(PTYCHO_EINVAL, "ptycho_get_object: NULL handle");
    return get_complex(h, h->d_obj, (size_t)h->M * h->M, dst, dst_on_device);
}

extern "C" int ptycho_get_probe(ptycho_handle h, void *dst, int dst_on_device) {
    if (!h) return pm::fail(PTYCHO_EINVAL, "ptycho_get_probe: NULL handle");
    return get_complex(h, h->d_probe, (size_t)h->Q * h->N * h->N, dst, dst_on_device);
}

extern "C" void ptycho_destroy(ptycho_handle h) { free_ctx(h); }

extern "C" int ptycho_set_timing(ptycho_handle h, int enable) {
    if (!h) return pm::fail(PTYCHO_EINVAL, "ptycho_set_timing: NULL handle");
    h->timing = enable != 0;
    for (int s = 0; s < ST_COUNT; ++s) { h->stage_ms[s] = 0.0; h->stage_launches[s] = 0; }
    return PTYCHO_OK;
}

extern "C" int ptycho_stage_times(ptycho_handle h, double *ms, long long *launches) {
    if (!h || !ms || !launches) return pm::fail(PTYCHO_EINVAL, "ptycho_stage_times: NULL argument");
    for (int s = 0; s < ST_COUNT; ++s) { ms[s] = h->stage_ms[s]; launches[s] = h->stage_launches[s]; }
    return PTYCHO_OK;
}

extern "C" int ptycho_debug_wait_timeout(ptycho_handle h, int enable) {
    if (!h) return pm::fail(PTYCHO_EINVAL, "ptycho_debug_wait_timeout: NULL handle");
    if (!h->exit_tma)
        return pm::fail(PTYCHO_EINVAL, "ptycho_debug_wait_timeout: the handle's exit-wave kernel (N = %d) has no "
                                       "bounded waits to exercise; the hook needs N = 256", h->N);
    if (enable < 0 || enable > 2)
        return pm::fail(PTYCHO_EINVAL, "ptycho_debug_wait_timeout: enable = %d not in {0, 1, 2}", enable);
    h->inject_wait = enable;
    return PTYCHO_OK;
}

extern "C" int ptycho_get_colouring(ptycho_handle h, int32_t *h_colour, int *n_colours) {
    if (!h || !h_colour || !n_colours) return pm::fail(PTYCHO_EINVAL, "ptycho_get_colouring: NULL argument");
    if (h->algorithm != PTYCHO_ALG_EPIE_COLOUR)
        return pm::fail(PTYCHO_EINVAL, "ptycho_get_colouring: the handle does not use ePIE by colour");
    for (int j = 0; j < h->J; ++j) h_colour[j] = h->colour_of[j];
    *n_colours = (int)h->colour_start.size() - 1;
    return PTYCHO_OK;
}

// ---------------------------------------------------------------------------------------
// Batches of independent reconstructions (many datasets of uneven sizes).  One iteration of a
// batch = one exit-wave launch per class of small datasets (N = 16 or 64 radix, or N = 64
// tensor-core DFT), whose persistent CTAs walk the concatenated positions of every dataset of
// the class, plus, per dataset, the N = 256 exit-wave kernel (if any), the object update, the
// probe update and the error reduction on the dataset's own branch (stream); branches run
// concurrently and join on the batch stream.  With PTYCHO_BATCH_GRAPH the iteration is
// captured once as a CUDA graph and replayed.  PTYCHO_BATCH_AUTOTUNE times candidate launch
// shapes on the batch's own data (state restored afterwards) and keeps the fastest.
struct ptycho_batch_ctx {
    struct Class {
        int kind = 0;                         // 4 or 8: radix kernel of that R; 64: tensor-core DFT
        std::vector<int> members;
        ExitArgs *d_table = nullptr;
        pm::Dft64Exit *d_gtable = nullptr;
        int *d_start = nullptr;               // prefix of positions (radix) or patch groups (tensor)
        int units = 0;
        int grid = 0, grid_max = 0;
        size_t smem = 0;
    };
    std::vector<ptycho_ctx *> hs;
    cudaStream_t user_st = nullptr;           // the caller's stream (may be the legacy default stream)
    cudaStream_t st = nullptr;                // the batch's own stream (capturable)
    cudaEvent_t ev_user = nullptr;
    int flags = 0;
    int sms = 0;
    std::vector<cudaStream_t> side, cls_st;
    cudaEvent_t ev_fork = nullptr, ev_done = nullptr;
    std::vector<cudaEvent_t> ev_join, ev_cls, ev_in;
    std::vector<Class> cls;
    std::vector<int> cls_of;
    cudaGraphExec_t exec = nullptr;
    std::vector<char> cap_mask;
    int *d_status = nullptr;
    std::string describe;
    // one persistent exit-wave launch for every single-mode radix dataset (k_exit_wave_all)
    bool one_launch = false;
    std::vector<char> in_all;                 // dataset i's exit waves are in the one launch
    int4 *d_units = nullptr;
    int nunits = 0, grid_all = 0;
    ExitArgs *d_etab = nullptr;
    TmaArgs *d_ttab = nullptr;
    TmaMaps *d_mtab = nullptr;
    float2 *d_slot = nullptr;                 // one 256 x 256 slot per CTA of the one launch
};

namespace {

void free_batch(ptycho_batch_ctx *b) {
    if (!b) return;
    if (b->st) cudaStreamSynchronize(b->st);
    if (b->exec) cudaGraphExecDestroy(b->exec);
    for (auto &c : b->cls) {
        if (c.d_table) cudaFree(c.d_table);
        if (c.d_gtable) cudaFree(c.d_gtable);
        if (c.d_start) cudaFree(c.d_start);
    }
    for (cudaStream_t s : b->side) if (s) cudaStreamDestroy(s);
    for (cudaStream_t s : b->cls_st) if (s) cudaStreamDestroy(s);
    for (cudaEvent_t e : b->ev_join) if (e) cudaEventDestroy(e);
    for (cudaEvent_t e : b->ev_cls) if (e) cudaEventDestroy(e);
    for (cudaEvent_t e : b->ev_in) if (e) cudaEventDestroy(e);
    if (b->ev_fork) cudaEventDestroy(b->ev_fork);
    if (b->ev_user) cudaEventDestroy(b->ev_user);
    if (b->st) cudaStreamDestroy(b->st);
    if (b->ev_done) cudaEventDestroy(b->ev_done);
    if (b->d_status) cudaFree(b->d_status);
    void *ptrs[] = {b->d_units, b->d_etab, b->d_ttab, b->d_mtab, b->d_slot};
    for (void *q : ptrs)
        if (q) cudaFree(q);
    delete b;
}

int launch_class(ptycho_batch_ctx *b, const ptycho_batch_ctx::Class &c, cudaStream_t s) {
    if (c.kind == 64)
        return pm::dft64_exit_multi_launch(c.d_gtable, c.d_start, (int)c.members.size(), c.units, b->d_status, c.grid,
                                           s);
    ExitArgs a{};
    a.table = c.d_table;
    a.ustart = c.d_start;
    a.ntable = (int)c.members.size();
    a.J = c.units;
    a.Q = 1;
    if (c.kind == 4) k_exit_wave<4, XM_FULL><<<c.grid, kThreads, c.smem, s>>>(a);
    else if (c.kind == 128) k_exit_wave128<XM_FULL><<<c.grid, kThreads128, c.smem, s>>>(a);
    else k_exit_wave<8, XM_FULL><<<c.grid, kThreads, c.smem, s>>>(a);
    PM_LAUNCHED("k_exit_wave (datasets)");
    return PTYCHO_OK;
}

// Enqueue one iteration of every dataset on the batch stream (fork / join over side streams).
int enqueue_iteration(ptycho_batch_ctx *b, const std::vector<char> &upd) {
    if (b->one_launch) {
        k_exit_wave_all<<<b->grid_all, kAllThreads, all_smem_bytes(), b->st>>>(b->d_units, b->nunits, b->d_etab,
                                                                               b->d_ttab, b->d_mtab, b->d_status);
        PM_LAUNCHED("k_exit_wave_all");
    }
    PM_CUDA(cudaEventRecord(b->ev_fork, b->st));
    for (size_t c = 0; c < b->cls.size() && !b->one_launch; ++c) {
        PM_CUDA(cudaStreamWaitEvent(b->cls_st[c], b->ev_fork, 0));
        int rc = launch_class(b, b->cls[c], b->cls_st[c]);
        if (rc) return rc;
        PM_CUDA(cudaEventRecord(b->ev_cls[c], b->cls_st[c]));
    }
    for (size_t i = 0; i < b->hs.size(); ++i) {
        ptycho_ctx *h = b->hs[i];
        cudaStream_t s = b->side[i];
        PM_CUDA(cudaStreamWaitEvent(s, b->ev_fork, 0));
        const int c = b->one_launch ? -1 : b->cls_of[i];
        if (c >= 0) PM_CUDA(cudaStreamWaitEvent(s, b->ev_cls[c], 0));
        cudaStream_t saved = h->st;
        const bool timing = h->timing;                 // no per-stage events inside a batch
        h->st = s;
        h->timing = false;
        const bool exit_done = b->one_launch ? b->in_all[i] != 0 : c >= 0;
        const int rc = iterate_one(h, h->d_err_batch, 0, upd[i] != 0, exit_done);
        h->st = saved;
        h->timing = timing;
        if (rc) return rc;
        PM_CUDA(cudaEventRecord(b->ev_join[i], s));
        PM_CUDA(cudaStreamWaitEvent(b->st, b->ev_join[i], 0));
    }
    return PTYCHO_OK;
}

std::vector<char> update_mask(const ptycho_batch_ctx *b) {
    std::vector<char> m(b->hs.size());
    for (size_t i = 0; i < b->hs.size(); ++i) m[i] = b->hs[i]->iter >= b->hs[i]->probe_update_start;
    return m;
}

// n_iter iterations; graph mode re-captures when the set of probe-updating datasets changes.
int run_iterations(ptycho_batch_ctx *b, int n_iter, bool graph) {
    for (int it = 0; it < n_iter; ++it) {
        const std::vector<char> m = update_mask(b);
        int rc;
        if (graph) {
            if (!b->exec || m != b->cap_mask) {
                if (b->exec) { PM_CUDA(cudaGraphExecDestroy(b->exec)); b->exec = nullptr; }
                PM_CUDA(cudaStreamBeginCapture(b->st, cudaStreamCaptureModeThreadLocal));
                rc = enqueue_iteration(b, m);
                cudaGraph_t g = nullptr;
                const cudaError_t e = cudaStreamEndCapture(b->st, &g);
                if (rc) { if (g) cudaGraphDestroy(g); return rc; }
                if (e != cudaSuccess) return pm::cuda_fail(e, "cudaStreamEndCapture");
                const cudaError_t e2 = cudaGraphInstantiate(&b->exec, g, 0);
                cudaGraphDestroy(g);
                if (e2 != cudaSuccess) { b->exec = nullptr; return pm::cuda_fail(e2, "cudaGraphInstantiate"); }
                b->cap_mask = m;
            }
            PM_CUDA(cudaGraphLaunch(b->exec, b->st));
        } else if ((rc = enqueue_iteration(b, m))) {
            return rc;
        }
        for (ptycho_ctx *h : b->hs) ++h->iter;
    }
    return PTYCHO_OK;
}

// N = 256 kernels: rows per TMA stage (16 or 32); re-derives the grid, slot buffer and maps.
int retune_tma(ptycho_ctx *h, int B) {
    int per_sm = 0, sms = 0, dev = 0, rc;
    PM_CUDA(cudaGetDevice(&dev));
    PM_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    if (B == 32) rc = setup_tma_kernel<32, XM_FULL>(h, &per_sm);
    else rc = setup_tma_kernel<16, XM_FULL>(h, &per_sm);
    if (rc) return rc;
    h->tma_batch = B;
    const int grid = std::max(1, std::min(h->J, sms * per_sm));
    if (grid != h->grid_exit) {
        PM_CUDA(cudaStreamSynchronize(h->st));
        if ((rc = hfree(h, &h->d_slot))) return rc;
        h->grid_exit = grid;
        if ((rc = halloc(h, &h->d_slot, (size_t)exit_slots(grid) * h->N * h->N))) return rc;
        if ((rc = alloc_tail(h))) return rc;
        PM_CUDA(cudaStreamSynchronize(h->st));         // the batch's streams use the new buffers
    }
    return encode_exit_tma(h);
}

double time_iterations(ptycho_batch_ctx *b, int n, int *rc) {
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    *rc = run_iterations(b, 1, false);                     // warm-up
    if (!*rc) cudaEventRecord(e0, b->st);
    if (!*rc) *rc = run_iterations(b, n, false);
    float ms = 0.f;
    if (!*rc) {
        cudaEventRecord(e1, b->st);
        cudaEventSynchronize(e1);
        cudaEventElapsedTime(&ms, e0, e1);
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return ms;
}

// Autotuner results by problem shape (class kind + dataset sizes), kept for the process: a
// later batch of the same shapes reuses the choice without timing again.
std::mutex g_tune_mu;
std::map<std::string, int> g_tune_cache;

const char *class_name(int kind) {
    return kind == 64 ? "dftgemm64" : (kind == 8 ? "radix64" : (kind == 128 ? "radix128" : "radix16"));
}

std::string class_key(const ptycho_batch_ctx *b, const ptycho_batch_ctx::Class &c) {
    std::string k = "k" + std::to_string(c.kind) + ":";
    for (int m : c.members) k += std::to_string(b->hs[m]->J) + "/" + std::to_string(b->hs[m]->M) + ",";
    return k;
}

int setup_one_launch(ptycho_batch_ctx *b);

// Datasets the one persistent exit-wave launch can take (single mode, radix FFT), and the key
// of the tuner's choice between it and the per-size launches for this set of shapes.
int one_launch_eligible(const ptycho_batch_ctx *b, std::string *key) {
    int n = 0;
    *key = "one:";
    for (const ptycho_ctx *h : b->hs)
        if (h->Q == 1 && !h->fft_gemm) {
            ++n;
            *key += std::to_string(h->N) + "/" + std::to_string(h->J) + "/" + std::to_string(h->M) + ",";
        }
    return n;
}

// Coordinate search over the launch shapes, on the batch's own data; object, probe and
// iteration counters are restored afterwards.  Last, the tuned per-size launches are timed
// against the one persistent launch for all eligible datasets, and the faster is kept.
int autotune(ptycho_batch_ctx *b) {
    const int reps = 3;
    std::vector<float2 *> so(b->hs.size()), sp(b->hs.size());
    std::vector<long long> sit(b->hs.size());
    int rc = PTYCHO_OK;
    bool need = false;                     // anything not in the cache?  (else no snapshot)
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        for (const auto &c : b->cls) need = need || (!b->one_launch && !g_tune_cache.count(class_key(b, c)));
        std::string bkey = "tma:";
        bool any = false;
        for (ptycho_ctx *h : b->hs)
            if (h->exit_tma && !h->fft_gemm && h->Q == 1 && h->algorithm == PTYCHO_ALG_AP && !b->one_launch) {
                bkey += std::to_string(h->J) + "/" + std::to_string(h->M) + ",";
                any = true;
            }
        need = need || (any && !g_tune_cache.count(bkey));
        std::string okey;
        need = need || (!b->one_launch && one_launch_eligible(b, &okey) >= 2 && !g_tune_cache.count(okey));
    }
    for (size_t i = 0; i < b->hs.size() && !rc && need; ++i) {
        ptycho_ctx *h = b->hs[i];
        rc = dalloc(&so[i], (size_t)h->M * h->M);
        if (!rc) rc = dalloc(&sp[i], (size_t)h->Q * h->N * h->N);
        if (!rc) {
            cudaMemcpyAsync(so[i], h->d_obj, (size_t)h->M * h->M * sizeof(float2), cudaMemcpyDeviceToDevice, b->st);
            cudaMemcpyAsync(sp[i], h->d_probe, (size_t)h->Q * h->N * h->N * sizeof(float2), cudaMemcpyDeviceToDevice,
                            b->st);
        }
        sit[i] = h->iter;
    }
    std::string rep = "{";
    char buf[256];
    int cached = 0;
    // grids of the multi-dataset classes
    for (size_t c = 0; c < b->cls.size() && !rc && !b->one_launch; ++c) {
        auto &k = b->cls[c];
        const std::string key = class_key(b, k);
        {
            std::lock_guard<std::mutex> lk(g_tune_mu);
            auto it = g_tune_cache.find(key);
            if (it != g_tune_cache.end()) {
                k.grid = it->second;
                ++cached;
                std::snprintf(buf, sizeof buf, "%s\"class_%s_grid\": %d", rep.size() > 1 ? ", " : "",
                              class_name(k.kind), k.grid);
                rep += buf;
                continue;
            }
        }
        std::vector<int> cand;
        for (int m : {1, 2, 3, 4, 6, 8}) {
            const int g = std::min(k.units, std::min(k.grid_max, m * b->sms));
            if (g >= 1 && std::find(cand.begin(), cand.end(), g) == cand.end()) cand.push_back(g);
        }
        if (k.kind == 64) cand = {std::min(k.units, b->sms / 2), std::min(k.units, b->sms)};
        int best = k.grid;
        double best_ms = 1e30;
        std::string tried;
        for (int g : cand) {
            if (g < 1) continue;
            k.grid = g;
            const double ms = time_iterations(b, reps, &rc);
            if (rc) break;
            std::snprintf(buf, sizeof buf, "%s%d:%.3f", tried.empty() ? "" : ",", g, ms / reps);
            tried += buf;
            if (ms < best_ms) { best_ms = ms; best = g; }
        }
        k.grid = best;
        {
            std::lock_guard<std::mutex> lk(g_tune_mu);
            g_tune_cache[key] = best;
        }
        std::snprintf(buf, sizeof buf, "%s\"class_%s_grid\": %d, \"class_%s_tried_ms\": \"%s\"",
                      rep.size() > 1 ? ", " : "", class_name(k.kind), best, class_name(k.kind), tried.c_str());
        rep += buf;
    }
    // rows per TMA stage of the N = 256 datasets (all together)
    std::vector<ptycho_ctx *> big;
    for (ptycho_ctx *h : b->hs)
        if (h->exit_tma && !h->fft_gemm && h->Q == 1 && h->algorithm == PTYCHO_ALG_AP && !b->one_launch)
            big.push_back(h);
    std::string bkey = "tma:";
    for (ptycho_ctx *h : big) bkey += std::to_string(h->J) + "/" + std::to_string(h->M) + ",";
    int bcached = 0;
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        auto it = g_tune_cache.find(bkey);
        if (it != g_tune_cache.end()) bcached = it->second;
    }
    if (!big.empty() && !rc && bcached) {
        for (ptycho_ctx *h : big)
            if (!rc && h->tma_batch != bcached) rc = retune_tma(h, bcached);
        ++cached;
        std::snprintf(buf, sizeof buf, "%s\"tma_rows_n256\": %d", rep.size() > 1 ? ", " : "", bcached);
        rep += buf;
    } else if (!big.empty() && !rc) {
        int best = 16;
        double best_ms = 1e30;
        std::string tried;
        for (int B : {16, 32}) {
            for (ptycho_ctx *h : big)
                if (!rc) rc = retune_tma(h, B);
            if (rc) break;
            const double ms = time_iterations(b, reps, &rc);
            if (rc) break;
            std::snprintf(buf, sizeof buf, "%s%d:%.3f", tried.empty() ? "" : ",", B, ms / reps);
            tried += buf;
            if (ms < best_ms) { best_ms = ms; best = B; }
        }
        for (ptycho_ctx *h : big)
            if (!rc) rc = retune_tma(h, best);
        {
            std::lock_guard<std::mutex> lk(g_tune_mu);
            g_tune_cache[bkey] = best;
        }
        std::snprintf(buf, sizeof buf, "%s\"tma_rows_n256\": %d, \"tma_rows_tried_ms\": \"%s\"",
                      rep.size() > 1 ? ", " : "", best, tried.c_str());
        rep += buf;
    }
    // one persistent launch for every eligible dataset, or the per-size launches tuned above
    std::string okey;
    if (!rc && !b->one_launch && one_launch_eligible(b, &okey) >= 2) {
        int choice = -1;
        {
            std::lock_guard<std::mutex> lk(g_tune_mu);
            auto it = g_tune_cache.find(okey);
            if (it != g_tune_cache.end()) choice = it->second;
        }
        if (choice >= 0) {
            ++cached;
            if (choice == 1) rc = setup_one_launch(b);
            std::snprintf(buf, sizeof buf, "%s\"one_launch\": %d", rep.size() > 1 ? ", " : "", choice);
        } else {
            const double t_sizes = time_iterations(b, reps, &rc);
            if (!rc) rc = setup_one_launch(b);
            const double t_one = rc ? 0.0 : time_iterations(b, reps, &rc);
            choice = (!rc && b->one_launch && t_one < t_sizes) ? 1 : 0;
            if (!rc) {
                std::lock_guard<std::mutex> lk(g_tune_mu);
                g_tune_cache[okey] = choice;
            }
            std::snprintf(buf, sizeof buf, "%s\"one_launch\": %d, \"one_launch_tried_ms\": \"sizes:%.3f,one:%.3f\"",
                          rep.size() > 1 ? ", " : "", choice, t_sizes / reps, t_one / reps);
        }
        rep += buf;
        if (!rc && choice == 0) b->one_launch = false;      // its tables stay allocated, unused
    }
    for (size_t i = 0; i < b->hs.size(); ++i) {
        ptycho_ctx *h = b->hs[i];
        if (so[i]) cudaMemcpyAsync(h->d_obj, so[i], (size_t)h->M * h->M * sizeof(float2), cudaMemcpyDeviceToDevice, b->st);
        if (sp[i])
            cudaMemcpyAsync(h->d_probe, sp[i], (size_t)h->Q * h->N * h->N * sizeof(float2), cudaMemcpyDeviceToDevice,
                            b->st);
        if (need) h->iter = sit[i];
    }
    cudaStreamSynchronize(b->st);
    for (size_t i = 0; i < b->hs.size(); ++i) {
        if (so[i]) cudaFree(so[i]);
        if (sp[i]) cudaFree(sp[i]);
    }
    std::snprintf(buf, sizeof buf, "%s\"from_cache\": %d", rep.size() > 1 ? ", " : "", cached);
    b->describe = rep + buf + "}";
    return rc;
}

// The unit list and dataset tables of the one persistent exit-wave launch (k_exit_wave_all):
// every single-mode, full-batch, radix-FFT dataset; the others keep their own launches.
int setup_one_launch(ptycho_batch_ctx *b) {
    const int n = (int)b->hs.size();
    b->in_all.assign(n, 0);
    std::vector<ExitArgs> et(n);
    std::vector<TmaArgs> tt(n);
    std::vector<int4> units;
    const int kinds[4] = {256, 128, 64, 16};
    for (int k : kinds)
        for (int i = 0; i < n; ++i) {
            ptycho_ctx *h = b->hs[i];
            if (h->Q != 1 || h->fft_gemm || h->N != k) continue;
            b->in_all[i] = 1;
            const int per = (k <= 64) ? 4 : 1;             // positions per unit (one per CTA quarter)
            for (int j0 = 0; j0 < h->J; j0 += per) units.push_back(make_int4(k, i, j0, std::min(per, h->J - j0)));
        }
    if (units.empty()) return PTYCHO_OK;
    b->grid_all = std::min<int>((int)units.size(), b->sms);
    bool any256 = false;
    for (int i = 0; i < n; ++i) {
        ptycho_ctx *h = b->hs[i];
        ExitArgs a{};
        a.obj = h->d_obj; a.probe = h->d_probe; a.amp = h->d_amp; a.pos = h->d_pos; a.psi = h->d_psi;
        a.err = h->d_err_pos; a.M = h->M; a.J = h->J; a.Q = 1;
        et[i] = a;
        tt[i] = tma_args(h);
        tt[i].status = b->d_status;
        tt[i].list = nullptr;
        tt[i].count = 0;
        any256 = any256 || (b->in_all[i] && h->N == 256);
    }
    int rc;
    std::vector<TmaMaps> mt(n);
    if (any256 && (rc = dalloc(&b->d_slot, (size_t)b->grid_all * 256 * 256))) return rc;
    for (int i = 0; i < n; ++i) {
        ptycho_ctx *h = b->hs[i];
        if (b->in_all[i] && h->N == 256 &&
            (rc = encode_tma_maps(&mt[i], h->d_probe, h->d_psi, b->d_slot, 1, h->J, b->grid_all, 32)))
            return rc;
    }
    if ((rc = dalloc(&b->d_units, units.size())) || (rc = dalloc(&b->d_etab, (size_t)n)) ||
        (rc = dalloc(&b->d_ttab, (size_t)n)) || (rc = dalloc(&b->d_mtab, (size_t)n)))
        return rc;
    PM_CUDA(cudaMemcpy(b->d_units, units.data(), units.size() * sizeof(int4), cudaMemcpyHostToDevice));
    PM_CUDA(cudaMemcpy(b->d_etab, et.data(), n * sizeof(ExitArgs), cudaMemcpyHostToDevice));
    PM_CUDA(cudaMemcpy(b->d_ttab, tt.data(), n * sizeof(TmaArgs), cudaMemcpyHostToDevice));
    PM_CUDA(cudaMemcpy(b->d_mtab, mt.data(), n * sizeof(TmaMaps), cudaMemcpyHostToDevice));
    PM_CUDA(cudaFuncSetAttribute(k_exit_wave_all, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)all_smem_bytes()));
    b->nunits = (int)units.size();
    b->one_launch = true;
    return PTYCHO_OK;
}

}  // namespace

extern "C" int ptycho_batch_create(ptycho_batch *out, const ptycho_handle *handles, int n, int flags,
                                   void *cuda_stream) {
    if (!out) return pm::fail(PTYCHO_EINVAL, "ptycho_batch_create: out is NULL");
    *out = nullptr;
    if (!handles || n < 1) return pm::fail(PTYCHO_EINVAL, "ptycho_batch_create: need n >= 1 handles");
    if (flags & ~(PTYCHO_BATCH_GRAPH | PTYCHO_BATCH_AUTOTUNE | PTYCHO_BATCH_ONE_LAUNCH))
        return pm::fail(PTYCHO_EINVAL, "ptycho_batch_create: unknown flags 0x%x", flags);
    for (int i = 0; i < n; ++i) {
        if (!handles[i]) return pm::fail(PTYCHO_EINVAL, "ptycho_batch_create: handle %d is NULL", i);
        if (handles[i]->algorithm != PTYCHO_ALG_AP)
            return pm::fail(PTYCHO_EINVAL, "ptycho_batch_create: handle %d is not a full-batch (AP) handle", i);
        if (handles[i]->timing)
            return pm::fail(PTYCHO_EINVAL, "ptycho_batch_create: handle %d has stage timing enabled", i);
        for (int k = 0; k < i; ++k)
            if (handles[k] == handles[i])
                return pm::fail(PTYCHO_EINVAL, "ptycho_batch_create: handle %d appears twice", i);
    }
    ptycho_batch_ctx *b = new (std::nothrow) ptycho_batch_ctx();
    if (!b) return pm::fail(PTYCHO_ENOMEM, "ptycho_batch_create: host allocation failed");
    b->user_st = (cudaStream_t)cuda_stream;
    b->flags = flags;
    int rc = PTYCHO_OK, dev = 0;
    auto bail = [&](int r) { free_batch(b); return r; };
    cudaError_t e;
    if ((e = cudaStreamCreateWithFlags(&b->st, cudaStreamNonBlocking)) ||
        (e = cudaEventCreateWithFlags(&b->ev_user, cudaEventDisableTiming)) ||
        (e = cudaEventRecord(b->ev_user, b->user_st)) || (e = cudaStreamWaitEvent(b->st, b->ev_user, 0)))
        return bail(pm::cuda_fail(e, "ptycho_batch_create: stream"));
    if ((e = cudaGetDevice(&dev)) || (e = cudaDeviceGetAttribute(&b->sms, cudaDevAttrMultiProcessorCount, dev)))
        return bail(pm::cuda_fail(e, "ptycho_batch_create: device query"));
    b->hs.assign(handles, handles + n);
    b->cls_of.assign(n, -1);
    // classes of datasets served by one multi-dataset exit-wave launch
    for (int i = 0; i < n; ++i) {
        ptycho_ctx *h = b->hs[i];
        if (h->Q != 1 || h->exit_tma || (h->fft_gemm && h->N != 64)) continue;   // own launch on its branch
        const int kind = h->fft_gemm ? 64 : h->R;
        int c = -1;
        for (size_t k = 0; k < b->cls.size(); ++k)
            if (b->cls[k].kind == kind) c = (int)k;
        if (c < 0) {
            b->cls.emplace_back();
            b->cls.back().kind = kind;
            c = (int)b->cls.size() - 1;
        }
        b->cls[c].members.push_back(i);
        b->cls_of[i] = c;
    }
    if ((rc = dalloc(&b->d_status, 1))) return bail(rc);
    if ((e = cudaMemsetAsync(b->d_status, 0, sizeof(int), b->st))) return bail(pm::cuda_fail(e, "clear status"));
    for (auto &c : b->cls) {
        const int nm = (int)c.members.size();
        std::vector<int> start(nm + 1, 0);
        if (c.kind == 64) {
            std::vector<pm::Dft64Exit> t(nm);
            for (int m = 0; m < nm; ++m) {
                ptycho_ctx *h = b->hs[c.members[m]];
                t[m] = pm::Dft64Exit{h->d_obj, h->d_probe, h->d_amp, h->d_pos, h->d_psi, h->d_err_pos, b->d_status, h->M,
                                     h->J};
                start[m + 1] = start[m] + pm::dft64_groups(h->J);
            }
            if ((rc = dalloc(&c.d_gtable, nm))) return bail(rc);
            if ((e = cudaMemcpy(c.d_gtable, t.data(), nm * sizeof(pm::Dft64Exit), cudaMemcpyHostToDevice)))
                return bail(pm::cuda_fail(e, "copy dataset table"));
            c.grid_max = b->sms;
        } else {
            std::vector<ExitArgs> t(nm);
            for (int m = 0; m < nm; ++m) {
                ptycho_ctx *h = b->hs[c.members[m]];
                ExitArgs a{};
                a.obj = h->d_obj; a.probe = h->d_probe; a.amp = h->d_amp; a.pos = h->d_pos; a.psi = h->d_psi;
                a.err = h->d_err_pos; a.M = h->M; a.J = h->J; a.Q = 1;
                t[m] = a;
                start[m + 1] = start[m] + h->J;
            }
            if ((rc = dalloc(&c.d_table, nm))) return bail(rc);
            if ((e = cudaMemcpy(c.d_table, t.data(), nm * sizeof(ExitArgs), cudaMemcpyHostToDevice)))
                return bail(pm::cuda_fail(e, "copy dataset table"));
            int per_sm = 0;
            c.smem = b->hs[c.members[0]]->exit_smem;
            if (c.kind == 4) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_exit_wave<4, XM_FULL>, kThreads, c.smem);
            else if (c.kind == 128)
                e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_exit_wave128<XM_FULL>, kThreads128, c.smem);
            else e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_exit_wave<8, XM_FULL>, kThreads, c.smem);
            if (e) return bail(pm::cuda_fail(e, "occupancy query"));
            c.grid_max = std::max(1, per_sm) * b->sms;
        }
        c.units = start[nm];
        c.grid = std::max(1, std::min(c.units, c.grid_max));
        if ((rc = dalloc(&c.d_start, nm + 1))) return bail(rc);
        if ((e = cudaMemcpy(c.d_start, start.data(), (nm + 1) * sizeof(int), cudaMemcpyHostToDevice)))
            return bail(pm::cuda_fail(e, "copy dataset prefix"));
    }
    b->side.assign(n, nullptr);
    b->ev_join.assign(n, nullptr);
    b->ev_in.assign(n, nullptr);
    for (int i = 0; i < n; ++i) {
        if ((e = cudaStreamCreateWithFlags(&b->side[i], cudaStreamNonBlocking)) ||
            (e = cudaEventCreateWithFlags(&b->ev_join[i], cudaEventDisableTiming)) ||
            (e = cudaEventCreateWithFlags(&b->ev_in[i], cudaEventDisableTiming)))
            return bail(pm::cuda_fail(e, "ptycho_batch_create: streams"));
    }
    if ((flags & PTYCHO_BATCH_ONE_LAUNCH) && (rc = setup_one_launch(b))) return bail(rc);
    b->cls_st.assign(b->cls.size(), nullptr);
    b->ev_cls.assign(b->cls.size(), nullptr);
    for (size_t c = 0; c < b->cls.size(); ++c)
        if ((e = cudaStreamCreateWithFlags(&b->cls_st[c], cudaStreamNonBlocking)) ||
            (e = cudaEventCreateWithFlags(&b->ev_cls[c], cudaEventDisableTiming)))
            return bail(pm::cuda_fail(e, "ptycho_batch_create: streams"));
    if ((e = cudaEventCreateWithFlags(&b->ev_fork, cudaEventDisableTiming)) ||
        (e = cudaEventCreateWithFlags(&b->ev_done, cudaEventDisableTiming)))
        return bail(pm::cuda_fail(e, "ptycho_batch_create: events"));
    // order after the handles' own pending work
    for (int i = 0; i < n; ++i) {
        if ((e = cudaEventRecord(b->ev_in[i], b->hs[i]->st)) || (e = cudaStreamWaitEvent(b->st, b->ev_in[i], 0)))
            return bail(pm::cuda_fail(e, "ptycho_batch_create: ordering"));
    }
    if (flags & PTYCHO_BATCH_AUTOTUNE) {
        if ((rc = autotune(b))) return bail(rc);
    } else {
        b->describe = "{}";
    }
    if ((e = cudaStreamSynchronize(b->st))) return bail(pm::cuda_fail(e, "ptycho_batch_create: synchronise"));
    if ((e = cudaStreamSynchronize(b->user_st))) return bail(pm::cuda_fail(e, "ptycho_batch_create: synchronise"));
    *out = b;
    return PTYCHO_OK;
}

extern "C" int ptycho_batch_iterate(ptycho_batch b, int n_iter, double *h_err) {
    pm::NvtxRange range("ptycho_batch_iterate");
    if (!b) return pm::fail(PTYCHO_EINVAL, "ptycho_batch_iterate: NULL batch");
    if (n_iter < 0) return pm::fail(PTYCHO_EINVAL, "ptycho_batch_iterate: n_iter = %d < 0", n_iter);
    if (n_iter == 0) return PTYCHO_OK;
    PM_CUDA(cudaEventRecord(b->ev_user, b->user_st));
    PM_CUDA(cudaStreamWaitEvent(b->st, b->ev_user, 0));
    for (size_t i = 0; i < b->hs.size(); ++i) {
        PM_CUDA(cudaEventRecord(b->ev_in[i], b->hs[i]->st));
        PM_CUDA(cudaStreamWaitEvent(b->st, b->ev_in[i], 0));
    }
    int rc = run_iterations(b, n_iter, (b->flags & PTYCHO_BATCH_GRAPH) != 0);
    if (rc) return rc;
    PM_CUDA(cudaEventRecord(b->ev_done, b->st));
    PM_CUDA(cudaStreamWaitEvent(b->user_st, b->ev_done, 0));
    for (ptycho_ctx *h : b->hs) PM_CUDA(cudaStreamWaitEvent(h->st, b->ev_done, 0));
    if (h_err) {
        // status words: the batch's own (shared launches) and every member's (kernels on the
        // member's branch write the handle's word)
        std::vector<int> status(b->hs.size() + 1, 0);
        for (size_t i = 0; i < b->hs.size(); ++i) {
            PM_CUDA(cudaMemcpyAsync(h_err + i, b->hs[i]->d_err_batch, sizeof(double), cudaMemcpyDeviceToHost, b->st));
            PM_CUDA(cudaMemcpyAsync(&status[i], b->hs[i]->d_status, sizeof(int), cudaMemcpyDeviceToHost, b->st));
        }
        PM_CUDA(cudaMemcpyAsync(&status[b->hs.size()], b->d_status, sizeof(int), cudaMemcpyDeviceToHost, b->st));
        PM_CUDA(cudaStreamSynchronize(b->st));
        for (size_t i = 0; i <= b->hs.size(); ++i)
            if (status[i])
                return pm::fail(PTYCHO_ETIMEDOUT, "ptycho_batch_iterate: a bounded device wait gave up (%s)",
                                i < b->hs.size() ? "a dataset's own kernels" : "a shared multi-dataset launch");
        for (size_t i = 0; i < b->hs.size(); ++i)
            if (!std::isfinite(h_err[i]))
                return pm::fail(PTYCHO_ENONFINITE, "ptycho_batch_iterate: error of dataset %zu is not finite", i);
    }
    return PTYCHO_OK;
}

extern "C" int ptycho_batch_describe(ptycho_batch b, char *buf, int len) {
    if (!b || !buf || len < 1) return pm::fail(PTYCHO_EINVAL, "ptycho_batch_describe: NULL argument");
    std::snprintf(buf, (size_t)len, "%s", b->describe.c_str());
    return PTYCHO_OK;
}

extern "C" void ptycho_batch_destroy(ptycho_batch b) { free_batch(b); }
