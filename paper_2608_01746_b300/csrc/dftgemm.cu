// Split-BF16 (3-term) DFT-as-GEMM on the fifth-generation tensor cores, N = 64.
//
// The unitary 2-D DFT of Eq. 3 (and its inverse) is computed as four real GEMMs per batch of
// patches, each of the form D = G B^T with
//   G  [128 x 128]  the 64-point DFT matrix F[u][r] = exp(-2 pi i u r / 64) as a real matrix
//                   over interleaved (re, im) indices: G[2u + s'][2r + s]
//   B  [128 x 128]  one row per transformed vector (2 patches x 64 vectors), interleaved re/im
//   D  [128 x 128]  FP32 in tensor memory: lane 2u + s' of column n = part s' of (F b_n)[u].
// Every operand is split x = hi + lo with hi = bf16(x), lo = bf16(x - hi), and the product is
// taken as G_hi B_hi + G_hi B_lo + G_lo B_hi (the lo x lo term, ~2^-18 relative, is dropped);
// accumulation is FP32 in TMEM.
//
// A CTA runs two independent pipelines of 256 threads (named barriers 1 and 2), each with its
// own 2-patch group, operand buffers, 128 TMEM columns and mbarrier, sharing the DFT matrix:
// while one pipeline's warps convert a pass result into the next operand, the other's MMAs
// keep the tensor core busy.  The pass structure keeps a whole group on chip.  Lane 2h + s of a pass's result
// holds part s of entry h of every transformed vector, i.e. one full vector of the NEXT
// pass's operand (which transforms along the other axis), so each epilogue reads its TMEM lane
// and writes one contiguous operand row:
//   pass 1  b_(p,c) = x_p[., c]            -> W_p = F x_p              (columns)
//   pass 2  b_(p,u) = W_p[u, .]            -> Psi_p = F x_p F          (rows; Psi^T per lane)
//   exit-wave form only:
//   modulus Psi' = A Psi / |Psi| (Psi' = A where Psi = 0), error (|Psi| - A)^2 per position
//   pass 3  b_(p,v) = conj(Psi')[., v]     -> V_p = F conj(Psi')
//   pass 4  b_(p,w) = V_p[w, .]            -> F conj(Psi') F = N conj(psi')
// so the inverse transform is the forward one applied by conjugation, and the 1/N unitary
// scale is applied in the epilogues (a power of two, exact).
#include <cuda_bf16.h>
#include <mutex>

#include "common.cuh"
#include "dftgemm.h"
#include "tcgen05.cuh"
#include "tma.cuh"

namespace {

using namespace pm;

constexpr int kN = 64;                     // transform length
constexpr int kK = 2 * kN;                 // real K: interleaved (re, im)
constexpr int kRows = 2 * kN;              // rows of G = MMA M
constexpr int kP = 2;                      // patches per pipeline group
constexpr int kCols = kP * kN;             // MMA N
constexpr int kPipes = 2;                  // independent pipelines per CTA
constexpr int kPipeThreads = 256;          // 8 warps: (TMEM lane quarter) x (patch)
constexpr int kThreads = kPipes * kPipeThreads;
constexpr uint32_t kLBO = 128;             // next core matrix along K
constexpr uint32_t kSBO = (kK / 8) * 128;  // next 8-row group
constexpr uint32_t kGBytes = kRows * kK * 2;
constexpr uint32_t kBBytes = kCols * kK * 2;
constexpr uint32_t kSmemBytes = 2 * kGBytes + kPipes * 2 * kBBytes + 1024;   // + alignment slack
constexpr uint32_t kTmemCols = 256;

static_assert(kCols <= 256 && kCols % 16 == 0, "MMA N");
static_assert(kTmemCols >= kPipes * kCols, "accumulator columns");

// G_hi then G_lo in the core-matrix layout; filled once per device by k_fill_dft64.
__device__ uint4 g_dft64[2 * kGBytes / 16];

enum { MODE_EXIT = 0, MODE_DFT = 1 };

struct Args {
    const float2 *obj;      // exit: object [M][M]
    const float2 *probe;    // exit: probe [N][N]
    const float *amp;       // exit: amplitudes [J][kx][ky] (DC at 0)
    const int2 *pos;        // exit: (row, column) of each patch
    float2 *psi;            // exit: psi' [J][N][N]
    double *err;            // exit: Fourier error per position
    const float2 *in;       // dft: [J][N][N]
    float2 *out;            // dft: [J][N][N]
    int inverse;            // dft: 1 = unitary inverse
    int *status;            // set to 1 when a bounded wait gives up
    int M, J;               // object side; number of patches / transforms
    // exit, several datasets: group g belongs to dataset d with gstart[d] <= g < gstart[d + 1]
    const pm::Dft64Exit *table;
    const int *gstart;
    int ntable;
};

using tc::split2;

__global__ void k_fill_dft64() {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= kRows * kK) return;
    const int m = i / kK, k = i % kK;
    const int u = m >> 1, sp = m & 1, r = k >> 1, s = k & 1;
    double sn, cs;
    sincospi(2.0 * (double)((u * r) % kN) / (double)kN, &sn, &cs);
    // Re y = cos Re x + sin Im x,  Im y = -sin Re x + cos Im x   (y = e^{-i theta} x)
    const double g = (sp == s) ? cs : (sp == 0 ? sn : -sn);
    const __nv_bfloat16 hi = __float2bfloat16_rn((float)g);
    const __nv_bfloat16 lo = __float2bfloat16_rn((float)(g - (double)__bfloat162float(hi)));
    uint16_t *gw = reinterpret_cast<uint16_t *>(g_dft64);
    const uint32_t off = tc::core_offset(m, k, kK) / 2;
    gw[off] = __bfloat16_as_ushort(hi);
    gw[kGBytes / 2 + off] = __bfloat16_as_ushort(lo);
}

// Operand of pass 1: B[p N + c][2 r + s] = x_p[r][c], 4 rows (16 bytes) per store; thread
// (p, c) of each half of the block takes half of the row quads.
template <int MODE>
__device__ __forceinline__ void fill_input(const Args &a, int j0, int np, uint8_t *bh, uint8_t *bl) {
    const int tid = threadIdx.x & (kPipeThreads - 1);
    const int pc = tid & (kCols - 1), rhalf = tid / kCols;
    const int p = pc >> 6, c = pc & (kN - 1);
    const int n = p * kN + c;
    const bool live = p < np;
    const float2 *x0 = nullptr, *x1 = nullptr;
    if (live) {
        if constexpr (MODE == MODE_EXIT) {
            const int2 pj = a.pos[j0 + p];
            x0 = a.obj + (size_t)pj.x * a.M + pj.y + c;
            x1 = a.probe + c;
        } else {
            x0 = a.in + (size_t)(j0 + p) * kN * kN + c;
        }
    }
    constexpr int kRq = kN / 4 / (kPipeThreads / kCols);
#pragma unroll 2
    for (int rq = rhalf * kRq; rq < (rhalf + 1) * kRq; ++rq) {
        uint32_t h[4], l[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int r = 4 * rq + q;
            float2 z = make_float2(0.f, 0.f);
            if (live) {
                if constexpr (MODE == MODE_EXIT) {
                    z = cmul(__ldg(x1 + (size_t)r * kN), __ldg(x0 + (size_t)r * a.M));
                } else {
                    z = __ldg(x0 + (size_t)r * kN);
                    if (a.inverse) z.y = -z.y;
                }
            }
            split2(z, h[q], l[q]);
        }
        const uint32_t off = tc::core_offset(n, 8 * rq, kK);
        *reinterpret_cast<uint4 *>(bh + off) = make_uint4(h[0], h[1], h[2], h[3]);
        *reinterpret_cast<uint4 *>(bl + off) = make_uint4(l[0], l[1], l[2], l[3]);
    }
}

// Two consecutive entries (c, c + 1), c even, of operand row n.
__device__ __forceinline__ void put_pair(uint8_t *bh, uint8_t *bl, int n, int c, float2 z0, float2 z1) {
    uint32_t h0, l0, h1, l1;
    split2(z0, h0, l0);
    split2(z1, h1, l1);
    const uint32_t off = tc::core_offset(n, 2 * c, kK);
    *reinterpret_cast<uint2 *>(bh + off) = make_uint2(h0, h1);
    *reinterpret_cast<uint2 *>(bl + off) = make_uint2(l0, l1);
}

// Reads the 64 accumulator columns of patch p in this thread's lane and hands the thread the
// complex entries c, c + 1 (c = 4 i + 2 part) of its lane pair's vector: lanes 2h and 2h + 1
// hold the real and imaginary rows of the same index h, and swap halves with one shuffle per
// two entries.
// The two 32-column halves are read one after the other (32 live registers, not 64).
template <typename F>
__device__ __forceinline__ void for_pairs(uint32_t lane_addr, int p, int part, F &&f) {
#pragma unroll
    for (int ch = 0; ch < 2; ++ch) {
        uint32_t v[32];
        tc::ld_32cols(lane_addr + (uint32_t)(p * kN + 32 * ch), v);
        tc::wait_ld();
#pragma unroll
        for (int i = 0; i < 32; i += 4) {
            const float a0 = __uint_as_float(v[i]), a1 = __uint_as_float(v[i + 1]);
            const float a2 = __uint_as_float(v[i + 2]), a3 = __uint_as_float(v[i + 3]);
            const float y0 = __shfl_xor_sync(0xffffffffu, part ? a0 : a2, 1);
            const float y1 = __shfl_xor_sync(0xffffffffu, part ? a1 : a3, 1);
            const float2 z0 = part ? make_float2(y0, a2) : make_float2(a0, y0);
            const float2 z1 = part ? make_float2(y1, a3) : make_float2(a1, y1);
            f(ch * 32 + i + 2 * part, z0, z1);
        }
    }
}

// Named barrier of one pipeline (ids 1, 2; id 0 is __syncthreads).
__device__ __forceinline__ void pipe_sync(int pipe) {
    asm volatile("bar.sync %0, %1;" ::"r"(pipe + 1), "r"(kPipeThreads) : "memory");
}

// Barrier of one pipeline that also returns the AND of `v` over its threads.
__device__ __forceinline__ bool pipe_and(int pipe, bool v) {
    uint32_t out;
    asm volatile(
        "{\n\t.reg .pred q, r;\n\t"
        "setp.ne.u32 q, %1, 0;\n\t"
        "bar.red.and.pred r, %2, %3, q;\n\t"
        "selp.u32 %0, 1, 0, r;\n\t}"
        : "=r"(out)
        : "r"((uint32_t)v), "r"(pipe + 1), "r"(kPipeThreads)
        : "memory");
    return out != 0;
}

// One GEMM pass D = G_hi B_hi + G_hi B_lo + G_lo B_hi of one pipeline.  Every thread of the
// pipeline calls it; returns false (for all of them) when the completion wait gave up.
template <int NCOLS = kCols>
__device__ __forceinline__ bool mma_pass(int pipe, uint32_t tmem, uint32_t gh, uint32_t bh, uint64_t *bar,
                                         uint32_t &phase) {
    tma::fence_async_smem();          // operand writes -> visible to the tensor core
    tc::fence_before();
    pipe_sync(pipe);
    // Warp 0 of the pipeline issues the MMAs and polls their completion; the other warps sleep
    // in the closing barrier instead of spinning (spinning warps would take issue slots from
    // the other pipeline's epilogue).
    const bool waiter = ((threadIdx.x & (kPipeThreads - 1)) >> 5) == 0;
    bool ok = true;
    if (waiter) {
      if ((threadIdx.x & (kPipeThreads - 1)) == 0) {
        tc::fence_after();
        constexpr uint32_t idesc = tc::idesc_bf16_f32(kRows, NCOLS);
        const uint32_t gl = gh + kGBytes, bl = bh + (uint32_t)NCOLS * kK * 2;
#pragma unroll
        for (int t = 0; t < 3; ++t) {
            const uint32_t ab = (t == 2) ? gl : gh;
            const uint32_t bb = (t == 1) ? bl : bh;
#pragma unroll
            for (int ks = 0; ks < kK / 16; ++ks)
                tc::mma_bf16(tmem, tc::smem_desc(ab + ks * 256, kLBO, kSBO), tc::smem_desc(bb + ks * 256, kLBO, kSBO),
                             idesc, (uint32_t)((t | ks) != 0));
        }
        tc::commit(bar);
      }
      __syncwarp();
      ok = tma::mbar_wait(bar, phase);
      tc::fence_before();
    }
    const bool all = pipe_and(pipe, ok);
    tc::fence_after();
    if (all) phase ^= 1;
    return all;
}

template <int MODE>
__global__ void __launch_bounds__(kThreads, 1) k_dft64_gemm(Args a) {
    extern __shared__ uint8_t smem_raw[];
    uint8_t *sm = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
    __shared__ uint64_t bars[kPipes];
    __shared__ uint32_t tmem_slot;
    __shared__ double s_err[kThreads / 32];

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int pipe = tid / kPipeThreads, ptid = tid & (kPipeThreads - 1);
    uint8_t *sG = sm;
    uint8_t *sBh = sm + 2 * kGBytes + pipe * 2 * kBBytes;
    uint8_t *sBl = sBh + kBBytes;
    uint64_t *bar = &bars[pipe];
    for (int i = tid; i < (int)(2 * kGBytes / 16); i += kThreads) reinterpret_cast<uint4 *>(sG)[i] = g_dft64[i];
    if (warp == 0) tc::alloc(&tmem_slot, kTmemCols);
    if (tid == 0) {
        for (int q = 0; q < kPipes; ++q) tma::mbar_init(&bars[q], 1);
        tma::fence_barrier_init();
    }
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    const uint32_t tmem = tmem_slot + (uint32_t)(pipe * kCols);   // this pipeline's columns
    const uint32_t gh = tc::smem_addr(sG), bh = tc::smem_addr(sBh);
    uint32_t phase = 0;

    const int row = 32 * (warp & 3) + lane;        // accumulator lane 2 h + part
    const int half = row >> 1, part = row & 1;
    const int p = (warp >> 2) & (kP - 1);          // this warp's patch in the group
    const uint32_t lane_addr = tmem + ((uint32_t)(32 * (warp & 3)) << 16);
    const float invN = 1.0f / (float)kN;
    const int ngroups = a.table ? __ldg(a.gstart + a.ntable) : (a.J + kP - 1) / kP;
    bool failed = false;

    for (int grp = blockIdx.x * kPipes + pipe; grp < ngroups; grp += gridDim.x * kPipes) {
        Args c = a;
        int lg = grp;
        if (a.table) {
            int lo = 0, hi = a.ntable - 1;
            while (lo < hi) {
                const int mid = (lo + hi + 1) >> 1;
                if (__ldg(a.gstart + mid) <= grp) lo = mid;
                else hi = mid - 1;
            }
            const pm::Dft64Exit &e = a.table[lo];
            c.obj = e.obj;
            c.probe = e.probe;
            c.amp = e.amp;
            c.pos = e.pos;
            c.psi = e.psi;
            c.err = e.err;
            c.M = e.M;
            c.J = e.J;
            lg = grp - __ldg(a.gstart + lo);
        }
        const int j0 = lg * kP;
        const int np = min(kP, c.J - j0);
        fill_input<MODE>(c, j0, np, sBh, sBl);
        if (!mma_pass(pipe, tmem, gh, bh, bar, phase)) { failed = true; break; }
        const bool live = p < np;                  // warp-uniform
        // pass-2 operand: rows of W_p
        if (live)
            for_pairs(lane_addr, p, part,
                      [&](int c, float2 z0, float2 z1) { put_pair(sBh, sBl, p * kN + half, c, z0, z1); });
        if (!mma_pass(pipe, tmem, gh, bh, bar, phase)) { failed = true; break; }
        if constexpr (MODE == MODE_DFT) {
            // lane (v, part) holds part of Psi_p[u][v] for every u
            if (live) {
                float2 *o = c.out + (size_t)(j0 + p) * kN * kN + half;
                const float sy = c.inverse ? -invN : invN;
                for_pairs(lane_addr, p, part, [&](int c, float2 z0, float2 z1) {
                    o[(size_t)c * kN] = make_float2(z0.x * invN, z0.y * sy);
                    o[(size_t)(c + 1) * kN] = make_float2(z1.x * invN, z1.y * sy);
                });
            }
        } else {
            // modulus constraint against A_j[v][u], then conj(Psi') as the pass-3 operand
            float ep = 0.f;
            if (live) {
                const float *amp = c.amp + (size_t)(j0 + p) * kN * kN + (size_t)half * kN;
                for_pairs(lane_addr, p, part, [&](int c, float2 z0, float2 z1) {
                    const float2 A2 = __ldg(reinterpret_cast<const float2 *>(amp + c));
                    // z = N Psi (the forward pass unscaled); A Psi / |Psi| = A z / |z|
                    float2 z[2] = {z0, z1};
                    const float A[2] = {A2.x, A2.y};
#pragma unroll
                    for (int q = 0; q < 2; ++q) {
                        const float mag2 = cabs2(z[q]);
                        if (mag2 > 0.f) {
                            const float inv = rsqrtf(mag2);
                            const float dm = mag2 * inv * invN - A[q];
                            ep += dm * dm;
                            z[q] = cscale(z[q], A[q] * inv);
                        } else {
                            ep += A[q] * A[q];
                            z[q] = make_float2(A[q], 0.f);
                        }
                        z[q].y = -z[q].y;
                    }
                    put_pair(sBh, sBl, p * kN + half, c, z[0], z[1]);
                });
            }
            if (!mma_pass(pipe, tmem, gh, bh, bar, phase)) { failed = true; break; }
            if (live)
                for_pairs(lane_addr, p, part,
                          [&](int c, float2 z0, float2 z1) { put_pair(sBh, sBl, p * kN + half, c, z0, z1); });
            if (!mma_pass(pipe, tmem, gh, bh, bar, phase)) { failed = true; break; }
            // lane (x, part) holds part of N conj(psi'_p)[w][x] for every w
            if (live) {
                float2 *o = c.psi + (size_t)(j0 + p) * kN * kN + half;
                for_pairs(lane_addr, p, part, [&](int c, float2 z0, float2 z1) {
                    o[(size_t)c * kN] = make_float2(z0.x * invN, -z0.y * invN);
                    o[(size_t)(c + 1) * kN] = make_float2(z1.x * invN, -z1.y * invN);
                });
            }
            // Fourier error per position: fixed-order sums over lanes, then over the 4 warps
            double d = (double)ep;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) d += __shfl_xor_sync(0xffffffffu, d, o);
            if (lane == 0) s_err[warp] = d;
            pipe_sync(pipe);
            if (ptid < np) {
                const double *se = s_err + pipe * (kPipeThreads / 32) + 4 * ptid;
                c.err[j0 + ptid] = ((se[0] + se[1]) + se[2]) + se[3];
            }
        }
    }
    if (failed) {
        if (ptid == 0) atomicExch(a.status, 1);
        tma::mbar_wait(bar, phase);           // let MMAs still in flight finish (bounded)
    }
    tc::fence_before();
    __syncthreads();
    if (warp == 0) {
        tc::fence_after();
        tc::dealloc(tmem, kTmemCols);
    }
}

// ---------------------------------------------------------------------------------------------
// N = 128: each 128-point transform is two 64-point GEMM halves (even / odd samples) and a
// radix-2 butterfly in the epilogue:  X[h] = E[h] + w O[h],  X[h + 64] = E[h] - w O[h],
// w = W_128^h.  One patch per group, one 256-thread pipeline per CTA: the operand has 256 rows
// (parity b, vector index), the accumulator 256 TMEM columns (b 128 + vector index).
//   pass 1  b_(r%2, c)  = psi[r][c], K index r / 2        -> rows W[u][c], u = h, h + 64
//   pass 2  b_(c%2, u)  = W[u][c], K index c / 2          -> Psi[u][v], v = h, h + 64
//   modulus, conj; pass 3 b_(u%2, v) = conj Psi'[u][v]     -> V[k][v]
//   pass 4  b_(v%2, k)  = V[k][v]                           -> N conj(psi')[k][x]
constexpr int kN2 = 128;
constexpr int kCols2 = 2 * kN2;                           // 256 operand rows / accumulator columns
constexpr uint32_t kB2Bytes = kCols2 * kK * 2;           // 64 KB per split term
constexpr uint32_t kSmem2 = 2 * kGBytes + 2 * kB2Bytes + 1024;
constexpr int kThreads2 = 256;

// One word (re, im) of operand row n at K index 2 q.
__device__ __forceinline__ void put1(uint8_t *bh, uint8_t *bl, int n, int q, float2 z) {
    uint32_t h, l;
    split2(z, h, l);
    const uint32_t off = tc::core_offset(n, 2 * q, kK);
    *reinterpret_cast<uint32_t *>(bh + off) = h;
    *reinterpret_cast<uint32_t *>(bl + off) = l;
}

// Columns [c0, c0 + 32) of both halves of this lane: complex E (column c) and O (column 128 + c)
// after the lane-pair exchange (the thread owns c = c0 + 4 i + 2 part + {0, 1}), then the
// butterfly with w: f(c, X_lo(c), X_hi(c), X_lo(c + 1), X_hi(c + 1)).
template <typename F>
__device__ __forceinline__ void butterfly_pairs(uint32_t lane_addr, int c0, int part, float2 w, F &&f) {
    uint32_t ve[32], vo[32];
    tc::ld_32cols(lane_addr + (uint32_t)c0, ve);
    tc::ld_32cols(lane_addr + (uint32_t)(kN2 + c0), vo);
    tc::wait_ld();
#pragma unroll
    for (int i = 0; i < 32; i += 4) {
        const float e0 = __uint_as_float(ve[i]), e1 = __uint_as_float(ve[i + 1]);
        const float e2 = __uint_as_float(ve[i + 2]), e3 = __uint_as_float(ve[i + 3]);
        const float o0 = __uint_as_float(vo[i]), o1 = __uint_as_float(vo[i + 1]);
        const float o2 = __uint_as_float(vo[i + 2]), o3 = __uint_as_float(vo[i + 3]);
        const float ye0 = __shfl_xor_sync(0xffffffffu, part ? e0 : e2, 1);
        const float ye1 = __shfl_xor_sync(0xffffffffu, part ? e1 : e3, 1);
        const float yo0 = __shfl_xor_sync(0xffffffffu, part ? o0 : o2, 1);
        const float yo1 = __shfl_xor_sync(0xffffffffu, part ? o1 : o3, 1);
        const float2 Ea = part ? make_float2(ye0, e2) : make_float2(e0, ye0);
        const float2 Eb = part ? make_float2(ye1, e3) : make_float2(e1, ye1);
        const float2 wOa = cmul(w, part ? make_float2(yo0, o2) : make_float2(o0, yo0));
        const float2 wOb = cmul(w, part ? make_float2(yo1, o3) : make_float2(o1, yo1));
        f(c0 + i + 2 * part, cadd(Ea, wOa), csub(Ea, wOa), cadd(Eb, wOb), csub(Eb, wOb));
    }
}

// Operand of pass 1: row (r % 2, c), K index r / 2 = psi[r][c]; thread (b, c) writes 4
// consecutive rows of its parity per 16-byte store.
template <int MODE>
__device__ __forceinline__ void fill_input128(const Args &a, int j, uint8_t *bh, uint8_t *bl) {
    const int tid = threadIdx.x;
    const int c = tid & (kN2 - 1), b = tid >> 7;
    const int n = b * kN2 + c;
    const float2 *x0, *x1 = nullptr;
    if constexpr (MODE == MODE_EXIT) {
        const int2 pj = a.pos[j];
        x0 = a.obj + (size_t)pj.x * a.M + pj.y + c;
        x1 = a.probe + c;
    } else {
        x0 = a.in + (size_t)j * kN2 * kN2 + c;
    }
#pragma unroll 2
    for (int q4 = 0; q4 < kN2 / 8; ++q4) {           // 4 values (K indices 4 q4 .. 4 q4 + 3) per store
        uint32_t h[4], l[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int r = 2 * (4 * q4 + q) + b;
            float2 z;
            if constexpr (MODE == MODE_EXIT) {
                z = cmul(__ldg(x1 + (size_t)r * kN2), __ldg(x0 + (size_t)r * a.M));
            } else {
                z = __ldg(x0 + (size_t)r * kN2);
                if (a.inverse) z.y = -z.y;
            }
            split2(z, h[q], l[q]);
        }
        const uint32_t off = tc::core_offset(n, 8 * q4, kK);
        *reinterpret_cast<uint4 *>(bh + off) = make_uint4(h[0], h[1], h[2], h[3]);
        *reinterpret_cast<uint4 *>(bl + off) = make_uint4(l[0], l[1], l[2], l[3]);
    }
}

template <int MODE>
__global__ void __launch_bounds__(kThreads2, 1) k_dft128_gemm(Args a) {
    extern __shared__ uint8_t smem_raw[];
    uint8_t *sm = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
    uint8_t *sG = sm;
    uint8_t *sBh = sm + 2 * kGBytes;
    uint8_t *sBl = sBh + kB2Bytes;
    __shared__ uint64_t bar;
    __shared__ uint32_t tmem_slot;
    __shared__ double s_err[kThreads2 / 32];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    for (int i = tid; i < (int)(2 * kGBytes / 16); i += kThreads2) reinterpret_cast<uint4 *>(sG)[i] = g_dft64[i];
    if (warp == 0) tc::alloc(&tmem_slot, 256);
    if (tid == 0) {
        tma::mbar_init(&bar, 1);
        tma::fence_barrier_init();
    }
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    const uint32_t tmem = tmem_slot;
    const uint32_t gh = tc::smem_addr(sG), bh = tc::smem_addr(sBh);
    uint32_t phase = 0;
    const int row = 32 * (warp & 3) + lane;              // TMEM lane 2 h + part
    const int h = row >> 1, part = row & 1;
    const int cbase = (warp >> 2) * 64;                  // this warp's vector indices: cbase .. + 63
    const uint32_t lane_addr = tmem + ((uint32_t)(32 * (warp & 3)) << 16);
    float ws, wc;
    sincospif(-2.0f * (float)h / (float)kN2, &ws, &wc);   // w = W_128^h (forward sign)
    const float2 w = make_float2(wc, ws);
    const float invN = 1.0f / (float)kN2;
    bool failed = false;
    for (int j = blockIdx.x; j < a.J; j += gridDim.x) {
        fill_input128<MODE>(a, j, sBh, sBl);
        if (!mma_pass<kCols2>(0, tmem, gh, bh, &bar, phase)) { failed = true; break; }
        // pass-2 operand: row (c % 2, u), K index c / 2 = W[u][c], u = h and h + 64
#pragma unroll 1
        for (int c0 = cbase; c0 < cbase + 64; c0 += 32)
            butterfly_pairs(lane_addr, c0, part, w, [&](int c, float2 la, float2 ha, float2 lb, float2 hb) {
                put1(sBh, sBl, h, c >> 1, la);
                put1(sBh, sBl, h + 64, c >> 1, ha);
                put1(sBh, sBl, kN2 + h, c >> 1, lb);
                put1(sBh, sBl, kN2 + h + 64, c >> 1, hb);
            });
        if (!mma_pass<kCols2>(0, tmem, gh, bh, &bar, phase)) { failed = true; break; }
        // lane (h, part): Psi[u][h] and Psi[u][h + 64] for u = c (even) and c + 1
        if constexpr (MODE == MODE_DFT) {
            float2 *o = a.out + (size_t)j * kN2 * kN2;
            const float sy = a.inverse ? -invN : invN;
#pragma unroll 1
            for (int c0 = cbase; c0 < cbase + 64; c0 += 32)
                butterfly_pairs(lane_addr, c0, part, w, [&](int u, float2 la, float2 ha, float2 lb, float2 hb) {
                    o[(size_t)u * kN2 + h] = make_float2(la.x * invN, la.y * sy);
                    o[(size_t)u * kN2 + h + 64] = make_float2(ha.x * invN, ha.y * sy);
                    o[(size_t)(u + 1) * kN2 + h] = make_float2(lb.x * invN, lb.y * sy);
                    o[(size_t)(u + 1) * kN2 + h + 64] = make_float2(hb.x * invN, hb.y * sy);
                });
        } else {
            float ep = 0.f;
            const float *amp = a.amp + (size_t)j * kN2 * kN2;    // amp[kx][ky]
            auto proj = [&](float2 z, float A) {        // z = N Psi (unscaled): A z / |z|
                const float mag2 = cabs2(z);
                if (mag2 > 0.f) {
                    const float inv = rsqrtf(mag2);
                    const float dm = mag2 * inv * invN - A;
                    ep += dm * dm;
                    z = cscale(z, A * inv);
                } else {
                    ep += A * A;
                    z = make_float2(A, 0.f);
                }
                z.y = -z.y;
                return z;
            };
#pragma unroll 1
            for (int c0 = cbase; c0 < cbase + 64; c0 += 32)
                butterfly_pairs(lane_addr, c0, part, w, [&](int u, float2 la, float2 ha, float2 lb, float2 hb) {
                    const float2 A_lo = __ldg(reinterpret_cast<const float2 *>(amp + (size_t)h * kN2 + u));
                    const float2 A_hi = __ldg(reinterpret_cast<const float2 *>(amp + (size_t)(h + 64) * kN2 + u));
                    // pass-3 operand: row (u % 2, v), K index u / 2 = conj Psi'[u][v]
                    put1(sBh, sBl, h, u >> 1, proj(la, A_lo.x));
                    put1(sBh, sBl, h + 64, u >> 1, proj(ha, A_hi.x));
                    put1(sBh, sBl, kN2 + h, u >> 1, proj(lb, A_lo.y));
                    put1(sBh, sBl, kN2 + h + 64, u >> 1, proj(hb, A_hi.y));
                });
            if (!mma_pass<kCols2>(0, tmem, gh, bh, &bar, phase)) { failed = true; break; }
#pragma unroll 1
            for (int c0 = cbase; c0 < cbase + 64; c0 += 32)
                butterfly_pairs(lane_addr, c0, part, w, [&](int v, float2 la, float2 ha, float2 lb, float2 hb) {
                    put1(sBh, sBl, h, v >> 1, la);
                    put1(sBh, sBl, h + 64, v >> 1, ha);
                    put1(sBh, sBl, kN2 + h, v >> 1, lb);
                    put1(sBh, sBl, kN2 + h + 64, v >> 1, hb);
                });
            if (!mma_pass<kCols2>(0, tmem, gh, bh, &bar, phase)) { failed = true; break; }
            // lane (x = h, part): N conj(psi')[k][h], [k][h + 64] for k = c (even), c + 1
            float2 *o = a.psi + (size_t)j * kN2 * kN2;
#pragma unroll 1
            for (int c0 = cbase; c0 < cbase + 64; c0 += 32)
                butterfly_pairs(lane_addr, c0, part, w, [&](int k, float2 la, float2 ha, float2 lb, float2 hb) {
                    o[(size_t)k * kN2 + h] = make_float2(la.x * invN, -la.y * invN);
                    o[(size_t)k * kN2 + h + 64] = make_float2(ha.x * invN, -ha.y * invN);
                    o[(size_t)(k + 1) * kN2 + h] = make_float2(lb.x * invN, -lb.y * invN);
                    o[(size_t)(k + 1) * kN2 + h + 64] = make_float2(hb.x * invN, -hb.y * invN);
                });
            double d = (double)ep;
#pragma unroll
            for (int o2 = 16; o2 > 0; o2 >>= 1) d += __shfl_xor_sync(0xffffffffu, d, o2);
            if (lane == 0) s_err[warp] = d;
            __syncthreads();
            if (tid == 0) {
                double sum = 0.0;
                for (int q = 0; q < kThreads2 / 32; ++q) sum += s_err[q];
                a.err[j] = sum;
            }
        }
    }
    if (failed) {
        if (tid == 0) atomicExch(a.status, 1);
        tma::mbar_wait(&bar, phase);
    }
    tc::fence_before();
    __syncthreads();
    if (warp == 0) {
        tc::fence_after();
        tc::dealloc(tmem, 256);
    }
}

int launch128(const Args &a, int mode, int sm_count, cudaStream_t st) {
    if (a.J <= 0) return PTYCHO_OK;
    const int grid = a.J < sm_count ? a.J : sm_count;
    if (mode == MODE_EXIT)
        k_dft128_gemm<MODE_EXIT><<<grid, kThreads2, kSmem2, st>>>(a);
    else
        k_dft128_gemm<MODE_DFT><<<grid, kThreads2, kSmem2, st>>>(a);
    PM_LAUNCHED("k_dft128_gemm");
    return PTYCHO_OK;
}

std::mutex g_mu;
bool g_ready[64] = {};

int launch(const Args &a, int mode, int sm_count, cudaStream_t st, int total_groups = -1) {
    const int ngroups = total_groups >= 0 ? total_groups : (a.J + kP - 1) / kP;
    if (ngroups <= 0) return PTYCHO_OK;
    const int ctas = (ngroups + kPipes - 1) / kPipes;
    const int grid = ctas < sm_count ? ctas : sm_count;
    if (mode == MODE_EXIT)
        k_dft64_gemm<MODE_EXIT><<<grid, kThreads, kSmemBytes, st>>>(a);
    else
        k_dft64_gemm<MODE_DFT><<<grid, kThreads, kSmemBytes, st>>>(a);
    PM_LAUNCHED("k_dft64_gemm");
    return PTYCHO_OK;
}

}  // namespace

namespace pm {

int dft64_prepare(int *sm_count) {
    int dev = 0;
    PM_CUDA(cudaGetDevice(&dev));
    PM_CUDA(cudaDeviceGetAttribute(sm_count, cudaDevAttrMultiProcessorCount, dev));
    std::lock_guard<std::mutex> lk(g_mu);
    if (dev >= 0 && dev < 64 && g_ready[dev]) return PTYCHO_OK;
    PM_CUDA(cudaFuncSetAttribute(k_dft64_gemm<MODE_EXIT>, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemBytes));
    PM_CUDA(cudaFuncSetAttribute(k_dft64_gemm<MODE_DFT>, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemBytes));
    PM_CUDA(cudaFuncSetAttribute(k_dft128_gemm<MODE_EXIT>, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmem2));
    PM_CUDA(cudaFuncSetAttribute(k_dft128_gemm<MODE_DFT>, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmem2));
    k_fill_dft64<<<(kRows * kK + 255) / 256, 256>>>();
    PM_LAUNCHED("k_fill_dft64");
    PM_CUDA(cudaDeviceSynchronize());
    if (dev >= 0 && dev < 64) g_ready[dev] = true;
    return PTYCHO_OK;
}

int dft64_matrix(const void **d_matrix) {
    int sms = 0, rc = dft64_prepare(&sms);
    if (rc) return rc;
    void *p = nullptr;
    PM_CUDA(cudaGetSymbolAddress(&p, g_dft64));
    *d_matrix = p;
    return PTYCHO_OK;
}

int dft64_exit_launch(const Dft64Exit &e, int sm_count, cudaStream_t st) {
    Args a{};
    a.obj = e.obj;
    a.probe = e.probe;
    a.amp = e.amp;
    a.pos = e.pos;
    a.psi = e.psi;
    a.err = e.err;
    a.status = e.status;
    a.M = e.M;
    a.J = e.J;
    return launch(a, MODE_EXIT, sm_count, st);
}

int dft64_groups(int J) { return (J + kP - 1) / kP; }

int dft128_exit_launch(const Dft64Exit &e, int sm_count, cudaStream_t st) {
    Args a{};
    a.obj = e.obj;
    a.probe = e.probe;
    a.amp = e.amp;
    a.pos = e.pos;
    a.psi = e.psi;
    a.err = e.err;
    a.status = e.status;
    a.M = e.M;
    a.J = e.J;
    return launch128(a, MODE_EXIT, sm_count, st);
}

int dft64_exit_multi_launch(const Dft64Exit *d_table, const int *d_gstart, int ntable, int total_groups,
                            int *d_status, int grid_cap, cudaStream_t st) {
    Args a{};
    a.table = d_table;
    a.gstart = d_gstart;
    a.ntable = ntable;
    a.status = d_status;
    return launch(a, MODE_EXIT, grid_cap, st, total_groups);
}

}  // namespace pm

extern "C" int dft2_split_bf16(const void *d_in, void *d_out, int B, int N, int inverse, int *d_status,
                               void *cuda_stream) {
    if (N != 64 && N != 128) return pm::fail(PTYCHO_EINVAL, "dft2_split_bf16: N = %d unsupported (64 or 128)", N);
    if (B < 0) return pm::fail(PTYCHO_EINVAL, "dft2_split_bf16: B = %d < 0", B);
    if (inverse != 0 && inverse != 1) return pm::fail(PTYCHO_EINVAL, "dft2_split_bf16: inverse must be 0 or 1");
    if (B == 0) return PTYCHO_OK;
    if (!d_in || !d_out || !d_status) return pm::fail(PTYCHO_EINVAL, "dft2_split_bf16: NULL pointer");
    int sms = 0;
    int rc = pm::dft64_prepare(&sms);
    if (rc) return rc;
    Args a{};
    a.in = static_cast<const float2 *>(d_in);
    a.out = static_cast<float2 *>(d_out);
    a.inverse = inverse;
    a.status = d_status;
    a.J = B;
    if (N == 128) return launch128(a, MODE_DFT, sms, static_cast<cudaStream_t>(cuda_stream));
    return launch(a, MODE_DFT, sms, static_cast<cudaStream_t>(cuda_stream));
}
