// N = 256 exit-wave kernel (k_exit_wave_tma) and its per-unit body, shared with the one-launch
// batch kernel.  Included by ptycho.cu inside its internal namespace, after the exit-wave modes
// XM_* and the FFT / TMA / complex helpers it uses.
#pragma once

// ---------------------------------------------------------------------------------------
// N = 256 exit-wave kernel: one 512-thread CTA per SM, persistent over positions, with a
// TMA pipeline through a per-CTA 512 KB tile slot that stays in L2.  Batches are 32 rows or
// columns (one per 16-thread FFT group); every batch of tile data is a bulk tensor copy that
// runs while the previous batch is transformed.
//
//   phase R   rows r = 32 b + g: probe rows arrive by TMA (double-buffered), object patch rows
//             by register-prefetched loads (the patch origin x is not 16-byte aligned);
//             psi = P * O_j, forward row FFT, written (128-byte swizzle) to a staging buffer
//             that is TMA-stored column-major into the slot.
//   phase C   32 slot columns per TMA load (double-buffered); forward column FFT, modulus
//             replacement against A_j (loads issued before the FFT), inverse column FFT;
//             results TMA-stored (128-byte swizzle) into psi_j, row-major.
//   phase R'  32 rows of psi_j per TMA load, inverse row FFT, TMA-stored back in place.
// FFT exchanges happen in place in the group's own staged row or column.  Waits are bounded
// (tma.cuh); on a timeout the kernel sets *a.status and returns.
struct TmaArgs {
    const float2 *obj;
    const float *amp;        // [J][N][N] column-major per position
    const int2 *pos;
    double *err;             // [J] Fourier error per position (XM_FULL)
    int *status;             // set to 1 if a bounded wait gave up
    const int *list;         // XM_FULL: if not NULL, process positions list[0 .. count)
    int count;
    int M, J, Q;
    int inject_wait;         // test hook: wait on a barrier nothing arrives on (short limit) first
};

struct TmaMaps {
    CUtensorMap prow;        // probe rows ([Q N] rows) box {256 c, B r}
    CUtensorMap slot_r;      // slot, column-major    box {16 r, 256 c}, 128-byte swizzle
    CUtensorMap slot_c;      // slot, column-major    box {256 r, 32 c}
    CUtensorMap psi_c;       // psi, row-major        box {16 c, 256 r}, 128-byte swizzle
    CUtensorMap psi_r;       // psi, row-major        box {256 c, 32 r}  (loads)
    CUtensorMap psi_w;       // psi, row-major        box {256 c, 16 r}  (stores)
};

// Batch = rows or columns per pipeline stage = FFT groups per CTA (16 threads each).  32:
// one 512-thread CTA per SM; 16: two 256-thread CTAs per SM, each with its own position.
template <int B>
__host__ __device__ constexpr size_t tma_buf_bytes() { return (size_t)B * 256 * sizeof(float2); }
template <int B>
__host__ __device__ constexpr size_t tma_smem_bytes() { return 1024 /*alignment slack*/ + 3 * tma_buf_bytes<B>() + 256 * sizeof(float2) + 64; }

// Per-CTA state of the N = 256 pipeline (shared by every unit the CTA processes).
struct TmaPipe {
    unsigned char *base;     // 1024-byte aligned: stage 0, stage 1, staging buffer (B x 256 float2 each)
    const float2 *tw;        // tw[k1 * 16 + t] = W_256^(t k1)
    uint64_t *bar;           // stage mbarriers [2] (+ [2] for the test hook)
    uint32_t *pending;       // thread 0: bit s = a load into stage s is in flight
    double *s_red;           // [threads / 32]
    uint32_t parity;         // bit s: phase parity of bar[s]
    bool failed;             // uniform after each barrier
    bool timed_out;          // this thread's waits
    int slot_col;            // this CTA's slot columns
    uint64_t pol_keep, pol_stream;
};

// Every copy carries an L2 cache policy: the probe rows, the slot and the intermediate psi
// columns (re-read by this CTA within the position) are kept, data read for the last time and
// the final psi_j' rows are evicted first (measured at lab scale: DRAM traffic 2.47 -> 1.24 MB per
// position with B = 32).  One unit: position j (or (j, m) for the mixed-state forms).  After a
// wait gives up the unit returns with p.failed set (uniformly) before waiting again, so the parity
// of a stage whose wait failed stays that of the load still in flight (tma_pipe_finish drains it).
// Returns the updated mutable state: bits 0-1 parity, bit 2 failed, bit 3 timed out.
__host__ __device__ constexpr uint32_t tma_state(uint32_t parity, bool failed, bool timed_out) {
    return parity | (failed ? 4u : 0u) | (timed_out ? 8u : 0u);
}

template <int B, int XM>
__device__ __forceinline__ uint32_t tma_unit(const TmaPipe &p, const TmaArgs &a, const TmaMaps &tm, int u) {
    constexpr int R = 16, N = 256, NB = N / B;
    constexpr int kTmaThreads = B * 16, kTmaBatch = B;
    constexpr size_t kTmaBuf = tma_buf_bytes<B>();
    constexpr bool kFull = (XM == XM_FULL || XM == XM_LIST);
    namespace T = pm::tma;
    const int tid = threadIdx.x;
    const int t = tid & 15, g = tid >> 4;                        // g in [0, B)
    const int h = g >> 4, gl = g & 15;                           // 16-wide box of the batch, row in it
    auto bin = [&](int s) { return (float2 *)(p.base + s * kTmaBuf); };
    float2 *bout = (float2 *)(p.base + 2 * kTmaBuf);
    const float2 *tw = p.tw;
    uint64_t *bar = p.bar;
    const float invN = 1.0f / (float)N;
    const int M = a.M;
    uint32_t parity = p.parity;
    bool failed = p.failed, timed_out = p.timed_out;
    auto wait_stage = [&](int s) {
        if (T::mbar_wait(&bar[s], (parity >> s) & 1u)) {
            if (tid == 0) *p.pending &= ~(1u << s);
            parity ^= 1u << s;
        } else {
            timed_out = true;
        }
    };
    // Barrier A of every batch: the batch's input buffer is consumed, the staging buffer's
    // previous store has finished reading it (thread 0 waited just before), and a timed-out
    // wait anywhere in the CTA is agreed on.
    auto barrier_a = [&]() {
        if (tid == 0) T::wait_read<0>();
        if (__syncthreads_or(timed_out)) failed = true;
    };
    // Staging buffer written: thread 0 stores it.
    auto publish = [&](const CUtensorMap *map, int x0, int y0, int dx, int dy, uint64_t pol) {
        T::fence_async_smem();
        __syncthreads();
        if (tid == 0) {
            T::store_2d_hint(map, x0, y0, bout, pol);
            if constexpr (B == 32) T::store_2d_hint(map, x0 + dx, y0 + dy, bout + 4096, pol);
            T::commit();
        }
    };
    auto prefetch = [&](int s, const CUtensorMap *map, int x, int y, uint64_t pol) {
        if (tid == 0) {
            *p.pending |= 1u << s;
            T::mbar_expect_tx(&bar[s], (uint32_t)kTmaBuf);
            T::load_2d_hint(bin(s), map, x, y, &bar[s], pol);
        }
    };
    const int slot_col = p.slot_col;
    const int j = kFull ? u : u / a.Q;
    const int prow0 = kFull ? 0 : (u % a.Q) * N;                  // first probe row of the mode
    float err = 0.f;
    if constexpr (XM != XM_INV) {
        const int2 pj = a.pos[j];
        // ---- phase R: forward row FFTs -> slot (column-major)
        prefetch(0, &tm.prow, 0, prow0, p.pol_keep);
        prefetch(1, &tm.prow, 0, prow0 + kTmaBatch, p.pol_keep);
        float2 pO[R];                                             // object row of the next batch
        {
            const float2 *orow = a.obj + (size_t)(pj.x + g) * M + pj.y;
#pragma unroll
            for (int m = 0; m < R; ++m) pO[m] = __ldg(orow + t + R * m);
        }
        for (int b = 0; b < NB; ++b) {
            const int s = b & 1;
            wait_stage(s);
            float2 *row = bin(s) + g * 256;
            float2 d[R];
#pragma unroll
            for (int m = 0; m < R; ++m) d[m] = cmul(row[t + R * m], pO[m]);
            if (b + 1 < NB) {
                const float2 *orow = a.obj + (size_t)(pj.x + kTmaBatch * (b + 1) + g) * M + pj.y;
#pragma unroll
                for (int m = 0; m < R; ++m) pO[m] = __ldg(orow + t + R * m);
            }
            pm::fft_group_xs<R, -1>(d, row, tw, t);
            barrier_a();
            if (failed) return tma_state(parity, failed, timed_out);
            if (b + 2 < NB) prefetch(s, &tm.prow, 0, prow0 + kTmaBatch * (b + 2), p.pol_keep);
            float2 *ob = bout + h * 4096;
#pragma unroll
            for (int m = 0; m < R; ++m) ob[T::swz128_index(t + R * m, gl)] = d[m];
            publish(&tm.slot_r, kTmaBatch * b, slot_col, 16, 0, p.pol_keep);
        }
        if (tid == 0) T::wait_all<0>();                          // slot complete before phase C reads it
        prefetch(0, &tm.slot_c, 0, slot_col, p.pol_stream);
        prefetch(1, &tm.slot_c, 0, slot_col + kTmaBatch, p.pol_stream);
        // ---- phase C: column FFTs (modulus replacement and inverse column FFTs in XM_FULL)
        for (int b = 0; b < NB; ++b) {
            const int s = b & 1;
            const int c = kTmaBatch * b + g;
            float A[R];                                           // A[k2] = |F psi| target at ky = t + 16 k2
            if constexpr (kFull) {
                const float4 *amp = reinterpret_cast<const float4 *>(a.amp + ((size_t)j * N + c) * N + t * R);
#pragma unroll
                for (int v = 0; v < R / 4; ++v) {
                    const float4 q = T::ldg_hint(amp + v, p.pol_stream);
                    A[4 * v] = q.x; A[4 * v + 1] = q.y; A[4 * v + 2] = q.z; A[4 * v + 3] = q.w;
                }
            }
            wait_stage(s);
            float2 *col = bin(s) + g * 256;
            float2 d[R];
#pragma unroll
            for (int m = 0; m < R; ++m) d[m] = col[t + R * m];
            pm::fft_group_xs<R, -1>(d, col, tw, t);
            if constexpr (kFull) {
                // d = N Psi (unnormalised transforms).  The projection A Psi / |Psi| does not
                // depend on the scale of Psi, and the inverse transform's 1/N is folded into the
                // projected amplitude, so neither unitary scaling costs a pass of its own.
#pragma unroll
                for (int m = 0; m < R; ++m) {
                    const float2 X = d[m];
                    const float mag2 = cabs2(X);
                    if (mag2 > 0.f) {
                        const float inv = rsqrtf(mag2);
                        const float dm = mag2 * inv * invN - A[m];
                        err += dm * dm;
                        d[m] = cscale(X, A[m] * invN * inv);
                    } else {
                        err += A[m] * A[m];
                        d[m] = make_float2(A[m] * invN, 0.f);
                    }
                }
                pm::fft_group_xs<R, +1>(d, col, tw, t);
            } else {
#pragma unroll
                for (int m = 0; m < R; ++m) d[m] = cscale(d[m], invN);
            }
            barrier_a();
            if (failed) return tma_state(parity, failed, timed_out);
            if (b + 2 < NB) prefetch(s, &tm.slot_c, 0, slot_col + kTmaBatch * (b + 2), p.pol_stream);
            float2 *ob = bout + h * 4096;
#pragma unroll
            for (int m = 0; m < R; ++m) ob[T::swz128_index(t + R * m, gl)] = d[m];
            publish(&tm.psi_c, kTmaBatch * b, u * N, 16, 0, p.pol_keep);
        }
    } else {
        // ---- phase C (XM_INV): inverse column FFTs of psi[j][m] in place
        auto load_psi_cols = [&](int s, int c0) {
            if (tid == 0) {
                *p.pending |= 1u << s;
                T::mbar_expect_tx(&bar[s], (uint32_t)kTmaBuf);
                T::load_2d(bin(s), &tm.psi_c, c0, u * N, &bar[s]);
                if constexpr (B == 32) T::load_2d(bin(s) + 4096, &tm.psi_c, c0 + 16, u * N, &bar[s]);
            }
        };
        if (tid == 0) T::wait_all<0>();
        load_psi_cols(0, 0);
        load_psi_cols(1, kTmaBatch);
        for (int b = 0; b < NB; ++b) {
            const int s = b & 1;
            wait_stage(s);
            float2 d[R];
            const float2 *colsw = bin(s) + h * 4096;
#pragma unroll
            for (int m = 0; m < R; ++m) d[m] = colsw[T::swz128_index(t + R * m, gl)];
            if (__syncthreads_or(timed_out)) failed = true;   // batch read: regions free
            if (failed) return tma_state(parity, failed, timed_out);
            pm::fft_group_xs<R, +1>(d, bin(s) + g * 256, tw, t);
            barrier_a();
            if (failed) return tma_state(parity, failed, timed_out);
            if (b + 2 < NB) load_psi_cols(s, kTmaBatch * (b + 2));
            float2 *ob = bout + h * 4096;
#pragma unroll
            for (int m = 0; m < R; ++m) ob[T::swz128_index(t + R * m, gl)] = d[m];
            publish(&tm.psi_c, kTmaBatch * b, u * N, 16, 0, p.pol_keep);
        }
    }
    if constexpr (XM != XM_FWD) {
        if (tid == 0) T::wait_all<0>();                          // psi columns complete before R'
        prefetch(0, &tm.psi_r, 0, u * N, p.pol_stream);
        prefetch(1, &tm.psi_r, 0, u * N + kTmaBatch, p.pol_stream);
        // ---- phase R': inverse row FFTs of psi[u] -> psi'
        for (int b = 0; b < NB; ++b) {
            const int s = b & 1;
            wait_stage(s);
            float2 *row = bin(s) + g * 256;
            float2 d[R];
#pragma unroll
            for (int m = 0; m < R; ++m) d[m] = row[t + R * m];
            pm::fft_group_xs<R, +1>(d, row, tw, t);
            barrier_a();
            if (failed) return tma_state(parity, failed, timed_out);
            if (b + 2 < NB) prefetch(s, &tm.psi_r, 0, u * N + kTmaBatch * (b + 2), p.pol_stream);
            if constexpr (kFull) {                               // 1/N already applied in phase C
#pragma unroll
                for (int m = 0; m < R; ++m) bout[g * 256 + t + R * m] = d[m];
            } else {
#pragma unroll
                for (int m = 0; m < R; ++m) bout[g * 256 + t + R * m] = cscale(d[m], invN);
            }
            publish(&tm.psi_w, 0, u * N + kTmaBatch * b, 0, 16, p.pol_stream);
        }
    }
    if constexpr (kFull) {
        double e = (double)err;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) e += __shfl_xor_sync(0xffffffffu, e, o);
        if ((tid & 31) == 0) p.s_red[tid >> 5] = e;
        __syncthreads();
        if (tid == 0) {
            double sum = 0.0;
            for (int w = 0; w < kTmaThreads / 32; ++w) sum += p.s_red[w];
            a.err[j] = sum;
        }
    }
    if (tid == 0) T::wait_all<0>();                              // psi[u] complete; buffers free for u + 1
    __syncthreads();
    return tma_state(parity, failed, timed_out);
}

__device__ __forceinline__ void tma_apply(TmaPipe &p, uint32_t st) {
    p.parity = st & 3u;
    p.failed = (st & 4u) != 0;
    p.timed_out = (st & 8u) != 0;
}

// Sets up the pipeline state (mbarriers, twiddles, policies); ends with a block barrier.
__device__ __forceinline__ void tma_pipe_init(TmaPipe &p, unsigned char *base, float2 *tw, uint64_t *bar,
                                              uint32_t *pending, double *s_red, int slot_col) {
    namespace T = pm::tma;
    const int tid = threadIdx.x;
    p.base = base;
    p.tw = tw;
    p.bar = bar;
    p.pending = pending;
    p.s_red = s_red;
    p.parity = 0u;
    p.failed = false;
    p.timed_out = false;
    p.slot_col = slot_col;
    p.pol_keep = T::policy_keep();
    p.pol_stream = T::policy_stream();
    for (int i = tid; i < 256; i += blockDim.x) {
        double sn, cs;
        sincospi(-2.0 * (double)((i >> 4) * (i & 15)) / 256.0, &sn, &cs);
        tw[i] = make_float2((float)cs, (float)sn);
    }
    if (tid == 0) {
        *pending = 0u;
        T::mbar_init(&bar[0], 1);
        T::mbar_init(&bar[1], 1);
        T::fence_barrier_init();
    }
    __syncthreads();
}

// Test hook (ptycho_debug_wait_timeout): a wait on a barrier that nothing arrives on, limited to
// ~2^20 cycles, before any copy is issued; the CTA then takes the timeout path.
__device__ __forceinline__ void tma_pipe_inject_wait(TmaPipe &p) {
    namespace T = pm::tma;
    if (threadIdx.x == 0) {
        T::mbar_init(&p.bar[2], 1);
        T::fence_barrier_init();
        if (!T::mbar_wait_for(&p.bar[2], 0u, 1ll << 20)) p.timed_out = true;
    }
    if (__syncthreads_or(p.timed_out)) p.failed = true;
}

// After a timeout: let every load still in flight land (bounded) before the CTA's shared memory
// is released, then drain the bulk stores and report.
__device__ __forceinline__ void tma_pipe_finish(TmaPipe &p, int *status) {
    namespace T = pm::tma;
    if (threadIdx.x == 0) {
#pragma unroll
        for (int s = 0; s < 2; ++s)
            if (p.failed && ((*p.pending >> s) & 1u)) T::mbar_wait(&p.bar[s], (p.parity >> s) & 1u);
        T::wait_all<0>();
        if (p.failed) atomicExch(status, 1);
    }
}

template <int B, int XM>
__global__ void __launch_bounds__(B * 16, 32 / B)
k_exit_wave_tma(TmaArgs a, const __grid_constant__ TmaMaps tm) {
    constexpr size_t kTmaBuf = tma_buf_bytes<B>();
    extern __shared__ unsigned char smem_raw[];
    unsigned char *base = (unsigned char *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    __shared__ double s_red[B * 16 / 32];
    __shared__ uint32_t s_pending;
    TmaPipe p;
    tma_pipe_init(p, base, (float2 *)(base + 3 * kTmaBuf), (uint64_t *)(base + 3 * kTmaBuf + 256 * sizeof(float2)),
                  &s_pending, s_red, blockIdx.x * 256);
    constexpr bool kFull = (XM == XM_FULL || XM == XM_LIST);
    const int units = (XM == XM_LIST) ? a.count : (kFull ? a.J : a.J * a.Q);
    if (a.inject_wait) tma_pipe_inject_wait(p);
    for (int iu = blockIdx.x; iu < units && !p.failed; iu += gridDim.x)
        tma_apply(p, tma_unit<B, XM>(p, a, tm, (XM == XM_LIST) ? a.list[iu] : iu));
    tma_pipe_finish(p, a.status);
}

