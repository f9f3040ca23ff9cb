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
    int inject_wait;         // test hook: 1 = wait on a barrier nothing arrives on (short limit)
                             // first; 2 = part 0 of every split tail unit skips its first arrival
    const uint4 *gmat;       // tensor-core form: the split 64-point DFT matrix (64 KB, global)
    // Tail split (XM_FULL without a list): the first launch takes units [0, tail_base); a second,
    // cooperative launch shares each unit tail_base .. J-1 among `split` consecutive CTAs, part q
    // taking batches [q NB / split, (q + 1) NB / split) of every phase, with two hand-offs
    // through tail_sync[unit - tail_base] (zeroed before that launch); the parts' per-batch error
    // sums meet in tail_err[(unit - tail_base) * 16 + batch].  Unsplit: tail_base = J.
    int split, tail_base;
    int *tail_sync;
    double *tail_err;
    // XM_INV (mixed state): if not NULL, the mode-summed modulus constraint's per-pixel scale
    // A / sqrt(sum_m |Psi_m|^2), [J][N][N] in the amplitude order (column kx, then thread t's rows
    // t + 16 k2 contiguous); each loaded spectrum is multiplied by it before the inverse FFTs
    const float *fscale;
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
    // tensor-core form only
    unsigned char *gs;       // the split DFT matrix in shared memory (G_hi, G_lo)
    unsigned char *op;       // operand of one pass (B_hi, B_lo: 64 rows x 128 K each)
    uint32_t tmem;           // 64 FP32 accumulator columns
    uint32_t mphase;         // phase parity of the MMA barrier bar[3]
    float2 twq[3];           // W_256^(q u), q = 1, 2, 3, for this thread's accumulator lane u
};

// ---------------------------------------------------------------------------------------
// Tensor-core 256-point DFT of the 16 vectors of one stage buffer (the fft_path DFTGEMM form
// at N = 256), in place, by 256 threads.  256 = 4 x 64: the 64-point DFTs of the four decimated
// sub-sequences x[4 r + q] are one split-BF16 GEMM against the resident 64-point matrix (operand
// row 4 v + q, K index 2 r + s; accumulator lane 2 u + s', column 4 v + q holds part s' of
// E_q[u]); the epilogue combines them with a radix-4 step,
//   X[u + 64 m] = sum_q (-i)^(q m) W_256^(q u) E_q[u],
// lane pairs (s' = 0, 1) exchanging their halves with one shuffle per value.  The inverse is
// the forward transform by conjugation (unnormalised, like the radix path).  Returns false
// (uniformly) when the MMA completion wait gave up.
__device__ __forceinline__ bool tc_dft256(float2 *buf, bool inverse, const TmaPipe &p, uint32_t &mphase) {
    namespace T = pm::tma;
    const int tid = threadIdx.x;
    {
        const int v = tid >> 4, t = tid & 15, q = t & 3;
        unsigned char *oh = p.op, *ol = p.op + 16384;
#pragma unroll 4
        for (int sI = 0; sI < 16; ++sI) {
            const int e = 16 * sI + t;                            // element of vector v
            float2 z = buf[v * 256 + e];
            if (inverse) z.y = -z.y;
            uint32_t hw, lw;
            pm::tc::split2(z, hw, lw);
            const uint32_t off = pm::tc::core_offset(4 * v + q, 2 * (e >> 2), 128);
            *reinterpret_cast<uint32_t *>(oh + off) = hw;
            *reinterpret_cast<uint32_t *>(ol + off) = lw;
        }
    }
    T::fence_async_smem();                                        // operand writes -> tensor core
    pm::tc::fence_before();
    __syncthreads();
    if (tid == 0) {
        pm::tc::fence_after();
        constexpr uint32_t idesc = pm::tc::idesc_bf16_f32(128, 64);
        const uint32_t gh = pm::tc::smem_addr(p.gs), gl = gh + 32768;
        const uint32_t bh = pm::tc::smem_addr(p.op), bl = bh + 16384;
#pragma unroll
        for (int term = 0; term < 3; ++term) {                    // hi hi, hi lo, lo hi
            const uint32_t ab = (term == 2) ? gl : gh, bb = (term == 1) ? bl : bh;
#pragma unroll
            for (int ks = 0; ks < 8; ++ks)
                pm::tc::mma_bf16(p.tmem, pm::tc::smem_desc(ab + ks * 256, 128, 2048),
                                 pm::tc::smem_desc(bb + ks * 256, 128, 2048), idesc, (uint32_t)((term | ks) != 0));
        }
        pm::tc::commit(&p.bar[3]);
    }
    const bool ok = T::mbar_wait(&p.bar[3], mphase);
    if (__syncthreads_or(!ok)) return false;                      // the MMAs are drained at the end
    mphase ^= 1u;
    pm::tc::fence_after();
    const int w = tid >> 5, lane = tid & 31, lq = w & 3, ch = w >> 2;
    const int u = 16 * lq + (lane >> 1), part = lane & 1;
    uint32_t r[32];
    pm::tc::ld_32cols(p.tmem + ((uint32_t)(32 * lq) << 16) + (uint32_t)(32 * ch), r);
    pm::tc::wait_ld();
#pragma unroll
    for (int vv = 0; vv < 8; ++vv) {
        float2 E[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const float a = __uint_as_float(r[4 * vv + q]);
            const float y = __shfl_xor_sync(0xffffffffu, a, 1);
            E[q] = part ? make_float2(y, a) : make_float2(a, y);
        }
        const float2 Y1 = cmul(p.twq[0], E[1]), Y2 = cmul(p.twq[1], E[2]), Y3 = cmul(p.twq[2], E[3]);
        const float2 A0 = cadd(E[0], Y2), A1 = csub(E[0], Y2), B0 = cadd(Y1, Y3), B1 = csub(Y1, Y3);
        const float2 mB1 = make_float2(B1.y, -B1.x);              // -i B1
        float2 X0, X1;
        if (part == 0) { X0 = cadd(A0, B0); X1 = cadd(A1, mB1); }  // m = 0, 1
        else { X0 = csub(A0, B0); X1 = csub(A1, mB1); }            // m = 2, 3
        if (inverse) { X0.y = -X0.y; X1.y = -X1.y; }
        float2 *o = buf + (8 * ch + vv) * 256 + u + 128 * part;
        o[0] = X0;
        o[64] = X1;
    }
    pm::tc::fence_before();
    __syncthreads();                                              // buffer complete, TMEM read
    return true;
}

// Every copy carries an L2 cache policy: the probe rows, the slot and the intermediate psi
// columns (re-read by this CTA within the position) are kept, data read for the last time and
// the final psi_j' rows are evicted first (measured at lab scale: DRAM traffic 2.47 -> 1.24 MB per
// position with B = 32).  One unit: position j (or (j, m) for the mixed-state forms).  After a
// wait gives up the unit returns with p.failed set (uniformly) before waiting again, so the parity
// of a stage whose wait failed stays that of the load still in flight (tma_pipe_finish drains it).
// Hand-off between the CTAs sharing a tail unit (thread 0; its bulk stores of the phase have
// completed): release one arrival on the counter, then wait (bounded, ~1 s) until `target`
// arrivals, with async-proxy fences on both sides so that the partners' TMA stores are seen by
// this CTA's TMA loads.  Returns false when the wait gave up.
// skip_arrival (test hook only): wait without arriving, so that the partners' waits run out.
__device__ __forceinline__ bool tail_handoff(int *ctr, int target, bool skip_arrival = false) {
    asm volatile("fence.proxy.async.global;" ::: "memory");
    if (!skip_arrival) asm volatile("red.release.gpu.global.add.s32 [%0], 1;" ::"l"(ctr) : "memory");
    const long long start = clock64();
    for (uint32_t i = 0; i < (1u << 26); ++i) {
        int v;
        asm volatile("ld.acquire.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(ctr) : "memory");
        if (v >= target) {
            asm volatile("fence.proxy.async.global;" ::: "memory");
            return true;
        }
        if (clock64() - start > (1ll << 31)) break;
        __nanosleep(64);
    }
    return false;
}

// Returns the updated mutable state: bits 0-1 parity, bit 2 failed, bit 3 timed out, bit 4 the
// MMA barrier's phase parity (tensor-core form).
__host__ __device__ constexpr uint32_t tma_state(uint32_t parity, bool failed, bool timed_out, uint32_t mphase = 0) {
    return parity | (failed ? 4u : 0u) | (timed_out ? 8u : 0u) | (mphase << 4);
}

// TC: the 256-point transforms on the tensor cores (tc_dft256) instead of the FP32 radix FFT;
// 16-row stages, one-mode XM_FULL only.
// SPLIT: part q of S of a tail unit (the CTAs blockIdx / S of the tail launch share it; its slot
// at slot_override); otherwise the whole unit with a compile-time batch range.  The Fourier error is summed per batch (warps in order, then
// batches in order), so a split and an unsplit unit give the same error bit for bit.
template <int B, int XM, bool TC = false, bool SPLIT = false>
__device__ __forceinline__ uint32_t tma_unit(const TmaPipe &p, const TmaArgs &a, const TmaMaps &tm, int u,
                                             int q = 0, int S = 1, int slot_override = -1) {
    static_assert(!TC || (B == 16 && XM == XM_FULL), "tensor-core form: 16-row stages, XM_FULL");
    constexpr int R = 16, N = 256, NB = N / B;
    constexpr int kTmaThreads = B * 16, kTmaBatch = B;
    constexpr size_t kTmaBuf = tma_buf_bytes<B>();
    constexpr bool kFull = (XM == XM_FULL || XM == XM_LIST);
    namespace T = pm::tma;
    const int tid = threadIdx.x;
    // group g = one 256-point vector, thread t of 16 (g in [0, B)).  A warp holds groups 2w and
    // 2w + 1, interleaved by eights: lanes 0-7 and 24-31 are group 2w (t = 0-7, 8-15), lanes
    // 8-23 group 2w + 1 (t = 8-15, 0-7).  Each half-warp then holds t = 0-7 of one group and
    // t = 8-15 of the other, so its 8-byte accesses to the two vectors' rows (2 KB apart, the
    // same banks), to the exchange and to the 128-byte-swizzled staging (rows t and t + 8 share
    // a swizzle phase) fall on 16 distinct bank pairs.
    const int t = tid & 15, g = (tid >> 4) ^ ((tid >> 3) & 1);
    const int h = g >> 4, gl = g & 15;                           // 16-wide box of the batch, row in it
    auto bin = [&](int s) { return (float2 *)(p.base + s * kTmaBuf); };
    float2 *bout = (float2 *)(p.base + 2 * kTmaBuf);
    const float2 *tw = p.tw;
    uint64_t *bar = p.bar;
    const float invN = 1.0f / (float)N;
    const int M = a.M;
    uint32_t parity = p.parity, mphase = p.mphase;
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
    const int slot_col = slot_override >= 0 ? slot_override : p.slot_col;
    const int j = kFull ? u : u / a.Q;
    const int prow0 = kFull ? 0 : (u % a.Q) * N;                  // first probe row of the mode
    const int b0 = SPLIT ? q * (NB / S) : 0, b1 = SPLIT ? b0 + NB / S : NB;   // this part's batches
    // (only b0 and b1 stay live: the split, its factor and the tail index are derived from them)
    auto parts = [&]() { return NB / (b1 - b0); };
    auto tail_index = [&]() { return (int)blockIdx.x / parts(); };
    double *s_wsum = p.s_red;                                     // [2][32] warp sums, by batch parity
    double *s_berr = p.s_red + 64;                                // [NB] per-batch error sums
    // per-batch error: warp sums in FP32, then the batch's sum over warps in order (double)
    auto batch_error = [&](float eb, int b) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) eb += __shfl_xor_sync(0xffffffffu, eb, o);
        if ((tid & 31) == 0) s_wsum[(b & 1) * 32 + (tid >> 5)] = (double)eb;
    };
    auto batch_error_sum = [&](int b) {                           // thread 0, after a block barrier
        double e = 0.0;
        for (int w = 0; w < kTmaThreads / 32; ++w) e += s_wsum[(b & 1) * 32 + w];
        s_berr[b] = e;
    };
    auto handoff = [&](int target) {                              // every thread; uniform result
        bool ok = true;
        if (tid == 0)
            ok = tail_handoff(a.tail_sync + tail_index(), target, a.inject_wait == 2 && b0 == 0 && target == parts());
        if (__syncthreads_or(!ok)) failed = true;
    };
    if constexpr (XM != XM_INV) {
        const int2 pj = a.pos[j];
        // ---- phase R: forward row FFTs -> slot (column-major)
        prefetch(0, &tm.prow, 0, prow0 + kTmaBatch * b0, p.pol_keep);
        prefetch(1, &tm.prow, 0, prow0 + kTmaBatch * (b0 + 1), p.pol_keep);
        float2 pO[R];                                             // object row of the next batch
        {
            const float2 *orow = a.obj + (size_t)(pj.x + kTmaBatch * b0 + g) * M + pj.y;
#pragma unroll
            for (int m = 0; m < R; ++m) pO[m] = __ldg(orow + t + R * m);
        }
        for (int b = b0; b < b1; ++b) {
            const int s = b & 1;
            wait_stage(s);
            float2 *row = bin(s) + g * 256;
            float2 d[R];
#pragma unroll
            for (int m = 0; m < R; ++m) d[m] = cmul(row[t + R * m], pO[m]);
            if (b + 1 < b1) {
                const float2 *orow = a.obj + (size_t)(pj.x + kTmaBatch * (b + 1) + g) * M + pj.y;
#pragma unroll
                for (int m = 0; m < R; ++m) pO[m] = __ldg(orow + t + R * m);
            }
            if constexpr (TC) {
#pragma unroll
                for (int m = 0; m < R; ++m) row[t + R * m] = d[m];
                __syncthreads();
                if (!tc_dft256(bin(s), false, p, mphase)) failed = true;
                else {
#pragma unroll
                    for (int m = 0; m < R; ++m) d[m] = row[t + R * m];
                }
            } else {
                pm::fft_group_xs<R, -1>(d, row, tw, t);
            }
            barrier_a();
            if (failed) return tma_state(parity, failed, timed_out, mphase);
            if (b + 2 < b1) prefetch(s, &tm.prow, 0, prow0 + kTmaBatch * (b + 2), p.pol_keep);
            float2 *ob = bout + h * 4096;
#pragma unroll
            for (int m = 0; m < R; ++m) ob[T::swz128_index(t + R * m, gl)] = d[m];
            publish(&tm.slot_r, kTmaBatch * b, slot_col, 16, 0, p.pol_keep);
        }
        if (tid == 0) T::wait_all<0>();                          // slot complete before phase C reads it
        if (b1 - b0 < NB) {
            handoff(parts());                                    // every part's rows are in the slot
            if (failed) return tma_state(parity, failed, timed_out, mphase);
        }
        prefetch(0, &tm.slot_c, 0, slot_col + kTmaBatch * b0, p.pol_stream);
        prefetch(1, &tm.slot_c, 0, slot_col + kTmaBatch * (b0 + 1), p.pol_stream);
        // ---- phase C: column FFTs (modulus replacement and inverse column FFTs in XM_FULL)
        float4 An[R / 4];                                         // amplitudes of the next column
        if constexpr (kFull) {
            const float4 *amp = reinterpret_cast<const float4 *>(a.amp + ((size_t)j * N + kTmaBatch * b0 + g) * N + t * R);
#pragma unroll
            for (int v = 0; v < R / 4; ++v) An[v] = T::ldg_hint(amp + v, p.pol_stream);
        }
        for (int b = b0; b < b1; ++b) {
            const int s = b & 1;
            const int c = kTmaBatch * b + g;
            float A[R];                                           // A[k2] = |F psi| target at ky = t + 16 k2
            if constexpr (kFull) {
#pragma unroll
                for (int v = 0; v < R / 4; ++v) {
                    A[4 * v] = An[v].x; A[4 * v + 1] = An[v].y; A[4 * v + 2] = An[v].z; A[4 * v + 3] = An[v].w;
                }
                if (b + 1 < b1) {
                    const float4 *amp =
                        reinterpret_cast<const float4 *>(a.amp + ((size_t)j * N + c + kTmaBatch) * N + t * R);
#pragma unroll
                    for (int v = 0; v < R / 4; ++v) An[v] = T::ldg_hint(amp + v, p.pol_stream);
                }
            }
            wait_stage(s);
            float2 *col = bin(s) + g * 256;
            float2 d[R];
            if constexpr (TC) {
                if (__syncthreads_or(timed_out)) failed = true;           // stage arrived everywhere
                if (failed || !tc_dft256(bin(s), false, p, mphase)) {
                    failed = true;
                    return tma_state(parity, failed, timed_out, mphase);
                }
            }
#pragma unroll
            for (int m = 0; m < R; ++m) d[m] = col[t + R * m];
            if constexpr (!TC) pm::fft_group_xs<R, -1>(d, col, tw, t);
            if constexpr (kFull) {
                // d = N Psi (unnormalised transforms).  The projection A Psi / |Psi| does not
                // depend on the scale of Psi, and the inverse transform's 1/N is folded into the
                // projected amplitude, so neither unitary scaling costs a pass of its own.
                float eb = 0.f;
#pragma unroll
                for (int m = 0; m < R; ++m) {
                    const float2 X = d[m];
                    const float mag2 = cabs2(X);
                    if (mag2 > 0.f) {
                        const float inv = rsqrtf(mag2);
                        const float dm = mag2 * inv * invN - A[m];
                        eb += dm * dm;
                        d[m] = cscale(X, A[m] * invN * inv);
                    } else {
                        eb += A[m] * A[m];
                        d[m] = make_float2(A[m] * invN, 0.f);
                    }
                }
                batch_error(eb, b);
                if constexpr (TC) {
#pragma unroll
                    for (int m = 0; m < R; ++m) col[t + R * m] = d[m];
                    __syncthreads();
                    if (!tc_dft256(bin(s), true, p, mphase)) failed = true;
                    else {
#pragma unroll
                        for (int m = 0; m < R; ++m) d[m] = col[t + R * m];
                    }
                } else {
                    pm::fft_group_xs<R, +1>(d, col, tw, t);
                }
            } else {
#pragma unroll
                for (int m = 0; m < R; ++m) d[m] = cscale(d[m], invN);
            }
            barrier_a();
            if (failed) return tma_state(parity, failed, timed_out, mphase);
            if (kFull && tid == 0) batch_error_sum(b);
            if (b + 2 < b1) prefetch(s, &tm.slot_c, 0, slot_col + kTmaBatch * (b + 2), p.pol_stream);
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
        // the modulus scales of the next column (one column batch ahead, like the amplitudes)
        const float *fs_j = a.fscale ? a.fscale + (size_t)j * N * N : nullptr;
        float4 Fn[R / 4];
        if (fs_j) {
            const float4 *f = reinterpret_cast<const float4 *>(fs_j + (size_t)g * N + t * R);
#pragma unroll
            for (int v = 0; v < R / 4; ++v) Fn[v] = T::ldg_hint(f + v, p.pol_keep);
        }
        for (int b = 0; b < NB; ++b) {
            const int s = b & 1;
            wait_stage(s);
            float2 d[R];
            const float2 *colsw = bin(s) + h * 4096;
#pragma unroll
            for (int m = 0; m < R; ++m) d[m] = colsw[T::swz128_index(t + R * m, gl)];
            if (fs_j) {
                const float F[R] = {Fn[0].x, Fn[0].y, Fn[0].z, Fn[0].w, Fn[1].x, Fn[1].y, Fn[1].z, Fn[1].w,
                                    Fn[2].x, Fn[2].y, Fn[2].z, Fn[2].w, Fn[3].x, Fn[3].y, Fn[3].z, Fn[3].w};
                if (b + 1 < NB) {
                    const float4 *f =
                        reinterpret_cast<const float4 *>(fs_j + (size_t)(kTmaBatch * (b + 1) + g) * N + t * R);
#pragma unroll
                    for (int v = 0; v < R / 4; ++v) Fn[v] = T::ldg_hint(f + v, p.pol_keep);
                }
#pragma unroll
                for (int m = 0; m < R; ++m) d[m] = cscale(d[m], F[m]);
            }
            if (__syncthreads_or(timed_out)) failed = true;   // batch read: regions free
            if (failed) return tma_state(parity, failed, timed_out, mphase);
            pm::fft_group_xs<R, +1>(d, bin(s) + g * 256, tw, t);
            barrier_a();
            if (failed) return tma_state(parity, failed, timed_out, mphase);
            if (b + 2 < NB) load_psi_cols(s, kTmaBatch * (b + 2));
            float2 *ob = bout + h * 4096;
#pragma unroll
            for (int m = 0; m < R; ++m) ob[T::swz128_index(t + R * m, gl)] = d[m];
            publish(&tm.psi_c, kTmaBatch * b, u * N, 16, 0, p.pol_keep);
        }
    }
    if constexpr (XM != XM_FWD) {
        if (tid == 0) T::wait_all<0>();                          // psi columns complete before R'
        if (b1 - b0 < NB) {
            if (kFull && tid == 0)
                for (int b = b0; b < b1; ++b) a.tail_err[tail_index() * 16 + b] = s_berr[b];
            handoff(2 * parts());                                // every part's columns are in psi
            if (failed) return tma_state(parity, failed, timed_out, mphase);
            if (kFull && b0 == 0 && tid == 0)
                for (int b = 0; b < NB; ++b)
                    if (b >= b1) s_berr[b] = __ldcg(a.tail_err + tail_index() * 16 + b);
        }
        prefetch(0, &tm.psi_r, 0, u * N + kTmaBatch * b0, p.pol_stream);
        prefetch(1, &tm.psi_r, 0, u * N + kTmaBatch * (b0 + 1), p.pol_stream);
        // ---- phase R': inverse row FFTs of psi[u] -> psi'
        for (int b = b0; b < b1; ++b) {
            const int s = b & 1;
            wait_stage(s);
            float2 *row = bin(s) + g * 256;
            float2 d[R];
            if constexpr (TC) {
                if (__syncthreads_or(timed_out)) failed = true;
                if (failed || !tc_dft256(bin(s), true, p, mphase)) {
                    failed = true;
                    return tma_state(parity, failed, timed_out, mphase);
                }
            }
#pragma unroll
            for (int m = 0; m < R; ++m) d[m] = row[t + R * m];
            if constexpr (!TC) pm::fft_group_xs<R, +1>(d, row, tw, t);
            barrier_a();
            if (failed) return tma_state(parity, failed, timed_out, mphase);
            if (b + 2 < b1) prefetch(s, &tm.psi_r, 0, u * N + kTmaBatch * (b + 2), p.pol_stream);
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
        if (b0 == 0 && tid == 0) {
            double sum = 0.0;
            for (int b = 0; b < NB; ++b) sum += s_berr[b];
            a.err[j] = sum;
        }
    }
    if (tid == 0) T::wait_all<0>();                              // psi[u] complete; buffers free for u + 1
    __syncthreads();
    return tma_state(parity, failed, timed_out, mphase);
}

__device__ __forceinline__ void tma_apply(TmaPipe &p, uint32_t st) {
    p.parity = st & 3u;
    p.failed = (st & 4u) != 0;
    p.timed_out = (st & 8u) != 0;
    p.mphase = (st >> 4) & 1u;
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
    p.gs = nullptr;
    p.op = nullptr;
    p.tmem = 0;
    p.mphase = 0;
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

// Dynamic shared memory of the kernel: stages, staging, twiddles, barriers; the tensor-core
// form adds the split DFT matrix (64 KB) and one pass's operand (32 KB).
template <int B, bool TC>
__host__ __device__ constexpr size_t tma_kernel_smem() {
    return tma_smem_bytes<B>() + (TC ? (size_t)1024 + 65536 + 32768 : 0);
}

// TAIL = false: the units [0, tail_base) (all of them unless the tail is split), persistent,
// one CTA per unit.  TAIL = true (XM_FULL, a separate launch after it, cooperative, split CTAs
// per tail unit): CTA c takes part c mod split of unit tail_base + c / split, in the slot of
// CTA (c / split) * split, which the finished first launch no longer uses.
template <int B, int XM, bool TC = false, bool TAIL = false>
__global__ void __launch_bounds__(B * 16, TC ? 1 : 32 / B)
k_exit_wave_tma(TmaArgs a, const __grid_constant__ TmaMaps tm) {
    constexpr size_t kTmaBuf = tma_buf_bytes<B>();
    extern __shared__ unsigned char smem_raw[];
    unsigned char *base = (unsigned char *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    __shared__ double s_red[96];                  // warp sums [2][32], per-batch error sums [NB]
    __shared__ uint32_t s_pending;
    __shared__ uint32_t s_tmem;
    TmaPipe p;
    if constexpr (TC) {
        // split DFT matrix into shared memory, TMEM for the accumulators, per-lane radix-4 twiddles
        unsigned char *gs = base + 3 * kTmaBuf + 256 * sizeof(float2) + 1024;
        for (int i = threadIdx.x; i < 65536 / 16; i += blockDim.x) reinterpret_cast<uint4 *>(gs)[i] = a.gmat[i];
        if (threadIdx.x < 32) pm::tc::alloc(&s_tmem, 64);
    }
    tma_pipe_init(p, base, (float2 *)(base + 3 * kTmaBuf), (uint64_t *)(base + 3 * kTmaBuf + 256 * sizeof(float2)),
                  &s_pending, s_red, blockIdx.x * 256);
    if constexpr (TC) {
        p.gs = base + 3 * kTmaBuf + 256 * sizeof(float2) + 1024;
        p.op = p.gs + 65536;
        if (threadIdx.x == 0) {
            pm::tma::mbar_init(&p.bar[3], 1);
            pm::tma::fence_barrier_init();
        }
        pm::tc::fence_before();
        __syncthreads();
        pm::tc::fence_after();
        p.tmem = s_tmem;
        const int u = 16 * ((threadIdx.x >> 5) & 3) + ((threadIdx.x & 31) >> 1);
#pragma unroll
        for (int q = 1; q < 4; ++q) {
            double sn, cs;
            sincospi(-2.0 * (double)(q * u) / 256.0, &sn, &cs);
            p.twq[q - 1] = make_float2((float)cs, (float)sn);
        }
    }
    constexpr bool kFull = (XM == XM_FULL || XM == XM_LIST);
    const int units = (XM == XM_LIST) ? a.count : (kFull ? a.J : a.J * a.Q);
    if (a.inject_wait == 1) tma_pipe_inject_wait(p);
    if constexpr (TAIL) {
        static_assert(XM == XM_FULL, "split tails: XM_FULL only");
        const int ti = (int)blockIdx.x / a.split;
        if (!p.failed && a.tail_base + ti < units)
            tma_apply(p, tma_unit<B, XM, TC, true>(p, a, tm, a.tail_base + ti, (int)blockIdx.x % a.split, a.split,
                                                   ti * a.split * 256));
    } else {
        const int nunits = (XM == XM_FULL && a.list == nullptr) ? a.tail_base : units;
        for (int iu = blockIdx.x; iu < nunits && !p.failed; iu += gridDim.x)
            tma_apply(p, tma_unit<B, XM, TC>(p, a, tm, (XM == XM_LIST) ? a.list[iu] : iu));
    }
    tma_pipe_finish(p, a.status);
    if constexpr (TC) {
        // an MMA whose completion wait gave up may still be running: wait once more (bounded),
        // then release the TMEM columns
        if (p.failed && threadIdx.x == 0) pm::tma::mbar_wait(&p.bar[3], p.mphase);
        pm::tc::fence_before();
        __syncthreads();
        if (threadIdx.x < 32) {
            pm::tc::fence_after();
            pm::tc::dealloc(p.tmem, 64);
        }
    }
}
