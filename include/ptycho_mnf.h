/*
 * ptycho_mnf.h -- C ABI of the B300 (sm_103a) library for Multi-Scale Non-Linear Fusion of
 * multi-exposure diffraction stacks and the iterative ptychographic reconstruction that
 * consumes the fused patterns.
 *
 * Conventions shared by every entry point
 *   - Every int-returning call returns PTYCHO_OK (0) or a negative PTYCHO_E* code; the message
 *     of the last failure on the calling host thread is ptycho_last_error() (library-owned,
 *     valid until the next failing call on that thread).
 *   - Invalid arguments are rejected before any device work or allocation (PTYCHO_EINVAL).
 *   - "device" pointers are CUDA device addresses on the current device; "host" pointers are
 *     ordinary host memory.  Caller-owned buffers stay caller-owned; the library never frees
 *     them and never keeps them past the call (it copies what it needs).
 *   - cuda_stream is a cudaStream_t (NULL = legacy default stream).  All device work of a call
 *     is enqueued on that stream; calls return without waiting unless stated otherwise.
 *   - Complex numbers are interleaved (re, im) float32 pairs ("complex64"), row-major arrays.
 *   - Detector patterns are stored with their DC term at the array centre (index N/2, N/2).
 */
#ifndef PTYCHO_MNF_H
#define PTYCHO_MNF_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
    PTYCHO_OK = 0,
    PTYCHO_EINVAL = -1,     /* bad argument (sizes, ranges, NULL pointers) */
    PTYCHO_ENOMEM = -2,     /* a device allocation failed */
    PTYCHO_ECUDA = -3,      /* a CUDA call failed; the CUDA error string is in the message */
    PTYCHO_ENONFINITE = -4, /* the reconstruction error became NaN or Inf */
    PTYCHO_ETIMEDOUT = -5   /* a bounded device wait gave up */
};

/* Base layer of the per-exposure collapse (§3.4.4): the paper propagates the base from the
 * Gaussian pyramid without weight modulation.  MEAN = G_{L-1}[E_k] / K (default), SUM =
 * G_{L-1}[E_k] (Eq. 10 literally), WEIGHTED = G_{L-1}[W_k] * G_{L-1}[E_k]. */
enum { PTYCHO_BASE_MEAN = 0, PTYCHO_BASE_SUM = 1, PTYCHO_BASE_WEIGHTED = 2 };

/* Pyramid input domain: RADIANCE = I_k * t_max / t_k (default), RAW = I_k as recorded. */
enum { PTYCHO_DOMAIN_RADIANCE = 0, PTYCHO_DOMAIN_RAW = 1 };

typedef struct {
    float mu;          /* centre of the exposure-quality curve, Eq. 5 (default 0.5)        */
    float sigma;       /* width of the exposure-quality curve, Eq. 5 (default 0.2), > 0     */
    int levels;        /* pyramid levels L (§3.4.2), >= 1, with N / 2^(L-1) >= 4            */
    float delta0;      /* quantiser step of the finest level, Eq. 8; 0 disables quantising */
    float delta_ratio; /* Delta_l = delta0 * delta_ratio^l (l = 0 finest), > 0             */
    float clip;        /* detector full scale in counts; Ibar = min(I, clip) / clip, > 0    */
    int base_mode;     /* PTYCHO_BASE_*                                                     */
    int domain;        /* PTYCHO_DOMAIN_*                                                   */
} fuse_params;

/*
 * fuse_stack -- Multi-Scale Non-Linear Fusion of every position's exposure bracket
 * (§3.4: Eq. 5 weights normalised to sum 1, Eq. 6 Gaussian and Eq. 7 Laplacian pyramids,
 * modulation and Eq. 8 quantisation, Eq. 9 per-exposure collapse, Eq. 10 sum over k).
 *
 *   d_raw    device, uint16 counts [J][K][N][N] (the bracket S_j of Eq. 1), read-only
 *   J        positions, >= 0 (0 is a no-op)
 *   K        exposures per position, 1 <= K <= 8
 *   N        detector side, a power of two, 8 <= N <= 1024
 *   h_t      host, [K] exposure times t_k > 0 (only their ratios matter)
 *   p        host, fusion parameters (see fuse_params)
 *   d_fused  device, float32 [J][N][N] output I_MNF (DC-centred like the input), caller-owned
 *   cuda_stream  stream for all work
 * Scratch: the call takes stream-ordered device scratch (about 4 (2K + 1) N^2 / 3 bytes per
 * position) and releases it on the same stream.  Returns PTYCHO_EINVAL for bad sizes or
 * parameters, PTYCHO_ENOMEM / PTYCHO_ECUDA on device failures.  Asynchronous.
 */
int fuse_stack(const uint16_t *d_raw, int J, int K, int N, const float *h_t,
               const fuse_params *p, float *d_fused, void *cuda_stream);

/*
 * fuse_stack_noalloc -- the same fusion as fuse_stack, for callers that cannot allocate device
 * memory (for example while another framework's caching allocator holds nearly all of it, or
 * inside a latency-critical loop where an allocation, which can synchronise the device, is
 * not acceptable).  The paper has no counterpart: this is a deployment variant of the
 * library.  Arguments, layouts and results are those of fuse_stack.
 *   - Scratch lives in a 16 MiB array compiled into the library: every GPU that loads the
 *     library holds it until the process exits.  The call allocates and frees nothing.
 *   - Positions are processed in chunks that fit the array; a configuration whose single
 *     position needs more than 16 MiB of scratch (about 4 (2K + 1) N^2 / 3 bytes) is rejected
 *     with PTYCHO_EINVAL and a message naming the sizes.
 *   - A call on a stream that is not being captured looks up the array's device address for
 *     the current device (and context); a captured call reuses the address found by the
 *     device's last uncaptured call.  So make one uncaptured call on a device before any
 *     stream capture, and again after a cudaDeviceReset (which invalidates the address).
 *   - All calls share the array: calls whose work may overlap on the GPU (different streams,
 *     other host threads) race on it and must be serialised by the caller.
 */
int fuse_stack_noalloc(const uint16_t *d_raw, int J, int K, int N, const float *h_t,
                       const fuse_params *p, float *d_fused, void *cuda_stream);

/*
 * fuse_stack_host -- fuse_stack for a stack that is still in host memory: the same fusion and
 * results (bit for bit), with the host-to-device copy overlapped with the fusion.  Positions
 * are copied in chunks on a copy stream of the library (one per device, created by the first
 * call) and each chunk is fused on cuda_stream as soon as it has landed, so the copy of one
 * chunk runs under the fusion of the previous one.  The paper has no counterpart: this is a
 * deployment variant of the library for data arriving from the host.
 *   h_raw            host, uint16 [J][K][N][N], read-only, caller-owned; page-locked (pinned)
 *                    memory is needed for the copies to overlap the fusion (pageable memory
 *                    works, with copies that do not overlap)
 *   d_raw            device, uint16 [J][K][N][N], caller-owned staging buffer, overwritten
 *   chunk_positions  positions per chunk, > 0; 0 = J / 8 (eight chunks)
 *   others           as fuse_stack
 * Ordering: the copies start after the work already queued on cuda_stream (d_raw may still be
 * in use), and work queued on cuda_stream after the call runs after every copy and the whole
 * fusion.  h_raw must stay valid and unchanged until then.  Asynchronous.
 */
int fuse_stack_host(const uint16_t *h_raw, uint16_t *d_raw, int J, int K, int N, const float *h_t,
                    const fuse_params *p, float *d_fused, int chunk_positions, void *cuda_stream);

/*
 * fuse_sli -- Standard Linear Integration, the linear HDR comparator the paper evaluates MNF
 * against (§1, §2.2, "SLI"): per pixel t_max * sum_{k: I_k < clip} I_k / sum_{k: I_k < clip} t_k
 * (count rate over the unsaturated exposures, in longest-exposure units); a pixel saturated in
 * every exposure takes the shortest exposure's clipped rate.  Same raw / output layouts as
 * fuse_stack, any N in [1, 4096], 1 <= K <= 8.  Allocates nothing.  Asynchronous.
 */
int fuse_sli(const uint16_t *d_raw, int J, int K, int N, const float *h_t, float clip, float *d_fused,
             void *cuda_stream);

/*
 * dft2_split_bf16 -- batch of unitary 2-D DFTs (the F of Eq. 3; inverse = F^-1) computed on the
 * tensor cores as split-BF16 (3-term) DFT-by-GEMM with FP32 accumulation: every operand x is
 * split into hi = bf16(x) and lo = bf16(x - hi), and each real GEMM takes
 * G_hi B_hi + G_hi B_lo + G_lo B_hi (the lo x lo term is dropped).  The paper prescribes no
 * FFT algorithm; this is the precision form offered beside the FP32 radix path.
 *   d_in, d_out  device, complex64 [B][N][N] row-major, DC at index 0; may be the same buffer
 *   B            transforms, >= 0 (0 is a no-op)
 *   N            64 or 128 (other sizes: PTYCHO_EINVAL); 128 = two 64-point halves and a
 *                radix-2 butterfly per pass
 *   inverse      0 forward (exp(-2 pi i k n / N), 1/N), 1 inverse (exp(+...), 1/N)
 *   d_status     device int, caller-owned; set to 1 if a bounded device wait gave up (never
 *                cleared by the library)
 * The first call on a device builds the split DFT matrix (a 64 KB array compiled into the
 * library) and synchronises the device; make it before any stream capture.  Asynchronous.
 */
int dft2_split_bf16(const void *d_in, void *d_out, int B, int N, int inverse, int *d_status, void *cuda_stream);

typedef struct ptycho_ctx *ptycho_handle;

/* Reconstruction engines (the paper cites PIE / ePIE / difference map without choosing one):
 *   AP           full-batch alternating projections (default): all exit waves from the same
 *                (O, P), least-squares object update, then least-squares probe update.
 *   EPIE_COLOUR  ePIE (Maiden and Rodenburg 2009) run colour by colour: positions are coloured
 *                greedily in index order so that patches of one colour never overlap; per
 *                colour, every member's exit-wave update Delta = psi' - P O_j is computed from
 *                the current (O, P), O_j += alpha conj(P) Delta / max|P|^2 is scattered without
 *                atomics (disjoint patches), and P += (beta / n_colour) sum conj(O_j) Delta /
 *                max|O_j|^2.  One probe mode only. */
enum { PTYCHO_ALG_AP = 0, PTYCHO_ALG_EPIE_COLOUR = 1 };

/* FFT form of the exit-wave step (the paper prescribes none):
 *   RADIX_FP32        FP32 radix FFTs on the CUDA cores (default; N = 16, 64, 128, 256)
 *   DFTGEMM_BF16X3    split-BF16 3-term DFT-by-GEMM on the tensor cores, FP32 accumulation
 *                     (see dft2_split_bf16); N = 64, 128 or 256 (256 = four 64-point GEMMs of
 *                     the decimated quarters x[4 r + q] and a radix-4 epilogue, in the N = 256
 *                     kernel's TMA slot pipeline); one probe mode, algorithm AP. */
enum { PTYCHO_FFT_RADIX_FP32 = 0, PTYCHO_FFT_DFTGEMM_BF16X3 = 1 };

typedef struct {
    int M;                  /* object side (M x M complex64), M >= N                          */
    int N;                  /* probe / detector side: 16, 64, 128 or 256 (128: one mode)      */
    int J;                  /* scan positions, >= 1                                           */
    int modes;              /* incoherent probe modes Q, 1..8 (Eq. 4 with a discrete spectrum:
                               I = sum_m |F(P_m O_j)|^2, shared object); 1 = coherent Eq. 3   */
    const int32_t *h_pos;   /* host [J][2] (y, x) top-left patch corner, 0 <= y, x <= M - N   */
    const float *d_fused;   /* device [J][N][N] fused intensities, DC-centred (fuse_stack's
                               output); A = sqrt(max(I, 0)) is formed once here              */
    const void *obj0;       /* complex64 [M][M] initial object                                */
    const void *probe0;     /* complex64 [modes][N][N] initial probe modes                    */
    int init_on_device;     /* 1: obj0 / probe0 are device pointers, 0: host pointers         */
    float alpha_O;          /* object regulariser relative to max sum_j |P|^2 (>= 0)          */
    float alpha_P;          /* probe regulariser relative to max sum_j |O_j|^2 (>= 0)         */
    int probe_update_start; /* first iteration (counted from init) that updates the probe     */
    int algorithm;          /* PTYCHO_ALG_AP (default) or PTYCHO_ALG_EPIE_COLOUR              */
    float epie_alpha;       /* ePIE object step (> 0; 1 is standard), EPIE_COLOUR only        */
    float epie_beta;        /* ePIE probe step (>= 0; 1 is standard), EPIE_COLOUR only        */
    int fft_path;           /* PTYCHO_FFT_RADIX_FP32 (default) or PTYCHO_FFT_DFTGEMM_BF16X3    */
    void *cuda_stream;      /* stream for all work of this handle                             */
} ptycho_desc;

/*
 * ptycho_init -- set up a reconstruction (§3.3 forward model, Eqs. 2-3).  Copies positions,
 * fused intensities (as amplitudes with DC moved to index 0), initial object and probe into
 * handle-owned device memory; the caller may free its inputs when the call returns.  Builds
 * the per-tile position lists of the object update on the host.  Synchronises the stream.
 * Returns PTYCHO_EINVAL (sizes, N unsupported, position out of range, NULL pointers),
 * PTYCHO_ENOMEM, PTYCHO_ECUDA.  *out is NULL on failure.
 */
int ptycho_init(ptycho_handle *out, const ptycho_desc *d);

/*
 * ptycho_iterate -- run n_iter >= 0 iterations of full-batch alternating projections:
 * per position psi_j' = F^-1[A_j F(P O_j) / |F(P O_j)|] (Eqs. 2-3 and the modulus
 * constraint), then the least-squares object update from all psi_j', then (from iteration
 * probe_update_start on) the least-squares probe update from the new object.  With modes > 1
 * every mode's spectrum is scaled by A_j / sqrt(sum_m |F(P_m O_j)|^2), the object update sums
 * over modes and each mode gets its own least-squares probe update.
 *   h_err  host [n_iter] or NULL: per-iteration Fourier error
 *          sum_j sum_q (|Psi_j| - A_j)^2 / sum_j sum_q A_j^2 measured before each projection.
 * With h_err the call synchronises and returns PTYCHO_ENONFINITE if any error is NaN/Inf, or
 * PTYCHO_ETIMEDOUT if a bounded device wait of an exit-wave kernel gave up (that status stays
 * set for the life of the handle); without it the call is asynchronous.
 * Launches (N = 256, one mode, AP): when J is not a multiple of the persistent grid G of the
 * exit-wave kernel and J mod G <= G / 2, the J mod G leftover positions of each iteration run
 * in a second, cooperative launch (a memset of the hand-off counters, then 2-8 CTAs per
 * position), so that the last round takes a fraction of a position's time; a cooperative launch
 * waits until the whole grid is resident, i.e. for other work on the device to leave room.  Not
 * used while the stream is being captured (graphs) — the results are the same either way.
 */
int ptycho_iterate(ptycho_handle h, int n_iter, double *h_err);

/* Copy the current object (complex64 [M][M]) / probe modes (complex64 [modes][N][N]) into dst,
 * a device pointer if dst_on_device else a host pointer.  A host copy synchronises the stream. */
int ptycho_get_object(ptycho_handle h, void *dst, int dst_on_device);
int ptycho_get_probe(ptycho_handle h, void *dst, int dst_on_device);

/* EPIE_COLOUR handles: the colour of every position (host [J]) and the number of colours. */
int ptycho_get_colouring(ptycho_handle h, int32_t *h_colour, int *n_colours);

/* Release every device resource of the handle (waits for its stream; work of other streams
 * on the handle's buffers, e.g. a batch, must be finished or destroyed first).  The buffers go
 * back to the library's memory pool (see ptycho_release_memory), ordered on the handle's stream;
 * destroy the handle before that stream (if the stream is gone, they are freed after a device
 * synchronisation instead).  NULL is a no-op. */
void ptycho_destroy(ptycho_handle h);

/*
 * ptycho_release_memory -- the library's stream-ordered device allocations (reconstruction
 * buffers of ptycho_init, scratch of fuse_stack / fuse_stack_host and of the warm-start
 * stitching) come from one memory pool per device that keeps freed memory for the next
 * allocation instead of returning it to the device, so that creating a reconstruction after
 * destroying one, or fusing the next scan, maps no new pages.  This call hands the memory that
 * no handle or call in flight holds back to the device (memory that live handles hold stays
 * theirs and returns to the pool when they are destroyed).  The pools live as long as the
 * process: the library is not usable across a cudaDeviceReset.  Returns PTYCHO_OK or
 * PTYCHO_ECUDA.
 */
int ptycho_release_memory(void);

/* Per-stage device timing with CUDA events on the handle's stream (for measurement only).
 * While enabled, ptycho_iterate records events at the stage boundaries (one event between two
 * consecutive stages) and synchronises at its end.
 * Stages: 0 exit-wave kernel (patch, FFT, modulus, inverse FFT), 1 object update,
 * 2 probe update, 3 error reduction (ePIE by colour only: the alternating projections form the
 * error inside stage 1).  ms[s] is the summed device time of stage s and
 * launches[s] the number of kernel launches it made since timing was (re-)enabled. */
int ptycho_set_timing(ptycho_handle h, int enable);
int ptycho_stage_times(ptycho_handle h, double *ms /*[4]*/, long long *launches /*[4]*/);

/*
 * Batches of independent reconstructions: many datasets of uneven sizes (positions, object and
 * probe sides) advanced together, iteration by iteration.  The paper reconstructs one scan at a
 * time; batching is a throughput form of the same iteration for many scans.
 *   ptycho_batch_create  groups n existing full-batch (AP) handles (any N, modes, fft_path;
 *                        stage timing off; each handle at most once).  Datasets of one probe
 *                        size and FFT form with N <= 64 share one persistent exit-wave launch per
 *                        iteration; every dataset's other kernels run on its own branch, and the
 *                        branches run concurrently.  flags: PTYCHO_BATCH_GRAPH captures an
 *                        iteration as a CUDA graph and replays it (re-captured when the set of
 *                        datasets updating their probe changes); PTYCHO_BATCH_AUTOTUNE times
 *                        candidate launch shapes (persistent grid sizes; rows per TMA stage at
 *                        N = 256; then the tuned per-size launches against the one persistent
 *                        launch below, when two or more datasets can share it) on the datasets
 *                        themselves, keeps the fastest and restores every object and probe
 *                        (results are unaffected).  PTYCHO_BATCH_ONE_LAUNCH
 *                        computes the exit waves of every single-mode radix-FFT dataset, of any
 *                        N, in ONE persistent launch per iteration (units ordered by cost and
 *                        dealt to one 512-thread CTA per SM; N <= 64 positions four at a time per
 *                        CTA); results are bit-identical to the per-size launches, and the
 *                        per-size launch grids are then not tuned.  The handles stay
 *                        owned by the caller, must outlive the batch, belong to one batch at a
 *                        time, and must not be iterated while a batch call is in flight
 *                        (ptycho_iterate between batch calls is fine).  The batch runs on a stream of its
 *                        own, ordered after `cuda_stream` and the handles' streams at each
 *                        call and before their later work.  Synchronises `cuda_stream`.
 *   ptycho_batch_iterate n_iter iterations of every dataset, the same arithmetic as
 *                        ptycho_iterate on each handle.  h_err: host [n] or NULL, each dataset's
 *                        Fourier error of the last iteration (then the call synchronises and
 *                        reports PTYCHO_ENONFINITE, or PTYCHO_ETIMEDOUT if a bounded wait of any
 *                        dataset's kernels gave up).  Later calls on a handle are ordered after
 *                        the batch's work.
 *   ptycho_batch_describe  the autotuner's choices and timings as a JSON object text.
 */
typedef struct ptycho_batch_ctx *ptycho_batch;
enum { PTYCHO_BATCH_GRAPH = 1, PTYCHO_BATCH_AUTOTUNE = 2, PTYCHO_BATCH_ONE_LAUNCH = 4 };
int ptycho_batch_create(ptycho_batch *out, const ptycho_handle *handles, int n, int flags, void *cuda_stream);
int ptycho_batch_iterate(ptycho_batch b, int n_iter, double *h_err);
int ptycho_batch_describe(ptycho_batch b, char *buf, int len);
void ptycho_batch_destroy(ptycho_batch b);

/* Message of the last failing call on this host thread ("" if none). */
const char *ptycho_last_error(void);

/*
 * Test hooks for the failure paths (no counterpart in the paper; for the library's own tests).
 *   ptycho_debug_wait_timeout  enable = 1: every later exit-wave launch of the handle first
 *       waits, with a limit of about 2^20 SM cycles, on a barrier that nothing arrives on, before
 *       it issues any copy; the wait gives up, the kernel sets the handle's status word and
 *       returns, and ptycho_iterate with h_err reports PTYCHO_ETIMEDOUT.  enable = 2: in the
 *       split last round of an iteration (see ptycho_iterate), the first CTA of every leftover
 *       position does not arrive at its first hand-off, so the other CTAs' waits (limit about
 *       2^31 SM cycles, ~1 s) give up: PTYCHO_ETIMEDOUT the same way (a handle whose positions
 *       leave no split round runs normally).  enable = 0 switches the hook off.  The device
 *       context stays usable.  The status word is sticky: the handle keeps reporting the
 *       timeout, so destroy it.  Handles whose exit-wave kernel has no bounded waits (N != 256)
 *       get PTYCHO_EINVAL.
 *   ptycho_debug_fail_alloc  nth > 0: the nth device allocation the library makes from now on
 *       (any entry point, any thread) fails as if the device were out of memory, and the call
 *       that made it returns PTYCHO_ENOMEM after releasing what it had allocated; nth = 0
 *       switches the hook off.  Process-wide.
 */
int ptycho_debug_wait_timeout(ptycho_handle h, int enable);
int ptycho_debug_fail_alloc(int nth);

#ifdef __cplusplus
}
#endif

#endif /* PTYCHO_MNF_H */
