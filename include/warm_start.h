/*
 * warm_start.h -- C ABI of the learned warm start: a convolutional encoder-decoder that predicts
 * coarse object patches from fused diffraction patterns, trained and run on the GPU with the
 * library's own kernels, and the stitching of its predictions into the initial object of the
 * reconstruction (§3.3 iterates from that object instead of a flat one).  The paper has no
 * network; this is the learned-initialisation form of the workload, with the plain flat start
 * as its fallback.
 *
 * Conventions are those of ptycho_mnf.h (status codes, ptycho_last_error(), device/host
 * pointers, streams).  Precision: weights and activations are stored in BF16, every contraction
 * runs on the tensor cores with FP32 accumulation, master weights / Adam moments / biases /
 * loss are FP32.
 */
#ifndef WARM_START_H
#define WARM_START_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/*
 * gemm_bf16 -- C[M][N] = A[M][K] B[N][K]^T on the tensor cores (tcgen05, FP32 accumulation).
 *   d_A, d_B  device, BF16 row-major (K contiguous); d_C device, FP32 row-major
 *   M % 128 == 0, N % 64 == 0, K % 64 == 0 (PTYCHO_EINVAL otherwise); K == 0 zero-fills C
 *   d_status  device int, set to 1 if a bounded device wait gave up
 * Asynchronous.
 */
int gemm_bf16(const void *d_A, const void *d_B, float *d_C, int M, int N, int K, int *d_status, void *cuda_stream);

/* Layer modes: 3 x 3 convolution with one pixel of zero padding at stride 1 (S1), at stride 2
 * (S2, halves the side), or after nearest-neighbour 2x up-sampling (UP, doubles the side). */
enum { WS_MODE_S1 = 0, WS_MODE_S2 = 1, WS_MODE_UP = 2 };

typedef struct wsnet_ctx *wsnet;

/*
 * wsnet_create -- a chain of nlayers convolution layers, ReLU after every layer but the last.
 *   cin, cout, mode  host [nlayers]; cin[i] == cout[i - 1]
 *   in_side          side of the square input; max_batch >= 1 samples per call
 *   seed             He-normal initial weights (std sqrt(2 / (9 cin))), zero biases
 * The network owns its weights, Adam state and all scratch for max_batch samples.
 */
int wsnet_create(wsnet *out, const int *cin, const int *cout, const int *mode, int nlayers, int in_side,
                 int max_batch, unsigned long long seed, void *cuda_stream);

/* Layer parameters (FP32, host): w [cout][cin][3][3], b [cout]; set / get, and the gradients
 * of the last wsnet_backward.  These synchronise the network's stream. */
int wsnet_set_params(wsnet n, int layer, const float *h_w, const float *h_b);
int wsnet_get_params(wsnet n, int layer, float *h_w, float *h_b);
int wsnet_get_grads(wsnet n, int layer, float *h_dw, float *h_db);

/* d_x device BF16 [B][cin_0][in_side][in_side]; d_y device FP32 [B][cout_last][side][side].
 * 1 <= B <= max_batch.  Asynchronous. */
int wsnet_forward(wsnet n, const void *d_x, int B, float *d_y);

/* Forward, mean-squared-error loss against d_t (device FP32, the output's shape) and the
 * gradients of every layer (kept for wsnet_get_grads / wsnet_adam).  h_loss (host) or NULL:
 * with it the call synchronises and reports PTYCHO_ENONFINITE / PTYCHO_ETIMEDOUT. */
int wsnet_backward(wsnet n, const void *d_x, const float *d_t, int B, double *h_loss);

/* One Adam step (beta1 0.9, beta2 0.999, eps 1e-8) with the current gradients. */
int wsnet_adam(wsnet n, float lr);

/* wsnet_backward followed by wsnet_adam. */
int wsnet_train_step(wsnet n, const void *d_x, const float *d_t, int B, float lr, double *h_loss);

void wsnet_destroy(wsnet n);

/* Network input from fused patterns: d_fused device FP32 [J][N][N] (DC-centred) ->
 * d_x device BF16 [J][1][N/2][N/2] = log(1 + 2x2-binned max(I, 0)) / 10.  Asynchronous. */
int ws_preprocess(const float *d_fused, int J, int N, void *d_x, void *cuda_stream);

/* Training targets: d_t device FP32 [J][2][N/4][N/4] = the object d_obj (complex64 [M][M])
 * under each window d_pos (device int32 [J][2], (row, column) top-left), 4 x 4 mean-pooled,
 * (real, imaginary).  Asynchronous. */
int ws_targets(const void *d_obj, int M, const int32_t *d_pos, int J, int N, float *d_t, void *cuda_stream);

/* Initial object from predicted coarse patches d_pred (device FP32 [J][2][N/4][N/4]): on the
 * (M/4)^2 grid, each position's patch at (row / 4, column / 4) weighted by the 4 x 4 mean of
 * |P|^2 of d_probe (complex64 [N][N]); coarse pixels with weight below 1e-3 of the maximum take
 * 1 (the flat object); bilinear up-sampling by 4 (coarse pixel i centred on 4 i + 1.5, edges
 * clamped) into d_obj (complex64 [M][M]).  Stream-ordered scratch.  Asynchronous. */
int ws_stitch(const float *d_pred, const int32_t *d_pos, int J, const void *d_probe, int N, int M, void *d_obj,
              void *cuda_stream);

#ifdef __cplusplus
}
#endif

#endif /* WARM_START_H */
