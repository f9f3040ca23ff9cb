/*
 * measure.h -- measurement entry points of the library (no counterpart in the paper, which
 * reports no hardware figures; they supply the measured denominators of the roofline).
 */
#ifndef PTYCHO_MEASURE_H
#define PTYCHO_MEASURE_H

#ifdef __cplusplus
extern "C" {
#endif

/*
 * measure_fp32_fma -- enqueue one launch of `blocks` blocks x measure_fma_threads_per_block()
 * threads, each thread running `iters` x 128 dependent-free FP32 FMAs (16 independent chains),
 * on cuda_stream; the caller times it with CUDA events on that stream.
 *   d_sink  device, float [blocks * threads], caller-owned (receives the chain sums so that the
 *           work cannot be optimised away)
 *   flops   host, receives the launch's FP32 flops (an FMA counts 2)
 * Returns PTYCHO_EINVAL for blocks < 1, iters < 1 or NULL pointers; asynchronous.
 */
int measure_fp32_fma(int blocks, int iters, float *d_sink, double *flops, void *cuda_stream);

/* Threads per block of measure_fp32_fma's launches. */
int measure_fma_threads_per_block(void);

#ifdef __cplusplus
}
#endif

#endif /* PTYCHO_MEASURE_H */
