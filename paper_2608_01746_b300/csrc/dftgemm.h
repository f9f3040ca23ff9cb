// Internal interface between the reconstruction engine and the split-BF16 tensor-core DFT
// (N = 64 and 128; the Dft64Exit record serves both), see dftgemm.cu.
#pragma once

#include <cuda_runtime.h>

namespace pm {

struct Dft64Exit {
    const float2 *obj;      // object [M][M]
    const float2 *probe;    // probe [64][64]
    const float *amp;       // amplitudes [J][kx][ky], DC at index 0
    const int2 *pos;        // (row, column) of each patch's top-left corner
    float2 *psi;            // out: psi' [J][64][64] row-major
    double *err;            // out: Fourier error per position
    int *status;            // set to 1 if a bounded wait gave up
    int M, J;
};

// Once per device (synchronises the device the first time): builds the split DFT matrix and
// sets the kernels' shared-memory limit.  Returns the device's SM count.
int dft64_prepare(int *sm_count);

// psi_j' = F^-1[A_j F(P O_j) / |F(P O_j)|] for every j, tensor-core DFTs; one launch.
int dft64_exit_launch(const Dft64Exit &e, int sm_count, cudaStream_t st);

// The same for N = 128 (two 64-point halves and a radix-2 butterfly per pass; one launch).
int dft128_exit_launch(const Dft64Exit &e, int sm_count, cudaStream_t st);

// Device address of the split 64-point DFT matrix (G_hi then G_lo, 128 x 128 BF16 each in the
// tcgen05 core-matrix layout, 64 KB), built by dft64_prepare (which this call makes first).
int dft64_matrix(const void **d_matrix);

// Patch groups the kernel makes of J positions (the unit of work of one pipeline).
int dft64_groups(int J);

// One launch over several datasets: d_table[d] (device) describes dataset d, whose groups are
// d_gstart[d] .. d_gstart[d + 1] - 1 (device prefix, d_gstart[ntable] = total_groups).  At most
// grid_cap CTAs.
int dft64_exit_multi_launch(const Dft64Exit *d_table, const int *d_gstart, int ntable, int total_groups,
                            int *d_status, int grid_cap, cudaStream_t st);

}  // namespace pm
