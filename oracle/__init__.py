"""FP64 CPU oracle for the paper's hot path: Multi-Scale Non-Linear Fusion (§3.4) and the
iterative ptychographic reconstruction that consumes the fused patterns (§3.3), plus the learned
warm start's network, gradients, optimiser and patch stitching (``oracle.cnn``).

TEST INFRASTRUCTURE ONLY.  This package is the slow, plain, obviously-correct statement of what
the CUDA library computes.  Only the test suite, the smoke check and the benchmark's CPU-baseline
leg may import it.  It shares no code with the CUDA path: the library never imports it and it
never imports the library.

Parity status: every function here is pinned by tests against closed forms, library routines or
brute force (see ``tests/test_oracle_*.py``), except the absolute convergence behaviour of the
reconstruction on noisy fused data (time to a given NRMSE), which depends on unpublished
constants and is reported, not pinned ("parity unpinned" for that figure only).
"""
from .mnf import FuseParams, exposure_weights, radiance, blur_down, upsample, \
    gaussian_pyramid, laplacian_pyramid, quantise, mnf_position, mnf_stack, sli_position, \
    sli_stack
from .ptycho import fft2u, ifft2u, amplitudes, modulus_projection, reconstruct, \
    iterate_once, exit_wave_update, object_update, probe_update, illumination, nrmse, \
    fourier_error, modes_modulus_projection, iterate_once_modes, reconstruct_modes, \
    greedy_colouring, epie_by_colour
from . import cnn

__all__ = [
    "FuseParams", "sli_position", "sli_stack", "exposure_weights", "radiance", "blur_down", "upsample", "gaussian_pyramid",
    "laplacian_pyramid", "quantise", "mnf_position", "mnf_stack", "fft2u", "ifft2u",
    "amplitudes", "modulus_projection", "reconstruct", "iterate_once", "exit_wave_update",
    "object_update", "probe_update",
    "illumination", "nrmse", "fourier_error", "modes_modulus_projection", "iterate_once_modes",
    "reconstruct_modes", "greedy_colouring", "epie_by_colour", "cnn",
]
