"""Helpers for the GPU-vs-oracle parity tests (CPU side only)."""
import numpy as np

import oracle

# FP32 unit roundoff.  A detail coefficient is a few dozen FP32 multiply-adds deep (25-tap
# filters per level, the weight normalisation, the up-sampling), so the GPU's value may sit up
# to ~32 u of its own operand scale away from the FP64 value.
U32 = 2.0 ** -24
TIE_SLACK = 32 * U32


def tie_mask(raw, times, p: oracle.FuseParams):
    """Level-0 pixels whose fused value may legitimately differ between FP32 and FP64 by one
    quantiser step: the footprint of every coefficient whose FP64 ratio Lhat / Delta lies within
    FP32 reach of a rounding tie (both sides round the same ratio; only a tie can flip it).

    Returns (mask, n_ties, n_coeffs)."""
    raw = np.asarray(raw, dtype=np.float64)
    K, N, _ = raw.shape
    L = p.levels
    mask = np.zeros((N, N), bool)
    if p.delta0 == 0.0 or L < 2:
        return mask, 0, 0
    W = oracle.exposure_weights(raw, p.clip, p.mu, p.sigma)
    E = oracle.radiance(raw, times, p.domain)
    n_ties = 0
    n_coeffs = 0
    for k in range(K):
        ge = oracle.gaussian_pyramid(E[k], L)
        gw = oracle.gaussian_pyramid(W[k], L)
        for l in range(L - 1):
            d = p.delta(l)
            up = oracle.upsample(ge[l + 1])
            ratio = gw[l] * (ge[l] - up) / d
            scale = np.abs(gw[l]) * (np.abs(ge[l]) + np.abs(up)) / d + np.abs(ratio)
            frac = np.abs(ratio - np.floor(ratio) - 0.5)
            ties = frac <= TIE_SLACK * scale + 1e-6
            n_ties += int(ties.sum())
            n_coeffs += ties.size
            if ties.any():
                r = 2 ** (l + 1)            # support of U2^l of an impulse at level l
                ys, xs = np.nonzero(ties)
                for y, x in zip(ys, xs):
                    cy, cx = y << l, x << l
                    mask[max(0, cy - r):cy + r + 1, max(0, cx - r):cx + r + 1] = True
    return mask, n_ties, n_coeffs


def tie_allowance(raw, times, p: oracle.FuseParams):
    """Per level-0 pixel, how far the FP32 fusion may sit from the FP64 oracle because of
    quantiser decisions that FP32 cannot take reliably: every detail coefficient (exposure k,
    level l) whose FP64 ratio Lhat / Delta_l lies within FP32 reach of a rounding tie (see
    tie_mask) may round either way, which moves R_l^(k) by Delta_l there; the up-sampling U2 is
    a max-norm contraction, so the output moves by at most Delta_l inside the coefficient's
    footprint (radius 2^(l+1) - 2 at level 0; 2^(l+1) is used).  The allowances of overlapping
    footprints add up.

    Returns (allowance [N][N], n_ties, n_coeffs)."""
    raw = np.asarray(raw, dtype=np.float64)
    K, N, _ = raw.shape
    L = p.levels
    allow = np.zeros((N, N))
    if p.delta0 == 0.0 or L < 2:
        return allow, 0, 0
    W = oracle.exposure_weights(raw, p.clip, p.mu, p.sigma)
    E = oracle.radiance(raw, times, p.domain)
    n_ties = 0
    n_coeffs = 0
    for k in range(K):
        ge = oracle.gaussian_pyramid(E[k], L)
        gw = oracle.gaussian_pyramid(W[k], L)
        for l in range(L - 1):
            d = p.delta(l)
            up = oracle.upsample(ge[l + 1])
            ratio = gw[l] * (ge[l] - up) / d
            scale = np.abs(gw[l]) * (np.abs(ge[l]) + np.abs(up)) / d + np.abs(ratio)
            frac = np.abs(ratio - np.floor(ratio) - 0.5)
            ties = frac <= TIE_SLACK * scale + 1e-6
            n_ties += int(ties.sum())
            n_coeffs += ties.size
            r = 2 ** (l + 1)
            for y, x in zip(*np.nonzero(ties)):
                cy, cx = y << l, x << l
                allow[max(0, cy - r):cy + r + 1, max(0, cx - r):cx + r + 1] += d
    return allow, n_ties, n_coeffs


def rel_l2(a, b):
    b = np.asarray(b)
    return float(np.linalg.norm(np.asarray(a) - b) / max(np.linalg.norm(b), 1e-300))
