"""FP64 oracle of Multi-Scale Non-Linear Fusion (MNF), §3.4 of the paper.

TEST INFRASTRUCTURE ONLY (see the package docstring).  Plain numpy in float64, one scan
position at a time, following the four stages of §3.4 in the paper's order:

  §3.4.1  exposure quality  W_k = exp(-(Ibar_k - mu)^2 / (2 sigma^2)), then sum_k W_k = 1  (Eq. 5)
  §3.4.2  pyramids          G_{l+1} = D2(G_l * w_G)  (Eq. 6),  L_l = G_l - U2(G_{l+1})  (Eq. 7)
  §3.4.3  modulation        Lhat_l = G_l[W_k] * L_l[E_k];  Ltilde = Delta_l round(Lhat/Delta_l) (Eq. 8)
  §3.4.4  per-exposure collapse R_{l-1} = U2(R_l) + Ltilde_{l-1}  (Eq. 9), I = sum_k R_0^(k) (Eq. 10)

Readings of points the paper leaves open (each is a parameter or documented default):
  * Ibar = min(I, clip) / clip: normalised by the detector full scale, so saturated pixels
    give Ibar = 1 (§3.4.1 only says Ibar lies in [0, 1]).
  * mu = 0.5, sigma = 0.2 by default (§3.4.1 gives no values).
  * The pyramid input is the radiance E_k = I_k * t_max / t_k (domain "radiance", default);
    domain "raw" feeds I_k itself, as Eq. 7 is literally written.
  * w_G = [1, 4, 6, 4, 1] / 16 per axis (Burt-Adelson); D2 keeps even indices; U2 inserts zeros
    and filters with 2 w_G per axis; every border is mirrored without repeating the edge
    sample (reflect-101) on the grid being filtered.  Needs N / 2^(L-1) >= 4.
  * Levels: l = 0 is the finest; G_0 .. G_{L-1}; details L_0 .. L_{L-2}.
  * Delta_l = delta0 * delta_ratio^l (coarser levels get larger steps, §3.4.3); delta0 = 0
    turns the quantiser off.  round() is round-half-to-even.
  * Eq. 9 is read as the recursive collapse from the base R_{L-1} down to R_0 (the literal
    text up-samples the image Gaussian at each level, which would discard all but the
    finest detail).
  * Base R_{L-1}^(k) (§3.4.4 says it comes from the Gaussian pyramid, unweighted):
      "mean"      G_{L-1}[E_k] / K   (default: keeps base and details on one scale)
      "sum"       G_{L-1}[E_k]       (Eq. 10 taken literally)
      "weighted"  G_{L-1}[W_k] * G_{L-1}[E_k]
"""
from __future__ import annotations

import dataclasses

import numpy as np

W_G = np.array([1.0, 4.0, 6.0, 4.0, 1.0]) / 16.0

BASE_MODES = ("mean", "sum", "weighted")


@dataclasses.dataclass(frozen=True)
class FuseParams:
    levels: int = 4
    mu: float = 0.5
    sigma: float = 0.2
    delta0: float = 0.5
    delta_ratio: float = 2.0
    clip: float = 4095.0
    base_mode: str = "mean"
    domain: str = "radiance"

    def delta(self, level: int) -> float:
        return self.delta0 * self.delta_ratio ** level


def exposure_weights(raw: np.ndarray, clip: float, mu: float, sigma: float) -> np.ndarray:
    """Eq. 5 and the normalisation after it (§3.4.1).  raw: [K, ...] counts -> W [K, ...]."""
    raw = np.asarray(raw, dtype=np.float64)
    ibar = np.minimum(raw, clip) / clip
    w = np.exp(-((ibar - mu) ** 2) / (2.0 * sigma * sigma))
    total = w.sum(axis=0)
    K = raw.shape[0]
    safe = total > 1e-300
    return np.where(safe, w / np.where(safe, total, 1.0), 1.0 / K)


def radiance(raw: np.ndarray, times, domain: str = "radiance") -> np.ndarray:
    """E_k = I_k * t_max / t_k (radiance in longest-exposure counts) or I_k itself ("raw")."""
    raw = np.asarray(raw, dtype=np.float64)
    if domain == "raw":
        return raw.copy()
    t = np.asarray(times, dtype=np.float64)
    return raw * (t.max() / t)[:, None, None]


def blur_down(x: np.ndarray) -> np.ndarray:
    """Eq. 6: G_{l+1}[i, j] = sum_{a,b} w[a] w[b] G_l[2i + a - 2, 2j + b - 2], reflect-101."""
    n = x.shape[0]
    xp = np.pad(x, 2, mode="reflect")          # numpy "reflect" = mirror without the edge
    m = n // 2
    out = np.zeros((m, m))
    for a in range(5):
        for b in range(5):
            out += W_G[a] * W_G[b] * xp[a:a + 2 * m:2, b:b + 2 * m:2]
    return out


def upsample(x: np.ndarray) -> np.ndarray:
    """U2 of §3.4.2: insert zeros to double the grid, then filter with 2 w_G along each axis
    (reflect-101 on the doubled grid)."""
    n = x.shape[0]
    z = np.zeros((2 * n, 2 * n))
    z[::2, ::2] = x
    zp = np.pad(z, 2, mode="reflect")
    out = np.zeros((2 * n, 2 * n))
    for a in range(5):
        for b in range(5):
            out += (2.0 * W_G[a]) * (2.0 * W_G[b]) * zp[a:a + 2 * n, b:b + 2 * n]
    return out


def gaussian_pyramid(x: np.ndarray, levels: int) -> list:
    """G_0 = x, G_{l+1} = D2(G_l * w_G) for l = 0 .. L-2 (Eq. 6)."""
    g = [np.asarray(x, dtype=np.float64)]
    for _ in range(levels - 1):
        g.append(blur_down(g[-1]))
    return g


def laplacian_pyramid(g: list) -> list:
    """L_l = G_l - U2(G_{l+1}) for l = 0 .. L-2 (Eq. 7)."""
    return [g[l] - upsample(g[l + 1]) for l in range(len(g) - 1)]


def quantise(lhat: np.ndarray, delta: float) -> np.ndarray:
    """Eq. 8: Delta * round(Lhat / Delta), ties to even; delta == 0 leaves Lhat unchanged."""
    if delta == 0.0:
        return lhat.copy()
    return delta * np.rint(lhat / delta)


def mnf_position(raw: np.ndarray, times, p: FuseParams, return_coeffs: bool = False):
    """Fuse one position's bracket raw[K][N][N] (DC-centred counts) into I_MNF[N][N].

    With ``return_coeffs`` also returns, per detail level l, the array Lhat / Delta_l of shape
    [K, n_l, n_l] (empty list when the quantiser is off), used to locate rounding ties.
    """
    if p.base_mode not in BASE_MODES:
        raise ValueError(p.base_mode)
    raw = np.asarray(raw, dtype=np.float64)
    K, N, _ = raw.shape
    L = p.levels
    if N % (1 << (L - 1)) or (N >> (L - 1)) < 4:
        raise ValueError("N / 2^(L-1) must be an integer >= 4")
    W = exposure_weights(raw, p.clip, p.mu, p.sigma)            # §3.4.1
    E = radiance(raw, times, p.domain)
    fused = np.zeros((N, N))
    ratios = [np.zeros((K, N >> l, N >> l)) for l in range(L - 1)]
    for k in range(K):
        ge = gaussian_pyramid(E[k], L)                            # §3.4.2
        gw = gaussian_pyramid(W[k], L)
        lap = laplacian_pyramid(ge)
        detail = []
        for l in range(L - 1):                                    # §3.4.3
            lhat = gw[l] * lap[l]
            d = p.delta(l)
            if d != 0.0:
                ratios[l][k] = lhat / d
            detail.append(quantise(lhat, d))
        if p.base_mode == "mean":                                 # §3.4.4
            r = ge[L - 1] / K
        elif p.base_mode == "sum":
            r = ge[L - 1].copy()
        else:
            r = gw[L - 1] * ge[L - 1]
        for l in range(L - 2, -1, -1):                            # Eq. 9, recursive reading
            r = upsample(r) + detail[l]
        fused += r                                                # Eq. 10
    if return_coeffs:
        return fused, (ratios if p.delta0 != 0.0 else [])
    return fused


def mnf_stack(raw: np.ndarray, times, p: FuseParams) -> np.ndarray:
    """Positions are independent (§3.4): fuse raw[J][K][N][N] -> I_MNF[J][N][N]."""
    raw = np.asarray(raw)
    return np.stack([mnf_position(raw[j], times, p) for j in range(raw.shape[0])])


def sli_position(raw: np.ndarray, times, clip: float) -> np.ndarray:
    """Standard Linear Integration, the linear HDR baseline the paper compares against (§1,
    §2.2): per pixel, the exposure-time-weighted mean count rate over the unsaturated exposures,
    in longest-exposure units, t_max * sum_{k: I_k < clip} I_k / sum_{k: I_k < clip} t_k.  A
    pixel saturated in every exposure takes the shortest exposure's clipped rate."""
    raw = np.asarray(raw, dtype=np.float64)
    t = np.asarray(times, dtype=np.float64)
    ok = raw < clip
    num = np.sum(np.where(ok, raw, 0.0), axis=0)
    den = np.sum(np.where(ok, t[:, None, None], 0.0), axis=0)
    kmin = int(np.argmin(t))
    fallback = raw[kmin] / t[kmin]
    return t.max() * np.where(den > 0, num / np.where(den > 0, den, 1.0), fallback)


def sli_stack(raw: np.ndarray, times, clip: float) -> np.ndarray:
    raw = np.asarray(raw)
    return np.stack([sli_position(raw[j], times, clip) for j in range(raw.shape[0])])
