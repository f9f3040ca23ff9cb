"""Seeded synthetic ptychographic scans: the one input generator shared by tests, bench and smoke.

This module holds none of the fusion or reconstruction arithmetic.  It draws a ground-truth
object and probe, lays out a scan, and simulates the detector: the far-field forward model
(§3.3, Eqs. 2-3: psi_j = P * O(r - r_j), I = |F psi|^2), a bracket of K exposures whose mean
counts scale with exposure time (§2.1, Eq. 1), Poisson counting and a detector clip (the
saturation of §2.3).  The paper's data are private, so these scans stand in for its workloads;
the recipe follows the workload table of the design notes (object amplitude U[0.5, 1], phase a
Gaussian-smoothed random field, soft circular probe with quadratic phase, raster or Fermat-spiral
scan).

Two back ends produce the same distributions from the same seed recipe:
  * ``make_scan``        numpy (PCG64), used by the CPU tests and the oracle-sized cases;
  * ``make_scan_torch``  object/probe/positions from numpy, frames simulated with torch on a
                         device (used for the lab-scale workload, where numpy would take minutes).
The two draw different Poisson streams, so their frames differ value by value.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

__all__ = ["ScanConfig", "CONFIGS", "make_object", "make_probe", "make_probe_modes",
           "raster_positions", "spiral_positions", "make_scan", "make_scan_torch", "seed_for",
           "batched_configs", "WARM_NET"]


@dataclasses.dataclass(frozen=True)
class ScanConfig:
    name: str
    M: int                      # object side (pixels)
    N: int                      # probe / detector side (pixels)
    scan: str                   # "raster" or "spiral"
    radius: float               # probe aperture radius (pixels)
    times: tuple                # relative exposure times t_k, ascending
    peak: float                 # expected counts of the brightest pixel in the longest frame
    clip: int                   # detector full scale (counts)
    levels: int                 # pyramid levels L
    n_iter: int                 # reconstruction iterations
    n_side: int = 0             # raster: positions per side
    step: int = 0               # raster: step (pixels)
    jitter: int = 0             # raster: uniform integer jitter in [-jitter, jitter]
    J: int = 0                  # spiral: number of positions
    phase_sigma: float = 4.0    # smoothing of the object phase field (pixels)
    modes: int = 1              # incoherent probe modes (one per wavelength)
    bandwidth: float = 0.1      # wavelengths span lambda_0 (1 +- bandwidth)

    @property
    def K(self) -> int:
        return len(self.times)

    @property
    def n_pos(self) -> int:
        return self.n_side * self.n_side if self.scan == "raster" else self.J


CONFIGS = {
    # 256^2 object, 64^2 probe, 10x10 raster step 8 with +-1 px jitter, exposures 1/10/100,
    # 1e4 peak counts in the longest frame, 12-bit clip, 4 levels, 50 iterations.
    "small": ScanConfig("small", M=256, N=64, scan="raster", radius=20.0, times=(1.0, 10.0, 100.0),
                        peak=1e4, clip=4095, levels=4, n_iter=50, n_side=10, step=8, jitter=1),
    # 1024^2 object, 256^2 probe, 1600 Fermat-spiral positions, exposures 1/4/16/64/256,
    # 1e6 peak counts, 16-bit clip, 6 levels, 200 iterations.
    "lab": ScanConfig("lab", M=1024, N=256, scan="spiral", radius=80.0,
                      times=(1.0, 4.0, 16.0, 64.0, 256.0), peak=1e6, clip=65535, levels=6,
                      n_iter=200, J=1600),
    # Mixed state: the lab scan with 8 probe modes over +-10% bandwidth, 100 iterations.
    "mixed": ScanConfig("mixed", M=1024, N=256, scan="spiral", radius=80.0,
                        times=(1.0, 4.0, 16.0, 64.0, 256.0), peak=1e6, clip=65535, levels=6,
                        n_iter=100, J=1600, modes=8),
    # The same construction on the small scan (fast enough for the oracle).
    "mixed_small": ScanConfig("mixed_small", M=256, N=64, scan="raster", radius=20.0,
                              times=(1.0, 10.0, 100.0), peak=1e4, clip=4095, levels=4, n_iter=20,
                              n_side=10, step=8, jitter=1, modes=8),
    # The small scan's construction (64^2 probe, 3 exposures, 12-bit clip, 4 levels) on a
    # 1024^2 object with a 96 x 96 raster, step 10: 9216 positions, enough to fill the GPU.
    "wide64": ScanConfig("wide64", M=1024, N=64, scan="raster", radius=20.0, times=(1.0, 10.0, 100.0),
                         peak=1e4, clip=4095, levels=4, n_iter=50, n_side=96, step=10, jitter=1),
    # The same with a 128^2 probe (radius 40): 48 x 48 raster, step 18 (2304 positions).
    "wide128": ScanConfig("wide128", M=1024, N=128, scan="raster", radius=40.0, times=(1.0, 10.0, 100.0),
                          peak=1e4, clip=4095, levels=4, n_iter=50, n_side=48, step=18, jitter=1),
    # Reduced cases for the CPU tests (same construction, smaller sizes).
    "tiny": ScanConfig("tiny", M=64, N=16, scan="raster", radius=5.0, times=(1.0, 10.0, 100.0),
                       peak=1e4, clip=4095, levels=3, n_iter=30, n_side=5, step=4, jitter=1,
                       phase_sigma=2.0),
    "mid": ScanConfig("mid", M=160, N=64, scan="raster", radius=20.0, times=(1.0, 10.0, 100.0),
                      peak=1e4, clip=4095, levels=4, n_iter=20, n_side=5, step=16, jitter=1),
    # The same construction with a 128^2 probe (radius 40): 5 x 5 raster, step 24, 256^2 object.
    "mid128": ScanConfig("mid128", M=256, N=128, scan="raster", radius=40.0, times=(1.0, 10.0, 100.0),
                         peak=1e4, clip=4095, levels=4, n_iter=20, n_side=5, step=24, jitter=1),
}


# The warm-start network of the learned-initialisation workload: 8 convolution layers (3 x 3
# kernels) as (input channels, output channels, mode), mode "s1" stride 1, "s2" stride 2, "up"
# nearest 2x up-sampling then stride 1; ReLU after every layer but the last.  Four stride-2
# layers bring a 128^2 input to an 8^2 bottleneck, so the bottleneck sees most of the pattern
# (a far-field pattern mixes every object pixel into every detector pixel).  Input: the fused
# pattern binned to (N/2)^2, one channel; output: the (N/4)^2 coarse object patch, two channels
# (real, imaginary).  2.05 M weights (the widest layers at the 8^2 bottleneck and the first
# up-sampling step).
WARM_NET = ((1, 32, "s2"), (32, 64, "s2"), (64, 128, "s2"), (128, 256, "s2"), (256, 384, "s1"),
            (384, 192, "up"), (192, 64, "up"), (64, 2, "up"))


def batched_configs(seed: int | None = None, count: int = 64) -> list:
    """The uneven multi-dataset workload: ``count`` scans built like the small scan (exposures
    1/10/100, 1e4 peak counts, 12-bit clip, 4 pyramid levels, 50 iterations), each with its own
    probe side N drawn from {64, 128, 256} (aperture radius 5N/16), an n x n raster with n drawn from
    [7, 30] (capped so the scan fits a 1024-pixel object; step N/8, +-1 px jitter) and the
    smallest object side M in [256, 1024], a multiple of 32, that holds it."""
    rng = np.random.default_rng(seed_for("batched") if seed is None else seed)
    out = []
    for d in range(count):
        N = int(rng.choice([64, 128, 256]))
        step = N // 8
        n_max = min(30, (1024 - N - 2) // step + 1)
        n = int(rng.integers(7, n_max + 1))
        span = N + (n - 1) * step + 2
        M = max(256, -(-span // 32) * 32)
        out.append(ScanConfig(f"batched{d}", M=M, N=N, scan="raster", radius=5.0 * N / 16.0,
                              times=(1.0, 10.0, 100.0), peak=1e4, clip=4095, levels=4, n_iter=50,
                              n_side=n, step=step, jitter=1))
    return out


def seed_for(name: str) -> int:
    order = ["small", "lab", "mixed", "batched", "warm", "tiny", "mid", "mixed_small", "wide64", "mid128", "wide128"]
    return 1000 + (order.index(name) if name in order else 99)


def _smooth_field(rng: np.random.Generator, M: int, sigma: float) -> np.ndarray:
    """White noise low-passed with a periodic Gaussian of std ``sigma`` pixels."""
    noise = rng.standard_normal((M, M))
    f = np.fft.fftfreq(M)
    g = np.exp(-2.0 * (math.pi * sigma) ** 2 * (f[:, None] ** 2 + f[None, :] ** 2))
    return np.real(np.fft.ifft2(np.fft.fft2(noise) * g))


def make_object(rng: np.random.Generator, M: int, phase_sigma: float = 4.0) -> np.ndarray:
    """Amplitude iid U[0.5, 1]; phase a smoothed random field scaled to max |phi| = pi/2."""
    amp = rng.uniform(0.5, 1.0, size=(M, M))
    phi = _smooth_field(rng, M, phase_sigma)
    phi *= (math.pi / 2.0) / np.max(np.abs(phi))
    return amp * np.exp(1j * phi)


def make_probe(N: int, radius: float) -> np.ndarray:
    """Soft circular aperture (1 inside, Gaussian roll-off of width radius/10) with phase
    pi r^2 / radius^2.  Unscaled; ``make_scan`` sets the photon scale."""
    c = (N - 1) / 2.0
    yy, xx = np.mgrid[0:N, 0:N]
    r = np.hypot(yy - c, xx - c)
    w = radius / 10.0
    amp = np.where(r <= radius, 1.0, np.exp(-((r - radius) ** 2) / (2.0 * w * w)))
    return amp * np.exp(1j * math.pi * r * r / (radius * radius))


def make_probe_modes(N: int, radius: float, modes: int, bandwidth: float) -> np.ndarray:
    """Q probe modes, one per wavelength lambda_m = lambda_0 (1 + b (2m/(Q-1) - 1)): mode m is the
    probe magnified by lambda_m / lambda_0, P_m(r) = P(r lambda_0 / lambda_m); equal spectral
    weights (1/Q of the power each).  One mode returns the plain probe."""
    if modes == 1:
        return make_probe(N, radius)[None]
    out = []
    for m in range(modes):
        lam = 1.0 + bandwidth * (2.0 * m / (modes - 1) - 1.0)
        out.append(make_probe(N, radius * lam) / math.sqrt(modes))
    return np.stack(out)


def raster_positions(rng: np.random.Generator, M: int, N: int, n_side: int, step: int,
                     jitter: int) -> np.ndarray:
    """Top-left (y, x) of each patch: an n_side^2 raster centred on the object, integer jitter."""
    span = (n_side - 1) * step + N
    origin = (M - span) // 2
    gy, gx = np.mgrid[0:n_side, 0:n_side]
    pos = np.stack([origin + gy.ravel() * step, origin + gx.ravel() * step], axis=1)
    if jitter:
        pos = pos + rng.integers(-jitter, jitter + 1, size=pos.shape)
    return np.clip(pos, 0, M - N).astype(np.int32)


def spiral_positions(M: int, N: int, J: int) -> np.ndarray:
    """Fermat spiral (golden angle 137.508 deg) of J patch centres fitted into the disk of
    radius (M - N)/2 about the object centre; returns rounded top-left (y, x)."""
    golden = math.radians(137.508)
    n = np.arange(J, dtype=np.float64)
    rmax = (M - N) / 2.0
    r = rmax * np.sqrt(n / max(J - 1, 1))
    th = n * golden
    cy = M / 2.0 + r * np.sin(th)
    cx = M / 2.0 + r * np.cos(th)
    pos = np.stack([np.rint(cy - N / 2.0), np.rint(cx - N / 2.0)], axis=1)
    return np.clip(pos, 0, M - N).astype(np.int32)


def _positions(cfg: ScanConfig, rng: np.random.Generator) -> np.ndarray:
    if cfg.scan == "raster":
        return raster_positions(rng, cfg.M, cfg.N, cfg.n_side, cfg.step, cfg.jitter)
    return spiral_positions(cfg.M, cfg.N, cfg.J)


def _far_field_intensity(obj: np.ndarray, probes: np.ndarray, pos: np.ndarray) -> np.ndarray:
    """sum_m |F[P_m * O_j]|^2 over the probe modes (one mode: the coherent intensity), unitary
    2-D DFT, DC moved to the array centre (detector layout)."""
    Q, N, _ = probes.shape
    out = np.empty((len(pos), N, N))
    for j, (y, x) in enumerate(pos):
        psi = probes * obj[y:y + N, x:x + N][None]
        f = np.fft.fftshift(np.fft.fft2(psi, norm="ortho"), axes=(-2, -1))
        out[j] = np.sum(np.abs(f) ** 2, axis=0)
    return out


def make_scan(cfg: ScanConfig | str, seed: int | None = None, noise: bool = True,
              clip: bool = True, times: tuple | None = None, frames_for=None) -> dict:
    """Ground truth plus a K-exposure raw stack ``raw[J][K][N][N]`` (uint16, DC-centred).

    The probe is scaled so that the brightest expected pixel of the longest exposure holds
    ``cfg.peak`` counts; frame k has mean ``I * t_k / t_max``.  ``noise=False`` rounds the mean
    instead of drawing Poisson counts; ``clip=False`` keeps counts above full scale (stored as
    float64 in ``raw`` then).  ``frames_for`` (position indices) simulates frames for those
    positions only (``raw`` then has one row per listed position).  Returns a dict with obj,
    probe (scaled), pos, times, clip_value, intensity (expected counts at t_max) and raw.
    """
    if isinstance(cfg, str):
        cfg = CONFIGS[cfg]
    if seed is None:
        seed = seed_for(cfg.name)
    times = tuple(cfg.times if times is None else times)
    rng = np.random.default_rng(seed)
    obj = make_object(rng, cfg.M, cfg.phase_sigma)
    probe = make_probe_modes(cfg.N, cfg.radius, cfg.modes, cfg.bandwidth)
    pos = _positions(cfg, rng)
    inten = _far_field_intensity(obj, probe, pos)
    scale = cfg.peak / inten.max()
    probe = probe * math.sqrt(scale)
    inten = inten * scale
    tmax = max(times)
    K = len(times)
    sel = np.arange(len(pos)) if frames_for is None else np.asarray(frames_for)
    raw = np.empty((len(sel), K, cfg.N, cfg.N), dtype=np.float64)
    for k, t in enumerate(times):
        lam = inten[sel] * (t / tmax)
        raw[:, k] = rng.poisson(lam) if noise else np.rint(lam)
    if clip:
        raw = np.minimum(raw, cfg.clip).astype(np.uint16)
    if cfg.modes == 1:
        probe = probe[0]                # single mode: [N][N] as before; else [Q][N][N]
    return {"cfg": cfg, "obj": obj, "probe": probe, "pos": pos, "times": np.asarray(times),
            "clip_value": float(cfg.clip), "intensity": inten, "raw": raw, "seed": seed}


def make_scan_torch(cfg: ScanConfig | str, seed: int | None = None, device="cuda",
                    chunk: int = 64) -> dict:
    """Same recipe as ``make_scan``; frames simulated with torch on ``device``.

    Returns obj/probe/pos as numpy (complex128 / int32), ``raw`` as a device tensor of dtype
    torch.uint16 with shape [J][K][N][N] and ``intensity`` (expected counts of the longest
    exposure, noiseless and unclipped, DC-centred) as a float32 device tensor [J][N][N].
    """
    import torch

    if isinstance(cfg, str):
        cfg = CONFIGS[cfg]
    if seed is None:
        seed = seed_for(cfg.name)
    rng = np.random.default_rng(seed)
    obj = make_object(rng, cfg.M, cfg.phase_sigma)
    probe = make_probe_modes(cfg.N, cfg.radius, cfg.modes, cfg.bandwidth)
    pos = _positions(cfg, rng)
    J, N, K = len(pos), cfg.N, cfg.K
    dev = torch.device(device)
    o_t = torch.from_numpy(obj.astype(np.complex64)).to(dev)
    p_t = torch.from_numpy(probe.astype(np.complex64)).to(dev)
    ys = torch.from_numpy(pos[:, 0].astype(np.int64)).to(dev)
    xs = torch.from_numpy(pos[:, 1].astype(np.int64)).to(dev)
    ar = torch.arange(N, device=dev)
    inten = torch.empty((J, N, N), dtype=torch.float32, device=dev)
    for s in range(0, J, chunk):
        e = min(J, s + chunk)
        rows = (ys[s:e, None] + ar[None, :])[:, :, None]
        cols = (xs[s:e, None] + ar[None, :])[:, None, :]
        acc = torch.zeros((e - s, N, N), dtype=torch.float32, device=dev)
        patch = o_t[rows, cols]
        for m in range(p_t.shape[0]):
            f = torch.fft.fftshift(torch.fft.fft2(p_t[m][None] * patch, norm="ortho"), dim=(-2, -1))
            acc += f.real ** 2 + f.imag ** 2
        inten[s:e] = acc
    scale = cfg.peak / float(inten.max())
    inten *= scale
    probe = probe * math.sqrt(scale)
    gen = torch.Generator(device=dev)
    gen.manual_seed(int(seed))
    tmax = max(cfg.times)
    raw = torch.empty((J, K, N, N), dtype=torch.uint16, device=dev)
    for s in range(0, J, chunk):
        e = min(J, s + chunk)
        for k, t in enumerate(cfg.times):
            lam = inten[s:e] * float(t / tmax)
            cnt = torch.poisson(lam, generator=gen).clamp_(max=float(cfg.clip))
            raw[s:e, k] = cnt.to(torch.int32).to(torch.uint16)
    if cfg.modes == 1:
        probe = probe[0]
    return {"cfg": cfg, "obj": obj, "probe": probe, "pos": pos, "times": np.asarray(cfg.times),
            "clip_value": float(cfg.clip), "raw": raw, "intensity": inten, "seed": seed}
