"""FP64 oracle of the learned warm start: a convolutional encoder-decoder that maps a fused
diffraction pattern to a coarse object patch, its gradients and its optimiser, and the stitching
of predicted patches into an initial object.

TEST INFRASTRUCTURE ONLY (see the package docstring).  The paper itself has no network; this
follows the warm-start form of the workload (a small CNN whose predictions seed the plain
reconstruction of §3.3).  Plain numpy in float64, written from the definitions:

  conv layer   y[b, o, i, j] = bias[o] + sum_{c, u, v} w[o, c, u, v] x_in[b, c, s i + u - 1, s j + v - 1]
               with zero padding; mode "s1" (s = 1), "s2" (s = 2, half the side), "up" (x_in is
               the nearest-neighbour 2x up-sampling of x, then s = 1: twice the side)
  activation   ReLU after every layer except the last
  loss         L = mean((y - t)^2) over every element
  Adam         m = b1 m + (1 - b1) g, v = b2 v + (1 - b2) g^2,
               w -= lr (m / (1 - b1^k)) / (sqrt(v / (1 - b2^k)) + eps)   (step k = 1, 2, ...)

Storage precision: the workload fixes BF16 storage for the network (weights, activations), so
``network_forward`` / ``network_backward`` take an optional ``store`` function applied where the
stored form is what later arithmetic reads: every activation after its ReLU, and every dL/dz
that enters a contraction (the weight and input gradients; the bias gradient sums dL/dz as
computed).  ``store=None`` is exact FP64 throughout.

Readings (the workload names the network, not its data transforms):
  * input   x = log(1 + 2x2-binned fused intensity, clipped at 0) / 10, the DC-centred pattern as
            fused (N x N -> N/2 x N/2)
  * target  the object under the probe window, 4 x 4 mean-pooled: (N/4)^2 complex values, as two
            channels (real, imaginary)
  * stitch  coarse object (M/4)^2: per position, the patch at (y // 4, x // 4) weighted by the
            4 x 4 mean of |P|^2; pixels whose weight sum is below 1e-3 of the maximum take 1
            (the flat object); then bilinear up-sampling by 4 (coarse pixel i centred on fine
            4 i + 1.5, edges clamped)
"""
from __future__ import annotations

import numpy as np

MODES = ("s1", "s2", "up")


def _input_of(x: np.ndarray, mode: str) -> np.ndarray:
    if mode == "up":
        return np.repeat(np.repeat(x, 2, axis=2), 2, axis=3)
    return x


def out_side(h: int, mode: str) -> int:
    return h // 2 if mode == "s2" else (2 * h if mode == "up" else h)


def conv_forward(x, w, b, mode: str):
    """x [B][C][H][W], w [O][C][3][3], b [O] -> y [B][O][H'][W'] (definition in the module doc)."""
    if mode not in MODES:
        raise ValueError(mode)
    xi = _input_of(np.asarray(x, np.float64), mode)
    s = 2 if mode == "s2" else 1
    B, C, H, W = xi.shape
    Ho, Wo = H // s, W // s
    xp = np.pad(xi, ((0, 0), (0, 0), (1, 1), (1, 1)))
    y = np.zeros((B, w.shape[0], Ho, Wo))
    for u in range(3):
        for v in range(3):
            tap = xp[:, :, u:u + s * Ho:s, v:v + s * Wo:s]          # x_in[s i + u - 1, s j + v - 1]
            y += np.einsum("bchw,oc->bohw", tap, w[:, :, u, v])
    return y + b[None, :, None, None]


def conv_backward(x, w, dy, mode: str):
    """Gradients of sum(dy * conv_forward(x, w, b)) with respect to x, w and b."""
    x = np.asarray(x, np.float64)
    xi = _input_of(x, mode)
    s = 2 if mode == "s2" else 1
    B, C, H, W = xi.shape
    Ho, Wo = dy.shape[2], dy.shape[3]
    xp = np.pad(xi, ((0, 0), (0, 0), (1, 1), (1, 1)))
    dxp = np.zeros_like(xp)
    dw = np.zeros_like(w, dtype=np.float64)
    for u in range(3):
        for v in range(3):
            tap = xp[:, :, u:u + s * Ho:s, v:v + s * Wo:s]
            dw[:, :, u, v] = np.einsum("bohw,bchw->oc", dy, tap)
            dxp[:, :, u:u + s * Ho:s, v:v + s * Wo:s] += np.einsum("bohw,oc->bchw", dy, w[:, :, u, v])
    dxi = dxp[:, :, 1:H + 1, 1:W + 1]
    if mode == "up":                                                 # adjoint of the repetition
        dx = dxi.reshape(B, C, H // 2, 2, W // 2, 2).sum(axis=(3, 5))
    else:
        dx = dxi
    db = dy.sum(axis=(0, 2, 3))
    return dx, dw, db


def relu(x):
    return np.maximum(x, 0.0)


def network_forward(layers, params, x, store=None):
    """layers: [(cin, cout, mode)]; params: [(w, b)].  Returns the output and the per-layer inputs
    and pre-activations needed by the backward pass."""
    acts, pre = [np.asarray(x, np.float64)], []
    h = acts[0]
    for i, ((cin, cout, mode), (w, b)) in enumerate(zip(layers, params)):
        z = conv_forward(h, w, b, mode)
        pre.append(z)
        if i == len(layers) - 1:
            h = z
        else:
            h = relu(z)
            if store is not None:
                h = store(h)
        acts.append(h)
    return h, acts, pre


def mse(y, t):
    y = np.asarray(y, np.float64)
    d = y - t
    return float(np.mean(d * d)), 2.0 * d / d.size


def network_backward(layers, params, acts, pre, dout, store=None):
    """Parameter gradients [(dw, db)] and the input gradient, by the chain rule layer by layer."""
    grads = [None] * len(layers)
    g = dout
    for i in range(len(layers) - 1, -1, -1):
        if i != len(layers) - 1:
            g = g * (pre[i] > 0.0)
        db = g.sum(axis=(0, 2, 3))
        gs = g if store is None else store(g)
        dx, dw, _ = conv_backward(acts[i], params[i][0], gs, layers[i][2])
        grads[i] = (dw, db)
        g = dx
    return grads, g


def adam_step(w, g, m, v, k: int, lr: float, b1: float = 0.9, b2: float = 0.999, eps: float = 1e-8):
    """One Adam update (step number k >= 1); returns new (w, m, v)."""
    m = b1 * m + (1.0 - b1) * g
    v = b2 * v + (1.0 - b2) * g * g
    mh = m / (1.0 - b1 ** k)
    vh = v / (1.0 - b2 ** k)
    return w - lr * mh / (np.sqrt(vh) + eps), m, v


def preprocess(fused: np.ndarray) -> np.ndarray:
    """[J][N][N] fused intensity -> [J][1][N/2][N/2] network input (module doc)."""
    f = np.maximum(np.asarray(fused, np.float64), 0.0)
    J, N, _ = f.shape
    binned = f.reshape(J, N // 2, 2, N // 2, 2).sum(axis=(2, 4))
    return (np.log1p(binned) / 10.0)[:, None]


def targets(obj: np.ndarray, pos, N: int) -> np.ndarray:
    """[J][2][N/4][N/4]: the object under each probe window, 4 x 4 mean-pooled (re, im)."""
    out = []
    for y, x in pos:
        p = obj[y:y + N, x:x + N].reshape(N // 4, 4, N // 4, 4).mean(axis=(1, 3))
        out.append(np.stack([p.real, p.imag]))
    return np.array(out)


def stitch(pred: np.ndarray, pos, probe: np.ndarray, M: int) -> np.ndarray:
    """Initial object [M][M] from predicted coarse patches pred [J][2][N/4][N/4] (module doc)."""
    N = probe.shape[0]
    n, Mc = N // 4, M // 4
    wgt = (np.abs(probe) ** 2).reshape(n, 4, n, 4).mean(axis=(1, 3))
    num = np.zeros((Mc, Mc), complex)
    den = np.zeros((Mc, Mc))
    for j, (y, x) in enumerate(pos):
        cy, cx = y // 4, x // 4
        num[cy:cy + n, cx:cx + n] += wgt * (pred[j, 0] + 1j * pred[j, 1])
        den[cy:cy + n, cx:cx + n] += wgt
    ok = den >= 1e-3 * den.max()
    coarse = np.where(ok, num / np.where(ok, den, 1.0), 1.0 + 0j)
    # bilinear: fine pixel f sits at coarse coordinate (f - 1.5) / 4, clamped to [0, Mc - 1]
    c = np.clip((np.arange(M) - 1.5) / 4.0, 0.0, Mc - 1.0)
    i0 = np.minimum(np.floor(c).astype(int), Mc - 2)
    t = c - i0
    rows = coarse[i0] * (1 - t)[:, None] + coarse[i0 + 1] * t[:, None]
    return rows[:, i0] * (1 - t)[None, :] + rows[:, i0 + 1] * t[None, :]
