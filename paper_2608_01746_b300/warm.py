"""Learned warm start for the reconstruction: training data from the forward model, training of
the warm-start network, and the initial object it predicts for a scan, with the flat start as
fallback and judge.

Orchestration only: every arithmetic step runs in the library's kernels (fusion, network
forward / backward / Adam on the tensor cores, input and target transforms, stitching, the
reconstruction); this module moves tensors between those calls.

  training set  for each random object (the scan recipe of ``synth`` with a fresh seed): the
                bracket of every scan position simulated by the forward model, fused (MNF),
                binned and log-scaled (the network input); the object under the window,
                4 x 4 mean-pooled (the target)
  warm start    predict every position's coarse patch, stitch them into an initial object
  judge         one iteration from the warm start and one from the flat start; the start whose
                first Fourier error (measured before its projection) is lower is kept, so the
                warm start never starts the reconstruction worse than the flat object
"""
from __future__ import annotations

import numpy as np

from . import api, synth


def training_set(cfg: synth.ScanConfig, seeds, device="cuda", stream=None):
    """Network inputs X (bfloat16 [S][1][N/2][N/2]) and targets T (float32 [S][2][N/4][N/4])
    from len(seeds) random objects scanned with ``cfg``."""
    import torch
    params = api.fuse_params(levels=cfg.levels, clip=float(cfg.clip))
    xs, ts = [], []
    for s in seeds:
        sc = synth.make_scan_torch(cfg, seed=int(s), device=device)
        fused = api.fuse_stack(sc["raw"], cfg.times, params, stream=stream)
        xs.append(api.ws_preprocess(fused, stream=stream))
        obj = torch.from_numpy(sc["obj"].astype(np.complex64)).to(device)
        pos = torch.from_numpy(np.ascontiguousarray(sc["pos"], dtype=np.int32)).to(device)
        ts.append(api.ws_targets(obj, pos, cfg.N, stream=stream))
        del sc, fused
    return torch.cat(xs), torch.cat(ts)


def train(net: api.WsNet, X, T, epochs: int, batch: int, lr: float, seed: int = 0, log_every: int = 0):
    """Adam on shuffled minibatches; returns the per-epoch mean training loss."""
    import torch
    S = X.shape[0]
    gen = torch.Generator(device="cpu").manual_seed(seed)
    history = []
    for ep in range(epochs):
        perm = torch.randperm(S, generator=gen).to(X.device)
        Xp, Tp = X[perm].contiguous(), T[perm].contiguous()
        losses = []
        for i, b0 in enumerate(range(0, S - batch + 1, batch)):
            want = bool(log_every) and i % log_every == 0
            loss = api.wsnet_train_step(net, Xp[b0:b0 + batch], Tp[b0:b0 + batch], lr, loss=want)
            if want:
                losses.append(loss)
        history.append(float(np.mean(losses)) if losses else None)
    return history

def predict(net: api.WsNet, X, batch: int):
    import torch
    out = torch.empty((X.shape[0], net.out_channels, net.out_side, net.out_side), dtype=torch.float32,
                      device=X.device)
    for b0 in range(0, X.shape[0], batch):
        b1 = min(X.shape[0], b0 + batch)
        api.wsnet_forward(net, X[b0:b1].contiguous(), out=out[b0:b1])
    return out


def warm_object(net: api.WsNet, fused, pos, probe, M: int, batch: int | None = None, stream=None):
    """Initial object complex64 [M][M] (device) for a scan: fused float32 [J][N][N] (device),
    pos [J][2] (host or device int32), probe complex64 [N][N] (device)."""
    import torch
    X = api.ws_preprocess(fused, stream=stream)
    pred = predict(net, X, batch or net.max_batch)
    pos_d = torch.as_tensor(np.ascontiguousarray(pos, dtype=np.int32)).to(fused.device) \
        if not isinstance(pos, torch.Tensor) else pos
    return api.ws_stitch(pred, pos_d, probe, M, stream=stream)


def judged_start(fused, pos, probe0, obj_warm, obj_flat, **init_kw):
    """One iteration from each start; keep the handle whose first Fourier error is lower.
    Returns (handle, chosen, errors) with chosen in {"warm", "flat"}; the other handle is
    destroyed."""
    hw = api.ptycho_init(fused, pos, obj_warm, probe0, **init_kw)
    hf = api.ptycho_init(fused, pos, obj_flat, probe0, **init_kw)
    ew = float(api.ptycho_iterate(hw, 1)[0])
    ef = float(api.ptycho_iterate(hf, 1)[0])
    if ew <= ef:
        api.ptycho_destroy(hf)
        return hw, "warm", (ew, ef)
    api.ptycho_destroy(hw)
    return hf, "flat", (ew, ef)
