"""Training and evaluation helpers for the learned level predictor (an addition to the paper's method).

The predictor is trained on the GPU by the library's own kernels (``Mlp``: BF16 forward / backward, FP32 Adam). Its
training set comes from the library as well: a map run with the plain variance rule records the features of every new
block (``Map.set_feature_capture``), and each record is labelled with the level its block holds at the end of the
run. This module only joins keys to labels, draws minibatches and loops; no step of the map's per-frame path runs
here.
"""
from __future__ import annotations

import numpy as np

from . import MLP_HIDDEN, MLP_IN, MLP_LEVELS, MLP_PARAMS, Mlp


def init_weights(seed: int) -> np.ndarray:
    """He-normal weights (std sqrt(2 / fan_in)), zero biases, packed W1, b1, W2, b2, W3, b3; float32."""
    rng = np.random.default_rng(seed)
    parts = []
    for fan_in, fan_out in ((MLP_IN, MLP_HIDDEN), (MLP_HIDDEN, MLP_HIDDEN), (MLP_HIDDEN, MLP_LEVELS)):
        parts.append(rng.standard_normal(fan_in * fan_out) * np.sqrt(2.0 / fan_in))
        parts.append(np.zeros(fan_out))
    w = np.concatenate(parts).astype(np.float32)
    assert w.size == MLP_PARAMS
    return w


def constant_level_weights(level: int) -> np.ndarray:
    """BF16 bit patterns of a network that answers `level` for every input: zero weights, output bias 4 at `level`.
    Set as a map's predictor it starts every new block at that level (the bound a perfect "go coarse" predictor can
    reach at most)."""
    w = np.zeros(MLP_PARAMS, dtype=np.uint16)
    w[MLP_PARAMS - MLP_LEVELS + level] = 0x4080  # 4.0 in BF16
    return w


def _packed(keys: np.ndarray) -> np.ndarray:
    k = np.asarray(keys, dtype=np.int64) + (1 << 20)
    return (k[:, 0] << 42) | (k[:, 1] << 21) | k[:, 2]


def level_labels(captured_keys: np.ndarray, map_keys: np.ndarray, map_levels: np.ndarray) -> np.ndarray:
    """Level each captured block holds in the map (map_keys sorted by key, as extracted); -1 if it is absent."""
    ck, mk = _packed(captured_keys), _packed(map_keys)
    pos = np.searchsorted(mk, ck)
    pos_c = np.minimum(pos, max(len(mk) - 1, 0))
    found = (len(mk) > 0) & (mk[pos_c] == ck) if len(mk) else np.zeros(len(ck), bool)
    return np.where(found, np.asarray(map_levels, dtype=np.int64)[pos_c], -1).astype(np.int32)


def train(x, y, epochs: int = 20, batch: int = 4096, lr: float = 1e-3, seed: int = 0, device: int = 0,
          init: np.ndarray | None = None):
    """Train on features x (n, 16) float32 and labels y (n,) int32 (CUDA tensors). Returns (Mlp, per-epoch mean
    loss). Minibatches are drawn by a seeded permutation each epoch."""
    import torch
    net = Mlp(init_weights(seed) if init is None else init, device)
    n = x.shape[0]
    gen = torch.Generator(device=x.device)
    gen.manual_seed(seed)
    loss_buf = torch.zeros(max(1, (n + batch - 1) // batch), dtype=torch.float32, device=x.device)
    history = []
    for _ in range(epochs):
        perm = torch.randperm(n, generator=gen, device=x.device)
        xs, ys = x[perm].contiguous(), y[perm].contiguous()
        nb = 0
        for s in range(0, n, batch):
            e = min(n, s + batch)
            net.train_step(xs[s:e], ys[s:e], lr, loss_buf[nb:nb + 1])
            nb += 1
        history.append(float(loss_buf[:nb].mean().item()))
    return net, history


def predicted_levels(net: Mlp, x, n_levels: int = 3):
    """First-argmax level of each sample, clamped to n_levels - 1 (as the map applies it); int32 CUDA tensor."""
    import torch
    return net.predict(x).argmax(dim=1).clamp(max=n_levels - 1).to(torch.int32)
