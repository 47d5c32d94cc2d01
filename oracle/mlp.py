"""Float64 oracle of the level predictor's training (test infrastructure only).

The learned level predictor is an addition to the paper's method (Sec. 3.2.1 allocates every new block at the finest
level). This module is the plain reference its GPU training kernels are checked against: the network
16 -> 64 -> 64 -> 3 with GELU, softmax cross-entropy averaged over the batch, the gradient of that loss by the chain
rule written out layer by layer, and one Adam step, all in float64 numpy with the exact erf.

``act_round=True`` rounds the two hidden activations to BF16 in the forward pass, as the GPU network does, and takes
the derivative of each rounding as 1 (straight-through); the GPU gradient is compared with that variant. Without it
the loss is a smooth function of the weights, and its gradient is pinned against central differences.

Parameter vector layout (shared definition with the C ABI, restated): W1 [16][64] input-major, b1 [64], W2 [64][64],
b2 [64], W3 [64][3], b3 [3]; 5443 values.
"""
from __future__ import annotations

import numpy as np
from scipy.special import erf

N_IN, N_HID, N_OUT = 16, 64, 3
SHAPES = [("W1", (N_IN, N_HID)), ("b1", (N_HID,)), ("W2", (N_HID, N_HID)), ("b2", (N_HID,)), ("W3", (N_HID, N_OUT)),
          ("b3", (N_OUT,))]
N_PARAMS = sum(int(np.prod(s)) for _, s in SHAPES)


def unpack(theta: np.ndarray) -> dict:
    out, o = {}, 0
    for name, shape in SHAPES:
        k = int(np.prod(shape))
        out[name] = np.asarray(theta[o:o + k], dtype=np.float64).reshape(shape)
        o += k
    return out


def pack(p: dict) -> np.ndarray:
    return np.concatenate([np.asarray(p[name], dtype=np.float64).reshape(-1) for name, _ in SHAPES])


def bf16_round(x: np.ndarray) -> np.ndarray:
    """Nearest BF16 value (ties to even) of each element, via its float32 value."""
    f = np.asarray(x, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    finite = (u & 0x7F800000) != 0x7F800000
    r = ((u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000).astype(np.uint32)
    out = np.where(finite, r, u.astype(np.uint32)).astype(np.uint32).view(np.float32)
    return out.astype(np.float64)


def bf16_bits(x: np.ndarray) -> np.ndarray:
    """BF16 bit patterns (uint16) of the BF16-rounded values of x."""
    return (bf16_round(x).astype(np.float32).view(np.uint32) >> 16).astype(np.uint16)


def from_bf16_bits(b: np.ndarray) -> np.ndarray:
    return (np.asarray(b, dtype=np.uint16).astype(np.uint32) << 16).view(np.float32).astype(np.float64)


def gelu(a: np.ndarray) -> np.ndarray:
    """x Phi(x) = x (1 + erf(x / sqrt 2)) / 2."""
    return 0.5 * a * (1.0 + erf(a / np.sqrt(2.0)))


def gelu_prime(a: np.ndarray) -> np.ndarray:
    """Phi(x) + x phi(x)."""
    return 0.5 * (1.0 + erf(a / np.sqrt(2.0))) + a * np.exp(-0.5 * a * a) / np.sqrt(2.0 * np.pi)


def forward(theta: np.ndarray, x: np.ndarray, act_round: bool = False) -> dict:
    """Pre-activations, activations and logits for a batch x (n, 16)."""
    p = unpack(theta)
    x = np.asarray(x, dtype=np.float64)
    a1 = x @ p["W1"] + p["b1"]
    h1 = gelu(a1)
    if act_round:
        h1 = bf16_round(h1)
    a2 = h1 @ p["W2"] + p["b2"]
    h2 = gelu(a2)
    if act_round:
        h2 = bf16_round(h2)
    z = h2 @ p["W3"] + p["b3"]
    return dict(x=x, a1=a1, h1=h1, a2=a2, h2=h2, z=z)


def loss(theta: np.ndarray, x: np.ndarray, y: np.ndarray, act_round: bool = False) -> float:
    """Mean softmax cross-entropy: mean_i (log sum_c exp z_ic - z_iy_i)."""
    z = forward(theta, x, act_round)["z"]
    zmax = z.max(axis=1, keepdims=True)
    lse = zmax[:, 0] + np.log(np.exp(z - zmax).sum(axis=1))
    return float(np.mean(lse - z[np.arange(len(y)), y]))


def loss_and_grad(theta: np.ndarray, x: np.ndarray, y: np.ndarray, act_round: bool = False):
    """Loss and its gradient with respect to theta (same layout), by back-propagation."""
    f = forward(theta, x, act_round)
    p = unpack(theta)
    n = x.shape[0]
    z = f["z"]
    e = np.exp(z - z.max(axis=1, keepdims=True))
    prob = e / e.sum(axis=1, keepdims=True)
    onehot = np.zeros_like(z)
    onehot[np.arange(n), y] = 1.0
    dz = (prob - onehot) / n                           # d loss / d logits
    g = {"W3": f["h2"].T @ dz, "b3": dz.sum(axis=0)}
    da2 = (dz @ p["W3"].T) * gelu_prime(f["a2"])      # through h2 = GELU(a2)
    g["W2"] = f["h1"].T @ da2
    g["b2"] = da2.sum(axis=0)
    da1 = (da2 @ p["W2"].T) * gelu_prime(f["a1"])     # through h1 = GELU(a1)
    g["W1"] = f["x"].T @ da1
    g["b1"] = da1.sum(axis=0)
    lse = np.log(e.sum(axis=1)) + z.max(axis=1)
    return float(np.mean(lse - z[np.arange(n), y])), pack(g)


def adam_step(theta, m1, m2, grad, step: int, lr: float, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update (Kingma & Ba, Algorithm 1) with bias correction; step counts from 1."""
    m1 = beta1 * m1 + (1.0 - beta1) * grad
    m2 = beta2 * m2 + (1.0 - beta2) * grad * grad
    mh = m1 / (1.0 - beta1 ** step)
    vh = m2 / (1.0 - beta2 ** step)
    return theta - lr * mh / (np.sqrt(vh) + eps), m1, m2


def init_params(seed: int, scale: float = 1.0) -> np.ndarray:
    """He-style random initial weights (normal, std sqrt(2 / fan_in) times scale), zero biases."""
    rng = np.random.default_rng(seed)
    p = {}
    for name, shape in SHAPES:
        if name.startswith("W"):
            p[name] = rng.standard_normal(shape) * np.sqrt(2.0 / shape[0]) * scale
        else:
            p[name] = np.zeros(shape)
    return pack(p)
