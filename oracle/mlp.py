"""FP64 oracle of the dimension predictor network -- test infrastructure.

The paper has no learned component; this network maps spectrum features of a
data set to the target dimension its certified search returns.  Architecture:
68 -> 256 -> 256 -> 1 with GELU activations (exact, erf form), mean squared
error on y = log m, Adam (Kingma & Ba 2015) with bias correction.  The
library computes the same network with BF16 weights and FP32 accumulation;
the parity tests feed the oracle the BF16-rounded weights, widened exactly.

Parameter vector layout (shared with the library's set/get calls):
    W1 [256][68], b1 [256], W2 [256][256], b2 [256], w3 [256], b3 [1]

Parity unpinned: the network's accuracy as a predictor (no reference value
exists); only its forward/backward/Adam arithmetic is pinned.
"""
from __future__ import annotations

import math

import numpy as np
from scipy.special import erf

IN, H1, H2 = 68, 256, 256
SIZES = [("W1", (H1, IN)), ("b1", (H1,)), ("W2", (H2, H1)), ("b2", (H2,)), ("w3", (H2,)),
         ("b3", (1,))]
NPARAM = sum(int(np.prod(s)) for _, s in SIZES)


def unpack(vec: np.ndarray) -> dict:
    out, off = {}, 0
    for name, shape in SIZES:
        k = int(np.prod(shape))
        out[name] = np.asarray(vec[off:off + k], dtype=np.float64).reshape(shape)
        off += k
    return out


def pack(p: dict) -> np.ndarray:
    return np.concatenate([np.asarray(p[name], dtype=np.float64).ravel() for name, _ in SIZES])


def gelu(x):
    """GELU(x) = x Phi(x) with the exact normal CDF."""
    return 0.5 * x * (1.0 + erf(x / math.sqrt(2.0)))


def gelu_grad(x):
    """d/dx x Phi(x) = Phi(x) + x phi(x)."""
    return 0.5 * (1.0 + erf(x / math.sqrt(2.0))) + x * np.exp(-0.5 * x * x) / math.sqrt(2.0 * math.pi)


def forward(p: dict, X: np.ndarray):
    X = np.asarray(X, dtype=np.float64)
    z1 = X @ p["W1"].T + p["b1"]
    h1 = gelu(z1)
    z2 = h1 @ p["W2"].T + p["b2"]
    h2 = gelu(z2)
    y = h2 @ p["w3"] + p["b3"][0]
    return y, (X, z1, h1, z2, h2)


def loss_and_grads(p: dict, X: np.ndarray, t: np.ndarray):
    """Mean squared error and its gradient with respect to every parameter."""
    y, (X, z1, h1, z2, h2) = forward(p, X)
    t = np.asarray(t, dtype=np.float64)
    B = X.shape[0]
    r = y - t
    loss = float(np.mean(r * r))
    dy = 2.0 * r / B
    g = {"w3": h2.T @ dy, "b3": np.array([dy.sum()])}
    dz2 = np.outer(dy, p["w3"]) * gelu_grad(z2)
    g["W2"] = dz2.T @ h1
    g["b2"] = dz2.sum(axis=0)
    dz1 = (dz2 @ p["W2"]) * gelu_grad(z1)
    g["W1"] = dz1.T @ X
    g["b1"] = dz1.sum(axis=0)
    return loss, g


def adam_step(vec, grad, m, v, step, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update (step counts from 1); returns new (vec, m, v)."""
    m = beta1 * m + (1.0 - beta1) * grad
    v = beta2 * v + (1.0 - beta2) * grad * grad
    mhat = m / (1.0 - beta1 ** step)
    vhat = v / (1.0 - beta2 ** step)
    return vec - lr * mhat / (np.sqrt(vhat) + eps), m, v


def bf16_round(x: np.ndarray) -> np.ndarray:
    """Round float32 values to bfloat16 (round to nearest even), returned as float64."""
    u = np.ascontiguousarray(x, dtype=np.float32).view(np.uint32).astype(np.uint64)
    r = ((u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000).astype(np.uint32)
    return r.view(np.float32).astype(np.float64)


def with_bf16_weights(vec: np.ndarray) -> dict:
    """The parameters as the library's forward pass sees them: weights in BF16."""
    p = unpack(np.asarray(vec, dtype=np.float32).astype(np.float64))
    for name in ("W1", "W2", "w3"):
        p[name] = bf16_round(p[name])
    return p
