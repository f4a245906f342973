"""FP64 reference of the cluster-proposal network -- TEST INFRASTRUCTURE ONLY.

The proposal network is not in the paper; its shape comes from the target
specification: segment end points (6 numbers) -> 128 -> 128 -> 256 cluster
logits, GELU between layers, BF16 weights with FP32 accumulation.  GELU is
taken in its tanh form, one of the two forms its authors give (Hendrycks &
Gimpel, "Gaussian Error Linear Units", 2016): 0.5 z (1 + tanh(sqrt(2/pi)
(z + 0.044715 z^3))); it differs from the erf definition by at most 4.8e-4.  Reading
used here (and by the GPU kernels): the inputs of every layer (features and
hidden activations) and the weights are rounded to BF16; products and sums
are exact-then-rounded in the kernels (FP32) and FP64 here; biases stay
FP32.  Features: each end point normalised by the mesh extent to [-1, 1]
(clamped to [-4, 4]), zero-padded to 16 inputs.

Loss: mean binary cross-entropy with logits over the 256 clusters and the
batch; label c = 1 if the segment meets a triangle of cluster c (cluster =
one of 256 equal ranges of the Morton-ordered leaves).  Optimiser: Adam.
"""
from __future__ import annotations

import math

import numpy as np

D_IN, D_PAD, D_H, D_OUT = 6, 16, 128, 256


def bf16_round(x):
    """Round to the nearest BF16 value (8 significant bits, ties to even),
    directly from FP64, returned as float64."""
    m, e = np.frexp(np.asarray(x, dtype=np.float64))   # x = m 2^e, 0.5 <= |m| < 1
    return np.ldexp(np.round(m * 256.0), e - 8)


GELU_C = math.sqrt(2.0 / math.pi)
GELU_A = 0.044715


def gelu(z):
    """GELU, tanh form: 0.5 z (1 + tanh(c (z + a z^3))), c = sqrt(2 / pi)."""
    return 0.5 * z * (1.0 + np.tanh(GELU_C * (z + GELU_A * z ** 3)))


def gelu_grad(z):
    """d/dz of gelu: 0.5 (1 + t) + 0.5 z (1 - t^2) c (1 + 3 a z^2)."""
    t = np.tanh(GELU_C * (z + GELU_A * z ** 3))
    return 0.5 * (1.0 + t) + 0.5 * z * (1.0 - t * t) * GELU_C * (1.0 + 3.0 * GELU_A * z * z)


def features(ray_from, ray_to, lo, hi):
    """[n, 16] features: both end points mapped by the extent to [-1, 1]."""
    lo = np.asarray(lo, np.float64)
    hi = np.asarray(hi, np.float64)
    span = np.where(hi > lo, hi - lo, 1.0)
    f = np.concatenate([(np.asarray(ray_from, np.float64) - lo) / span, (np.asarray(ray_to, np.float64) - lo) / span], 1)
    f = np.clip(2.0 * f - 1.0, -4.0, 4.0)
    x = np.zeros((len(f), D_PAD))
    x[:, :D_IN] = f
    return x


def init_params(seed: int):
    """He-style normal init (FP32 master copies as float64 arrays)."""
    rng = np.random.default_rng([seed, 0x4D4C50])
    p = {
        "W1": rng.normal(0, math.sqrt(2.0 / D_IN), (D_PAD, D_H)),
        "b1": np.zeros(D_H),
        "W2": rng.normal(0, math.sqrt(2.0 / D_H), (D_H, D_H)),
        "b2": np.zeros(D_H),
        "W3": rng.normal(0, math.sqrt(1.0 / D_H), (D_H, D_OUT)),
        "b3": np.zeros(D_OUT),
    }
    p["W1"][D_IN:] = 0.0
    return {k: v.astype(np.float32).astype(np.float64) for k, v in p.items()}


def forward(p, x):
    """Returns (logits, cache) with BF16 weights and BF16 layer inputs."""
    W1, W2, W3 = (bf16_round(p[k]) for k in ("W1", "W2", "W3"))
    a0 = bf16_round(x)
    z1 = a0 @ W1 + p["b1"]
    a1 = bf16_round(gelu(z1))
    z2 = a1 @ W2 + p["b2"]
    a2 = bf16_round(gelu(z2))
    z3 = a2 @ W3 + p["b3"]
    return z3, dict(a0=a0, z1=z1, a1=a1, z2=z2, a2=a2, W1=W1, W2=W2, W3=W3)


def bce_loss(logits, y):
    """Mean binary cross-entropy with logits."""
    z = logits
    return float(np.mean(np.maximum(z, 0) - z * y + np.log1p(np.exp(-np.abs(z)))))


def backward(p, cache, logits, y):
    """Gradients of the mean BCE loss.  The BF16 roundings are treated as
    identity (straight-through), as the GPU backward does."""
    n = logits.shape[0]
    dz3 = (1.0 / (1.0 + np.exp(-logits)) - y) / (n * D_OUT)
    g = {"W3": cache["a2"].T @ dz3, "b3": dz3.sum(0)}
    da2 = dz3 @ cache["W3"].T
    dz2 = da2 * gelu_grad(cache["z2"])
    g["W2"] = cache["a1"].T @ dz2
    g["b2"] = dz2.sum(0)
    da1 = dz2 @ cache["W2"].T
    dz1 = da1 * gelu_grad(cache["z1"])
    g["W1"] = cache["a0"].T @ dz1
    g["b1"] = dz1.sum(0)
    return g


def adam_step(p, g, state, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam step on the FP32 master weights (state: m, v, t)."""
    t = state.get("t", 0) + 1
    state["t"] = t
    out = {}
    for k in p:
        m = state.setdefault("m_" + k, np.zeros_like(p[k]))
        v = state.setdefault("v_" + k, np.zeros_like(p[k]))
        m[...] = b1 * m + (1 - b1) * g[k]
        v[...] = b2 * v + (1 - b2) * g[k] ** 2
        mh = m / (1 - b1 ** t)
        vh = v / (1 - b2 ** t)
        out[k] = p[k] - lr * mh / (np.sqrt(vh) + eps)
    return out


def top4(logits):
    """Indices of the 4 largest logits per row, largest first (ties: lower
    index first)."""
    order = np.argsort(-logits, axis=1, kind="stable")
    return order[:, :4]
