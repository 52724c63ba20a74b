"""Plain FP64 CPU reference of the learned sub-grid correction network.

TEST INFRASTRUCTURE ONLY (the test suite and the smoke check use it; the GPU
library never does).  The network is not in the paper; it is the small
convolutional correction added to coarse runs: three 3x3 convolutions with
zero padding, 3 -> 32 -> 32 -> 3 channels, ReLU after the first two.

    y[o, i, j] = b[o] + sum_c sum_{u,v in 0..2} w[o, c, u, v] x[c, i+u-1, j+v-1]

Forward and backward are written out directly (np.einsum over shifted views).
`bf16` optionally rounds chosen tensors to bfloat16 (round to nearest even),
so the reference can take the same rounding decisions as the GPU kernels,
which store weights and activations in bfloat16 and accumulate in FP32.
"""
from __future__ import annotations

import numpy as np


def bf16(x: np.ndarray) -> np.ndarray:
    """Round to the nearest bfloat16 (ties to even), returned as float64."""
    f = np.ascontiguousarray(x, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    u = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def conv3x3(x: np.ndarray, w: np.ndarray, b: np.ndarray) -> np.ndarray:
    """x (C, H, W), w (O, C, 3, 3), b (O,) -> (O, H, W), zero padding."""
    C, H, W = x.shape
    xp = np.pad(x, ((0, 0), (1, 1), (1, 1)))
    y = np.zeros((w.shape[0], H, W))
    for u in range(3):
        for v in range(3):
            y += np.einsum("oc,chw->ohw", w[:, :, u, v], xp[:, u:u + H, v:v + W])
    return y + b[:, None, None]


def conv3x3_input_grad(gy: np.ndarray, w: np.ndarray) -> np.ndarray:
    """d/dx of sum(gy * conv3x3(x, w, b)): (O, H, W) -> (C, H, W)."""
    O, H, W = gy.shape
    gp = np.pad(gy, ((0, 0), (1, 1), (1, 1)))
    gx = np.zeros((w.shape[1], H, W))
    for u in range(3):
        for v in range(3):
            # x[c, i+u-1, j+v-1] feeds y[o, i, j]: so gx[c, p, q] gets gy[o, p-u+1, q-v+1]
            gx += np.einsum("oc,ohw->chw", w[:, :, u, v], gp[:, 2 - u:2 - u + H, 2 - v:2 - v + W])
    return gx


def conv3x3_weight_grad(gy: np.ndarray, x: np.ndarray):
    """(d/dw, d/db) of sum(gy * conv3x3(x, w, b))."""
    C, H, W = x.shape
    xp = np.pad(x, ((0, 0), (1, 1), (1, 1)))
    gw = np.zeros((gy.shape[0], C, 3, 3))
    for u in range(3):
        for v in range(3):
            gw[:, :, u, v] = np.einsum("ohw,chw->oc", gy, xp[:, u:u + H, v:v + W])
    return gw, gy.sum(axis=(1, 2))


def forward(x, p, quantize=False):
    """Returns (out, cache).  p: dict w1 b1 w2 b2 w3 b3.  With quantize, the
    input, weights and the two hidden activations are rounded to bfloat16
    where the GPU stores them."""
    q = bf16 if quantize else (lambda a: a)
    w1, w2, w3 = q(p["w1"]), q(p["w2"]), q(p["w3"])
    x0 = q(x)
    h1 = q(np.maximum(conv3x3(x0, w1, p["b1"]), 0.0))
    h2 = q(np.maximum(conv3x3(h1, w2, p["b2"]), 0.0))
    out = conv3x3(h2, w3, p["b3"])
    return out, (x0, h1, h2, w1, w2, w3)


def backward(gout, cache, quantize=False):
    """Gradients of sum(gout * out) w.r.t. the parameters.  With quantize, the
    back-propagated activation gradients are rounded to bfloat16 where the GPU
    stores them."""
    q = bf16 if quantize else (lambda a: a)
    x0, h1, h2, w1, w2, w3 = cache
    g = {}
    g["w3"], g["b3"] = conv3x3_weight_grad(gout, h2)
    gh2 = q(conv3x3_input_grad(q(gout), w3) * (h2 > 0))
    g["w2"], g["b2"] = conv3x3_weight_grad(gh2, h1)
    gh1 = q(conv3x3_input_grad(gh2, w2) * (h1 > 0))
    g["w1"], g["b1"] = conv3x3_weight_grad(gh1, x0)
    return g


def mse(out, target):
    d = out - target
    return float(np.mean(d * d)), 2.0 * d / d.size


def init_params(seed: int, c_hidden: int = 32, scale: float = 1.0):
    """He-style initial weights (seeded), zero biases."""
    rng = np.random.default_rng(seed)
    p = {}
    for k, (o, c) in enumerate([(c_hidden, 3), (c_hidden, c_hidden), (3, c_hidden)], start=1):
        std = scale * np.sqrt(2.0 / (9 * c))
        p[f"w{k}"] = rng.normal(0.0, std, size=(o, c, 3, 3))
        p[f"b{k}"] = np.zeros(o)
    p["w3"] *= 0.1
    return p
