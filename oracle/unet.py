"""Oracle: the learned warm start's network (a small U-Net) and its gradients.

Test infrastructure only (see ``oracle/__init__``).

The paper's method has no network; the learned warm start maps the step-one
image and the long-baseline dirty image [i^_L, i~_H1] to a starting image x0
for step two (Sect. 3.3), whose FISTA run then starts from alpha_0 = W^H x0 / M
and still runs to its own tolerance, so the network only changes the starting
point.  This module defines that network plainly, in FP64 numpy, as the
reference for the CUDA kernels:

* layout: images are [H, W, C] arrays (channels last);
* conv3x3: zero-padded 'same' cross-correlation,
  y[p, co] = b[co] + sum_{dy, dx in -1..1} sum_ci w[co, dy+1, dx+1, ci] x[p + (dy, dx), ci];
* encoder level l (l < levels - 1): conv3x3 + ReLU, conv3x3 + ReLU, its output
  is the skip s_l, then 2x2 average pooling;
* bottom level: conv3x3 + ReLU, conv3x3 + ReLU;
* decoder level l: nearest-neighbour 2x upsampling of the level below,
  concatenation [up, s_l] along channels, conv3x3 + ReLU, conv3x3 + ReLU;
* head: conv3x3 to one channel, plus the first input channel (the step-one
  image), so the network learns a correction to it.
Widths: C 2^l channels at level l.

Mixed precision (optional, `quantize=True`) follows the CUDA path's rounding
points exactly: inputs, weights and every stored activation (after ReLU and
after pooling) are rounded to bfloat16 (round to nearest even); the head's
output is not; in the backward pass every pre-activation gradient is rounded
to bfloat16 before it enters a product.  Sums are exact here (FP64); the CUDA
path accumulates in FP32.
"""
from __future__ import annotations

from dataclasses import dataclass
from typing import Dict, List

import numpy as np


# ---------------------------------------------------------------------------
# bfloat16 rounding (round to nearest, ties to even, of the FP32 value)
# ---------------------------------------------------------------------------
def bf16(x: np.ndarray) -> np.ndarray:
    """Round to the nearest bfloat16 (the upper 16 bits of an IEEE float32,
    ties to even); returned as float64."""
    f = np.ascontiguousarray(np.asarray(x, dtype=np.float32))
    u = f.view(np.uint32).astype(np.uint64)
    lsb = (u >> 16) & 1
    r = ((u + 0x7FFF + lsb) >> 16) << 16
    return r.astype(np.uint32).view(np.float32).astype(np.float64)


# ---------------------------------------------------------------------------
# layers
# ---------------------------------------------------------------------------
def conv3x3(x: np.ndarray, w: np.ndarray, b: np.ndarray) -> np.ndarray:
    """'same' cross-correlation; x [H, W, Ci], w [Co, 3, 3, Ci], b [Co]."""
    H, W, _ = x.shape
    xp = np.pad(x, ((1, 1), (1, 1), (0, 0)))
    y = np.broadcast_to(b, (H, W, w.shape[0])).astype(np.float64).copy()
    for ky in range(3):
        for kx in range(3):
            y += xp[ky:ky + H, kx:kx + W, :] @ w[:, ky, kx, :].T
    return y


def conv3x3_grad_input(g: np.ndarray, w: np.ndarray) -> np.ndarray:
    """Adjoint of conv3x3 in x: dx[p, ci] = sum_taps sum_co g[p - tap, co] w[co, tap, ci]."""
    H, W, _ = g.shape
    dx = np.zeros((H, W, w.shape[3]))
    gp = np.pad(g, ((1, 1), (1, 1), (0, 0)))
    for ky in range(3):
        for kx in range(3):
            # output p - (ky - 1, kx - 1) read input p through tap (ky, kx)
            dx += gp[2 - ky:2 - ky + H, 2 - kx:2 - kx + W, :] @ w[:, ky, kx, :]
    return dx


def conv3x3_grad_weight(x: np.ndarray, g: np.ndarray) -> np.ndarray:
    """dw[co, tap, ci] = sum_p g[p, co] x[p + tap, ci]."""
    H, W, ci = x.shape
    xp = np.pad(x, ((1, 1), (1, 1), (0, 0)))
    dw = np.zeros((g.shape[2], 3, 3, ci))
    g2 = g.reshape(H * W, -1)
    for ky in range(3):
        for kx in range(3):
            dw[:, ky, kx, :] = g2.T @ xp[ky:ky + H, kx:kx + W, :].reshape(H * W, ci)
    return dw


def avgpool2(x: np.ndarray) -> np.ndarray:
    H, W, C = x.shape
    return x.reshape(H // 2, 2, W // 2, 2, C).mean(axis=(1, 3))


def avgpool2_grad(g: np.ndarray) -> np.ndarray:
    return np.repeat(np.repeat(g, 2, axis=0), 2, axis=1) / 4.0


def upsample2(x: np.ndarray) -> np.ndarray:
    return np.repeat(np.repeat(x, 2, axis=0), 2, axis=1)


def upsample2_grad(g: np.ndarray) -> np.ndarray:
    H, W, C = g.shape
    return g.reshape(H // 2, 2, W // 2, 2, C).sum(axis=(1, 3))


# ---------------------------------------------------------------------------
# the network
# ---------------------------------------------------------------------------
@dataclass
class UNetSpec:
    levels: int = 3
    width: int = 16
    in_channels: int = 2

    def conv_shapes(self) -> List[tuple]:
        """(c_out, c_in) of every conv, in execution order."""
        C, L = self.width, self.levels
        shapes = []
        cin = self.in_channels
        for lv in range(L):                      # encoder and bottom
            c = C << lv
            shapes += [(c, cin), (c, c)]
            cin = c
        for lv in range(L - 2, -1, -1):          # decoder
            c = C << lv
            shapes += [(c, (C << (lv + 1)) + c), (c, c)]
        shapes.append((1, C))                    # head
        return shapes


def init_params(spec: UNetSpec, rng: np.random.Generator) -> List[Dict[str, np.ndarray]]:
    """He-normal weights, zero biases."""
    out = []
    for co, ci in spec.conv_shapes():
        std = np.sqrt(2.0 / (9 * ci))
        out.append({"w": rng.standard_normal((co, 3, 3, ci)) * std, "b": np.zeros(co)})
    return out


def forward(spec: UNetSpec, params, x: np.ndarray, quantize: bool = False):
    """x [H, W, 2] -> (y [H, W], cache for backward)."""
    q = bf16 if quantize else (lambda a: a)
    L = spec.levels
    convs = iter(range(len(params)))
    cache = {"acts": [], "skips": [], "x": x}

    def conv_relu(a):
        i = next(convs)
        w = q(params[i]["w"])
        z = conv3x3(a, w, params[i]["b"])
        out = q(np.maximum(z, 0.0))
        cache["acts"].append((i, a, out))
        return out

    a = q(x)
    for lv in range(L):
        a = conv_relu(a)
        a = conv_relu(a)
        if lv < L - 1:
            cache["skips"].append(a)
            a = q(avgpool2(a))
    for lv in range(L - 2, -1, -1):
        a = np.concatenate([upsample2(a), cache["skips"][lv]], axis=2)
        a = conv_relu(a)
        a = conv_relu(a)
    i = next(convs)
    w = q(params[i]["w"])
    y = conv3x3(a, w, params[i]["b"])[:, :, 0] + x[:, :, 0]
    cache["head_in"] = (i, a)
    return y, cache


def loss(y: np.ndarray, target: np.ndarray) -> float:
    """Mean squared error over pixels."""
    return float(np.mean((y - target) ** 2))


def backward(spec: UNetSpec, params, cache, y: np.ndarray, target: np.ndarray,
             quantize: bool = False):
    """Gradients of the mean squared error: list of {"w", "b"} like params."""
    q = bf16 if quantize else (lambda a: a)
    L = spec.levels
    grads = [None] * len(params)
    H, W = y.shape
    g = (2.0 / (H * W)) * (y - target)
    i, a = cache["head_in"]
    gz = q(g[:, :, None])
    wq = q(params[i]["w"])
    grads[i] = {"w": conv3x3_grad_weight(a, gz), "b": gz.sum(axis=(0, 1))}
    ga = conv3x3_grad_input(gz, wq)
    acts = list(cache["acts"])

    def conv_relu_back(ga):
        i, a_in, out = acts.pop()
        gz = q(ga * (out > 0))
        wq = q(params[i]["w"])
        grads[i] = {"w": conv3x3_grad_weight(a_in, gz), "b": gz.sum(axis=(0, 1))}
        return conv3x3_grad_input(gz, wq)

    skip_grads = [None] * (L - 1)
    for lv in range(0, L - 1):                    # decoder, last level first
        ga = conv_relu_back(ga)
        ga = conv_relu_back(ga)
        c_up = ga.shape[2] - cache["skips"][lv].shape[2]
        skip_grads[lv] = ga[:, :, c_up:]
        ga = upsample2_grad(ga[:, :, :c_up])
    for lv in range(L - 1, -1, -1):               # bottom and encoder
        if lv < L - 1:
            ga = avgpool2_grad(ga) + skip_grads[lv]
        ga = conv_relu_back(ga)
        ga = conv_relu_back(ga)
    return grads


def adam_step(params, grads, state, lr: float, beta1: float = 0.9, beta2: float = 0.999,
              eps: float = 1e-8):
    """One Adam update (Kingma and Ba, 2015) of the FP64 master weights."""
    state["t"] = state.get("t", 0) + 1
    t = state["t"]
    for k, (p, g) in enumerate(zip(params, grads)):
        for name in ("w", "b"):
            m = state.setdefault(("m", k, name), np.zeros_like(p[name]))
            v = state.setdefault(("v", k, name), np.zeros_like(p[name]))
            m[...] = beta1 * m + (1 - beta1) * g[name]
            v[...] = beta2 * v + (1 - beta2) * g[name] ** 2
            mh = m / (1 - beta1 ** t)
            vh = v / (1 - beta2 ** t)
            p[name] = p[name] - lr * mh / (np.sqrt(vh) + eps)
