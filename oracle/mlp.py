"""Plain numpy reference of the learned proposal's features and MLP.

TEST INFRASTRUCTURE ONLY: the tests compare the CUDA kernels (mlp.cu) with
this; the product never imports it.  Binary64 arithmetic on the BF16 values
of the weights (the kernels accumulate in binary32, so the comparison has a
tolerance), except the features, which are recomputed in binary32 with the
same operations as the kernel (so they compare exactly).

Features: a 32 x 32 occupancy grid of a sample of m = min(n, 4096) points
(indices floor(j n / m)) over the sample's bounding box, as fractions of m.
MLP: 1024 -> 64 -> 64 -> 68, ReLU between; loss: softmax cross-entropy of
the 4 K-logits plus lam * mask * mean squared error of the 64 offsets, both
averaged over the batch; Adam (0.9, 0.999, 1e-8) with bias correction.
"""
from __future__ import annotations

import numpy as np

GRID, IN, HID, OUT, SAMPLE = 32, 1024, 64, 68, 4096
SHAPES = (("W1", (HID, IN)), ("b1", (HID,)), ("W2", (HID, HID)), ("b2", (HID,)), ("W3", (OUT, HID)), ("b3", (OUT,)))
N_PARAMS = sum(int(np.prod(s)) for _, s in SHAPES)


def bf16_round(a) -> np.ndarray:
    """binary32 -> nearest BF16 (ties to even), returned as binary32."""
    u = np.ascontiguousarray(a, np.float32).view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32)


def split(params):
    """Parameter views (binary64) in the kernels' row-major order."""
    p = np.asarray(params, np.float64)
    out, o = {}, 0
    for name, shape in SHAPES:
        k = int(np.prod(shape))
        out[name] = p[o:o + k].reshape(shape)
        o += k
    return out


def features(points) -> np.ndarray:
    p = np.ascontiguousarray(points, np.float32).reshape(-1, 2)
    n = p.shape[0]
    m = min(n, SAMPLE)
    idx = (np.arange(m, dtype=np.int64) * n) // m
    x, y = p[idx, 0], p[idx, 1]
    x0, x1, y0, y1 = x.min(), x.max(), y.min(), y.max()
    w, h = np.float32(x1 - x0), np.float32(y1 - y0)
    sx = np.float32(32) / w if w > 0 else np.float32(0)
    sy = np.float32(32) / h if h > 0 else np.float32(0)
    cx = np.minimum(GRID - 1, np.floor((x - x0) * sx).astype(np.int64))
    cy = np.minimum(GRID - 1, np.floor((y - y0) * sy).astype(np.int64))
    cnt = np.bincount(cy * GRID + cx, minlength=IN).astype(np.float32)
    return cnt * (np.float32(1) / np.float32(m))


def forward(X, params):
    P = split(params)
    X = np.asarray(X, np.float64)
    h1 = np.maximum(X @ P["W1"].T + P["b1"], 0.0)
    h2 = np.maximum(h1 @ P["W2"].T + P["b2"], 0.0)
    return h1, h2, h2 @ P["W3"].T + P["b3"]


def loss_grad(out, label, off, mask, lam):
    """Per-sample losses and d(mean loss)/d(out)."""
    B = out.shape[0]
    z = out[:, :4] - out[:, :4].max(1, keepdims=True)
    e = np.exp(z)
    sm = e / e.sum(1, keepdims=True)
    loss = -np.log(sm[np.arange(B), label])
    d = np.zeros_like(out)
    d[:, :4] = sm
    d[np.arange(B), label] -= 1.0
    diff = out[:, 4:] - off
    w = lam * np.asarray(mask, np.float64)[:, None]
    loss = loss + (w * diff * diff).sum(1) / 64.0
    d[:, 4:] = w * 2.0 * diff / 64.0
    return loss, d / B


def grads(X, params, label, off, mask, lam):
    """(per-sample losses, gradient of the batch-mean loss) in the kernels'
    parameter order."""
    P = split(params)
    X = np.asarray(X, np.float64)
    h1, h2, out = forward(X, params)
    loss, d3 = loss_grad(out, label, off, mask, lam)
    d2 = (d3 @ P["W3"]) * (h2 > 0)
    d1 = (d2 @ P["W2"]) * (h1 > 0)
    g = [d1.T @ X, d1.sum(0), d2.T @ h1, d2.sum(0), d3.T @ h2, d3.sum(0)]
    return loss, np.concatenate([a.ravel() for a in g])


def adam(master, g, m, v, step, lr, b1=0.9, b2=0.999, eps=1e-8):
    m = b1 * m + (1 - b1) * g
    v = b2 * v + (1 - b2) * g * g
    w = master - lr * (m / (1 - b1 ** step)) / (np.sqrt(v / (1 - b2 ** step)) + eps)
    return w, m, v
