"""FP64 reference of the cost model's perceptron (oracle, test-only).

h1 = relu(x W1 + b1), h2 = relu(h1 W2 + b2), y = h2 W3 + b3, loss = mean
(y - t)^2, with the weights rounded to BF16 (round to nearest even) as the
device model uses them.  Gradients by hand-written backpropagation; pinned by
tests/test_oracle_mlp.py against central finite differences of ``loss``.
"""
from __future__ import annotations

import numpy as np


def bf16_round(w: np.ndarray) -> np.ndarray:
    """Round FP32 values to BF16 (nearest, ties to even) and return FP64."""
    u = np.ascontiguousarray(w, dtype=np.float32).view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) >> 16 << 16
    return (u.astype(np.uint32)).view(np.float32).astype(np.float64)


def unpack(p: np.ndarray, din: int, hid: int):
    p = np.asarray(p, dtype=np.float64)
    o = 0
    W1 = p[o:o + din * hid].reshape(din, hid); o += din * hid
    b1 = p[o:o + hid]; o += hid
    W2 = p[o:o + hid * hid].reshape(hid, hid); o += hid * hid
    b2 = p[o:o + hid]; o += hid
    W3 = p[o:o + hid].reshape(hid, 1); o += hid
    b3 = p[o:o + 1]; o += 1
    assert o == p.size
    return W1, b1, W2, b2, W3, b3


def forward(params, x, din, hid, round_weights=True):
    W1, b1, W2, b2, W3, b3 = unpack(params, din, hid)
    if round_weights:
        W1, W2, W3 = bf16_round(W1), bf16_round(W2), bf16_round(W3)
    x = np.asarray(x, dtype=np.float64)
    z1 = x @ W1 + b1
    a1 = np.maximum(z1, 0.0)
    z2 = a1 @ W2 + b2
    a2 = np.maximum(z2, 0.0)
    y = (a2 @ W3).ravel() + b3[0]
    return y, (x, z1, a1, z2, a2, W1, W2, W3)


def loss(params, x, t, din, hid, round_weights=True):
    y, _ = forward(params, x, din, hid, round_weights)
    return float(np.mean((y - np.asarray(t, dtype=np.float64)) ** 2))


def gradients(params, x, t, din, hid, round_weights=True):
    """d loss / d params (same flat layout), derivatives taken with respect to
    the master parameters through the (straight-through) BF16 rounding."""
    y, (x, z1, a1, z2, a2, W1, W2, W3) = forward(params, x, din, hid, round_weights)
    B = x.shape[0]
    dy = 2.0 * (y - np.asarray(t, dtype=np.float64)) / B
    dW3 = a2.T @ dy[:, None]
    db3 = np.array([dy.sum()])
    da2 = dy[:, None] @ W3.T
    dz2 = da2 * (z2 > 0)
    dW2 = a1.T @ dz2
    db2 = dz2.sum(axis=0)
    da1 = dz2 @ W2.T
    dz1 = da1 * (z1 > 0)
    dW1 = x.T @ dz1
    db1 = dz1.sum(axis=0)
    return np.concatenate([dW1.ravel(), db1, dW2.ravel(), db2, dW3.ravel(), db3])
