"""FP64 reference of the router network (TEST INFRASTRUCTURE ONLY).

The router of the library is an MLP d -> 64 -> 64 -> 64 with ReLU hidden
layers and a softmax cross-entropy loss over 64 buckets.  This module holds
the plain definition, in numpy float64, that the GPU forward and backward
kernels are checked against: parameters packed as W1[64][d], b1[64],
W2[64][64], b2[64], W3[64][64], b3[64]; loss = mean over the batch of
log(sum_o exp(l_o)) - l_y.  It is pinned by central finite differences and by
the closed form of the zero network (loss = ln 64) in tests/test_oracle_pins.py.
"""
from __future__ import annotations

import numpy as np

H = 64
K = 64


def unpack(P: np.ndarray, d: int):
    P = np.asarray(P, dtype=np.float64)
    o = 0
    W1 = P[o:o + H * d].reshape(H, d); o += H * d
    b1 = P[o:o + H]; o += H
    W2 = P[o:o + H * H].reshape(H, H); o += H * H
    b2 = P[o:o + H]; o += H
    W3 = P[o:o + K * H].reshape(K, H); o += K * H
    b3 = P[o:o + K]; o += K
    assert o == P.size
    return W1, b1, W2, b2, W3, b3


def count(d: int) -> int:
    return H * d + H + H * H + H + K * H + K


def forward(P, Z):
    """Logits [B, 64] of the inputs Z [B, d]."""
    Z = np.asarray(Z, dtype=np.float64)
    W1, b1, W2, b2, W3, b3 = unpack(P, Z.shape[1])
    h1 = np.maximum(Z @ W1.T + b1, 0.0)
    h2 = np.maximum(h1 @ W2.T + b2, 0.0)
    return h2 @ W3.T + b3


def loss(P, Z, y) -> float:
    lg = forward(P, Z)
    mx = lg.max(axis=1, keepdims=True)
    lse = np.log(np.exp(lg - mx).sum(axis=1)) + mx[:, 0]
    return float(np.mean(lse - lg[np.arange(len(y)), y]))


def loss_and_grad(P, Z, y):
    """Mean cross-entropy and its gradient with respect to the packed parameters."""
    Z = np.asarray(Z, dtype=np.float64)
    y = np.asarray(y)
    B, d = Z.shape
    W1, b1, W2, b2, W3, b3 = unpack(P, d)
    a1 = Z @ W1.T + b1
    h1 = np.maximum(a1, 0.0)
    a2 = h1 @ W2.T + b2
    h2 = np.maximum(a2, 0.0)
    lg = h2 @ W3.T + b3
    mx = lg.max(axis=1, keepdims=True)
    e = np.exp(lg - mx)
    s = e.sum(axis=1, keepdims=True)
    p = e / s
    L = float(np.mean(np.log(s[:, 0]) + mx[:, 0] - lg[np.arange(B), y]))
    dl = p.copy()
    dl[np.arange(B), y] -= 1.0
    dl /= B
    gW3 = dl.T @ h2
    gb3 = dl.sum(axis=0)
    d2 = (dl @ W3) * (a2 > 0)
    gW2 = d2.T @ h1
    gb2 = d2.sum(axis=0)
    d1 = (d2 @ W2) * (a1 > 0)
    gW1 = d1.T @ Z
    gb1 = d1.sum(axis=0)
    return L, np.concatenate([gW1.ravel(), gb1, gW2.ravel(), gb2, gW3.ravel(), gb3])
