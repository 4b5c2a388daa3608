"""CPU FP64 reference of the learned pair scheduler's network.

TEST INFRASTRUCTURE ONLY: the gradient oracle of the GPU training kernels;
only the test suite calls it.

Network: 6 inputs -> 32 ReLU -> 32 ReLU -> 1 logit, mean binary cross-entropy
with logits.  Parameter layout (flat, 1313 values): W1[32][6], b1[32],
W2[32][32], b2[32], w3[32], b3.  The gradient is the textbook backward pass
(chain rule layer by layer), written out with numpy.
"""
from __future__ import annotations

import numpy as np

F, H = 6, 32
SIZES = [("W1", (H, F)), ("b1", (H,)), ("W2", (H, H)), ("b2", (H,)), ("w3", (H,)), ("b3", (1,))]
NPARAM = sum(int(np.prod(s)) for _, s in SIZES)


def unpack(w):
    w = np.asarray(w, dtype=np.float64)
    out, at = {}, 0
    for name, shape in SIZES:
        k = int(np.prod(shape))
        out[name] = w[at:at + k].reshape(shape)
        at += k
    return out


def forward(w, X):
    p = unpack(w)
    X = np.asarray(X, dtype=np.float64)
    a1 = X @ p["W1"].T + p["b1"]
    h1 = np.maximum(a1, 0.0)
    a2 = h1 @ p["W2"].T + p["b2"]
    h2 = np.maximum(a2, 0.0)
    z = h2 @ p["w3"] + p["b3"][0]
    return z, (X, a1, h1, a2, h2)


def loss(w, X, y):
    z, _ = forward(w, X)
    y = np.asarray(y, dtype=np.float64)
    return float(np.mean(np.maximum(z, 0) - z * y + np.log1p(np.exp(-np.abs(z)))))


def loss_grad(w, X, y):
    """Mean BCE-with-logits loss and its gradient (flat, parameter layout)."""
    p = unpack(w)
    z, (X, a1, h1, a2, h2) = forward(w, X)
    y = np.asarray(y, dtype=np.float64)
    n = len(y)
    L = float(np.mean(np.maximum(z, 0) - z * y + np.log1p(np.exp(-np.abs(z)))))
    dz = (1.0 / (1.0 + np.exp(-z)) - y) / n           # dL/dz
    g_w3 = h2.T @ dz
    g_b3 = np.array([dz.sum()])
    d2 = np.outer(dz, p["w3"]) * (a2 > 0)             # dL/da2
    g_W2 = d2.T @ h1
    g_b2 = d2.sum(0)
    d1 = (d2 @ p["W2"]) * (a1 > 0)                    # dL/da1
    g_W1 = d1.T @ X
    g_b1 = d1.sum(0)
    g = np.concatenate([g_W1.ravel(), g_b1, g_W2.ravel(), g_b2, g_w3, g_b3])
    return L, g
