"""ORACLE -- test infrastructure only.

Plain FP64 numpy reference of the small correction network the library trains on
the GPU (a ReLU MLP F -> H -> H -> 1 with mean-squared-error loss and Adam).  The
paper has no learned part; this is the reference that the GPU forward, backward
and optimiser kernels are checked against (analytic gradients here, and central
finite differences of the loss as the independent pin).

Parameter layout (shared with the library, one flat FP32 vector):
W1 [F x H] row-major, b1 [H], W2 [H x H], b2 [H], W3 [H], b3 [1].
"""
from __future__ import annotations

import numpy as np


def split(theta, F, H):
    theta = np.asarray(theta, dtype=np.float64)
    o = 0
    W1 = theta[o:o + F * H].reshape(F, H); o += F * H
    b1 = theta[o:o + H]; o += H
    W2 = theta[o:o + H * H].reshape(H, H); o += H * H
    b2 = theta[o:o + H]; o += H
    W3 = theta[o:o + H]; o += H
    b3 = theta[o:o + 1]; o += 1
    assert o == theta.size
    return W1, b1, W2, b2, W3, b3


def n_params(F, H):
    return F * H + H + H * H + H + H + 1


def bf16_round(a):
    """Round to the nearest BF16 value (8 significant bits, ties to even), by way
    of FP32 as a device does it; returned as float64."""
    u = np.asarray(a, dtype=np.float32).view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def forward(theta, X, F, H, act_bf16=False):
    """f(x) for every row of X (shape [B, F]).

    act_bf16: the first hidden layer is stored in BF16 before the second layer
    reads it -- the reading of inference on tensor cores, whose operands of the
    64 x 64 layer are BF16 (the network is defined with BF16 weights and
    features already; sums stay exact here)."""
    W1, b1, W2, b2, W3, b3 = split(theta, F, H)
    h1 = np.maximum(X @ W1 + b1, 0.0)
    if act_bf16:
        h1 = bf16_round(h1)
    h2 = np.maximum(h1 @ W2 + b2, 0.0)
    return h2 @ W3 + b3[0]


def loss(theta, X, y, F, H):
    """Mean squared error (1/B) sum (f(x_b) - y_b)^2."""
    r = forward(theta, X, F, H) - y
    return float(np.mean(r * r))


def grad(theta, X, y, F, H):
    """Analytic gradient of ``loss`` by back-propagation, flat like theta."""
    W1, b1, W2, b2, W3, b3 = split(theta, F, H)
    B = X.shape[0]
    z1 = X @ W1 + b1
    h1 = np.maximum(z1, 0.0)
    z2 = h1 @ W2 + b2
    h2 = np.maximum(z2, 0.0)
    out = h2 @ W3 + b3[0]
    d = 2.0 * (out - y) / B
    gW3 = h2.T @ d
    gb3 = np.array([d.sum()])
    dh2 = np.outer(d, W3) * (z2 > 0)
    gW2 = h1.T @ dh2
    gb2 = dh2.sum(axis=0)
    dh1 = (dh2 @ W2.T) * (z1 > 0)
    gW1 = X.T @ dh1
    gb1 = dh1.sum(axis=0)
    return np.concatenate([gW1.ravel(), gb1, gW2.ravel(), gb2, gW3, gb3])


def grad_fd(theta, X, y, F, H, idx, h=1e-6):
    """Central finite differences of the loss for the parameters listed in idx."""
    theta = np.asarray(theta, dtype=np.float64)
    out = np.empty(len(idx))
    for k, p in enumerate(idx):
        tp = theta.copy(); tp[p] += h
        tm = theta.copy(); tm[p] -= h
        out[k] = (loss(tp, X, y, F, H) - loss(tm, X, y, F, H)) / (2 * h)
    return out


def adam(theta, g, m, v, t, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam step (Kingma & Ba): returns the new (theta, m, v); t counts from 1."""
    m = beta1 * m + (1 - beta1) * g
    v = beta2 * v + (1 - beta2) * g * g
    mh = m / (1 - beta1 ** t)
    vh = v / (1 - beta2 ** t)
    return theta - lr * mh / (np.sqrt(vh) + eps), m, v
