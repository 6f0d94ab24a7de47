"""ORACLE -- test infrastructure only.

FP64 reference of the learned SC/PC selector: an MLP 8 -> 32 -> 32 -> 1 with
ReLU, trained on the mean squared error of y = log(t_PC / t_SC).  Plain numpy,
written step by step so that it can be checked by eye and by finite
differences.  The paper has no learned selector; this is the reference for the
library's own training kernels.

Flat parameter layout (1377 floats): W1[32][8], b1[32], W2[32][32], b2[32], W3[32], b3.
"""
from __future__ import annotations

import numpy as np

F, H = 8, 32
NW = H * F + H + H * H + H + H + 1


def unpack(w):
    w = np.asarray(w, dtype=np.float64)
    o = 0
    W1 = w[o:o + H * F].reshape(H, F); o += H * F
    b1 = w[o:o + H]; o += H
    W2 = w[o:o + H * H].reshape(H, H); o += H * H
    b2 = w[o:o + H]; o += H
    W3 = w[o:o + H]; o += H
    b3 = w[o]
    return W1, b1, W2, b2, W3, b3


def forward(w, X):
    """Returns the prediction for every row of X (already standardised)."""
    W1, b1, W2, b2, W3, b3 = unpack(w)
    X = np.asarray(X, dtype=np.float64)
    h1 = np.maximum(X @ W1.T + b1, 0.0)
    h2 = np.maximum(h1 @ W2.T + b2, 0.0)
    return h2 @ W3 + b3


def loss(w, X, Y):
    r = forward(w, X) - np.asarray(Y, dtype=np.float64)
    return float(np.mean(r * r))


def grad(w, X, Y):
    """Gradient of the mean squared error w.r.t. the flat parameters (backpropagation)."""
    W1, b1, W2, b2, W3, b3 = unpack(w)
    X = np.asarray(X, dtype=np.float64)
    Y = np.asarray(Y, dtype=np.float64)
    n = X.shape[0]
    z1 = X @ W1.T + b1
    h1 = np.maximum(z1, 0.0)
    z2 = h1 @ W2.T + b2
    h2 = np.maximum(z2, 0.0)
    yhat = h2 @ W3 + b3
    e = 2.0 * (yhat - Y) / n                 # dL/dyhat
    gW3 = h2.T @ e
    gb3 = e.sum()
    d2 = np.outer(e, W3) * (z2 > 0)          # dL/dz2
    gW2 = d2.T @ h1
    gb2 = d2.sum(axis=0)
    d1 = (d2 @ W2) * (z1 > 0)                # dL/dz1
    gW1 = d1.T @ X
    gb1 = d1.sum(axis=0)
    return np.concatenate([gW1.ravel(), gb1, gW2.ravel(), gb2, gW3, [gb3]])


def glorot_init(seed_stream: np.ndarray):
    """Glorot-uniform weights from a stream of uniform 64-bit integers (one per weight), zero biases."""
    w = np.zeros(NW)
    u = (seed_stream >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)
    o = 0
    for fan_out, fan_in, off in ((H, F, 0), (H, H, H * F + H), (1, H, H * F + H + H * H + H)):
        a = np.sqrt(6.0 / (fan_in + fan_out))
        m = fan_out * fan_in
        w[off:off + m] = (2.0 * u[off:off + m] - 1.0) * a
    return w
