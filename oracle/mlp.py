"""Oracle for the learned cost model: the same MLP in plain FP64 NumPy.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py). Forward pass
x -> relu(W1 x + b1) -> relu(W2 a1 + b2) -> W3 a2 + b3, loss = mean (y - t)^2,
and its gradient by the chain rule written out layer by layer. Parameters use
the library's flat layout: W1 [h1][n_in], b1 [h1], W2 [h2][h1], b2 [h2],
W3 [h2], b3.
"""

import numpy as np


def unpack(p, n_in, h1, h2):
    p = np.asarray(p, dtype=np.float64)
    o = 0

    def take(k, shape):
        nonlocal o
        a = p[o:o + k].reshape(shape)
        o += k
        return a
    W1 = take(h1 * n_in, (h1, n_in))
    b1 = take(h1, (h1,))
    W2 = take(h2 * h1, (h2, h1))
    b2 = take(h2, (h2,))
    W3 = take(h2, (h2,))
    b3 = take(1, (1,))
    assert o == p.size
    return W1, b1, W2, b2, W3, b3


def forward(p, X, n_in, h1, h2):
    W1, b1, W2, b2, W3, b3 = unpack(p, n_in, h1, h2)
    X = np.asarray(X, dtype=np.float64)
    z1 = X @ W1.T + b1
    a1 = np.maximum(z1, 0.0)
    z2 = a1 @ W2.T + b2
    a2 = np.maximum(z2, 0.0)
    y = a2 @ W3 + b3[0]
    return y, (X, z1, a1, z2, a2)


def loss_grad(p, X, t, n_in, h1, h2):
    W1, b1, W2, b2, W3, b3 = unpack(p, n_in, h1, h2)
    y, (X, z1, a1, z2, a2) = forward(p, X, n_in, h1, h2)
    t = np.asarray(t, dtype=np.float64)
    n = len(t)
    loss = float(np.mean((y - t) ** 2))
    dy = 2.0 * (y - t) / n                 # dL/dy
    gW3 = a2.T @ dy
    gb3 = np.array([dy.sum()])
    dz2 = np.outer(dy, W3) * (z2 > 0)      # dL/dz2
    gW2 = dz2.T @ a1
    gb2 = dz2.sum(axis=0)
    dz1 = (dz2 @ W2) * (z1 > 0)            # dL/dz1
    gW1 = dz1.T @ X
    gb1 = dz1.sum(axis=0)
    g = np.concatenate([gW1.ravel(), gb1, gW2.ravel(), gb2, gW3, gb3])
    return loss, g


def n_params(n_in, h1, h2):
    return h1 * n_in + h1 + h2 * h1 + h2 + h2 + 1
