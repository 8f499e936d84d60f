"""Plain FP64 CPU oracle for the learned bandwidth proposal.

TEST INFRASTRUCTURE ONLY.  Only the test suite and the benchmark's CPU
baseline may import it.  It shares no code with the CUDA library and never
imports it.  The paper points to bandwidth selection with the same FFT
machinery (Sec. 1, Sec. 5) but describes no network; these are the textbook
definitions the GPU side implements:

* ``standardize``   -- per-axis mean, population standard deviation,
                       correlation, skewness and mean excess kurtosis, and the
                       standardised samples (X - mean) / sd.
* ``features``      -- 32 x 32 block masses of a binned M x M grid
                       (8 sqrt(mass / n)), then the moments, log10(n)/4 and a
                       constant 1, zero-padded to 1088 entries.
* ``mlp_forward``   -- y = W3 relu(W2 relu(W1 x + b1) + b2) + b3.
* ``mlp_loss_grad`` -- loss (1/B) sum (y - t)^2 and its gradient with respect
                       to every parameter by the chain rule (backpropagation
                       written out layer by layer).
* ``theta_to_H``    -- log-Cholesky parameters (a, beta, c) to
                       H = R R^T, R = [[e^a, 0], [beta e^c, e^c]].

The network's ReLU masks are decisions taken on floating-point values, so a
comparison with a BF16 implementation takes them in that precision:
``bf16=True`` rounds (round to nearest even, 8-bit significand) the inputs,
the weights, the stored activations and the back-propagated gradients that
enter matrix products, exactly where a BF16-operand implementation holds
them; every sum stays FP64.

Parameters are one flat vector laid out as W1 (hidden x in, row-major), b1,
W2 (hidden x hidden), b2, W3 (out x hidden), b3.
"""
from __future__ import annotations

import numpy as np

FEAT_DIM = 1088


def standardize(X):
    """Moments (mean0, mean1, sd0, sd1, corr, skew0, skew1, excess kurtosis
    averaged over the axes) with population (1/n) normalisation, and Z."""
    X = np.asarray(X, dtype=np.float64)
    n = X.shape[0]
    mean = X.sum(axis=0) / n
    D = X - mean
    var = (D * D).sum(axis=0) / n
    sd = np.sqrt(var)
    corr = (D[:, 0] * D[:, 1]).sum() / n / (sd[0] * sd[1])
    Z = D / sd
    skew = (Z ** 3).sum(axis=0) / n
    kurt = 0.5 * ((Z ** 4).sum(axis=0) / n).sum() - 3.0
    mom = np.array([mean[0], mean[1], sd[0], sd[1], corr, skew[0], skew[1], kurt])
    return Z, mom


def features(counts, n, mom):
    """Block features of integer counts (units 2^-32) on an M x M grid."""
    counts = np.asarray(counts)
    M = counts.shape[0]
    w = M // 32
    mass = np.zeros((32, 32))
    for by in range(32):
        for bx in range(32):
            s = int(counts[by * w:(by + 1) * w, bx * w:(bx + 1) * w].astype(object).sum())
            mass[by, bx] = s / 2.0 ** 32 / n
    f = np.zeros(FEAT_DIM)
    f[:1024] = 8.0 * np.sqrt(mass).ravel()
    f[1024:1030] = [mom[4], mom[5], mom[6], mom[7], np.log10(n) / 4.0, 1.0]
    return f


def bf16_round(x):
    """Round to the nearest BF16 value (ties to even) via FP32."""
    f = np.asarray(x, dtype=np.float64).astype(np.float32)
    b = f.view(np.uint32).astype(np.uint64)
    b = (b + 0x7FFF + ((b >> 16) & 1)) & 0xFFFF0000
    return b.astype(np.uint32).view(np.float32).astype(np.float64)


def unpack(p, in_dim, hidden, out_dim):
    """Views W1, b1, W2, b2, W3, b3 of the flat parameter vector."""
    p = np.asarray(p, dtype=np.float64)
    sizes = [hidden * in_dim, hidden, hidden * hidden, hidden, out_dim * hidden, out_dim]
    parts, o = [], 0
    for s in sizes:
        parts.append(p[o:o + s])
        o += s
    assert o == p.size
    W1 = parts[0].reshape(hidden, in_dim)
    W2 = parts[2].reshape(hidden, hidden)
    W3 = parts[4].reshape(out_dim, hidden)
    return W1, parts[1], W2, parts[3], W3, parts[5]


def mlp_forward(p, X, in_dim, hidden, out_dim, bf16=False):
    """Outputs y (B x out) and the intermediate values the gradient needs."""
    r = bf16_round if bf16 else (lambda v: v)
    W1, b1, W2, b2, W3, b3 = unpack(p, in_dim, hidden, out_dim)
    W1, W2, W3 = r(W1), r(W2), r(W3)
    X = r(np.asarray(X, dtype=np.float64))
    z1 = X @ W1.T + b1
    a1 = r(np.maximum(z1, 0.0))
    z2 = a1 @ W2.T + b2
    a2 = r(np.maximum(z2, 0.0))
    y = a2 @ W3.T + b3
    return y, (X, z1, a1, z2, a2)


def mlp_loss_grad(p, X, T, in_dim, hidden, out_dim, bf16=False):
    """loss = (1/B) sum_b sum_j (y_bj - t_bj)^2 and d loss / d p (flat)."""
    r = bf16_round if bf16 else (lambda v: v)
    y, (X, z1, a1, z2, a2) = mlp_forward(p, X, in_dim, hidden, out_dim, bf16)
    W1, b1, W2, b2, W3, b3 = unpack(p, in_dim, hidden, out_dim)
    W2, W3 = r(W2), r(W3)
    B = X.shape[0]
    res = y - np.asarray(T, dtype=np.float64)
    loss = float((res * res).sum() / B)
    dy = 2.0 * res / B                  # d loss / d y
    db3 = dy.sum(axis=0)
    dy = r(dy)
    dW3 = dy.T @ a2
    da2 = dy @ W3
    dz2 = da2 * (z2 > 0)
    db2 = dz2.sum(axis=0)
    dz2 = r(dz2)
    dW2 = dz2.T @ a1
    da1 = dz2 @ W2
    dz1 = da1 * (z1 > 0)
    db1 = dz1.sum(axis=0)
    dz1 = r(dz1)
    dW1 = dz1.T @ X
    g = np.concatenate([dW1.ravel(), db1, dW2.ravel(), db2, dW3.ravel(), db3])
    return loss, g


def theta_to_H(theta):
    """H = R R^T with R = [[e^a, 0], [beta e^c, e^c]] for theta = (a, beta, c)."""
    a, beta, c = (float(v) for v in theta)
    R = np.array([[np.exp(a), 0.0], [beta * np.exp(c), np.exp(c)]])
    return R @ R.T
