"""Oracle of the variant-selector MLP -- TEST INFRASTRUCTURE ONLY (FP64, numpy).

Not a method of the paper: a small network standing in for the paper's analytical
performance model (Section 4.2) in choosing a member of the family.  Definition:

    x  (22)  features: (log2 m - 11)/3, (log2 n - 11)/3, (log2 k - 11)/3, dtype one-hot (3),
             then (b_c + 7)/7 for the 16 candidates, b_c the analytic model's log2 seconds
    h1 = relu(W1 x + b1)      W1: 64 x 22
    h2 = relu(W2 h1 + b2)     W2: 64 x 64
    y  = W3 h2 + b3           W3: 16 x 64  (the correction to b_c: predicted log2 seconds
                                            of candidate c are b_c + y_c)

    loss = sum_{i,c} mask_ic (y_ic - t_ic)^2 / sum_{i,c} mask_ic

with t the measured log2 seconds minus b, and mask 1 where a candidate was measured.
The flat parameter vector is [W1 (row-major), b1, W2, b2, W3, b3].
"""
from __future__ import annotations

import numpy as np

N_SHAPE, N_OUT, N_H = 6, 16, 64
N_IN = N_SHAPE + N_OUT
SHAPES = [("W1", (N_H, N_IN)), ("b1", (N_H,)), ("W2", (N_H, N_H)), ("b2", (N_H,)),
          ("W3", (N_OUT, N_H)), ("b3", (N_OUT,))]
N_PARAMS = sum(int(np.prod(s)) for _, s in SHAPES)


def unpack(theta: np.ndarray) -> dict:
    out, o = {}, 0
    for name, shp in SHAPES:
        size = int(np.prod(shp))
        out[name] = np.asarray(theta[o:o + size], dtype=np.float64).reshape(shp)
        o += size
    return out


def features(m, n, k, dtype, base=None) -> np.ndarray:
    """Feature rows for arrays of sizes, dtype codes (0 FP64, 1 INT8 split, 2 BF16 split)
    and the model's log2 seconds per candidate `base` [rows, 16] (zeros when None)."""
    m, n, k, dtype = (np.atleast_1d(np.asarray(v)) for v in (m, n, k, dtype))
    x = np.zeros((m.size, N_IN))
    x[:, 0] = (np.log2(m) - 11.0) / 3.0
    x[:, 1] = (np.log2(n) - 11.0) / 3.0
    x[:, 2] = (np.log2(k) - 11.0) / 3.0
    x[np.arange(m.size), 3 + dtype.astype(int)] = 1.0
    b = np.zeros((m.size, N_OUT)) if base is None else np.asarray(base, dtype=np.float64).reshape(m.size, N_OUT)
    x[:, N_SHAPE:] = (b + 7.0) / 7.0
    return x


def forward(theta: np.ndarray, X: np.ndarray):
    p = unpack(theta)
    z1 = X @ p["W1"].T + p["b1"]
    h1 = np.maximum(z1, 0.0)
    z2 = h1 @ p["W2"].T + p["b2"]
    h2 = np.maximum(z2, 0.0)
    y = h2 @ p["W3"].T + p["b3"]
    return y, (X, z1, h1, z2, h2)


def loss(theta, X, T, mask) -> float:
    y, _ = forward(theta, X)
    return float(np.sum(mask * (y - T) ** 2) / np.sum(mask))


def grad(theta, X, T, mask) -> np.ndarray:
    """d loss / d theta by the chain rule (reverse mode), as a flat vector."""
    p = unpack(theta)
    y, (X, z1, h1, z2, h2) = forward(theta, X)
    dy = 2.0 * mask * (y - T) / np.sum(mask)
    gW3 = dy.T @ h2
    gb3 = dy.sum(axis=0)
    dh2 = dy @ p["W3"]
    dz2 = dh2 * (z2 > 0)
    gW2 = dz2.T @ h1
    gb2 = dz2.sum(axis=0)
    dh1 = dz2 @ p["W2"]
    dz1 = dh1 * (z1 > 0)
    gW1 = dz1.T @ X
    gb1 = dz1.sum(axis=0)
    return np.concatenate([g.ravel() for g in (gW1, gb1, gW2, gb2, gW3, gb3)])


def adam(theta, g, m, v, step, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam update (Kingma and Ba, 2015); step counts from 1.  Returns new arrays."""
    m = b1 * m + (1 - b1) * g
    v = b2 * v + (1 - b2) * g * g
    mh = m / (1 - b1 ** step)
    vh = v / (1 - b2 ** step)
    return theta - lr * mh / (np.sqrt(vh) + eps), m, v


def init(seed: int) -> np.ndarray:
    """He-uniform initial weights, zero biases."""
    g = np.random.Generator(np.random.Philox(seed))
    parts = []
    for name, shp in SHAPES:
        if name.startswith("W"):
            lim = np.sqrt(6.0 / shp[1])
            parts.append(g.uniform(-lim, lim, size=shp).ravel())
        else:
            parts.append(np.zeros(shp).ravel())
    return np.concatenate(parts)
