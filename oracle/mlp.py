"""MLP selector oracle in float64 -- TEST INFRASTRUCTURE ONLY.

The paper's model kinds are decision trees and random forests and it names
neural networks as a further classifier the design admits (Section 3.1,
"model_type").  The learned selector here is that extension: features ->
signed log1p -> z-score with training-set statistics -> Linear(F,H) -> ReLU ->
Linear(H,H) -> ReLU -> Linear(H,V) -> softmax, trained with mean
cross-entropy against the fastest-variant label and Adam.

Flat parameter order (shared by the C ABI): W1 (H x F, row major), b1 (H),
W2 (H x H), b2 (H), W3 (V x H), b3 (V).  Written as plain numpy matrix
products and elementwise maps; no blocking or fusion.
"""
from __future__ import annotations

import numpy as np

ADAM_B1, ADAM_B2, ADAM_EPS = 0.9, 0.999, 1e-8


def num_params(F: int, H: int, V: int) -> int:
    return H * F + H + H * H + H + V * H + V


def unpack(theta, F: int, H: int, V: int):
    theta = np.asarray(theta, dtype=np.float64)
    o = 0
    out = []
    for shape in ((H, F), (H,), (H, H), (H,), (V, H), (V,)):
        n = int(np.prod(shape))
        out.append(theta[o:o + n].reshape(shape))
        o += n
    assert o == theta.size
    return out


def pack(parts) -> np.ndarray:
    return np.concatenate([np.asarray(p, dtype=np.float64).ravel() for p in parts])


def slog1p(f):
    """sign(f) * log(1 + |f|): compresses sizes spanning decades."""
    f = np.asarray(f, dtype=np.float64)
    return np.sign(f) * np.log1p(np.abs(f))


def feature_stats(Fraw):
    """Per-feature mean and population standard deviation of slog1p(features);
    a zero deviation becomes 1 so that a constant feature maps to 0."""
    z = slog1p(Fraw)
    mu = z.mean(axis=0)
    sd = z.std(axis=0)
    sd = np.where(sd > 0, sd, 1.0)
    return mu, sd


def normalise(Fraw, mu, sd):
    return (slog1p(Fraw) - mu) / sd


def forward(theta, Fraw, mu, sd, H: int, V: int):
    """Return (probabilities (B, V), cache for backward)."""
    Fraw = np.atleast_2d(np.asarray(Fraw, dtype=np.float64))
    F = Fraw.shape[1]
    W1, b1, W2, b2, W3, b3 = unpack(theta, F, H, V)
    x0 = normalise(Fraw, mu, sd)
    z1 = x0 @ W1.T + b1
    h1 = np.maximum(z1, 0.0)
    z2 = h1 @ W2.T + b2
    h2 = np.maximum(z2, 0.0)
    logits = h2 @ W3.T + b3
    m = logits.max(axis=1, keepdims=True)
    e = np.exp(logits - m)
    p = e / e.sum(axis=1, keepdims=True)
    return p, (x0, z1, h1, z2, h2, logits)


def loss(theta, Fraw, labels, mu, sd, H: int, V: int) -> float:
    """Mean cross-entropy -log p[label]."""
    p, _ = forward(theta, Fraw, mu, sd, H, V)
    lab = np.asarray(labels, dtype=np.int64)
    return float(-np.mean(np.log(p[np.arange(lab.size), lab])))


def grad(theta, Fraw, labels, mu, sd, H: int, V: int):
    """Return (loss, flat gradient of the mean cross-entropy)."""
    Fraw = np.atleast_2d(np.asarray(Fraw, dtype=np.float64))
    B, F = Fraw.shape
    W1, b1, W2, b2, W3, b3 = unpack(theta, F, H, V)
    p, (x0, z1, h1, z2, h2, _) = forward(theta, Fraw, mu, sd, H, V)
    lab = np.asarray(labels, dtype=np.int64)
    L = float(-np.mean(np.log(p[np.arange(B), lab])))
    d3 = p.copy()
    d3[np.arange(B), lab] -= 1.0
    d3 /= B                                   # dL/dlogits
    gW3 = d3.T @ h2
    gb3 = d3.sum(axis=0)
    d2 = (d3 @ W3) * (z2 > 0)                 # dL/dz2
    gW2 = d2.T @ h1
    gb2 = d2.sum(axis=0)
    d1 = (d2 @ W2) * (z1 > 0)                 # dL/dz1
    gW1 = d1.T @ x0
    gb1 = d1.sum(axis=0)
    return L, pack([gW1, gb1, gW2, gb2, gW3, gb3])


def adam_step(theta, g, m, v, t: int, lr: float = 1e-3):
    """One Adam update (Kingma & Ba 2015) at step t >= 1; returns new
    (theta, m, v)."""
    m = ADAM_B1 * m + (1.0 - ADAM_B1) * g
    v = ADAM_B2 * v + (1.0 - ADAM_B2) * g * g
    mh = m / (1.0 - ADAM_B1 ** t)
    vh = v / (1.0 - ADAM_B2 ** t)
    return theta - lr * mh / (np.sqrt(vh) + ADAM_EPS), m, v


def xavier_uniform(rng: np.random.Generator, F: int, H: int, V: int) -> np.ndarray:
    """Glorot-uniform weights, zero biases."""
    parts = []
    for fo, fi in ((H, F), (H, H), (V, H)):
        a = np.sqrt(6.0 / (fi + fo))
        parts.append(rng.uniform(-a, a, (fo, fi)))
        parts.append(np.zeros(fo))
    return pack(parts)


def train(theta, Fraw, labels, mu, sd, H: int, V: int, perms, batch: int = 256, lr: float = 1e-3):
    """Minibatch Adam over the given per-epoch permutations; the last
    minibatch of an epoch may be partial.  Returns (theta, last loss)."""
    theta = np.array(theta, dtype=np.float64)
    m = np.zeros_like(theta)
    v = np.zeros_like(theta)
    Fraw = np.atleast_2d(np.asarray(Fraw, dtype=np.float64))
    lab = np.asarray(labels, dtype=np.int64)
    t = 0
    L = float("nan")
    for perm in perms:
        for s in range(0, len(perm), batch):
            idx = np.asarray(perm[s:s + batch])
            L, g = grad(theta, Fraw[idx], lab[idx], mu, sd, H, V)
            t += 1
            theta, m, v = adam_step(theta, g, m, v, t, lr)
    return theta, L


def predict(theta, Fraw, mu, sd, H: int, V: int):
    """(argmax variant, max probability) per row; ties to the lowest index."""
    p, _ = forward(theta, Fraw, mu, sd, H, V)
    return p.argmax(axis=1), p.max(axis=1)
