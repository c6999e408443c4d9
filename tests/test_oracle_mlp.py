"""Pins of the float64 MLP oracle: finite differences, an independent autograd
formulation, uniform-logit cross-entropy and the closed-form first Adam step."""
import math

import numpy as np
import pytest
import torch

from oracle import mlp

F, H, V = 5, 16, 7


def _setup(seed=0, B=12):
    r = np.random.Generator(np.random.PCG64(seed))
    theta = mlp.xavier_uniform(r, F, H, V)
    theta += r.normal(scale=0.05, size=theta.size)  # non-zero biases too
    Fraw = np.exp(r.uniform(0, 12, (B, F)))
    lab = r.integers(0, V, B)
    mu, sd = mlp.feature_stats(Fraw)
    return theta, Fraw, lab, mu, sd


def test_uniform_logits_cross_entropy_is_ln_v():
    theta, Fraw, lab, mu, sd = _setup()
    W1, b1, W2, b2, W3, b3 = mlp.unpack(theta, F, H, V)
    zero = mlp.pack([W1, b1, W2, b2, np.zeros_like(W3), np.zeros_like(b3)])
    assert mlp.loss(zero, Fraw, lab, mu, sd, H, V) == pytest.approx(math.log(V), rel=1e-15)


def test_gradient_central_differences():
    theta, Fraw, lab, mu, sd = _setup(1)
    _, g = mlp.grad(theta, Fraw, lab, mu, sd, H, V)
    h = 1e-6
    r = np.random.Generator(np.random.PCG64(2))
    idx = r.choice(theta.size, 60, replace=False)
    num = np.empty(idx.size)
    for t, i in enumerate(idx):
        tp = theta.copy()
        tm = theta.copy()
        tp[i] += h
        tm[i] -= h
        num[t] = (mlp.loss(tp, Fraw, lab, mu, sd, H, V) - mlp.loss(tm, Fraw, lab, mu, sd, H, V)) / (2 * h)
    assert np.linalg.norm(num - g[idx]) <= 1e-6 * np.linalg.norm(g[idx])


def test_gradient_matches_autograd_formulation():
    theta, Fraw, lab, mu, sd = _setup(3, B=33)
    L, g = mlp.grad(theta, Fraw, lab, mu, sd, H, V)
    th = torch.tensor(theta, dtype=torch.float64, requires_grad=True)
    W1, b1, W2, b2, W3, b3 = [torch.as_tensor(p) for p in mlp.unpack(th.detach().numpy(), F, H, V)]
    ps = []
    o = 0
    for shape in ((H, F), (H,), (H, H), (H,), (V, H), (V,)):
        n = int(np.prod(shape))
        ps.append(th[o:o + n].reshape(shape))
        o += n
    x0 = torch.as_tensor(mlp.normalise(Fraw, mu, sd))
    net = torch.nn.functional.linear(x0, ps[0], ps[1]).relu()
    net = torch.nn.functional.linear(net, ps[2], ps[3]).relu()
    logits = torch.nn.functional.linear(net, ps[4], ps[5])
    lt = torch.nn.functional.cross_entropy(logits, torch.as_tensor(lab))
    lt.backward()
    assert L == pytest.approx(lt.item(), rel=1e-13)
    assert np.max(np.abs(th.grad.numpy() - g)) <= 1e-13 * np.max(np.abs(g))


def test_first_adam_step_closed_form():
    # at t = 1: m_hat = g and v_hat = g^2, so the step is lr * g / (|g| + eps)
    r = np.random.Generator(np.random.PCG64(4))
    theta = r.normal(size=50)
    g = r.normal(size=50)
    new, m, v = mlp.adam_step(theta, g, np.zeros(50), np.zeros(50), 1, lr=1e-3)
    assert np.allclose(new, theta - 1e-3 * g / (np.abs(g) + 1e-8), rtol=0, atol=1e-15)
    assert np.allclose(m, 0.1 * g) and np.allclose(v, 0.001 * g * g)


def test_training_fits_separable_labels():
    r = np.random.Generator(np.random.PCG64(5))
    Fraw = np.exp(r.uniform(0, 10, (400, 2)))
    lab = (np.log(Fraw[:, 0]) > 5).astype(int) + 2 * (np.log(Fraw[:, 1]) > 5).astype(int)
    mu, sd = mlp.feature_stats(Fraw)
    theta = mlp.xavier_uniform(r, 2, 32, 4)
    perms = [r.permutation(400) for _ in range(60)]
    theta, _ = mlp.train(theta, Fraw, lab, mu, sd, 32, 4, perms, batch=64, lr=1e-2)
    pred, conf = mlp.predict(theta, Fraw, mu, sd, 32, 4)
    assert np.mean(pred == lab) >= 0.97
    assert np.all((conf > 0.25) & (conf <= 1.0))


def test_feature_stats_constant_column():
    Fraw = np.array([[3.0, 1.0], [3.0, 2.0], [3.0, 7.0]])
    mu, sd = mlp.feature_stats(Fraw)
    assert sd[0] == 1.0 and mu[0] == pytest.approx(math.log(4.0))
    assert np.all(mlp.normalise(Fraw, mu, sd)[:, 0] == 0.0)
