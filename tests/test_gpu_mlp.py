"""Fused float32 MLP kernels against the float64 oracle (GPU)."""
import numpy as np
import pytest
import torch

import paper_2303_08873_b300 as ar
from oracle import mlp
from tests.gpu_util import dev, host

pytestmark = pytest.mark.gpu
F, H, V = 5, 64, 7


def _setup(seed, B):
    r = np.random.Generator(np.random.PCG64(seed))
    theta = mlp.xavier_uniform(r, F, H, V) + r.normal(scale=0.05, size=mlp.num_params(F, H, V))
    Fraw = np.exp(r.uniform(0, 14, (B, F)))
    lab = r.integers(0, V, B)
    # standardisation statistics of a training population, not of the batch
    # (a batch of one row would standardise every feature to exactly 0)
    mu, sd = mlp.feature_stats(np.exp(r.uniform(0, 14, (512, F))))
    return theta, Fraw, lab, mu, sd


def _parts(g):
    return mlp.unpack(g, F, H, V)


@pytest.mark.parametrize("B", [1, 37, 256])
def test_gradient_matches_oracle(B):
    theta, Fraw, lab, mu, sd = _setup(B, B)
    L, g = mlp.grad(theta, Fraw, lab, mu, sd, H, V)
    th32 = theta.astype(np.float32)
    # the oracle at the float32-rounded weights and statistics the kernel sees
    L, g = mlp.grad(th32.astype(np.float64), Fraw.astype(np.float32), lab, mu.astype(np.float32),
                    sd.astype(np.float32), H, V)
    grad = torch.zeros(mlp.num_params(F, H, V), dtype=torch.float32, device="cuda")
    loss = torch.zeros(1, dtype=torch.float32, device="cuda")
    ar.ar_mlp_grad(dev(th32), dev(mu, torch.float32), dev(sd, torch.float32), F, H, V, B,
                   dev(Fraw, torch.float32), dev(lab, torch.int32), grad, loss)
    gg = host(grad).astype(np.float64)
    assert abs(float(host(loss)[0]) - L) <= 1e-5 * max(1.0, abs(L))
    for name, a, b in zip(("W1", "b1", "W2", "b2", "W3", "b3"), _parts(gg), _parts(g)):
        assert np.linalg.norm(a - b) <= 1e-3 * np.linalg.norm(b) + 1e-12, name


def test_gradient_is_deterministic():
    theta, Fraw, lab, mu, sd = _setup(9, 200)
    args = (dev(theta, torch.float32), dev(mu, torch.float32), dev(sd, torch.float32), F, H, V, 200,
            dev(Fraw, torch.float32), dev(lab, torch.int32))
    g1 = torch.zeros(mlp.num_params(F, H, V), dtype=torch.float32, device="cuda")
    g2 = torch.zeros_like(g1)
    ar.ar_mlp_grad(*args, g1)
    ar.ar_mlp_grad(*args, g2)
    assert torch.equal(g1, g2)


def test_forward_matches_oracle():
    theta, Fraw, _, mu, sd = _setup(4, 3000)
    th32 = theta.astype(np.float32)
    p_ref, _ = mlp.forward(th32.astype(np.float64), Fraw.astype(np.float32), mu.astype(np.float32),
                           sd.astype(np.float32), H, V)
    B = Fraw.shape[0]
    probs = torch.zeros((B, V), dtype=torch.float32, device="cuda")
    var = torch.zeros(B, dtype=torch.int32, device="cuda")
    conf = torch.zeros(B, dtype=torch.float32, device="cuda")
    ar.ar_mlp_forward(dev(th32), dev(mu, torch.float32), dev(sd, torch.float32), F, H, V, B,
                      dev(Fraw, torch.float32), probs, var, conf)
    p = host(probs)
    assert np.max(np.abs(p - p_ref)) <= 1e-5
    top2 = np.sort(p_ref, axis=1)[:, -2:]
    clear = (top2[:, 1] - top2[:, 0]) > 1e-4
    assert np.array_equal(host(var)[clear], p_ref.argmax(axis=1)[clear])
    assert np.allclose(host(conf), p_ref.max(axis=1), atol=1e-5)


def test_adam_step_matches_oracle():
    r = np.random.Generator(np.random.PCG64(5))
    n = 5000
    th, g = r.normal(size=n), r.normal(size=n)
    m, v = r.normal(size=n) * 0.1, np.abs(r.normal(size=n)) * 0.01
    ref, mr, vr = mlp.adam_step(th, g, m, v, 7, lr=1e-3)
    tt, mt, vt = dev(th, torch.float32), dev(m, torch.float32), dev(v, torch.float32)
    ar.ar_mlp_adam(tt, dev(g, torch.float32), mt, vt, n, 7, 1e-3)
    assert np.max(np.abs(host(tt) - ref)) <= 1e-5 * np.max(np.abs(ref))
    assert np.allclose(host(mt), mr, rtol=1e-5, atol=1e-7)
    assert np.allclose(host(vt), vr, rtol=1e-5, atol=1e-9)


def test_fused_training_tracks_oracle_training():
    n, epochs, batch = 600, 3, 256
    theta, Fraw, lab, mu, sd = _setup(11, n)
    r = np.random.Generator(np.random.PCG64(12))
    perms = [r.permutation(n) for _ in range(epochs)]
    th32 = theta.astype(np.float32)
    ref, _ = mlp.train(th32.astype(np.float64), Fraw.astype(np.float32), lab, mu.astype(np.float32),
                       sd.astype(np.float32), H, V, perms, batch=batch, lr=1e-3)
    P = mlp.num_params(F, H, V)
    tt = dev(th32)
    am = torch.zeros(P, dtype=torch.float32, device="cuda")
    av = torch.zeros_like(am)
    ar.ar_mlp_train(tt, am, av, dev(mu, torch.float32), dev(sd, torch.float32), F, H, V, n,
                    dev(Fraw, torch.float32), dev(lab, torch.int32), dev(np.concatenate(perms), torch.int32),
                    epochs, batch, 1e-3)
    got = host(tt).astype(np.float64)
    # 9 Adam steps: float32 rounding may flip the sign of a tiny gradient and
    # move a weight by ~lr, so compare normwise
    assert np.linalg.norm(got - ref) <= 2e-3 * np.linalg.norm(ref - th32)


def test_region_mlp_model_trains_on_device_and_selects():
    # two features; the fastest variant depends on a threshold in each
    def cost(f, v):
        best = (1 if f[0] > 1e4 else 0) + (2 if f[1] > 50 else 0)
        return 1.0 if v == best else 2.0 + v

    r = ar.Region("m", 2, "mlp,64,epochs=300,seed=3", 10 ** 9)
    for v in range(4):
        r.register(f"v{v}", float(v), lambda a, v, x, s, u: 0)
    r.set_fake_timer(cost)
    rng = np.random.Generator(np.random.PCG64(2))
    pts = np.stack([np.exp(rng.uniform(0, 18, 300)), rng.uniform(0, 100, 300)], axis=1)
    for p in pts:
        r.profile(p.tolist(), reps=1)
    r.train()
    model = r.mlp()
    assert model["V"] == 4 and model["H"] == 64
    test = np.stack([np.exp(rng.uniform(0, 18, 200)), rng.uniform(0, 100, 200)], axis=1)
    want = [(1 if a > 1e4 else 0) + (2 if b > 50 else 0) for a, b in test]
    got = [r.select(p.tolist())[0] for p in test]
    assert np.mean(np.array(got) == np.array(want)) >= 0.9
    # device inference of the exported model agrees with the runtime's host inference
    var = torch.zeros(len(test), dtype=torch.int32, device="cuda")
    conf = torch.zeros(len(test), dtype=torch.float32, device="cuda")
    ar.ar_mlp_forward(dev(model["theta"]), dev(model["mu"]), dev(model["sd"]), 2, 64, 4, len(test),
                      dev(test, torch.float32), None, var, conf)
    assert np.mean(host(var) == np.array(got)) >= 0.99
