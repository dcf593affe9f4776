"""Pins of the oracle's lifetime regressor (dense ReLU network, MSE, Adam)."""
import numpy as np
import pytest


def _params(oracle_mod, seed=0, scale=0.3):
    rng = np.random.default_rng(seed)
    return rng.normal(scale=scale, size=oracle_mod.mlp_num_params())


def _unpack(oracle_mod, p):
    sizes = [(64, 6), (64, 64), (64, 64), (1, 64)]
    out, k = [], 0
    for o, i in sizes:
        W = p[k:k + o * i].reshape(o, i)
        k += o * i
        b = p[k:k + o]
        k += o
        out.append((W, b))
    assert k == len(p)
    return out


def test_parameter_count(oracle_mod):
    assert oracle_mod.mlp_num_params() == 6 * 64 + 64 + 2 * (64 * 64 + 64) + 64 + 1 == 8833


def test_forward_in_the_linear_regime_is_a_matrix_chain(oracle_mod):
    """With every pre-activation positive the ReLUs pass through, so the
    network is the affine map W4 W3 W2 W1 x + ... (numpy matrix products)."""
    p = _params(oracle_mod, 1, 0.05)
    layers = _unpack(oracle_mod, p)
    for W, b in layers[:3]:
        W[:] = np.abs(W)  # non-negative weights, biases and inputs keep every unit active
        b[:] = 0.1
    x = np.random.default_rng(2).uniform(0, 1, size=(50, 6))
    h = x.T
    for W, b in layers[:3]:
        h = W @ h + b[:, None]
        assert np.all(h > 0)
    W4, b4 = layers[3]
    want = (W4 @ h + b4[:, None]).ravel()
    assert np.allclose(oracle_mod.mlp_forward(p, x), want, rtol=1e-13, atol=1e-12)


def test_relu_cuts_negative_units(oracle_mod):
    p = _params(oracle_mod, 3)
    layers = _unpack(oracle_mod, p)
    for W, b in layers[:3]:
        b[:] = -1e6  # every hidden unit off
    x = np.random.default_rng(4).normal(size=(7, 6))
    assert np.allclose(oracle_mod.mlp_forward(p, x), layers[3][1][0])


def test_gradient_matches_central_differences(oracle_mod):
    p = _params(oracle_mod, 5)
    rng = np.random.default_rng(6)
    x = rng.normal(size=(32, 6))
    t = rng.normal(size=32)
    loss, g = oracle_mod.mlp_loss_grad(p, x, t)
    idx = rng.choice(len(p), size=200, replace=False)
    idx = np.concatenate([idx, [len(p) - 1, len(p) - 2, 0, 6 * 64]])  # output bias, last W, first W, b1
    h = 1e-6
    for i in idx:
        e = np.zeros_like(p)
        e[i] = h
        fd = (oracle_mod.mlp_loss_grad(p + e, x, t)[0] - oracle_mod.mlp_loss_grad(p - e, x, t)[0]) / (2 * h)
        assert g[i] == pytest.approx(fd, rel=1e-5, abs=1e-9)
    # the mean squared error itself
    y = oracle_mod.mlp_forward(p, x)
    assert loss == pytest.approx(np.mean((y - t) ** 2), rel=1e-14)


def test_adam_first_step_is_a_signed_unit_step(oracle_mod):
    n = oracle_mod.mlp_num_params()
    rng = np.random.default_rng(7)
    p, g = rng.normal(size=n), rng.normal(size=n)
    p1, m1, v1 = oracle_mod.mlp_adam(p, np.zeros(n), np.zeros(n), g, 1, lr=1e-3, eps=1e-15)
    # with bias correction the first step is lr * g / |g|
    assert np.allclose(p1, p - 1e-3 * np.sign(g), rtol=0, atol=1e-13)
    assert np.allclose(m1, 0.1 * g) and np.allclose(v1, 0.001 * g * g)


def test_training_reduces_the_loss(oracle_mod):
    rng = np.random.default_rng(8)
    x = rng.uniform(-1, 1, size=(256, 6))
    t = np.log1p(np.abs(x[:, 0]) + 0.5 * x[:, 1] ** 2)
    p = _params(oracle_mod, 9, 0.15)
    m = np.zeros_like(p)
    v = np.zeros_like(p)
    l0, _ = oracle_mod.mlp_loss_grad(p, x, t)
    for k in range(1, 301):
        _, g = oracle_mod.mlp_loss_grad(p, x, t)
        p, m, v = oracle_mod.mlp_adam(p, m, v, g, k, lr=3e-3)
    l1, _ = oracle_mod.mlp_loss_grad(p, x, t)
    assert l1 < 0.05 * l0
