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


def _pass_through(oracle_mod):
    """Parameters under which the network passes the first feature through
    unit 0 of every layer (weights 1, everything else 0)."""
    p = np.zeros(oracle_mod.mlp_num_params())
    H, IN = 64, 6
    k = 0
    for n_in, n_out in ((IN, H), (H, H), (H, H), (H, 1)):
        p[k + 0 * n_in + 0] = 1.0  # W[0][0]
        k += n_in * n_out + n_out
    return p


def test_bf16_pass_rounds_every_layer_input(oracle_mod):
    """Pinned by hand: 1 + 2^-8 lies halfway between the bfloat16 neighbours
    1 and 1 + 2^-7 and rounds to the even one (1); 1 + 3 * 2^-8 rounds up to
    1 + 2^-6; exact bfloat16 values pass unchanged; the double pass keeps them."""
    p = _pass_through(oracle_mod)
    x = np.zeros((4, 6))
    x[:, 0] = [1 + 2 ** -8, 1 + 3 * 2 ** -8, 0.75, -2.0]
    y16 = oracle_mod.mlp_forward_bf16act(p, x)
    y64 = oracle_mod.mlp_forward(p, x)
    assert list(y16) == [1.0, 1 + 2 ** -6, 0.75, 0.0]  # ReLU cuts the negative
    assert list(y64) == [1 + 2 ** -8, 1 + 3 * 2 ** -8, 0.75, 0.0]


def test_bf16_pass_equals_the_double_pass_on_exact_values(oracle_mod):
    """A sparse network whose hidden activations are the inputs scaled by
    powers of two (exact in bfloat16 for inputs with few significant bits):
    the two passes agree exactly; with inputs that need more than 8 bits they
    differ, by bfloat16 rounding only."""
    H, IN = 64, 6
    p = np.zeros(oracle_mod.mlp_num_params())
    k = 0
    W1 = p[k:k + H * IN].reshape(H, IN)
    for o in range(H):
        W1[o, o % IN] = 0.5
    k += H * IN + H
    W2 = p[k:k + H * H].reshape(H, H)
    np.fill_diagonal(W2, 2.0)
    k += H * H + H
    W3 = p[k:k + H * H].reshape(H, H)
    for o in range(H):
        W3[o, (o + 1) % H] = 1.0
    k += H * H + H
    p[k:k + H] = 2.0 ** -6
    rng = np.random.default_rng(5)
    x = rng.integers(0, 8, size=(50, IN)) * 0.25
    assert np.array_equal(oracle_mod.mlp_forward_bf16act(p, x), oracle_mod.mlp_forward(p, x))
    x2 = x + 2.0 ** -12  # now 12+ significant bits
    d = np.abs(oracle_mod.mlp_forward_bf16act(p, x2) - oracle_mod.mlp_forward(p, x2))
    assert d.max() > 0 and d.max() <= 2.0 ** -8 * (1 + np.abs(x2).max())
