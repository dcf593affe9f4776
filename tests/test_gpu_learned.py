"""The learned list-lifetime regressor and the learned rebuild rule on the GPU.

Regressor: forward pass and loss gradient of the GPU kernels (BF16 weights,
FP32 accumulation) against the FP64 oracle evaluated at the same BF16-rounded
weights; training reduces the loss.  Rule: traces from the plain rule, a
forced rollback, zero missed contacts, and the gain over the plain rule."""
import math

import numpy as np
import pytest

from paper_2307_03445_gb300 import scenes

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dem():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2307_03445_gb300 as dem

    dem.load_library()
    return dem


def _bf16(a):
    """Round float32 values to bfloat16 (nearest, ties to even) and back."""
    a = np.ascontiguousarray(a, np.float32)
    u = a.view(np.uint32).astype(np.uint64)
    r = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16
    return r.astype(np.uint32).view(np.float32)


def _data(n, seed):
    rng = np.random.default_rng(seed)
    x = rng.normal(size=(n, 6)).astype(np.float32)
    t = (np.tanh(x[:, 0]) + 0.3 * x[:, 1] * x[:, 2]).astype(np.float32)
    return x, t


def test_forward_matches_oracle(dem, oracle_mod):
    reg = dem.Regressor()
    p = reg.params()
    x, _ = _data(5000, 1)
    y = reg.forward(x)
    want = oracle_mod.mlp_forward(_bf16(p).astype(np.float64), x.astype(np.float64))
    scale = np.abs(want).max()
    assert np.abs(y - want).max() <= 1e-5 * max(scale, 1.0)


def test_gradient_matches_oracle(dem, oracle_mod):
    rng = np.random.default_rng(2)
    p = (rng.normal(size=oracle_mod.mlp_num_params()) * 0.2).astype(np.float32)
    reg = dem.Regressor(params=p)
    x, t = _data(3000, 3)
    loss, g = reg.loss_grad(x, t)
    loss_o, g_o = oracle_mod.mlp_loss_grad(_bf16(p).astype(np.float64), x.astype(np.float64),
                                           t.astype(np.float64))
    assert loss == pytest.approx(loss_o, rel=1e-5)
    assert np.linalg.norm(g - g_o) <= 1e-4 * np.linalg.norm(g_o)
    # per layer too (a transposed or misplaced block would show here)
    sizes = [64 * 6, 64, 64 * 64, 64, 64 * 64, 64, 64, 1]
    k = 0
    for s in sizes:
        a, b = g[k:k + s], g_o[k:k + s]
        assert np.linalg.norm(a - b) <= 1e-3 * np.linalg.norm(b) + 1e-12
        k += s


def test_training_reduces_the_loss(dem):
    reg = dem.Regressor()
    x, t = _data(20000, 4)
    l0, _ = reg.loss_grad(x, t)
    l1 = reg.train(x, t, steps=400, batch=2048, lr=2e-3, seed=1)
    assert l1 < 0.1 * l0


@pytest.fixture(scope="module")
def bed(dem):
    """A settled 0.25 x 0.25 m bed of the workload's clumps with the plate
    sliding on top (prepared like the benchmark bed, one patch)."""
    from paper_2307_03445_gb300 import workloads

    return workloads.bed_c5(n_clumps=6000, lx=0.25, ly=0.25, patch=0.25)


CAND = [1e-6, 2e-6, 4e-6, 8e-6, 1.6e-5, 3.2e-5]


def test_traces_are_well_formed(dem, bed):
    sc = bed
    with dem.Simulation(sc, margin=2e-5, rebuild_interval=20) as sim:
        x, t = sim.trace(3, 40, CAND)
    assert len(x) > 100 and len(x) % len(CAND) == 0
    assert np.all(np.isfinite(x)) and np.all(np.isfinite(t))
    assert t.min() >= 0.0 and t.max() <= math.log(40) + 1e-6
    # a larger margin never fails earlier than a smaller one in the same bin
    T = t.reshape(-1, len(CAND))
    assert np.all(np.diff(T, axis=1) >= -1e-6)


def _everlasting(dem):
    """A regressor that predicts everlasting lists: the smallest margin everywhere."""
    reg = dem.Regressor()
    p = np.zeros(reg.n_params, np.float32)
    p[-1] = 20.0  # output bias: ln(lifetime) = 20 for every query
    reg.set_params(p)
    return reg


@pytest.mark.parametrize("mode", ["halt", "rollback"])
def test_bad_predictions_never_miss_a_contact(dem, bed, mode):
    """With the smallest margin everywhere the certificate fails within a few
    steps (the plate drags clumps).  Halt mode cuts the interval short on the
    device and rebuilds; rollback mode replays the interval with the plain
    rule.  Either way no contact is missing and the trajectory is that of
    the plain rule."""
    from paper_2307_03445_gb300 import capi

    sc = bed
    reg = _everlasting(dem)
    m = capi.DEM_LEARNED_HALT if mode == "halt" else capi.DEM_LEARNED_ROLLBACK
    with dem.Simulation(sc, margin=2e-5, rebuild_interval=20) as plain:
        plain.step(400)
        pos_p = plain.state()[0]
    with dem.Simulation(sc, margin=2e-5, rebuild_interval=20) as sim:
        sim.set_learned_policy(reg, interval=200, safety=1.0, candidates=CAND, mode=m)
        sim.step(400)
        st = sim.stats()
        assert st["steps"] == 400 or mode == "rollback"
        if mode == "halt":
            assert st["early_rebuilds"] >= 1 and st["rollbacks"] == 0
        else:
            assert st["rollbacks"] >= 1
        assert sim.audit() == 0
        pos_l = sim.state()[0]
    moved = np.abs(pos_p - sc.pos).max()
    assert moved > 1e-6
    assert np.abs(pos_l - pos_p).max() <= 1e-3 * moved


def test_speed_floor_keeps_fast_clumps_listed(dem, bed):
    """A regressor that promises every bin an everlasting list gives every
    clump the smallest candidate (1 um), and over intervals of 200 steps the
    clumps the plate drags end them early; with the speed floor each clump's margin covers at least
    its own travel over the interval at its speed, so fewer intervals end
    early.  No contact is missed either way, and a negative or non-finite
    floor is refused."""
    sc = bed
    reg = _everlasting(dem)
    early = []
    for floor in (0.0, 1.5):
        with dem.Simulation(sc, margin=2e-5, rebuild_interval=20) as sim:
            sim.set_learned_policy(reg, interval=200, safety=1.0, candidates=CAND,
                                   speed_floor=floor)
            sim.step(400)
            st = sim.stats()
            assert st["steps"] == 400 and sim.audit() == 0
            early.append(st["early_rebuilds"])
    assert early[0] >= 1 and early[1] < early[0], early
    with dem.Simulation(sc, margin=2e-5, rebuild_interval=20) as sim:
        for bad in (-1.0, float("nan"), float("inf")):
            with pytest.raises(dem.DemError, match="INVALID"):
                sim.set_learned_policy(reg, interval=40, safety=1.0, candidates=CAND,
                                       speed_floor=bad)


def test_trained_rule_beats_the_plain_rule(dem, bed):
    """Trained on traces of the plain rule, the learned rule lists fewer pairs
    and rebuilds less often than the plain rule, with zero missed contacts."""
    sc = bed
    plain_K, plain_m = 20, 2e-5
    with dem.Simulation(sc, margin=plain_m, rebuild_interval=plain_K) as sim:
        sim.step(200)  # past the initial transient
        state = sim.state()
        x, t = sim.trace(6, 120, CAND)
    reg = dem.Regressor()
    reg.train(x, t, steps=600, batch=4096, lr=2e-3, seed=2)
    sc2 = scenes.Scene(**{**sc.__dict__, "pos": state[0], "quat": state[1], "vel": state[2],
                          "angvel": state[3]})
    n = 400
    with dem.Simulation(sc2, margin=plain_m, rebuild_interval=plain_K) as plain:
        plain.step(n)
        sp = plain.stats()
        assert plain.audit() == 0
    with dem.Simulation(sc2, margin=plain_m, rebuild_interval=plain_K) as sim:
        # the target interval times the safety factor stays inside the
        # traced window, where predicted lifetimes are not capped
        sim.set_learned_policy(reg, interval=60, safety=1.5, candidates=CAND)
        sim.step(n)
        sl = sim.stats()
        assert sim.audit() == 0
    # replays after a rollback count towards the learned run's work
    assert sl["rebuilds"] < sp["rebuilds"], (sl, sp)
    assert sl["pair_steps"] < sp["pair_steps"], (sl, sp)


def _sparse_exact_params(oracle_mod):
    """Hidden unit o takes input o % 6 (x 0.5), then itself (x 2), then unit
    o + 1 (x 1); the output sums the 64 units x 2^-6.  With inputs that are
    small multiples of 1/4 every product and partial sum is exact, so a
    misplaced row, column or K step shows up as an O(1) error."""
    H, IN = 64, 6
    p = np.zeros(oracle_mod.mlp_num_params(), np.float32)
    k = 0
    W1 = p[k:k + H * IN].reshape(H, IN)
    for o in range(H):
        W1[o, o % IN] = 0.5
    k += H * IN + H
    np.fill_diagonal(p[k:k + H * H].reshape(H, H), 2.0)
    k += H * H + H
    W3 = p[k:k + H * H].reshape(H, H)
    for o in range(H):
        W3[o, (o + 1) % H] = 1.0
    k += H * H + H
    p[k:k + H] = 2.0 ** -6
    return p


def test_tensor_core_forward_is_exact_on_an_exact_network(dem, oracle_mod):
    p = _sparse_exact_params(oracle_mod)
    reg = dem.Regressor(params=p)
    rng = np.random.default_rng(9)
    for n in (1, 127, 128, 129, 3001):
        x = (rng.integers(-4, 8, size=(n, 6)) * 0.25).astype(np.float32)
        want = oracle_mod.mlp_forward_bf16act(p.astype(np.float64), x.astype(np.float64))
        assert np.array_equal(reg.forward_tc(x).astype(np.float64), want), n
    reg.close()


def test_tensor_core_forward_matches_oracle(dem, oracle_mod):
    """The tcgen05 forward pass of a random network against the oracle pass
    with bfloat16 layer inputs at the same bfloat16 weights, over ragged row
    counts (partial last tiles).  The tensor cores sum the bfloat16 products
    with less than IEEE FP32 care, so activations near a bfloat16 rounding
    boundary may round the other way: the bound is a few bfloat16 steps."""
    rng = np.random.default_rng(8)
    p = (rng.normal(size=oracle_mod.mlp_num_params()) * 0.25).astype(np.float32)
    reg = dem.Regressor(params=p)
    pw = _bf16(p).astype(np.float64)
    for n in (1, 127, 128, 129, 5000, 70001):
        x = rng.normal(size=(n, 6)).astype(np.float32)
        y = reg.forward_tc(x)
        want = oracle_mod.mlp_forward_bf16act(pw, x.astype(np.float64))
        scale = max(np.abs(want).max(), 1.0)
        err = np.abs(y - want)
        assert err.max() <= 2e-2 * scale, n
        assert err.mean() <= 2e-3 * scale, n
    # and it agrees with the FP32-activation pass to bfloat16 accuracy
    x = rng.normal(size=(4096, 6)).astype(np.float32)
    yf = reg.forward(x)
    assert np.abs(reg.forward_tc(x) - yf).max() <= 5e-2 * max(np.abs(yf).max(), 1.0)
    reg.close()
