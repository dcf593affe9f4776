"""The two-level contact list (dem_set_outer_list): lists filtered from a
wider outer list must be exactly the lists of a fresh detection, a run with
it must be the run without it (bit-identical in deterministic mode) and the
oracle's run (FP64 tolerances), and a sphere that leaves its allowance around
the outer list must start a new one.  The oracle only ever sees generated
states."""
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


def _scene(prec, seed=21, n=500, margin=1e-4):
    """A packed lattice of clumps of a soft material (E 1e6 Pa: the initial
    overlaps push them apart slowly, so that they move by far less than the
    outer allowance over an outer list's life), at random speeds of a few
    cm/s."""
    sc = scenes.packed_scene(seed, n, precision=prec, compress=0.95, vel_scale=0.05, ang_scale=10.0)
    sc.E = np.full(len(sc.E), 1e6)
    if prec == scenes.PREC_FP32:
        sc.tpl_pos = sc.tpl_pos.astype(np.float32).astype(np.float64)
        sc.tpl_rad = sc.tpl_rad.astype(np.float32).astype(np.float64)
        scenes.snap_to_voxel_grid(sc)
    sc.bin_size = scenes.default_bin_size(sc, margin)
    return sc


def _fresh(oracle_mod, sc, pos, quat, margin, K, t):
    om = oracle_mod.OracleModel(sc)
    xs, owner, tsph = om.sphere_centres(sc.tpl, pos, quat)
    qc, rho = om.detect_coords(xs, tsph, margin)
    a, b = om.pairs_binned(owner, qc, rho)
    ws, ww = om.wall_candidates(xs, tsph, margin, t, sc.h * K)
    return a, b, ws, ww


@pytest.mark.parametrize("prec", [scenes.PREC_FP64, scenes.PREC_FP32])
def test_filtered_lists_are_the_fresh_detection(dem, prec):
    """Eight rebuilds 5 steps apart, an outer list at 3 x the margin serving
    four of them, against a context that detects every list afresh (both in
    deterministic mode, so their states stay bit-identical): after every
    rebuild the two lists, pairs and wall candidates, are the same, bit for
    bit.  (The fresh detection is the oracle's on generated states, tested
    elsewhere.)"""
    margin, K = 2e-4, 5
    sc = _scene(prec, margin=margin)
    sims = [dem.Simulation(sc, margin=margin, rebuild_interval=K) for _ in range(2)]
    try:
        for sim in sims:
            sim.set_deterministic(True)
        sims[1].set_outer_list(3.0, 4)
        for sim in sims:
            sim.step(1)
        for block in range(8):
            lists = []
            for sim in sims:
                sim.step(K)  # the last of these steps runs on a new list
                lists.append(sim.contacts())
            for x, y in zip(lists[0], lists[1]):
                assert np.array_equal(x, y), block
            assert len(lists[0][0]) > sc.n_clumps
            for x, y in zip(sims[0].state(), sims[1].state()):
                assert np.array_equal(x, y)
        st = sims[1].stats()
        assert st["rebuilds"] == 9 and st["outer_rebuilds"] == 3  # at rebuilds 1, 5 and 9
        assert sims[0].stats()["outer_rebuilds"] == 0
    finally:
        for sim in sims:
            sim.close()


@pytest.mark.parametrize("graphs", [False, True])
@pytest.mark.parametrize("prec", [scenes.PREC_FP64, scenes.PREC_FP32])
def test_outer_list_on_a_second_stream_is_the_fresh_detection(dem, prec, graphs):
    """The next outer list detected on a second stream while the steps run
    (async_detect): 12 rebuilds 5 steps apart against a context detecting
    every list afresh, both deterministic; lists and states bit-identical
    after every rebuild, and an outer list adopted every fourth rebuild."""
    margin, K = 2e-4, 5
    sc = _scene(prec, margin=margin)
    sims = [dem.Simulation(sc, margin=margin, rebuild_interval=K) for _ in range(2)]
    try:
        for sim in sims:
            sim.set_deterministic(True)
            sim.set_graphs(graphs)
        sims[1].set_outer_list(3.0, 4, async_detect=True)
        for sim in sims:
            sim.step(1)
        for block in range(11):
            lists = []
            for sim in sims:
                sim.step(K)
                lists.append(sim.contacts())
            for x, y in zip(lists[0], lists[1]):
                assert np.array_equal(x, y), block
            for x, y in zip(sims[0].state(), sims[1].state()):
                assert np.array_equal(x, y), block
        st = sims[1].stats()
        # built at rebuild 1, then started at rebuilds 4 and 8 and adopted at 5 and 9
        assert st["rebuilds"] == 12 and st["outer_rebuilds"] == 3
        # the same steps in one call (the detection overlaps them inside the call)
        for sim in sims:
            sim.step(4 * K + 3)
        for x, y in zip(sims[0].contacts(), sims[1].contacts()):
            assert np.array_equal(x, y)
        for x, y in zip(sims[0].state(), sims[1].state()):
            assert np.array_equal(x, y)
        assert sims[1].stats()["outer_rebuilds"] == 4
    finally:
        for sim in sims:
            sim.close()


def test_outer_list_on_a_second_stream_after_a_jump(dem, oracle_mod):
    """A state set from outside while an outer list detected on the second
    stream waits to be adopted: the allowance check rejects it, a new outer
    list is detected, and the list is the oracle's detection of that state."""
    margin, K = 1e-4, 5
    sc = _scene(scenes.PREC_FP64, seed=23)
    pos = sc.pos.copy()
    pos[::7, 0] += 1e-3
    with dem.Simulation(sc, margin=margin, rebuild_interval=K) as sim:
        sim.set_outer_list(3.0, 2, async_detect=True)
        sim.step(K + 1)  # rebuilds at steps 0 and 5: the one at 5 started the next list
        n_outer = sim.stats()["outer_rebuilds"]
        t = sim.stats()["time"]
        sim.set_state(pos, sc.quat, sc.vel, sc.angvel)
        sim.step(1)
        a, b, u, ws, ww, uw = sim.contacts()
        assert sim.stats()["outer_rebuilds"] == n_outer + 2  # adopted, rejected, detected
    ao, bo, wso, wwo = _fresh(oracle_mod, sc, pos, sc.quat, margin, K, t)
    assert np.array_equal(a, ao) and np.array_equal(b, bo)
    assert np.array_equal(ws, wso) and np.array_equal(ww, wwo)


def test_outer_list_fp64_trajectory_matches_oracle(dem, oracle_mod):
    """45 steps with a rebuild every 5, the lists filtered from outer lists:
    trajectory, lists and histories against the oracle's own run of the
    generated state, to the FP64 trajectory tolerances."""
    margin, K, nsteps = 2e-4, 5, 45
    sc = _scene(scenes.PREC_FP64, seed=24, margin=margin)
    with dem.Simulation(sc, margin=margin, rebuild_interval=K) as sim:
        sim.set_outer_list(3.0, 4)
        sim.step(nsteps)
        pos, quat, vel, w = sim.state()
        a, b, u, ws, ww, uw = sim.contacts()
        assert sim.stats()["outer_rebuilds"] == 3
    osim = oracle_mod.OracleSim(sc, margin, K)
    osim.step(nsteps)
    po, qo, vo, wo = osim.state()
    ao, bo, uo, wso, wwo, uwo = osim.contacts()
    osim.close()
    assert np.abs(pos - po).max() <= 1e-14 * (1 + np.abs(po).max())
    assert np.abs(vel - vo).max() <= 1e-10 * np.abs(vo).max()
    assert np.abs(w - wo).max() <= 1e-9 * np.abs(wo).max()
    assert np.array_equal(a, ao) and np.array_equal(b, bo)
    assert np.array_equal(ws, wso) and np.array_equal(ww, wwo)
    assert np.abs(uo).max() > 0 and np.abs(u - uo).max() <= 1e-8 * np.abs(uo).max()


def test_a_jump_past_the_allowance_starts_a_new_outer_list(dem, oracle_mod):
    """A generated state with clumps moved by 1 mm (far past m_out - m) set
    through dem_set_state after the context has built an outer list: the next
    rebuild finds them outside their allowance, detects a new outer list, and
    its list is the oracle's detection of that state."""
    margin, K = 1e-4, 5
    sc = _scene(scenes.PREC_FP64, seed=23)
    pos = sc.pos.copy()
    pos[::7, 0] += 1e-3
    with dem.Simulation(sc, margin=margin, rebuild_interval=K) as sim:
        sim.set_outer_list(3.0, 100)
        sim.step(K + 1)
        n_outer = sim.stats()["outer_rebuilds"]
        t = sim.stats()["time"]
        sim.set_state(pos, sc.quat, sc.vel, sc.angvel)
        sim.step(1)
        a, b, u, ws, ww, uw = sim.contacts()
        assert sim.stats()["outer_rebuilds"] == n_outer + 1
    ao, bo, wso, wwo = _fresh(oracle_mod, sc, pos, sc.quat, margin, K, t)
    assert np.array_equal(a, ao) and np.array_equal(b, bo)
    assert np.array_equal(ws, wso) and np.array_equal(ww, wwo)


def test_outer_list_arguments(dem):
    sc = _scene(scenes.PREC_FP64, n=50)
    with dem.Simulation(sc, margin=1e-4, rebuild_interval=5) as sim:
        for factor, n in ((1.0, 3), (0.5, 2), (float("nan"), 2), (2.0, -1)):
            with pytest.raises(dem.DemError, match="INVALID"):
                sim.set_outer_list(factor, n)
        sim.set_outer_list(2.0, 0)  # off
        sim.step(6)
        assert sim.stats()["outer_rebuilds"] == 0
