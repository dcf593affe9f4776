"""Parity of the CUDA path (through the C ABI) with the FP64 CPU oracle.

Bin registrations, pair lists and wall lists: bit-exact (integer predicate
on the same lattice).  Per-clump force and torque totals: within 1e-12 (FP64)
or 1e-5 (FP32_VOXEL) of the oracle, relative to the sum of the magnitudes of
the contributions to that total (the scale that bounds the rounding of a sum).
"""
import dataclasses
import math

import numpy as np
import pytest

from paper_2307_03445_gb300 import scenes
from tests.helpers import set_clumps, single_sphere_scene

pytestmark = pytest.mark.gpu

TOL = {scenes.PREC_FP64: 1e-12, scenes.PREC_FP32: 1e-5}


@pytest.fixture(scope="module")
def dem():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2307_03445_gb300 as dem

    dem.load_library()
    return dem


def _scene(seed, n, prec, compress=0.92, walls=True, bin_scale=1.0, margin=1e-4, **kw):
    sc = scenes.packed_scene(seed, n, precision=prec, compress=compress, walls=walls, **kw)
    if prec == scenes.PREC_FP32:
        # templates and state exactly representable in the FP32 voxel layout
        sc.tpl_pos = sc.tpl_pos.astype(np.float32).astype(np.float64)
        sc.tpl_rad = sc.tpl_rad.astype(np.float32).astype(np.float64)
        scenes.snap_to_voxel_grid(sc)
    sc.bin_size = bin_scale * scenes.default_bin_size(sc, margin)
    return sc


def _oracle_lists(oracle_mod, sc, margin, K):
    om = oracle_mod.OracleModel(sc)
    xs, owner, tsph = om.sphere_centres(sc.tpl, sc.pos, sc.quat)
    qc, rho = om.detect_coords(xs, tsph, margin)
    keys, ids = om.bin_entries(qc, rho)
    a, b = om.pairs_binned(owner, qc, rho)
    ws, ww = om.wall_candidates(xs, tsph, margin, 0.0, sc.h * K)
    return om, keys, ids, a, b, ws, ww


@pytest.mark.parametrize("prec", [scenes.PREC_FP64, scenes.PREC_FP32])
@pytest.mark.parametrize("seed,n,bin_scale", [(1, 333, 1.0), (2, 517, 0.45), (3, 1000, 2.2)])
def test_detection_bit_exact(dem, oracle_mod, prec, seed, n, bin_scale):
    margin, K = 1e-4, 10
    sc = _scene(seed, n, prec, bin_scale=bin_scale, margin=margin)
    with dem.Simulation(sc, margin=margin, rebuild_interval=K) as sim:
        sim.rebuild()
        keys, ids = sim.bins()
        a, b, u, ws, ww, uw = sim.contacts()
    om, k_o, i_o, a_o, b_o, ws_o, ww_o = _oracle_lists(oracle_mod, sc, margin, K)
    assert len(a_o) > n  # a dense case with many candidate pairs
    assert np.array_equal(keys, k_o) and np.array_equal(ids, i_o)
    assert np.array_equal(a, a_o) and np.array_equal(b, b_o)
    assert np.array_equal(ws, ws_o) and np.array_equal(ww, ww_o)
    assert np.all(u == 0) and np.all(uw == 0)


@pytest.mark.parametrize("prec", [scenes.PREC_FP64, scenes.PREC_FP32])
def test_autotuned_bins_stay_exact(dem, oracle_mod, prec):
    """The bin-size autotuner keeps the fastest factor; the state is unchanged
    and detection at the chosen bin edge is still the oracle's, bit for bit."""
    margin, K = 1e-4, 10
    sc = _scene(4, 700, prec, margin=margin)
    factors = (0.4, 0.7, 1.0, 2.0)
    with dem.Simulation(sc, margin=margin, rebuild_interval=K) as sim:
        sim.rebuild()
        before = sim.state()
        best, ms = sim.autotune_bins(factors, reps=2)
        assert best in factors and all(ms[f] is not None and ms[f] > 0 for f in factors)
        assert ms[best] == min(ms.values())
        after = sim.state()
        for x, y in zip(before, after):
            assert np.array_equal(x, y)
        keys, ids = sim.bins()
        a, b, *_ = sim.contacts()
        sim.step(12)  # steps and rebuilds run on the tuned grid
        assert sim.audit() == 0
    sc2 = dataclasses.replace(sc, bin_size=sc.bin_size * best)
    om, k_o, i_o, a_o, b_o, ws_o, ww_o = _oracle_lists(oracle_mod, sc2, margin, K)
    assert np.array_equal(keys, k_o) and np.array_equal(ids, i_o)
    assert np.array_equal(a, a_o) and np.array_equal(b, b_o)


def _compare_forces(sc, F, T, Fo, To, mag, tol):
    scaleF = np.maximum(mag[:, 0], 1e-300)
    scaleT = np.maximum(mag[:, 1], 1e-300)
    errF = np.abs(F - Fo).max(axis=1) / scaleF
    errT = np.abs(T - To).max(axis=1) / scaleT
    touched = mag[:, 0] > 0
    assert touched.sum() > 0.3 * len(F)
    assert errF[touched].max() <= tol, f"force error {errF[touched].max():.3e}"
    assert errT[touched].max() <= tol, f"torque error {errT[touched].max():.3e}"
    # untouched clumps get exactly nothing
    assert np.all(F[~touched] == 0) and np.all(T[~touched] == 0)
    return errF[touched].max(), errT[touched].max()


def _net_force_error(sc, F, Fo, mag):
    """Each clump's force error relative to its net force |F_ref|, floored
    at 1e-3 m |g| (a clump at rest under balanced contacts has a net force
    near zero whatever the precision), and the ratio of the contributions'
    sum to that net force (the cancellation that separates the two bounds)."""
    m = sc.tpl_mass[sc.tpl]
    g = float(np.linalg.norm(sc.g))
    net = np.maximum(np.linalg.norm(Fo, axis=1), 1e-3 * m * g)
    touched = mag[:, 0] > 0
    err = np.linalg.norm(F - Fo, axis=1)[touched] / net[touched]
    cancel = mag[touched, 0] / net[touched]
    return err, cancel


@pytest.mark.parametrize("prec", [scenes.PREC_FP64, scenes.PREC_FP32])
@pytest.mark.parametrize("seed,n", [(4, 300), (5, 777)])
def test_forces_match_oracle(dem, oracle_mod, prec, seed, n):
    margin, K = 1e-4, 10
    sc = _scene(seed, n, prec, margin=margin)
    with dem.Simulation(sc, margin=margin, rebuild_interval=K) as sim:
        F, T = sim.eval_forces()
        Fw = sim.wall_forces()
        st = sim.stats()
    om, _, _, a, b, ws, ww = _oracle_lists(oracle_mod, sc, margin, K)
    Fo, To, Fwo, _, _, act, mag = om.forces(sc.tpl, sc.pos, sc.quat, sc.vel, sc.angvel, 0.0, a, b,
                                            np.zeros((len(a), 3)), ws, ww, np.zeros((len(ws), 3)),
                                            with_mag=True)
    assert st["active_last"] == act
    _compare_forces(sc, F, T, Fo, To, mag, TOL[prec])
    # the error against the net force floored at 1e-3 m |g| (reading A17):
    # within TOL itself, on these cases where the contributions cancel by up
    # to 21x (reported)
    err, cancel = _net_force_error(sc, F, Fo, mag)
    assert err.max() <= TOL[prec], (err.max(), cancel.max())
    print(f"net-force error prec={prec} n={n}: median {np.median(err):.2e} p99 "
          f"{np.percentile(err, 99):.2e} max {err.max():.2e}; cancellation median "
          f"{np.median(cancel):.1f} max {cancel.max():.1f}")
    if len(ws):
        assert np.abs(Fw - Fwo).max() <= TOL[prec] * np.abs(Fwo).sum()


@pytest.mark.parametrize("prec", [scenes.PREC_FP64, scenes.PREC_FP32])
@pytest.mark.parametrize("mix", [1, 2])
def test_forces_match_oracle_min_max_mixing(dem, oracle_mod, prec, mix):
    """The min and max rules for mu and CoR (section 2.1: each sphere has its
    own mu and CoR; reading A2 mixes them per contact): forces and torques
    within the tolerance, on a bed where most listed pairs join spheres of
    different materials (E, nu, mu and CoR all differ between the three)."""
    margin, K = 1e-4, 10
    sc = _scene(5, 600, prec, margin=margin)
    sc.mix_rule = mix
    with dem.Simulation(sc, margin=margin, rebuild_interval=K) as sim:
        F, T = sim.eval_forces()
        st = sim.stats()
    om, _, _, a, b, ws, ww = _oracle_lists(oracle_mod, sc, margin, K)
    _, _, tsph = om.sphere_centres(sc.tpl, sc.pos, sc.quat)
    mats = np.asarray(sc.tpl_mat)[tsph]
    assert (mats[a] != mats[b]).sum() > 0.4 * len(a)
    assert len(set(np.asarray(sc.mu))) == 3 and len(set(np.asarray(sc.cor))) == 3
    Fo, To, _, _, _, act, mag = om.forces(sc.tpl, sc.pos, sc.quat, sc.vel, sc.angvel, 0.0, a, b,
                                          np.zeros((len(a), 3)), ws, ww, np.zeros((len(ws), 3)),
                                          with_mag=True)
    assert st["active_last"] == act
    _compare_forces(sc, F, T, Fo, To, mag, TOL[prec])
    # the rule matters on this bed: the mean rule moves some clump's force by
    # far more than the tolerance
    Fm = oracle_mod.OracleModel(dataclasses.replace(sc, mix_rule=0)).forces(
        sc.tpl, sc.pos, sc.quat, sc.vel, sc.angvel, 0.0, a, b, np.zeros((len(a), 3)), ws, ww,
        np.zeros((len(ws), 3)))[0]
    touched = mag[:, 0] > 0
    assert (np.abs(Fm - Fo).max(axis=1)[touched] / mag[touched, 0]).max() > 1e3 * TOL[prec]


def _run_both(dem, oracle_mod, sc, margin, K, nsteps, prec, graphs=False):
    sim = dem.Simulation(sc, margin=margin, rebuild_interval=K, precision=prec)
    sim.set_graphs(graphs)
    sim.step(nsteps)
    osim = oracle_mod.OracleSim(sc, margin, K)
    osim.step(nsteps)
    return sim, osim


@pytest.mark.parametrize("graphs", [False, True])
def test_fp64_trajectory_matches_oracle(dem, oracle_mod, graphs):
    """45 steps with a rebuild every 10, as ordinary launches and as one
    captured CUDA graph per list interval."""
    margin, K, nsteps = 2e-4, 10, 45
    sc = _scene(7, 250, scenes.PREC_FP64, margin=margin)
    sim, osim = _run_both(dem, oracle_mod, sc, margin, K, nsteps, scenes.PREC_FP64, graphs)
    pos, quat, vel, w = sim.state()
    po, qo, vo, wo = osim.state()
    vs = np.abs(vo).max()
    assert np.abs(pos - po).max() <= 1e-14 * (1 + np.abs(po).max())
    assert np.abs(vel - vo).max() <= 1e-10 * vs
    assert np.abs(quat - qo).max() <= 1e-12
    assert np.abs(w - wo).max() <= 1e-9 * np.abs(wo).max()
    a, b, u, ws, ww, uw = sim.contacts()
    ao, bo, uo, wso, wwo, uwo = osim.contacts()
    assert np.array_equal(a, ao) and np.array_equal(b, bo)
    assert np.array_equal(ws, wso) and np.array_equal(ww, wwo)
    assert np.abs(uo).max() > 0
    assert np.abs(u - uo).max() <= 1e-8 * np.abs(uo).max()
    if len(uwo):
        assert np.abs(uw - uwo).max() <= 1e-8 * max(np.abs(uwo).max(), 1e-30)
    sim.close()


@pytest.mark.parametrize("graphs", [False, True])
def test_fp32_voxel_trajectory_error_is_bounded(dem, oracle_mod, graphs):
    """Precision mode FP32_VOXEL against the FP64 oracle over 45 steps: the
    position and velocity errors stay at the level set by float forces."""
    margin, K, nsteps = 2e-4, 10, 45
    sc = _scene(8, 250, scenes.PREC_FP32, margin=margin, compress=1.0, jitter=0.05)
    sim, osim = _run_both(dem, oracle_mod, sc, margin, K, nsteps, scenes.PREC_FP32, graphs)
    pos, quat, vel, w = sim.state()
    po, qo, vo, wo = osim.state()
    dv = np.abs(vel - vo).max() / np.abs(vo - sc.vel).max()
    dx = np.abs(pos - po).max() / np.abs(po - sc.pos).max()
    # errors relative to the change over the run
    assert dv < 1e-5, dv
    assert dx < 1e-5, dx
    a, b, *_ = sim.contacts()
    ao, bo, *_ = osim.contacts()
    assert np.array_equal(a, ao) and np.array_equal(b, bo)
    sim.close()


def _wall_scene(prec, seed=9):
    """Clumps inside a cylinder with a floor, a cone pushed down through them
    and a tilted moving plane; a few clumps are placed just inside the reach
    of each wall so that every wall has contacts."""
    rng = np.random.default_rng(seed)
    half = math.radians(30.0)
    H = 0.01 / math.tan(half)
    tilt = np.array([0.0, -0.6, -0.8])
    walls = [scenes.plane((0, 0, 0), (0, 0, 1)), scenes.cylinder((0.03, 0.03, 0), (0, 0, 1), 0.025),
             scenes.cone((0.03, 0.03, 0.02), (0, 0, 1), half, H, vel=(0.0, 0.0, -0.01)),
             scenes.plane((0, 0.05, 0.05), tilt, vel=(0.2, 0.0, 0.0))]
    sc = scenes.packed_scene(seed, 400, precision=prec, compress=0.95, walls=False, vel_scale=0.02)
    sc.walls = walls
    n = len(sc.tpl)
    bound = sc.bounding_radius()[sc.tpl]
    r = 0.02 * np.sqrt(rng.random(n))
    th = 2 * math.pi * rng.random(n)
    z = 0.002 + 0.03 * rng.random(n)
    P = np.stack([0.03 + r * np.cos(th), 0.03 + r * np.sin(th), z], axis=1)
    near = rng.uniform(0.5, 1.1, size=n) * bound
    for i in range(0, 40):          # floor
        P[i, 2] = near[i]
    for i in range(40, 80):         # cylinder wall, from inside
        P[i, 0] = 0.03 + (0.025 - near[i]) * math.cos(th[i])
        P[i, 1] = 0.03 + (0.025 - near[i]) * math.sin(th[i])
    for i in range(80, 110):        # cone lateral surface, from outside
        t = rng.uniform(0.2, 0.9)
        on = np.array([t * H * math.tan(half), 0.0, t * H])
        nout = np.array([math.cos(half), 0.0, -math.sin(half)])
        q = on + near[i] * nout
        c, s_ = math.cos(th[i]), math.sin(th[i])
        P[i] = [0.03 + c * q[0], 0.03 + s_ * q[0], 0.02 + q[2]]
    for i in range(110, 130):       # below the cone tip
        P[i] = [0.03, 0.03, 0.02 - near[i]]
    for i in range(130, 160):       # tilted plane, from the grains' side
        base = np.array([rng.uniform(0.015, 0.045), 0.05, 0.05])
        along = np.array([0.0, 0.8, -0.6]) * rng.uniform(-0.004, 0.004)
        P[i] = base + along - tilt * near[i]
    sc.pos = P
    sc.lo, sc.hi = (0.0, 0.0, -1.0 / 128), (0.06, 0.06, 0.07)
    if prec == scenes.PREC_FP32:
        sc.tpl_pos = sc.tpl_pos.astype(np.float32).astype(np.float64)
        sc.tpl_rad = sc.tpl_rad.astype(np.float32).astype(np.float64)
        scenes.snap_to_voxel_grid(sc)
    sc.bin_size = scenes.default_bin_size(sc, 1e-4)
    return sc


@pytest.mark.parametrize("prec", [scenes.PREC_FP64, scenes.PREC_FP32])
def test_walls_plane_cylinder_cone(dem, oracle_mod, prec):
    margin, K = 1e-4, 10
    sc = _wall_scene(prec)
    with dem.Simulation(sc, margin=margin, rebuild_interval=K) as sim:
        F, T = sim.eval_forces()
        Fw = sim.wall_forces()
        Fl, Tl = sim.wall_loads()
        a, b, u, ws, ww, uw = sim.contacts()
    om, _, _, ao, bo, wso, wwo = _oracle_lists(oracle_mod, sc, margin, K)
    assert np.array_equal(ws, wso) and np.array_equal(ww, wwo)
    assert set(np.unique(ww)) == {0, 1, 2, 3}
    Fo, To, Fwo, _, _, act, mag, Two = om.forces(sc.tpl, sc.pos, sc.quat, sc.vel, sc.angvel, 0.0,
                                                 ao, bo, np.zeros((len(ao), 3)), wso, wwo,
                                                 np.zeros((len(wso), 3)), with_mag=True,
                                                 wall_torque=True)
    _compare_forces(sc, F, T, Fo, To, mag, TOL[prec])
    assert np.array_equal(Fl, Fw)
    extent = 0.07  # every lever arm about a wall's reference point is shorter
    for k in range(4):
        assert np.abs(Fw[k] - Fwo[k]).max() <= TOL[prec] * max(np.abs(Fwo).sum(), 1e-30)
        assert np.abs(Tl[k] - Two[k]).max() <= TOL[prec] * extent * np.abs(Fwo).sum()
        assert np.abs(Two[k]).max() > 0


@pytest.mark.parametrize("prec", [scenes.PREC_FP64, scenes.PREC_FP32])
def test_audit_finds_no_miss_with_an_adequate_margin(dem, prec):
    """While the displacement certificate holds (every clump moved less than
    the margin since the last rebuild), the exact check finds no miss."""
    sc = _scene(10, 400, prec, margin=2e-4, compress=1.1, jitter=0.02, vel_scale=0.05)
    certified = 0
    with dem.Simulation(sc, margin=2e-4, rebuild_interval=20) as sim:
        for _ in range(6):
            before = sim.stats()["guard_violations"]
            sim.step(15)
            if sim.stats()["guard_violations"] == before:
                certified += 1
                assert sim.audit() == 0
        assert sim.stats()["n_pairs"] > 30
    assert certified >= 3


def test_guard_and_audit_catch_a_margin_that_is_too_small(dem):
    sc = _scene(11, 300, scenes.PREC_FP64, margin=1e-7)
    sc.vel = sc.vel * 20.0  # 1 m/s class speeds: 1e-4 m per 100 steps
    with dem.Simulation(sc, margin=1e-7, rebuild_interval=100000) as sim:
        sim.step(100)
        assert sim.stats()["guard_violations"] > 0
        assert sim.audit() > 0


def test_degenerate_inputs(dem):
    # no clumps at all
    sc = single_sphere_scene([1e-3], g=(0, 0, -9.81))
    set_clumps(sc, [], np.zeros((0, 3)))
    with dem.Simulation(sc, margin=1e-5, rebuild_interval=5) as sim:
        sim.step(3)
        assert sim.contacts()[0].size == 0
    # one clump: falls freely, no pairs
    sc = single_sphere_scene([1e-3], g=(0, 0, -9.81), h=1e-5)
    set_clumps(sc, [0], [[0.0, 0.0, 0.0]])
    with dem.Simulation(sc, margin=1e-5, rebuild_interval=5) as sim:
        sim.step(10)
        pos, _, vel, _ = sim.state()
        assert vel[0, 2] == pytest.approx(-9.81 * 1e-4, rel=1e-12)
        assert pos[0, 2] == pytest.approx(-9.81 * 1e-10 * 55, rel=1e-12)
        assert sim.contacts()[0].size == 0
    # spheres outside the detection domain still collide
    sc = single_sphere_scene([1e-3, 1e-3], lo=(0, 0, 0), hi=(0.01, 0.01, 0.01))
    set_clumps(sc, [0, 1], [[-0.004, 0.005, 0.005], [-0.0021, 0.005, 0.005]])
    with dem.Simulation(sc, margin=1e-5, rebuild_interval=5, bin_size=2e-3) as sim:
        F, T = sim.eval_forces()
        assert F[1, 0] > 0 and F[0, 0] < 0


@pytest.mark.parametrize("case", ["one_bin", "wide_margin"])
def test_detection_extremes_bit_exact(dem, oracle_mod, case):
    """Degenerate binning: every registration in a single bin (the narrow phase
    walks 25 tiles of one bin); and a margin wide enough that the pair list
    outgrows the first pair buffer (2^16 pairs here; the find pass regrows
    it and runs again)."""
    if case == "one_bin":
        margin, K = 1e-4, 10
        sc = _scene(11, 300, scenes.PREC_FP64, margin=margin)
        sc.bin_size = 2.0  # one bin covers the whole domain
    else:
        margin, K = 2.5e-3, 10
        sc = _scene(12, 1500, scenes.PREC_FP64, margin=margin)
    with dem.Simulation(sc, margin=margin, rebuild_interval=K) as sim:
        sim.rebuild()
        keys, ids = sim.bins()
        a, b, *_ = sim.contacts()
        st = sim.stats()
    om, k_o, i_o, a_o, b_o, ws_o, ww_o = _oracle_lists(oracle_mod, sc, margin, K)
    if case == "one_bin":
        assert len(np.unique(keys)) == 1 and len(keys) > 25 * 32 - 32
    else:
        assert len(a_o) > max(2 * st["n_spheres"], 1 << 16)
    assert np.array_equal(keys, k_o) and np.array_equal(ids, i_o)
    assert np.array_equal(a, a_o) and np.array_equal(b, b_o)


def test_non_finite_input_rejected(dem):
    sc = single_sphere_scene([1e-3], g=(0, 0, -9.81))
    set_clumps(sc, [0], [[0.0, 0.0, np.nan]])
    with pytest.raises(dem.DemError, match="NONFINITE"):
        dem.Simulation(sc, margin=1e-5)


@pytest.mark.parametrize("prec", [scenes.PREC_FP64, scenes.PREC_FP32])
def test_set_state_converts_on_the_device(dem, oracle_mod, prec):
    """A state set after the first rebuild is staged as given and converted by
    kernels: quaternions and velocities unchanged; positions exact in FP64 and,
    in FP32_VOXEL, split into rint((x - lo) 2^20) voxels plus the float of the
    remainder (restated here in numpy); body-frame angular velocity that
    rotates back to the given one; sphere poses refreshed, so the forces are
    the oracle's for the new state.  Rejected states (a non-finite value, a
    position beyond the int32 voxel range) leave the records untouched."""
    margin, K, n = 1e-4, 10, 400
    sc = _scene(6, n, prec, margin=margin)
    rng = np.random.default_rng(17)
    pos = sc.pos + rng.uniform(-2e-6, 2e-6, sc.pos.shape)  # off the voxel lattice
    quat = scenes.random_quaternions(rng, n)
    vel = rng.normal(scale=0.1, size=(n, 3))
    angvel = rng.normal(scale=30.0, size=(n, 3))
    with dem.Simulation(sc, margin=margin, rebuild_interval=K) as sim:
        sim.rebuild()  # finalized: the state goes through the device kernels
        sim.set_state(pos, quat, vel, angvel)
        P, Q, V, W = sim.state()
        F, T = sim.eval_forces()
        bad = pos.copy()
        bad[7, 1] = np.inf
        with pytest.raises(dem.DemError, match="NONFINITE"):
            sim.set_state(bad, quat, vel, angvel)
        if prec == scenes.PREC_FP32:
            far = pos.copy()
            far[3, 0] = sc.lo[0] + 3000.0  # 3000 * 2^20 voxels > 2^31
            with pytest.raises(dem.DemError, match="INVALID"):
                sim.set_state(far, quat, vel, angvel)
        after = sim.state()
    assert np.array_equal(Q, quat) and np.array_equal(V, vel)
    if prec == scenes.PREC_FP64:
        expect = pos
    else:
        lo = np.asarray(sc.lo, dtype=np.float64)
        rel = pos - lo
        m = np.rint(rel * 2.0**20)
        off = (rel - m * 2.0**-20).astype(np.float32).astype(np.float64)
        expect = lo + (m * 2.0**-20 + off)
    assert np.array_equal(P, expect)
    assert np.abs(W - angvel).max() <= 1e-13 * np.abs(angvel).max()
    for x, y in zip(after, (P, Q, V, W)):
        assert np.array_equal(x, y)
    moved = dataclasses.replace(sc, pos=expect, quat=quat, vel=vel, angvel=angvel)
    om, _, _, a, b, ws, ww = _oracle_lists(oracle_mod, moved, margin, K)
    Fo, To, _, _, _, _, mag = om.forces(sc.tpl, expect, quat, vel, angvel, 0.0, a, b,
                                        np.zeros((len(a), 3)), ws, ww, np.zeros((len(ws), 3)),
                                        with_mag=True)
    _compare_forces(sc, F, T, Fo, To, mag, TOL[prec])


@pytest.mark.parametrize("prec", [scenes.PREC_FP64, scenes.PREC_FP32])
def test_deterministic_mode_is_bit_reproducible(dem, oracle_mod, prec):
    """The deterministic reduction: three runs (one with captured graphs) give
    bit-identical states after 45 steps with rebuilds, and the trajectory
    still matches the oracle to the precision mode's tolerance."""
    margin, K, nsteps = 2e-4, 10, 45
    if prec == scenes.PREC_FP64:
        sc = _scene(7, 250, prec, margin=margin)
    else:
        sc = _scene(8, 250, prec, margin=margin, compress=1.0, jitter=0.05)
    runs = []
    for graphs in (False, True, False):
        with dem.Simulation(sc, margin=margin, rebuild_interval=K, precision=prec) as sim:
            sim.set_deterministic(True)
            sim.set_graphs(graphs)
            sim.step(nsteps)
            runs.append(sim.state())
            assert sim.stats()["steps"] == nsteps
    for r in runs[1:]:
        for x, y in zip(runs[0], r):
            assert np.array_equal(x, y)
    osim = oracle_mod.OracleSim(sc, margin, K)
    osim.step(nsteps)
    po, qo, vo, wo = osim.state()
    pos, quat, vel, w = runs[0]
    if prec == scenes.PREC_FP64:
        assert np.abs(pos - po).max() <= 1e-14 * (1 + np.abs(po).max())
        assert np.abs(vel - vo).max() <= 1e-10 * np.abs(vo).max()
    else:
        assert np.abs(vel - vo).max() / np.abs(vo - sc.vel).max() < 1e-5
        assert np.abs(pos - po).max() / np.abs(po - sc.pos).max() < 1e-5


@pytest.mark.parametrize("prec", [scenes.PREC_FP32, scenes.PREC_FP64])
def test_launch_shapes_change_no_result(dem, prec):
    """Launch shapes (pair blocks per SM, update block, narrow chunk) change no
    result: in deterministic mode the state after 45 steps with rebuilds is
    bit-identical across shapes; the list and the bins are identical too.  The
    tile autotuner picks shapes from its sets, leaves the state, step count
    and counters as they were, and out-of-range shapes are refused."""
    margin, K, nsteps = 2e-4, 10, 45
    sc = _scene(8, 400, prec, margin=margin, compress=1.0, jitter=0.05)
    shapes = [None, dict(pairs_blocks_per_sm=2, update_block=64, narrow_chunk=3),
              dict(pairs_blocks_per_sm=16, update_block=256, narrow_chunk=1)]
    runs = []
    for sh in shapes:
        with dem.Simulation(sc, margin=margin, rebuild_interval=K) as sim:
            sim.set_deterministic(True)
            if sh:
                sim.set_tiles(**sh)
                assert sim.tiles() == sh
            sim.step(nsteps)
            sim.rebuild()
            a, b, _, ws, ww, _ = sim.contacts()
            runs.append((sim.state(), sim.bins(), (a, b, ws, ww)))
    for state, bins, lists in runs[1:]:
        for x, y in zip(runs[0][0], state):
            assert np.array_equal(x, y)
        for x, y in zip(runs[0][1] + runs[0][2], bins + lists):
            assert np.array_equal(x, y)
    with dem.Simulation(sc, margin=margin, rebuild_interval=K) as sim:
        sim.step(7)
        before, st0 = sim.state(), sim.stats()
        best = sim.autotune_tiles(steps=3, reps=1)
        assert best["pairs_blocks_per_sm"] in (2, 4, 8, 16)
        assert best["update_block"] in (64, 128, 256)
        assert best["narrow_chunk"] in (2, 4, 8, 16, 32)
        assert sim.tiles() == best
        for x, y in zip(before, sim.state()):
            assert np.array_equal(x, y)
        st1 = sim.stats()
        assert st1["steps"] == st0["steps"] and st1["rebuilds"] == st0["rebuilds"]
        for bad in (dict(update_block=100), dict(pairs_blocks_per_sm=0), dict(narrow_chunk=65)):
            with pytest.raises(dem.DemError, match="INVALID"):
                sim.set_tiles(**bad)
        assert sim.tiles() == best
        sim.step(5)  # still steps after tuning


def test_wall_motion_import_matches_the_motion_given_from_the_start(dem, oracle_mod):
    """Co-simulation hook: a plate held far above the clumps is moved, at step
    20, to 2 um above them and driven down at 0.5 m/s (dem_set_wall_motion);
    it reaches the bed and presses on it.  The run equals the oracle's run of
    the same scene whose plate had that motion from t = 0 (out of reach of the
    clumps until step 20 as well): the same trajectory to the FP64 trajectory
    tolerances, and the same loads on the plate (force and moment about its
    reference point) at the end."""
    margin, K, t1, t2 = 2e-4, 10, 20, 60
    sc = _scene(7, 250, scenes.PREC_FP64, margin=margin)
    # the highest sphere surface of the generated bed
    xs, _, tsph = oracle_mod.OracleModel(sc).sphere_centres(sc.tpl, sc.pos, sc.quat)
    top = float((xs[:, 2] + sc.tpl_rad[tsph]).max())
    v = np.array([0.0, 0.0, -0.5])
    near = np.array([0.0, 0.0, top + 2e-6])  # reached a few steps after the import
    sc_gpu = dataclasses.replace(sc, walls=list(sc.walls) + [scenes.plane((0, 0, top + 0.01), (0, 0, -1))],
                                 hi=(sc.hi[0], sc.hi[1], top + 0.02))
    p0 = near - v * (t1 * sc.h)
    sc_orc = dataclasses.replace(sc_gpu, walls=list(sc.walls) + [scenes.plane(p0, (0, 0, -1), vel=v)])
    plate = len(sc.walls)
    with dem.Simulation(sc_gpu, margin=margin, rebuild_interval=K) as sim:
        sim.step(t1)
        sim.set_wall_motion(plate, near, v)
        sim.step(t2 - t1)
        pos, quat, vel, w = sim.state()
        sim.eval_forces()
        Fl, Tl = sim.wall_loads()
        with pytest.raises(dem.DemError, match="INVALID"):
            sim.set_wall_motion(plate + 1, near, v)
    osim = oracle_mod.OracleSim(sc_orc, margin, K)
    osim.step(t2)
    po, qo, vo, wo = osim.state()
    assert np.abs(pos - po).max() <= 1e-14 * (1 + np.abs(po).max())
    assert np.abs(vel - vo).max() <= 1e-10 * np.abs(vo).max()
    assert np.abs(w - wo).max() <= 1e-9 * np.abs(wo).max()
    # the plate pushes on the bed by now: its loads with the oracle's own list
    # and histories at the end of its run (the lists were rebuilt at the same
    # steps; the histories agree to the trajectory tolerance)
    ao, bo, uo, wso, wwo, uwo = osim.contacts()
    om = oracle_mod.OracleModel(sc_orc)
    _, _, Fwo, _, _, _, Two = om.forces(sc.tpl, po, qo, vo, wo, t2 * sc.h, ao, bo, uo, wso, wwo,
                                        uwo, wall_torque=True)
    assert Fwo[plate][2] > 0 and Fl[plate][2] > 0  # the bed pushes the plate up
    scale = np.abs(Fwo[plate]).sum()
    assert np.abs(Fl[plate] - Fwo[plate]).max() <= 1e-7 * scale
    assert np.abs(Tl[plate] - Two[plate]).max() <= 1e-7 * scale * 0.1


def test_virtual_compressor_reaches_its_load_and_holds(dem):
    """Sample preparation's compressor, built on the co-simulation hook: a
    plate above the bed is driven down at 0.5 m/s until the grains push back
    with 0.2 N, then held; the load was reached before the step budget ran
    out, the plate moved by speed x time, and after 50 more steps it still
    carries load, the displacement certificate never failed and no contact
    is missing from the list."""
    from paper_2307_03445_gb300 import workloads

    margin, K = 2e-4, 10
    # a loose lattice (no initial overlaps) with slow clumps
    sc = _scene(13, 300, scenes.PREC_FP64, margin=margin, compress=1.1, jitter=0.02,
                vel_scale=0.01)
    top = float((sc.pos[:, 2] + sc.bounding_radius()[sc.tpl]).max()) + 2e-5
    plate = scenes.plane((0.0, 0.0, top), (0, 0, -1))
    sc2 = dataclasses.replace(sc, walls=list(sc.walls) + [plate], hi=(sc.hi[0], sc.hi[1], top + 0.01))
    k = len(sc.walls)
    with dem.Simulation(sc2, margin=margin, rebuild_interval=K) as sim:
        steps, push, p = workloads.compress(sim, plate, k, speed=0.5, load=0.2, max_steps=20_000)
        assert push >= 0.2 and steps < 20_000
        assert p[2] == pytest.approx(top - 0.5 * steps * sc.h, abs=1e-12)
        sim.step(50)
        F, T = sim.wall_loads()
        assert F[k][2] > 0.0  # still loaded: the grains push the held plate up
        assert sim.stats()["guard_violations"] == 0
        assert sim.audit() == 0


def test_set_state_uses_each_clumps_own_scene_corner(dem):
    """Two scenes in one context, the second shifted by (0.5, 0.25, 0.125) m:
    a state set on the device is split into voxel + offset against each
    clump's own scene corner (restated here in numpy)."""
    margin = 1e-4
    sc = _scene(6, 300, scenes.PREC_FP32, margin=margin)
    d = np.array([0.5, 0.25, 0.125])  # powers of two: the copy stays on the voxel grid
    walls2 = [dict(w, p=tuple(np.asarray(w["p"]) + d)) for w in sc.walls]
    sc2 = dataclasses.replace(sc, pos=sc.pos + d, lo=tuple(np.asarray(sc.lo) + d),
                              hi=tuple(np.asarray(sc.hi) + d), walls=walls2)
    rng = np.random.default_rng(23)
    n = len(sc.tpl)
    pos = np.concatenate([sc.pos, sc2.pos]) + rng.uniform(-2e-6, 2e-6, (2 * n, 3))
    quat = scenes.random_quaternions(rng, 2 * n)
    vel = rng.normal(scale=0.1, size=(2 * n, 3))
    angvel = rng.normal(scale=30.0, size=(2 * n, 3))
    with dem.Simulation(sc, margin=margin, rebuild_interval=10, extra_scenes=[sc2]) as sim:
        sim.rebuild()
        sim.set_state(pos, quat, vel, angvel)
        P, Q, V, W = sim.state()
        sim.step(3)  # and the scenes step
    lo = np.concatenate([np.tile(sc.lo, (n, 1)), np.tile(sc2.lo, (n, 1))])
    rel = pos - lo
    m = np.rint(rel * 2.0**20)
    off = (rel - m * 2.0**-20).astype(np.float32).astype(np.float64)
    assert np.array_equal(P, lo + (m * 2.0**-20 + off))
    assert np.array_equal(Q, quat) and np.array_equal(V, vel)


def _mesh_scene(prec, seed=12):
    """Clumps in a funnel built from 16 facets over a floor of 2 facets that
    rises at 1 cm/s; 180 clumps are placed within reach of a facet, over its
    face, beyond its edges or near its vertices (where neighbouring facets
    share the contact), the rest inside the funnel."""
    rng = np.random.default_rng(seed)
    walls = scenes.funnel_mesh(0.03, 0.03, 0.0, 0.035, 0.015, 0.027, 8)
    walls += scenes.mesh([(0.0, 0.0, 0.0), (0.06, 0.0, 0.0), (0.06, 0.06, 0.0), (0.0, 0.06, 0.0)],
                         [(0, 1, 2), (0, 2, 3)], (0.03, 0.03, 1.0), vel=(0.0, 0.0, 0.01))
    sc = scenes.packed_scene(seed, 400, precision=prec, compress=0.95, walls=False, vel_scale=0.02)
    sc.walls = walls
    n = len(sc.tpl)
    bound = sc.bounding_radius()[sc.tpl]
    z = 0.004 + 0.026 * rng.random(n)
    rad = (0.9 * (0.015 + 0.012 * z / 0.035) - 1.5 * bound) * np.sqrt(rng.random(n))
    th = 2 * math.pi * rng.random(n)
    P = np.stack([0.03 + rad * np.cos(th), 0.03 + rad * np.sin(th), z], axis=1)
    for i in range(180):
        f = walls[i % len(walls)]
        a, b, c, nf = (np.asarray(f[k]) for k in ("p", "b", "c", "n"))
        u, v = rng.random(2)
        if u + v > 1:
            u, v = 1 - u, 1 - v
        if i % 3 == 2:  # beyond an edge or a vertex
            u, v = u * 1.25 - 0.1, v * 1.25 - 0.1
        P[i] = a + u * (b - a) + v * (c - a) + rng.uniform(0.5, 1.1) * bound[i] * nf
    sc.pos = P
    sc.lo, sc.hi = (0.0, 0.0, -1.0 / 128), (0.06, 0.06, 0.07)
    if prec == scenes.PREC_FP32:
        sc.tpl_pos = sc.tpl_pos.astype(np.float32).astype(np.float64)
        sc.tpl_rad = sc.tpl_rad.astype(np.float32).astype(np.float64)
        scenes.snap_to_voxel_grid(sc)
    sc.bin_size = scenes.default_bin_size(sc, 1e-4)
    return sc


@pytest.mark.parametrize("prec", [scenes.PREC_FP64, scenes.PREC_FP32])
def test_mesh_facets_match_oracle(dem, oracle_mod, prec):
    """Sphere-facet candidate lists bit-exact; clump forces, per-facet loads
    and moments within the tolerance; a mesh's load is its facets' sum."""
    margin, K = 1e-4, 10
    sc = _mesh_scene(prec)
    with dem.Simulation(sc, margin=margin, rebuild_interval=K) as sim:
        F, T = sim.eval_forces()
        Fl, Tl = sim.wall_loads()
        a, b, u, ws, ww, uw = sim.contacts()
    om, _, _, ao, bo, wso, wwo = _oracle_lists(oracle_mod, sc, margin, K)
    assert np.array_equal(ws, wso) and np.array_equal(ww, wwo)
    assert len(np.unique(ww)) >= 16  # nearly every facet is reached
    Fo, To, Fwo, _, _, act, mag, Two = om.forces(sc.tpl, sc.pos, sc.quat, sc.vel, sc.angvel, 0.0,
                                                 ao, bo, np.zeros((len(ao), 3)), wso, wwo,
                                                 np.zeros((len(wso), 3)), with_mag=True,
                                                 wall_torque=True)
    _compare_forces(sc, F, T, Fo, To, mag, TOL[prec])
    scale = np.abs(Fwo).sum()
    extent = 0.07
    assert np.abs(Fl - Fwo).max() <= TOL[prec] * scale
    assert np.abs(Tl - Two).max() <= TOL[prec] * extent * scale
    assert np.abs(Fl[:16].sum(axis=0) - Fwo[:16].sum(axis=0)).max() <= TOL[prec] * scale
    assert (np.abs(Fwo).max(axis=1) > 0).sum() >= 14


def test_fp64_trajectory_in_a_box_mesh_matches_oracle(dem, oracle_mod):
    """A packed bed settling in a box made of 12 facets: 45 steps with a
    rebuild every 10 against the oracle, as the FP64 trajectory test does
    for analytic walls."""
    margin, K, nsteps = 2e-4, 10, 45
    sc = _scene(7, 250, scenes.PREC_FP64, margin=margin)
    planes = sc.walls
    lo, hi = np.array(sc.lo), np.array(sc.hi)
    x0 = max(w["p"][0] for w in planes if w["n"][0] > 0.5)
    x1 = min(w["p"][0] for w in planes if w["n"][0] < -0.5)
    y0 = max(w["p"][1] for w in planes if w["n"][1] > 0.5)
    y1 = min(w["p"][1] for w in planes if w["n"][1] < -0.5)
    z0 = max(w["p"][2] for w in planes if w["n"][2] > 0.5)
    sc.walls = scenes.box_mesh(x0, x1, y0, y1, z0, hi[2] - 1e-3)
    sim, osim = _run_both(dem, oracle_mod, sc, margin, K, nsteps, scenes.PREC_FP64)
    pos, quat, vel, w = sim.state()
    po, qo, vo, wo = osim.state()
    assert np.abs(pos - po).max() <= 1e-14 * (1 + np.abs(po).max())
    assert np.abs(vel - vo).max() <= 1e-10 * np.abs(vo).max()
    assert np.abs(w - wo).max() <= 1e-9 * np.abs(wo).max()
    a, b, u, ws, ww, uw = sim.contacts()
    ao, bo, uo, wso, wwo, uwo = osim.contacts()
    assert np.array_equal(ws, wso) and np.array_equal(ww, wwo) and len(ws) > 10
    assert np.abs(uw - uwo).max() <= 1e-8 * max(np.abs(uwo).max(), 1e-30)
    sim.close()
