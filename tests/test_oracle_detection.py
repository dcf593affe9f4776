"""Pins of the oracle's geometry and contact detection (section 2.2: enlarged
geometry, binning, exact pair predicate) against brute force, a library
rotation and hand-built cases."""
import math

import numpy as np
import pytest
from scipy.spatial.transform import Rotation

from paper_2307_03445_gb300 import scenes
from tests.helpers import set_clumps, single_sphere_scene

EPS = 2.0 ** -24


def test_sphere_centres_match_library_rotation(oracle_mod):
    sc = scenes.packed_scene(3, 40)
    om = oracle_mod.OracleModel(sc)
    xs, owner, tsph = om.sphere_centres(sc.tpl, sc.pos, sc.quat)
    # scipy uses scalar-last quaternions
    R = Rotation.from_quat(sc.quat[:, [1, 2, 3, 0]])
    ref = sc.pos[owner] + R[owner].apply(sc.tpl_pos[tsph])
    assert np.allclose(xs, ref, rtol=0, atol=1e-15)
    # owner / component bookkeeping
    counts = np.diff(sc.tpl_off)[sc.tpl]
    assert np.array_equal(np.bincount(owner, minlength=len(sc.tpl)), counts)


def test_quarter_turn_about_z(oracle_mod):
    sc = single_sphere_scene([1e-3])
    sc.tpl_off = np.array([0, 1], np.int32)
    sc.tpl_pos = np.array([[1e-3, 0.0, 0.0]])
    om = oracle_mod.OracleModel(sc)
    q = np.array([[math.cos(math.pi / 4), 0, 0, math.sin(math.pi / 4)]])
    xs, _, _ = om.sphere_centres([0], [[0.0, 0.0, 0.0]], q)
    assert np.allclose(xs[0], [0.0, 1e-3, 0.0], atol=1e-18)


@pytest.mark.parametrize("seed", [0, 1, 2, 3])
@pytest.mark.parametrize("bin_scale", [0.3, 1.0, 2.5])
def test_binned_pairs_equal_brute_force(oracle_mod, seed, bin_scale):
    sc = scenes.packed_scene(seed, 50, compress=1.0 + 0.05 * seed)
    margin = 2e-4 * (seed + 1)
    sc.bin_size = bin_scale * scenes.default_bin_size(sc, margin)
    om = oracle_mod.OracleModel(sc)
    xs, owner, tsph = om.sphere_centres(sc.tpl, sc.pos, sc.quat)
    assert len(xs) <= 250
    qc, rho = om.detect_coords(xs, tsph, margin)
    a, b = om.pairs_brute(owner, qc, rho)
    a2, b2 = om.pairs_binned(owner, qc, rho)
    assert len(a) > 20
    assert np.array_equal(a, a2) and np.array_equal(b, b2)
    assert np.all(a < b) and np.all(owner[a] != owner[b])


def test_bin_entries_cover_each_enlarged_box(oracle_mod):
    sc = scenes.packed_scene(5, 30)
    margin = 3e-4
    sc.bin_size = 0.5 * scenes.default_bin_size(sc, margin)
    om = oracle_mod.OracleModel(sc)
    xs, owner, tsph = om.sphere_centres(sc.tpl, sc.pos, sc.quat)
    qc, rho = om.detect_coords(xs, tsph, margin)
    keys, ids = om.bin_entries(qc, rho)
    dims, L = om.grid_dims()
    # sorted by (key, id)
    order = np.lexsort((ids, keys))
    assert np.array_equal(order, np.arange(len(keys)))
    # brute force: the set of bins whose closed cell meets the enlarged box
    for s in range(len(rho)):
        mine = set(keys[ids == s].tolist())
        lo = np.clip(np.floor_divide(qc[s] - rho[s], L), 0, dims - 1)
        hi = np.clip(np.floor_divide(qc[s] + rho[s], L), 0, dims - 1)
        want = {int((z * dims[1] + y) * dims[0] + x)
                for z in range(lo[2], hi[2] + 1) for y in range(lo[1], hi[1] + 1)
                for x in range(lo[0], hi[0] + 1)}
        assert mine == want


def _two_spheres(oracle_mod, gap, margin, r=1e-3):
    sc = single_sphere_scene([r, r], lo=(0.0, 0.0, 0.0), hi=(0.02, 0.02, 0.02))
    sc.bin_size = 4e-3
    x0 = 0.01
    set_clumps(sc, [0, 1], [[x0, 0.01, 0.01], [x0 + 2 * r + gap, 0.01, 0.01]])
    om = oracle_mod.OracleModel(sc)
    xs, owner, tsph = om.sphere_centres(sc.tpl, sc.pos, sc.quat)
    qc, rho = om.detect_coords(xs, tsph, margin)
    return om.pairs_binned(owner, qc, rho), (qc, rho)


def test_pair_inside_enlargement_is_listed(oracle_mod):
    margin = 5e-5
    (a, b), _ = _two_spheres(oracle_mod, 2 * margin - 4 * EPS, margin)
    assert list(zip(a, b)) == [(0, 1)]


def test_pair_beyond_enlargement_is_not_listed(oracle_mod):
    margin = 5e-5
    # the lattice rounds each centre by up to half a unit and adds one unit of slack
    (a, b), (qc, rho) = _two_spheres(oracle_mod, 2 * margin + 8 * EPS, margin)
    assert len(a) == 0


def test_touching_pair_listed_with_zero_margin(oracle_mod):
    (a, b), _ = _two_spheres(oracle_mod, 0.0, 0.0)
    assert list(zip(a, b)) == [(0, 1)]
    (a, b), _ = _two_spheres(oracle_mod, -1e-9, 0.0)
    assert list(zip(a, b)) == [(0, 1)]


def test_spheres_of_one_clump_never_pair(oracle_mod):
    sc = single_sphere_scene([1e-3])
    sc.tpl_off = np.array([0, 3], np.int32)
    sc.tpl_pos = np.array([[0.0, 0, 0], [1e-3, 0, 0], [2e-3, 0, 0]])
    sc.tpl_rad = np.full(3, 1e-3)
    sc.tpl_mat = np.zeros(3, np.int32)
    sc.lo, sc.hi, sc.bin_size = (0.0, 0.0, 0.0), (0.02, 0.02, 0.02), 1e-3
    set_clumps(sc, [0, 0], [[0.005, 0.01, 0.01], [0.0085, 0.01, 0.01]])
    om = oracle_mod.OracleModel(sc)
    xs, owner, tsph = om.sphere_centres(sc.tpl, sc.pos, sc.quat)
    qc, rho = om.detect_coords(xs, tsph, 1e-4)
    a, b = om.pairs_binned(owner, qc, rho)
    # only the two facing end spheres of the two clumps touch: (2, 3)
    assert list(zip(a, b)) == [(2, 3)]


def test_pair_spanning_many_bins_reported_once(oracle_mod):
    # tiny bins: both spheres span dozens of bins per axis, and they share many
    sc = single_sphere_scene([1e-3, 1e-3], lo=(0.0, 0.0, 0.0), hi=(0.02, 0.02, 0.02))
    sc.bin_size = 2.5e-4
    set_clumps(sc, [0, 1], [[0.01, 0.01, 0.01], [0.0112, 0.0103, 0.0098]])
    om = oracle_mod.OracleModel(sc)
    xs, owner, tsph = om.sphere_centres(sc.tpl, sc.pos, sc.quat)
    qc, rho = om.detect_coords(xs, tsph, 1e-4)
    keys, ids = om.bin_entries(qc, rho)
    shared = set(keys[ids == 0]) & set(keys[ids == 1])
    assert len(shared) > 100
    a, b = om.pairs_binned(owner, qc, rho)
    assert list(zip(a, b)) == [(0, 1)]


def test_spheres_outside_domain_are_clamped_not_lost(oracle_mod):
    sc = single_sphere_scene([1e-3, 1e-3], lo=(0.0, 0.0, 0.0), hi=(0.01, 0.01, 0.01))
    sc.bin_size = 2e-3
    set_clumps(sc, [0, 1], [[-0.004, 0.005, 0.005], [-0.0021, 0.005, 0.005]])
    om = oracle_mod.OracleModel(sc)
    xs, owner, tsph = om.sphere_centres(sc.tpl, sc.pos, sc.quat)
    qc, rho = om.detect_coords(xs, tsph, 0.0)
    a, b = om.pairs_binned(owner, qc, rho)
    assert list(zip(a, b)) == [(0, 1)]


# ---------------------------------------------------------------------------
# analytic boundaries
# ---------------------------------------------------------------------------
def _wall_model(oracle_mod, walls):
    sc = single_sphere_scene([1e-3], walls=walls)
    return oracle_mod.OracleModel(sc)


def test_plane_distance_and_motion(oracle_mod):
    om = _wall_model(oracle_mod, [scenes.plane((0, 0, 0.1), (0, 0, -2), vel=(0.3, 0.0, -0.5))])
    d, nw = om.wall_distance(0, 0.0, [1.0, 2.0, 0.07])
    assert d == pytest.approx(0.03, abs=1e-15) and np.allclose(nw, [0, 0, -1])
    d, _ = om.wall_distance(0, 0.02, [1.0, 2.0, 0.07])  # plane moved down by 1 cm
    assert d == pytest.approx(0.02, abs=1e-15)


def test_cylinder_distance(oracle_mod):
    om = _wall_model(oracle_mod, [scenes.cylinder((1.0, 1.0, 0.0), (0, 0, 1), 0.2)])
    d, nw = om.wall_distance(0, 0.0, [1.15, 1.0, 0.3])
    assert d == pytest.approx(0.05, abs=1e-15)
    assert np.allclose(nw, [-1.0, 0.0, 0.0])


def test_cone_distance_closed_forms(oracle_mod):
    half = math.radians(30.0)
    H = 0.01 / math.tan(half)
    om = _wall_model(oracle_mod, [scenes.cone((0.0, 0.0, 0.1), (0, 0, 1), half, H)])
    # straight below the tip
    d, nw = om.wall_distance(0, 0.0, [0.0, 0.0, 0.1 - 0.004])
    assert d == pytest.approx(0.004, abs=1e-15) and np.allclose(nw, [0, 0, -1])
    # off the lateral surface along its outward normal
    t = 0.4
    on = np.array([t * H * math.tan(half), 0.0, 0.1 + t * H])
    nout = np.array([math.cos(half), 0.0, -math.sin(half)])
    d, nw = om.wall_distance(0, 0.0, on + 0.003 * nout)
    assert d == pytest.approx(0.003, abs=1e-14) and np.allclose(nw, nout, atol=1e-12)
    # rotated about the axis: same distance
    c, s = math.cos(1.1), math.sin(1.1)
    p = on + 0.003 * nout
    d2, _ = om.wall_distance(0, 0.0, [c * p[0] - s * p[1], s * p[0] + c * p[1], p[2]])
    assert d2 == pytest.approx(0.003, abs=1e-14)
    # above the base disk
    d, nw = om.wall_distance(0, 0.0, [0.002, 0.0, 0.1 + H + 0.005])
    assert d == pytest.approx(0.005, abs=1e-14) and np.allclose(nw, [0, 0, 1])
    # inside the solid: negative
    d, _ = om.wall_distance(0, 0.0, [0.0, 0.0, 0.1 + 0.5 * H])
    assert d < 0
    # a moving cone: tip moves down 1 cm/s
    om2 = _wall_model(oracle_mod, [scenes.cone((0.0, 0.0, 0.1), (0, 0, 1), half, H, vel=(0, 0, -0.01))])
    d, _ = om2.wall_distance(0, 1.0, [0.0, 0.0, 0.09 - 0.004])
    assert d == pytest.approx(0.004, abs=1e-14)


def test_wall_candidates_use_margin_and_travel(oracle_mod):
    sc = single_sphere_scene([1e-3, 1e-3], walls=[scenes.plane((0, 0, 0), (0, 0, 1)),
                                                  scenes.plane((0, 0, 0.02), (0, 0, -1), vel=(0, 0, -0.1))])
    om = oracle_mod.OracleModel(sc)
    xs = np.array([[0.0, 0.0, 1e-3 + 1.5e-4], [0.0, 0.0, 0.02 - 1e-3 - 3e-4]])
    tsph = np.array([0, 1], np.int32)
    s, w = om.wall_candidates(xs, tsph, 2e-4, 0.0, 0.0)
    assert list(zip(s, w)) == [(0, 0)]
    # the top plate travels 0.1 m/s * 2e-3 s = 2e-4 m during the interval
    s, w = om.wall_candidates(xs, tsph, 2e-4, 0.0, 2e-3)
    assert list(zip(s, w)) == [(0, 0), (1, 1)]
