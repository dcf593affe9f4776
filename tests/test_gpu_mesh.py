"""Meshes of many facets (section 4's cone, funnel and wheel boundaries are
triangle meshes): facets registered in the detection bins, found through
them, against the oracle's test of every sphere against every facet.

Candidate lists bit-exact; clump forces, per-facet loads and moments within
the precision mode's tolerance; an FP64 trajectory with the cone moving into
the bed within the trajectory tolerances.
"""
import math

import numpy as np
import pytest

from paper_2307_03445_gb300 import scenes

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


def _sphere_centres(sc):
    """Sphere centres X + R(q) p of every clump (input preparation)."""
    w, x, y, z = (sc.quat[:, k] for k in range(4))
    R = np.stack([1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y),
                  2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x),
                  2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)],
                 axis=1).reshape(-1, 3, 3)
    out = []
    for i, t in enumerate(sc.tpl):
        s0, s1 = sc.tpl_off[t], sc.tpl_off[t + 1]
        out.append(sc.pos[i] + sc.tpl_pos[s0:s1] @ R[i].T)
    return out


def cone_bed(prec, seed=41, n=1500, nseg=32, nrings=9, depth=0.014, every=4):
    """A packed bed of clumps in a box of planes and an open cone of 544
    facets (30 degree half angle, 2 cm base) whose tip sits `depth` below the
    bed's top at its centre, pushed down at 1 cm/s.  Bed clumps with a sphere
    centre inside the cone or within 50 um of its side are taken out; then a
    clump of the smallest template is placed in front of every `every`-th
    facet, its bounding sphere 10 um into to 80 um clear of the facet's
    plane, and the bed clumps it would overlap are taken out too."""
    rng = np.random.default_rng(seed + 100)
    sc = scenes.packed_scene(seed, n, precision=prec, compress=0.95, vel_scale=0.02)
    bound_t = sc.bounding_radius()
    bound = bound_t[sc.tpl]
    top = float((sc.pos[:, 2] + bound).max())
    cx, cy = (float(v) for v in sc.pos[:, :2].mean(axis=0))
    half = math.radians(30.0)
    H = 0.01 / math.tan(half)
    tip = np.array([cx, cy, top - depth])
    mesh = scenes.cone_mesh(tuple(tip), half, H, nseg, nrings, vel=(0.0, 0.0, -0.01), base=False)
    keep = np.ones(len(sc.tpl), bool)
    for i, xs in enumerate(_sphere_centres(sc)):
        dz = xs[:, 2] - tip[2]
        rho = np.hypot(xs[:, 0] - cx, xs[:, 1] - cy)
        side = (rho - dz * math.tan(half)) * math.cos(half)  # outside the side (negative inside)
        keep[i] = not ((dz > -5e-5) & (dz < H + 5e-5) & (side < 5e-5)).any()
    small = int(np.argmin(bound_t))
    placed = []
    for f in mesh[::every]:
        a, b, c, nf = (np.asarray(f[k]) for k in ("p", "b", "c", "n"))
        centre = (a + b + c) / 3.0
        if centre[2] > top - 0.5 * bound_t[small]:
            continue  # above the bed
        placed.append(centre + nf * (bound_t[small] + rng.uniform(-1e-5, 8e-5)))
    placed = np.array(placed)
    for i in range(len(sc.tpl)):
        if keep[i] and len(placed):
            gap = np.linalg.norm(placed - sc.pos[i], axis=1) - bound[i] - bound_t[small]
            keep[i] = gap.min() > 0.0
    m = len(placed)
    sc.tpl = np.concatenate([sc.tpl[keep], np.full(m, small, np.int32)])
    sc.pos = np.concatenate([sc.pos[keep], placed])
    sc.quat = np.concatenate([sc.quat[keep], scenes.random_quaternions(rng, m)])
    sc.vel = np.concatenate([sc.vel[keep], rng.normal(scale=0.02, size=(m, 3))])
    sc.angvel = np.concatenate([sc.angvel[keep], np.zeros((m, 3))])
    sc.walls = list(sc.walls) + mesh
    sc.hi = (sc.hi[0], sc.hi[1], top + H + 0.01)
    if prec == scenes.PREC_FP32:
        sc.tpl_pos = sc.tpl_pos.astype(np.float32).astype(np.float64)
        sc.tpl_rad = sc.tpl_rad.astype(np.float32).astype(np.float64)
        scenes.snap_to_voxel_grid(sc)
    sc.bin_size = scenes.default_bin_size(sc, 1e-4)
    return sc, len(sc.walls) - len(mesh)


def _oracle_lists(oracle_mod, sc, margin, K):
    om = oracle_mod.OracleModel(sc)
    xs, owner, tsph = om.sphere_centres(sc.tpl, sc.pos, sc.quat)
    qc, rho = om.detect_coords(xs, tsph, margin)
    a, b = om.pairs_binned(owner, qc, rho)
    ws, ww = om.wall_candidates(xs, tsph, margin, 0.0, sc.h * K)
    return om, a, b, ws, ww


@pytest.mark.parametrize("prec", [scenes.PREC_FP64, scenes.PREC_FP32])
def test_cone_mesh_of_544_facets_matches_oracle(dem, oracle_mod, prec):
    margin, K = 1e-4, 10
    sc, first_facet = cone_bed(prec)
    n_facets = len(sc.walls) - first_facet
    assert n_facets == 544
    with dem.Simulation(sc, margin=margin, rebuild_interval=K) as sim:
        F, T = sim.eval_forces()
        Fl, Tl = sim.wall_loads()
        a, b, u, ws, ww, uw = sim.contacts()
    om, ao, bo, wso, wwo = _oracle_lists(oracle_mod, sc, margin, K)
    assert np.array_equal(a, ao) and np.array_equal(b, bo)
    assert np.array_equal(ws, wso) and np.array_equal(ww, wwo)
    hit = np.unique(ww[ww >= first_facet])
    assert len(hit) >= 200  # the spheres around the cone reach a large part of its facets
    Fo, To, Fwo, _, _, act, mag, Two = om.forces(sc.tpl, sc.pos, sc.quat, sc.vel, sc.angvel, 0.0,
                                                 ao, bo, np.zeros((len(ao), 3)), wso, wwo,
                                                 np.zeros((len(wso), 3)), with_mag=True,
                                                 wall_torque=True)
    touched = mag[:, 0] > 0
    errF = (np.abs(F - Fo).max(axis=1)[touched] / mag[touched, 0]).max()
    errT = (np.abs(T - To).max(axis=1)[touched] / mag[touched, 1]).max()
    assert errF <= TOL[prec] and errT <= TOL[prec], (errF, errT)
    scale = np.abs(Fwo).sum()
    extent = 0.1  # every lever arm about a facet's reference point is shorter
    assert np.abs(Fl - Fwo).max() <= TOL[prec] * scale
    assert np.abs(Tl - Two).max() <= TOL[prec] * extent * scale
    cone_load = Fwo[first_facet:].sum(axis=0)
    assert cone_load[2] > 0  # the bed pushes the cone up
    assert np.abs(Fl[first_facet:].sum(axis=0) - cone_load).max() <= TOL[prec] * scale


def test_cone_mesh_fp64_trajectory_matches_oracle(dem, oracle_mod):
    """45 steps with a rebuild every 10 while the cone moves into the bed:
    lists, histories and trajectory against the oracle, as the FP64
    trajectory test does for analytic walls."""
    margin, K, nsteps = 2e-4, 10, 45
    sc, first_facet = cone_bed(scenes.PREC_FP64, n=900)
    sim = dem.Simulation(sc, margin=margin, rebuild_interval=K, precision=scenes.PREC_FP64)
    sim.step(nsteps)
    osim = oracle_mod.OracleSim(sc, margin, K)
    osim.step(nsteps)
    pos, quat, vel, w = sim.state()
    po, qo, vo, wo = osim.state()
    assert np.abs(pos - po).max() <= 1e-14 * (1 + np.abs(po).max())
    assert np.abs(vel - vo).max() <= 1e-10 * np.abs(vo).max()
    assert np.abs(w - wo).max() <= 1e-9 * np.abs(wo).max()
    a, b, u, ws, ww, uw = sim.contacts()
    ao, bo, uo, wso, wwo, uwo = osim.contacts()
    assert np.array_equal(a, ao) and np.array_equal(b, bo)
    assert np.array_equal(ws, wso) and np.array_equal(ww, wwo)
    assert (ww >= first_facet).sum() > 50
    assert np.abs(uw - uwo).max() <= 1e-8 * max(np.abs(uwo).max(), 1e-30)
    sim.close()
    osim.close()
