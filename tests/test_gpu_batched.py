"""Batched independent scenes in one context (the batched sweep of scenes of
uneven size, each with its own friction, templates and materials): a merged
run must be each scene run alone, and each scene's forces the oracle's.

All scenes occupy the same region of space, so any contact across scenes, a
wrong per-scene grid, wall list, voxel corner or shifted template/material id
would change a scene's result.
"""
import numpy as np
import pytest

from paper_2307_03445_gb300 import scenes

pytestmark = pytest.mark.gpu

SIZES = (150, 420, 260)
SEEDS = (31, 32, 33)


@pytest.fixture(scope="module")
def dem():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2307_03445_gb300 as dem

    dem.load_library()
    return dem


def _parts(prec, margin):
    """Three dense scenes of 150, 420 and 260 clumps, each with its own 8
    templates, 3 materials (own mu and CoR) and box, at random velocities."""
    parts = []
    for seed, n in zip(SEEDS, SIZES):
        sc = scenes.packed_scene(seed, n, precision=prec, compress=0.95)
        if prec == scenes.PREC_FP32:
            sc.tpl_pos = sc.tpl_pos.astype(np.float32).astype(np.float64)
            sc.tpl_rad = sc.tpl_rad.astype(np.float32).astype(np.float64)
            scenes.snap_to_voxel_grid(sc)
        sc.bin_size = scenes.default_bin_size(sc, margin)
        parts.append(sc)
    return parts


def _offsets(parts):
    cl = np.cumsum([0] + [p.n_clumps for p in parts])
    sp = np.cumsum([0] + [p.n_spheres for p in parts])
    wl = np.cumsum([0] + [len(p.walls) for p in parts])
    return cl, sp, wl


@pytest.mark.parametrize("prec", [scenes.PREC_FP64, scenes.PREC_FP32])
def test_merged_run_equals_each_scene_alone(dem, prec):
    """Deterministic reduction and captured graphs, 25 steps with a rebuild
    every 10: every scene's state, pair list, wall list and tangential
    histories in the merged context are bit-identical to that scene's own run
    (ids shifted by the scenes before it)."""
    margin, K, nsteps = 2e-4, 10, 25
    parts = _parts(prec, margin)
    first, rest = scenes.merge_batch(parts)
    assert len(set(len(p.E) for p in parts)) == 1 and len(first.E) == 3 * len(parts)
    with dem.Simulation(first, margin=margin, rebuild_interval=K, precision=prec,
                        extra_scenes=rest) as sim:
        sim.set_deterministic(True)
        sim.set_graphs(True)
        sim.step(nsteps)
        merged = sim.state()
        ma, mb, mu_, mws, mww, muw = sim.contacts()
        assert sim.stats()["steps"] == nsteps
    cl, sp, wl = _offsets(parts)
    total_pairs = 0
    for k, p in enumerate(parts):
        with dem.Simulation(p, margin=margin, rebuild_interval=K, precision=prec) as one:
            one.set_deterministic(True)
            one.set_graphs(True)
            one.step(nsteps)
            alone = one.state()
            a, b, u, ws, ww, uw = one.contacts()
        for x, y in zip(merged, alone):
            assert np.array_equal(x[cl[k]:cl[k + 1]], y)
        sel = (ma >= sp[k]) & (ma < sp[k + 1])
        assert np.all((mb[sel] >= sp[k]) & (mb[sel] < sp[k + 1]))  # no pair across scenes
        assert np.array_equal(ma[sel] - sp[k], a) and np.array_equal(mb[sel] - sp[k], b)
        assert np.array_equal(mu_[sel], u)
        selw = (mws >= sp[k]) & (mws < sp[k + 1])
        assert np.all((mww[selw] >= wl[k]) & (mww[selw] < wl[k + 1]))  # own walls only
        assert np.array_equal(mws[selw] - sp[k], ws) and np.array_equal(mww[selw] - wl[k], ww)
        assert np.array_equal(muw[selw], uw)
        assert len(a) > p.n_clumps and np.abs(u).max() > 0
        total_pairs += len(a)
    assert total_pairs == len(ma)


def test_merged_fp64_forces_match_the_oracle_per_scene(dem, oracle_mod):
    """One force evaluation of the merged FP64 context: each scene's clump
    forces and torques against the oracle run on that scene alone, within
    1e-12 of the sum of the contribution magnitudes."""
    margin, K = 1e-4, 10
    parts = _parts(scenes.PREC_FP64, margin)
    first, rest = scenes.merge_batch(parts)
    with dem.Simulation(first, margin=margin, rebuild_interval=K, extra_scenes=rest) as sim:
        F, T = sim.eval_forces()
    cl, _, _ = _offsets(parts)
    for k, p in enumerate(parts):
        om = oracle_mod.OracleModel(p)
        xs, owner, tsph = om.sphere_centres(p.tpl, p.pos, p.quat)
        qc, rho = om.detect_coords(xs, tsph, margin)
        a, b = om.pairs_binned(owner, qc, rho)
        ws, ww = om.wall_candidates(xs, tsph, margin, 0.0, p.h * K)
        Fo, To, _, _, _, _, mag = om.forces(p.tpl, p.pos, p.quat, p.vel, p.angvel, 0.0, a, b,
                                            np.zeros((len(a), 3)), ws, ww, np.zeros((len(ws), 3)),
                                            with_mag=True)
        Fk, Tk = F[cl[k]:cl[k + 1]], T[cl[k]:cl[k + 1]]
        touched = mag[:, 0] > 0
        assert touched.sum() > 0.3 * p.n_clumps
        errF = (np.abs(Fk - Fo).max(axis=1)[touched] / mag[touched, 0]).max()
        errT = (np.abs(Tk - To).max(axis=1)[touched] / mag[touched, 1]).max()
        assert errF <= 1e-12 and errT <= 1e-12, (k, errF, errT)
        assert np.all(Fk[~touched] == 0) and np.all(Tk[~touched] == 0)
