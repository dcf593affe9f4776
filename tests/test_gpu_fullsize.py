"""Parity at the benchmark's full size: 11,000,000 clumps (about 34 million
spheres) of the paper-scale workload's templates and materials, FP32_VOXEL,
margin 2e-5 m, the launch configuration the benchmark times.  The oracle cannot
run the whole bed, so it checks sampled clumps one by one: for each, the
oracle takes the clump and every clump that can reach it, and computes

  * the bin registrations of the clump's spheres (bit-exact),
  * the listed sphere-sphere pairs and sphere-wall candidates that involve
    the clump's spheres (bit-exact),
  * the clump's total force and torque for a fresh list (1e-5 relative to
    the sum of the magnitudes of its contributions).

The state is generated (a lattice squeezed below the bounding diameter with
random velocities); it never comes from the GPU."""
import numpy as np
import pytest

from paper_2307_03445_gb300 import scenes

pytestmark = pytest.mark.gpu

N_CLUMPS = 11_000_000
MARGIN, K = 2e-5, 20
N_SAMPLES = 120
TOL = 1e-5


@pytest.fixture(scope="module")
def dem():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2307_03445_gb300 as dem

    dem.load_library()
    return dem


def _bed():
    sc = scenes.config5(n_clumps=N_CLUMPS)
    # templates exactly representable in float (the FP32_VOXEL layout)
    sc.tpl_pos = sc.tpl_pos.astype(np.float32).astype(np.float64)
    sc.tpl_rad = sc.tpl_rad.astype(np.float32).astype(np.float64)
    rng = np.random.default_rng(4321)
    bound = sc.bounding_radius()[sc.tpl]
    spacing = 0.9 * 2.0 * float(bound.mean())
    P = scenes.lattice_positions(N_CLUMPS, spacing, 0.0, 4.0, 0.0, 2.0, 0.0, rng, 0.1 * spacing)
    P[:, 2] += float(bound.max())
    sc.pos = P
    sc.quat = scenes.random_quaternions(rng, N_CLUMPS)
    sc.vel = rng.normal(scale=0.05, size=(N_CLUMPS, 3))
    sc.angvel = rng.normal(scale=20.0, size=(N_CLUMPS, 3))
    top = float(P[:, 2].max() + bound.max())
    sc.walls = scenes.box_walls(0.0, 4.0, 0.0, 2.0, 0.0, top=top, top_vel=(0.2, 0.0, 0.0))
    sc.hi = (4.0, 2.0, top + 0.01)
    scenes.snap_to_voxel_grid(sc)
    sc.bin_size = scenes.default_bin_size(sc, MARGIN)
    return sc


@pytest.fixture(scope="module")
def run(dem):
    sc = _bed()
    with dem.Simulation(sc, margin=MARGIN, rebuild_interval=K,
                        precision=dem.DEM_FP32_VOXEL) as sim:
        F, T = sim.eval_forces()
        keys, ids = sim.bins()
        a, b, _, ws, ww, _ = sim.contacts()
        Fw = sim.wall_forces()
        st = sim.stats()
    return sc, F, T, keys, ids, a, b, ws, ww, st, Fw


def _samples(sc):
    rng = np.random.default_rng(99)
    z = sc.pos[:, 2]
    low = np.flatnonzero(z < z.min() + 0.004)   # on the floor
    top = np.flatnonzero(z > z.max() - 0.004)   # under the plate
    side = np.flatnonzero(sc.pos[:, 0] < 0.006)  # at a side wall
    pick = [rng.choice(low, 15, replace=False), rng.choice(top, 15, replace=False),
            rng.choice(side, 15, replace=False),
            rng.choice(len(sc.tpl), N_SAMPLES - 45, replace=False)]
    return np.unique(np.concatenate(pick))


def test_full_size_matches_the_oracle_on_sampled_clumps(run, oracle_mod):
    from scipy.spatial import cKDTree

    sc, F, T, keys, ids, a, b, ws, ww, st, _ = run
    assert st["n_spheres"] == sc.n_spheres and st["n_pairs"] == len(a) > sc.n_spheres // 2
    counts = sc.sphere_counts()[sc.tpl]
    csph = np.concatenate([[0], np.cumsum(counts)])
    bound = sc.bounding_radius()
    tree = cKDTree(sc.pos)
    sample = _samples(sc)
    # GPU lists restricted to the sampled spheres, by global sphere id
    hit = np.zeros(sc.n_spheres, bool)
    for c in sample:
        hit[csph[c]:csph[c + 1]] = True
    sel = hit[a] | hit[b]
    gpu_pairs = set(zip(a[sel].tolist(), b[sel].tolist()))
    wsel = hit[ws]
    gpu_walls = set(zip(ws[wsel].tolist(), ww[wsel].tolist()))
    bsel = hit[ids]
    gpu_bins = set(zip(keys[bsel].tolist(), ids[bsel].tolist()))
    want_pairs, want_walls, want_bins = set(), set(), set()
    worst = 0.0
    for c in sample:
        # listed gaps are at most 2 m plus two lattice units (2^-24 m each)
        reach = bound[sc.tpl[c]] + bound.max() + 2.0 * MARGIN + 1e-6
        nb = [int(c)] + sorted(set(tree.query_ball_point(sc.pos[c], reach)) - {int(c)})
        sub = scenes.Scene(**{**sc.__dict__, "tpl": sc.tpl[nb], "pos": sc.pos[nb],
                              "quat": sc.quat[nb], "vel": sc.vel[nb], "angvel": sc.angvel[nb]})
        om = oracle_mod.OracleModel(sub)
        xs, owner, tsph = om.sphere_centres(sub.tpl, sub.pos, sub.quat)
        gid = np.concatenate([np.arange(csph[k], csph[k + 1]) for k in nb])
        n0 = int(counts[c])  # the sampled clump's spheres come first
        qc, rho = om.detect_coords(xs, tsph, MARGIN)
        k_o, i_o = om.bin_entries(qc[:n0], rho[:n0])
        want_bins |= set(zip(k_o.tolist(), gid[i_o].tolist()))
        pa, pb = om.pairs_brute(owner, qc, rho)
        mine = (pa < n0) | (pb < n0)
        ga, gb = gid[pa[mine]], gid[pb[mine]]  # a < b in global ids, as listed
        want_pairs |= set(zip(np.minimum(ga, gb).tolist(), np.maximum(ga, gb).tolist()))
        s_o, w_o = om.wall_candidates(xs, tsph, MARGIN, 0.0, sub.h * K)
        wm = s_o < n0
        want_walls |= set(zip(gid[s_o[wm]].tolist(), w_o[wm].tolist()))
        Fo, To, _, _, _, _, mag = om.forces(sub.tpl, sub.pos, sub.quat, sub.vel, sub.angvel, 0.0,
                                            pa, pb, np.zeros((len(pa), 3)), s_o, w_o,
                                            np.zeros((len(s_o), 3)), with_mag=True)
        if mag[0, 0] > 0:
            eF = np.abs(F[c] - Fo[0]).max() / mag[0, 0]
            eT = np.abs(T[c] - To[0]).max() / mag[0, 1]
            worst = max(worst, eF, eT)
        else:
            assert np.all(F[c] == 0) and np.all(T[c] == 0)
    assert gpu_bins == want_bins
    assert gpu_pairs == want_pairs and len(want_pairs) > len(sample)
    assert gpu_walls == want_walls and len(want_walls) > 0
    assert worst <= TOL, worst


def test_full_size_totals_balance(run):
    """Action and reaction at full size: every pair force enters two clumps
    with opposite signs, so the clump forces sum to minus the forces on the
    walls (float accumulators; relative to the sum of the magnitudes)."""
    sc, F, T, keys, ids, a, b, ws, ww, st, Fw = run
    assert st["active_last"] > 0 and len(ws) > 0
    assert np.all(np.isfinite(F)) and np.all(np.isfinite(T))
    scale = np.abs(F).sum()
    assert scale > 0
    assert np.abs(F.sum(axis=0) + Fw.sum(axis=0)).max() <= 1e-5 * scale
