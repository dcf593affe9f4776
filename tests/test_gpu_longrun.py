"""Long runs against the oracle, checked statistically.

Over thousands of steps two simulations of the same bed separate at the
particle level (the dynamics are chaotic), so a long run is compared through
a bulk property of its end state: the settled packing fraction (solid volume
fraction of the bed's interior).  A GPU run in FP64 stays within about 0.02 %
of the oracle's run of the same bed; an FP32_VOXEL run, whose roundings act
as noise, scatters around it by a standard deviation of about 0.5 % per bed
(measured over eight independent beds at mu = 0, 0.5 and 1, the mean
differences were +0.13, -0.07 and -0.14 %, each within 1.2 standard errors
of zero).  Realizations from tiny perturbations of one bed do not average
this scatter out: they keep that bed's own offset.  So twelve independent
beds (own templates and lattice) are each run by the oracle and by the GPU;
the mean relative difference must be within 0.5 % (3.5 standard errors at
0.5 % per bed) for both precisions, and no bed may be off by more than 2 %.
"""
import numpy as np
import pytest

from paper_2307_03445_gb300 import scenes
from tests.helpers import settling_box_scene
from tests.oracle_pool import run_many

pytestmark = pytest.mark.gpu

K = 20
SIDE = 0.06  # box footprint SIDE x SIDE
N_CLUMPS = 1600
E, H = 1e6, 3e-5  # a soft material resolved by 30 us steps
N_STEPS = 10_000  # 0.3 s: fall, rebound, rest
SEEDS = [5 + 10 * k for k in range(12)]  # independent beds (own templates and lattice)


@pytest.fixture(scope="module")
def dem():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2307_03445_gb300 as dem

    dem.load_library()
    return dem


def packing_fraction(oracle_mod, sc, pos, quat, n_points=200_000, seed=0):
    """Solid fraction of the slab from 2 r_max above the floor to 3 r_max
    below the 90th percentile of the sphere tops, 2 r_max inside the side
    walls, by sampling points (fixed seed) and testing each against every
    sphere within reach (a point inside any sphere of any clump is solid)."""
    from scipy.spatial import cKDTree

    xs, _, tsph = oracle_mod.OracleModel(sc).sphere_centres(sc.tpl, pos, quat)
    r = sc.tpl_rad[tsph]
    rmax = float(r.max())
    top = float(np.percentile(xs[:, 2] + r, 90))
    rng = np.random.default_rng(seed)
    pts = np.column_stack([rng.uniform(2 * rmax, SIDE - 2 * rmax, n_points),
                           rng.uniform(2 * rmax, SIDE - 2 * rmax, n_points),
                           rng.uniform(2 * rmax, top - 3 * rmax, n_points)])
    d, idx = cKDTree(xs).query(pts, k=32, distance_upper_bound=rmax)
    assert np.isinf(d[:, -1]).all()  # every sphere centre within reach was returned
    found = idx < len(xs)
    rr = np.where(found, r[np.minimum(idx, len(xs) - 1)], -1.0)
    return float(np.any(d <= rr, axis=1).mean())


def _bed(seed):
    sc = settling_box_scene(n=N_CLUMPS, side=SIDE, E=E, h=H, seed=seed)
    margin = 2.0 * 1.0 * sc.h * K  # speed bound 1 m/s, twice over
    sc.bin_size = scenes.default_bin_size(sc, margin)
    return sc, margin


@pytest.fixture(scope="module")
def settled(oracle_mod):
    """The oracle's settled packing fraction of every bed (runs in parallel)."""
    beds = [_bed(s) for s in SEEDS]
    ends = run_many([(sc, margin, K, N_STEPS) for sc, margin in beds])
    return [(sc, margin, packing_fraction(oracle_mod, sc, po, qo))
            for (sc, margin), (po, qo, _, _) in zip(beds, ends)]


@pytest.mark.parametrize("prec", [scenes.PREC_FP64, scenes.PREC_FP32])
def test_settled_packing_fraction_matches_the_oracle(dem, oracle_mod, settled, prec):
    rel = []
    for sc, margin, phi_o in settled:
        assert 0.5 < phi_o < 0.7  # a settled random packing of the clumps
        with dem.Simulation(sc, margin=margin, rebuild_interval=K, precision=prec) as sim:
            sim.step(N_STEPS)
            assert sim.audit() == 0
            st = sim.stats()
            pos, quat, vel, _ = sim.state()
        assert st["guard_violations"] == 0
        assert np.all(np.isfinite(pos)) and np.abs(vel).max() < 0.5
        # the bed came down from its start
        assert pos[:, 2].max() < sc.pos[:, 2].max()
        rel.append(packing_fraction(oracle_mod, sc, pos, quat) / phi_o - 1.0)
    rel = np.array(rel)
    print(f"packing fraction prec={prec}: mean {100 * rel.mean():+.3f} %, sd "
          f"{100 * rel.std(ddof=1):.3f} %, beds {np.round(100 * rel, 3).tolist()}")
    assert abs(rel.mean()) <= 0.005, rel
    assert np.abs(rel).max() <= 0.02, rel
