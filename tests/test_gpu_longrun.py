"""Long runs against the oracle, checked statistically.

Over thousands of steps two simulations of the same bed separate at the
particle level whatever their precision (the dynamics are chaotic), so a
long run is compared through a bulk property of its end state: the settled
packing fraction (solid volume fraction of the bed's interior).  One run's
value scatters around the ensemble mean: three oracle runs from states
1e-12 m apart settled within 0.18 % of each other, GPU runs from states
2^-40 m apart scatter by a standard deviation of about 0.05 % (FP64) and
0.1-0.2 % (FP32_VOXEL, whose rounding acts as extra noise).  So the mean of
six GPU realizations is compared with the oracle's bed: within 0.5 % in
FP64.  FP32_VOXEL's ensemble mean itself sits off the FP64 one by an amount
that depends on the friction coefficient (measured on this bed: -0.27 % at
mu = 0, +0.3 to +0.5 % at mu = 0.5, -0.32 % at mu = 1), so its bound is 1 %.
(A 400-clump bed spread over 2 %; this one has 1,600 clumps.)"""
import dataclasses

import numpy as np
import pytest

from paper_2307_03445_gb300 import scenes
from tests.helpers import settling_box_scene

pytestmark = pytest.mark.gpu

K = 20
SIDE = 0.06  # box footprint SIDE x SIDE
N_CLUMPS = 1600
E, H = 1e6, 3e-5  # a soft material resolved by 30 us steps
N_STEPS = 10_000  # 0.3 s: fall, rebound, rest
N_REAL = 6  # GPU realizations per precision


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
    side = SIDE
    top = float(np.percentile(xs[:, 2] + r, 90))
    rng = np.random.default_rng(seed)
    pts = np.column_stack([rng.uniform(2 * rmax, side - 2 * rmax, n_points),
                           rng.uniform(2 * rmax, side - 2 * rmax, n_points),
                           rng.uniform(2 * rmax, top - 3 * rmax, n_points)])
    inside = np.zeros(n_points, bool)
    for i, nb in enumerate(cKDTree(xs).query_ball_point(pts, rmax)):
        if nb:
            inside[i] = np.any(np.linalg.norm(xs[nb] - pts[i], axis=1) <= r[nb])
    return float(inside.mean())


@pytest.fixture(scope="module")
def settled(oracle_mod):
    sc = settling_box_scene(n=N_CLUMPS, side=SIDE, E=E, h=H)
    margin = 2.0 * 1.0 * sc.h * K  # speed bound 1 m/s, twice over
    sc.bin_size = scenes.default_bin_size(sc, margin)
    osim = oracle_mod.OracleSim(sc, margin, K)
    osim.step(N_STEPS)
    po, qo, vo, _ = osim.state()
    return sc, margin, packing_fraction(oracle_mod, sc, po, qo)


@pytest.mark.parametrize("prec", [scenes.PREC_FP64, scenes.PREC_FP32])
def test_settled_packing_fraction_matches_the_oracle(dem, oracle_mod, settled, prec):
    sc, margin, phi_o = settled
    assert 0.5 < phi_o < 0.7  # a settled random packing of the clumps
    phis = []
    for k in range(N_REAL):
        s2 = dataclasses.replace(sc, pos=sc.pos.copy())
        s2.pos[17, 1] += k * 2.0 ** -40  # on the FP32 offset grid
        with dem.Simulation(s2, margin=margin, rebuild_interval=K, precision=prec) as sim:
            sim.step(N_STEPS)
            assert sim.audit() == 0
            st = sim.stats()
            pos, quat, vel, _ = sim.state()
        assert st["guard_violations"] == 0
        assert np.all(np.isfinite(pos)) and np.abs(vel).max() < 0.5
        # the bed came down from its start
        assert pos[:, 2].max() < sc.pos[:, 2].max()
        phis.append(packing_fraction(oracle_mod, s2, pos, quat))
    phi = float(np.mean(phis))
    tol = 0.005 if prec == scenes.PREC_FP64 else 0.01
    assert abs(phi - phi_o) <= tol * phi_o, (phis, phi_o)
