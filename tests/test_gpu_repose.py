"""Angle of repose (section 4: grains flowing out of a container onto a
plate pile into a heap whose flank angle is measured), on the GPU path:
3,000 clumps of three overlapping spheres settle in a tube of 64 facets
(radius 5 cm) standing on the floor, the tube is lifted at 5 cm/s and the
column slumps into a heap; its angle, measured by workloads.repose_angle
(pinned on synthetic cones in tests/test_host_workloads.py), grows with the
friction coefficient and lies in the range granular heaps take.

Measured with this set-up (two seeds each): mu 0.1 gives 2.5-3.8 degrees,
mu 0.5 20-22, mu 0.9 21-24 (3,000 and 6,000 clumps alike); a fast lift
(20 cm/s) or a small column (750-1,500 clumps) gives flatter heaps whose
angle scatters by several degrees from run to run."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dem():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2307_03445_gb300 as dem

    dem.load_library()
    return dem


def _heap_angle(dem, mu, n=3000, radius=0.05, height=0.10, lift=0.05, t_settle=0.3, t_rest=0.4):
    from paper_2307_03445_gb300 import workloads

    sc, tube = workloads.repose_column_scene(n, mu, radius=radius, height=height)
    K = 20
    # a speed bound of 2 m/s at the spheres (translation plus rotation; the
    # heap's grains stay below 0.3 m/s), rebuilt every 20 steps
    margin = 2.0 * sc.h * K
    t_lift = 1.2 * height / lift
    with dem.Simulation(sc, margin=margin, rebuild_interval=K) as sim:
        sim.set_graphs(True)
        sim.step(int(round(t_settle / sc.h)))
        workloads.lift_walls(sim, sc, tube, (0.0, 0.0, lift))
        sim.step(int(round((t_lift + t_rest) / sc.h)))
        pos, quat, vel, angvel = sim.state()
        st = sim.stats()
        missed = sim.audit()
    xs, radii, owner = workloads.sphere_centres(sc, pos, quat)
    ang, hmax, rings = workloads.repose_angle(xs, radii, (0.0, 0.0), 0.0, 4e-3)
    spread = float(np.percentile(np.hypot(pos[:, 0], pos[:, 1]), 90))
    return ang, hmax, st, missed, spread


def test_repose_angle_grows_with_friction(dem):
    low = _heap_angle(dem, 0.1)
    high = _heap_angle(dem, 0.5)
    info = [(round(r[0], 2), round(r[1], 4), round(r[4], 4), r[2]["guard_violations"], r[3])
            for r in (low, high)]  # angle, apex height, 90 % radius, guard, missed
    print("repose (angle, apex, 90 % radius, guard, missed):", info)
    for ang, hmax, st, missed, spread in (low, high):
        assert missed == 0 and st["guard_violations"] == 0, info
    assert low[0] < 8.0, info  # a nearly frictionless heap spreads flat
    assert 12.0 < high[0] < 40.0 and high[1] > 0.015, info
    assert high[0] > low[0] + 10.0, info
    assert high[4] < low[4]  # and the rougher heap spreads less
