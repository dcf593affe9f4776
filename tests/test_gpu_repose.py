"""Angle of repose (section 4: grains flowing out of a container onto a
plate pile into a heap whose flank angle is measured), on the GPU path:
1,500 clumps of three overlapping spheres settle in a tube of 64 facets
standing on the floor, the tube is lifted at 0.2 m/s and the column slumps
into a heap; its angle, measured by workloads.repose_angle (pinned on
synthetic cones in tests/test_host_workloads.py), grows with the friction
coefficient and lies in the range granular heaps take."""
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


def _heap_angle(dem, mu, n=1500, t_settle=0.3, t_lift=0.6, t_rest=0.4):
    from paper_2307_03445_gb300 import workloads

    sc, tube = workloads.repose_column_scene(n, mu)
    K = 4
    # impacts on the soft contacts spin clumps up: a speed bound of 10 m/s
    # at the spheres (translation plus rotation), rebuilt every 4 steps
    margin = 10.0 * sc.h * K
    with dem.Simulation(sc, margin=margin, rebuild_interval=K) as sim:
        sim.set_graphs(True)
        sim.step(int(round(t_settle / sc.h)))
        workloads.lift_walls(sim, sc, tube, (0.0, 0.0, 0.2))
        sim.step(int(round((t_lift + t_rest) / sc.h)))
        pos, quat, vel, angvel = sim.state()
        st = sim.stats()
        missed = sim.audit()
    xs, radii, owner = workloads.sphere_centres(sc, pos, quat)
    ang, hmax, rings = workloads.repose_angle(xs, radii, (0.0, 0.0), 0.0, 4e-3)
    spread = float(np.percentile(np.hypot(pos[:, 0], pos[:, 1]), 90))
    return ang, hmax, st, missed, spread


def test_repose_angle_grows_with_friction(dem):
    low = _heap_angle(dem, 0.3)
    high = _heap_angle(dem, 0.9)
    info = [(round(r[0], 2), round(r[1], 4), round(r[4], 4), r[2]["guard_violations"], r[3])
            for r in (low, high)]  # angle, apex height, 90 % radius, guard, missed
    for ang, hmax, st, missed, spread in (low, high):
        # the exact audit of the final list; the certificate may fail for a
        # few clumps in 10^7 clump-steps (impacts on the soft contacts)
        assert missed == 0 and st["guard_violations"] < 1e-5 * st["steps"] * 1500, info
    assert 5.0 < high[0] < 50.0 and high[1] > 0.01, info
    assert high[0] > low[0] + 3.0, info
