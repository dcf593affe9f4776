"""Host logic of the sample-preparation compressor (no GPU): the loop that
drives a plate through the co-simulation hook, checked against a stand-in
simulation whose plate load grows once the plate has travelled a set
distance.  The library calls it makes are the ones the GPU test exercises."""
import numpy as np

from paper_2307_03445_gb300 import scenes, workloads


class FakeSim:
    """Time advances by h per step; the plate's load is stiffness x travel
    past `contact` once the plate has moved that far along its normal."""

    def __init__(self, h, t0, contact, stiffness, plate):
        self.h, self.t, self.contact, self.k, self.plate = h, t0, contact, stiffness, plate
        self.motions = []  # (time, point, vel) of every set_wall_motion call
        self.p = None
        self.v = None

    def stats(self):
        return {"time": self.t}

    def set_wall_motion(self, wall, point, vel):
        assert wall == self.plate
        self.motions.append((self.t, np.asarray(point, float).copy(), np.asarray(vel, float).copy()))
        self.p, self.v, self.t_set = np.asarray(point, float), np.asarray(vel, float), self.t

    def step(self, n):
        self.t += n * self.h

    def wall_loads(self):
        pos = self.p + self.v * (self.t - self.t_set)
        travel = float(np.dot(pos - self.motions[0][1], self.n))
        F = np.zeros((self.plate + 1, 3))
        F[self.plate] = -self.n * self.k * max(0.0, travel - self.contact)  # grains push back
        return F, np.zeros_like(F)


def test_compressor_drives_the_plate_until_the_load_then_holds_it():
    plate_wall = scenes.plane((0.1, 0.2, 0.3), (0, 0, -2), vel=(0.0, 0.0, 0.0))
    sim = FakeSim(h=1e-6, t0=5e-4, contact=3e-6, stiffness=1e5, plate=3)
    sim.n = np.array([0.0, 0.0, -1.0])
    steps, push, p = workloads.compress(sim, plate_wall, 3, speed=0.5, load=0.2, max_steps=1000,
                                        chunk=4)
    # travel to first contact 3 um, then 2 um more for 0.2 N at 1e5 N/m: 5 um at
    # 0.5 um per step, checked every 4 steps -> stops at the first multiple of 4 >= 10
    assert steps == 12 and push >= 0.2
    assert np.allclose(p, [0.1, 0.2, 0.3 - 0.5 * steps * 1e-6], rtol=0, atol=1e-15)
    (t0, p0, v0), (t1, p1, v1) = sim.motions
    assert t0 == 5e-4 and np.allclose(p0, [0.1, 0.2, 0.3]) and np.allclose(v0, [0, 0, -0.5])
    assert np.allclose(p1, p) and np.all(v1 == 0)  # held where it stopped


def test_compressor_stops_at_the_step_budget():
    plate_wall = scenes.plane((0.0, 0.0, 1.0), (0, 0, -1), vel=(0.0, 0.0, 0.1))
    sim = FakeSim(h=1e-5, t0=0.0, contact=1.0, stiffness=1.0, plate=0)  # never reached
    sim.n = np.array([0.0, 0.0, -1.0])
    steps, push, p = workloads.compress(sim, plate_wall, 0, speed=0.2, load=1.0, max_steps=25,
                                        chunk=10)
    assert steps == 25 and push == 0.0
    assert np.allclose(p, [0.0, 0.0, 1.0 - 0.2 * 25 * 1e-5], atol=1e-15)


def test_merge_batch_shifts_template_material_and_wall_ids():
    """One context of several scenes: through the merged tables every clump
    keeps its own templates (spheres, radii, masses) and every sphere and wall
    its own material values."""
    parts = [scenes.packed_scene(s, n) for s, n in ((31, 40), (32, 70), (33, 25))]
    first, rest = scenes.merge_batch(parts)
    for q, p in zip([first] + rest, parts):
        for t_new, t_old in zip(q.tpl, p.tpl):
            a, b = q.tpl_off[t_new], q.tpl_off[t_new + 1]
            c, d = p.tpl_off[t_old], p.tpl_off[t_old + 1]
            assert np.array_equal(q.tpl_pos[a:b], p.tpl_pos[c:d])
            assert np.array_equal(q.tpl_rad[a:b], p.tpl_rad[c:d])
            assert q.tpl_mass[t_new] == p.tpl_mass[t_old]
            for name in ("E", "nu", "mu", "cor"):
                assert np.array_equal(getattr(q, name)[q.tpl_mat[a:b]], getattr(p, name)[p.tpl_mat[c:d]])
        assert len(q.walls) == len(p.walls) > 0
        for wq, wp in zip(q.walls, p.walls):
            for name in ("E", "nu", "mu", "cor"):
                assert getattr(q, name)[wq["material"]] == getattr(p, name)[wp.get("material", 0)]


def test_repose_angle_of_synthetic_cones():
    """The heap measurement on spheres filling cones of known flank angle
    (20 and 32 degrees, 3 cm high): within half a degree, apex height within
    a sphere radius."""
    import math

    rng = np.random.default_rng(0)
    for ang in (20.0, 32.0):
        H = 0.03
        R = H / math.tan(math.radians(ang))
        pts = rng.uniform([-R, -R, 0.0], [R, R, H], size=(200000, 3))
        rho = np.hypot(pts[:, 0], pts[:, 1])
        pts = pts[pts[:, 2] <= H - math.tan(math.radians(ang)) * rho]
        got, hmax, rings = workloads.repose_angle(pts, np.full(len(pts), 1e-3), (0.0, 0.0), 0.0, 2e-3)
        assert abs(got - ang) < 0.5 and abs(hmax - (H + 1e-3)) < 1e-3 and rings >= 5
        # grains scattered on the floor beyond the toe do not move the flank
        far = np.column_stack([rng.uniform(R + 0.01, R + 0.1, 30) * np.cos(np.arange(30)),
                               rng.uniform(R + 0.01, R + 0.1, 30) * np.sin(np.arange(30)),
                               np.full(30, 1e-3)])
        got2, _, _ = workloads.repose_angle(np.vstack([pts, far]), np.full(len(pts) + 30, 1e-3),
                                            (0.0, 0.0), 0.0, 2e-3)
        assert got2 == got
