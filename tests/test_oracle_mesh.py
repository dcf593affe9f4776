"""Oracle pins for mesh facets (sphere-triangle contacts, the boundaries the
paper builds from meshes in section 4): in front of the facet's plane the
distance is the distance to the closed triangle, checked against brute
force over a dense sampling of the facet; in the facet's face region it is
exactly the plane wall's; beyond a vertex it is the distance to that vertex.
A facet is one-sided (reading B1): a centre behind its plane is at infinite
distance, so a sphere that reaches a facet from behind passes through it."""
import math
import numpy as np
import pytest

from paper_2307_03445_gb300 import scenes
from tests.helpers import set_clumps, single_sphere_scene

A, B, Cv = np.array([0.01, -0.004, 0.002]), np.array([0.026, 0.001, -0.003]), np.array([0.004, 0.018, 0.006])


def _model(oracle_mod, walls):
    return oracle_mod.OracleModel(single_sphere_scene([1e-3], walls=walls))


def _dense_facet(a, b, c, N=600):
    i, j = np.meshgrid(np.arange(N + 1), np.arange(N + 1), indexing="ij")
    keep = (i + j) <= N
    u, v = i[keep] / N, j[keep] / N
    return a + u[:, None] * (b - a) + v[:, None] * (c - a)


def _barycentric(a, b, c, x):
    e1, e2, d = b - a, c - a, x - a
    M = np.array([[e1 @ e1, e1 @ e2], [e1 @ e2, e2 @ e2]])
    return np.linalg.solve(M, [d @ e1, d @ e2])


def test_facet_distance_is_the_distance_to_the_closed_triangle(oracle_mod):
    tri = scenes.triangle(A, B, Cv)
    om = _model(oracle_mod, [tri])
    n = np.asarray(tri["n"])
    pts = _dense_facet(A, B, Cv)
    rng = np.random.default_rng(5)
    centre = (A + B + Cv) / 3
    regions = set()
    behind = 0
    for _ in range(150):
        x = centre + rng.uniform(-0.02, 0.02, 3) + rng.choice([-1, 1]) * rng.uniform(5e-4, 4e-3) * n
        d, nw = om.wall_distance(0, 0.0, x)
        if (x - A) @ n < 0:  # behind the plane: no contact, whatever the distance
            assert d == math.inf and np.array_equal(nw, n)
            behind += 1
            continue
        brute = np.sqrt(((pts - x) ** 2).sum(axis=1)).min()
        assert abs(abs(d) - brute) <= 2e-7, (x, d, brute)
        # the closest point x - |d| nw (face region: x - d n) lies on the facet
        cp = x - d * nw
        u, v = _barycentric(A, B, Cv, cp)
        assert u >= -1e-9 and v >= -1e-9 and u + v <= 1 + 1e-9
        assert abs(np.linalg.norm(nw) - 1.0) < 1e-12
        inside = np.allclose(nw, n, rtol=0, atol=0)
        regions.add(inside)
        assert d >= 0
        if inside:
            assert np.isclose(d, (x - A) @ n, rtol=0, atol=1e-17)
    assert regions == {True, False} and 40 < behind < 110


def test_facet_in_its_face_region_is_the_plane_wall_bit_for_bit(oracle_mod):
    """Same point p and normal: a sphere that stays over the facet's interior
    sees exactly the plane's distance, list and forces, through a whole
    trajectory (sliding and rolling under gravity)."""
    a, b, c = np.array([-0.04, -0.04, 0.0]), np.array([0.05, -0.03, 0.0]), np.array([-0.03, 0.05, 0.0])
    runs = []
    for wall in (scenes.triangle(a, b, c), scenes.plane(a, (0, 0, 1))):
        sc = single_sphere_scene([1e-3], g=(0.3, 0.0, -9.81), walls=[wall], mu=0.4, cor=0.6)
        # resting at about its static overlap, sliding along x
        set_clumps(sc, [0], [[0.0, 0.0, 1e-3 - 1.2e-7]], vel=[[0.05, 0.0, 0.0]])
        sim = oracle_mod.OracleSim(sc, margin=5e-5, rebuild_every=10)
        sim.step(3000)
        runs.append((sim.state(), sim.contacts()))
    (s1, c1), (s2, c2) = runs
    for x, y in zip(s1, s2):
        assert np.array_equal(x, y)
    assert np.array_equal(c1[3], c2[3]) and np.array_equal(c1[5], c2[5])
    assert len(c1[3]) == 1 and np.abs(c1[5]).max() > 0  # it touched and slid


def test_facet_vertex_and_edge_closed_forms(oracle_mod):
    tri = scenes.triangle(A, B, Cv)
    om = _model(oracle_mod, [tri])
    n = np.asarray(tri["n"])
    # beyond vertex B, away from both of its edges
    out = (B - A) / np.linalg.norm(B - A) + (B - Cv) / np.linalg.norm(B - Cv)
    x = B + 0.003 * out / np.linalg.norm(out) + 0.001 * n
    d, nw = om.wall_distance(0, 0.0, x)
    assert np.isclose(d, np.linalg.norm(x - B), rtol=1e-14)
    assert np.allclose(nw, (x - B) / np.linalg.norm(x - B), atol=1e-13)
    # off the middle of edge A-C, in the facet's plane, outwards
    e = Cv - A
    mid = A + 0.5 * e
    perp = np.cross(n, e)
    perp = perp / np.linalg.norm(perp)
    if perp @ (B - A) > 0:
        perp = -perp
    x = mid + 0.002 * perp + 0.0005 * n  # in front of the plane
    d, nw = om.wall_distance(0, 0.0, x)
    assert np.isclose(d, np.hypot(0.002, 0.0005), rtol=1e-13)
    # the same point mirrored behind the plane touches nothing
    d, nw = om.wall_distance(0, 0.0, x - 0.001 * n)
    assert d == math.inf


def test_moving_facet_is_the_translated_facet(oracle_mod):
    vel = np.array([0.01, -0.02, 0.03])
    t = 0.25
    om_m = _model(oracle_mod, [scenes.triangle(A, B, Cv, vel=tuple(vel))])
    om_s = _model(oracle_mod, [scenes.triangle(A + vel * t, B + vel * t, Cv + vel * t)])
    rng = np.random.default_rng(9)
    for _ in range(40):
        x = (A + B + Cv) / 3 + vel * t + rng.uniform(-0.02, 0.02, 3)
        d1, n1 = om_m.wall_distance(0, t, x)
        d2, n2 = om_s.wall_distance(0, 0.0, x)
        assert (d1 == d2 == math.inf or abs(d1 - d2) <= 1e-15) and np.allclose(n1, n2, atol=1e-12)


def test_mesh_helpers_orient_every_facet_towards_the_grains():
    box = scenes.box_mesh(-0.01, 0.02, -0.015, 0.01, 0.0, 0.03)
    assert len(box) == 12
    centre = np.array([0.005, -0.0025, 0.015])
    for f in box:
        a, b, c, n = (np.asarray(f[k]) for k in ("p", "b", "c", "n"))
        assert abs(np.linalg.norm(n) - 1) < 1e-15
        assert abs(n @ (b - a)) < 1e-15 and abs(n @ (c - a)) < 1e-15
        assert n @ (centre - a) > 0
    # the 12 facets tile the six faces: total area = box surface
    area = sum(0.5 * np.linalg.norm(np.cross(np.subtract(f["b"], f["p"]), np.subtract(f["c"], f["p"])))
               for f in box)
    assert np.isclose(area, 2 * (0.03 * 0.025 + 0.03 * 0.03 + 0.025 * 0.03), rtol=1e-13)
    fun = scenes.funnel_mesh(0.0, 0.0, 0.0, 0.02, 0.005, 0.015, 8)
    assert len(fun) == 16
    for f in fun:
        a, n = np.asarray(f["p"]), np.asarray(f["n"])
        assert n[0] * -a[0] + n[1] * -a[1] > 0  # towards the axis


def test_facet_box_is_the_workload_box():
    """The benchmark's box and sliding plate as facets: the same six planes
    (every facet lies in one of them, normal equal), 2 facets each, and only
    the top facets carry the plate's velocity."""
    from paper_2307_03445_gb300 import workloads

    planes = scenes.config5(n_clumps=1).walls
    facets = workloads.facet_box(planes)
    assert len(facets) == 12
    for pl in planes:
        n, p = np.asarray(pl["n"]), np.asarray(pl["p"])
        mine = [f for f in facets if np.allclose(f["n"], n, atol=1e-15)]
        assert len(mine) == 2
        for f in mine:
            for k in ("p", "b", "c"):
                assert abs((np.asarray(f[k]) - p) @ n) < 1e-15
            assert tuple(f["vel"]) == tuple(pl["vel"])


def test_facet_is_one_sided(oracle_mod):
    """A sphere thrown at a facet from its front rebounds exactly as from the
    plane wall.  A sphere whose centre lies 0.5 mm behind the facet, gliding
    along it, does not touch it: free flight, where the plane wall (which
    has no back side) pushes it out with an overlap of r + 0.5 mm."""
    a, b, c = np.array([-0.04, -0.04, 0.0]), np.array([0.05, -0.03, 0.0]), np.array([-0.03, 0.05, 0.0])
    out = {}
    for case, z0, v0 in (("front", 1.2e-3, (0.0, 0.0, -0.5)), ("behind", -0.5e-3, (0.05, 0.0, 0.0))):
        for wall in (scenes.triangle(a, b, c), scenes.plane(a, (0, 0, 1))):
            sc = single_sphere_scene([1e-3], walls=[wall], mu=0.3, cor=0.5)
            sc.bin_size = 4e-3
            set_clumps(sc, [0], [[0.0, 0.0, z0]], vel=[v0])
            sim = oracle_mod.OracleSim(sc, margin=5e-5, rebuild_every=10)
            sim.step(12000)
            out[(case, wall["type"])] = (sim.state(), sim.contacts())
    for x, y in zip(out[("front", scenes.WALL_TRIANGLE)][0], out[("front", scenes.WALL_PLANE)][0]):
        assert np.array_equal(x, y)
    assert out[("front", scenes.WALL_TRIANGLE)][0][2][0, 2] > 0  # bounced back up
    (pos, quat, vel, angvel), lists = out[("behind", scenes.WALL_TRIANGLE)]
    assert np.array_equal(vel[0], [0.05, 0.0, 0.0]) and len(lists[3]) == 0
    assert pos[0, 0] == pytest.approx(0.05 * 12000 * 1e-6, rel=1e-12) and pos[0, 2] == -0.5e-3
    assert out[("behind", scenes.WALL_PLANE)][0][2][0, 2] > 1.0  # the plane throws it out
