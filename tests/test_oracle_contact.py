"""Pins of the oracle's contact law (section 2.1, Eq. (1)-(4)) and its use in
whole simulations, against closed forms, invariants and textbook mechanics."""
import json
import math
import os

import numpy as np
import pytest
from scipy.integrate import quad

from paper_2307_03445_gb300 import scenes
from tests.helpers import set_clumps, single_sphere_scene, sphere_mass, triangle_clump_scene

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _estar(E, nu):
    return 1.0 / (2.0 * (1.0 - nu * nu) / E)


def collide(oracle_mod, r=1e-3, v0=0.5, E=1e8, nu=0.3, cor=1.0, mu=0.0, h=2e-7, nsteps=3000):
    """Head-on collision of two equal single spheres; returns overlap history and
    the final relative velocity."""
    sc = single_sphere_scene([r, r], E=E, nu=nu, mu=mu, cor=cor, h=h)
    sc.bin_size = 4 * r
    gap = 2e-6
    set_clumps(sc, [0, 1], [[-r - gap, 0, 0], [r + gap, 0, 0]],
               vel=[[0.5 * v0, 0, 0], [-0.5 * v0, 0, 0]])
    sim = oracle_mod.OracleSim(sc, margin=5e-5, rebuild_every=20)
    overl = []
    for _ in range(nsteps):
        sim.step(1)
        pos, quat, vel, angvel = sim.state()
        overl.append(2 * r - (pos[1, 0] - pos[0, 0]))
        if overl[-1] < -4 * gap and len(overl) > 10 and max(overl) > 0:
            break
    pos, quat, vel, angvel = sim.state()
    return np.array(overl), vel[1] - vel[0], sc


def test_elastic_peak_overlap_and_contact_time(oracle_mod):
    r, v0, E, nu = 1e-3, 0.5, 1e8, 0.3
    consts = json.load(open(os.path.join(GOLDEN, "hertz_constants.json")))
    ov, dv, sc = collide(oracle_mod, r=r, v0=v0, E=E, nu=nu)
    m = 0.5 * sphere_mass(r)
    R = 0.5 * r
    Es = _estar(E, nu)
    dmax = (15.0 * m * v0 ** 2 / (16.0 * Es * math.sqrt(R))) ** 0.4
    assert ov.max() == pytest.approx(dmax, rel=2e-4)
    integral = quad(lambda x: 1.0 / math.sqrt(1.0 - x ** 2.5), 0.0, 1.0, limit=200)[0]
    assert 2 * integral == pytest.approx(consts["contact_time_over_peak"], rel=1e-4)
    tc = 2.0 * integral * dmax / v0
    assert (ov > 0).sum() * sc.h == pytest.approx(tc, rel=3e-3)
    # elastic: the spheres separate with the approach speed, head-on stays head-on
    assert dv[0] == pytest.approx(v0, rel=1e-4)
    assert abs(dv[1]) < 1e-12 and abs(dv[2]) < 1e-12


@pytest.mark.parametrize("cor", [0.2, 0.5, 0.8])
@pytest.mark.parametrize("v0", [0.1, 1.0])
def test_restitution_reproduced(oracle_mod, cor, v0):
    """The normal law's damping turns an impact speed v0 into a rebound speed CoR * v0."""
    ov, dv, _ = collide(oracle_mod, v0=v0, cor=cor, E=1e9, h=1e-7, nsteps=20000)
    assert dv[0] / v0 == pytest.approx(cor, abs=1e-3)


def test_table1_material_rebound(oracle_mod):
    t1 = json.load(open(os.path.join(GOLDEN, "table1_digital_simulant.json")))
    r = t1["component_radius_mm"][-1] * 1e-3
    ov, dv, _ = collide(oracle_mod, r=r, v0=0.3, E=t1["E"], nu=t1["nu"], cor=t1["cor"],
                        mu=t1["mu"], h=5e-8, nsteps=40000)
    assert dv[0] / 0.3 == pytest.approx(t1["cor"], abs=1e-3)


def test_resting_sphere_static_overlap(oracle_mod):
    r, E, nu, g = 1e-3, 1e8, 0.3, 9.81
    floor = scenes.plane((0, 0, 0), (0, 0, 1))
    sc = single_sphere_scene([r], E=E, nu=nu, cor=0.2, mu=0.5, g=(0, 0, -g), walls=[floor])
    sc.bin_size = 4 * r
    set_clumps(sc, [0], [[0.0, 0.0, r]])
    sim = oracle_mod.OracleSim(sc, margin=2e-5, rebuild_every=50)
    sim.step(8000)
    pos, *_ = sim.state()
    W = sphere_mass(r) * g
    Es = 1.0 / (2.0 * (1.0 - nu * nu) / E)  # sphere and wall of the same material
    delta = (W / (4.0 / 3.0 * Es * math.sqrt(r))) ** (2.0 / 3.0)
    assert r - pos[0, 2] == pytest.approx(delta, rel=1e-6)


def test_static_column_overlaps(oracle_mod):
    """A vertical column of n equal spheres on a floor: contact k from the top
    carries k m g, so its overlap follows the Hertz static law with R = r/2."""
    r, E, nu, g, n = 1e-3, 1e8, 0.3, 9.81, 4
    floor = scenes.plane((0, 0, 0), (0, 0, 1))
    sc = single_sphere_scene([r] * n, E=E, nu=nu, cor=0.2, mu=0.5, g=(0, 0, -g), walls=[floor])
    sc.bin_size = 4 * r
    set_clumps(sc, list(range(n)), [[0.0, 0.0, r + 2 * r * k] for k in range(n)])
    sim = oracle_mod.OracleSim(sc, margin=2e-5, rebuild_every=50)
    sim.step(42000)
    pos, *_ = sim.state()
    m = sphere_mass(r)
    Es = 1.0 / (2.0 * (1.0 - nu * nu) / E)
    for k in range(1, n):  # between sphere k-1 and k; load of the spheres above
        W = (n - k) * m * g
        want = (W / (4.0 / 3.0 * Es * math.sqrt(0.5 * r))) ** (2.0 / 3.0)
        got = 2 * r - (pos[k, 2] - pos[k - 1, 2])
        assert got == pytest.approx(want, rel=1e-7)
    want0 = (n * m * g / (4.0 / 3.0 * Es * math.sqrt(r))) ** (2.0 / 3.0)
    assert r - pos[0, 2] == pytest.approx(want0, rel=1e-7)
    assert np.all(pos[:, :2] == 0.0)


@pytest.mark.parametrize("theta_deg,mu", [(20.0, 0.5), (35.0, 0.5), (30.0, 0.2)])
def test_incline_stick_and_slip(oracle_mod, theta_deg, mu):
    """Gravity tilted by theta (the paper's incline trick, section 5.1): a flat
    clump resting on its face sticks for tan(theta) < mu and otherwise slides
    with acceleration g (sin(theta) - mu cos(theta))."""
    g0 = 9.81
    th = math.radians(theta_deg)
    floor = scenes.plane((0, 0, 0), (0, 0, 1))
    sc = triangle_clump_scene(E=1e8, nu=0.3, cor=0.3, mu=mu, g=(g0 * math.sin(th), 0.0, -g0 * math.cos(th)),
                              walls=[floor], h=1e-6)
    sc.bin_size = 0.01
    r = sc.tpl_rad[0]
    set_clumps(sc, [0], [[0.0, 0.0, r]])
    sim = oracle_mod.OracleSim(sc, margin=1e-4, rebuild_every=10)
    sim.step(6000)  # normal oscillation decays
    p1, _, v1, _ = sim.state()
    n2 = 4000
    sim.step(n2)
    p2, q2, v2, w2 = sim.state()
    acc = (v2[0, 0] - v1[0, 0]) / (n2 * sc.h)
    if math.tan(th) < mu:
        assert abs(v2[0, 0]) < 1e-5
        assert abs(p2[0, 0] - p1[0, 0]) < 1e-7
    else:
        want = g0 * (math.sin(th) - mu * math.cos(th))
        assert acc == pytest.approx(want, rel=2e-3)
    # it neither lifts off nor spins about the slope normal
    assert abs(w2[0]).max() < 1e-2


def test_contact_moments_balance(oracle_mod):
    """With no walls and no gravity, sum over clumps of X x F + tau vanishes at
    every force evaluation (both bodies share one contact point, A4), and sum F
    vanishes (action and reaction, A3)."""
    sc = scenes.packed_scene(11, 64, walls=False)
    sc.bin_size = scenes.default_bin_size(sc, 1e-4)
    om = oracle_mod.OracleModel(sc)
    xs, owner, tsph = om.sphere_centres(sc.tpl, sc.pos, sc.quat)
    qc, rho = om.detect_coords(xs, tsph, 1e-4)
    a, b = om.pairs_binned(owner, qc, rho)
    rng = np.random.default_rng(0)
    u0 = rng.normal(scale=1e-6, size=(len(a), 3))
    F, T, _, _, _, act = om.forces(sc.tpl, sc.pos, sc.quat, sc.vel, sc.angvel, 0.0, a, b, u0)
    assert act > 30
    scale = np.abs(F).sum()
    assert np.abs(F.sum(axis=0)).max() < 1e-13 * scale
    L = (np.cross(sc.pos, F) + T).sum(axis=0)
    assert np.abs(L).max() < 1e-13 * scale * np.abs(sc.pos).max()


def _energy(sc, pos, quat, vel, angvel, om):
    """Kinetic energy plus the Hertz potential 8/15 E* sqrt(R) delta^(5/2) of
    every overlapping pair (the work integral of the elastic term of Eq. (1a))."""
    from scipy.spatial.transform import Rotation
    m = sc.tpl_mass[sc.tpl]
    I = sc.tpl_inertia[sc.tpl]
    R = Rotation.from_quat(quat[:, [1, 2, 3, 0]])
    wb = R.inv().apply(angvel)
    ke = 0.5 * (m * (vel ** 2).sum(1)).sum() + 0.5 * (I * wb ** 2).sum()
    xs, owner, tsph = om.sphere_centres(sc.tpl, pos, quat)
    pe = 0.0
    n = len(xs)
    for i in range(n):
        d = np.linalg.norm(xs[i + 1:] - xs[i], axis=1)
        rr = sc.tpl_rad[tsph[i]] + sc.tpl_rad[tsph[i + 1:]]
        ok = (owner[i + 1:] != owner[i]) & (d < rr)
        for j in np.nonzero(ok)[0]:
            ra, rb = sc.tpl_rad[tsph[i]], sc.tpl_rad[tsph[i + 1 + j]]
            Es, Gs, mu, e = om.pair_material(sc.tpl_mat[tsph[i]], sc.tpl_mat[tsph[i + 1 + j]])
            Rb = ra * rb / (ra + rb)
            pe += 8.0 / 15.0 * Es * math.sqrt(Rb) * (rr[j] - d[j]) ** 2.5
    return ke + pe


def test_energy_conserved_without_dissipation(oracle_mod):
    sc = scenes.packed_scene(4, 27, compress=0.97, walls=False, vel_scale=0.2, ang_scale=50.0)
    sc.cor = np.ones_like(sc.cor)
    sc.mu = np.zeros_like(sc.mu)
    sc.g = (0.0, 0.0, 0.0)
    sc.h = 2e-7
    sc.bin_size = scenes.default_bin_size(sc, 2e-4)
    om = oracle_mod.OracleModel(sc)
    sim = oracle_mod.OracleSim(sc, margin=2e-4, rebuild_every=20)
    e0 = _energy(sc, sc.pos, sc.quat, sc.vel, sc.angvel, om)
    sim.step(1500)
    e1 = _energy(sc, *sim.state(), om)
    assert abs(e1 - e0) / e0 < 1e-4


def test_linear_momentum_conserved(oracle_mod):
    sc = scenes.packed_scene(6, 40, walls=False)
    sc.g = (0.0, 0.0, 0.0)
    sc.bin_size = scenes.default_bin_size(sc, 1e-4)
    m = sc.tpl_mass[sc.tpl][:, None]
    p0 = (m * sc.vel).sum(0)
    sim = oracle_mod.OracleSim(sc, margin=1e-4, rebuild_every=10)
    sim.step(300)
    _, _, vel, _ = sim.state()
    p1 = (m * vel).sum(0)
    assert np.abs(p1 - p0).max() < 1e-12 * (m * np.abs(vel)).sum()


def test_deferred_rebuild_equals_every_step_rebuild(oracle_mod):
    """Section 2.2: with a margin that covers the motion between rebuilds, the
    deferred list gives the same trajectory as rebuilding every step, which
    requires the tangential history to survive each rebuild unchanged."""
    sc = scenes.packed_scene(8, 40, compress=0.98)
    sc.bin_size = scenes.default_bin_size(sc, 2e-4)
    a = oracle_mod.OracleSim(sc, margin=2e-4, rebuild_every=1)
    b = oracle_mod.OracleSim(sc, margin=2e-4, rebuild_every=25)
    assert a.step(200, audit=True) == 0
    assert b.step(200, audit=True) == 0
    sa, sb = a.state(), b.state()
    for x, y in zip(sa, sb):
        assert np.array_equal(x, y)
    # and the history is non-trivial: some contact carries a tangential displacement
    ua = a.contacts()[2]
    assert np.abs(ua).max() > 1e-9


def test_history_lost_if_not_carried(oracle_mod):
    """Control for the test above: a margin too small to keep pairs listed from
    one rebuild to the next changes the trajectory (the history matters)."""
    sc = scenes.packed_scene(8, 40, compress=0.98)
    sc.bin_size = scenes.default_bin_size(sc, 2e-4)
    a = oracle_mod.OracleSim(sc, margin=2e-4, rebuild_every=1)
    a.step(200)
    # rebuilding every step but through a fresh simulation each step drops u_t
    b_state = sc
    for _ in range(200):
        s = oracle_mod.OracleSim(b_state, margin=2e-4, rebuild_every=1)
        s.step(1)
        pos, quat, vel, angvel = s.state()
        b_state = scenes.Scene(**{**sc.__dict__, "pos": pos, "quat": quat, "vel": vel, "angvel": angvel})
    assert not np.array_equal(a.state()[0], b_state.pos)


def test_false_positive_has_no_force_and_resets_history(oracle_mod):
    sc = single_sphere_scene([1e-3, 1e-3], mu=0.5)
    om = oracle_mod.OracleModel(sc)
    args = dict(mat_a=0, mat_b=0, Xa=[0, 0, 0], Xb=[2.001e-3, 0, 0], va=[0, 0, 0], wa=[0, 0, 0],
                vb=[-1, 0.3, 0], wb=[0, 0, 0], ra=1e-3, rb=1e-3, ma=1e-5, mb=1e-5)
    act, F, u, *_ = om.contact(xa=[0, 0, 0], xb=[2.001e-3, 0, 0], u=[1e-7, 2e-7, 0], **args)
    assert not act and np.all(F == 0) and np.all(u == 0)


def test_tangential_history_update_and_cap(oracle_mod):
    """Eq. (3)-(4): u' = u + h v_t projected on the tangent plane; capped so
    that f k_t |u| = mu |F_n| when the friction force would exceed mu |F_n|."""
    E, nu, mu = 1e8, 0.3, 0.3
    sc = single_sphere_scene([1e-3, 1e-3], E=E, nu=nu, mu=mu, cor=1.0, h=1e-6)
    om = oracle_mod.OracleModel(sc)
    r, dn = 1e-3, 1e-6
    xb = [2 * r - dn, 0, 0]
    common = dict(mat_a=0, mat_b=0, xa=[0, 0, 0], xb=xb, Xa=[0, 0, 0], Xb=xb, va=[0, 0, 0],
                  wa=[0, 0, 0], wb=[0, 0, 0], ra=r, rb=r, ma=1e-5, mb=1e-5)
    Gs = 1.0 / (2 * 2.0 * (2.0 - nu) * (1.0 + nu) / E)
    f = math.sqrt(0.5 * r * dn)
    Fn = f * 4.0 / 3.0 * (1.0 / (2 * (1 - nu * nu) / E)) * dn
    # small slip: stays elastic; history gets the tangential increment only
    act, F, u, *_ = om.contact(vb=[0.5, 1e-4, 0], u=[0, 0, 0], **common)
    assert act
    assert u == pytest.approx([0.0, 1e-10, 0.0], abs=1e-22)
    assert F[1] == pytest.approx(-f * 8 * Gs * 1e-10, rel=1e-12)
    assert F[0] == pytest.approx(Fn, rel=1e-12)
    # large history: capped at mu |F_n|
    act, F, u, *_ = om.contact(vb=[0, 0, 0], u=[0, 1e-4, 0], **common)
    assert math.hypot(F[1], F[2]) == pytest.approx(mu * abs(F[0]), rel=1e-12)
    assert f * 8 * Gs * abs(u[1]) == pytest.approx(mu * abs(F[0]), rel=1e-12)
    # the normal component of a stored displacement is projected out (Eq. 3)
    act, F, u, *_ = om.contact(vb=[0, 0, 0], u=[3e-9, 2e-9, 0], **common)
    assert u[0] == 0.0 and u[1] == pytest.approx(2e-9, rel=1e-15)


def test_wall_moments_balance(oracle_mod):
    """Walls in the balance: for clumps pressed against moving box walls, the
    total moment about the origin of every load vanishes, sum over clumps of
    X x F + tau plus sum over walls of p_w(t) x F_w + tau_w, where tau_w is the
    moment the oracle reports for wall w about its reference point p_w(t) =
    p + v t; and the wall forces balance the clump forces."""
    sc = scenes.packed_scene(12, 64, walls=True, compress=0.9)
    rng = np.random.default_rng(3)
    for w in sc.walls:
        w["vel"] = tuple(rng.normal(scale=0.05, size=3))
    t = 0.37
    # the walls' positions at time t are where the packing put them at t = 0
    for w in sc.walls:
        w["p"] = tuple(np.asarray(w["p"]) - t * np.asarray(w["vel"]))
    sc.bin_size = scenes.default_bin_size(sc, 1e-4)
    om = oracle_mod.OracleModel(sc)
    xs, owner, tsph = om.sphere_centres(sc.tpl, sc.pos, sc.quat)
    qc, rho = om.detect_coords(xs, tsph, 1e-4)
    a, b = om.pairs_binned(owner, qc, rho)
    ws, ww = om.wall_candidates(xs, tsph, 1e-4, t, 0.0)
    F, T, Fw, _, _, act, Tw = om.forces(sc.tpl, sc.pos, sc.quat, sc.vel, sc.angvel, t, a, b,
                                        np.zeros((len(a), 3)), ws, ww, np.zeros((len(ws), 3)),
                                        wall_torque=True)
    loaded = np.abs(Fw).sum(axis=1) > 0
    assert loaded.sum() >= 3 and act > 30
    scale = np.abs(F).sum() + np.abs(Fw).sum()
    assert np.abs(F.sum(axis=0) + Fw.sum(axis=0)).max() < 1e-13 * scale
    pw = np.array([np.asarray(w["p"]) + t * np.asarray(w["vel"]) for w in sc.walls])
    L = (np.cross(sc.pos, F) + T).sum(axis=0) + (np.cross(pw, Fw) + Tw).sum(axis=0)
    assert np.abs(L).max() < 1e-13 * scale * (np.abs(sc.pos).max() + np.abs(pw).max())
    # and the wall moments are not trivially zero
    assert np.abs(Tw).max() > 1e-6 * np.abs(Fw).max() * np.abs(sc.pos).max()


def test_facet_moments_balance(oracle_mod):
    """The same balance with the box as 12 mesh facets, each translating with
    its own velocity (every vertex moves with it): clumps touching a face's
    two facets, edges and corners included."""
    sc = scenes.packed_scene(12, 64, walls=True, compress=0.9)
    pl = sc.walls
    x0 = max(w["p"][0] for w in pl if w["n"][0] > 0.5)
    x1 = min(w["p"][0] for w in pl if w["n"][0] < -0.5)
    y0 = max(w["p"][1] for w in pl if w["n"][1] > 0.5)
    y1 = min(w["p"][1] for w in pl if w["n"][1] < -0.5)
    z0 = max(w["p"][2] for w in pl if w["n"][2] > 0.5)
    rng = np.random.default_rng(4)
    t = 0.37
    sc.walls = []
    for f in scenes.box_mesh(x0, x1, y0, y1, z0, sc.hi[2]):
        v = rng.normal(scale=0.05, size=3)
        g = {k: tuple(np.asarray(f[k]) - t * v) for k in ("p", "b", "c")}
        sc.walls.append(dict(f, vel=tuple(v), **g))
    sc.bin_size = scenes.default_bin_size(sc, 1e-4)
    om = oracle_mod.OracleModel(sc)
    xs, owner, tsph = om.sphere_centres(sc.tpl, sc.pos, sc.quat)
    qc, rho = om.detect_coords(xs, tsph, 1e-4)
    a, b = om.pairs_binned(owner, qc, rho)
    ws, ww = om.wall_candidates(xs, tsph, 1e-4, t, 0.0)
    F, T, Fw, _, _, act, Tw = om.forces(sc.tpl, sc.pos, sc.quat, sc.vel, sc.angvel, t, a, b,
                                        np.zeros((len(a), 3)), ws, ww, np.zeros((len(ws), 3)),
                                        wall_torque=True)
    assert (np.abs(Fw).sum(axis=1) > 0).sum() >= 5 and act > 30
    scale = np.abs(F).sum() + np.abs(Fw).sum()
    assert np.abs(F.sum(axis=0) + Fw.sum(axis=0)).max() < 1e-13 * scale
    pw = np.array([np.asarray(w["p"]) + t * np.asarray(w["vel"]) for w in sc.walls])
    L = (np.cross(sc.pos, F) + T).sum(axis=0) + (np.cross(pw, Fw) + Tw).sum(axis=0)
    assert np.abs(L).max() < 1e-13 * scale * (np.abs(sc.pos).max() + np.abs(pw).max())
    assert np.abs(Tw).max() > 1e-6 * np.abs(Fw).max() * np.abs(sc.pos).max()
