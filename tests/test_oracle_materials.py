"""Pins of the oracle's mixing of two spheres' materials into one contact
(section 2.1: every component sphere carries its own E, nu, mu and CoR, and
Eq. (1) takes one effective value of each per contact).

The mixing of E and nu follows Hertz and Mindlin: the two bodies' normal and
tangential compliances add.  It is pinned three ways, none of which retypes
the oracle's expression: the limit of a rigid partner (the textbook contact
of an elastic sphere with a rigid flat), the additivity of compliances across
the three material pairs (a, a), (b, b), (a, b), and whole collisions whose
peak overlap is the Hertz closed form.  The mixing of mu and CoR (mean, min or
max of the two values) is pinned by rebounds and by stick/slip on a tilted
plane of another material.
"""
import math

import numpy as np
import pytest

from paper_2307_03445_gb300 import scenes
from tests.helpers import set_clumps, single_sphere_scene, sphere_mass, triangle_clump_scene

# two materials of the benchmark's family with different E and nu (the tests
# fail on a swapped index only when both differ)
E2 = np.array([5e7, 1e9])
NU2 = np.array([0.25, 0.35])


def _model(oracle_mod, E, nu, mu=(0.5, 0.5), cor=(0.5, 0.5), mix=0):
    sc = single_sphere_scene([1e-3, 1e-3], E=E, nu=nu, mu=mu, cor=cor, mats=[0, 1])
    sc.mix_rule = mix
    return oracle_mod.OracleModel(sc)


def test_rigid_partner_limit(oracle_mod):
    """Against a rigid body the effective moduli are the elastic body's own
    plane-strain modulus E/(1 - nu^2) (Hertz, sphere on a rigid flat) and
    G/(2 - nu) with G = E / (2 (1 + nu)) (Mindlin); either order of the pair."""
    for k in (0, 1):
        E = np.array([E2[k], 1e40])
        nu = np.array([NU2[k], 0.45])
        om = _model(oracle_mod, E, nu)
        G = E2[k] / (2.0 * (1.0 + NU2[k]))
        for ia, ib in ((0, 1), (1, 0)):
            Es, Gs, _, _ = om.pair_material(ia, ib)
            assert Es == pytest.approx(E2[k] / (1.0 - NU2[k] ** 2), rel=1e-13)
            assert Gs == pytest.approx(G / (2.0 - NU2[k]), rel=1e-13)


def test_compliances_add(oracle_mod):
    """The compliance 1/E* of a mixed pair is the mean of those of the two
    like pairs (each body's deformation adds to the approach), and the same
    for 1/G*; a like pair of identical spheres has E* = E / (2 (1 - nu^2))."""
    rng = np.random.default_rng(3)
    for _ in range(20):
        E = rng.choice([5e7, 1e8, 5e8, 1e9], size=2, replace=False)
        nu = rng.uniform(0.1, 0.45, size=2)
        om = _model(oracle_mod, E, nu)
        Eab, Gab, _, _ = om.pair_material(0, 1)
        Eaa, Gaa, _, _ = om.pair_material(0, 0)
        Ebb, Gbb, _, _ = om.pair_material(1, 1)
        assert 1.0 / Eab == pytest.approx(0.5 * (1.0 / Eaa + 1.0 / Ebb), rel=1e-13)
        assert 1.0 / Gab == pytest.approx(0.5 * (1.0 / Gaa + 1.0 / Gbb), rel=1e-13)
        assert Eaa == pytest.approx(E[0] / (2.0 * (1.0 - nu[0] ** 2)), rel=1e-13)
        assert Ebb == pytest.approx(E[1] / (2.0 * (1.0 - nu[1] ** 2)), rel=1e-13)
        G = E / (2.0 * (1.0 + nu))
        assert Gaa == pytest.approx(G[0] / (2.0 * (2.0 - nu[0])), rel=1e-13)
        assert om.pair_material(1, 0)[:2] == (Eab, Gab)


@pytest.mark.parametrize("rule,pick", [(0, lambda a, b: 0.5 * (a + b)), (1, min), (2, max)])
def test_mu_and_cor_rules(oracle_mod, rule, pick):
    om = _model(oracle_mod, E2, NU2, mu=(0.2, 0.7), cor=(0.3, 0.8), mix=rule)
    for ia, ib in ((0, 1), (1, 0)):
        _, _, mu, e = om.pair_material(ia, ib)
        assert mu == pick(0.2, 0.7) and e == pick(0.3, 0.8)
    # like pairs keep their own values under every rule
    assert om.pair_material(0, 0)[2:] == (0.2, 0.3)
    assert om.pair_material(1, 1)[2:] == (0.7, 0.8)


def collide_two(oracle_mod, ra, rb, E, nu, cor, mix=0, v0=0.5, h=2e-7, nsteps=20000):
    """Head-on collision of two single spheres of materials 0 and 1 with the
    centre of mass at rest; returns the overlap history, the approach speed
    and the relative velocity after separation."""
    sc = single_sphere_scene([ra, rb], E=E, nu=nu, mu=(0.0, 0.0), cor=cor, h=h, mats=[0, 1])
    sc.mix_rule = mix
    sc.bin_size = 4 * max(ra, rb)
    ma, mb = sphere_mass(ra), sphere_mass(rb)
    gap = 2e-6
    set_clumps(sc, [0, 1], [[-ra - gap, 0, 0], [rb + gap, 0, 0]],
               vel=[[v0 * mb / (ma + mb), 0, 0], [-v0 * ma / (ma + mb), 0, 0]])
    sim = oracle_mod.OracleSim(sc, margin=5e-5, rebuild_every=20)
    ov = []
    for _ in range(nsteps):
        sim.step(1)
        pos, _, vel, _ = sim.state()
        ov.append(ra + rb - (pos[1, 0] - pos[0, 0]))
        if ov[-1] < -4 * gap and max(ov) > 0:
            break
    pos, _, vel, _ = sim.state()
    p = ma * vel[0] + mb * vel[1]
    return np.array(ov), vel[1] - vel[0], p, (ma, mb)


def test_two_material_elastic_peak_overlap(oracle_mod):
    """Spheres of 1 and 1.5 mm, E = 5e7 / 1e9 Pa, nu = 0.25 / 0.35, CoR 1: the
    peak overlap is Hertz's (15 m v0^2 / (16 E* sqrt(R)))^(2/5) with
    1/E* = (1 - nu_a^2)/E_a + (1 - nu_b^2)/E_b, R and m the reduced radius and
    mass; the spheres separate with the approach speed and momentum stays 0."""
    ra, rb, v0 = 1e-3, 1.5e-3, 0.5
    ov, dv, p, (ma, mb) = collide_two(oracle_mod, ra, rb, E2, NU2, (1.0, 1.0), v0=v0)
    Es = 1.0 / ((1.0 - NU2[0] ** 2) / E2[0] + (1.0 - NU2[1] ** 2) / E2[1])
    R = ra * rb / (ra + rb)
    m = ma * mb / (ma + mb)
    dmax = (15.0 * m * v0 ** 2 / (16.0 * Es * math.sqrt(R))) ** 0.4
    assert ov.max() == pytest.approx(dmax, rel=2e-4)
    assert dv[0] == pytest.approx(v0, rel=1e-4)
    assert abs(p[0]) < 1e-12 * ma * v0


@pytest.mark.parametrize("rule,want", [(0, 0.5), (1, 0.3), (2, 0.7)])
def test_two_material_restitution_follows_the_rule(oracle_mod, rule, want):
    """Spheres of CoR 0.3 and 0.7 rebound with the mixed CoR of the rule
    (mean 0.5, min 0.3, max 0.7), to the 1e-3 of the single-material pin."""
    E = np.array([1e9, 1e9])
    ov, dv, _, _ = collide_two(oracle_mod, 1e-3, 1e-3, E, NU2, (0.3, 0.7), mix=rule, v0=0.3,
                               h=1e-7, nsteps=40000)
    assert dv[0] / 0.3 == pytest.approx(want, abs=1e-3)


@pytest.mark.parametrize("rule,mu_eff", [(0, 0.4), (1, 0.2), (2, 0.6)])
def test_incline_friction_follows_the_rule(oracle_mod, rule, mu_eff):
    """A flat clump of material 0 (mu 0.2) on a plane of material 1 (mu 0.6)
    under gravity tilted by 30 degrees (tan = 0.577): it slides with
    g (sin - mu cos) for the mean (0.4) and min (0.2) rules and sticks for
    the max rule (0.6)."""
    g0, th = 9.81, math.radians(30.0)
    floor = scenes.plane((0, 0, 0), (0, 0, 1), material=1)
    sc = triangle_clump_scene(E=(1e8, 1e8), nu=(0.3, 0.3), cor=(0.3, 0.3), mu=(0.2, 0.6),
                              g=(g0 * math.sin(th), 0.0, -g0 * math.cos(th)), walls=[floor], h=1e-6)
    sc.mix_rule = rule
    sc.bin_size = 0.01
    r = sc.tpl_rad[0]
    set_clumps(sc, [0], [[0.0, 0.0, r]])
    sim = oracle_mod.OracleSim(sc, margin=1e-4, rebuild_every=10)
    sim.step(6000)
    p1, _, v1, _ = sim.state()
    n2 = 4000
    sim.step(n2)
    p2, _, v2, _ = sim.state()
    if math.tan(th) < mu_eff:
        assert abs(v2[0, 0]) < 1e-5 and abs(p2[0, 0] - p1[0, 0]) < 1e-7
    else:
        acc = (v2[0, 0] - v1[0, 0]) / (n2 * sc.h)
        assert acc == pytest.approx(g0 * (math.sin(th) - mu_eff * math.cos(th)), rel=2e-3)
