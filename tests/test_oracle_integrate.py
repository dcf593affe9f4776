"""Pins of the oracle's explicit integration of the equations of motion
(section 2.1, Eq. (5a), (5b)) against closed-form motions."""
import math

import numpy as np
import pytest
from scipy.spatial.transform import Rotation

from paper_2307_03445_gb300 import scenes
from tests.helpers import set_clumps, single_sphere_scene


def _free_model(oracle_mod, g=(0.3, -1.0, -9.81), h=1e-5):
    sc = scenes.packed_scene(2, 1, walls=False)
    sc.g = g
    sc.h = h
    sc.bin_size = 0.01
    return sc, oracle_mod.OracleModel(sc)


def test_free_flight_matches_semi_implicit_euler_closed_form(oracle_mod):
    sc, om = _free_model(oracle_mod)
    g = np.array(sc.g)
    x0, v0 = sc.pos.copy(), sc.vel.copy()
    pos, quat, vel, angvel = sc.pos, sc.quat, sc.vel, np.zeros((1, 3))
    n = 500
    for _ in range(n):
        pos, quat, vel, angvel = om.integrate(sc.tpl, pos, quat, vel, angvel, np.zeros((1, 3)), np.zeros((1, 3)))
    h = sc.h
    assert np.allclose(vel, v0 + n * h * g, rtol=0, atol=1e-13)
    want = x0 + n * h * v0 + h * h * g * n * (n + 1) / 2
    assert np.allclose(pos, want, rtol=0, atol=1e-13)


def test_spin_about_a_principal_axis_is_uniform(oracle_mod):
    sc, om = _free_model(oracle_mod, g=(0.0, 0.0, 0.0), h=1e-6)
    w = 150.0
    quat = np.array([[1.0, 0.0, 0.0, 0.0]])
    angvel = np.array([[0.0, 0.0, w]])  # body axes = world axes at start; z is principal
    pos, vel = sc.pos.copy(), np.zeros((1, 3))
    n = 4000
    for _ in range(n):
        pos, quat, vel, angvel = om.integrate(sc.tpl, pos, quat, vel, angvel, np.zeros((1, 3)), np.zeros((1, 3)))
    th = n * sc.h * w
    assert quat[0] == pytest.approx([math.cos(th / 2), 0, 0, math.sin(th / 2)], abs=1e-12)
    assert angvel[0] == pytest.approx([0.0, 0.0, w], abs=1e-9)


def test_torque_free_body_keeps_angular_momentum(oracle_mod):
    sc, om = _free_model(oracle_mod, g=(0.0, 0.0, 0.0), h=1e-6)
    I = sc.tpl_inertia[sc.tpl[0]]
    assert len(set(np.round(I / I.max(), 3))) == 3  # asymmetric top
    angvel = np.array([[40.0, -70.0, 55.0]])
    quat, pos, vel = sc.quat.copy(), sc.pos.copy(), np.zeros((1, 3))

    def L(q, w):
        R = Rotation.from_quat(q[0, [1, 2, 3, 0]])
        return R.apply(I * R.inv().apply(w[0]))

    L0 = L(quat, angvel)
    n = 2000
    for _ in range(n):
        pos, quat, vel, angvel = om.integrate(sc.tpl, pos, quat, vel, angvel, np.zeros((1, 3)), np.zeros((1, 3)))
    # the explicit gyroscopic update is first order: drift of order n (h |w|)^2 |L|
    hw = sc.h * np.linalg.norm([40.0, -70.0, 55.0])
    assert np.linalg.norm(L(quat, angvel) - L0) <= 3 * n * hw * hw * np.linalg.norm(L0)
    assert np.linalg.norm(quat) == pytest.approx(1.0, abs=1e-15)


def test_applied_force_and_torque(oracle_mod):
    sc = single_sphere_scene([1e-3], g=(0.0, 0.0, 0.0), h=1e-6)
    set_clumps(sc, [0], [[0.0, 0.0, 0.0]])
    om = oracle_mod.OracleModel(sc)
    m, I = sc.tpl_mass[0], sc.tpl_inertia[0, 0]
    F = np.array([[1e-3, 0.0, 0.0]])
    T = np.array([[0.0, 2e-9, 0.0]])
    pos, quat, vel, angvel = om.integrate(sc.tpl, sc.pos, sc.quat, sc.vel, sc.angvel, F, T)
    assert vel[0] == pytest.approx([sc.h * 1e-3 / m, 0, 0], rel=1e-14)
    assert pos[0] == pytest.approx([sc.h * sc.h * 1e-3 / m, 0, 0], rel=1e-14)
    assert angvel[0] == pytest.approx([0, sc.h * 2e-9 / I, 0], rel=1e-12)
