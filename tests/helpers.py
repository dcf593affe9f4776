"""Small scene builders shared by the tests (inputs only, no method arithmetic)."""
import math

import numpy as np

from paper_2307_03445_gb300 import scenes

RHO = scenes.DENSITY


def sphere_mass(r):
    return RHO * 4.0 / 3.0 * math.pi * r ** 3


def single_sphere_scene(radii, E=1e8, nu=0.3, mu=0.5, cor=0.5, h=1e-6, g=(0.0, 0.0, 0.0),
                        walls=(), lo=(-0.05, -0.05, -0.05), hi=(0.05, 0.05, 0.05), n_mat=None,
                        mats=None):
    """Templates that are single spheres (exact mass and inertia)."""
    radii = np.asarray(radii, float)
    n = len(radii)
    if n_mat is None:
        E, nu, mu, cor = (np.atleast_1d(np.asarray(v, float)) for v in (E, nu, mu, cor))
    sc = scenes.Scene(
        "spheres",
        tpl_off=np.arange(n + 1, dtype=np.int32),
        tpl_pos=np.zeros((n, 3)),
        tpl_rad=radii.copy(),
        tpl_mat=np.zeros(n, np.int32) if mats is None else np.asarray(mats, np.int32),
        tpl_mass=np.array([sphere_mass(r) for r in radii]),
        tpl_inertia=np.array([[0.4 * sphere_mass(r) * r * r] * 3 for r in radii]),
        E=np.atleast_1d(E), nu=np.atleast_1d(nu), mu=np.atleast_1d(mu), cor=np.atleast_1d(cor),
        h=h, g=tuple(g), lo=tuple(lo), hi=tuple(hi), bin_size=0.01, walls=list(walls))
    return sc


def set_clumps(sc, tpl, pos, vel=None, angvel=None, quat=None):
    n = len(tpl)
    sc.tpl = np.asarray(tpl, np.int32)
    sc.pos = np.asarray(pos, float).reshape(n, 3)
    sc.quat = np.tile([1.0, 0.0, 0.0, 0.0], (n, 1)) if quat is None else np.asarray(quat, float)
    sc.vel = np.zeros((n, 3)) if vel is None else np.asarray(vel, float).reshape(n, 3)
    sc.angvel = np.zeros((n, 3)) if angvel is None else np.asarray(angvel, float).reshape(n, 3)
    return sc


def triangle_clump_scene(r=1e-3, arm=1.2e-3, **kw):
    """One flat clump of three equal spheres at the corners of an equilateral
    triangle in its xy plane (a clump that cannot roll on its face)."""
    p = np.array([[arm * math.cos(2 * math.pi * k / 3), arm * math.sin(2 * math.pi * k / 3), 0.0]
                  for k in range(3)])
    m, com, I = scenes.union_mass_properties(p, [r, r, r])
    w, V = np.linalg.eigh(I)
    sc = single_sphere_scene([r], **kw)
    sc.tpl_off = np.array([0, 3], np.int32)
    sc.tpl_pos = p - com
    sc.tpl_rad = np.array([r, r, r])
    sc.tpl_mat = np.zeros(3, np.int32)
    sc.tpl_mass = np.array([m])
    sc.tpl_inertia = np.array([np.diag(I)])
    return sc
