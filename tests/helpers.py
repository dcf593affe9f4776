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


def settling_box_scene(n=400, seed=5, side=0.03, E=1e7, h=1e-5):
    """Clumps of three overlapping spheres (the 1,000-clump workload's
    templates, 20 of them) on a jittered lattice above the floor of a
    side x side box, at rest; a soft material (E, CoR 0.3) so that a step of
    h resolves the contacts and the bed settles within a few thousand steps.
    Templates and positions are exact in the FP32 voxel layout, so every
    precision mode starts from the same state."""
    sc = scenes.config1(seed=seed, n_clumps=n, n_templates=20)
    sc.E, sc.cor, sc.mu = np.array([E]), np.array([0.3]), np.array([0.5])
    sc.h = h
    rng = np.random.default_rng(seed + 1)
    bound = sc.bounding_radius()[sc.tpl]
    sp = 2.0 * float(bound.max()) + 2e-4
    P = scenes.lattice_positions(n, sp, 0.0, side, 0.0, side, 0.0, rng, 0.1 * sp)
    P[:, 2] += float(bound.max())
    sc.pos = P
    sc.quat = scenes.random_quaternions(rng, n)
    sc.vel, sc.angvel = np.zeros((n, 3)), np.zeros((n, 3))
    sc.walls = scenes.box_walls(0.0, side, 0.0, side, 0.0)
    sc.lo = (-2.0 ** -9, -2.0 ** -9, -2.0 ** -9)  # on the FP32 offset grid
    sc.hi = (side + 0.002, side + 0.002, float(P[:, 2].max()) + 0.01)
    sc.tpl_pos = sc.tpl_pos.astype(np.float32).astype(np.float64)
    sc.tpl_rad = sc.tpl_rad.astype(np.float32).astype(np.float64)
    scenes.snap_to_voxel_grid(sc)
    return sc
