"""Benchmark workloads built with the library itself.

The paper-scale bed (11,000,000 clumps, ~34,000,000 spheres in a 4 x 2 m box
with a plate sliding on top) is prepared the way the paper prepares its test
beds (section 4.1): one patch of clumps is spawned on size-layered lattices,
settled under gravity, then copy-pasted side by side to fill the box.  The
patch is settled with softer contacts and a longer time step (a preparation
setting, not the measured one); the measured run then uses the workload's own
materials and dt = 1e-6 s from that settled, copied bed.
"""
from __future__ import annotations

import math
import time

import numpy as np

from . import Simulation, scenes


def _prep_scene(base: scenes.Scene, n_patch: int, foot: float, rng):
    sc = scenes.Scene(
        "patch", base.tpl_off, base.tpl_pos, base.tpl_rad, base.tpl_mat, base.tpl_mass,
        base.tpl_inertia, np.full(len(base.E), 5e7), np.full(len(base.E), 0.3),
        np.full(len(base.E), 0.5), np.full(len(base.E), 0.2), h=5e-6, g=(0.0, 0.0, -9.81),
        lo=(0.0, 0.0, 0.0), hi=(foot, foot, 2.0), bin_size=0.0,
        walls=scenes.box_walls(0.0, foot, 0.0, foot, 0.0), precision=scenes.PREC_FP32)
    tpl = rng.integers(0, len(base.tpl_mass), size=n_patch).astype(np.int32)
    bound = sc.bounding_radius()[tpl]
    P = scenes.layered_positions(bound, 0.0, foot, 0.0, foot, 0.0, gap=4e-4, rng=rng,
                                 jitter=1e-4)
    sc.tpl = tpl
    sc.pos = P
    sc.quat = scenes.random_quaternions(rng, n_patch)
    sc.vel = np.zeros((n_patch, 3))
    sc.angvel = np.zeros((n_patch, 3))
    sc.hi = (foot, foot, float(P[:, 2].max()) + 0.05)
    return sc


def settle(sc: scenes.Scene, t_end: float, v_bound=6.0, K=10, log=None, chunk=2000):
    """Runs the scene until simulated time t_end; returns the final state."""
    sim = Simulation(sc, margin=v_bound * sc.h * K * 1.5, rebuild_interval=K)
    n = int(round(t_end / sc.h))
    done = 0
    t0 = time.time()
    while done < n:
        k = min(chunk, n - done)
        sim.step(k)
        done += k
    if log:
        st = sim.stats()
        log(f"settled {sc.n_clumps} clumps for {n} steps in {time.time() - t0:.1f} s "
            f"({st['rebuilds']} rebuilds, {st['n_pairs']} pairs)")
    out = sim.state()
    sim.close()
    return out


def bed_c5(n_clumps=11_000_000, lx=4.0, ly=2.0, patch=0.25, seed=1239, log=None,
           settle_time=None, stiffen_time=6e-3, spatial_order=True):
    """The paper-scale bed: a settled patch copy-pasted over lx x ly; with
    spatial_order the clumps are numbered along a space-filling curve."""
    base = scenes.config5(seed=seed, n_clumps=1, lx=lx, ly=ly)
    rng = np.random.default_rng(seed + 1)
    nx, ny = int(round(lx / patch)), int(round(ly / patch))
    tiles = nx * ny
    n_patch = int(math.ceil(n_clumps / tiles))
    psc = _prep_scene(base, n_patch, patch, rng)
    fall = math.sqrt(2.0 * float(psc.pos[:, 2].max()) / 9.81)
    t_end = settle_time if settle_time is not None else fall + 0.15
    pos, quat, vel, angvel = settle(psc, t_end, log=log)
    # stiffen: the workload's own materials and time step, until the elastic
    # energy stored by the softer preparation contacts has been released
    psc.E, psc.nu, psc.mu, psc.cor = base.E, base.nu, base.mu, base.cor
    psc.h = base.h
    psc.pos, psc.quat, psc.vel, psc.angvel = pos, quat, vel, angvel
    pos, quat, vel, angvel = settle(psc, stiffen_time, v_bound=2.0, K=20, log=log)
    # copy-paste the patch over the box
    P = np.concatenate([pos + np.array([i * patch, j * patch, 0.0])
                        for j in range(ny) for i in range(nx)])[:n_clumps]
    Q = np.concatenate([quat] * tiles)[:n_clumps]
    T = np.concatenate([psc.tpl] * tiles)[:n_clumps]
    if spatial_order:
        # number the clumps along a Morton curve (cells of the largest clump)
        perm = scenes.morton_order(P, (0.0, 0.0, 0.0), 2.0 * float(base.bounding_radius().max()))
        P, Q, T = P[perm], Q[perm], T[perm]
    top = float((P[:, 2] + base.bounding_radius()[T]).max())
    sc = base
    sc.tpl = T
    sc.pos = P
    sc.quat = Q
    sc.vel = np.zeros((len(T), 3))
    sc.angvel = np.zeros((len(T), 3))
    plate = top + 1e-4
    sc.walls = scenes.box_walls(0.0, lx, 0.0, ly, 0.0, top=plate, top_vel=(0.2, 0.0, 0.0))
    sc.hi = (lx, ly, plate + 0.01)
    return sc


def compress(sim, plate_wall: dict, plate: int, speed: float, load: float, max_steps: int,
             chunk: int = 10):
    """Virtual compressor (section 4.1: the beds are compacted by a plate
    before a test).  Drives the plane wall `plate` (its dict as given at
    creation, `plate_wall`, whose normal points into the grains) into the bed
    at `speed` m/s along its normal, checking the load on it every `chunk`
    steps, until the grains push back with at least `load` newtons or
    `max_steps` steps have run; then holds the plate where it is.  Returns
    (steps run, final load, plate position).  Uses the library's wall loads
    and wall motion calls (the co-simulation hook)."""
    n = np.asarray(plate_wall["n"], float)
    n = n / np.linalg.norm(n)
    t0 = sim.stats()["time"]
    p = np.asarray(plate_wall["p"], float) + np.asarray(plate_wall["vel"], float) * t0
    sim.set_wall_motion(plate, p, speed * n)
    steps, push = 0, 0.0
    while steps < max_steps:
        k = min(chunk, max_steps - steps)
        sim.step(k)
        steps += k
        F, _ = sim.wall_loads()
        push = -float(np.dot(F[plate], n))  # grains push the plate back along -n
        if push >= load:
            break
    p = p + speed * n * (sim.stats()["time"] - t0)
    sim.set_wall_motion(plate, p, np.zeros(3))
    return steps, push, p


def facet_box(walls):
    """The same axis-aligned box as mesh facets: the floor, the four sides and
    the top plate of `walls` (planes) become 12 facets; the two top facets
    keep the plate's sliding velocity."""
    def plane_at(axis, sign):
        return next(w for w in walls if w["type"] == scenes.WALL_PLANE and w["n"][axis] * sign > 0.5)

    x0, x1 = plane_at(0, 1)["p"][0], plane_at(0, -1)["p"][0]
    y0, y1 = plane_at(1, 1)["p"][1], plane_at(1, -1)["p"][1]
    top = plane_at(2, -1)
    facets = scenes.box_mesh(x0, x1, y0, y1, plane_at(2, 1)["p"][2], top["p"][2])
    for f in facets:
        if f["n"][2] < -0.5:
            f["vel"] = tuple(top["vel"])
    return facets
