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

import dataclasses
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


def settled_bed(base: scenes.Scene, n_clumps: int, x0: float, x1: float, y0: float, y1: float,
                seed: int, inside=None, log=None, stiffen_time=4e-3, gap=4e-4):
    """A bed of `n_clumps` clumps of `base`'s templates (drawn uniformly),
    spawned on size-layered lattices over [x0, x1] x [y0, y1] (only the sites
    for which inside(x, y, bounding radius) holds, the lowest first), settled
    under gravity with soft preparation contacts at dt 5e-6 s, then run with
    `base`'s own materials and dt for `stiffen_time`; clumps numbered along a
    Morton curve.  `base.walls` must hold the clumps (the preparation uses
    them).  Returns a copy of `base` with the settled state."""
    rng = np.random.default_rng(seed)
    nt = len(base.tpl_mass)
    bound_t = base.bounding_radius()
    z0 = float(base.walls[0]["p"][2])  # the floor is the first wall
    spare = 1.0
    while True:
        m = int(n_clumps * spare) + 16
        tpl = rng.integers(0, nt, size=m).astype(np.int32)
        P = scenes.layered_positions(bound_t[tpl], x0, x1, y0, y1, z0, gap=gap, rng=rng,
                                     jitter=1e-4)
        keep = np.ones(m, bool) if inside is None else inside(P[:, 0], P[:, 1], bound_t[tpl] + gap)
        idx = np.nonzero(keep)[0]
        if len(idx) >= n_clumps:
            break
        spare *= 1.5
    idx = idx[np.argsort(P[idx, 2], kind="stable")][:n_clumps]
    P, tpl = P[idx], tpl[idx]
    soft = scenes.Scene(
        "prep", base.tpl_off, base.tpl_pos, base.tpl_rad, base.tpl_mat, base.tpl_mass,
        base.tpl_inertia, np.full(len(base.E), 5e7), np.full(len(base.E), 0.3),
        np.full(len(base.E), 0.5), np.full(len(base.E), 0.2), h=5e-6, g=base.g,
        lo=base.lo, hi=(base.hi[0], base.hi[1], float(P[:, 2].max()) + 0.05), bin_size=0.0,
        walls=[w for w in base.walls if np.allclose(w.get("vel", (0.0, 0.0, 0.0)), 0.0)],
        precision=scenes.PREC_FP32)
    soft.tpl, soft.pos = tpl, P
    soft.quat = scenes.random_quaternions(rng, n_clumps)
    soft.vel, soft.angvel = np.zeros((n_clumps, 3)), np.zeros((n_clumps, 3))
    fall = math.sqrt(2.0 * float(P[:, 2].max()) / 9.81)
    pos, quat, vel, angvel = settle(soft, fall + 0.15, log=log)
    soft.E, soft.nu, soft.mu, soft.cor, soft.h = base.E, base.nu, base.mu, base.cor, base.h
    soft.pos, soft.quat, soft.vel, soft.angvel = pos, quat, vel, angvel
    pos, quat, vel, angvel = settle(soft, stiffen_time, v_bound=2.0, K=20, log=log)
    perm = scenes.morton_order(pos, base.lo, 2.0 * float(bound_t.max()))
    out = dataclasses.replace(base)  # the dataclass fields (not attributes set on base)
    out.tpl, out.pos, out.quat = tpl[perm], pos[perm], quat[perm]
    out.vel, out.angvel = vel[perm], angvel[perm]
    out.hi = (base.hi[0], base.hi[1], max(base.hi[2], float(pos[:, 2].max()) + 0.05))
    return out


def insert_cone_mesh(sc: scenes.Scene, depth=0.005, nseg=32, nrings=9, speed=0.01,
                     half_angle_deg=30.0, base_diameter=0.02):
    """Adds an open cone of nseg (2 nrings - 1) facets (section 4's cone
    penetration test: 30 degree half angle, 2 cm base) whose tip sits `depth`
    below the bed's top at the centre of the bed's footprint, pushed down at
    `speed`; the clumps with a sphere centre inside the cone's side are taken
    out.  Returns the new scene (clump numbering kept in order)."""
    half = math.radians(half_angle_deg)
    H = 0.5 * base_diameter / math.tan(half)
    bound_t = sc.bounding_radius()
    top = float((sc.pos[:, 2] + bound_t[sc.tpl]).max())
    cx = 0.5 * (sc.lo[0] + sc.hi[0])
    cy = 0.5 * (sc.lo[1] + sc.hi[1])
    tip = np.array([cx, cy, top - depth])
    mesh = scenes.cone_mesh(tuple(tip), half, H, nseg, nrings, vel=(0.0, 0.0, -speed), base=False)
    # only clumps near the cone can reach inside it
    near = np.nonzero((np.abs(sc.pos[:, 0] - cx) < 0.5 * base_diameter + 0.02) &
                      (np.abs(sc.pos[:, 1] - cy) < 0.5 * base_diameter + 0.02) &
                      (sc.pos[:, 2] > tip[2] - 0.02))[0]
    keep = np.ones(len(sc.tpl), bool)
    for i in near:
        q = sc.quat[i]
        w, x, y, z = q
        R = np.array([[1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)],
                      [2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)],
                      [2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)]])
        s0, s1 = sc.tpl_off[sc.tpl[i]], sc.tpl_off[sc.tpl[i] + 1]
        xs = sc.pos[i] + sc.tpl_pos[s0:s1] @ R.T
        dz = xs[:, 2] - tip[2]
        side = (np.hypot(xs[:, 0] - cx, xs[:, 1] - cy) - dz * math.tan(half)) * math.cos(half)
        keep[i] = not ((dz > -5e-5) & (dz < H + 5e-5) & (side < 5e-5)).any()
    out = scenes.Scene(**{**sc.__dict__})
    for k in ("tpl", "pos", "quat", "vel", "angvel"):
        setattr(out, k, getattr(sc, k)[keep])
    out.walls = list(sc.walls) + mesh
    out.hi = (sc.hi[0], sc.hi[1], max(sc.hi[2], top + H + 0.01))
    return out


def repose_angle(xs, radii, centre, z_floor, bin_width, lo_frac=0.2, hi_frac=0.8, min_count=5):
    """Angle of repose of a heap [degrees] (section 4's angle-of-repose test):
    the heap's top surface h(rho) is the highest sphere top above the floor
    in each ring of width `bin_width` around the vertical axis through
    `centre`, over the rings from the axis outwards up to the first one that
    holds fewer than `min_count` spheres (grains scattered beyond the heap's
    toe are not part of its flank); a least-squares line h = a - b rho over
    those rings whose height lies between lo_frac and hi_frac of the apex
    height (the flank, without the rounded apex and the toe) gives the angle
    atan(b).  Returns (angle, apex height, rings used)."""
    xs = np.asarray(xs, float)
    top = xs[:, 2] + np.asarray(radii, float) - z_floor
    rho = np.hypot(xs[:, 0] - centre[0], xs[:, 1] - centre[1])
    k = np.floor(rho / bin_width).astype(np.int64)
    nb = int(k.max()) + 1
    h = np.full(nb, -np.inf)
    np.maximum.at(h, k, top)
    cnt = np.bincount(k, minlength=nb)
    short = np.nonzero(cnt < min_count)[0]
    end = int(short[0]) if len(short) else nb
    mid = (np.arange(nb) + 0.5) * bin_width
    ok = np.zeros(nb, bool)
    ok[:end] = True
    if not ok.any():
        raise ValueError("no ring near the axis holds enough spheres")
    hmax = float(h[ok].max())
    sel = ok & (h >= lo_frac * hmax) & (h <= hi_frac * hmax)
    if sel.sum() < 3:
        raise ValueError("too few rings on the heap's flank to fit a slope")
    b, a = np.polyfit(mid[sel], h[sel], 1)
    return math.degrees(math.atan(-b)), hmax, int(sel.sum())


def repose_column_scene(n_clumps, mu, seed=7, radius=0.04, height=0.12, nseg=32, E=1e7, h=1e-5):
    """The angle-of-repose set-up (section 4: a heap formed by grains flowing
    out of a container onto a flat plate; here the container is a tube of
    2 nseg facets, grains inside, standing on a floor at z = 0, which is
    lifted once the grains have settled in it: lift_walls).  n_clumps clumps
    of three overlapping 1-2 mm spheres (the first workload's templates) on
    a jittered lattice inside the tube, at rest.  Soft contacts (E, CoR 0.3)
    and friction mu; dt = h.  Returns (scene, wall ids of the tube)."""
    sc = scenes.config1(seed=seed, n_clumps=n_clumps, n_templates=20)
    sc.E, sc.nu, sc.mu, sc.cor = (np.array([E]), np.array([0.3]), np.array([mu]), np.array([0.3]))
    sc.h = h
    rng = np.random.default_rng(seed + 1)
    bound = float(sc.bounding_radius().max())
    sp = 2.0 * bound + 2e-4
    side = 2.0 * (radius - bound)
    P = scenes.lattice_positions(4 * n_clumps, sp, -0.5 * side, 0.5 * side, -0.5 * side,
                                 0.5 * side, 0.0, rng, 0.1 * sp)
    P = P[np.hypot(P[:, 0], P[:, 1]) <= radius - bound - 1e-4][:n_clumps]
    if len(P) < n_clumps or P[:, 2].max() + bound > height:
        raise ValueError("the tube does not hold that many clumps")
    sc.pos = P
    sc.quat = scenes.random_quaternions(rng, n_clumps)
    sc.vel, sc.angvel = np.zeros((n_clumps, 3)), np.zeros((n_clumps, 3))
    tube = scenes.funnel_mesh(0.0, 0.0, 0.0, height, radius, radius, nseg)
    sc.walls = [scenes.plane((0.0, 0.0, 0.0), (0, 0, 1))] + tube
    R = 0.2
    sc.lo = (-R, -R, -2.0 ** -9)
    sc.hi = (R, R, height + 0.05)
    sc.precision = scenes.PREC_FP32
    return sc, list(range(1, 1 + len(tube)))


def lift_walls(sim, scene: scenes.Scene, walls, vel):
    """Gives the walls `walls` of `scene` (as created, not moving before) the
    translation velocity `vel` from now on, through the co-simulation hook."""
    t = sim.stats()["time"]
    for k in walls:
        w = scene.walls[k]
        p = np.asarray(w["p"], float) + np.asarray(w.get("vel", (0.0, 0.0, 0.0)), float) * t
        sim.set_wall_motion(k, p, np.asarray(vel, float))


def sphere_centres(sc: scenes.Scene, pos, quat):
    """Sphere centres X + R(q) p and radii of every clump of a state (for
    measurements on the host, e.g. repose_angle); returns (centres, radii,
    owner clump of each sphere)."""
    pos, quat = np.asarray(pos, float), np.asarray(quat, float)
    w, x, y, z = (quat[:, k] for k in range(4))
    R = np.stack([1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y),
                  2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x),
                  2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)],
                 axis=1).reshape(-1, 3, 3)
    counts = np.diff(sc.tpl_off)[sc.tpl]
    owner = np.repeat(np.arange(len(sc.tpl)), counts)
    tsph = np.concatenate([np.arange(sc.tpl_off[t], sc.tpl_off[t + 1]) for t in sc.tpl]) \
        if len(sc.tpl) else np.zeros(0, np.int64)
    xs = pos[owner] + np.einsum("nij,nj->ni", R[owner], sc.tpl_pos[tsph])
    return xs, sc.tpl_rad[tsph], owner
