"""Seeded synthetic inputs: clump templates, materials, boundaries, initial states.

This module holds no arithmetic of the simulation method.  It only draws the
inputs that the paper's workloads are shaped like (section 3: clumps of 1-6
overlapping spheres with per-sphere E, nu, mu, CoR; section 4.1: beds spawned
on a lattice with gaps set by the largest clump).  Mass and principal inertia
of each clump template are properties of the input geometry (the union of its
spheres at the grain density); they are computed here once, by voxel
sampling, and handed identically to every consumer.

Every generator is deterministic for a given seed.
"""
from __future__ import annotations

from dataclasses import dataclass, field
import math

import numpy as np

DENSITY = 2600.0  # kg/m^3; the paper gives no grain density
WALL_PLANE, WALL_CYLINDER, WALL_CONE, WALL_TRIANGLE = 0, 1, 2, 3
PREC_FP64, PREC_FP32 = 0, 1


@dataclass
class Scene:
    name: str
    # clump templates
    tpl_off: np.ndarray
    tpl_pos: np.ndarray
    tpl_rad: np.ndarray
    tpl_mat: np.ndarray
    tpl_mass: np.ndarray
    tpl_inertia: np.ndarray
    # materials
    E: np.ndarray
    nu: np.ndarray
    mu: np.ndarray
    cor: np.ndarray
    # world
    h: float
    g: tuple
    lo: tuple
    hi: tuple
    bin_size: float
    walls: list = field(default_factory=list)
    mix_rule: int = 0
    precision: int = PREC_FP64
    # clumps
    tpl: np.ndarray = None
    pos: np.ndarray = None
    quat: np.ndarray = None
    vel: np.ndarray = None
    angvel: np.ndarray = None
    steps: int = 0
    seed: int = 0

    @property
    def n_clumps(self) -> int:
        return 0 if self.tpl is None else len(self.tpl)

    @property
    def n_spheres(self) -> int:
        counts = np.diff(self.tpl_off)
        return int(counts[self.tpl].sum())

    def sphere_counts(self):
        return np.diff(self.tpl_off)

    def bounding_radius(self):
        """Per-template radius of the bounding sphere about the CoM."""
        out = np.zeros(len(self.tpl_mass))
        for t in range(len(out)):
            s = slice(self.tpl_off[t], self.tpl_off[t + 1])
            out[t] = np.max(np.linalg.norm(self.tpl_pos[s], axis=1) + self.tpl_rad[s])
        return out

    def copy_state(self):
        return (self.pos.copy(), self.quat.copy(), self.vel.copy(), self.angvel.copy())


# ---------------------------------------------------------------------------
# clump templates
# ---------------------------------------------------------------------------
def _ball_points(rng, n, radius):
    v = rng.normal(size=(n, 3))
    v /= np.linalg.norm(v, axis=1, keepdims=True)
    r = radius * rng.random(n) ** (1.0 / 3.0)
    return v * r[:, None]


def union_mass_properties(centres, radii, density=DENSITY, cells=96):
    """Mass, centre of mass and inertia tensor of a union of spheres (voxel sampling)."""
    centres = np.asarray(centres, float)
    radii = np.asarray(radii, float)
    if len(radii) == 1:
        m = density * 4.0 / 3.0 * math.pi * radii[0] ** 3
        return m, centres[0].copy(), np.eye(3) * 0.4 * m * radii[0] ** 2
    lo = (centres - radii[:, None]).min(axis=0)
    hi = (centres + radii[:, None]).max(axis=0)
    dx = float((hi - lo).max()) / cells
    axes = [lo[k] + dx * (np.arange(int(math.ceil((hi[k] - lo[k]) / dx))) + 0.5) for k in range(3)]
    X, Y, Z = np.meshgrid(*axes, indexing="ij")
    P = np.stack([X.ravel(), Y.ravel(), Z.ravel()], axis=1)
    inside = np.zeros(len(P), bool)
    for c, r in zip(centres, radii):
        inside |= ((P - c) ** 2).sum(axis=1) <= r * r
    P = P[inside]
    dm = density * dx ** 3
    m = dm * len(P)
    com = P.mean(axis=0)
    Q = P - com
    r2 = (Q ** 2).sum(axis=1)
    I = dm * (np.eye(3) * r2.sum() - Q.T @ Q)
    return m, com, I


def make_template(rng, radii, spread, density=DENSITY, cells=96):
    """Component spheres with centres uniform in a ball of radius ``spread``,
    expressed in the principal frame about the union's centre of mass."""
    radii = np.asarray(radii, float)
    c = _ball_points(rng, len(radii), spread) if len(radii) > 1 else np.zeros((1, 3))
    m, com, I = union_mass_properties(c, radii, density, cells)
    w, V = np.linalg.eigh(I)
    if np.linalg.det(V) < 0:
        V[:, 0] = -V[:, 0]
    p = (c - com) @ V
    return p, radii, m, w


def _templates_from_lists(rng, radius_lists, spreads, n_mat, cells=96):
    off, pos, rad, mat, mass, inert = [0], [], [], [], [], []
    for radii, spread in zip(radius_lists, spreads):
        p, r, m, I = make_template(rng, radii, spread, cells=cells)
        pos.append(p)
        rad.append(r)
        mat.append(rng.integers(0, n_mat, size=len(r)))
        mass.append(m)
        inert.append(I)
        off.append(off[-1] + len(r))
    return (np.array(off, np.int32), np.concatenate(pos), np.concatenate(rad),
            np.concatenate(mat).astype(np.int32), np.array(mass), np.array(inert))


def random_quaternions(rng, n):
    """Uniform random unit quaternions (w, x, y, z)."""
    u1, u2, u3 = rng.random(n), rng.random(n), rng.random(n)
    a, b = np.sqrt(1 - u1), np.sqrt(u1)
    q = np.stack([a * np.sin(2 * math.pi * u2), a * np.cos(2 * math.pi * u2),
                  b * np.sin(2 * math.pi * u3), b * np.cos(2 * math.pi * u3)], axis=1)
    return q


def lognormal_radii(rng, n, median, sigma, lo, hi):
    return np.clip(median * np.exp(sigma * rng.normal(size=n)), lo, hi)


# ---------------------------------------------------------------------------
# boundaries
# ---------------------------------------------------------------------------
def plane(p, n, vel=(0.0, 0.0, 0.0), material=0):
    n = np.asarray(n, float)
    n = n / np.linalg.norm(n)
    return {"type": WALL_PLANE, "p": tuple(map(float, p)), "n": tuple(n), "vel": tuple(vel),
            "material": material}


def cylinder(p, axis, radius, material=0):
    a = np.asarray(axis, float)
    a = a / np.linalg.norm(a)
    return {"type": WALL_CYLINDER, "p": tuple(map(float, p)), "n": tuple(a), "radius": float(radius),
            "vel": (0.0, 0.0, 0.0), "material": material}


def cone(tip, axis, half_angle, height, vel=(0.0, 0.0, 0.0), material=0):
    a = np.asarray(axis, float)
    a = a / np.linalg.norm(a)
    return {"type": WALL_CONE, "p": tuple(map(float, tip)), "n": tuple(a),
            "half_angle": float(half_angle), "height": float(height), "vel": tuple(vel),
            "material": material}


def triangle(a, b, c, vel=(0.0, 0.0, 0.0), material=0):
    """One mesh facet; the grains are on the side of (b - a) x (c - a)."""
    a, b, c = (np.asarray(v, float) for v in (a, b, c))
    n = np.cross(b - a, c - a)
    n = n / np.linalg.norm(n)
    return {"type": WALL_TRIANGLE, "p": tuple(map(float, a)), "b": tuple(map(float, b)),
            "c": tuple(map(float, c)), "n": tuple(map(float, n)), "vel": tuple(vel),
            "material": material}


def mesh(vertices, faces, grains_at, vel=(0.0, 0.0, 0.0), material=0):
    """Facets of a triangle mesh, each oriented so that its normal points to
    the side of its plane where the point grains_at lies."""
    v = np.asarray(vertices, float)
    out = []
    for i, j, k in faces:
        a, b, c = v[i], v[j], v[k]
        if np.dot(np.cross(b - a, c - a), np.asarray(grains_at, float) - a) < 0:
            b, c = c, b
        out.append(triangle(a, b, c, vel=vel, material=material))
    return out


def box_mesh(x0, x1, y0, y1, z0, z1, material=0):
    """The six faces of a box as 12 facets, grains inside."""
    v = [(x, y, z) for z in (z0, z1) for y in (y0, y1) for x in (x0, x1)]
    quads = [(0, 1, 3, 2), (4, 5, 7, 6), (0, 1, 5, 4), (2, 3, 7, 6), (0, 2, 6, 4), (1, 3, 7, 5)]
    faces = [f for q in quads for f in ((q[0], q[1], q[2]), (q[0], q[2], q[3]))]
    centre = (0.5 * (x0 + x1), 0.5 * (y0 + y1), 0.5 * (z0 + z1))
    return mesh(v, faces, centre, material=material)


def funnel_mesh(cx, cy, z0, z1, r0, r1, nseg, material=0):
    """The side of a funnel (a frustum from radius r0 at height z0 to r1 at
    z1, open at both ends) as 2 nseg facets, grains inside."""
    ang = 2 * np.pi * np.arange(nseg) / nseg
    v = [(cx + r * np.cos(t), cy + r * np.sin(t), z) for z, r in ((z0, r0), (z1, r1)) for t in ang]
    faces = []
    for i in range(nseg):
        j = (i + 1) % nseg
        faces += [(i, j, nseg + j), (i, nseg + j, nseg + i)]
    out = []
    for f in faces:
        # orient towards the axis at the facet's own height
        zc = np.mean([v[k][2] for k in f])
        out.append(mesh(v, [f], (cx, cy, zc), material=material)[0])
    return out


def cone_mesh(tip, half_angle, height, nseg, nrings, vel=(0.0, 0.0, 0.0), material=0, base=True):
    """A cone with its tip at `tip`, its axis along +z and its flat base
    (radius height * tan(half_angle)) at tip + height, as facets with the
    grains outside: nseg around, nrings bands along the side (a fan at the
    tip), and (base=True) a fan of nseg over the base; nseg (2 nrings - 1)
    side facets plus nseg base facets."""
    tx, ty, tz = (float(v) for v in tip)
    rb = height * math.tan(half_angle)
    ang = 2 * np.pi * np.arange(nseg) / nseg
    ring = lambda k: [(tx + rb * k / nrings * np.cos(t), ty + rb * k / nrings * np.sin(t),
                       tz + height * k / nrings) for t in ang]
    v = [(tx, ty, tz)]
    for k in range(1, nrings + 1):
        v += ring(k)
    base_c = len(v)
    v.append((tx, ty, tz + height))
    at = lambda k, i: 1 + (k - 1) * nseg + (i % nseg)  # vertex i of ring k >= 1
    side = [(0, at(1, i), at(1, i + 1)) for i in range(nseg)]
    for k in range(1, nrings):
        for i in range(nseg):
            side += [(at(k, i), at(k + 1, i), at(k + 1, i + 1)), (at(k, i), at(k + 1, i + 1), at(k, i + 1))]
    out = []
    vv = np.asarray(v, float)
    for f in side:
        c = vv[list(f)].mean(axis=0)
        outward = c + np.array([c[0] - tx, c[1] - ty, 0.0])  # radially away from the axis
        out.append(mesh(v, [f], outward, vel=vel, material=material)[0])
    for i in range(nseg if base else 0):
        out.append(mesh(v, [(base_c, at(nrings, i), at(nrings, i + 1))],
                        (tx, ty, tz + 2.0 * height), vel=vel, material=material)[0])
    return out


def box_walls(x0, x1, y0, y1, z0, top=None, top_vel=(0.0, 0.0, 0.0)):
    w = [plane((0, 0, z0), (0, 0, 1)), plane((x0, 0, 0), (1, 0, 0)), plane((x1, 0, 0), (-1, 0, 0)),
         plane((0, y0, 0), (0, 1, 0)), plane((0, y1, 0), (0, -1, 0))]
    if top is not None:
        w.append(plane((0, 0, top), (0, 0, -1), vel=top_vel))
    return w


# ---------------------------------------------------------------------------
# placement
# ---------------------------------------------------------------------------
def lattice_positions(n, spacing, x0, x1, y0, y1, z0, rng=None, jitter=0.0):
    """n sites filling x fastest, then y, then z upward, starting at z0."""
    nx = max(1, int((x1 - x0) // spacing))
    ny = max(1, int((y1 - y0) // spacing))
    i = np.arange(n)
    ix, iy, iz = i % nx, (i // nx) % ny, i // (nx * ny)
    P = np.stack([x0 + (ix + 0.5) * spacing, y0 + (iy + 0.5) * spacing,
                  z0 + (iz + 0.5) * spacing], axis=1)
    if rng is not None and jitter > 0:
        P += rng.uniform(-jitter, jitter, size=P.shape)
    return P


def layered_positions(bound, x0, x1, y0, y1, z0, gap=2e-4, rng=None, jitter=0.0):
    """Spawn sites for clumps of bounding radii ``bound``: clumps sorted from
    the largest, filled layer by layer on square lattices whose spacing is set
    by the largest clump of the layer (the paper's batch spawning with gaps
    set by the largest element, applied per size class).  Returns positions in
    the input order."""
    bound = np.asarray(bound, float)
    order = np.argsort(-bound, kind="stable")
    P = np.zeros((len(bound), 3))
    i, z = 0, z0
    while i < len(order):
        s = 2.0 * bound[order[i]] + gap
        nx = max(1, int((x1 - x0) // s))
        ny = max(1, int((y1 - y0) // s))
        k = min(nx * ny, len(order) - i)
        idx = order[i:i + k]
        j = np.arange(k)
        P[idx, 0] = x0 + (j % nx + 0.5) * s
        P[idx, 1] = y0 + (j // nx + 0.5) * s
        P[idx, 2] = z + 0.5 * s
        if rng is not None and jitter > 0:
            P[idx, :2] += rng.uniform(-jitter, jitter, size=(k, 2))
        z += s
        i += k
    return P


def morton_order(pos, lo, cell):
    """Permutation that sorts points along a Z-order (Morton) curve of cells
    of edge ``cell`` from corner ``lo`` (21 bits per axis): neighbours in space
    get nearby indices, so their records share cache lines."""
    q = np.floor((np.asarray(pos, float) - np.asarray(lo, float)) / cell).astype(np.int64)
    q = np.clip(q, 0, (1 << 21) - 1).astype(np.uint64)
    key = np.zeros(len(q), np.uint64)
    for bit in range(21):
        for k in range(3):
            key |= ((q[:, k] >> np.uint64(bit)) & np.uint64(1)) << np.uint64(3 * bit + k)
    return np.argsort(key, kind="stable")


def _finish(sc: Scene, rng, pos, tpl, vel_scale=0.0, ang_scale=0.0):
    n = len(tpl)
    sc.tpl = np.asarray(tpl, np.int32)
    sc.pos = np.asarray(pos, float)
    sc.quat = random_quaternions(rng, n)
    sc.vel = rng.normal(scale=vel_scale, size=(n, 3)) if vel_scale > 0 else np.zeros((n, 3))
    sc.angvel = rng.normal(scale=ang_scale, size=(n, 3)) if ang_scale > 0 else np.zeros((n, 3))
    return sc


def default_bin_size(sc: Scene, margin: float) -> float:
    return 2.0 * (float(np.max(sc.tpl_rad)) + margin)


# ---------------------------------------------------------------------------
# the five workload shapes
# ---------------------------------------------------------------------------
def config1(seed=1235, n_clumps=1000, n_templates=None):
    """1,000 clumps of 3 overlapping spheres (r ~ U(1, 2) mm, centres within
    1 mm of the CoM), one material (E 1e8, nu 0.3, mu 0.5, CoR 0.5), settling
    in a 5 x 5 x 10 cm box of planes, dt 1e-6 s, FP64."""
    rng = np.random.default_rng(seed)
    nt = n_clumps if n_templates is None else n_templates
    radii = [rng.uniform(1e-3, 2e-3, size=3) for _ in range(nt)]
    off, pos, rad, mat, mass, inert = _templates_from_lists(rng, radii, [1e-3] * nt, 1)
    sc = Scene("c1", off, pos, rad, mat, mass, inert, np.array([1e8]), np.array([0.3]),
               np.array([0.5]), np.array([0.5]), h=1e-6, g=(0.0, 0.0, -9.81),
               lo=(-0.005, -0.005, -0.005), hi=(0.055, 0.055, 0.155), bin_size=0.0,
               walls=box_walls(0.0, 0.05, 0.0, 0.05, 0.0), precision=PREC_FP64, steps=1000,
               seed=seed)
    bound = 2.0 * sc.bounding_radius().max() + 0.4e-3
    tpl = np.arange(n_clumps) % nt
    P = lattice_positions(n_clumps, bound, 0.0, 0.05, 0.0, 0.05, 0.0, rng, 0.2e-3)
    _finish(sc, rng, P, tpl)
    return sc


def polydisperse_templates(rng, n_templates, counts, median, sigma, rmin, rmax, n_mat, cells=96):
    radius_lists = [lognormal_radii(rng, int(k), median, sigma, rmin, rmax) for k in counts]
    spreads = [0.8 * float(np.mean(r)) for r in radius_lists]
    return _templates_from_lists(rng, radius_lists, spreads, n_mat, cells)


def four_materials(rng):
    E = np.array([5e7, 1e8, 5e8, 1e9])
    nu = np.full(4, 0.3)
    mu = rng.uniform(0.3, 0.8, size=4)
    cor = rng.uniform(0.2, 0.8, size=4)
    return E, nu, mu, cor


def config2(seed=1236, n_clumps=200_000, footprint=0.25):
    """200,000 clumps from 20 templates of U{1..5} spheres (r lognormal, median
    1.5 mm, sigma 0.4, clipped 0.5-5 mm), 4 materials per sphere, box settling,
    FP32 forces with voxel positions."""
    rng = np.random.default_rng(seed)
    counts = rng.integers(1, 6, size=20)
    off, pos, rad, mat, mass, inert = polydisperse_templates(rng, 20, counts, 1.5e-3, 0.4,
                                                             0.5e-3, 5e-3, 4)
    E, nu, mu, cor = four_materials(rng)
    sc = Scene("c2", off, pos, rad, mat, mass, inert, E, nu, mu, cor, h=1e-6,
               g=(0.0, 0.0, -9.81), lo=(0.0, 0.0, 0.0), hi=(footprint, footprint, 1.0),
               bin_size=0.0, walls=box_walls(0.0, footprint, 0.0, footprint, 0.0),
               precision=PREC_FP32, steps=20_000, seed=seed)
    spacing = 2.0 * sc.bounding_radius().max() + 0.4e-3
    tpl = rng.integers(0, 20, size=n_clumps)
    P = lattice_positions(n_clumps, spacing, 0.0, footprint, 0.0, footprint, 0.0, rng, 0.2e-3)
    height = P[:, 2].max() + spacing
    sc.hi = (footprint, footprint, max(1.0, height))
    _finish(sc, rng, P, tpl)
    return sc


def config5_templates(rng):
    """30 templates of 1-6 spheres with a mean of about 3.1 spheres."""
    weights = np.array([0.12, 0.18, 0.30, 0.18, 0.12, 0.10])
    counts = rng.choice(np.arange(1, 7), size=30, p=weights)
    return counts


def config5(seed=1239, n_clumps=11_000_000, lx=4.0, ly=2.0, lz=0.3, plate_speed=0.2):
    """Paper-scale bed: 11,000,000 clumps from 30 templates of 1-6 spheres (r
    lognormal, median 2 mm, sigma 0.4, clipped 0.5-6 mm), 4 materials, a
    4 x 2 x 0.3 m box with a flat rigid plate sliding at 0.2 m/s on top."""
    rng = np.random.default_rng(seed)
    counts = config5_templates(rng)
    off, pos, rad, mat, mass, inert = polydisperse_templates(rng, 30, counts, 2e-3, 0.4,
                                                             0.5e-3, 6e-3, 4)
    E, nu, mu, cor = four_materials(rng)
    sc = Scene("c5", off, pos, rad, mat, mass, inert, E, nu, mu, cor, h=1e-6,
               g=(0.0, 0.0, -9.81), lo=(0.0, 0.0, 0.0), hi=(lx, ly, lz), bin_size=0.0,
               walls=box_walls(0.0, lx, 0.0, ly, 0.0, top=lz, top_vel=(plate_speed, 0.0, 0.0)),
               precision=PREC_FP32, steps=5000, seed=seed)
    sc.tpl = rng.integers(0, 30, size=n_clumps).astype(np.int32)
    return sc


def config3(seed=1237, n_clumps=1_000_000, radius=0.2, n_templates=100):
    """Clumps as in the first workload settling into a cylinder of radius
    0.2 m, with an analytic cone (30 degree half angle, 2 cm base) pushed down
    at 1 cm/s; FP32 forces / FP64 integration."""
    rng = np.random.default_rng(seed)
    radii = [rng.uniform(1e-3, 2e-3, size=3) for _ in range(n_templates)]
    off, pos, rad, mat, mass, inert = _templates_from_lists(rng, radii, [1e-3] * n_templates, 1)
    half = math.radians(30.0)
    cone_h = 0.01 / math.tan(half)
    sc = Scene("c3", off, pos, rad, mat, mass, inert, np.array([1e8]), np.array([0.3]),
               np.array([0.5]), np.array([0.5]), h=1e-6, g=(0.0, 0.0, -9.81),
               lo=(-radius, -radius, 0.0), hi=(radius, radius, 1.0), bin_size=0.0,
               walls=[plane((0, 0, 0), (0, 0, 1)), cylinder((0, 0, 0), (0, 0, 1), radius)],
               precision=PREC_FP32, steps=50_000, seed=seed)
    sc.cone = cone((0.0, 0.0, 0.0), (0, 0, 1), half, cone_h, vel=(0.0, 0.0, -0.01))
    sc.tpl = (np.arange(n_clumps) % n_templates).astype(np.int32)
    return sc


def config4_scene_sizes(seed=1238, n_scenes=64, lo=5_000, hi=100_000):
    rng = np.random.default_rng(seed)
    return np.round(np.exp(rng.uniform(math.log(lo), math.log(hi), size=n_scenes))).astype(np.int64)


def config4(seed=1238, n_scenes=64, lo=5_000, hi=100_000):
    """The batched sensitivity sweep: n_scenes independent box-settling scenes
    of log-uniform size, each with its own friction coefficient and template
    set, merged into one template / material table (merge_batch)."""
    rng = np.random.default_rng(seed)
    sizes = config4_scene_sizes(seed, n_scenes, lo, hi)
    mus = rng.uniform(0.2, 0.9, size=n_scenes)
    return [batched_scene(seed * 1000 + i, int(n), float(mu)) for i, (n, mu) in enumerate(zip(sizes, mus))]


def merge_batch(parts):
    """Scenes with their own templates and materials -> (first, rest) for one
    context: `first` carries the concatenated template and material tables,
    and the clumps and walls of every scene refer to them through shifted
    ids.  All scenes must share dt, g and precision."""
    first = parts[0]
    for p in parts[1:]:
        if p.h != first.h or tuple(p.g) != tuple(first.g) or p.precision != first.precision:
            raise ValueError("batched scenes must share dt, g and precision")
    off, pos, rad, mat, mass, inert = [np.zeros(1, np.int32)], [], [], [], [], []
    E, nu, mu, cor = [], [], [], []
    t_base, s_base, m_base = 0, 0, 0
    out = []
    for p in parts:
        off.append(np.asarray(p.tpl_off[1:], np.int32) + s_base)
        pos.append(p.tpl_pos)
        rad.append(p.tpl_rad)
        mat.append(np.asarray(p.tpl_mat, np.int32) + m_base)
        mass.append(p.tpl_mass)
        inert.append(p.tpl_inertia)
        E.append(p.E); nu.append(p.nu); mu.append(p.mu); cor.append(p.cor)
        q = Scene(**{**p.__dict__})
        q.tpl = np.asarray(p.tpl, np.int32) + t_base
        # a wall's material is an index into its own scene's table too
        q.walls = [dict(w, material=int(w.get("material", 0)) + m_base) for w in p.walls]
        out.append(q)
        t_base += len(p.tpl_mass)
        s_base += int(p.tpl_off[-1])
        m_base += len(p.E)
    tables = dict(tpl_off=np.concatenate(off), tpl_pos=np.concatenate(pos),
                  tpl_rad=np.concatenate(rad), tpl_mat=np.concatenate(mat),
                  tpl_mass=np.concatenate(mass), tpl_inertia=np.concatenate(inert),
                  E=np.concatenate(E), nu=np.concatenate(nu), mu=np.concatenate(mu),
                  cor=np.concatenate(cor))
    for q in out:
        for k, v in tables.items():
            setattr(q, k, v)
    return out[0], out[1:]


def batched_scene(seed, n_clumps, mu):
    """One scene of the batched sensitivity sweep: its own friction coefficient
    and template set of U{1..5} spheres, box footprint proportional to sqrt(N)."""
    rng = np.random.default_rng(seed)
    counts = rng.integers(1, 6, size=10)
    # coarser voxel sampling of the template mass properties (64 scenes x 10
    # templates); the values are inputs, shared by every consumer
    off, pos, rad, mat, mass, inert = polydisperse_templates(rng, 10, counts, 1.5e-3, 0.4,
                                                             0.5e-3, 5e-3, 1, cells=48)
    spacing = 0.0
    foot = 0.0
    sc = Scene("c4", off, pos, rad, mat, mass, inert, np.array([1e8]), np.array([0.3]),
               np.array([mu]), np.array([0.5]), h=1e-6, g=(0.0, 0.0, -9.81),
               lo=(0.0, 0.0, 0.0), hi=(1.0, 1.0, 1.0), bin_size=0.0, walls=[],
               precision=PREC_FP32, steps=10_000, seed=seed)
    spacing = 2.0 * sc.bounding_radius().max() + 0.4e-3
    foot = spacing * math.ceil(math.sqrt(n_clumps / 10.0))  # about 10 layers deep
    P = lattice_positions(n_clumps, spacing, 0.0, foot, 0.0, foot, 0.0, rng, 0.2e-3)
    sc.walls = box_walls(0.0, foot, 0.0, foot, 0.0)
    sc.hi = (foot, foot, P[:, 2].max() + spacing)
    tpl = rng.integers(0, 10, size=n_clumps)
    _finish(sc, rng, P, tpl)
    return sc


# ---------------------------------------------------------------------------
# small dense scenes for parity tests
# ---------------------------------------------------------------------------
def packed_scene(seed, n_clumps, precision=PREC_FP64, compress=0.92, n_templates=8,
                 vel_scale=0.05, ang_scale=20.0, n_mat=3, walls=True, jitter=0.15):
    """A small lattice of polydisperse clumps squeezed below their bounding
    diameter, so that many sphere pairs overlap by a spread of depths, with
    random linear and angular velocities and several materials."""
    rng = np.random.default_rng(seed)
    counts = rng.integers(1, 6, size=n_templates)
    off, pos, rad, mat, mass, inert = polydisperse_templates(rng, n_templates, counts, 1.5e-3,
                                                             0.4, 0.5e-3, 4e-3, n_mat)
    E = np.array([5e7, 1e8, 5e8, 1e9][:n_mat])
    nu = np.array([0.3, 0.25, 0.35, 0.3][:n_mat])
    mu = rng.uniform(0.2, 0.8, size=n_mat)
    cor = rng.uniform(0.2, 0.9, size=n_mat)
    sc = Scene("packed", off, pos, rad, mat, mass, inert, E, nu, mu, cor, h=1e-6,
               g=(0.0, 0.0, -9.81), lo=(0.0, 0.0, 0.0), hi=(1.0, 1.0, 1.0), bin_size=0.0,
               precision=precision, seed=seed)
    bound = sc.bounding_radius()
    tpl = rng.integers(0, n_templates, size=n_clumps)
    spacing = compress * 2.0 * float(np.mean(bound[tpl]))
    side = spacing * math.ceil(n_clumps ** (1.0 / 3.0))
    P = lattice_positions(n_clumps, spacing, 0.0, side, 0.0, side, 0.0, rng, jitter * spacing)
    P += 0.01
    sc.lo = (0.0, 0.0, 0.0)
    top = float(P[:, 2].max()) + 0.02
    sc.hi = (side + 0.02, side + 0.02, top)
    if walls:
        zf = float(P[:, 2].min()) - 0.5 * spacing
        sc.walls = box_walls(0.01 - 0.3 * spacing, 0.01 + side + 0.3 * spacing,
                             0.01 - 0.3 * spacing, 0.01 + side + 0.3 * spacing, zf)
    _finish(sc, rng, P, tpl, vel_scale, ang_scale)
    return sc


# ---------------------------------------------------------------------------
# snapping an FP64 state onto the FP32 voxel representation
# ---------------------------------------------------------------------------
def snap_to_voxel_grid(sc: Scene, voxel_log2=20, offset_bits=44):
    """Round positions to multiples of 2^-offset_bits m relative to the domain
    corner and orientations to float32, so that the same state is exactly
    representable both in FP64 and as (int voxel, float offset, float quat)."""
    q = 2.0 ** -offset_bits
    lo = np.asarray(sc.lo)
    if not np.all(np.round(lo / q) * q == lo):
        raise ValueError("domain corner must lie on the offset grid")
    sc.pos = lo + np.round((sc.pos - lo) / q) * q
    qf = sc.quat.astype(np.float32)
    qf = qf / np.linalg.norm(qf.astype(np.float64), axis=1, keepdims=True).astype(np.float32)
    sc.quat = qf.astype(np.float64)
    return sc
