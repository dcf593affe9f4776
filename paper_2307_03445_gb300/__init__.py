"""GB300 clump-of-spheres DEM (arXiv 2307.03445 hot path) -- Python binding.

The binding marshals numpy arrays and torch device pointers into the C ABI of
libdem.so (include/dem.h); every step of the method runs in the CUDA kernels.

    from paper_2307_03445_gb300 import Simulation, scenes
    sc = scenes.config1()
    sim = Simulation(sc, margin=5e-5, rebuild_interval=10)
    sim.step(1000)
    pos, quat, vel, angvel = sim.state()
"""
from __future__ import annotations

import ctypes as C

import numpy as np

from . import capi
from .capi import (DEM_FP32_VOXEL, DEM_FP64, DEM_GUARD_COUNT, DEM_GUARD_OFF,
                   DEM_GUARD_ROLLBACK, DemError)

__all__ = ["Simulation", "Regressor", "DemError", "DEM_FP64", "DEM_FP32_VOXEL", "DEM_GUARD_OFF",
           "DEM_GUARD_COUNT", "DEM_GUARD_ROLLBACK", "load_library"]


def load_library():
    return capi.load()


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _i32(a):
    return np.ascontiguousarray(a, dtype=np.int32)


def _pd(a):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _pi(a):
    return a.ctypes.data_as(C.POINTER(C.c_int))


def walls_to_c(walls, scene_of=None):
    arr = (capi.DemWall * max(1, len(walls)))()
    for i, w in enumerate(walls):
        arr[i].type = int(w["type"])
        arr[i].material = int(w.get("material", 0))
        for k in range(3):
            arr[i].p[k] = float(w["p"][k])
            arr[i].n[k] = float(w["n"][k])
            arr[i].vel[k] = float(w.get("vel", (0.0, 0.0, 0.0))[k])
            arr[i].b[k] = float(w.get("b", (0.0, 0.0, 0.0))[k])
            arr[i].c[k] = float(w.get("c", (0.0, 0.0, 0.0))[k])
        arr[i].radius = float(w.get("radius", 0.0))
        arr[i].half_angle = float(w.get("half_angle", 0.0))
        arr[i].height = float(w.get("height", 0.0))
        arr[i].scene = int(w.get("scene", -1)) if scene_of is None else int(scene_of[i])
    return arr


class Simulation:
    """One context of libdem.so holding one or more scenes.

    scene: a ``scenes.Scene`` (templates, materials, walls, world, clumps).
    margin: enlargement of every sphere for the contact list [m]; if None,
        v_bound * dt * rebuild_interval.
    extra_scenes: further Scene objects sharing templates/materials/dt/g with
        the first one (batched independent systems).
    allocator: optional (alloc, free) Python callables for the context's
        device memory: alloc(nbytes) -> device address (256-byte aligned),
        free(address); None = the library's stream-ordered allocator.
    """

    def __init__(self, scene, margin=None, rebuild_interval=10, v_bound=0.5, precision=None,
                 guard=DEM_GUARD_COUNT, device=0, stream=None, bin_size=None, max_contacts=0,
                 extra_scenes=(), extra_walls=(), allocator=None):
        self.lib = capi.load()
        self.scene = scene
        prec = scene.precision if precision is None else precision
        self._keep = []
        p = capi.DemParams()
        p.dt = float(scene.h)
        for k in range(3):
            p.g[k] = float(scene.g[k])
            p.domain_lo[k] = float(scene.lo[k])
            p.domain_hi[k] = float(scene.hi[k])
        p.precision = int(prec)
        p.bin_size = float(bin_size if bin_size is not None else (scene.bin_size or 0.0))
        p.margin_policy = 0
        p.rebuild_interval = int(rebuild_interval)
        p.v_bound = float(v_bound)
        p.margin = float(margin) if margin is not None else 0.0
        p.mix_rule = int(getattr(scene, "mix_rule", 0))
        mats = [_f64(getattr(scene, k)) for k in ("E", "nu", "mu", "cor")]
        self._keep += mats
        p.n_materials = len(mats[0])
        p.E, p.nu, p.mu, p.cor = (_pd(m) for m in mats)
        walls = [dict(w, scene=0) for w in scene.walls]
        for si, sc2 in enumerate(extra_scenes, start=1):
            walls += [dict(w, scene=si) for w in sc2.walls]
        walls += list(extra_walls)
        warr = walls_to_c(walls)
        self._keep.append(warr)
        p.n_walls = len(walls)
        p.walls = C.cast(warr, C.POINTER(capi.DemWall))
        p.max_contacts = int(max_contacts)
        p.guard = int(guard)
        p.cuda_stream = stream
        p.device = int(device)
        if allocator is not None:
            a_fn, f_fn = allocator
            p.alloc = capi.ALLOC_FN(lambda n, user: a_fn(int(n)))
            p.free = capi.FREE_FN(lambda ptr, user: f_fn(int(ptr)))
            self._keep += [p.alloc, p.free]  # the callbacks must outlive the context
        ctx = C.c_void_p()
        rc = self.lib.dem_create(C.byref(p), C.byref(ctx))
        if rc != 0:
            raise DemError(rc, self.lib.dem_last_error(None).decode())
        self.ctx = ctx
        self._check(self.lib.dem_load_clump_templates(
            ctx, len(scene.tpl_mass), _pi(_i32(scene.tpl_off)), _pd(_f64(scene.tpl_pos).reshape(-1)),
            _pd(_f64(scene.tpl_rad)), _pi(_i32(scene.tpl_mat)), _pd(_f64(scene.tpl_mass)),
            _pd(_f64(scene.tpl_inertia).reshape(-1))))
        self.n_walls = len(walls)
        self.scene_ids = [0]
        for sc2 in extra_scenes:
            sid = C.c_int()
            lo, hi = _f64(sc2.lo), _f64(sc2.hi)
            self._check(self.lib.dem_add_scene(ctx, _pd(lo), _pd(hi),
                                               float(sc2.bin_size or p.bin_size), C.byref(sid)))
            self.scene_ids.append(sid.value)
        self.n = 0
        if scene.tpl is not None and len(scene.tpl):
            self.add_clumps(scene.tpl, scene.pos, scene.quat, scene.vel, scene.angvel, 0)
        for sid, sc2 in zip(self.scene_ids[1:], extra_scenes):
            self.add_clumps(sc2.tpl, sc2.pos, sc2.quat, sc2.vel, sc2.angvel, sid)

    # ------------------------------------------------------------------
    def _check(self, rc):
        if rc != 0:
            raise DemError(rc, self.lib.dem_last_error(self.ctx).decode())

    def add_clumps(self, tpl, pos, quat, vel, angvel, scene=0):
        tpl = _i32(tpl)
        arr = [_f64(a) for a in (pos, quat, vel, angvel)]
        self._check(self.lib.dem_add_clumps(self.ctx, len(tpl), _pi(tpl), *(_pd(a) for a in arr),
                                            int(scene)))
        self.n += len(tpl)

    def step(self, n=1):
        self._check(self.lib.dem_step(self.ctx, int(n)))

    def state(self, out=None):
        """(pos, quat, vel, angvel) as float64 host arrays; `out` may give four
        C-contiguous float64 arrays of shapes (n,3), (n,4), (n,3), (n,3) to
        fill (e.g. views of pinned host memory)."""
        n = self.n
        if out is None:
            out = [np.zeros((n, 3)), np.zeros((n, 4)), np.zeros((n, 3)), np.zeros((n, 3))]
        for o, w in zip(out, (3, 4, 3, 3)):
            if o.dtype != np.float64 or o.shape != (n, w) or not o.flags.c_contiguous:
                raise ValueError("state(out=...) wants C-contiguous float64 arrays of the state's shapes")
        self._check(self.lib.dem_get_state(self.ctx, *(o.ctypes.data for o in out), 0))
        return tuple(out)

    def state_device(self, pos, quat, vel, angvel):
        """Writes the state into device buffers (e.g. torch CUDA tensors, float64)."""
        ptrs = [t.data_ptr() if t is not None else None for t in (pos, quat, vel, angvel)]
        self._check(self.lib.dem_get_state(self.ctx, *ptrs, 1))

    def set_state(self, pos, quat, vel, angvel):
        arr = [_f64(a) for a in (pos, quat, vel, angvel)]
        self._check(self.lib.dem_set_state(self.ctx, *(_pd(a) for a in arr)))

    def rebuild(self):
        self._check(self.lib.dem_rebuild(self.ctx))

    def eval_forces(self):
        self._check(self.lib.dem_eval_forces(self.ctx))
        F, T = np.zeros((self.n, 3)), np.zeros((self.n, 3))
        self._check(self.lib.dem_get_forces(self.ctx, _pd(F), _pd(T)))
        return F, T

    def wall_forces(self):
        F = np.zeros((max(1, self.n_walls), 3))
        self._check(self.lib.dem_get_wall_forces(self.ctx, _pd(F)))
        return F[: self.n_walls]

    def wall_loads(self):
        """(force, moment about the wall's reference point) per wall, from the
        last force evaluation."""
        F = np.zeros((max(1, self.n_walls), 3))
        T = np.zeros((max(1, self.n_walls), 3))
        self._check(self.lib.dem_get_wall_loads(self.ctx, _pd(F), _pd(T)))
        return F[: self.n_walls], T[: self.n_walls]

    def set_wall_motion(self, wall, point, vel):
        """From now on wall `wall` moves as point + vel * (t' - t_now)."""
        p, v = _f64(point), _f64(vel)
        if p.shape != (3,) or v.shape != (3,):
            raise ValueError("point and vel are 3-vectors")
        self._check(self.lib.dem_set_wall_motion(self.ctx, int(wall), _pd(p), _pd(v)))

    def contacts(self):
        npair, nw = C.c_longlong(), C.c_longlong()
        self._check(self.lib.dem_num_contacts(self.ctx, C.byref(npair), C.byref(nw)))
        a, b = np.zeros(npair.value, np.int32), np.zeros(npair.value, np.int32)
        u = np.zeros((npair.value, 3))
        ws, ww = np.zeros(nw.value, np.int32), np.zeros(nw.value, np.int32)
        uw = np.zeros((nw.value, 3))
        self._check(self.lib.dem_get_contacts(self.ctx, _pi(a), _pi(b), _pd(u), _pi(ws), _pi(ww),
                                              _pd(uw)))
        return a, b, u, ws, ww, uw

    def bins(self):
        n = C.c_longlong()
        self._check(self.lib.dem_get_bins(self.ctx, 0, None, None, C.byref(n)))
        keys, ids = np.zeros(n.value, np.uint32), np.zeros(n.value, np.int32)
        self._check(self.lib.dem_get_bins(self.ctx, n.value,
                                          keys.ctypes.data_as(C.POINTER(C.c_uint)), _pi(ids),
                                          C.byref(n)))
        return keys, ids

    def audit(self):
        m = C.c_longlong()
        self._check(self.lib.dem_audit(self.ctx, C.byref(m)))
        return m.value

    def stats(self):
        s = capi.DemStats()
        self._check(self.lib.dem_get_stats(self.ctx, C.byref(s)))
        return {k: getattr(s, k) for k, _ in capi.DemStats._fields_}

    def reset_stats(self):
        self._check(self.lib.dem_reset_stats(self.ctx))

    def set_timing(self, on=True):
        self._check(self.lib.dem_set_timing(self.ctx, 1 if on else 0))

    def autotune_bins(self, factors=(0.35, 0.5, 0.7, 1.0, 1.5), reps=2):
        """Times rebuilds at each bin-edge factor and keeps the fastest.
        Returns (best factor, {factor: mean rebuild ms or None})."""
        f = _f64(factors)
        ms = np.zeros(len(f))
        best = C.c_double()
        self._check(self.lib.dem_autotune_bins(self.ctx, len(f), _pd(f), int(reps), C.byref(best),
                                               _pd(ms)))
        return best.value, {float(a): (float(b) if b >= 0 else None) for a, b in zip(f, ms)}

    def tiles(self):
        """Launch shapes: {pairs_blocks_per_sm, update_block, narrow_chunk}."""
        t = capi.DemTiles()
        self._check(self.lib.dem_get_tiles(self.ctx, C.byref(t)))
        return {k: getattr(t, k) for k, _ in capi.DemTiles._fields_}

    def set_tiles(self, **kw):
        """Sets some launch shapes (the others keep their values)."""
        cur = self.tiles()
        unknown = set(kw) - set(cur)
        if unknown:
            raise ValueError(f"unknown launch shapes {sorted(unknown)}")
        cur.update(kw)
        t = capi.DemTiles(**{k: int(v) for k, v in cur.items()})
        self._check(self.lib.dem_set_tiles(self.ctx, C.byref(t)))

    def autotune_tiles(self, steps=10, reps=2):
        """Times the launch shapes one at a time and keeps the fastest; the
        state is unchanged.  Returns the chosen shapes."""
        t = capi.DemTiles()
        self._check(self.lib.dem_autotune_tiles(self.ctx, int(steps), int(reps), C.byref(t)))
        return {k: getattr(t, k) for k, _ in capi.DemTiles._fields_}

    def set_deterministic(self, on=True):
        """Bit-reproducible force sums (per-contact slots summed in a fixed order)."""
        self._check(self.lib.dem_set_deterministic(self.ctx, 1 if on else 0))

    def set_outer_list(self, factor=3.0, n_inner=4, async_detect=False):
        """Two-level contact list (see include/dem.h): an outer list at factor x
        the margin serves the next n_inner rebuilds; n_inner=0 turns it off.
        async_detect builds the next outer list on a second stream while the
        steps run."""
        self._check(self.lib.dem_set_outer_list(self.ctx, float(factor), int(n_inner),
                                                1 if async_detect else 0))

    def set_graphs(self, on=True):
        """Run the steps between rebuilds as one captured CUDA graph."""
        self._check(self.lib.dem_set_graphs(self.ctx, 1 if on else 0))

    def set_learned_policy(self, regressor, interval=40, safety=1.5, candidates=None,
                           mode=capi.DEM_LEARNED_HALT, speed_floor=0.0):
        """Learned rebuild rule (see include/dem.h); regressor=None restores the plain rule."""
        if regressor is None:
            self._check(self.lib.dem_set_learned_policy(self.ctx, None, None))
            self._regressor = None
            return
        cand = _f64(candidates)
        self._cand = cand
        lp = capi.DemLearnedParams(int(interval), float(safety), len(cand), _pd(cand), int(mode),
                                   float(speed_floor))
        self._check(self.lib.dem_set_learned_policy(self.ctx, regressor.h, C.byref(lp)))
        self._regressor = regressor  # keep it alive while in use

    def trace(self, windows, window, candidates, cap=None):
        """Training samples (x: n x 6, t: n) from `windows` windows of the plain rule."""
        cand = _f64(candidates)
        if cap is None:
            cap = 1 << 22
        x = np.zeros((cap, 6), np.float32)
        t = np.zeros(cap, np.float32)
        n = C.c_longlong()
        self._check(self.lib.dem_trace(self.ctx, int(windows), int(window), len(cand), _pd(cand),
                                       int(cap), x.ctypes.data_as(C.POINTER(C.c_float)),
                                       t.ctypes.data_as(C.POINTER(C.c_float)), C.byref(n)))
        return x[: n.value].copy(), t[: n.value].copy()

    def close(self):
        if getattr(self, "ctx", None):
            self.lib.dem_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


def _pf(a):
    return a.ctypes.data_as(C.POINTER(C.c_float))


class Regressor:
    """The learned list-lifetime regressor of libdem.so (6 -> 3x64 ReLU -> 1,
    BF16 weights, FP32 accumulation, Adam), trained and run on the GPU."""

    def __init__(self, device=0, params=None):
        self.lib = capi.load()
        h = C.c_void_p()
        rc = self.lib.dem_mlp_create(int(device), C.byref(h))
        if rc != 0:
            raise DemError(rc, "dem_mlp_create failed")
        self.h = h
        self.n_params = int(self.lib.dem_mlp_num_params())
        if params is not None:
            self.set_params(params)

    def _check(self, rc):
        if rc != 0:
            raise DemError(rc, "regressor call failed")

    def set_params(self, p):
        p = np.ascontiguousarray(p, np.float32)
        assert p.size == self.n_params
        self._check(self.lib.dem_mlp_set_params(self.h, _pf(p)))

    def params(self):
        p = np.zeros(self.n_params, np.float32)
        self._check(self.lib.dem_mlp_get_params(self.h, _pf(p)))
        return p

    def forward(self, x):
        x = np.ascontiguousarray(x, np.float32).reshape(-1, 6)
        y = np.zeros(len(x), np.float32)
        self._check(self.lib.dem_mlp_forward(self.h, len(x), _pf(x), _pf(y)))
        return y

    def forward_tc(self, x):
        """Forward pass on the tensor cores (bfloat16 layer inputs, FP32 sums)."""
        x = np.ascontiguousarray(x, np.float32).reshape(-1, 6)
        y = np.zeros(len(x), np.float32)
        self._check(self.lib.dem_mlp_forward_tc(self.h, len(x), _pf(x), _pf(y)))
        return y

    def loss_grad(self, x, t):
        x = np.ascontiguousarray(x, np.float32).reshape(-1, 6)
        t = np.ascontiguousarray(t, np.float32)
        g = np.zeros(self.n_params, np.float32)
        loss = C.c_double()
        self._check(self.lib.dem_mlp_loss_grad(self.h, len(x), _pf(x), _pf(t), C.byref(loss), _pf(g)))
        return loss.value, g

    def loss_grad_noalloc(self, x, t):
        """loss_grad without device allocation (fixed scratch of
        DEM_MLP_NOALLOC_MAX_ROWS rows; calls on one device must not overlap)."""
        x = np.ascontiguousarray(x, np.float32).reshape(-1, 6)
        t = np.ascontiguousarray(t, np.float32)
        if len(x) > capi.DEM_MLP_NOALLOC_MAX_ROWS:
            raise ValueError(f"{len(x)} rows exceed the fixed scratch of "
                             f"{capi.DEM_MLP_NOALLOC_MAX_ROWS} rows")
        g = np.zeros(self.n_params, np.float32)
        loss = C.c_double()
        self._check(self.lib.dem_mlp_loss_grad_noalloc(self.h, len(x), _pf(x), _pf(t),
                                                       C.byref(loss), _pf(g)))
        return loss.value, g

    def train(self, x, t, steps=500, batch=4096, lr=1e-3, seed=0):
        x = np.ascontiguousarray(x, np.float32).reshape(-1, 6)
        t = np.ascontiguousarray(t, np.float32)
        loss = C.c_double()
        self._check(self.lib.dem_mlp_train(self.h, len(x), _pf(x), _pf(t), int(steps), int(batch),
                                           float(lr), int(seed), C.byref(loss)))
        return loss.value

    def close(self):
        if getattr(self, "h", None):
            self.lib.dem_mlp_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
