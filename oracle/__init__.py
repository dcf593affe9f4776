"""FP64 CPU oracle for the clump-of-spheres DEM hot path -- TEST INFRASTRUCTURE.

Only the test suite, the package smoke check and the benchmark's CPU-baseline
leg may import this module.  The product path (the CUDA library and its
binding) never imports, links or executes anything here.

The arithmetic lives in ``dem_oracle.c`` (plain, single-threaded, double
precision C written from the paper, arXiv 2307.03445, section 2.1 Eq. (1)-(5)
and section 2.2).  This module compiles it with gcc and wraps it with ctypes;
it holds no arithmetic of the method itself.

Parity status of each function (pins live in ``tests/test_oracle_*.py``):
  sphere_centres, detect_coords   pinned: hand rotations, brute force
  bin_entries, pairs_binned       pinned: O(N^2) brute force, hand cases
  wall_distance / candidates      pinned: closed-form distances to plane,
                                  cylinder and cone
  contact / forces                pinned: Hertz closed forms (peak overlap,
                                  contact time, static overlap), CoR, Coulomb
                                  stick/slip on a tilted plane, momentum
  integrate                       pinned: free flight, torque-free rotation
                                  invariants, energy at CoR = 1, mu = 0
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "dem_oracle.c")
_LIB_PATH = os.path.join(_HERE, "libdem_oracle.so")
_lock = threading.Lock()
_lib = None

WALL_PLANE, WALL_CYLINDER, WALL_CONE, WALL_TRIANGLE = 0, 1, 2, 3
MIX_MEAN, MIX_MIN, MIX_MAX = 0, 1, 2


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (no FMA contraction) into oracle/libdem_oracle.so."""
    if not force and os.path.exists(_LIB_PATH) and os.path.getmtime(_LIB_PATH) >= max(
        os.path.getmtime(_SRC), os.path.getmtime(os.path.join(_HERE, "dem_oracle.h"))
    ):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fPIC",
           "-shared", "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class Wall(C.Structure):
    _fields_ = [("type", C.c_int), ("material", C.c_int), ("p", C.c_double * 3),
                ("n", C.c_double * 3), ("radius", C.c_double), ("half_angle", C.c_double),
                ("height", C.c_double), ("vel", C.c_double * 3), ("b", C.c_double * 3),
                ("c", C.c_double * 3)]


class Model(C.Structure):
    _fields_ = [("n_tpl", C.c_int), ("tpl_off", C.POINTER(C.c_int)),
                ("tpl_pos", C.POINTER(C.c_double)), ("tpl_rad", C.POINTER(C.c_double)),
                ("tpl_mat", C.POINTER(C.c_int)), ("tpl_mass", C.POINTER(C.c_double)),
                ("tpl_inertia", C.POINTER(C.c_double)), ("n_mat", C.c_int),
                ("E", C.POINTER(C.c_double)), ("nu", C.POINTER(C.c_double)),
                ("mu", C.POINTER(C.c_double)), ("cor", C.POINTER(C.c_double)),
                ("mix_rule", C.c_int), ("n_walls", C.c_int), ("walls", C.POINTER(Wall)),
                ("h", C.c_double), ("g", C.c_double * 3), ("lo", C.c_double * 3),
                ("hi", C.c_double * 3), ("bin_size", C.c_double)]


_D = C.POINTER(C.c_double)
_I = C.POINTER(C.c_int)
_L = C.POINTER(C.c_longlong)
_U = C.POINTER(C.c_uint)
_M = C.POINTER(Model)


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = C.CDLL(build())
            sig = {
                "orc_num_spheres": (C.c_longlong, [_M, C.c_int, _I]),
                "orc_sphere_centres": (None, [_M, C.c_int, _I, _D, _D, _D, _I, _I]),
                "orc_detect_coords": (None, [_M, C.c_longlong, _D, _I, _D, _L, _L]),
                "orc_grid_dims": (None, [_M, _L, _L]),
                "orc_bin_entries": (C.c_longlong, [_M, C.c_longlong, _L, _L, C.c_longlong, _U, _I]),
                "orc_pairs_brute": (C.c_longlong, [C.c_longlong, _I, _L, _L, C.c_longlong, _I, _I]),
                "orc_pairs_binned": (C.c_longlong, [_M, C.c_longlong, _I, _L, _L, C.c_longlong, _I, _I]),
                "orc_wall_distance": (C.c_double, [C.POINTER(Wall), C.c_double, _D, _D]),
                "orc_wall_candidates": (C.c_longlong, [_M, C.c_longlong, _D, _I, _D, C.c_double,
                                                        C.c_double, C.c_longlong, _I, _I]),
                "orc_pair_material": (None, [_M, C.c_int, C.c_int, _D, _D, _D, _D]),
                "orc_contact": (C.c_int, [_M, C.c_int, C.c_int, _D, _D, _D, _D, _D, _D, _D, _D,
                                          C.c_double, C.c_double, C.c_double, C.c_double, _D,
                                          C.c_double, _D, _D, _D, _D]),
                "orc_forces": (C.c_longlong, [_M, C.c_int, _I, _D, _D, _D, _D, C.c_double,
                                              C.c_longlong, _I, _I, _D, C.c_longlong, _I, _I, _D,
                                              _D, _D, _D, _D, _D]),
                "orc_integrate": (None, [_M, C.c_int, _I, _D, _D, _D, _D, _D, _D]),
                "orc_sim_create": (C.c_void_p, [_M, C.c_int, _I, _D, _D, _D, _D, C.c_double, C.c_int]),
                "orc_sim_step": (C.c_longlong, [C.c_void_p, C.c_int, C.c_int]),
                "orc_sim_get_state": (None, [C.c_void_p, _D, _D, _D, _D]),
                "orc_sim_num_contacts": (C.c_longlong, [C.c_void_p, _L]),
                "orc_sim_get_contacts": (None, [C.c_void_p, _I, _I, _D, _I, _I, _D]),
                "orc_sim_last_forces": (None, [C.c_void_p, _D, _D]),
                "orc_sim_time": (C.c_double, [C.c_void_p]),
                "orc_sim_active": (C.c_longlong, [C.c_void_p]),
                "orc_sim_destroy": (None, [C.c_void_p]),
                "orc_mlp_num_params": (C.c_int, []),
                "orc_mlp_forward": (None, [_D, C.c_longlong, _D, _D]),
                "orc_mlp_forward_bf16act": (None, [_D, C.c_longlong, _D, _D]),
                "orc_mlp_loss_grad": (C.c_double, [_D, C.c_longlong, _D, _D, _D]),
                "orc_mlp_adam": (None, [_D, _D, _D, _D, C.c_int, C.c_double, C.c_double,
                                        C.c_double, C.c_double]),
            }
            for name, (res, args) in sig.items():
                f = getattr(lib, name)
                f.restype = res
                f.argtypes = args
            _lib = lib
    return _lib


def _p(a, ct):
    return a.ctypes.data_as(C.POINTER(ct)) if a is not None else None


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _i32(a):
    return np.ascontiguousarray(a, dtype=np.int32)


class OracleModel:
    """Owns the numpy arrays behind an ``orc_model`` (templates, materials, walls, world).

    ``scene`` is any object with the attributes produced by the seeded scene
    generators: tpl_off, tpl_pos, tpl_rad, tpl_mat, tpl_mass, tpl_inertia, E, nu,
    mu, cor, mix_rule, walls (list of dicts), h, g, lo, hi, bin_size.
    """

    def __init__(self, scene):
        self.lib = _load()
        self._keep = {}
        k = self._keep
        k["tpl_off"] = _i32(scene.tpl_off)
        k["tpl_pos"] = _f64(scene.tpl_pos).reshape(-1)
        k["tpl_rad"] = _f64(scene.tpl_rad)
        k["tpl_mat"] = _i32(scene.tpl_mat)
        k["tpl_mass"] = _f64(scene.tpl_mass)
        k["tpl_inertia"] = _f64(scene.tpl_inertia).reshape(-1)
        for name in ("E", "nu", "mu", "cor"):
            k[name] = _f64(getattr(scene, name))
        walls = list(scene.walls)
        warr = (Wall * max(1, len(walls)))()
        for i, w in enumerate(walls):
            warr[i].type = int(w["type"])
            warr[i].material = int(w.get("material", 0))
            for j in range(3):
                warr[i].p[j] = float(w["p"][j])
                warr[i].n[j] = float(w["n"][j])
                warr[i].vel[j] = float(w.get("vel", (0.0, 0.0, 0.0))[j])
                warr[i].b[j] = float(w.get("b", (0.0, 0.0, 0.0))[j])
                warr[i].c[j] = float(w.get("c", (0.0, 0.0, 0.0))[j])
            warr[i].radius = float(w.get("radius", 0.0))
            warr[i].half_angle = float(w.get("half_angle", 0.0))
            warr[i].height = float(w.get("height", 0.0))
        k["walls"] = warr
        m = Model()
        m.n_tpl = len(k["tpl_mass"])
        m.tpl_off = _p(k["tpl_off"], C.c_int)
        m.tpl_pos = _p(k["tpl_pos"], C.c_double)
        m.tpl_rad = _p(k["tpl_rad"], C.c_double)
        m.tpl_mat = _p(k["tpl_mat"], C.c_int)
        m.tpl_mass = _p(k["tpl_mass"], C.c_double)
        m.tpl_inertia = _p(k["tpl_inertia"], C.c_double)
        m.n_mat = len(k["E"])
        m.E, m.nu, m.mu, m.cor = (_p(k[n], C.c_double) for n in ("E", "nu", "mu", "cor"))
        m.mix_rule = int(getattr(scene, "mix_rule", 0))
        m.n_walls = len(walls)
        m.walls = C.cast(warr, C.POINTER(Wall))
        m.h = float(scene.h)
        for j in range(3):
            m.g[j] = float(scene.g[j])
            m.lo[j] = float(scene.lo[j])
            m.hi[j] = float(scene.hi[j])
        m.bin_size = float(scene.bin_size)
        self.m = m
        self.n_walls = len(walls)

    @property
    def ptr(self):
        return C.byref(self.m)

    # ---- geometry / detection -------------------------------------------
    def num_spheres(self, tpl):
        tpl = _i32(tpl)
        return int(self.lib.orc_num_spheres(self.ptr, len(tpl), _p(tpl, C.c_int)))

    def sphere_centres(self, tpl, pos, quat):
        tpl, pos, quat = _i32(tpl), _f64(pos), _f64(quat)
        ns = self.num_spheres(tpl)
        xs = np.zeros((ns, 3))
        owner = np.zeros(ns, np.int32)
        tsph = np.zeros(ns, np.int32)
        self.lib.orc_sphere_centres(self.ptr, len(tpl), _p(tpl, C.c_int), _p(pos, C.c_double),
                                    _p(quat, C.c_double), _p(xs, C.c_double),
                                    _p(owner, C.c_int), _p(tsph, C.c_int))
        return xs, owner, tsph

    def detect_coords(self, xs, tsph, margin):
        xs, tsph = _f64(xs), _i32(tsph)
        ns = len(tsph)
        mg = _f64(np.broadcast_to(np.asarray(margin, np.float64), (ns,)))
        qc = np.zeros((ns, 3), np.int64)
        rho = np.zeros(ns, np.int64)
        self.lib.orc_detect_coords(self.ptr, ns, _p(xs, C.c_double), _p(tsph, C.c_int),
                                   _p(mg, C.c_double), _p(qc, C.c_longlong), _p(rho, C.c_longlong))
        return qc, rho

    def need_bins(self):
        """The oracle takes the bin edge literally (a zero edge would be a grid
        of one lattice unit per bin); the library's default edge depends on the
        margin, which the model does not know, so binning needs an explicit one."""
        if not self.m.bin_size > 0.0:
            raise ValueError("the oracle needs an explicit bin edge (scene.bin_size > 0)")

    def grid_dims(self):
        self.need_bins()
        dims = np.zeros(3, np.int64)
        L = np.zeros(1, np.int64)
        self.lib.orc_grid_dims(self.ptr, _p(dims, C.c_longlong), _p(L, C.c_longlong))
        return dims, int(L[0])

    def bin_entries(self, qc, rho):
        self.need_bins()
        qc, rho = np.ascontiguousarray(qc, np.int64), np.ascontiguousarray(rho, np.int64)
        ns = len(rho)
        n = self.lib.orc_bin_entries(self.ptr, ns, _p(qc, C.c_longlong), _p(rho, C.c_longlong),
                                     0, None, None)
        keys = np.zeros(n, np.uint32)
        ids = np.zeros(n, np.int32)
        self.lib.orc_bin_entries(self.ptr, ns, _p(qc, C.c_longlong), _p(rho, C.c_longlong), n,
                                 _p(keys, C.c_uint), _p(ids, C.c_int))
        return keys, ids

    def pairs_brute(self, owner, qc, rho):
        owner = _i32(owner)
        qc, rho = np.ascontiguousarray(qc, np.int64), np.ascontiguousarray(rho, np.int64)
        ns = len(rho)
        args = (ns, _p(owner, C.c_int), _p(qc, C.c_longlong), _p(rho, C.c_longlong))
        n = self.lib.orc_pairs_brute(*args, 0, None, None)
        a = np.zeros(n, np.int32)
        b = np.zeros(n, np.int32)
        self.lib.orc_pairs_brute(*args, n, _p(a, C.c_int), _p(b, C.c_int))
        return a, b

    def pairs_binned(self, owner, qc, rho):
        self.need_bins()
        owner = _i32(owner)
        qc, rho = np.ascontiguousarray(qc, np.int64), np.ascontiguousarray(rho, np.int64)
        ns = len(rho)
        args = (self.ptr, ns, _p(owner, C.c_int), _p(qc, C.c_longlong), _p(rho, C.c_longlong))
        n = self.lib.orc_pairs_binned(*args, 0, None, None)
        a = np.zeros(n, np.int32)
        b = np.zeros(n, np.int32)
        self.lib.orc_pairs_binned(*args, n, _p(a, C.c_int), _p(b, C.c_int))
        return a, b

    def wall_distance(self, k, t, x):
        x = _f64(x)
        nw = np.zeros(3)
        d = self.lib.orc_wall_distance(C.byref(self._keep["walls"][k]), float(t),
                                       _p(x, C.c_double), _p(nw, C.c_double))
        return d, nw

    def wall_candidates(self, xs, tsph, margin, t, travel_time):
        xs, tsph = _f64(xs), _i32(tsph)
        ns = len(tsph)
        mg = _f64(np.broadcast_to(np.asarray(margin, np.float64), (ns,)))
        args = (self.ptr, ns, _p(xs, C.c_double), _p(tsph, C.c_int), _p(mg, C.c_double),
                float(t), float(travel_time))
        n = self.lib.orc_wall_candidates(*args, 0, None, None)
        s = np.zeros(n, np.int32)
        w = np.zeros(n, np.int32)
        self.lib.orc_wall_candidates(*args, n, _p(s, C.c_int), _p(w, C.c_int))
        return s, w

    # ---- contact law ------------------------------------------------------
    def pair_material(self, ia, ib):
        out = [C.c_double() for _ in range(4)]
        self.lib.orc_pair_material(self.ptr, ia, ib, *(C.byref(o) for o in out))
        return tuple(o.value for o in out)

    def contact(self, mat_a, mat_b, xa, xb, Xa, Xb, va, wa, vb, wb, ra, rb, ma, mb,
                u, n_wall=None, delta_wall=0.0):
        """One contact; returns (active, F on b, new u, lever arm a, lever arm b)."""
        z = np.zeros(3)
        arr = [_f64(v) if v is not None else z.copy() for v in (xa, xb, Xa, Xb, va, wa, vb, wb)]
        u = _f64(u).copy()
        nw = _f64(n_wall) if n_wall is not None else z.copy()
        F, ca, cb = np.zeros(3), np.zeros(3), np.zeros(3)
        act = self.lib.orc_contact(self.ptr, mat_a, mat_b, *(_p(v, C.c_double) for v in arr),
                                   float(ra), float(rb), float(ma), float(mb),
                                   _p(nw, C.c_double), float(delta_wall), _p(u, C.c_double),
                                   _p(F, C.c_double), _p(ca, C.c_double), _p(cb, C.c_double))
        return bool(act), F, u, ca, cb

    def forces(self, tpl, pos, quat, vel, angvel, t, pa, pb, up, ws=None, ww=None, uw=None,
               with_mag=False, wall_torque=False):
        """Clump forces/torques for one step; returns (F, T, Fwall, up_new, uw_new, n_active)
        and, with ``with_mag``, the per-clump sums of |F| and |torque| over its contacts;
        with ``wall_torque``, also (last) the moment on each wall about its reference point
        at time t."""
        tpl, pos, quat, vel, angvel = _i32(tpl), _f64(pos), _f64(quat), _f64(vel), _f64(angvel)
        pa, pb = _i32(pa), _i32(pb)
        up = _f64(up).reshape(-1, 3).copy()
        ws = _i32(ws if ws is not None else np.zeros(0, np.int32))
        ww = _i32(ww if ww is not None else np.zeros(0, np.int32))
        uw = _f64(uw if uw is not None else np.zeros((0, 3))).reshape(-1, 3).copy()
        n = len(tpl)
        F = np.zeros((n, 3))
        T = np.zeros((n, 3))
        Fw = np.zeros((max(1, self.n_walls), 3))
        Tw = np.zeros((max(1, self.n_walls), 3))
        mag = np.zeros((n, 2))
        act = self.lib.orc_forces(self.ptr, n, _p(tpl, C.c_int), _p(pos, C.c_double),
                                  _p(quat, C.c_double), _p(vel, C.c_double),
                                  _p(angvel, C.c_double), float(t), len(pa), _p(pa, C.c_int),
                                  _p(pb, C.c_int), _p(up, C.c_double), len(ws), _p(ws, C.c_int),
                                  _p(ww, C.c_int), _p(uw, C.c_double), _p(F, C.c_double),
                                  _p(T, C.c_double), _p(Fw, C.c_double), _p(Tw, C.c_double),
                                  _p(mag, C.c_double))
        out = (F, T, Fw[: self.n_walls], up, uw, int(act)) + ((mag,) if with_mag else ())
        return out + ((Tw[: self.n_walls],) if wall_torque else ())

    def integrate(self, tpl, pos, quat, vel, angvel, F, T):
        tpl = _i32(tpl)
        pos, quat, vel, angvel = (_f64(a).copy() for a in (pos, quat, vel, angvel))
        F, T = _f64(F), _f64(T)
        self.lib.orc_integrate(self.ptr, len(tpl), _p(tpl, C.c_int), _p(pos, C.c_double),
                               _p(quat, C.c_double), _p(vel, C.c_double),
                               _p(angvel, C.c_double), _p(F, C.c_double), _p(T, C.c_double))
        return pos, quat, vel, angvel


class OracleSim:
    """A whole oracle simulation with the list rebuilt every ``rebuild_every`` steps."""

    def __init__(self, scene, margin, rebuild_every, state=None):
        self.model = OracleModel(scene)
        self.model.need_bins()
        self.lib = self.model.lib
        st = state if state is not None else scene
        self.tpl = _i32(st.tpl)
        self.n = len(self.tpl)
        arr = [_f64(getattr(st, k)) for k in ("pos", "quat", "vel", "angvel")]
        self.h = self.lib.orc_sim_create(self.model.ptr, self.n, _p(self.tpl, C.c_int),
                                         *(_p(a, C.c_double) for a in arr), float(margin),
                                         int(rebuild_every))

    def step(self, nsteps=1, audit=False):
        return int(self.lib.orc_sim_step(self.h, int(nsteps), int(bool(audit))))

    def state(self):
        n = self.n
        pos, quat, vel, angvel = np.zeros((n, 3)), np.zeros((n, 4)), np.zeros((n, 3)), np.zeros((n, 3))
        self.lib.orc_sim_get_state(self.h, *(_p(a, C.c_double) for a in (pos, quat, vel, angvel)))
        return pos, quat, vel, angvel

    def contacts(self):
        nw = C.c_longlong()
        npair = self.lib.orc_sim_num_contacts(self.h, C.byref(nw))
        a, b = np.zeros(npair, np.int32), np.zeros(npair, np.int32)
        u = np.zeros((npair, 3))
        ws, ww = np.zeros(nw.value, np.int32), np.zeros(nw.value, np.int32)
        uw = np.zeros((nw.value, 3))
        self.lib.orc_sim_get_contacts(self.h, _p(a, C.c_int), _p(b, C.c_int), _p(u, C.c_double),
                                      _p(ws, C.c_int), _p(ww, C.c_int), _p(uw, C.c_double))
        return a, b, u, ws, ww, uw

    def last_forces(self):
        F, T = np.zeros((self.n, 3)), np.zeros((self.n, 3))
        self.lib.orc_sim_last_forces(self.h, _p(F, C.c_double), _p(T, C.c_double))
        return F, T

    def time(self):
        return float(self.lib.orc_sim_time(self.h))

    def active(self):
        return int(self.lib.orc_sim_active(self.h))

    def close(self):
        if self.h:
            self.lib.orc_sim_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ---------------------------------------------------------------------------
# learned lifetime regressor (FP64 reference of the GPU training kernels)
# ---------------------------------------------------------------------------
MLP_IN, MLP_H = 6, 64


def mlp_num_params():
    return int(_load().orc_mlp_num_params())


def mlp_forward(params, x):
    params, x = _f64(params), _f64(x).reshape(-1, MLP_IN)
    y = np.zeros(len(x))
    _load().orc_mlp_forward(_p(params, C.c_double), len(x), _p(x, C.c_double), _p(y, C.c_double))
    return y


def mlp_forward_bf16act(params, x):
    """Forward pass with bfloat16-rounded layer inputs and double sums."""
    params, x = _f64(params), _f64(x).reshape(-1, MLP_IN)
    y = np.zeros(len(x))
    _load().orc_mlp_forward_bf16act(_p(params, C.c_double), len(x), _p(x, C.c_double),
                                    _p(y, C.c_double))
    return y


def mlp_loss_grad(params, x, t):
    params, x, t = _f64(params), _f64(x).reshape(-1, MLP_IN), _f64(t)
    g = np.zeros(mlp_num_params())
    loss = _load().orc_mlp_loss_grad(_p(params, C.c_double), len(x), _p(x, C.c_double),
                                     _p(t, C.c_double), _p(g, C.c_double))
    return float(loss), g


def mlp_adam(params, m, v, grad, step, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8):
    params, m, v = (_f64(a).copy() for a in (params, m, v))
    grad = _f64(grad)
    _load().orc_mlp_adam(_p(params, C.c_double), _p(m, C.c_double), _p(v, C.c_double),
                         _p(grad, C.c_double), int(step), lr, beta1, beta2, eps)
    return params, m, v
