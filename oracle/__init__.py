"""FP64 CPU oracle for the plenoctree luminaire path.

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the
bench's CPU-baseline leg are the only callers. The product library never
imports this package and shares no code with it.

``render.c`` (plain C, FP64) holds the render oracle: SH basis from the
associated-Legendre recursion, point -> leaf descent, and the exact per-leaf
segment integral of Eq. 3 with exponential or linear (Eq. 4) transmittance
and alpha = 1 - T (Eq. 5); and a path tracer that uses the luminaire as an
emitter (Eq. 2, Sec. 5 "Sampling") with its random numbers passed in.
``mlp.py`` holds the learned-part oracle.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import tempfile

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "render.c")
_SO = os.path.join(_HERE, "_build", "liboracle.so")
_lib = None

EXPONENTIAL, LINEAR, LINEAR_LITERAL = 0, 1, 2
RELU, SIGMOID = 0, 1


def build(force: bool = False) -> str:
    """Compile render.c (gcc, FP64, OpenMP over rays) in-tree."""
    os.makedirs(os.path.dirname(_SO), exist_ok=True)
    if not force and os.path.exists(_SO) and os.path.getmtime(_SO) >= os.path.getmtime(_SRC):
        return _SO
    fd, tmp = tempfile.mkstemp(suffix=".so", dir=os.path.dirname(_SO))
    os.close(fd)
    subprocess.run(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off",
                    _SRC, "-o", tmp, "-lm"], check=True)
    os.replace(tmp, _SO)
    return _SO


class _Tree(ctypes.Structure):
    _fields_ = [("depth", ctypes.c_int32), ("sh_degree", ctypes.c_int32),
                ("n_nodes", ctypes.c_int64), ("n_leaves", ctypes.c_int64),
                ("child", ctypes.c_void_p), ("sigma", ctypes.c_void_p), ("sh", ctypes.c_void_p),
                ("bbox_min", ctypes.c_double * 3), ("bbox_max", ctypes.c_double * 3)]


class _Params(ctypes.Structure):
    _fields_ = [("transmittance", ctypes.c_int32), ("activation", ctypes.c_int32),
                ("l_max", ctypes.c_double), ("t_stop", ctypes.c_double), ("sigma_min", ctypes.c_double),
                ("saturate", ctypes.c_int32), ("proxy", ctypes.c_int32), ("sphere", ctypes.c_double * 4)]


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        P = ctypes.c_void_p
        lib.oracle_sh_basis.restype = None
        lib.oracle_sh_basis.argtypes = [ctypes.c_int, ctypes.c_double, ctypes.c_double, ctypes.c_double, P]
        lib.oracle_lookup.restype = None
        lib.oracle_lookup.argtypes = [P, P, P, ctypes.c_int64, P, P]
        lib.oracle_render.restype = ctypes.c_int64
        lib.oracle_render.argtypes = [P, P, ctypes.c_int64, P, P, P, P, P, P, P, P, P, ctypes.c_int]
        lib.oracle_trace.restype = ctypes.c_int32
        lib.oracle_trace.argtypes = [P, P, P, ctypes.c_int32, P, P]
        lib.oracle_max_threads.restype = ctypes.c_int
        _lib = lib
    return _lib


class _Bound:
    """Keeps the numpy arrays referenced by a ctypes tree struct alive."""

    def __init__(self, tree):
        self.child = np.ascontiguousarray(tree.child, np.int32)
        self.sigma = np.ascontiguousarray(tree.sigma, np.float32)
        self.sh = np.ascontiguousarray(tree.sh, np.float32)
        s = _Tree()
        s.depth, s.sh_degree = int(tree.depth), int(tree.sh_degree)
        s.n_nodes, s.n_leaves = self.child.shape[0], self.sigma.shape[0]
        s.child, s.sigma, s.sh = self.child.ctypes.data, self.sigma.ctypes.data, self.sh.ctypes.data
        s.bbox_min[:] = tuple(getattr(tree, "bbox_min", (0.0, 0.0, 0.0)))
        s.bbox_max[:] = tuple(getattr(tree, "bbox_max", (1.0, 1.0, 1.0)))
        self.struct = s


def _params(transmittance=EXPONENTIAL, activation=RELU, l_max=1.0, t_stop=0.0, sigma_min=0.0, saturate=False,
            sphere=None):
    """sphere = (cx, cy, cz, radius) in world units selects the sphere proxy."""
    p = _Params()
    p.transmittance, p.activation = transmittance, activation
    p.l_max, p.t_stop, p.sigma_min = l_max, t_stop, sigma_min
    p.saturate = int(bool(saturate))
    p.proxy = 0 if sphere is None else 1
    p.sphere[:] = (0.0, 0.0, 0.0, 0.0) if sphere is None else tuple(float(v) for v in sphere)
    return p


def max_threads() -> int:
    return int(_load().oracle_max_threads())


def sh_basis(degree: int, d) -> np.ndarray:
    """Y_k(d), k = l(l+1)+m, FP64, for one direction d."""
    lib = _load()
    out = np.zeros(25, np.float64)
    lib.oracle_sh_basis(degree, float(d[0]), float(d[1]), float(d[2]), out.ctypes.data)
    return out[: (degree + 1) ** 2]


def lookup(tree, pts, dirs=None):
    """Leaf id per point (unit-cube coords, float32 [n,3]); -1 empty octant,
    -2 outside.  Returns (leaf int64[n], level int32[n])."""
    lib = _load()
    b = _Bound(tree)
    pts = np.ascontiguousarray(pts, np.float32)
    n = pts.shape[0]
    d = None if dirs is None else np.ascontiguousarray(dirs, np.float32)
    leaf = np.empty(n, np.int64)
    lev = np.empty(n, np.int32)
    lib.oracle_lookup(ctypes.byref(b.struct), pts.ctypes.data, None if d is None else d.ctypes.data, n,
                      leaf.ctypes.data, lev.ctypes.data)
    return leaf, lev


def render(tree, rays, transmittance=EXPONENTIAL, activation=RELU, l_max=1.0, t_stop=0.0, sigma_min=0.0,
           saturate=False, sphere=None, n_threads: int = 0) -> dict:
    """Exact FP64 render of float32 rays [n,6].  Returns a dict of arrays:
    rgb [n,3], T [n], bound [n,3] (per-channel error scale), cond [n,3]
    (sensitivity to optical-depth errors), n_leaf, n_sh,
    n_cell, status (0 ok, 1 iteration cap, 2 lookup failure, 3 invalid ray:
    NaN/Inf component or zero direction, with NaN outputs)."""
    lib = _load()
    b = _Bound(tree)
    rays = np.ascontiguousarray(rays, np.float32)
    n = rays.shape[0]
    out = {"rgb": np.zeros((n, 3)), "T": np.ones(n), "bound": np.zeros((n, 3)), "cond": np.zeros((n, 3)),
           "n_leaf": np.zeros(n, np.int32), "n_sh": np.zeros(n, np.int32), "n_cell": np.zeros(n, np.int32),
           "status": np.zeros(n, np.int32)}
    p = _params(transmittance, activation, l_max, t_stop, sigma_min, saturate, sphere)
    lib.oracle_render(ctypes.byref(b.struct), rays.ctypes.data, n, ctypes.byref(p),
                      *(out[k].ctypes.data for k in ("rgb", "T", "bound", "cond", "n_leaf", "n_sh", "n_cell",
                                                      "status")),
                      int(n_threads))
    return out


def trace(tree, ray, max_cells: int = 100000, **kw):
    """Ordered cells crossed by one ray: (leaf int64[m] with -1 = empty
    octant, t float64[m,2] = [t_in, t_out])."""
    lib = _load()
    b = _Bound(tree)
    ray = np.ascontiguousarray(ray, np.float32).reshape(6)
    leaf = np.empty(max_cells, np.int64)
    t = np.empty((max_cells, 2), np.float64)
    p = _params(**kw)
    m = lib.oracle_trace(ctypes.byref(b.struct), ctypes.byref(p), ray.ctypes.data, max_cells,
                         leaf.ctypes.data, t.ctypes.data)
    return leaf[:m].copy(), t[:m].copy()


class _PtScene(ctypes.Structure):
    _fields_ = [("room_min", ctypes.c_double * 3), ("room_max", ctypes.c_double * 3),
                ("albedo", (ctypes.c_double * 3) * 6), ("cam_pos", ctypes.c_double * 3),
                ("cam_target", ctypes.c_double * 3), ("cam_up", ctypes.c_double * 3), ("fov_y", ctypes.c_double),
                ("width", ctypes.c_int32), ("height", ctypes.c_int32), ("max_bounces", ctypes.c_int32),
                ("emitter", ctypes.c_int32), ("box_radiance", ctypes.c_double * 3)]


def _pt_scene(sc: dict) -> _PtScene:
    s = _PtScene()
    for k in ("room_min", "room_max", "cam_pos", "cam_target", "cam_up", "box_radiance"):
        getattr(s, k)[:] = tuple(float(v) for v in sc[k])
    for w in range(6):
        s.albedo[w][:] = tuple(float(v) for v in sc["albedo"][w])
    s.fov_y = float(sc["fov_y"])
    s.width, s.height = int(sc["width"]), int(sc["height"])
    s.max_bounces, s.emitter = int(sc["max_bounces"]), int(sc["emitter"])
    return s


def pt_render(tree, scene: dict, uniforms, n_threads: int = 0, **params) -> np.ndarray:
    """Radiance of each path [n, 3] (FP64) of the path tracer with the
    luminaire as emitter.  uniforms [n, 2 + 5 * max_bounces] in [0, 1); path
    p is pixel p % (width * height).  scene: dict with the fields of
    plo_pt_scene; params: the render parameters of the luminaire queries."""
    lib = _load()
    if not getattr(lib, "_pt_sigs", False):
        lib.oracle_pt_render.restype = None
        lib.oracle_pt_render.argtypes = [ctypes.c_void_p] * 4 + [ctypes.c_int64, ctypes.c_int, ctypes.c_void_p]
        lib._pt_sigs = True
    b = _Bound(tree)
    u = np.ascontiguousarray(uniforms, np.float64)
    n = u.shape[0]
    assert u.shape[1] == 2 + 5 * int(scene["max_bounces"])
    out = np.zeros((n, 3))
    p = _params(**params)
    s = _pt_scene(scene)
    lib.oracle_pt_render(ctypes.byref(b.struct), ctypes.byref(p), ctypes.byref(s), u.ctypes.data, n, int(n_threads),
                         out.ctypes.data)
    return out
