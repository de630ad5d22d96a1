"""Seeded synthetic inputs shared by the oracle and the CUDA path.

This package holds none of the rendering method's arithmetic. It builds a
procedural luminaire octree in the canonical host tree format and draws ray
sets, both from a counter-based generator (``luminaire.c``), so the same seed
gives the same inputs to the FP64 oracle and to the GPU library.

The workloads stand in for the paper's Mitsuba luminaires (Sec. 6.1), which
are not available: a helical emissive coil inside a spherical glass-like
shell, with per-leaf values drawn as the workload description states.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import tempfile
from dataclasses import dataclass, field, replace

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "luminaire.c")
_SO = os.path.join(_HERE, "_build", "libplogen.so")

_lib = None


def build(force: bool = False) -> str:
    """Compile luminaire.c into an in-tree shared library (gcc, OpenMP)."""
    os.makedirs(os.path.dirname(_SO), exist_ok=True)
    if not force and os.path.exists(_SO) and os.path.getmtime(_SO) >= os.path.getmtime(_SRC):
        return _SO
    fd, tmp = tempfile.mkstemp(suffix=".so", dir=os.path.dirname(_SO))
    os.close(fd)
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off",
           _SRC, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _SO)
    return _SO


class _Params(ctypes.Structure):
    _fields_ = [
        ("depth", ctypes.c_int32),
        ("sh_degree", ctypes.c_int32),
        ("seed", ctypes.c_uint64),
        ("shell_center", ctypes.c_double * 3),
        ("shell_radius", ctypes.c_double),
        ("shell_half_thickness", ctypes.c_double),
        ("coil_center_xy", ctypes.c_double * 2),
        ("coil_radius", ctypes.c_double),
        ("coil_tube_radius", ctypes.c_double),
        ("coil_z0", ctypes.c_double),
        ("coil_z1", ctypes.c_double),
        ("coil_turns", ctypes.c_double),
        ("emissive_fraction", ctypes.c_double),
        ("sigma_log10_min", ctypes.c_double),
        ("sigma_log10_max", ctypes.c_double),
        ("dc_log10_min", ctypes.c_double),
        ("dc_log10_max", ctypes.c_double),
        ("band_rel_std", ctypes.c_double),
    ]


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        P = ctypes.c_void_p
        lib.plogen_build.restype = P
        lib.plogen_build.argtypes = [ctypes.POINTER(_Params), ctypes.POINTER(ctypes.c_int64),
                                     ctypes.POINTER(ctypes.c_int64)]
        lib.plogen_fill.restype = ctypes.c_int
        lib.plogen_fill.argtypes = [P, P, P, P, P]
        lib.plogen_free.restype = None
        lib.plogen_free.argtypes = [P]
        lib.plogen_rays_sphere.restype = None
        lib.plogen_rays_sphere.argtypes = [ctypes.c_uint64, ctypes.c_int64, P, ctypes.c_double, P]
        lib.plogen_rays_room.restype = ctypes.c_int64
        lib.plogen_rays_room.argtypes = [ctypes.c_uint64, ctypes.c_int64, P, P, P, P, ctypes.c_int64, P]
        _lib = lib
    return _lib


@dataclass(frozen=True)
class Luminaire:
    """Procedural luminaire recipe (all lengths in unit-cube coordinates)."""
    depth: int = 6
    sh_degree: int = 2
    seed: int = 20220711
    shell_center: tuple = (0.5, 0.5, 0.5)
    shell_radius: float = 0.42
    shell_half_thickness: float = 0.014
    coil_center_xy: tuple = (0.5, 0.5)
    coil_radius: float = 0.2
    coil_tube_radius: float = 0.03
    coil_z0: float = 0.25
    coil_z1: float = 0.75
    coil_turns: float = 5.0
    emissive_fraction: float = 0.3
    sigma_log10: tuple = (-2.0, 3.0)
    dc_log10: tuple = (-2.0, 4.0)
    band_rel_std: float = 0.1

    def with_(self, **kw) -> "Luminaire":
        return replace(self, **kw)


# Depth-6 tree, SH degree 2: the 65,536-ray, ~20k-leaf workload.
LUMINAIRE_D6 = Luminaire()
# Depth-10 tree, SH degree 3: the ~30M-leaf workload rendered by 16M rays.
LUMINAIRE_D10 = Luminaire(depth=10, sh_degree=3, shell_half_thickness=0.0057, coil_tube_radius=0.015)


@dataclass
class HostTree:
    """Canonical host tree (numpy arrays), the format plo_build_tree reads."""
    depth: int
    sh_degree: int
    child: np.ndarray          # int32 [n_nodes, 8]
    sigma: np.ndarray          # float32 [n_leaves]
    sh: np.ndarray             # float32 [n_leaves, 3, K]
    leaf_xyz: np.ndarray | None = None  # int32 [n_leaves, 3] coords at level depth (generator only)
    bbox_min: tuple = (0.0, 0.0, 0.0)
    bbox_max: tuple = (1.0, 1.0, 1.0)
    meta: dict = field(default_factory=dict)

    @property
    def K(self) -> int:
        return (self.sh_degree + 1) ** 2

    @property
    def n_nodes(self) -> int:
        return int(self.child.shape[0])

    @property
    def n_leaves(self) -> int:
        return int(self.sigma.shape[0])


def luminaire_tree(rec: Luminaire = LUMINAIRE_D6, with_sh: bool = True) -> HostTree:
    """Build the procedural luminaire octree for recipe `rec`."""
    lib = _load()
    p = _Params()
    p.depth, p.sh_degree, p.seed = rec.depth, rec.sh_degree, rec.seed
    p.shell_center[:] = rec.shell_center
    p.shell_radius, p.shell_half_thickness = rec.shell_radius, rec.shell_half_thickness
    p.coil_center_xy[:] = rec.coil_center_xy
    p.coil_radius, p.coil_tube_radius = rec.coil_radius, rec.coil_tube_radius
    p.coil_z0, p.coil_z1, p.coil_turns = rec.coil_z0, rec.coil_z1, rec.coil_turns
    p.emissive_fraction = rec.emissive_fraction
    p.sigma_log10_min, p.sigma_log10_max = rec.sigma_log10
    p.dc_log10_min, p.dc_log10_max = rec.dc_log10
    p.band_rel_std = rec.band_rel_std
    nn, nl = ctypes.c_int64(), ctypes.c_int64()
    h = lib.plogen_build(ctypes.byref(p), ctypes.byref(nn), ctypes.byref(nl))
    if not h:
        raise MemoryError("plogen_build failed (bad parameters or out of memory)")
    try:
        K = (rec.sh_degree + 1) ** 2
        child = np.empty((nn.value, 8), np.int32)
        sigma = np.empty(nl.value, np.float32)
        sh = np.empty((nl.value, 3, K), np.float32) if with_sh else None
        xyz = np.empty((nl.value, 3), np.int32)
        lib.plogen_fill(h, child.ctypes.data, sigma.ctypes.data,
                        sh.ctypes.data if sh is not None else None, xyz.ctypes.data)
    finally:
        lib.plogen_free(h)
    if sh is None:
        sh = np.zeros((nl.value, 3, K), np.float32)
    return HostTree(rec.depth, rec.sh_degree, child, sigma, sh, xyz, meta={"recipe": rec})


def rays_sphere(n: int, seed: int = 7, radius: float = 3.0, center=(0.5, 0.5, 0.5)) -> np.ndarray:
    """float32 [n, 6]: origins uniform on a sphere about the cube centre,
    each aimed at a uniform point of the unit cube."""
    lib = _load()
    out = np.empty((n, 6), np.float32)
    c = np.asarray(center, np.float64)
    lib.plogen_rays_sphere(seed, n, c.ctypes.data, radius, out.ctypes.data)
    return out


ROOM_LO = (-4.5, -4.5, -1.0)
ROOM_HI = (5.5, 5.5, 2.0)


def rays_room(n: int, seed: int = 11, room_lo=ROOM_LO, room_hi=ROOM_HI,
              box_lo=(0.0, 0.0, 0.0), box_hi=(1.0, 1.0, 1.0), max_attempts: int = 1 << 20,
              return_attempts: bool = False):
    """float32 [n, 6]: origins uniform in a 10x10x3 room outside the cube,
    cosine-weighted directions about the direction to the cube centre, kept
    only when the ray meets the cube."""
    lib = _load()
    out = np.empty((n, 6), np.float32)
    arrs = [np.asarray(v, np.float64) for v in (room_lo, room_hi, box_lo, box_hi)]
    tot = lib.plogen_rays_room(seed, n, *(a.ctypes.data for a in arrs), max_attempts, out.ctypes.data)
    if tot < 0:
        raise RuntimeError("rays_room: a ray exceeded max_attempts")
    return (out, int(tot)) if return_attempts else out
