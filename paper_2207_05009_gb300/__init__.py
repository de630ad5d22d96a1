"""Python binding of libplo (include/plo.h): plenoctree luminaire rendering on
GB300.  Argument marshalling only: every step of the path runs in the
library's CUDA kernels; PyTorch supplies device memory and the current stream.

There is no CPU fallback.  If libplo.so cannot be built or loaded, or no CUDA
device is present, the calls raise.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import numpy as np

from . import _build

__all__ = ["PloError", "Tree", "RenderParams", "load", "render", "render_host", "lookup", "trace",
           "PREC_FP32", "PREC_FP16", "PREC_BF16", "LAYOUT_OCTREE", "LAYOUT_BRICKS", "LAYOUT_DEFAULT", "TRANS_EXP", "TRANS_LINEAR", "TRANS_LINEAR_LITERAL",
           "ACT_RELU", "ACT_SIGMOID", "PROXY_BOX", "PROXY_SPHERE"]

PREC_FP32, PREC_FP16, PREC_BF16 = 0, 1, 2
LAYOUT_OCTREE, LAYOUT_BRICKS = 0, 1
LAYOUT_DEFAULT = LAYOUT_OCTREE
TRANS_EXP, TRANS_LINEAR, TRANS_LINEAR_LITERAL = 0, 1, 2
ACT_RELU, ACT_SIGMOID = 0, 1
PROXY_BOX, PROXY_SPHERE = 0, 1
RAY_OK, RAY_STEP_LIMIT, RAY_INVALID = 0, 1, 3

STATUS_NAMES = {0: "PLO_OK", -1: "PLO_ERR_INVALID_ARG", -2: "PLO_ERR_BAD_TREE", -3: "PLO_ERR_OOM",
                -4: "PLO_ERR_CUDA", -5: "PLO_ERR_TRAVERSAL_LIMIT", -6: "PLO_ERR_TIMEOUT",
                -7: "PLO_ERR_UNSUPPORTED"}


class PloError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


class TreeDesc(ctypes.Structure):
    _fields_ = [("depth", ctypes.c_int32), ("sh_degree", ctypes.c_int32),
                ("n_nodes", ctypes.c_int64), ("n_leaves", ctypes.c_int64),
                ("child", ctypes.c_void_p), ("sigma", ctypes.c_void_p), ("sh", ctypes.c_void_p),
                ("bbox_min", ctypes.c_float * 3), ("bbox_max", ctypes.c_float * 3)]


class _RenderParams(ctypes.Structure):
    _fields_ = [("transmittance", ctypes.c_int32), ("activation", ctypes.c_int32),
                ("l_max", ctypes.c_float), ("t_stop", ctypes.c_float), ("sigma_min", ctypes.c_float),
                ("max_steps", ctypes.c_int32), ("saturate", ctypes.c_int32), ("proxy", ctypes.c_int32),
                ("sphere", ctypes.c_float * 4)]


class TreeInfo(ctypes.Structure):
    _fields_ = [("depth", ctypes.c_int32), ("sh_degree", ctypes.c_int32), ("precision", ctypes.c_int32),
                ("top_levels", ctypes.c_int32), ("n_nodes", ctypes.c_int64), ("n_leaves", ctypes.c_int64),
                ("n_sh_records", ctypes.c_int64), ("node_bytes", ctypes.c_int64), ("sh_bytes", ctypes.c_int64),
                ("sh_record_stride", ctypes.c_int32), ("device", ctypes.c_int32), ("layout", ctypes.c_int32),
                ("brick_log", ctypes.c_int32), ("n_bricks", ctypes.c_int64), ("brick_bytes", ctypes.c_int64),
                ("top_nodes", ctypes.c_int64)]


class BuildOptions(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int32), ("layout", ctypes.c_int32), ("brick_log", ctypes.c_int32)]


@dataclass
class RenderParams:
    transmittance: int = TRANS_EXP
    activation: int = ACT_RELU
    l_max: float = 1.0
    t_stop: float = 0.0
    sigma_min: float = 0.0
    max_steps: int = 0
    saturate: bool = False
    sphere: tuple | None = None  # (cx, cy, cz, radius) selects the sphere proxy

    def _c(self) -> _RenderParams:
        p = _RenderParams()
        p.transmittance, p.activation = self.transmittance, self.activation
        p.l_max, p.t_stop, p.sigma_min, p.max_steps = self.l_max, self.t_stop, self.sigma_min, self.max_steps
        p.saturate = int(bool(self.saturate))
        p.proxy = PROXY_BOX if self.sphere is None else PROXY_SPHERE
        if self.sphere is not None:
            p.sphere[:] = tuple(float(v) for v in self.sphere)
        return p

    @classmethod
    def paper_heuristics(cls, **kw) -> "RenderParams":
        """sigma_min = 0.1 and alpha_max = 0.9 (t_stop = 0.1, saturated rays
        opaque), the values Sec. 6.2 sets empirically."""
        kw.setdefault("sigma_min", 0.1)
        kw.setdefault("t_stop", 0.1)
        kw.setdefault("saturate", True)
        return cls(**kw)


_lib = None


def load(build: bool = True) -> ctypes.CDLL:
    """Loads libplo.so (building it first when sources are newer)."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.build() if build else _build.LIB
    if not os.path.exists(path):
        raise RuntimeError(f"libplo.so not found at {path}; run __graft_entry__.build()")
    lib = ctypes.CDLL(path)
    P, I32, I64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64
    sigs = {
        "plo_validate_tree": (I32, [P]),
        "plo_build_tree": (I32, [P, I32, P]),
        "plo_build_tree_ex": (I32, [P, P, P]),
        "plo_tree_free": (None, [P]),
        "plo_tree_get_info": (I32, [P, P]),
        "plo_render_rays": (I32, [P, P, I64, P, P, P, P, P]),
        "plo_render_rays_host": (I32, [P, P, I64, P, P, P, P]),
        "plo_render_rays_host_noalloc": (I32, [P, P, I64, P, P, P, P]),
        "plo_lookup_points": (I32, [P, P, P, I64, P, P, P]),
        "plo_trace_rays": (I32, [P, P, I64, P, I32, P, P, P, P]),
        "plo_tree_check": (I32, [P, P]),
        "plo_last_error": (ctypes.c_char_p, []),
        "plo_version": (ctypes.c_char_p, []),
    }
    for name, (res, args) in sigs.items():
        fn = getattr(lib, name)
        fn.restype, fn.argtypes = res, args
    _lib = lib
    return lib


def _check(status: int):
    if status != 0:
        raise PloError(status, load().plo_last_error().decode())


def _desc(host_tree):
    """ctypes descriptor for a canonical host tree (keeps arrays alive)."""
    child = np.ascontiguousarray(host_tree.child, np.int32)
    sigma = np.ascontiguousarray(host_tree.sigma, np.float32)
    sh = np.ascontiguousarray(host_tree.sh, np.float32)
    d = TreeDesc()
    d.depth, d.sh_degree = int(host_tree.depth), int(host_tree.sh_degree)
    d.n_nodes, d.n_leaves = child.shape[0], sigma.shape[0]
    d.child = child.ctypes.data if child.size else None
    d.sigma = sigma.ctypes.data if sigma.size else None
    d.sh = sh.ctypes.data if sh.size else None
    d.bbox_min[:] = tuple(getattr(host_tree, "bbox_min", (0.0, 0.0, 0.0)))
    d.bbox_max[:] = tuple(getattr(host_tree, "bbox_max", (1.0, 1.0, 1.0)))
    return d, (child, sigma, sh)


def validate(host_tree) -> None:
    """Host-only validation of a canonical tree (raises PloError)."""
    d, keep = _desc(host_tree)
    _check(load().plo_validate_tree(ctypes.byref(d)))


def _stream(stream=None):
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else None


def _require(t, name: str, shape, dtype, cuda: bool = True):
    """Checks a caller-supplied tensor before its pointer reaches the library,
    which trusts the sizes it is given: dtype, exact shape, contiguity, and
    device memory (cuda) or host memory."""
    shape = tuple(int(x) for x in shape)
    if t.dtype != dtype or tuple(t.shape) != shape or not t.is_contiguous():
        raise ValueError(f"{name} must be a contiguous {dtype} tensor of shape {shape}, "
                         f"got {t.dtype} {tuple(t.shape)}{'' if t.is_contiguous() else ' (not contiguous)'}")
    if bool(t.is_cuda) != cuda:
        raise ValueError(f"{name} must be in {'CUDA device' if cuda else 'host'} memory")


def _require_rays_targets(rays, rgb_gt, alpha_gt):
    """Training rays [R, 6] with targets rgb [R, 3] and alpha [R] on the device."""
    import torch
    if rays.ndim != 2:
        raise ValueError("rays must have shape [n_rays, 6]")
    R = rays.shape[0]
    _require_all((rays, "rays", (R, 6), torch.float32), (rgb_gt, "rgb_gt", (R, 3), torch.float32),
                 (alpha_gt, "alpha_gt", (R,), torch.float32))


def _require_all(*specs, cuda: bool = True):
    """_require over several (tensor, name, shape, dtype) specs (None tensors
    skipped): every shape, dtype and layout first, then every device, so a
    caller learns of the first malformed buffer whatever memory it is in."""
    specs = [sp for sp in specs if sp[0] is not None]
    for t, name, shape, dtype in specs:
        _require(t, name, shape, dtype, cuda=bool(t.is_cuda))
    for t, name, shape, dtype in specs:
        _require(t, name, shape, dtype, cuda=cuda)


def _require_np(a, name: str, shape, dtype):
    """The same for a numpy array in host memory."""
    shape = tuple(int(x) for x in shape)
    if a.dtype != dtype or a.shape != shape or not a.flags.c_contiguous:
        raise ValueError(f"{name} must be a C-contiguous {np.dtype(dtype)} array of shape {shape}, "
                         f"got {a.dtype} {a.shape}")


class Tree:
    """A packed plenoctree on the current CUDA device (plo_build_tree)."""

    def __init__(self, host_tree, precision: int = PREC_FP32, layout: int = LAYOUT_DEFAULT, brick_log: int = 0):
        lib = load()
        d, keep = _desc(host_tree)
        h = ctypes.c_void_p()
        opt = BuildOptions(precision, layout, brick_log)
        _check(lib.plo_build_tree_ex(ctypes.byref(d), ctypes.byref(opt), ctypes.byref(h)))
        self._h = h
        self.precision = precision
        self.layout = layout

    @property
    def handle(self):
        return self._h

    def info(self) -> dict:
        inf = TreeInfo()
        _check(load().plo_tree_get_info(self._h, ctypes.byref(inf)))
        return {k: getattr(inf, k) for k, _ in TreeInfo._fields_}

    def check(self, stream=None) -> None:
        _check(load().plo_tree_check(self._h, _stream(stream)))

    def export(self):
        """plo_tree_export: the packed tree as a canonical host tree (plogen
        HostTree; 16-bit leaves dequantised)."""
        from plogen import HostTree
        inf = self.info()
        K = (inf["sh_degree"] + 1) ** 2
        child = np.empty((inf["n_nodes"], 8), np.int32)
        sigma = np.empty(inf["n_leaves"], np.float32)
        sh = np.empty((inf["n_leaves"], 3, K), np.float32)
        lib = load()
        fn = lib.plo_tree_export
        fn.restype, fn.argtypes = ctypes.c_int32, [ctypes.c_void_p] * 4
        _check(fn(self._h, ctypes.c_void_p(child.ctypes.data), ctypes.c_void_p(sigma.ctypes.data),
                  ctypes.c_void_p(sh.ctypes.data)))
        return HostTree(inf["depth"], inf["sh_degree"], child, sigma, sh)

    def free(self):
        if getattr(self, "_h", None) and self._h.value:
            load().plo_tree_free(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


def render(tree: Tree, rays, params: RenderParams | None = None, rgb=None, T=None, status=None, stream=None):
    """plo_render_rays on CUDA tensors: rays float32 [n, 6] -> (rgb [n,3], T [n], status [n] or None)."""
    import torch
    params = params or RenderParams()
    if not (rays.is_cuda and rays.dtype == torch.float32 and rays.is_contiguous() and rays.ndim == 2
            and rays.shape[1] == 6):
        raise ValueError("rays must be a contiguous float32 CUDA tensor of shape [n, 6]")
    n = rays.shape[0]
    rgb = rgb if rgb is not None else torch.empty((n, 3), device=rays.device, dtype=torch.float32)
    T = T if T is not None else torch.empty(n, device=rays.device, dtype=torch.float32)
    _require(rgb, "rgb", (n, 3), torch.float32)
    _require(T, "T", (n,), torch.float32)
    if status is not None:
        _require(status, "status", (n,), torch.int32)
    p = params._c()
    _check(load().plo_render_rays(tree.handle, _ptr(rays), n, ctypes.byref(p), _ptr(rgb), _ptr(T), _ptr(status),
                                  _stream(stream)))
    return rgb, T, status


def render_host(tree: Tree, rays: np.ndarray, params: RenderParams | None = None, rgb=None, T=None, stream=None):
    """plo_render_rays_host: rays in host memory (numpy or pinned CPU tensor)."""
    params = params or RenderParams()
    import torch
    if isinstance(rays, torch.Tensor):
        n = rays.shape[0]
        _require(rays, "rays", (n, 6), torch.float32, cuda=False)
        rp = rays.data_ptr()
        rgb = rgb if rgb is not None else torch.empty((n, 3), dtype=torch.float32, pin_memory=rays.is_pinned())
        T = T if T is not None else torch.empty(n, dtype=torch.float32, pin_memory=rays.is_pinned())
        _require(rgb, "rgb", (n, 3), torch.float32, cuda=False)
        _require(T, "T", (n,), torch.float32, cuda=False)
        op, tp = rgb.data_ptr(), T.data_ptr()
    else:
        rays = np.ascontiguousarray(rays, np.float32)
        if rays.ndim != 2 or rays.shape[1] != 6:
            raise ValueError(f"rays must have shape [n, 6], got {rays.shape}")
        n = rays.shape[0]
        rp = rays.ctypes.data
        rgb = rgb if rgb is not None else np.empty((n, 3), np.float32)
        T = T if T is not None else np.empty(n, np.float32)
        _require_np(rgb, "rgb", (n, 3), np.float32)
        _require_np(T, "T", (n,), np.float32)
        op, tp = rgb.ctypes.data, T.ctypes.data
    p = params._c()
    _check(load().plo_render_rays_host(tree.handle, ctypes.c_void_p(rp), n, ctypes.byref(p), ctypes.c_void_p(op),
                                       ctypes.c_void_p(tp), _stream(stream)))
    return rgb, T


NOALLOC_MAX_RAYS = 262144


def render_host_noalloc(tree: Tree, rays: np.ndarray, params: RenderParams | None = None, stream=None):
    """plo_render_rays_host_noalloc: host rays (numpy, at most NOALLOC_MAX_RAYS)
    staged through the library's fixed device array; allocates no device
    memory.  Returns (rgb [n,3], T [n]) as numpy arrays."""
    params = params or RenderParams()
    rays = np.ascontiguousarray(rays, np.float32)
    if rays.ndim != 2 or rays.shape[1] != 6:
        raise ValueError(f"rays must have shape [n, 6], got {rays.shape}")
    n = rays.shape[0]
    rgb = np.empty((n, 3), np.float32)
    T = np.empty(n, np.float32)
    p = params._c()
    _check(load().plo_render_rays_host_noalloc(tree.handle, ctypes.c_void_p(rays.ctypes.data), n, ctypes.byref(p),
                                               ctypes.c_void_p(rgb.ctypes.data), ctypes.c_void_p(T.ctypes.data),
                                               _stream(stream)))
    return rgb, T


def lookup(tree: Tree, points, dirs=None, stream=None):
    """plo_lookup_points: points float32 [n,3] CUDA -> (leaf int64 [n], level int32 [n])."""
    import torch
    n = points.shape[0]
    _require(points, "points", (n, 3), torch.float32)
    if dirs is not None:
        _require(dirs, "dirs", (n, 3), torch.float32)
    leaf = torch.empty(n, device=points.device, dtype=torch.int64)
    level = torch.empty(n, device=points.device, dtype=torch.int32)
    _check(load().plo_lookup_points(tree.handle, _ptr(points), _ptr(dirs), n, _ptr(leaf), _ptr(level),
                                    _stream(stream)))
    return leaf, level


def trace(tree: Tree, rays, max_cells: int, params: RenderParams | None = None, stream=None):
    """plo_trace_rays: -> (leaf int64 [n, max_cells], t float32 [n, max_cells, 2], count int32 [n])."""
    import torch
    params = params or RenderParams()
    n = rays.shape[0]
    _require(rays, "rays", (n, 6), torch.float32)
    leaf = torch.full((n, max_cells), -3, device=rays.device, dtype=torch.int64)
    t = torch.zeros((n, max_cells, 2), device=rays.device, dtype=torch.float32)
    cnt = torch.zeros(n, device=rays.device, dtype=torch.int32)
    p = params._c()
    _check(load().plo_trace_rays(tree.handle, _ptr(rays), n, ctypes.byref(p), max_cells, _ptr(leaf), _ptr(t),
                                 _ptr(cnt), _stream(stream)))
    return leaf, t, cnt


# ---------------------------------------------------------------- learned part
LOSS_PAPER, LOSS_REG, LOSS_MSE = 0, 1, 2
MLP_DZ_BASE = 16
ARCH_LINEAR_HEAD, ARCH_PAPER = 0, 1


class MlpDesc(ctypes.Structure):
    _fields_ = [("sh_degree", ctypes.c_int32), ("transmittance", ctypes.c_int32), ("loss", ctypes.c_int32),
                ("total_steps", ctypes.c_int32), ("l_max", ctypes.c_float), ("eps", ctypes.c_float),
                ("lr0", ctypes.c_float), ("lr1", ctypes.c_float), ("init_radiance", ctypes.c_float),
                ("arch", ctypes.c_int32), ("seed", ctypes.c_uint64)]


def _load_mlp_sigs(lib):
    P, I32, I64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64
    sigs = {
        "plo_mlp_param_count": (I64, [I32]),
        "plo_mlp_param_count_arch": (I64, [I32, I32]),
        "plo_mlp_train_step_hier": (I32, [P, P, P, P, P, I32, I32, I32, P, P, P, P]),
        "plo_hier_samples": (I32, [P, I32, I32, I32, P, P, P, P, P, P, P]),
        "plo_mlp_create": (I32, [P, ctypes.c_uint64, P]),
        "plo_mlp_free": (None, [P]),
        "plo_mlp_set_params": (I32, [P, P, I64]),
        "plo_mlp_get_params": (I32, [P, P, I64]),
        "plo_mlp_get_grads": (I32, [P, P, I64]),
        "plo_mlp_forward": (I32, [P, P, I64, P, P]),
        "plo_mlp_train_step": (I32, [P, P, P, P, I32, I32, P, P, P]),
        "plo_mlp_check": (I32, [P, P]),
        "plo_mlp_step": (I64, [P]),
        "plo_gemm_bf16": (I32, [P, P, I32, I32, I32, I32, P, P, P, P, P, P]),
        "plo_wgrad_bf16": (I32, [P, I32, P, I32, I32, P, P, P, P]),
        "plo_distill": (I32, [P, I32, I32, ctypes.c_float, I32, P, P]),
        "plo_mlp_save": (I32, [P, ctypes.c_char_p]),
        "plo_mlp_load": (I32, [ctypes.c_char_p, P]),
        "plo_mlp_checkpoint_info": (I32, [ctypes.c_char_p, P, P]),
        "plo_mlp_get_activation": (I32, [P, I32, P, I64, P]),
        "plo_mlp_quad": (I32, [P, P, P, P, P, P, I32, I32, P, P, P]),
    }
    for name, (res, args) in sigs.items():
        fn = getattr(lib, name)
        fn.restype, fn.argtypes = res, args


def mlp_lib():
    lib = load()
    if not getattr(lib, "_mlp_sigs", False):
        _load_mlp_sigs(lib)
        lib._mlp_sigs = True
    return lib


class Mlp:
    """The NeRF-SH network on the current device (plo_mlp_*)."""

    def __init__(self, l_max: float, loss: int = LOSS_PAPER, transmittance: int = TRANS_EXP, total_steps: int = 1000,
                 lr0: float = 5e-4, lr1: float = 5e-6, eps: float = 0.01, seed: int = 1, jitter_seed: int = 2,
                 init_radiance: float = 0.0, arch: int = ARCH_LINEAR_HEAD):
        lib = mlp_lib()
        d = MlpDesc()
        d.sh_degree, d.transmittance, d.loss, d.total_steps = 3, transmittance, loss, total_steps
        d.l_max, d.eps, d.lr0, d.lr1, d.seed = l_max, eps, lr0, lr1, jitter_seed
        d.init_radiance, d.arch = init_radiance, arch
        h = ctypes.c_void_p()
        _check(lib.plo_mlp_create(ctypes.byref(d), seed, ctypes.byref(h)))
        self._h = h
        self.arch = arch
        self.n_params = int(lib.plo_mlp_param_count_arch(3, arch))

    @property
    def handle(self):
        return self._h

    def set_params(self, flat: np.ndarray):
        flat = np.ascontiguousarray(flat, np.float32)
        _check(mlp_lib().plo_mlp_set_params(self._h, ctypes.c_void_p(flat.ctypes.data), flat.size))

    def get_params(self) -> np.ndarray:
        out = np.empty(self.n_params, np.float32)
        _check(mlp_lib().plo_mlp_get_params(self._h, ctypes.c_void_p(out.ctypes.data), out.size))
        return out

    def get_grads(self) -> np.ndarray:
        out = np.empty(self.n_params, np.float32)
        _check(mlp_lib().plo_mlp_get_grads(self._h, ctypes.c_void_p(out.ctypes.data), out.size))
        return out

    def forward(self, points, stream=None):
        import torch
        n = points.shape[0]
        _require(points, "points", (n, 3), torch.float32)
        raw = torch.empty((n, 49), device=points.device, dtype=torch.float32)
        _check(mlp_lib().plo_mlp_forward(self._h, _ptr(points), n, _ptr(raw), _stream(stream)))
        return raw

    def train_step(self, rays, rgb_gt, alpha_gt, n_samples: int = 128, jitter=None, loss_out=None, stream=None):
        import torch
        R = rays.shape[0] if rays.ndim == 2 else -1
        _require_all((jitter, "jitter", (R, n_samples), torch.float32),
                     (loss_out, "loss_out", (1,), torch.float32))
        _require_rays_targets(rays, rgb_gt, alpha_gt)
        loss_out = loss_out if loss_out is not None else torch.empty(1, device=rays.device, dtype=torch.float32)
        _check(mlp_lib().plo_mlp_train_step(self._h, _ptr(rays), _ptr(rgb_gt), _ptr(alpha_gt), rays.shape[0],
                                            n_samples, _ptr(jitter), _ptr(loss_out), _stream(stream)))
        return loss_out

    def check(self, stream=None):
        _check(mlp_lib().plo_mlp_check(self._h, _stream(stream)))

    @staticmethod
    def train_step_hier(coarse: "Mlp", fine: "Mlp", rays, rgb_gt, alpha_gt, n_coarse: int = 64, n_fine: int = 128,
                        jitter=None, xi=None, loss_out=None, stream=None):
        """plo_mlp_train_step_hier: one coarse/fine step (Sec. 4.3-4.4)."""
        import torch
        R = rays.shape[0] if rays.ndim == 2 else -1
        _require_all((jitter, "jitter", (R, n_coarse), torch.float32), (xi, "xi", (R, n_fine), torch.float32),
                     (loss_out, "loss_out", (1,), torch.float32))
        _require_rays_targets(rays, rgb_gt, alpha_gt)
        loss_out = loss_out if loss_out is not None else torch.empty(1, device=rays.device, dtype=torch.float32)
        _check(mlp_lib().plo_mlp_train_step_hier(coarse._h, fine._h, _ptr(rays), _ptr(rgb_gt), _ptr(alpha_gt),
                                                 rays.shape[0], n_coarse, n_fine, _ptr(jitter), _ptr(xi),
                                                 _ptr(loss_out), _stream(stream)))
        return loss_out

    def distill(self, depth: int, samples: int = 8, sigma_thresh: float = 0.01, precision: int = PREC_FP32,
                stream=None) -> "Tree":
        """plo_distill: the network as a plenoctree of the given depth."""
        h = ctypes.c_void_p()
        _check(mlp_lib().plo_distill(self._h, depth, samples, sigma_thresh, precision, ctypes.byref(h),
                                     _stream(stream)))
        t = Tree.__new__(Tree)
        t._h = h
        t.precision = precision
        return t

    @property
    def step(self) -> int:
        return int(mlp_lib().plo_mlp_step(self._h))

    def save(self, path: str) -> None:
        """plo_mlp_save: the network and its Adam state to a checkpoint file."""
        _check(mlp_lib().plo_mlp_save(self._h, os.fsencode(path)))

    @classmethod
    def load(cls, path: str) -> "Mlp":
        """plo_mlp_load: a network on the current device from a checkpoint."""
        lib = mlp_lib()
        h = ctypes.c_void_p()
        _check(lib.plo_mlp_load(os.fsencode(path), ctypes.byref(h)))
        desc = MlpDesc()
        _check(lib.plo_mlp_checkpoint_info(os.fsencode(path), ctypes.byref(desc), None))
        net = cls.__new__(cls)
        net._h = h
        net.arch = desc.arch
        net.n_params = int(lib.plo_mlp_param_count_arch(desc.sh_degree, desc.arch))
        return net

    def activation(self, layer: int, n_rows: int, stream=None):
        """plo_mlp_get_activation: bf16 input of `layer` for the first n_rows
        samples of the last forward or training step."""
        import torch
        cols = 64 if layer == 0 else (128 if layer == 9 else 256)  # MLP_DZ_BASE + l: d loss / d Z_l
        out = torch.empty((n_rows, cols), device="cuda", dtype=torch.bfloat16)
        _check(mlp_lib().plo_mlp_get_activation(self._h, layer, _ptr(out), n_rows, _stream(stream)))
        return out

    def quad(self, rays, raw, delta, rgb_gt, alpha_gt, n_samples: int, stream=None):
        """plo_mlp_quad: (ray_out [R, 5] = C^ rgb, alpha^, loss; d loss / d raw
        [R * n_samples, 49]) for given raw outputs and segment lengths."""
        import torch
        R = rays.shape[0] if rays.ndim == 2 else -1
        M = R * n_samples
        _require_all((raw, "raw", (M, 49), torch.float32), (delta, "delta", (M,), torch.float32))
        _require_rays_targets(rays, rgb_gt, alpha_gt)
        ray_out = torch.empty((R, 5), device=rays.device, dtype=torch.float32)
        draw = torch.empty((M, 49), device=rays.device, dtype=torch.float32)
        _check(mlp_lib().plo_mlp_quad(self._h, _ptr(rays), _ptr(raw), _ptr(delta), _ptr(rgb_gt), _ptr(alpha_gt),
                                      R, n_samples, _ptr(ray_out), _ptr(draw), _stream(stream)))
        return ray_out, draw


    def free(self):
        if getattr(self, "_h", None) and self._h.value:
            mlp_lib().plo_mlp_free(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


def checkpoint_info(path: str) -> tuple[dict, int]:
    """plo_mlp_checkpoint_info: (network description, step) of a checkpoint
    file, read on the host without a GPU."""
    lib = mlp_lib()
    desc = MlpDesc()
    step = ctypes.c_int64()
    _check(lib.plo_mlp_checkpoint_info(os.fsencode(path), ctypes.byref(desc), ctypes.byref(step)))
    return {k: getattr(desc, k) for k, _ in MlpDesc._fields_}, int(step.value)


def gemm_bf16(A, B, epilogue: int, bias=None, mask=None, out=None, err=None, bits=None, stream=None):
    """plo_gemm_bf16 on CUDA tensors (A [M][K], B [N][K] bf16); bits: int32
    [M][N / 32], written by epilogue 0 and read by epilogue 3."""
    import torch
    if A.ndim != 2 or B.ndim != 2:
        raise ValueError("A and B must be 2-D")
    M, K = A.shape
    N = B.shape[0]
    odt = torch.float32 if epilogue == 1 else torch.bfloat16
    _require_all((A, "A", (M, K), torch.bfloat16), (B, "B", (N, K), torch.bfloat16),
                 (bias, "bias", (N,), torch.float32), (mask, "mask", (M, N), torch.bfloat16),
                 (bits, "bits", (M, N // 32), torch.int32), (out, "out", (M, N), odt),
                 (err, "err", (1,), torch.int32))
    if out is None:
        out = torch.empty((M, N), device=A.device, dtype=odt)
    err = err if err is not None else torch.zeros(1, device=A.device, dtype=torch.int32)
    _check(mlp_lib().plo_gemm_bf16(_ptr(A), _ptr(B), M, N, K, epilogue, _ptr(bias), _ptr(mask), _ptr(bits), _ptr(out),
                                   _ptr(err), _stream(stream)))
    return out, err


def hier_samples(rays, t, delta, w, xi, stream=None):
    """plo_hier_samples: merged coarse + fine parameters and lengths
    ([n_rays][n_coarse + n_fine]) for coarse t, delta, w and fine xi."""
    import torch
    if t.ndim != 2 or xi.ndim != 2:
        raise ValueError("t and xi must be 2-D")
    n, nc = t.shape
    nf = xi.shape[1]
    f32 = torch.float32
    _require_all((rays, "rays", (n, 6), f32), (t, "t", (n, nc), f32), (delta, "delta", (n, nc), f32),
                 (w, "w", (n, nc), f32), (xi, "xi", (n, nf), f32))
    t_out = torch.empty((n, nc + nf), device=t.device, dtype=torch.float32)
    d_out = torch.empty_like(t_out)
    _check(mlp_lib().plo_hier_samples(_ptr(rays), n, nc, nf, _ptr(t), _ptr(delta), _ptr(w), _ptr(xi), _ptr(t_out),
                                      _ptr(d_out), _stream(stream)))
    return t_out, d_out


def wgrad_bf16(dZ, H, dW, db=None, err=None, stream=None):
    """plo_wgrad_bf16: dW [n_out][n_in] (fp32) += dZ^T H; db [n_out] (fp32,
    optional) += the column sums of dZ."""
    import torch
    if dZ.ndim != 2 or H.ndim != 2:
        raise ValueError("dZ and H must be 2-D")
    M, n_out = dZ.shape
    n_in = H.shape[1]
    _require_all((dZ, "dZ", (M, n_out), torch.bfloat16), (H, "H", (M, n_in), torch.bfloat16),
                 (dW, "dW", (n_out, n_in), torch.float32), (db, "db", (n_out,), torch.float32),
                 (err, "err", (1,), torch.int32))
    err = err if err is not None else torch.zeros(1, device=dZ.device, dtype=torch.int32)
    _check(mlp_lib().plo_wgrad_bf16(_ptr(dZ), dZ.shape[1], _ptr(H), H.shape[1], dZ.shape[0], _ptr(dW), _ptr(db),
                                    _ptr(err), _stream(stream)))
    return dW, err


# ---------------------------------------------------------------- path tracer with the luminaire as emitter
PT_OCTREE, PT_CONSTANT_BOX = 0, 1


OCTOPT_SIGMA, OCTOPT_SH, OCTOPT_GRAD_SIGMA, OCTOPT_GRAD_SH, OCTOPT_NEIGHBOURS = 0, 1, 2, 3, 4


class OctOptConfig(ctypes.Structure):
    _fields_ = [("transmittance", ctypes.c_int32), ("loss", ctypes.c_int32), ("l_max", ctypes.c_float),
                ("eps", ctypes.c_float), ("lr_sigma", ctypes.c_float), ("lr_sh", ctypes.c_float),
                ("lr_decay", ctypes.c_float), ("total_steps", ctypes.c_int32), ("tv_sigma", ctypes.c_float),
                ("tv_sh", ctypes.c_float), ("max_rays", ctypes.c_int64), ("max_cells", ctypes.c_int32)]


def _octopt_lib():
    lib = load()
    if not getattr(lib, "_octopt_sigs", False):
        P, I32, I64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64
        sigs = {
            "plo_octopt_create": (I32, [P, P, P]),
            "plo_octopt_free": (None, [P]),
            "plo_octopt_grad": (I32, [P, P, P, P, I64, P, P, P]),
            "plo_octopt_step": (I32, [P, P, P, P, I64, P, P, P]),
            "plo_octopt_read": (I32, [P, I32, P, P]),
            "plo_octopt_write": (I32, [P, I32, P, P]),
            "plo_octopt_check": (I32, [P, P]),
            "plo_octopt_build_tree": (I32, [P, P, P]),
        }
        for name, (res, args) in sigs.items():
            fn = getattr(lib, name)
            fn.restype, fn.argtypes = res, args
        lib._octopt_sigs = True
    return lib


class OctOpt:
    """Direct optimisation of an octree's leaves (plo_octopt_*): raw
    densities and SH coefficients fitted to rendered targets with the
    paper's loss, TV regularisers and Adam, on the structure of `init`."""

    def __init__(self, init, l_max: float, max_rays: int, loss: int = LOSS_PAPER, transmittance: int = TRANS_EXP,
                 eps: float = 0.01, lr_sigma: float = 0.1, lr_sh: float = 0.05, lr_decay: float = 0.1,
                 total_steps: int = 1000, tv_sigma: float = 0.0, tv_sh: float = 0.0, max_cells: int = 0):
        lib = _octopt_lib()
        d, keep = _desc(init)
        c = OctOptConfig(transmittance, loss, l_max, eps, lr_sigma, lr_sh, lr_decay, total_steps, tv_sigma, tv_sh,
                         max_rays, max_cells)
        h = ctypes.c_void_p()
        _check(lib.plo_octopt_create(ctypes.byref(d), ctypes.byref(c), ctypes.byref(h)))
        self._h = h
        self.n_leaves = int(init.sigma.shape[0])
        self.K = (int(init.sh_degree) + 1) ** 2
        self.max_rays = int(max_rays)

    @property
    def handle(self):
        return self._h

    def _run(self, fn, rays, rgb_gt, alpha_gt, ray_out, loss_out, stream):
        import torch
        R = rays.shape[0] if rays.ndim == 2 else -1
        if R > self.max_rays:
            raise ValueError(f"{R} rays exceed max_rays = {self.max_rays}")
        _require_all((ray_out, "ray_out", (R, 5), torch.float32), (loss_out, "loss_out", (3,), torch.float32))
        _require_rays_targets(rays, rgb_gt, alpha_gt)
        loss_out = loss_out if loss_out is not None else torch.empty(3, device=rays.device, dtype=torch.float32)
        _check(fn(self._h, _ptr(rays), _ptr(rgb_gt), _ptr(alpha_gt), R, _ptr(ray_out), _ptr(loss_out),
                  _stream(stream)))
        return loss_out

    def grad(self, rays, rgb_gt, alpha_gt, ray_out=None, loss_out=None, stream=None):
        """plo_octopt_grad; returns the device tensor (mean loss, TV(s), TV(k))."""
        return self._run(_octopt_lib().plo_octopt_grad, rays, rgb_gt, alpha_gt, ray_out, loss_out, stream)

    def step(self, rays, rgb_gt, alpha_gt, ray_out=None, loss_out=None, stream=None):
        """plo_octopt_step (gradient and one Adam update)."""
        return self._run(_octopt_lib().plo_octopt_step, rays, rgb_gt, alpha_gt, ray_out, loss_out, stream)

    def _shape(self, what):
        if what in (OCTOPT_SIGMA, OCTOPT_GRAD_SIGMA):
            return (self.n_leaves,), np.float32
        if what in (OCTOPT_SH, OCTOPT_GRAD_SH):
            return (self.n_leaves, 3, self.K), np.float32
        if what == OCTOPT_NEIGHBOURS:
            return (self.n_leaves, 3), np.int32
        raise ValueError(f"unknown array {what}")

    def read(self, what: int) -> np.ndarray:
        """One PLO_OCTOPT_* array, copied to the host (synchronous)."""
        import torch
        shape, dt = self._shape(what)
        out = np.empty(shape, dt)
        lib = _octopt_lib()
        _check(lib.plo_octopt_read(self._h, what, ctypes.c_void_p(out.ctypes.data), _stream(None)))
        torch.cuda.current_stream().synchronize()
        return out

    def write(self, what: int, values: np.ndarray) -> None:
        import torch
        shape, dt = self._shape(what)
        values = np.ascontiguousarray(values, dt)
        _require_np(values, "values", shape, dt)
        _check(_octopt_lib().plo_octopt_write(self._h, what, ctypes.c_void_p(values.ctypes.data), _stream(None)))
        torch.cuda.current_stream().synchronize()

    def check(self, stream=None) -> None:
        _check(_octopt_lib().plo_octopt_check(self._h, _stream(stream)))

    def build_tree(self, precision: int = PREC_FP32, layout: int = LAYOUT_DEFAULT, brick_log: int = 0) -> "Tree":
        """plo_octopt_build_tree: the current parameters as a renderable Tree
        (render it with ACT_SIGMOID and this optimiser's l_max)."""
        t = Tree.__new__(Tree)
        h = ctypes.c_void_p()
        opt = BuildOptions(precision, layout, brick_log)
        _check(_octopt_lib().plo_octopt_build_tree(self._h, ctypes.byref(opt), ctypes.byref(h)))
        t._h, t.precision, t.layout = h, precision, layout
        return t

    def free(self):
        if getattr(self, "_h", None) and self._h.value:
            _octopt_lib().plo_octopt_free(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


class PtScene(ctypes.Structure):
    _fields_ = [("room_min", ctypes.c_float * 3), ("room_max", ctypes.c_float * 3),
                ("albedo", (ctypes.c_float * 3) * 6), ("cam_pos", ctypes.c_float * 3),
                ("cam_target", ctypes.c_float * 3), ("cam_up", ctypes.c_float * 3), ("fov_y", ctypes.c_float),
                ("width", ctypes.c_int32), ("height", ctypes.c_int32), ("max_bounces", ctypes.c_int32),
                ("emitter", ctypes.c_int32), ("box_radiance", ctypes.c_float * 3)]

    @classmethod
    def from_dict(cls, sc: dict) -> "PtScene":
        s = cls()
        for k in ("room_min", "room_max", "cam_pos", "cam_target", "cam_up", "box_radiance"):
            getattr(s, k)[:] = tuple(float(v) for v in sc[k])
        for w in range(6):
            s.albedo[w][:] = tuple(float(v) for v in sc["albedo"][w])
        s.fov_y = float(sc["fov_y"])
        s.width, s.height = int(sc["width"]), int(sc["height"])
        s.max_bounces, s.emitter = int(sc["max_bounces"]), int(sc["emitter"])
        return s


def pt_render(tree: Tree, scene: dict, spp: int, params: RenderParams | None = None, seed: int = 1, uniforms=None,
              samples: bool = False, stream=None):
    """plo_pt_render: (image [H, W, 3], per-sample radiance [spp, H, W, 3] or None)."""
    import torch
    lib = load()
    if not getattr(lib, "_pt_sigs", False):
        P = ctypes.c_void_p
        lib.plo_pt_render.restype = ctypes.c_int32
        lib.plo_pt_render.argtypes = [P, P, P, ctypes.c_int32, ctypes.c_uint64, P, P, P, P]
        lib._pt_sigs = True
    s = PtScene.from_dict(scene)
    if uniforms is not None:
        _require(uniforms, "uniforms", (spp * s.width * s.height, 2 + 5 * s.max_bounces), torch.float32)
    p = (params or RenderParams())._c()
    img = torch.empty((s.height, s.width, 3), device="cuda", dtype=torch.float32)
    smp = torch.empty((spp, s.height, s.width, 3), device="cuda", dtype=torch.float32) if samples else None
    _check(lib.plo_pt_render(tree.handle, ctypes.byref(p), ctypes.byref(s), spp, seed, _ptr(uniforms), _ptr(img),
                             _ptr(smp), _stream(stream)))
    return img, smp


# ---------------------------------------------------------------- batched render
class BatchConfig(ctypes.Structure):
    _fields_ = [("claim_rays", ctypes.c_int32), ("blocks_per_sm", ctypes.c_int32), ("top_nodes", ctypes.c_int32)]


def _batch_lib():
    lib = load()
    if not getattr(lib, "_batch_sigs", False):
        P, I32 = ctypes.c_void_p, ctypes.c_int32
        sigs = {
            "plo_batch_create": (I32, [P, I32, P, P, P]),
            "plo_batch_free": (None, [P]),
            "plo_batch_set_config": (I32, [P, P]),
            "plo_batch_get_config": (I32, [P, P]),
            "plo_batch_render": (I32, [P, P, P, P, P, P]),
            "plo_batch_capture": (I32, [P, P, P, P, P, P]),
            "plo_batch_replay": (I32, [P, P]),
            "plo_batch_autotune": (I32, [P, P, P, P, I32, P, P, P]),
        }
        for name, (res, args) in sigs.items():
            fn = getattr(lib, name)
            fn.restype, fn.argtypes = res, args
        lib._batch_sigs = True
    return lib


class Batch:
    """Several trees rendered by one persistent launch (plo_batch_*).  Rays of
    tree t are rows offsets[t]:offsets[t+1] of one concatenated array."""

    def __init__(self, trees, offsets, params: RenderParams | None = None):
        lib = _batch_lib()
        self._trees = list(trees)  # keep the trees alive
        arr = (ctypes.c_void_p * len(trees))(*[t.handle.value for t in trees])
        offs = np.ascontiguousarray(offsets, np.int64)
        self.n_rays = int(offs[-1])
        p = (params or RenderParams())._c()
        h = ctypes.c_void_p()
        _check(lib.plo_batch_create(arr, len(trees), ctypes.c_void_p(offs.ctypes.data), ctypes.byref(p),
                                    ctypes.byref(h)))
        self._h = h

    def config(self) -> dict:
        c = BatchConfig()
        _check(_batch_lib().plo_batch_get_config(self._h, ctypes.byref(c)))
        return {"claim_rays": c.claim_rays, "blocks_per_sm": c.blocks_per_sm, "top_nodes": c.top_nodes}

    def set_config(self, claim_rays: int, blocks_per_sm: int, top_nodes: int):
        c = BatchConfig(claim_rays, blocks_per_sm, top_nodes)
        _check(_batch_lib().plo_batch_set_config(self._h, ctypes.byref(c)))

    def _require_buffers(self, rays, rgb, T, status=None):
        import torch
        n = self.n_rays
        _require_all((rays, "rays", (n, 6), torch.float32), (rgb, "rgb", (n, 3), torch.float32),
                     (T, "T", (n,), torch.float32), (status, "status", (n,), torch.int32))

    def render(self, rays, rgb, T, status=None, stream=None):
        self._require_buffers(rays, rgb, T, status)
        _check(_batch_lib().plo_batch_render(self._h, _ptr(rays), _ptr(rgb), _ptr(T), _ptr(status), _stream(stream)))

    def capture(self, rays, rgb, T, status=None, stream=None):
        self._require_buffers(rays, rgb, T, status)
        _check(_batch_lib().plo_batch_capture(self._h, _ptr(rays), _ptr(rgb), _ptr(T), _ptr(status),
                                              _stream(stream)))

    def replay(self, stream=None):
        _check(_batch_lib().plo_batch_replay(self._h, _stream(stream)))

    def autotune(self, rays, rgb, T, reps: int = 2, stream=None):
        self._require_buffers(rays, rgb, T)
        c = BatchConfig()
        ms = ctypes.c_float()
        _check(_batch_lib().plo_batch_autotune(self._h, _ptr(rays), _ptr(rgb), _ptr(T), reps, _stream(stream),
                                               ctypes.byref(c), ctypes.byref(ms)))
        return {"claim_rays": c.claim_rays, "blocks_per_sm": c.blocks_per_sm, "top_nodes": c.top_nodes}, ms.value

    def free(self):
        if getattr(self, "_h", None) and self._h.value:
            _batch_lib().plo_batch_free(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


def autotune_cached(batch: "Batch", key: str, rays, rgb, T, reps: int = 2, path: str | None = None):
    """Applies the launch shape cached for (this GPU, key) in a JSON file
    (default ~/.cache/plo/autotune.json), autotuning and recording it when
    absent.  Returns (config, source) with source 'cache' or 'tuned'."""
    import json
    import torch
    path = path or os.path.join(os.path.expanduser("~"), ".cache", "plo", "autotune.json")
    gpu = torch.cuda.get_device_name()
    full = f"{gpu}|{key}"
    try:
        with open(path) as f:
            cache = json.load(f)
    except (OSError, ValueError):
        cache = {}
    if full in cache:
        c = cache[full]
        batch.set_config(c["claim_rays"], c["blocks_per_sm"], c["top_nodes"])
        return c, "cache"
    cfg, ms = batch.autotune(rays, rgb, T, reps=reps)
    cache[full] = dict(cfg, ms=ms)
    os.makedirs(os.path.dirname(path), exist_ok=True)
    tmp = path + f".{os.getpid()}.tmp"
    with open(tmp, "w") as f:
        json.dump(cache, f, indent=1)
    os.replace(tmp, path)
    return cfg, "tuned"


# ---------------------------------------------------------------- test hooks
def debug_fail_alloc_after(n: int) -> None:
    """The n-th following device allocation of the library fails (n < 0: off)."""
    lib = load()
    lib.plo_debug_fail_alloc_after.restype = None
    lib.plo_debug_fail_alloc_after.argtypes = [ctypes.c_int32]
    lib.plo_debug_fail_alloc_after(n)


def debug_gemm_stall(A, B, out, err, wait_limit: int, stream=None):
    """plo_debug_gemm_stall: a GEMM whose pipeline waits run out."""
    import torch
    M = A.shape[0]
    _require_all((A, "A", (M, 64), torch.bfloat16), (B, "B", (256, 64), torch.bfloat16),
                 (out, "out", (M, 256), torch.bfloat16), (err, "err", (1,), torch.int32))
    lib = load()
    fn = lib.plo_debug_gemm_stall
    fn.restype = ctypes.c_int32
    fn.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p,
                   ctypes.c_uint32, ctypes.c_void_p]
    _check(fn(_ptr(A), _ptr(B), A.shape[0], _ptr(out), _ptr(err), wait_limit, _stream(stream)))
