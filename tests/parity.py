"""Parity metrics between the CUDA path and the FP64 oracle, plus an
independent numpy emulation of the 16-bit leaf encoding (used to render the
exact dequantised tree with the oracle)."""
from __future__ import annotations

import numpy as np

from plogen import HostTree

# FP32 leaves: 1e-4 relative per channel; FP16 leaves: 2e-3 relative.
RTOL_FP32 = 1e-4
RTOL_FP16 = 2e-3


def radiance_errors(rgb, T, ref):
    """Per-ray, per-channel error relative to the oracle's error scale
    sum_i w_i sum_k |c_k Y_k| (which equals |L_e| when nothing cancels), and
    the transmittance error relative to max(T, 1e-3)."""
    rgb = np.asarray(rgb, np.float64)
    T = np.asarray(T, np.float64)
    scale = np.maximum(ref["bound"], 1e-30)
    e_c = np.abs(rgb - ref["rgb"]) / scale
    e_c[(ref["bound"] == 0) & (rgb == 0)] = 0.0
    e_T = np.abs(T - ref["T"]) / np.maximum(ref["T"], 1e-3)
    return e_c, e_T


def assert_radiance_close(rgb, T, ref, rtol, mask=None, what=""):
    e_c, e_T = radiance_errors(rgb, T, ref)
    if mask is not None:
        e_c, e_T = e_c[mask], e_T[mask]
    worst_c = float(e_c.max()) if e_c.size else 0.0
    worst_T = float(e_T.max()) if e_T.size else 0.0
    if worst_c > rtol or worst_T > rtol:
        i = int(np.argmax(e_c.max(axis=1))) if e_c.size else -1
        raise AssertionError(f"{what}: worst radiance error {worst_c:.3e}, worst T error {worst_T:.3e} "
                             f"(tolerance {rtol:g}); worst ray {i}")
    return worst_c, worst_T


def quantise_tree(tree: HostTree, precision: str) -> HostTree:
    """The tree the 16-bit leaves represent exactly: sigma rounded to
    binary16/bfloat16, and per leaf with non-zero SH, coefficients scaled by
    2^-e (e = frexp exponent of max|c|, clamped to [-126, 127]), rounded to
    nearest-even, and scaled back."""
    import torch

    def rnd(x32):
        if precision == "fp16":
            return x32.astype(np.float16).astype(np.float64)
        return torch.from_numpy(np.ascontiguousarray(x32)).to(torch.bfloat16).to(torch.float64).numpy()

    sig = rnd(tree.sigma.astype(np.float32)).astype(np.float32)
    sh = tree.sh.astype(np.float32).copy()
    flat = sh.reshape(sh.shape[0], -1)
    m = np.abs(flat).max(axis=1)
    nz = m > 0
    e = np.frexp(m)[1].astype(np.int64)
    e = np.clip(e, -126, 127)
    scaled = np.ldexp(flat, -e[:, None]).astype(np.float32)
    deq = np.ldexp(rnd(scaled), e[:, None])
    flat[nz] = deq[nz].astype(np.float32)
    return HostTree(tree.depth, tree.sh_degree, tree.child, sig, flat.reshape(sh.shape),
                    bbox_min=tree.bbox_min, bbox_max=tree.bbox_max)
