"""Parity metrics between the CUDA path and the FP64 oracle, plus an
independent numpy emulation of the 16-bit leaf encoding (used to render the
exact dequantised tree with the oracle)."""
from __future__ import annotations

import numpy as np

from plogen import HostTree

# FP32 leaves: 1e-4 relative per channel; FP16 leaves: 2e-3 relative.
RTOL_FP32 = 1e-4
RTOL_FP16 = 2e-3
# BF16 leaves: each coefficient keeps 8 significant bits, so its rounding
# error is at most 2^-8 (3.9e-3) of its magnitude and the SH sum's at most
# 2^-8 of sum_k |c_k Y_k|, the metric's scale; 4e-3 leaves 2% for the
# 24-bit density's 2^-17 relative error carried through the optical depth.
RTOL_BF16 = 4e-3


# Absolute radiance floor, relative to the largest error scale of the ray
# set: covers sliver segments (length ~1e-14 of t) at shared cell edges that
# one walk visits and the other does not.
ATOL_REL = 1e-9
# FP32 optical depths carry an absolute error ~2e-7 * OD (segment lengths
# and sigma * dt roundings); the linear models turn it into an absolute
# transmittance error (T = 1 - OD cancels), which moves the radiance by at
# most eta * cond with cond = sum_i OD_i |Phi_i| from the oracle.
COND_ETA_LINEAR = 1e-6


def radiance_errors(rgb, T, ref, rtol, cond_eta=0.0):
    """Normalised errors (<= 1 passes): per channel
    |g - o| / (rtol * bound + atol + cond_eta * cond), bound being the
    oracle's error scale sum_i w_i sum_k |c_k Y_k| (= |L_e| when nothing
    cancels); T: |g - o| / (rtol * max(T, 1e-3))."""
    rgb = np.asarray(rgb, np.float64)
    T = np.asarray(T, np.float64)
    atol = ATOL_REL * ref["bound"].max(axis=0, keepdims=True)
    scale = rtol * ref["bound"] + atol + cond_eta * ref["cond"] + 1e-300
    e_c = np.abs(rgb - ref["rgb"]) / scale
    e_c[(ref["bound"] == 0) & (rgb == ref["rgb"])] = 0.0
    e_T = np.abs(T - ref["T"]) / (rtol * np.maximum(ref["T"], 1e-3))
    return e_c, e_T


def relative_errors(rgb, T, ref):
    """Plain relative errors for reporting: max |g - o| / bound (channels with
    a non-zero scale) and max |T_g - T_o| / max(T_o, 1e-3)."""
    b = ref["bound"]
    m = b > 0
    e_c = (np.abs(np.asarray(rgb, np.float64) - ref["rgb"])[m] / b[m]).max() if m.any() else 0.0
    e_T = (np.abs(np.asarray(T, np.float64) - ref["T"]) / np.maximum(ref["T"], 1e-3)).max()
    return float(e_c), float(e_T)


def assert_radiance_close(rgb, T, ref, rtol, mask=None, what="", cond_eta=0.0):
    """Radiance per channel within rtol of the error scale (plus the absolute
    floor and, for the linear models, cond_eta * cond); T within rtol
    relative (floor 1e-3)."""
    e_c, e_T = radiance_errors(rgb, T, ref, rtol, cond_eta)
    if mask is not None:
        e_c, e_T = e_c[mask], e_T[mask]
    worst_c = float(e_c.max()) if e_c.size else 0.0
    worst_T = float(e_T.max()) if e_T.size else 0.0
    if worst_c > 1.0 or worst_T > 1.0:
        i = int(np.argmax(e_c.max(axis=1))) if e_c.size else -1
        raise AssertionError(f"{what}: radiance error {worst_c:.3g} x tolerance, T error {worst_T:.3g} x "
                             f"tolerance (rtol {rtol:g}); worst ray {i}")
    return worst_c, worst_T


def quantise_tree(tree: HostTree, precision: str) -> HostTree:
    """The tree the 16-bit leaves represent exactly: sigma rounded to a
    24-bit float (16-bit mantissa, nearest-even), and per leaf with non-zero
    SH, coefficients scaled by 2^-e, rounded to binary16/bfloat16
    (nearest-even), and scaled back; e is the frexp exponent of max|c| (minus
    15 for binary16, so the largest coefficient lands in [2^14, 2^15)),
    clamped to [-126, 127]."""
    import torch

    def sigma24(x32):
        b = np.ascontiguousarray(x32, np.float32).view(np.uint32) & np.uint32(0x7FFFFFFF)
        b = ((b.astype(np.uint64) + 0x3F + ((b >> 7) & 1)) >> 7) << 7
        return b.astype(np.uint32).view(np.float32)

    def rnd(x32):
        if precision == "fp16":
            return x32.astype(np.float16).astype(np.float64)
        return torch.from_numpy(np.ascontiguousarray(x32)).to(torch.bfloat16).to(torch.float64).numpy()

    sig = sigma24(tree.sigma.astype(np.float32))
    sh = tree.sh.astype(np.float32).copy()
    flat = sh.reshape(sh.shape[0], -1)
    m = np.abs(flat).max(axis=1)
    nz = m > 0
    e = np.frexp(m)[1].astype(np.int64)
    if precision == "fp16":
        e = e - 15
    e = np.clip(e, -126, 127)
    scaled = np.ldexp(flat, -e[:, None]).astype(np.float32)
    deq = np.ldexp(rnd(scaled), e[:, None])
    flat[nz] = deq[nz].astype(np.float32)
    return HostTree(tree.depth, tree.sh_degree, tree.child, sig, flat.reshape(sh.shape),
                    bbox_min=tree.bbox_min, bbox_max=tree.bbox_max)
