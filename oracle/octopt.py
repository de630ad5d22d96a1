"""FP64 oracle for optimising the octree's leaves directly from rendered
targets, the alternative to training a network and projecting it onto the
octree that Sec. 7 ("Limitations -- Precomputation cost") names: fit the SH
octree itself, with a total-variation regulariser against aliasing at
discontinuities (as Plenoxels does on its grid).

TEST INFRASTRUCTURE ONLY (tests and smoke).  Plain numpy over the oracle's
own exact cell walk (``oracle.trace``) and its quadrature, loss and Adam
(``oracle.mlp``).  The paper gives no formulas for this variant; the reading
taken here:

  - parameters, per leaf i: a raw density s_i and 3K SH coefficients k_i
    (channel-major); sigma_i = max(0, s_i) and the emission
    L_max sigmoid(sum_k k_{i,ch,k} Y_k(d)) as for the network (Sec. 4.2,
    Eq. 6);
  - render: the octree's own exact per-leaf segments (the cells the ray
    crosses, Sec. 5), composited with Eq. 3-5 (exponential or linear
    transmittance), so the forward pass equals ``oracle.render`` of the tree
    with sigma = max(0, s) and the sigmoid activation;
  - loss: the paper's (Sec. 4.3, Eq. 7-9) as for the network
    (``oracle.mlp.loss_terms``), averaged over the rays;
  - TV, per leaf i and per channel x (the raw density; each SH
    coefficient): sqrt(eps + sum_a (x_{n_a(i)} - x_i)^2) over the axes a,
    where n_a(i) is the leaf that holds the point just across i's upper face
    on axis a, at the face's centre (c_i + (h_i + 2^-(D+1)) e_a, with c_i,
    h_i the leaf's centre and half size in the unit cube and D the tree
    depth); an axis without such a leaf (outside the cube, an empty octant)
    adds nothing.  TV_sigma and TV_sh are the means over the leaves of the
    density term and of the sum of the SH terms;
  - objective: loss + lambda_sigma TV_sigma + lambda_sh TV_sh;
  - update: Adam (``oracle.mlp.adam_update``) on (s, k), the step size of
    each group decaying exponentially by the factor `lr_decay` over
    `total` steps (Sec. 4.4's schedule for the network).
"""
from __future__ import annotations

import numpy as np

import oracle as _oracle
from oracle import mlp as _mlp

TV_EPS = 1e-8


def leaf_boxes(child: np.ndarray, n_leaves: int):
    """Unit-cube box of every leaf: (lo float64[n_leaves, 3], size
    float64[n_leaves]), from the canonical child table."""
    lo = np.zeros((n_leaves, 3))
    size = np.ones(n_leaves)
    if child.shape[0] == 0:
        return lo, size
    stack = [(0, (0.0, 0.0, 0.0), 1.0)]
    while stack:
        nid, base, s = stack.pop()
        h = s / 2
        for slot in range(8):
            clo = (base[0] + h * (slot & 1), base[1] + h * ((slot >> 1) & 1), base[2] + h * ((slot >> 2) & 1))
            e = int(child[nid, slot])
            if e >= 0:
                stack.append((e, clo, h))
            elif e <= -2:
                lo[-e - 2] = clo
                size[-e - 2] = h
    return lo, size


def neighbour_points(tree):
    """float32 [n_leaves, 3, 3]: per leaf and axis a, the point just across
    the leaf's upper face a, at the face's centre."""
    lo, size = leaf_boxes(np.asarray(tree.child), tree.n_leaves)
    delta = 2.0 ** -(tree.depth + 1)
    pts = np.repeat((lo + size[:, None] / 2)[:, None, :], 3, axis=1)
    for a in range(3):
        pts[:, a, a] = lo[:, a] + size + delta
    return pts.astype(np.float32)


def neighbours(tree) -> np.ndarray:
    """int64 [n_leaves, 3]: the leaf n_a(i), or -1 (outside, empty octant)."""
    pts = neighbour_points(tree).reshape(-1, 3)
    leaf, _ = _oracle.lookup(tree, pts)
    return np.where(leaf >= 0, leaf, -1).reshape(-1, 3)


def structure(tree):
    """The tree with zero densities and coefficients: its walk crosses every
    cell to the far side of the proxy (nothing saturates)."""
    from types import SimpleNamespace
    return SimpleNamespace(depth=tree.depth, sh_degree=tree.sh_degree, child=tree.child,
                           sigma=np.zeros(tree.n_leaves, np.float32),
                           sh=np.zeros((tree.n_leaves, 3, (tree.sh_degree + 1) ** 2), np.float32),
                           bbox_min=getattr(tree, "bbox_min", (0.0, 0.0, 0.0)),
                           bbox_max=getattr(tree, "bbox_max", (1.0, 1.0, 1.0)))


def segments(tree, rays):
    """Per ray, the leaves it crosses in order and their segment lengths:
    (leaf int64 [R, N], delta float64 [R, N]) padded with leaf -1, delta 0."""
    st = structure(tree)
    per = []
    for r in rays:
        leaf, t = _oracle.trace(st, r)
        keep = leaf >= 0
        per.append((leaf[keep], (t[:, 1] - t[:, 0])[keep]))
    N = max([len(p[0]) for p in per] + [1])
    L = np.full((len(rays), N), -1, np.int64)
    D = np.zeros((len(rays), N))
    for i, (lf, dl) in enumerate(per):
        L[i, : len(lf)] = lf
        D[i, : len(dl)] = dl
    return L, D


def tv(x: np.ndarray, nb: np.ndarray, eps: float = TV_EPS):
    """Total variation of the per-leaf channels x [n_leaves, C] over the
    neighbour table nb [n_leaves, 3]: (value, gradient [n_leaves, C])."""
    n, C = x.shape
    diff = np.zeros((n, 3, C))
    for a in range(3):
        has = nb[:, a] >= 0
        diff[has, a] = x[nb[has, a]] - x[has]
    s = np.sqrt(eps + (diff ** 2).sum(1))  # [n, C]
    val = s.sum() / n
    g = np.zeros_like(x, dtype=np.float64)
    for a in range(3):
        q = diff[:, a] / s / n
        has = nb[:, a] >= 0
        g -= q
        np.add.at(g, nb[has, a], q[has])
    return val, g


def loss_and_grads(tree, s, k, rays, C_gt, alpha_gt, l_max_scale, transmittance="exp", kind="paper",
                   lam_sigma=0.0, lam_sh=0.0, segs=None, nb=None, denom=None):
    """Objective and its gradient for raw densities s [n_leaves] and
    coefficients k [n_leaves, 3K] on world-space rays [R, 6] against targets
    C_gt [R, 3], alpha_gt [R].  `denom` overrides the loss's held-constant
    denominator (``oracle.mlp.loss_terms``).  Returns (objective, ds, dk,
    extras)."""
    K = (tree.sh_degree + 1) ** 2
    L, D = segments(tree, rays) if segs is None else segs
    R, N = L.shape
    valid = L >= 0
    idx = np.where(valid, L, 0)
    raw = np.concatenate([s[idx][..., None], k[idx]], axis=2)  # [R, N, 1 + 3K]
    raw[~valid] = 0.0
    d = rays[:, 3:].astype(np.float64)
    d = d / np.linalg.norm(d, axis=1, keepdims=True)
    Y = _mlp.sh_matrix(d, tree.sh_degree)
    C, alpha, cache = _mlp.composite(raw, D, Y, l_max_scale, transmittance)
    per_ray, dC, dA = _mlp.loss_terms(C, alpha, C_gt, alpha_gt, l_max_scale, kind, denom=denom)
    draw = _mlp.composite_backward(cache, dC / R, dA / R)
    draw[~valid] = 0.0
    ds = np.zeros(len(s))
    dk = np.zeros((len(s), 3 * K))
    np.add.at(ds, L[valid], draw[..., 0][valid])
    np.add.at(dk, L[valid], draw[..., 1:][valid])
    obj = per_ray.mean()
    tv_s = tv_k = 0.0
    if lam_sigma or lam_sh:
        nb = neighbours(tree) if nb is None else nb
        tv_s, g_s = tv(s[:, None].astype(np.float64), nb)
        tv_k, g_k = tv(k.astype(np.float64), nb)
        obj += lam_sigma * tv_s + lam_sh * tv_k
        ds += lam_sigma * g_s[:, 0]
        dk += lam_sh * g_k
    return obj, ds, dk, dict(C=C, alpha=alpha, loss=per_ray.mean(), tv_sigma=tv_s, tv_sh=tv_k, segs=(L, D))


def adam_steps(tree, s, k, batches, l_max_scale, lr_sigma, lr_sh, lr_decay, total, transmittance="exp",
               kind="paper", lam_sigma=0.0, lam_sh=0.0, start_step=0):
    """Adam over the batches [(rays, C_gt, alpha_gt)], one update per batch.
    Returns (s, k, per-step objectives)."""
    s, k = s.astype(np.float64).copy(), k.astype(np.float64).copy()
    ms, vs = np.zeros_like(s), np.zeros_like(s)
    mk, vk = np.zeros_like(k), np.zeros_like(k)
    nb = neighbours(tree) if (lam_sigma or lam_sh) else None
    objs = []
    for j, (rays, C_gt, a_gt) in enumerate(batches):
        step = start_step + j + 1
        obj, ds, dk, _ = loss_and_grads(tree, s, k, rays, C_gt, a_gt, l_max_scale, transmittance, kind,
                                        lam_sigma, lam_sh, nb=nb)
        objs.append(obj)
        f = lr_decay ** (min(step - 1, total) / max(total, 1))
        s, ms, vs = _mlp.adam_update(s, ds, ms, vs, step, lr_sigma * f)
        k, mk, vk = _mlp.adam_update(k, dk, mk, vk, step, lr_sh * f)
    return s, k, objs
