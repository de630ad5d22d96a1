"""Hand-built canonical trees and brute-force references for the tests.

Everything here is independent of both the oracle and the CUDA library: the
brute-force point -> cell rule is written as box membership over an explicit
list of cell boxes, not as a descent.
"""
from __future__ import annotations

import math

import numpy as np

from plogen import HostTree


def _K(deg):
    return (deg + 1) ** 2


def uniform_tree(depth: int, sigma: float, coeffs, sh_degree: int = 2) -> HostTree:
    """Full tree of the given depth whose leaves all hold (sigma, coeffs).
    depth 0 gives the single-leaf tree (no nodes, the root is leaf 0)."""
    K = _K(sh_degree)
    coeffs = np.asarray(coeffs, np.float32).reshape(3, K)
    if depth == 0:
        return HostTree(0, sh_degree, np.zeros((0, 8), np.int32), np.array([sigma], np.float32),
                        coeffs[None].copy())
    child, leaves = [], 0
    # breadth-first full tree
    level_nodes = [0]
    child.append(None)
    for lev in range(depth):
        nxt = []
        for nid in level_nodes:
            row = []
            for _ in range(8):
                if lev == depth - 1:
                    row.append(-leaves - 2)
                    leaves += 1
                else:
                    cid = len(child)
                    child.append(None)
                    row.append(cid)
                    nxt.append(cid)
            child[nid] = row
        level_nodes = nxt
    sig = np.full(leaves, sigma, np.float32)
    sh = np.broadcast_to(coeffs, (leaves, 3, K)).copy()
    return HostTree(depth, sh_degree, np.array(child, np.int32), sig, sh)


def random_tree(depth: int, rng: np.random.Generator, sh_degree: int = 2, p_split: float = 0.6,
                p_empty: float = 0.25, emissive: float = 0.5, sigma_range=(1e-2, 1e2)) -> HostTree:
    """Random sparse octree: each child of a node is split (if above the max
    depth), empty or a leaf."""
    K = _K(sh_degree)
    child = [[-1] * 8]
    sig, sh = [], []

    def new_leaf():
        s = float(np.exp(rng.uniform(np.log(sigma_range[0]), np.log(sigma_range[1]))))
        c = np.zeros((3, K), np.float32)
        if rng.random() < emissive:
            dc = rng.uniform(0.1, 10.0, 3)
            c[:, 0] = dc
            c[:, 1:] = rng.normal(0.0, 0.3, (3, K - 1)) * dc[:, None]
        sig.append(s)
        sh.append(c)
        return -(len(sig) - 1) - 2

    def fill(nid, lev):
        for s in range(8):
            r = rng.random()
            if lev + 1 < depth and r < p_split:
                cid = len(child)
                child.append([-1] * 8)
                fill(cid, lev + 1)
                child[nid][s] = cid
            elif r < p_split + (1 - p_split) * p_empty:
                child[nid][s] = -1
            else:
                child[nid][s] = new_leaf()

    fill(0, 0)
    if not sig:
        child[0][0] = new_leaf()
    return HostTree(depth, sh_degree, np.array(child, np.int32), np.array(sig, np.float32),
                    np.array(sh, np.float32).reshape(-1, 3, K))


def cell_boxes(tree: HostTree):
    """Every cell of the tree that is a leaf or an empty octant:
    (ids int64[m] (-1 = empty), lo float64[m,3], size float64[m])."""
    ids, los, sizes = [], [], []
    if tree.n_nodes == 0:
        return np.array([0]), np.zeros((1, 3)), np.ones(1)
    stack = [(0, (0.0, 0.0, 0.0), 1.0)]
    while stack:
        nid, lo, size = stack.pop()
        h = size / 2
        for s in range(8):
            clo = (lo[0] + h * (s & 1), lo[1] + h * ((s >> 1) & 1), lo[2] + h * ((s >> 2) & 1))
            e = int(tree.child[nid, s])
            if e >= 0:
                stack.append((e, clo, h))
            else:
                ids.append(-1 if e == -1 else -e - 2)
                los.append(clo)
                sizes.append(h)
    return np.array(ids, np.int64), np.array(los), np.array(sizes)


def brute_force_cell(boxes, p, d=None):
    """Index into `boxes` of the cell that owns point p under the tie rule
    (on a shared face the point belongs to the cell the direction points
    into; faces of the root box are closed), or -1 outside."""
    ids, lo, size = boxes
    hi = lo + size[:, None]
    p = np.asarray(p, np.float64)
    if np.any(p < 0) or np.any(p > 1):
        return -1
    dd = np.zeros(3) if d is None else np.asarray(d, np.float64)
    ok = np.ones(len(ids), bool)
    for a in range(3):
        x = p[a]
        up = dd[a] >= 0
        inside = (lo[:, a] < x) & (x < hi[:, a])
        on_lo = (x == lo[:, a]) & (up | (lo[:, a] == 0.0))
        on_hi = (x == hi[:, a]) & ((not up) | (hi[:, a] == 1.0))
        ok &= inside | on_lo | on_hi
    idx = np.nonzero(ok)[0]
    assert len(idx) == 1, f"point {p} owned by {len(idx)} cells"
    return int(idx[0])


def chord(o, d, lo=(0, 0, 0), hi=(1, 1, 1)):
    """[t0, t1] of the ray o + t d inside the box, by intersecting with each
    face plane and keeping the hits that lie on the box (independent of any
    slab formulation).  Returns None for a miss."""
    o, d = np.asarray(o, np.float64), np.asarray(d, np.float64)
    ts = []
    for a in range(3):
        if d[a] == 0:
            continue
        for plane in (lo[a], hi[a]):
            t = (plane - o[a]) / d[a]
            q = o + t * d
            q[a] = plane
            if all(lo[b] - 1e-12 <= q[b] <= hi[b] + 1e-12 for b in range(3)):
                ts.append(t)
    if len(ts) < 2:
        return None
    t0, t1 = min(ts), max(ts)
    if t1 <= max(t0, 0.0):
        return None
    return max(t0, 0.0), t1


def cartesian_table(x, y, z):
    """Real orthonormal SH, l <= 4, no Condon-Shortley phase, k = l(l+1)+m
    (standard Cartesian table; degree 4 from the associated Legendre
    functions P_4^m and cos / sin(m phi) written as polynomials of x, y, z)."""
    pi = math.pi
    return np.array([
        0.5 * math.sqrt(1 / pi),
        math.sqrt(3 / (4 * pi)) * y,
        math.sqrt(3 / (4 * pi)) * z,
        math.sqrt(3 / (4 * pi)) * x,
        0.5 * math.sqrt(15 / pi) * x * y,
        0.5 * math.sqrt(15 / pi) * y * z,
        0.25 * math.sqrt(5 / pi) * (3 * z * z - 1),
        0.5 * math.sqrt(15 / pi) * x * z,
        0.25 * math.sqrt(15 / pi) * (x * x - y * y),
        0.25 * math.sqrt(35 / (2 * pi)) * y * (3 * x * x - y * y),
        0.5 * math.sqrt(105 / pi) * x * y * z,
        0.25 * math.sqrt(21 / (2 * pi)) * y * (5 * z * z - 1),
        0.25 * math.sqrt(7 / pi) * z * (5 * z * z - 3),
        0.25 * math.sqrt(21 / (2 * pi)) * x * (5 * z * z - 1),
        0.25 * math.sqrt(105 / pi) * z * (x * x - y * y),
        0.25 * math.sqrt(35 / (2 * pi)) * x * (x * x - 3 * y * y),
        0.75 * math.sqrt(35 / pi) * x * y * (x * x - y * y),
        0.75 * math.sqrt(35 / (2 * pi)) * y * z * (3 * x * x - y * y),
        0.75 * math.sqrt(5 / pi) * x * y * (7 * z * z - 1),
        0.75 * math.sqrt(5 / (2 * pi)) * y * z * (7 * z * z - 3),
        3 / 16 * math.sqrt(1 / pi) * (35 * z ** 4 - 30 * z * z + 3),
        0.75 * math.sqrt(5 / (2 * pi)) * x * z * (7 * z * z - 3),
        3 / 8 * math.sqrt(5 / pi) * (x * x - y * y) * (7 * z * z - 1),
        0.75 * math.sqrt(35 / (2 * pi)) * x * z * (x * x - 3 * y * y),
        3 / 16 * math.sqrt(35 / pi) * (x ** 4 - 6 * x * x * y * y + y ** 4),
    ])


def brute_force_cells(boxes, P, d):
    """Vectorised brute_force_cell for points P [n,3] sharing direction d:
    returns the owning cell index per point (asserts exactly one)."""
    ids, lo, size = boxes
    hi = lo + size[:, None]
    P = np.asarray(P, np.float64)
    ok = np.ones((len(P), len(ids)), bool)
    for a in range(3):
        x = P[:, a:a + 1]
        up = d[a] >= 0
        inside = (lo[None, :, a] < x) & (x < hi[None, :, a])
        on_lo = (x == lo[None, :, a]) & (up | (lo[None, :, a] == 0.0))
        on_hi = (x == hi[None, :, a]) & ((not up) | (hi[None, :, a] == 1.0))
        ok &= inside | on_lo | on_hi
    assert np.all(ok.sum(1) == 1)
    return np.argmax(ok, axis=1)


def ball_chord(o, d, centre, radius):
    """[t0, t1] of the ray o + t d (any |d|) inside the ball, from the impact
    parameter: the closest approach t_m = (c - o).d / |d|^2 and the half chord
    sqrt(r^2 - h^2) / |d|.  None for a miss."""
    o, d, c = (np.asarray(v, np.float64) for v in (o, d, centre))
    dd = float(d @ d)
    tm = float((c - o) @ d) / dd
    h2 = float(np.sum((o + tm * d - c) ** 2))
    if h2 >= radius * radius:
        return None
    s = math.sqrt(radius * radius - h2) / math.sqrt(dd)
    t0, t1 = tm - s, tm + s
    if t1 <= max(t0, 0.0):
        return None
    return max(t0, 0.0), t1


def midpoint_quadrature(tree, ray, h, model="exp", act="relu", l_max=1.0, ball=None):
    """Brute-force Riemann sum of Eq. 3 along one ray: midpoint samples of
    step ~h, the cell of each sample found by box membership, Phi from the
    Cartesian SH table, transmittance from the running sum of sigma h
    (exponential, or the literal linear form of Eq. 4).  `ball` = (centre,
    radius) restricts the integral to the part of the ray inside the ball.
    Returns (rgb, T)."""
    o, d = np.asarray(ray[:3], np.float64), np.asarray(ray[3:], np.float64)
    ch = chord(o, d)
    if ch is not None and ball is not None:
        bc = ball_chord(o, d, *ball)
        ch = None if bc is None else (max(ch[0], bc[0]), min(ch[1], bc[1]))
        if ch is not None and ch[1] <= ch[0]:
            ch = None
    if ch is None:
        return np.zeros(3), 1.0
    t0, t1 = ch
    n = max(1, int(math.ceil((t1 - t0) / h)))
    hh = (t1 - t0) / n
    t = t0 + (np.arange(n) + 0.5) * hh
    P = np.clip(o[None] + t[:, None] * d[None], 0.0, 1.0)
    boxes = cell_boxes(tree)
    cid = boxes[0][brute_force_cells(boxes, P, d)]
    sig = np.where(cid >= 0, tree.sigma[np.maximum(cid, 0)].astype(np.float64), 0.0)
    dn = d / np.linalg.norm(d)
    Y = cartesian_table(*dn)[: tree.K]
    s = np.einsum("nck,k->nc", tree.sh[np.maximum(cid, 0)].astype(np.float64), Y)
    phi = np.maximum(s, 0.0) if act == "relu" else l_max / (1 + np.exp(-s))
    phi[cid < 0] = 0.0
    od_before = np.concatenate([[0.0], np.cumsum(sig * hh)[:-1]]) + 0.5 * sig * hh
    T = np.exp(-od_before) if model == "exp" else np.maximum(0.0, 1.0 - od_before)
    rgb = (T[:, None] * sig[:, None] * phi * hh).sum(0)
    od = float((sig * hh).sum())
    Tend = math.exp(-od) if model == "exp" else max(0.0, 1.0 - od)
    return rgb, Tend
