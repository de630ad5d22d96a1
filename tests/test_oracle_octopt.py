"""Pins of the direct leaf optimisation oracle (oracle/octopt.py) against the
exact-segment render, brute-force neighbours, closed forms of the total
variation, central differences of the whole objective and Adam's first
step."""
from __future__ import annotations

import numpy as np
import pytest

import oracle
import plogen
from oracle import octopt
from tests.trees import brute_force_cell, cell_boxes, random_tree, uniform_tree


def _problem(seed, depth=3, deg=2, n_rays=48):
    rng = np.random.default_rng(seed)
    tree = random_tree(depth, rng, sh_degree=deg, p_split=0.5, p_empty=0.2)
    K = tree.K
    s = rng.uniform(0.5, 3.0, tree.n_leaves)
    s[rng.random(tree.n_leaves) < 0.2] = -0.7  # some leaves below the ReLU's kink
    k = rng.normal(0.0, 0.8, (tree.n_leaves, 3 * K))
    rays = plogen.rays_sphere(n_rays, seed=seed + 3)
    C_gt = rng.uniform(0.0, 2.0, (n_rays, 3))
    a_gt = rng.uniform(0.0, 1.0, n_rays)
    return tree, s, k, rays, C_gt, a_gt


@pytest.mark.parametrize("trans", ["exp", "linear"])
def test_forward_equals_exact_segment_render(trans):
    tree, s, k, rays, C_gt, a_gt = _problem(1)
    l_max = 2.5
    t = plogen.HostTree(tree.depth, tree.sh_degree, tree.child, np.maximum(s, 0).astype(np.float32),
                        k.reshape(-1, 3, tree.K).astype(np.float32))
    # the exact render reads float32 leaves: feed the same values to both
    s32 = t.sigma.astype(np.float64)
    k32 = t.sh.reshape(-1, 3 * tree.K).astype(np.float64)
    _, _, _, ex = octopt.loss_and_grads(tree, s32, k32, rays, C_gt, a_gt, l_max, trans)
    ref = oracle.render(t, rays, transmittance=0 if trans == "exp" else 1, activation=1, l_max=l_max)
    assert np.all(ref["status"] == 0)
    np.testing.assert_allclose(ex["C"], ref["rgb"], rtol=1e-9, atol=1e-12)
    np.testing.assert_allclose(1.0 - ex["alpha"], ref["T"], rtol=1e-9, atol=1e-12)


def test_neighbours_match_brute_force_ownership():
    rng = np.random.default_rng(4)
    tree = random_tree(4, rng, p_split=0.55, p_empty=0.2)
    nb = octopt.neighbours(tree)
    pts = octopt.neighbour_points(tree)
    boxes = cell_boxes(tree)
    for i in range(tree.n_leaves):
        for a in range(3):
            j = brute_force_cell(boxes, pts[i, a].astype(np.float64))
            want = -1 if j < 0 else int(boxes[0][j])
            assert nb[i, a] == want, (i, a)


def test_neighbours_of_a_uniform_grid_are_index_steps():
    tree = uniform_tree(2, 1.0, np.zeros(27))
    lo, size = octopt.leaf_boxes(tree.child, tree.n_leaves)
    ijk = np.rint(lo * 4).astype(int)
    where = {tuple(v): i for i, v in enumerate(ijk)}
    nb = octopt.neighbours(tree)
    for i, v in enumerate(ijk):
        for a in range(3):
            w = v.copy()
            w[a] += 1
            assert nb[i, a] == where.get(tuple(w), -1)
    assert np.all(size == 0.25)


def test_tv_closed_forms():
    tree = uniform_tree(2, 1.0, np.zeros(27))
    nb = octopt.neighbours(tree)
    n = tree.n_leaves
    # a constant field: only the eps floor, zero gradient
    val, g = octopt.tv(np.full((n, 2), 3.0), nb)
    assert val == pytest.approx(2 * np.sqrt(octopt.TV_EPS))
    assert np.all(g == 0.0)
    # a unit ramp along x: 48 of the 64 cells step by 1 to their x neighbour
    lo, _ = octopt.leaf_boxes(tree.child, n)
    x = np.rint(lo[:, :1] * 4)
    val, _ = octopt.tv(x, nb)
    assert val == pytest.approx((48 * np.sqrt(1 + octopt.TV_EPS) + 16 * np.sqrt(octopt.TV_EPS)) / 64, rel=1e-12)
    # x + 2y: sqrt(5) where both neighbours exist, 1 or 2 on the faces
    x = np.rint(lo[:, 0] * 4) + 2 * np.rint(lo[:, 1] * 4)
    val, _ = octopt.tv(x[:, None], nb)
    hx, hy = np.rint(lo[:, 0] * 4) < 3, np.rint(lo[:, 1] * 4) < 3
    want = np.sqrt(octopt.TV_EPS + hx * 1.0 + hy * 4.0).sum() / 64
    assert val == pytest.approx(want, rel=1e-12)


@pytest.mark.parametrize("trans,kind,seed", [("exp", "paper", 2), ("linear", "paper", 3), ("exp", "mse", 5)])
def test_objective_gradient_matches_central_differences(trans, kind, seed):
    tree, s, k, rays, C_gt, a_gt = _problem(seed)
    lam_s, lam_k = 0.03, 0.01
    args = (rays, C_gt, a_gt, 2.0, trans, kind, lam_s, lam_k)
    obj, ds, dk, ex = octopt.loss_and_grads(tree, s, k, *args)
    segs, nb = ex["segs"], octopt.neighbours(tree)
    # the loss holds its denominator constant: keep it at the base point's
    den = ex["C"] / 2.0 + 0.01
    f = lambda s_, k_: octopt.loss_and_grads(tree, s_, k_, *args, segs=segs, nb=nb, denom=den)[0]
    rng = np.random.default_rng(seed)
    h = 1e-4  # the paper loss reaches 1e4 (denominators near eps): larger steps keep roundoff down
    hit = np.unique(segs[0][segs[0] >= 0])
    for i in rng.choice(hit, 6, replace=False):
        if abs(s[i]) > 10 * h:
            e = np.zeros_like(s)
            e[i] = h
            fd = (f(s + e, k) - f(s - e, k)) / (2 * h)
            assert ds[i] == pytest.approx(fd, rel=1e-5, abs=1e-8), ("sigma", i)
        for c in rng.choice(k.shape[1], 3, replace=False):
            e = np.zeros_like(k)
            e[i, c] = h
            fd = (f(s, k + e) - f(s, k - e)) / (2 * h)
            assert dk[i, c] == pytest.approx(fd, rel=1e-5, abs=1e-8), ("sh", i, c)
    # a leaf no ray crosses moves only by the regulariser
    missed = np.setdiff1d(np.arange(tree.n_leaves), hit)
    if len(missed):
        _, ds0, dk0, _ = octopt.loss_and_grads(tree, s, k, rays, C_gt, a_gt, 2.0, trans, kind, segs=segs)
        assert np.all(ds0[missed] == 0.0) and np.all(dk0[missed] == 0.0)


def test_adam_first_step_is_a_signed_step_of_the_decayed_rate():
    tree, s, k, rays, C_gt, a_gt = _problem(6, n_rays=24)
    obj, ds, dk, _ = octopt.loss_and_grads(tree, s, k, rays, C_gt, a_gt, 2.0)
    s1, k1, objs = octopt.adam_steps(tree, s, k, [(rays, C_gt, a_gt)], 2.0, 0.1, 0.05, 0.01, 100)
    assert objs[0] == pytest.approx(obj)
    np.testing.assert_allclose(s1, s - 0.1 * ds / (np.abs(ds) + 1e-8), rtol=1e-12, atol=1e-15)
    np.testing.assert_allclose(k1, k - 0.05 * dk / (np.abs(dk) + 1e-8), rtol=1e-12, atol=1e-15)
    # the rate at update j (1-based) is lr * decay^((j - 1) / total)
    s5, _, _ = octopt.adam_steps(tree, s, k, [(rays, C_gt, a_gt)], 2.0, 0.1, 0.05, 0.01, 4, start_step=4)
    m = 0.1 * ds
    v = 0.001 * ds * ds
    want = s - 0.1 * 0.01 * (m / (1 - 0.9 ** 5)) / (np.sqrt(v / (1 - 0.999 ** 5)) + 1e-8)
    np.testing.assert_allclose(s5, want, rtol=1e-12, atol=1e-15)
