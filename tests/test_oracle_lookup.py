"""Pins for the oracle's point -> leaf descent: brute force over explicit
cell boxes on tiny trees, at random and adversarial points (on mid-planes,
corners, the closed root faces, outside)."""
import itertools

import numpy as np
import pytest

import oracle
from tests.trees import brute_force_cell, cell_boxes, random_tree, uniform_tree


def adversarial_points(depth, rng, n_rand=300):
    g = np.arange(0, 2 ** depth + 1) / 2 ** depth
    pts = [np.array(p) for p in itertools.product([0.0, 0.5, 1.0, g[1], g[-2]], repeat=3)]
    for _ in range(n_rand):
        p = rng.random(3)
        k = rng.integers(0, 4)
        for a in rng.choice(3, size=k, replace=False):
            p[a] = rng.choice(g)        # exactly on a cell plane
        pts.append(p)
    return np.array(pts, np.float32)


@pytest.mark.parametrize("seed", range(6))
def test_descent_matches_brute_force(seed):
    rng = np.random.default_rng(seed)
    depth = 1 + seed % 4
    tree = random_tree(depth, rng)
    boxes = cell_boxes(tree)
    pts = adversarial_points(depth, rng)
    dirs = rng.normal(size=(len(pts), 3)).astype(np.float32)
    dirs[rng.random(dirs.shape) < 0.2] = 0.0
    for use_dir in (False, True):
        leaf, _ = oracle.lookup(tree, pts, dirs if use_dir else None)
        for i, p in enumerate(pts):
            j = brute_force_cell(boxes, p, dirs[i] if use_dir else None)
            assert leaf[i] == boxes[0][j], (p, dirs[i] if use_dir else None)


def test_outside_points():
    tree = uniform_tree(2, 1.0, np.zeros((3, 9)))
    pts = np.array([[-1e-7, 0.5, 0.5], [0.5, 1.0000001, 0.5], [2, 2, 2], [0.5, 0.5, -0.0]], np.float32)
    leaf, _ = oracle.lookup(tree, pts)
    assert list(leaf[:3]) == [-2, -2, -2]
    assert leaf[3] >= 0  # -0.0 is inside the closed root box


def test_depth0_root_leaf():
    tree = uniform_tree(0, 2.0, np.ones((3, 9)))
    leaf, lev = oracle.lookup(tree, np.array([[0.0, 1.0, 0.3]], np.float32))
    assert leaf[0] == 0 and lev[0] == 0
