"""Pins for the oracle's render (Eq. 3-5): closed forms for uniform and
stacked leaves, telescoping of the weights, bounds, misses, empty octants,
early stop, and convergence of a brute-force midpoint quadrature of Eq. 3 to
the exact per-segment sum."""
import math

import numpy as np
import pytest

import oracle
import plogen
from plogen import HostTree
from tests.trees import ball_chord, cartesian_table, chord, midpoint_quadrature, random_tree, uniform_tree

EXP, LIN, LIT = oracle.EXPONENTIAL, oracle.LINEAR, oracle.LINEAR_LITERAL


def coeffs9(rng):
    c = np.zeros((3, 9))
    c[:, 0] = rng.uniform(1, 5, 3)
    c[:, 1:4] = rng.normal(0, 0.5, (3, 3))
    return c.astype(np.float32)


def emission(coeffs, d, act="relu", l_max=1.0):
    dn = np.asarray(d, np.float64)
    dn = dn / np.linalg.norm(dn)
    s = coeffs.astype(np.float64) @ cartesian_table(*dn)[: coeffs.shape[1]]
    return np.maximum(s, 0) if act == "relu" else l_max / (1 + np.exp(-s))


@pytest.mark.parametrize("depth", [0, 1, 3])
def test_uniform_leaf_closed_forms(depth):
    rng = np.random.default_rng(depth)
    c = coeffs9(rng)
    sigma = float(np.float32(1.7))  # the tree stores float32
    tree = uniform_tree(depth, sigma, c)
    rays = plogen.rays_sphere(256, seed=3)
    inside = np.concatenate([rng.uniform(0.05, 0.95, (32, 3)), rng.normal(size=(32, 3))], 1)
    inside[:, 3:] /= np.linalg.norm(inside[:, 3:], axis=1, keepdims=True)
    rays = np.concatenate([rays, inside.astype(np.float32)])
    for model in (EXP, LIN, LIT):
        out = oracle.render(tree, rays, transmittance=model)
        assert np.all(out["status"] == 0)
        for i, r in enumerate(rays):
            ch = chord(r[:3], r[3:])
            L = 0.0 if ch is None else ch[1] - ch[0]
            col = emission(c, r[3:])
            if model == EXP:
                T = math.exp(-sigma * L)
                C = col * (1 - T)
            else:
                T = max(0.0, 1 - sigma * L)
                C = col * (1 - T) if model == LIN else col * (1 - T * T) / 2
            assert out["T"][i] == pytest.approx(T, rel=1e-12, abs=1e-15)
            np.testing.assert_allclose(out["rgb"][i], C, rtol=1e-11, atol=1e-13)


def test_sigmoid_activation_uniform():
    rng = np.random.default_rng(5)
    c = coeffs9(rng) - 3.0
    tree = uniform_tree(2, 0.8, c)
    rays = plogen.rays_sphere(64, seed=9)
    out = oracle.render(tree, rays, activation=oracle.SIGMOID, l_max=7.5)
    for i, r in enumerate(rays):
        ch = chord(r[:3], r[3:])
        L = 0.0 if ch is None else ch[1] - ch[0]
        T = math.exp(-float(np.float32(0.8)) * L)
        np.testing.assert_allclose(out["rgb"][i], emission(c, r[3:], "sigmoid", 7.5) * (1 - T), rtol=1e-11)


def two_stack_tree(s1, c1, s2, c2):
    """Depth-1 tree: the z < 1/2 half holds (s1, c1), the upper half (s2, c2)."""
    child = np.array([[-2, -3, -4, -5, -6, -7, -8, -9]], np.int32)
    sig = np.array([s1] * 4 + [s2] * 4, np.float32)
    sh = np.stack([c1] * 4 + [c2] * 4).astype(np.float32)
    return HostTree(1, 2, child, sig, sh)


def test_two_stacked_leaves():
    rng = np.random.default_rng(2)
    c1, c2 = coeffs9(rng), coeffs9(rng)
    s1, s2 = 3.0, float(np.float32(0.4))
    tree = two_stack_tree(s1, c1, s2, c2)
    e1, e2 = math.exp(-s1 * 0.5), math.exp(-s2 * 0.5)
    up = np.array([[0.3, 0.7, -1.0, 0, 0, 1]], np.float32)
    down = np.array([[0.3, 0.7, 2.0, 0, 0, -1]], np.float32)
    o = oracle.render(tree, up)
    np.testing.assert_allclose(o["rgb"][0], emission(c1, (0, 0, 1)) * (1 - e1) +
                               e1 * emission(c2, (0, 0, 1)) * (1 - e2), rtol=1e-12)
    assert o["T"][0] == pytest.approx(e1 * e2, rel=1e-13)
    o = oracle.render(tree, down)
    np.testing.assert_allclose(o["rgb"][0], emission(c2, (0, 0, -1)) * (1 - e2) +
                               e2 * emission(c1, (0, 0, -1)) * (1 - e1), rtol=1e-12)


@pytest.mark.parametrize("model", [EXP, LIN])
def test_weights_telescope_to_alpha(model):
    # same SH in every leaf, random sigma: L_e = Phi * sum w = Phi * (1 - T)
    rng = np.random.default_rng(11)
    tree = random_tree(4, rng, emissive=1.0, sigma_range=(0.05, 20.0))
    c = coeffs9(rng)
    tree.sh[:] = c
    rays = plogen.rays_sphere(300, seed=4)
    out = oracle.render(tree, rays, transmittance=model)
    for i, r in enumerate(rays):
        np.testing.assert_allclose(out["rgb"][i], emission(c, r[3:]) * (1 - out["T"][i]), rtol=1e-11,
                                   atol=1e-14)


def test_radiance_bounded_by_brightest_leaf_and_error_scale():
    rng = np.random.default_rng(12)
    tree = random_tree(4, rng)
    rays = plogen.rays_sphere(500, seed=5)
    out = oracle.render(tree, rays)
    for i, r in enumerate(rays):
        cmax = max(emission(tree.sh[j], r[3:]).max() for j in range(tree.n_leaves))
        assert np.all(out["rgb"][i] <= cmax * (1 - out["T"][i]) * (1 + 1e-12) + 1e-15)
        assert np.all(out["rgb"][i] <= out["bound"][i] * (1 + 1e-12) + 1e-300)


def test_misses_and_axis_parallel_outside_slab():
    tree = uniform_tree(2, 5.0, np.ones((3, 9)))
    rays = np.array([
        [2.0, 2.0, 2.0, 1, 0, 0],            # parallel to x, outside y/z slabs
        [0.5, 0.5, -1.0, 0, 0, -1],          # pointing away
        [1.5, 0.5, 0.5, 0, 1, 0],            # d_x = 0 and x outside
        [-1, -1, -1, 0.6, 0.8, 0.0],         # z = -1 plane, never enters
    ], np.float32)
    out = oracle.render(tree, rays)
    np.testing.assert_array_equal(out["rgb"], 0.0)
    np.testing.assert_array_equal(out["T"], 1.0)
    np.testing.assert_array_equal(out["n_cell"], 0)


def test_empty_octants_change_nothing():
    rng = np.random.default_rng(13)
    tree = random_tree(4, rng, p_empty=0.5)
    filled = HostTree(tree.depth, tree.sh_degree, tree.child.copy(), tree.sigma.copy(), tree.sh.copy())
    sig, sh = list(filled.sigma), list(filled.sh)
    for idx in zip(*np.nonzero(filled.child == -1)):
        filled.child[idx] = -len(sig) - 2
        sig.append(0.0)
        sh.append(np.full((3, 9), 3.0, np.float32))
    filled.sigma, filled.sh = np.array(sig, np.float32), np.array(sh, np.float32)
    rays = plogen.rays_sphere(400, seed=6)
    a, b = oracle.render(tree, rays), oracle.render(filled, rays)
    np.testing.assert_allclose(a["rgb"], b["rgb"], rtol=1e-12, atol=1e-300)
    np.testing.assert_allclose(a["T"], b["T"], rtol=1e-13)


@pytest.mark.parametrize("seed", range(4))
def test_midpoint_quadrature_converges_to_segment_sum(seed):
    rng = np.random.default_rng(100 + seed)
    tree = random_tree(1 + seed % 3, rng, emissive=0.8, sigma_range=(0.1, 4.0))
    rays = list(plogen.rays_sphere(3, seed=20 + seed))
    rays.append(np.array([0.25, 0.5, -1.0, 0.0, 0.0, 1.0], np.float32))  # lies on two cell planes
    for model, mname in ((EXP, "exp"), (LIT, "lin")):
        out = oracle.render(tree, np.array(rays), transmittance=model)
        for i, r in enumerate(rays):
            errs = []
            for h in (4e-3, 1e-3, 2.5e-4):
                rgb, T = midpoint_quadrature(tree, r, h, model=mname)
                scale = max(np.abs(out["rgb"][i]).max(), 1e-3)
                errs.append(np.abs(rgb - out["rgb"][i]).max() / scale)
            assert errs[-1] < 3e-3, errs
            assert errs[-1] <= errs[0] + 1e-12, errs


def test_early_stop_within_tail_bound():
    tree = plogen.luminaire_tree(plogen.LUMINAIRE_D6)
    rays = plogen.rays_sphere(4096, seed=8)
    full = oracle.render(tree, rays)
    stop = oracle.render(tree, rays, t_stop=1e-4)
    stopped = stop["n_leaf"] < full["n_leaf"]
    assert stopped.any()
    assert np.all(stop["n_leaf"] <= full["n_leaf"])
    assert np.all(stop["T"][stopped] < 1e-4)
    # after the stop the rest of the ray adds at most T_stop * max_leaf Phi(d)
    absc = np.abs(tree.sh.astype(np.float64))
    for i in np.nonzero(stopped)[0]:
        d = rays[i, 3:].astype(np.float64)
        Y = np.abs(cartesian_table(*(d / np.linalg.norm(d))))[: tree.K]
        cap = (absc @ Y).max(axis=0)
        gap = np.abs(stop["rgb"][i] - full["rgb"][i])
        assert np.all(gap <= stop["T"][i] * cap * (1 + 1e-9) + 1e-12)
    np.testing.assert_array_equal(stop["rgb"][~stopped], full["rgb"][~stopped])


def test_sigma_min_equals_zeroed_tree():
    rng = np.random.default_rng(14)
    tree = random_tree(3, rng, sigma_range=(1e-3, 1.0))
    zeroed = HostTree(tree.depth, tree.sh_degree, tree.child, np.where(tree.sigma < 0.1, 0, tree.sigma)
                      .astype(np.float32), tree.sh)
    rays = plogen.rays_sphere(300, seed=15)
    a = oracle.render(tree, rays, sigma_min=0.1)
    b = oracle.render(zeroed, rays)
    np.testing.assert_array_equal(a["rgb"], b["rgb"])
    np.testing.assert_array_equal(a["T"], b["T"])


def test_world_bbox_scales_lengths():
    c = coeffs9(np.random.default_rng(3))
    tree = uniform_tree(2, 0.3, c)
    tree.bbox_min, tree.bbox_max = (-1.0, -2.0, 0.0), (3.0, 2.0, 4.0)
    rays = plogen.rays_sphere(64, seed=2, radius=9.0, center=(1.0, 0.0, 2.0))
    out = oracle.render(tree, rays)
    for i, r in enumerate(rays):
        ch = chord(r[:3], r[3:], tree.bbox_min, tree.bbox_max)
        L = 0.0 if ch is None else ch[1] - ch[0]
        T = math.exp(-float(np.float32(0.3)) * L)
        assert out["T"][i] == pytest.approx(T, rel=1e-12)
        np.testing.assert_allclose(out["rgb"][i], emission(c, r[3:]) * (1 - T), rtol=1e-11)


def test_trace_is_ordered_and_contiguous():
    tree = plogen.luminaire_tree(plogen.LUMINAIRE_D6)
    for r in plogen.rays_sphere(50, seed=16):
        leaf, t = oracle.trace(tree, r)
        if len(leaf) == 0:
            continue
        assert np.all(t[:, 1] >= t[:, 0])
        np.testing.assert_array_equal(t[1:, 0], t[:-1, 1])
        ch = chord(r[:3], r[3:])
        assert t[0, 0] == pytest.approx(ch[0], abs=1e-12)
        assert t[-1, 1] == pytest.approx(ch[1], abs=1e-12)


def corner_rays(rng, n, grid=64):
    """Diagonal rays from grid points: they cross many cells exactly through
    shared corners and edges."""
    g = np.arange(grid + 1) / grid
    out = []
    for _ in range(n):
        o = rng.choice(g, 3) - 2.0
        s = rng.choice([-1.0, 1.0], 3)
        o = np.where(s > 0, o, 3.0 - (o + 2.0))
        out.append(np.concatenate([o, s / np.sqrt(3)]))
    return np.array(out, np.float32)


def test_corner_rays_progress_and_closed_form():
    rng = np.random.default_rng(21)
    rays = corner_rays(rng, 400)
    c = coeffs9(rng)
    sig = float(np.float32(2.5))
    tree = uniform_tree(4, sig, c)
    out = oracle.render(tree, rays)
    assert np.all(out["status"] == 0)
    for i, r in enumerate(rays):
        ch = chord(r[:3], r[3:])
        L = 0.0 if ch is None else ch[1] - ch[0]
        T = math.exp(-sig * L)
        assert out["T"][i] == pytest.approx(T, rel=1e-12, abs=1e-15)
        np.testing.assert_allclose(out["rgb"][i], emission(c, r[3:]) * (1 - T), rtol=1e-11, atol=1e-13)
    # sparse luminaire tree: every corner ray terminates, and its segments tile the chord
    d6 = plogen.luminaire_tree(plogen.LUMINAIRE_D6)
    out = oracle.render(d6, rays)
    assert np.all(out["status"] == 0)
    for r in rays[:100]:
        leaf, t = oracle.trace(d6, r)
        ch = chord(r[:3], r[3:])
        if ch is None:
            assert len(leaf) == 0
            continue
        np.testing.assert_array_equal(t[1:, 0], t[:-1, 1])
        assert t[0, 0] == pytest.approx(ch[0], abs=1e-12) and t[-1, 1] == pytest.approx(ch[1], abs=1e-12)


def test_corner_rays_match_midpoint_quadrature():
    rng = np.random.default_rng(22)
    tree = random_tree(3, rng, emissive=0.8, sigma_range=(0.1, 4.0))
    rays = corner_rays(rng, 6, grid=8)
    out = oracle.render(tree, rays)
    assert np.all(out["status"] == 0)
    for i, r in enumerate(rays):
        rgb, T = midpoint_quadrature(tree, r, 2.5e-4)
        scale = max(np.abs(out["rgb"][i]).max(), 1e-3)
        assert np.abs(rgb - out["rgb"][i]).max() / scale < 3e-3


# ---------------------------------------------------------------- proxy sphere and the paper's
# render heuristics (Sec. 5 proxy geometry; Sec. 6 sigma_min / alpha_max)

@pytest.mark.parametrize("model", [EXP, LIN])
def test_sphere_proxy_uniform_closed_form(model):
    rng = np.random.default_rng(21)
    c = coeffs9(rng)
    sigma = float(np.float32(2.3))
    tree = uniform_tree(2, sigma, c)
    centre, radius = (0.5, 0.47, 0.53), 0.41
    rays = plogen.rays_sphere(256, seed=22)
    inside = np.concatenate([rng.uniform(0.3, 0.7, (32, 3)), rng.normal(size=(32, 3))], 1)
    inside[:, 3:] /= np.linalg.norm(inside[:, 3:], axis=1, keepdims=True)
    rays = np.concatenate([rays, inside.astype(np.float32)])
    out = oracle.render(tree, rays, transmittance=model, sphere=(*centre, radius))
    assert np.all(out["status"] == 0)
    hits = 0
    for i, r in enumerate(rays):
        ch = ball_chord(r[:3], r[3:], centre, radius)  # the ball lies inside the cube
        L = 0.0 if ch is None else ch[1] - ch[0]
        hits += L > 0
        T = math.exp(-sigma * L) if model == EXP else max(0.0, 1.0 - sigma * L)
        assert out["T"][i] == pytest.approx(T, rel=1e-10, abs=1e-13)
        np.testing.assert_allclose(out["rgb"][i], emission(c, r[3:]) * (1 - T), rtol=1e-10, atol=1e-12)
    assert hits > 100


def test_sphere_enclosing_the_box_changes_nothing():
    tree = plogen.luminaire_tree(plogen.LUMINAIRE_D6)
    rays = plogen.rays_sphere(2048, seed=23)
    a = oracle.render(tree, rays)
    b = oracle.render(tree, rays, sphere=(0.5, 0.5, 0.5, 0.87))  # sqrt(3)/2 < 0.87
    for k in ("rgb", "T", "n_cell"):
        np.testing.assert_array_equal(a[k], b[k])


def test_sphere_proxy_cut_matches_midpoint_quadrature():
    # a ball that cuts through cells: brute force restricted to the ball
    rng = np.random.default_rng(24)
    tree = random_tree(3, rng, sigma_range=(0.1, 8.0))
    ball = ((0.45, 0.55, 0.5), 0.33)
    rays = plogen.rays_sphere(24, seed=25, radius=2.0)
    out = oracle.render(tree, rays, sphere=(*ball[0], ball[1]))
    errs = np.zeros((len(rays), 2))
    for i, r in enumerate(rays):
        for j, h in enumerate((1e-3, 2.5e-4)):
            rgb, T = midpoint_quadrature(tree, r, h, ball=ball)
            scale = max(1.0, np.abs(rgb).max())
            errs[i, j] = max(np.abs(rgb - out["rgb"][i]).max() / scale, abs(T - out["T"][i]))
    # midpoint errors are O(h) but not monotone ray by ray
    assert errs[:, 1].max() < 2e-3, errs
    assert errs[:, 1].mean() < 0.6 * errs[:, 0].mean(), errs.mean(0)


def test_saturation_sets_T_to_zero_after_early_stop():
    rng = np.random.default_rng(26)
    c1, c2 = coeffs9(rng), coeffs9(rng)
    s1, s2 = 6.0, float(np.float32(0.4))  # T after the first half: e^-3 < 0.1
    tree = two_stack_tree(s1, c1, s2, c2)
    e1 = math.exp(-s1 * 0.5)
    up = np.array([[0.3, 0.7, -1.0, 0, 0, 1]], np.float32)
    down = np.array([[0.3, 0.7, 2.0, 0, 0, -1]], np.float32)
    plain = oracle.render(tree, up, t_stop=0.1)
    sat = oracle.render(tree, up, t_stop=0.1, saturate=True)
    np.testing.assert_allclose(sat["rgb"][0], emission(c1, (0, 0, 1)) * (1 - e1), rtol=1e-12)
    np.testing.assert_array_equal(sat["rgb"], plain["rgb"])
    assert plain["T"][0] == pytest.approx(e1, rel=1e-13)
    assert sat["T"][0] == 0.0 and sat["n_leaf"][0] == 1
    # a ray that never gets below t_stop keeps its T
    e2 = math.exp(-s2 * 0.5)
    sat = oracle.render(tree, down, t_stop=e2 * 0.5, saturate=True)
    full = oracle.render(tree, down)
    assert sat["T"][0] == pytest.approx(e2 * e1, rel=1e-13) or sat["T"][0] == 0.0
    assert sat["T"][0] == 0.0  # e2 * e1 < e2 / 2: saturated after the second leaf
    np.testing.assert_array_equal(sat["rgb"], full["rgb"])
    sat = oracle.render(tree, down, t_stop=1e-3, saturate=True)
    assert sat["T"][0] == pytest.approx(e2 * e1, rel=1e-13)


def test_sphere_proxy_world_bbox():
    c = coeffs9(np.random.default_rng(27))
    tree = uniform_tree(2, 0.3, c)
    tree.bbox_min, tree.bbox_max = (-1.0, -2.0, 0.0), (3.0, 2.0, 4.0)
    centre, radius = (1.2, -0.3, 2.1), 1.6
    rays = plogen.rays_sphere(128, seed=28, radius=9.0, center=(1.0, 0.0, 2.0))
    out = oracle.render(tree, rays, sphere=(*centre, radius))
    for i, r in enumerate(rays):
        ch = ball_chord(r[:3], r[3:], centre, radius)
        L = 0.0 if ch is None else ch[1] - ch[0]
        T = math.exp(-float(np.float32(0.3)) * L)
        assert out["T"][i] == pytest.approx(T, rel=1e-11)
        np.testing.assert_allclose(out["rgb"][i], emission(c, r[3:]) * (1 - T), rtol=1e-10, atol=1e-13)
