"""GPU parity of the direct leaf optimisation (plo_octopt_*, the Sec. 7
alternative to the network): forward pass, loss, TV values, the gradients of
every leaf element by element and the neighbour table against the FP64
oracle (oracle/octopt.py); Adam against the oracle's update on the GPU's own
gradients; a fit that recovers a tree from its renders; edge cases."""
import numpy as np
import pytest

import paper_2207_05009_gb300 as plo
import plogen
from oracle import octopt as ooct
from tests.trees import random_tree

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_cuda(cuda_available):
    import torch
    return torch


def _problem(seed, depth=4, deg=2, n=512, l_max=2.0):
    rng = np.random.default_rng(seed)
    tree = random_tree(depth, rng, sh_degree=deg, p_split=0.5, p_empty=0.2)
    nl, K = tree.n_leaves, tree.K
    s = rng.uniform(0.5, 3.0, nl).astype(np.float32)
    s[rng.random(nl) < 0.2] = -0.7
    k = rng.normal(0.0, 0.8, (nl, 3, K)).astype(np.float32)
    rays = plogen.rays_sphere(n, seed=seed + 3)
    C_gt = rng.uniform(0.0, l_max, (n, 3)).astype(np.float32)
    a_gt = rng.uniform(0.0, 1.0, n).astype(np.float32)
    init = plogen.HostTree(tree.depth, deg, tree.child, np.maximum(s, 0.0), k)
    return tree, init, s, k, rays, C_gt, a_gt


def _dev(torch, *arrs):
    return [torch.from_numpy(np.ascontiguousarray(a)).cuda() for a in arrs]


def _close(name, got, want, rtol, atol_frac):
    """|got - want| <= rtol |want| + atol_frac max|want| element-wise."""
    got, want = np.asarray(got, np.float64), np.asarray(want, np.float64)
    atol = atol_frac * max(np.abs(want).max(), 1e-30)
    err = np.abs(got - want)
    bad = err > rtol * np.abs(want) + atol
    assert not bad.any(), (f"{name}: {bad.sum()} of {bad.size} off; max err {err.max():.3e}, "
                           f"max|want| {np.abs(want).max():.3e}, worst rel {np.max(err / (np.abs(want) + atol)):.3e}")


@pytest.mark.parametrize("trans,kind,seed", [(plo.TRANS_EXP, plo.LOSS_PAPER, 1), (plo.TRANS_LINEAR, plo.LOSS_PAPER, 2),
                                             (plo.TRANS_EXP, plo.LOSS_MSE, 3), (plo.TRANS_EXP, plo.LOSS_REG, 4)])
def test_gradients_match_oracle(torch_cuda, trans, kind, seed):
    torch = torch_cuda
    l_max, lam_s, lam_k = 2.0, 0.03, 0.01
    tree, init, s, k, rays, C_gt, a_gt = _problem(seed, l_max=l_max)
    n = rays.shape[0]
    opt = plo.OctOpt(init, l_max, max_rays=n, loss=kind, transmittance=trans, tv_sigma=lam_s, tv_sh=lam_k)
    opt.write(plo.OCTOPT_SIGMA, s)
    dr, dc, da = _dev(torch, rays, C_gt, a_gt)
    ray_out = torch.empty((n, 5), device="cuda", dtype=torch.float32)
    loss = opt.grad(dr, dc, da, ray_out=ray_out)
    opt.check()
    gs, gk = opt.read(plo.OCTOPT_GRAD_SIGMA), opt.read(plo.OCTOPT_GRAD_SH).reshape(tree.n_leaves, -1)
    tname = "exp" if trans == plo.TRANS_EXP else "linear"
    kname = {plo.LOSS_PAPER: "paper", plo.LOSS_MSE: "mse", plo.LOSS_REG: "reg"}[kind]
    obj, ds, dk, ex = ooct.loss_and_grads(tree, s.astype(np.float64), k.reshape(tree.n_leaves, -1).astype(np.float64),
                                          rays, C_gt.astype(np.float64), a_gt.astype(np.float64), l_max, tname, kname,
                                          lam_s, lam_k)
    ro = ray_out.cpu().numpy()
    _close("C", ro[:, :3], ex["C"], 1e-4, 1e-5)
    _close("alpha", ro[:, 3], ex["alpha"], 1e-4, 1e-5)
    lo = loss.cpu().numpy()
    assert lo[0] == pytest.approx(ex["loss"], rel=2e-3)
    assert lo[1] == pytest.approx(ex["tv_sigma"], rel=1e-4)
    assert lo[2] == pytest.approx(ex["tv_sh"], rel=1e-4)
    _close("d/ds", gs, ds, 3e-3, 3e-4)
    _close("d/dk", gk, dk, 3e-3, 3e-4)


def test_neighbour_table_is_bit_exact(torch_cuda):
    rng = np.random.default_rng(9)
    tree = random_tree(5, rng, p_split=0.55, p_empty=0.2)
    opt = plo.OctOpt(tree, 1.0, max_rays=1)
    np.testing.assert_array_equal(opt.read(plo.OCTOPT_NEIGHBOURS), ooct.neighbours(tree))


def test_adam_matches_oracle_update_over_steps(torch_cuda):
    torch = torch_cuda
    tree, init, s, k, rays, C_gt, a_gt = _problem(5, n=256)
    lr_s, lr_k, decay, total = 0.05, 0.02, 0.1, 3
    opt = plo.OctOpt(init, 2.0, max_rays=256, lr_sigma=lr_s, lr_sh=lr_k, lr_decay=decay, total_steps=total,
                     tv_sigma=0.01, tv_sh=0.01)
    opt.write(plo.OCTOPT_SIGMA, s)
    from oracle import mlp as omlp
    p = [opt.read(plo.OCTOPT_SIGMA).astype(np.float64), opt.read(plo.OCTOPT_SH).astype(np.float64).ravel()]
    m = [np.zeros_like(x) for x in p]
    v = [np.zeros_like(x) for x in p]
    for t in range(1, 6):
        sub = slice(50 * t, 50 * t + 200)
        opt.step(*_dev(torch, rays[sub], C_gt[sub], a_gt[sub]))
        g = [opt.read(plo.OCTOPT_GRAD_SIGMA).astype(np.float64), opt.read(plo.OCTOPT_GRAD_SH).astype(np.float64).ravel()]
        f = decay ** (min(t - 1, total) / total)
        for i, lr in enumerate((lr_s, lr_k)):
            p[i], m[i], v[i] = omlp.adam_update(p[i], g[i], m[i], v[i], t, lr * f)
        got = [opt.read(plo.OCTOPT_SIGMA), opt.read(plo.OCTOPT_SH).ravel()]
        for i, lr in enumerate((lr_s, lr_k)):
            err = np.abs(got[i] - p[i])
            assert err.max() <= 1e-5 * lr * t + 2e-7 * np.abs(p[i]).max(), (t, i, err.max())
        p = [x.astype(np.float64) for x in got]  # continue from the GPU's own rounding


def test_fit_recovers_a_tree_from_its_renders(torch_cuda):
    torch = torch_cuda
    rng = np.random.default_rng(12)
    l_max = 4.0
    gt = random_tree(4, rng, sh_degree=2, p_split=0.5, p_empty=0.2, sigma_range=(0.5, 8.0), emissive=1.0)
    gt.sh[:] = rng.normal(0.0, 1.0, gt.sh.shape)
    gtt = plo.Tree(gt)
    prm = plo.RenderParams(activation=plo.ACT_SIGMOID, l_max=l_max)

    def batch(seed, n):
        r = torch.from_numpy(plogen.rays_sphere(n, seed=seed)).cuda()
        rgb, T, _ = plo.render(gtt, r, prm)
        return r, rgb, (1.0 - T).contiguous()

    init = plogen.HostTree(gt.depth, 2, gt.child, np.full(gt.n_leaves, 1.0, np.float32),
                           np.zeros_like(gt.sh))
    n = 8192
    opt = plo.OctOpt(init, l_max, max_rays=n, lr_sigma=0.1, lr_sh=0.1, lr_decay=0.1, total_steps=400,
                     tv_sigma=1e-4, tv_sh=1e-4)
    losses = []
    for it in range(400):
        loss = opt.step(*batch(1000 + it, n))
        if it % 50 == 0 or it == 399:
            losses.append(float(loss[0]))
    opt.check()
    assert losses[-1] < 0.1 * losses[0], losses
    # held-out rays: the packed result renders what the optimiser composites
    r, rgb, a = batch(77, 4096)
    out = torch.empty((4096, 5), device="cuda")
    opt.grad(r, rgb, a, ray_out=out)
    fit = opt.build_tree()
    rgb_f, T_f, _ = plo.render(fit, r, prm)
    o = out.cpu().numpy()
    np.testing.assert_allclose(rgb_f.cpu().numpy(), o[:, :3], rtol=1e-4, atol=1e-5 * l_max)
    np.testing.assert_allclose(1.0 - T_f.cpu().numpy(), o[:, 3], rtol=1e-4, atol=1e-5)
    a_rmse = float(np.sqrt(np.mean((o[:, 3] - a.cpu().numpy()) ** 2)))
    a0 = float(np.sqrt(np.mean(a.cpu().numpy() ** 2)))
    rel = float(np.linalg.norm(o[:, :3] - rgb.cpu().numpy()) / np.linalg.norm(rgb.cpu().numpy()))
    assert a_rmse < 0.1 * a0 and rel < 0.1, (a_rmse, a0, rel)


def test_edge_cases(torch_cuda):
    torch = torch_cuda
    tree, init, s, k, rays, C_gt, a_gt = _problem(7, depth=3, n=64)
    opt = plo.OctOpt(init, 2.0, max_rays=64, max_cells=4)
    before = opt.read(plo.OCTOPT_SH)
    e = torch.empty((0, 6), device="cuda")
    opt.step(e, torch.empty((0, 3), device="cuda"), torch.empty(0, device="cuda"))
    np.testing.assert_array_equal(opt.read(plo.OCTOPT_SH), before)
    # rays crossing more than max_cells cells are left out and flagged
    out = torch.empty((64, 5), device="cuda")
    opt.grad(*_dev(torch, rays, C_gt, a_gt), ray_out=out)
    with pytest.raises(plo.PloError) as ei:
        opt.check()
    assert ei.value.status == -5
    o = out.cpu().numpy()
    assert np.isnan(o[:, 0]).any()
    opt.check()  # the flag was cleared
    # rays that miss the box contribute nothing
    miss = np.tile(np.array([[5.0, 5.0, 5.0, 1.0, 0.0, 0.0]], np.float32), (8, 1))
    opt2 = plo.OctOpt(init, 2.0, max_rays=8)
    loss = opt2.grad(*_dev(torch, miss, np.zeros((8, 3), np.float32), np.zeros(8, np.float32)))
    assert float(loss[0]) == 0.0
    assert not opt2.read(plo.OCTOPT_GRAD_SIGMA).any() and not opt2.read(plo.OCTOPT_GRAD_SH).any()
    with pytest.raises(ValueError):
        opt2.grad(*_dev(torch, rays[:9], C_gt[:9], a_gt[:9]))
