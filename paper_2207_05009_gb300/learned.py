"""The learned part end to end (Sec. 4.2-4.4, Sec. 5): training targets
rendered from a ground-truth octree by the plain renderer, NeRF-SH training
with the library's kernels, distillation back into an octree, and the error of
that octree's renders against the ground truth.  Every step runs in libplo;
this module only sequences the calls."""
from __future__ import annotations

import time
from dataclasses import dataclass

import numpy as np

from . import (ACT_SIGMOID, ARCH_PAPER, LOSS_PAPER, PREC_FP32, Mlp, RenderParams, Tree, render)


def target_batches(gt_tree: Tree, ray_sets):
    """(rays, L_e, alpha) on the device for each float32 [n, 6] ray array,
    rendered from the ground-truth tree (exponential T, max(0,.) emission)."""
    import torch
    out = []
    for rays_np in ray_sets:
        rays = torch.from_numpy(np.ascontiguousarray(rays_np, np.float32)).cuda()
        rgb, T, _ = render(gt_tree, rays)
        out.append((rays, rgb, 1.0 - T))
    torch.cuda.synchronize()
    return out


def emission_scale(batches):
    """L_max (largest target radiance) and the mean emission of the opaque
    part of the rays (mean L_e / mean alpha), the network's starting level."""
    l_max = max(float(b[1].max().item()) for b in batches)
    mean_c = sum(float(b[1].mean().item()) for b in batches) / len(batches)
    mean_a = sum(float(b[2].mean().item()) for b in batches) / len(batches)
    return l_max, mean_c / max(mean_a, 1e-3)


def train(batches, steps: int, loss: int = LOSS_PAPER, n_samples: int = 128, l_max=None, init_radiance=None,
          seed: int = 1, lr0: float = 5e-4, lr1: float = 5e-6):
    """Trains a fresh network for `steps` steps cycling over the batches.
    Returns (network, per-step losses, seconds)."""
    import torch
    lm, c0 = emission_scale(batches)
    l_max = l_max or lm
    net = Mlp(l_max=l_max, loss=loss, total_steps=max(steps, 1), lr0=lr0, lr1=lr1, seed=seed,
              init_radiance=c0 if init_radiance is None else init_radiance)
    losses = torch.empty(max(steps, 1), device="cuda")
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for k in range(steps):
        rays, rgb, alpha = batches[k % len(batches)]
        net.train_step(rays, rgb, alpha, n_samples=n_samples, loss_out=losses[k:k + 1])
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    net.check()
    return net, losses[:steps].cpu().numpy(), dt


def train_hier(batches, steps: int, n_coarse: int = 64, n_fine: int = 128, l_max=None, init_radiance=None,
               seed: int = 1, lr0: float = 5e-4, lr1: float = 5e-6, arch: int = ARCH_PAPER):
    """The paper's full setup (Sec. 4.2-4.4): coarse and fine networks with
    the 128-wide SH output layer, N_c + N_f samples, loss L_c + L_f + L_alpha.
    Returns (coarse, fine, per-step losses, seconds)."""
    import torch
    lm, c0 = emission_scale(batches)
    l_max = l_max or lm
    kw = dict(l_max=l_max, loss=LOSS_PAPER, total_steps=max(steps, 1), lr0=lr0, lr1=lr1, arch=arch,
              init_radiance=c0 if init_radiance is None else init_radiance)
    coarse = Mlp(seed=seed, jitter_seed=2 * seed, **kw)
    fine = Mlp(seed=seed + 1, jitter_seed=2 * seed + 1, **kw)
    losses = torch.empty(max(steps, 1), device="cuda")
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for k in range(steps):
        rays, rgb, alpha = batches[k % len(batches)]
        Mlp.train_step_hier(coarse, fine, rays, rgb, alpha, n_coarse=n_coarse, n_fine=n_fine,
                            loss_out=losses[k:k + 1])
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    coarse.check()
    fine.check()
    return coarse, fine, losses[:steps].cpu().numpy(), dt


@dataclass
class DistillError:
    """Error of a distilled octree's renders against ground-truth renders."""
    rel_l2_radiance: float   # ||L_e - L_e_gt|| / ||L_e_gt|| over all rays and channels
    psnr: float              # PSNR of L_e / L_max clipped to [0, 1]
    alpha_rmse: float        # RMSE of alpha = 1 - T
    leaves: int
    distill_s: float


def tree_error(tree: Tree, l_max: float, test_batches):
    """(rel_l2_radiance, psnr, alpha_rmse) of a tree rendered with the
    sigmoid emission of scale l_max against the ground-truth batches."""
    import torch
    params = RenderParams(activation=ACT_SIGMOID, l_max=l_max)
    se_c = ss_c = se_n = se_a = 0.0
    n = 0
    for rays, rgb_gt, alpha_gt in test_batches:
        rgb, T, _ = render(tree, rays, params)
        alpha = 1.0 - T
        d = (rgb - rgb_gt).double()
        se_c += float((d * d).sum())
        ss_c += float((rgb_gt.double() ** 2).sum())
        dn = (rgb / l_max).clamp(0, 1).double() - (rgb_gt / l_max).clamp(0, 1).double()
        se_n += float((dn * dn).sum())
        da = (alpha - alpha_gt).double()
        se_a += float((da * da).sum())
        n += rays.shape[0]
    torch.cuda.synchronize()
    mse_n = se_n / (3 * n)
    return (float(np.sqrt(se_c / max(ss_c, 1e-300))), float(10 * np.log10(1.0 / max(mse_n, 1e-30))),
            float(np.sqrt(se_a / n)))


def distilled_error(net: Mlp, l_max: float, test_batches, depth: int, samples: int = 8,
                    sigma_thresh: float = 0.01, precision: int = PREC_FP32) -> DistillError:
    import torch
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    tree = net.distill(depth, samples=samples, sigma_thresh=sigma_thresh, precision=precision)
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    rel, psnr, a_rmse = tree_error(tree, l_max, test_batches)
    leaves = tree.info()["n_leaves"]
    tree.free()
    return DistillError(rel_l2_radiance=rel, psnr=psnr, alpha_rmse=a_rmse, leaves=int(leaves), distill_s=dt)
