"""Parity at the full sizes of the benchmark, in its launch configuration.

- The depth-10 luminaire (31.9M leaves, SH degree 3) and the 16,777,216 room
  rays that bench.py times, rendered by the same call (one launch over all
  rays, warps claiming rays from the shared counter), FP32 and FP16 leaves.
- The depth-6 luminaire stored with FP16 and BF16 leaves on the same 16M
  rays: against the oracle on the exactly dequantised tree (arithmetic) and
  on the FP32 leaves (storage error).
- The 8-luminaire batch (depths 7-10, ~12M rays): the graph-captured
  persistent launch equals 8 separate launches bit for bit, and both match
  the oracle.
The FP64 oracle checks samples spread evenly over each output array, the
last ray included (Eq. 3-5).
"""
import os

import numpy as np
import pytest

import bench
import oracle
import paper_2207_05009_gb300 as plo
import plogen
from tests.parity import RTOL_BF16, RTOL_FP16, RTOL_FP32, assert_radiance_close, quantise_tree

pytestmark = pytest.mark.gpu

N_FULL = 1 << 24
CORES = len(os.sched_getaffinity(0))


def spread(n, k):
    """k indices spread evenly over [0, n), plus the last."""
    return np.unique(np.concatenate([np.linspace(0, n - 1, k).astype(np.int64), [n - 1]]))


@pytest.fixture(scope="module")
def room_rays(cuda_available):
    import torch
    rays_np = plogen.rays_room(N_FULL, seed=bench.shard_seed(0))
    return rays_np, torch.from_numpy(rays_np).cuda()


def render_all(torch, tree, rays, precision, layout=plo.LAYOUT_DEFAULT):
    n = rays.shape[0]
    rgb = torch.empty((n, 3), device="cuda")
    T = torch.empty(n, device="cuda")
    st = torch.full((n,), -7, dtype=torch.int32, device="cuda")
    t = plo.Tree(tree, precision, layout)
    plo.render(t, rays, plo.RenderParams(), rgb=rgb, T=T, status=st)
    torch.cuda.synchronize()
    t.check()
    assert int((st != 0).sum().item()) == 0, "a ray reported a status"
    return rgb, T


def test_full_size_workload_sampled_parity(room_rays):
    import torch
    rays_np, rays = room_rays
    tree = plogen.luminaire_tree(plogen.LUMINAIRE_D10.with_(depth=10))  # the bench's tree
    idx = spread(N_FULL, 1 << 18)
    ref = oracle.render(tree, rays_np[idx], n_threads=CORES)
    sel = torch.from_numpy(idx).cuda()
    for prec, rtol, name, layout in ((plo.PREC_FP32, RTOL_FP32, "fp32", plo.LAYOUT_DEFAULT),
                                     (plo.PREC_FP16, RTOL_FP16, "fp16", plo.LAYOUT_DEFAULT),
                                     (plo.PREC_FP32, RTOL_FP32, "fp32 octree layout", plo.LAYOUT_OCTREE)):
        rgb, T = render_all(torch, tree, rays, prec, layout)
        assert_radiance_close(rgb[sel].cpu().numpy(), T[sel].cpu().numpy(), ref, rtol,
                              what=f"full-size {name} launch vs oracle")
        del rgb, T


def test_16bit_leaves_depth6_on_16m_rays(room_rays):
    import torch
    rays_np, rays = room_rays
    tree = plogen.luminaire_tree(plogen.LUMINAIRE_D6)
    idx = spread(N_FULL, 1 << 17)
    sel = torch.from_numpy(idx).cuda()
    ref = oracle.render(tree, rays_np[idx], n_threads=CORES)
    for prec, name in ((plo.PREC_FP16, "fp16"), (plo.PREC_BF16, "bf16")):
        rgb, T = render_all(torch, tree, rays, prec)
        g_rgb, g_T = rgb[sel].cpu().numpy(), T[sel].cpu().numpy()
        ref_q = oracle.render(quantise_tree(tree, name), rays_np[idx], n_threads=CORES)
        assert_radiance_close(g_rgb, g_T, ref_q, RTOL_FP32, what=f"{name} leaves vs dequantised oracle")
        rtol = RTOL_FP16 if name == "fp16" else RTOL_BF16
        assert_radiance_close(g_rgb, g_T, ref, rtol, what=f"{name} leaves vs FP32-leaf oracle")


def test_batch_of_8_luminaires_full_size(cuda_available):
    import torch
    recs, counts = bench.batch_workload()
    hosts = [plogen.luminaire_tree(r) for r in recs]
    trees = [plo.Tree(h, plo.PREC_FP32) for h in hosts]
    rays_l = [plogen.rays_room(int(c), seed=300 + i) for i, c in enumerate(counts)]
    offs = np.concatenate([[0], np.cumsum(counts)])
    n = int(offs[-1])
    d_rays = torch.from_numpy(np.concatenate(rays_l)).cuda()
    rgb = torch.full((n, 3), -1.0, device="cuda")
    T = torch.full((n,), -1.0, device="cuda")
    batch = plo.Batch(trees, offs)
    batch.capture(d_rays, rgb, T)
    batch.replay()
    torch.cuda.synchronize()
    ref_rgb = torch.empty_like(rgb)
    ref_T = torch.empty_like(T)
    for t, (lo, hi) in zip(trees, zip(offs[:-1], offs[1:])):
        plo.render(t, d_rays[lo:hi], rgb=ref_rgb[lo:hi], T=ref_T[lo:hi])
    torch.cuda.synchronize()
    assert torch.equal(rgb, ref_rgb) and torch.equal(T, ref_T)
    for h, r, (lo, hi) in zip(hosts, rays_l, zip(offs[:-1], offs[1:])):
        idx = spread(int(hi - lo), 4096)
        ref = oracle.render(h, r[idx], n_threads=CORES)
        sel = torch.from_numpy(idx + int(lo)).cuda()
        assert_radiance_close(rgb[sel].cpu().numpy(), T[sel].cpu().numpy(), ref, RTOL_FP32,
                              what=f"batched depth-{h.depth} luminaire vs oracle")
