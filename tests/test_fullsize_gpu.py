"""Parity at the full size of the benchmark, in its launch configuration.

The depth-10 luminaire (31.9M leaves, SH degree 3) and the 16,777,216 room
rays that bench.py times, rendered by the same call (one launch over all
rays, warps claiming rays from the shared counter); the FP64 oracle checks a
sample of 262,145 of the outputs spread evenly over the array, the last ray
included (Eq. 3-5).
"""
import os

import numpy as np
import pytest

import bench
import oracle
import paper_2207_05009_gb300 as plo
from tests.parity import RTOL_FP16, RTOL_FP32, assert_radiance_close

pytestmark = pytest.mark.gpu


def test_full_size_workload_sampled_parity(cuda_available):
    import torch
    _, tree, rays_np, _ = bench.workload(10, 1 << 24, seed=bench.shard_seed(0))
    n = len(rays_np)
    idx = np.unique(np.concatenate([np.linspace(0, n - 1, 1 << 18).astype(np.int64), [n - 1]]))
    ref = oracle.render(tree, rays_np[idx], n_threads=len(os.sched_getaffinity(0)))
    rays = torch.from_numpy(rays_np).cuda()
    rgb = torch.empty((n, 3), device="cuda")
    T = torch.empty(n, device="cuda")
    st = torch.full((n,), -7, dtype=torch.int32, device="cuda")
    sel = torch.from_numpy(idx).cuda()
    for prec, rtol, name in ((plo.PREC_FP32, RTOL_FP32, "fp32"), (plo.PREC_FP16, RTOL_FP16, "fp16")):
        t = plo.Tree(tree, prec)
        plo.render(t, rays, plo.RenderParams(), rgb=rgb, T=T, status=st)
        torch.cuda.synchronize()
        t.check()
        assert int((st != 0).sum().item()) == 0, "a ray reported a status"
        assert_radiance_close(rgb[sel].cpu().numpy(), T[sel].cpu().numpy(), ref, rtol,
                              what=f"full-size {name} launch vs oracle")
        del t
