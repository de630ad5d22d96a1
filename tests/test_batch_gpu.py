"""Batched render of several luminaires in one persistent launch (one ray
queue, mixed depths, SH degrees and leaf precisions): identical per-ray
results to separate plo_render_rays launches, through a direct launch, a
captured CUDA graph, and after autotuning."""
import numpy as np
import pytest

import paper_2207_05009_gb300 as plo
import plogen

pytestmark = pytest.mark.gpu


def test_batch_equals_separate_launches(cuda_available, tmp_path):
    import torch
    recs = [plogen.LUMINAIRE_D6, plogen.LUMINAIRE_D6.with_(depth=7, sh_degree=3, seed=5),
            plogen.LUMINAIRE_D6.with_(depth=5, sh_degree=1, seed=6), plogen.LUMINAIRE_D6.with_(depth=8, seed=7)]
    precs = [plo.PREC_FP32, plo.PREC_FP16, plo.PREC_FP32, plo.PREC_BF16]
    trees = [plo.Tree(plogen.luminaire_tree(r), p) for r, p in zip(recs, precs)]
    counts = [70_001, 1_000, 250_037, 33]
    offs = np.concatenate([[0], np.cumsum(counts)])
    rays_np = np.concatenate([plogen.rays_sphere(c, seed=50 + i) for i, c in enumerate(counts)])
    rays = torch.from_numpy(rays_np).cuda()
    n = len(rays_np)
    ref_rgb = torch.empty((n, 3), device="cuda")
    ref_T = torch.empty(n, device="cuda")
    for t, (a, b) in zip(trees, zip(offs[:-1], offs[1:])):
        plo.render(t, rays[a:b], rgb=ref_rgb[a:b], T=ref_T[a:b])
    batch = plo.Batch(trees, offs)
    rgb = torch.full((n, 3), -1.0, device="cuda")
    T = torch.full((n,), -1.0, device="cuda")
    st = torch.full((n,), -9, dtype=torch.int32, device="cuda")
    batch.render(rays, rgb, T, st)
    torch.cuda.synchronize()
    assert torch.equal(rgb, ref_rgb) and torch.equal(T, ref_T)
    assert int(st.max()) == 0 and int(st.min()) == 0
    # captured graph, replayed twice
    rgb2 = torch.full((n, 3), -1.0, device="cuda")
    T2 = torch.full((n,), -1.0, device="cuda")
    batch.capture(rays, rgb2, T2)
    batch.replay()
    torch.cuda.synchronize()
    assert torch.equal(rgb2, ref_rgb) and torch.equal(T2, ref_T)
    rgb2.fill_(-1.0)
    batch.replay()
    torch.cuda.synchronize()
    assert torch.equal(rgb2, ref_rgb)
    # autotune (cached in a file) keeps the results identical
    cfg, src = plo.autotune_cached(batch, "test", rays, rgb, T, path=str(tmp_path / "tune.json"))
    assert src == "tuned" and cfg["claim_rays"] % 32 == 0
    cfg2, src2 = plo.autotune_cached(batch, "test", rays, rgb, T, path=str(tmp_path / "tune.json"))
    assert src2 == "cache" and cfg2["claim_rays"] == cfg["claim_rays"]
    rgb.fill_(-1.0)
    batch.render(rays, rgb, T)
    torch.cuda.synchronize()
    assert torch.equal(rgb, ref_rgb) and torch.equal(T, ref_T)
