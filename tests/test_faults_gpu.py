"""Failure detection without faulting the GPU: injected device-allocation
failures surface as PLO_ERR_OOM with everything already allocated released,
and a tensor-core pipeline whose barrier waits run out (a producer that
issues no loads) reports its error word and leaves the context usable."""
import numpy as np
import pytest

import paper_2207_05009_gb300 as plo
import plogen

pytestmark = pytest.mark.gpu


def test_allocation_failures_are_reported_and_cleaned_up(cuda_available):
    import torch
    tree = plogen.luminaire_tree(plogen.LUMINAIRE_D6)
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for k in range(4):  # fail the 1st .. 4th allocation of plo_build_tree
        plo.debug_fail_alloc_after(k)
        with pytest.raises(plo.PloError) as ei:
            plo.Tree(tree)
        assert ei.value.status == -3, str(ei.value)
    plo.debug_fail_alloc_after(0)
    with pytest.raises(plo.PloError) as ei:
        plo.Mlp(l_max=1.0)
    assert ei.value.status == -3
    plo.debug_fail_alloc_after(-1)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert abs(free1 - free0) < (64 << 20)  # nothing of the failed builds is left behind
    t = plo.Tree(tree)  # and the library works again
    rgb, T, _ = plo.render(t, torch.from_numpy(plogen.rays_sphere(1000, seed=1)).cuda())
    torch.cuda.synchronize()
    assert torch.isfinite(rgb).all()


def test_pipeline_wait_gives_up_and_context_survives(cuda_available):
    import torch
    g = torch.Generator(device="cuda").manual_seed(1)
    A = torch.randn(256, 64, device="cuda", generator=g).to(torch.bfloat16)
    B = torch.randn(256, 64, device="cuda", generator=g).to(torch.bfloat16)
    out = torch.zeros(256, 256, device="cuda", dtype=torch.bfloat16)
    err = torch.zeros(1, device="cuda", dtype=torch.int32)
    plo.debug_gemm_stall(A, B, out, err, wait_limit=1 << 14)
    torch.cuda.synchronize()
    assert int(err.item()) & 2
    # the context is still usable: a normal GEMM right after is correct
    bias = torch.zeros(256, device="cuda")
    res, err2 = plo.gemm_bf16(A, B, 1, bias=bias)
    torch.cuda.synchronize()
    assert int(err2.item()) == 0
    ref = A.float() @ B.float().t()
    assert float((res - ref).abs().max()) < 1e-3 * float(ref.abs().max())
