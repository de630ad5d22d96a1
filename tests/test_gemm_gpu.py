"""tcgen05 GEMM building blocks vs a plain PyTorch FP32 reference of the same
op on the same bf16 inputs."""
import numpy as np
import pytest

import paper_2207_05009_gb300 as plo

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_cuda(cuda_available):
    import torch
    return torch


def rel_err(a, b):
    return float((a - b).abs().max() / (b.abs().max() + 1e-30))


@pytest.mark.parametrize("N,K", [(256, 64), (256, 256), (64, 256)])
@pytest.mark.parametrize("M", [128, 1000, 65536 + 64])
def test_gemm_epilogues(torch_cuda, N, K, M):
    torch = torch_cuda
    g = torch.Generator(device="cuda").manual_seed(M + N + K)
    A = (torch.randn(M, K, device="cuda", generator=g) * 0.5).to(torch.bfloat16)
    B = (torch.randn(N, K, device="cuda", generator=g) * 0.1).to(torch.bfloat16)
    bias = torch.randn(N, device="cuda", generator=g) * 0.1
    ref = A.float() @ B.float().t()
    out, err = plo.gemm_bf16(A, B, 1, bias=bias)
    torch.cuda.synchronize()
    assert int(err.item()) == 0
    assert rel_err(out, ref + bias) < 1e-5
    out, err = plo.gemm_bf16(A, B, 0, bias=bias)
    r = torch.relu(ref + bias).to(torch.bfloat16)
    assert (out.float() - r.float()).abs().max() <= 2 ** -7 * r.float().abs().max() + 1e-6
    mask = torch.randn(M, N, device="cuda", generator=g).to(torch.bfloat16)
    mask[::7] = 0.0
    out, err = plo.gemm_bf16(A, B, 2, mask=mask)
    r = (ref * (mask.float() > 0)).to(torch.bfloat16)
    torch.cuda.synchronize()
    assert int(err.item()) == 0
    assert (out.float() - r.float()).abs().max() <= 2 ** -7 * r.float().abs().max() + 1e-6
    # ReLU with its positive outputs as bits, then the same mask applied from
    # those bits: bit-identical to the bf16-mask epilogue with the ReLU output
    bits = torch.full((M, N // 32), -1, device="cuda", dtype=torch.int32)
    h, err = plo.gemm_bf16(A, B, 0, bias=bias, bits=bits)
    h2, _ = plo.gemm_bf16(A, B, 0, bias=bias)
    torch.cuda.synchronize()
    assert torch.equal(h, h2)
    # bits from the fp32 pre-activation: positive exactly where the bf16
    # ReLU output is (no pre-activation is small enough to round to zero)
    want = (h.float() > 0).reshape(M, N // 32, 32).to(torch.int64)
    want = (want << torch.arange(32, device="cuda", dtype=torch.int64)).sum(-1)
    assert torch.equal(bits.to(torch.int64) & 0xFFFFFFFF, want)
    out_b, err = plo.gemm_bf16(A, B, 3, bits=bits)
    out_m, _ = plo.gemm_bf16(A, B, 2, mask=h)
    torch.cuda.synchronize()
    assert int(err.item()) == 0
    assert torch.equal(out_b, out_m)


@pytest.mark.parametrize("n_out,n_in,M", [(256, 256, 64), (256, 256, 524288), (64, 256, 4096), (256, 64, 8192)])
def test_weight_gradient(torch_cuda, n_out, n_in, M):
    torch = torch_cuda
    g = torch.Generator(device="cuda").manual_seed(n_out * 7 + n_in + M)
    dZ = (torch.randn(M, n_out, device="cuda", generator=g) * 0.1).to(torch.bfloat16)
    H = torch.relu(torch.randn(M, n_in, device="cuda", generator=g)).to(torch.bfloat16)
    dW = torch.full((n_out, n_in), 0.5, device="cuda")
    db = torch.full((n_out,), -0.25, device="cuda")
    dW, err = plo.wgrad_bf16(dZ, H, dW, db=db)
    ref = dZ.float().t() @ H.float() + 0.5
    ref_db = dZ.double().sum(0).float() - 0.25
    torch.cuda.synchronize()
    assert int(err.item()) == 0
    assert rel_err(dW, ref) < 1e-4
    # the bias gradient (column sums of dZ) from the same pass
    assert rel_err(db, ref_db) < 1e-4
    # without db the weight gradient alone
    dW2 = torch.zeros((n_out, n_in), device="cuda")
    plo.wgrad_bf16(dZ, H, dW2)
    torch.cuda.synchronize()
    assert rel_err(dW2, ref - 0.5) < 1e-4
