"""The Python binding checks the buffers a caller hands it before any
pointer reaches the library (which trusts the sizes it is given), on CPU."""
import numpy as np
import pytest
import torch

import paper_2207_05009_gb300 as plo


def test_require_rejects_wrong_shape_dtype_layout_and_device():
    ok = torch.zeros(4, 3)
    plo._require(ok, "rgb", (4, 3), torch.float32, cuda=False)
    with pytest.raises(ValueError, match="shape"):
        plo._require(torch.zeros(5, 3), "rgb", (4, 3), torch.float32, cuda=False)
    with pytest.raises(ValueError, match="float32"):
        plo._require(torch.zeros(4, 3, dtype=torch.float64), "rgb", (4, 3), torch.float32, cuda=False)
    with pytest.raises(ValueError, match="not contiguous"):
        plo._require(torch.zeros(3, 4).t(), "rgb", (4, 3), torch.float32, cuda=False)
    with pytest.raises(ValueError, match="CUDA"):
        plo._require(ok, "rgb", (4, 3), torch.float32, cuda=True)


def test_host_render_checks_its_buffers_before_the_library():
    rays = np.zeros((8, 6), np.float32)
    with pytest.raises(ValueError, match="rgb"):
        plo.render_host(None, rays, rgb=np.zeros((7, 3), np.float32))
    with pytest.raises(ValueError, match="T"):
        plo.render_host(None, rays, T=np.zeros(8, np.float64))
    with pytest.raises(ValueError, match=r"\[n, 6\]"):
        plo.render_host(None, np.zeros((8, 5), np.float32))
    with pytest.raises(ValueError, match="rgb"):
        plo.render_host(None, torch.zeros(8, 6), rgb=torch.zeros(8, 4))
    with pytest.raises(ValueError, match=r"\[n, 6\]"):
        plo.render_host_noalloc(None, np.zeros((8, 3), np.float32))


def test_device_render_rejects_host_rays():
    with pytest.raises(ValueError, match="CUDA"):
        plo.render(None, torch.zeros(8, 6))


def test_device_render_rejects_rays_of_the_wrong_rank():
    with pytest.raises(ValueError, match=r"\[n, 6\]"):
        plo.render(None, torch.zeros(8, 2, 6))


def test_batch_checks_its_buffers_against_the_ray_count():
    b = plo.Batch.__new__(plo.Batch)  # no library handle: the checks run first
    b.n_rays = 16
    rays, rgb, T = torch.zeros(16, 6), torch.zeros(16, 3), torch.zeros(16)
    with pytest.raises(ValueError, match="rays"):
        b.render(torch.zeros(15, 6), rgb, T)
    with pytest.raises(ValueError, match="rgb"):
        b.capture(rays, torch.zeros(16, 4), T)
    with pytest.raises(ValueError, match="T"):
        b.autotune(rays, rgb, torch.zeros(16, dtype=torch.float64))
    with pytest.raises(ValueError, match="status"):
        b.render(rays, rgb, T, status=torch.zeros(16, dtype=torch.int64))
    with pytest.raises(ValueError, match="CUDA"):  # right shapes, host memory
        b.render(rays, rgb, T)


def test_network_calls_check_their_buffers():
    net = plo.Mlp.__new__(plo.Mlp)
    rays, rgb, alpha = torch.zeros(64, 6), torch.zeros(64, 3), torch.zeros(64)
    with pytest.raises(ValueError, match="points"):
        net.forward(torch.zeros(10, 4))
    with pytest.raises(ValueError, match="rgb_gt"):
        net.train_step(rays, torch.zeros(63, 3), alpha)
    with pytest.raises(ValueError, match="alpha_gt"):
        net.train_step(rays, rgb, torch.zeros(64, 1))
    with pytest.raises(ValueError, match="jitter"):
        net.train_step(rays, rgb, alpha, n_samples=32, jitter=torch.zeros(64, 16))
    with pytest.raises(ValueError, match="xi"):
        plo.Mlp.train_step_hier(net, net, rays, rgb, alpha, n_coarse=64, n_fine=128, xi=torch.zeros(64, 64))


def test_tensor_core_entry_points_check_their_buffers():
    bf = torch.bfloat16
    A, B = torch.zeros(128, 64, dtype=bf), torch.zeros(256, 64, dtype=bf)
    with pytest.raises(ValueError, match="B"):
        plo.gemm_bf16(A, torch.zeros(256, 32, dtype=bf), 1)
    with pytest.raises(ValueError, match="bias"):
        plo.gemm_bf16(A, B, 1, bias=torch.zeros(255))
    with pytest.raises(ValueError, match="mask"):
        plo.gemm_bf16(A, B, 2, mask=torch.zeros(128, 256))
    with pytest.raises(ValueError, match="bits"):
        plo.gemm_bf16(A, B, 0, bits=torch.zeros(128, 7, dtype=torch.int32))
    with pytest.raises(ValueError, match="out"):
        plo.gemm_bf16(A, B, 1, out=torch.zeros(128, 256, dtype=bf))
    with pytest.raises(ValueError, match="dW"):
        plo.wgrad_bf16(torch.zeros(64, 256, dtype=bf), torch.zeros(64, 64, dtype=bf), torch.zeros(64, 256))
    with pytest.raises(ValueError, match="db"):
        plo.wgrad_bf16(torch.zeros(64, 256, dtype=bf), torch.zeros(64, 64, dtype=bf), torch.zeros(256, 64),
                       db=torch.zeros(64))
    with pytest.raises(ValueError, match="delta"):
        plo.hier_samples(torch.zeros(8, 6), torch.zeros(8, 64), torch.zeros(8, 63), torch.zeros(8, 64),
                         torch.zeros(8, 128))


def test_network_handle_class_keeps_its_methods():
    # the class must keep free / __del__ (a module-level function defined in
    # the middle of the class once swallowed them)
    for name in ("free", "__del__", "save", "load", "quad", "activation", "train_step", "distill"):
        assert callable(getattr(plo.Mlp, name)), name
    assert callable(plo.checkpoint_info)


def test_leaf_optimiser_checks_its_buffers():
    opt = plo.OctOpt.__new__(plo.OctOpt)  # no library handle: the checks run first
    opt.n_leaves, opt.K, opt.max_rays = 10, 9, 64
    rays, rgb, alpha = torch.zeros(64, 6), torch.zeros(64, 3), torch.zeros(64)
    with pytest.raises(ValueError, match="rgb_gt"):
        opt.grad(rays, torch.zeros(63, 3), alpha)
    with pytest.raises(ValueError, match="alpha_gt"):
        opt.step(rays, rgb, torch.zeros(64, 2))
    with pytest.raises(ValueError, match="ray_out"):
        opt.grad(rays, rgb, alpha, ray_out=torch.zeros(64, 4))
    with pytest.raises(ValueError, match="loss_out"):
        opt.step(rays, rgb, alpha, loss_out=torch.zeros(2))
    with pytest.raises(ValueError, match="max_rays"):
        opt.grad(torch.zeros(65, 6), torch.zeros(65, 3), torch.zeros(65))
    with pytest.raises(ValueError, match="values"):
        opt.write(plo.OCTOPT_SH, np.zeros((10, 3, 8), np.float32))
    with pytest.raises(ValueError, match="unknown array"):
        opt.read(99)
    for name in ("free", "__del__", "grad", "step", "read", "write", "check", "build_tree"):
        assert callable(getattr(plo.OctOpt, name)), name
