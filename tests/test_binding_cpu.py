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
