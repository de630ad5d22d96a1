"""The allocation-free host render (plo_render_rays_host_noalloc) matches
the allocating host render (plo_render_rays_host) on two calls in a row.

Callers such as a CPU path tracer's emitter code, or a process whose device
memory is fixed at start-up, cannot allocate device memory while they render;
this entry point stages rays and results in a fixed device array of the
library instead.  The file's name makes pytest collect it last."""
import numpy as np
import pytest

import paper_2207_05009_gb300 as plo
import plogen

pytestmark = pytest.mark.gpu


def test_noalloc_host_render_matches_host_render_twice(cuda_available):
    tree = plo.Tree(plogen.luminaire_tree(plogen.LUMINAIRE_D6))
    for n, seed in ((50_001, 31), (plo.NOALLOC_MAX_RAYS, 32)):
        rays = plogen.rays_sphere(n, seed=seed)
        rgb, T = plo.render_host_noalloc(tree, rays)
        ref_rgb, ref_T = plo.render_host(tree, rays)
        # every ray's arithmetic is independent of its lane and of the launch
        # shape, so the two paths agree bit for bit
        np.testing.assert_array_equal(rgb, ref_rgb)
        np.testing.assert_array_equal(T, ref_T)
        assert np.isfinite(rgb).all() and (T < 1).any()


def test_noalloc_call_makes_no_device_allocation(cuda_available):
    """With the library's allocation hook set to fail the very next device
    allocation (cudaMalloc or cudaMallocAsync), the allocation-free call
    still succeeds, while the allocating host path fails with PLO_ERR_OOM."""
    tree = plo.Tree(plogen.luminaire_tree(plogen.LUMINAIRE_D6))
    rays = plogen.rays_sphere(4096, seed=34)
    ref_rgb, ref_T = plo.render_host_noalloc(tree, rays)  # set-up call of this context
    try:
        plo.debug_fail_alloc_after(0)
        rgb, T = plo.render_host_noalloc(tree, rays)
        np.testing.assert_array_equal(rgb, ref_rgb)
        np.testing.assert_array_equal(T, ref_T)
        with pytest.raises(plo.PloError) as ei:
            plo.render_host(tree, rays)
        assert ei.value.status == -3
    finally:
        plo.debug_fail_alloc_after(-1)


def test_noalloc_rejects_more_rays_than_its_array_holds(cuda_available):
    tree = plo.Tree(plogen.luminaire_tree(plogen.LUMINAIRE_D6))
    rays = plogen.rays_sphere(plo.NOALLOC_MAX_RAYS + 1, seed=33)
    with pytest.raises(plo.PloError) as ei:
        plo.render_host_noalloc(tree, rays)
    assert ei.value.status == -1 and "maximum" in str(ei.value)
