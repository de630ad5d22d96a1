"""Host-side checks of plo_octopt_create (no GPU): every configuration
field is validated, and unsupported trees are refused, before any device
work."""
import numpy as np
import pytest

import paper_2207_05009_gb300 as plo
import plogen
from tests.trees import uniform_tree


def _tree():
    return uniform_tree(2, 1.0, np.zeros(27))


@pytest.mark.parametrize("kw", [dict(transmittance=plo.TRANS_LINEAR_LITERAL), dict(transmittance=7), dict(loss=3),
                                dict(l_max=0.0), dict(l_max=float("inf")), dict(eps=-1.0), dict(lr_sigma=-0.1),
                                dict(lr_sh=float("nan")), dict(lr_decay=0.0), dict(lr_decay=1.5),
                                dict(total_steps=0), dict(tv_sigma=-1.0), dict(tv_sh=float("inf")),
                                dict(max_cells=-1)])
def test_bad_config_is_refused(kw):
    args = dict(l_max=1.0, max_rays=16)
    args.update(kw)
    l_max = args.pop("l_max")
    with pytest.raises(plo.PloError) as ei:
        plo.OctOpt(_tree(), l_max, **args)
    assert ei.value.status == -1


def test_bad_max_rays_and_tree_are_refused():
    with pytest.raises(plo.PloError) as ei:
        plo.OctOpt(_tree(), 1.0, max_rays=0)
    assert ei.value.status == -1
    t = _tree()
    t.sigma[3] = -1.0  # the initial densities must be a valid tree's
    with pytest.raises(plo.PloError) as ei:
        plo.OctOpt(t, 1.0, max_rays=4)
    assert ei.value.status == -2
    # depth 11: a chain of nodes down to one leaf
    child = np.full((11, 8), -1, np.int32)
    for i in range(10):
        child[i, 0] = i + 1
    child[10, 0] = -2
    deep = plogen.HostTree(11, 0, child, np.ones(1, np.float32), np.zeros((1, 3, 1), np.float32))
    plo.validate(deep)
    with pytest.raises(plo.PloError) as ei:
        plo.OctOpt(deep, 1.0, max_rays=4)
    assert ei.value.status == -7
