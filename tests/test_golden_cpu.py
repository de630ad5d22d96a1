"""The constants the paper prints (tests/golden/paper_constants.json, each
with the section that states it) against the defaults of the FP64 oracle
and of the library's binding: the network's shape and output count, the
loss's epsilon, the sample counts, the learning-rate schedule's ends, the
distillation's threshold and sample count, the octree depth and the
render heuristics."""
import inspect
import json
import os

import pytest

import oracle.mlp as omlp
import paper_2207_05009_gb300 as plo
import plogen

_GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_constants.json")))
C = {c["name"]: c["value"] for c in _GOLD["constants"]}


def default(fn, name):
    return inspect.signature(fn).parameters[name].default


def test_every_constant_is_cited():
    for c in _GOLD["constants"]:
        assert c["cite"].startswith("Sec. "), c


def test_network_shape():
    assert omlp.DEPTH == C["trunk_layers"]
    assert omlp.WIDTH == C["trunk_width"]
    assert omlp.FEAT == C["output_hidden_width"]
    l_max = C["l_max_default"]
    shapes = omlp.layer_shapes_paper(l_max=l_max)
    assert sum(1 for o, _ in shapes if o == C["trunk_width"]) == C["trunk_layers"]
    # the output layer: 3 (l_max + 1)^2 SH coefficients from the 128-wide layer
    assert shapes[-1] == (3 * (l_max + 1) ** 2, C["output_hidden_width"])
    assert 3 * (l_max + 1) ** 2 == 27


def test_training_constants():
    assert default(plo.Mlp.__init__, "lr0") == C["lr_start"] == default(omlp.lr_at, "lr0")
    assert default(plo.Mlp.__init__, "lr1") == C["lr_end"] == default(omlp.lr_at, "lr1")
    total = 1000
    assert omlp.lr_at(0, total) == pytest.approx(C["lr_start"], rel=1e-12)
    assert omlp.lr_at(total, total) == pytest.approx(C["lr_end"], rel=1e-12)
    assert default(plo.Mlp.__init__, "eps") == C["hdr_loss_eps"] == default(omlp.loss_terms, "eps")
    assert default(plo.Mlp.train_step_hier, "n_coarse") == C["n_coarse"]
    assert default(plo.Mlp.train_step_hier, "n_fine") == C["n_fine"]


def test_distillation_constants():
    assert default(plo.Mlp.distill, "sigma_thresh") == C["distill_sigma_threshold"]
    assert default(omlp.distill_dense, "sigma_thresh") == C["distill_sigma_threshold"]
    # the device distillation takes 1..256 samples per kept voxel: the
    # paper's count is the largest (its GPU parity runs at 4 and 256)
    with open(os.path.join(os.path.dirname(os.path.dirname(__file__)), "include", "plo.h")) as f:
        assert f"(1..{C['distill_samples_per_voxel']})" in f.read()
    assert plogen.LUMINAIRE_D10.depth == C["octree_depth"]


def test_render_heuristics():
    p = plo.RenderParams.paper_heuristics()
    assert p.sigma_min == C["sigma_min"]
    assert p.t_stop == pytest.approx(1.0 - C["alpha_max"])
    assert p.saturate
