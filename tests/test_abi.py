"""CPU-side checks of the C ABI: the library builds and loads, exports every
function include/plo.h declares, and the host validator rejects malformed
trees (no GPU needed: validation runs before any CUDA call)."""
import ctypes
import os
import re

import numpy as np
import pytest

import paper_2207_05009_gb300 as plo
import plogen
from plogen import HostTree
from tests.trees import random_tree, uniform_tree

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            src = open(os.path.join(ROOT, "include", fn)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names |= set(re.findall(r"\b(plo_[a-z0-9_]+)\s*\(", src))
    return sorted(names)


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("plo_build_tree", "plo_render_rays", "plo_tree_free", "plo_last_error"):
        assert required in names


def test_library_exports_every_declared_symbol():
    lib = plo.load()
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_version_string():
    assert b"sm_103a" in plo.load().plo_version()


def _expect(tree, status):
    with pytest.raises(plo.PloError) as ei:
        plo.validate(tree)
    assert ei.value.status == status, str(ei.value)


def test_validator_accepts_good_trees():
    plo.validate(plogen.luminaire_tree(plogen.LUMINAIRE_D6))
    plo.validate(uniform_tree(0, 1.0, np.ones((3, 9))))
    plo.validate(HostTree(0, 2, np.zeros((0, 8), np.int32), np.zeros(0, np.float32), np.zeros((0, 3, 9), np.float32)))
    plo.validate(random_tree(5, np.random.default_rng(0)))


def test_validator_rejects_malformed_trees():
    BAD, ARG = -2, -1
    base = random_tree(3, np.random.default_rng(1), p_split=0.9)
    # child index out of range
    t = HostTree(base.depth, 2, base.child.copy(), base.sigma, base.sh)
    t.child[0, 0] = base.n_nodes + 5
    _expect(t, BAD)
    # cycle back to the root
    t = HostTree(base.depth, 2, base.child.copy(), base.sigma, base.sh)
    inner = np.argwhere(t.child >= 1)[0]
    t.child[t.child[tuple(inner)], 0] = 0
    _expect(t, BAD)
    # leaf referenced twice
    t = HostTree(base.depth, 2, base.child.copy(), base.sigma, base.sh)
    leaves = np.argwhere(t.child <= -2)
    t.child[tuple(leaves[1])] = t.child[tuple(leaves[0])]
    _expect(t, BAD)
    # leaf id out of range
    t = HostTree(base.depth, 2, base.child.copy(), base.sigma, base.sh)
    t.child[tuple(leaves[0])] = -base.n_leaves - 10
    _expect(t, BAD)
    # node below the declared depth
    t = HostTree(1, 2, base.child, base.sigma, base.sh)
    _expect(t, BAD)
    # negative and NaN sigma, NaN SH
    for field, val in (("sigma", -1.0), ("sigma", np.nan), ("sh", np.inf)):
        t = HostTree(base.depth, 2, base.child, base.sigma.copy(), base.sh.copy())
        getattr(t, field).reshape(-1)[0] = val
        _expect(t, BAD)
    # parameter errors
    _expect(HostTree(17, 2, base.child, base.sigma, base.sh), ARG)
    _expect(HostTree(base.depth, 5, base.child, base.sigma, np.zeros((base.n_leaves, 3, 36), np.float32)), ARG)
    plo.validate(HostTree(base.depth, 4, base.child, base.sigma, np.zeros((base.n_leaves, 3, 25), np.float32)))
    t = HostTree(base.depth, 2, base.child, base.sigma, base.sh)
    t.bbox_min, t.bbox_max = (0, 0, 0), (1, 0, 1)
    _expect(t, ARG)
    # two leaves without nodes
    _expect(HostTree(0, 2, np.zeros((0, 8), np.int32), np.ones(2, np.float32), np.zeros((2, 3, 9), np.float32)), BAD)


def test_build_rejects_bad_precision_before_any_device_work():
    t = uniform_tree(1, 1.0, np.ones((3, 9)))
    with pytest.raises(plo.PloError) as ei:
        plo.Tree(t, 7)
    assert ei.value.status == -1 and "precision" in str(ei.value)
    with pytest.raises(plo.PloError) as ei:
        bad = t.child.copy()
        bad[0, 3] = 99
        plo.Tree(HostTree(1, 2, bad, t.sigma, t.sh), plo.PREC_FP16)
    assert ei.value.status == -2


def test_missing_library_fails_loudly(tmp_path):
    """Without the CUDA library the binding raises; there is no fallback."""
    import subprocess
    import sys
    code = ("import sys; sys.path.insert(0, %r)\n"
            "import paper_2207_05009_gb300 as plo\n"
            "from paper_2207_05009_gb300 import _build\n"
            "_build.LIB = %r\n"
            "plo._lib = None\n"
            "try:\n"
            "    plo.load(build=False)\n"
            "except RuntimeError as e:\n"
            "    print('raised:', e)\n"
            "    sys.exit(0)\n"
            "sys.exit(1)\n") % (ROOT, str(tmp_path / "absent" / "libplo.so"))
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0, r.stdout + r.stderr
    assert "libplo.so not found" in r.stdout
