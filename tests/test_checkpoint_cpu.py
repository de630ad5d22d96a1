"""The network checkpoint format (plo_mlp_save / plo_mlp_load) on CPU: a file
written from the format's description is read back by the library's
host-only header reader, and malformed files are rejected."""
import numpy as np
import pytest

import paper_2207_05009_gb300 as plo
from tests import ckpt_format

DESC = dict(arch=plo.ARCH_LINEAR_HEAD, sh_degree=3, transmittance=plo.TRANS_EXP, loss=plo.LOSS_PAPER,
            total_steps=5000, l_max=4096.5, eps=0.01, lr0=5e-4, lr1=5e-6, init_radiance=37.25,
            seed=18446744073709551557)


def n_weights(arch):
    n_out = 49
    blocks = [(256, 63)] + [(256, 256)] * 7
    blocks += [(n_out, 256)] if arch == plo.ARCH_LINEAR_HEAD else [(1, 256), (128, 256), (n_out - 1, 128)]
    return sum(r * c for r, c in blocks)


def make(path, desc=DESC, step=1234, n=None):
    n = n if n is not None else int(plo.mlp_lib().plo_mlp_param_count_arch(3, desc["arch"]))
    rng = np.random.default_rng(0)
    ckpt_format.write(path, desc, step, rng.random(n), rng.random(n), rng.random(n),
                      rng.integers(0, 1 << 16, n_weights(desc["arch"])))


@pytest.mark.parametrize("arch", [plo.ARCH_LINEAR_HEAD, plo.ARCH_PAPER])
def test_header_round_trips(tmp_path, arch):
    path = str(tmp_path / "net.plomlp")
    desc = dict(DESC, arch=arch)
    make(path, desc)
    got, step = plo.checkpoint_info(path)
    assert step == 1234
    for k, v in desc.items():
        assert got[k] == pytest.approx(v, rel=0, abs=0) if isinstance(v, int) else np.float32(got[k]) == np.float32(v)
    head, blobs = ckpt_format.read(path)
    assert head["n_params"] == plo.mlp_lib().plo_mlp_param_count_arch(3, arch)
    assert blobs["master"].size == head["n_params"]


def test_malformed_files_are_rejected(tmp_path):
    good = str(tmp_path / "good.plomlp")
    make(good)
    data = open(good, "rb").read()
    cases = {
        "magic": b"XLOMLP01" + data[8:],
        "truncated": data[:-10],
        "header": data[:8] + (10 ** 9).to_bytes(8, "little") + data[16:],
    }
    for name, blob in cases.items():
        p = str(tmp_path / f"{name}.plomlp")
        open(p, "wb").write(blob)
        with pytest.raises(plo.PloError) as ei:
            plo.checkpoint_info(p)
        assert ei.value.status == -1, name
    wrong_n = str(tmp_path / "n.plomlp")
    make(wrong_n, n=1000)
    with pytest.raises(plo.PloError, match="n_params"):
        plo.checkpoint_info(wrong_n)
    bad_desc = str(tmp_path / "d.plomlp")
    make(bad_desc, dict(DESC, loss=7))
    with pytest.raises(plo.PloError, match="loss"):
        plo.checkpoint_info(bad_desc)
    with pytest.raises(plo.PloError):
        plo.checkpoint_info(str(tmp_path / "missing.plomlp"))
