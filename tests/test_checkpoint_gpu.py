"""Checkpoint and resume of a training run (plo_mlp_save / plo_mlp_load):
ten steps, save, load into a fresh network, ten more steps, against twenty
uninterrupted steps.  The sample jitter is drawn from (seed, step) in both
runs, so the resumed run also checks that the random stream is restored."""
import numpy as np
import pytest

import paper_2207_05009_gb300 as plo
import plogen
from tests import ckpt_format

pytestmark = pytest.mark.gpu

LR0 = 5e-4


def batches(torch, n, R=64, seed=70):
    rng = np.random.default_rng(seed)
    out = []
    for k in range(n):
        rays = torch.from_numpy(plogen.rays_sphere(R, seed=seed + k)).cuda()
        C = torch.from_numpy(rng.uniform(0, 5, (R, 3)).astype(np.float32)).cuda()
        a = torch.from_numpy(rng.uniform(0, 1, R).astype(np.float32)).cuda()
        out.append((rays, C, a))
    return out


@pytest.mark.parametrize("arch", [plo.ARCH_LINEAR_HEAD, plo.ARCH_PAPER])
def test_resume_matches_uninterrupted_training(cuda_available, tmp_path, arch):
    import torch
    data = batches(torch, 20)
    kw = dict(l_max=6.0, total_steps=15, seed=3, jitter_seed=9, init_radiance=1.5, arch=arch, lr0=LR0)
    straight = plo.Mlp(**kw)
    for rays, C, a in data:
        straight.train_step(rays, C, a, n_samples=32)
    first = plo.Mlp(**kw)
    for rays, C, a in data[:10]:
        first.train_step(rays, C, a, n_samples=32)
    path10 = str(tmp_path / "step10.plomlp")
    first.save(path10)
    desc, step = plo.checkpoint_info(path10)
    assert step == 10 and desc["arch"] == arch and desc["seed"] == 9
    first.free()
    resumed = plo.Mlp.load(path10)
    assert resumed.step == 10
    for rays, C, a in data[10:]:
        resumed.train_step(rays, C, a, n_samples=32)
    torch.cuda.synchronize()
    straight.check()
    resumed.check()
    assert resumed.step == 20
    p_s, p_r = straight.get_params(), resumed.get_params()
    # Weight gradients are summed with float atomics, so two runs differ in
    # the last bits of every gradient; where a gradient is itself at the
    # rounding level (near zero), Adam's m / sqrt(v) turns that noise into
    # a step of up to ~lr, so a few parameters may differ by that much, and
    # ten more steps let the two trajectories drift apart by ~1e-4 lr
    # (measured median for the paper architecture: 2.6e-4 lr).  A lost Adam
    # moment or jitter stream changes every update by O(lr), a lost step
    # count the learning rate 20x: either moves the median past 1e-2 lr.
    d = np.abs(p_s.astype(np.float64) - p_r)
    assert np.median(d) <= 1e-3 * LR0 and np.percentile(d, 99) <= 3e-2 * LR0, (np.median(d),
                                                                               np.percentile(d, 99), d.max())
    assert d.max() <= 20 * LR0
    a_path, b_path = str(tmp_path / "a.plomlp"), str(tmp_path / "b.plomlp")
    straight.save(a_path)
    resumed.save(b_path)
    (ha, ba), (hb, bb) = ckpt_format.read(a_path), ckpt_format.read(b_path)
    assert ha["step"] == hb["step"] == 20
    # Adam's moments are averages of the gradients the two runs saw, which
    # differ as the parameters drift (measured median 2.5e-3 relative); a
    # lost first moment would leave out 0.9^10 = 35% of its weight, a lost
    # second moment about half of it
    for name in ("adam_m", "adam_v"):
        rel = np.abs(bb[name].astype(np.float64) - ba[name]) / (np.abs(ba[name]) + 1e-30)
        assert np.median(rel) <= 3e-2, (name, np.median(rel))
    np.testing.assert_array_equal(bb["master"], p_r)


def test_load_rejects_weights_that_do_not_match_the_masters(cuda_available, tmp_path):
    import torch
    net = plo.Mlp(l_max=6.0, init_radiance=1.5)
    rays, C, a = batches(torch, 1)[0]
    net.train_step(rays, C, a, n_samples=32)
    good = str(tmp_path / "good.plomlp")
    net.save(good)
    head, blobs = ckpt_format.read(good)
    data = bytearray(open(good, "rb").read())
    o = head["weights_bf16_offset"] + 2 * 1000
    data[o] ^= 0x40  # flip a bit of one bf16 weight
    bad = str(tmp_path / "bad.plomlp")
    open(bad, "wb").write(bytes(data))
    with pytest.raises(plo.PloError, match="bf16"):
        plo.Mlp.load(bad)
    again = plo.Mlp.load(good)
    np.testing.assert_array_equal(again.get_params(), net.get_params())
