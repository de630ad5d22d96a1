"""GPU parity of the learned part: network forward, training gradients and
loss against the FP64 oracle (oracle/mlp.py) on the same bf16-rounded
weights, plus a short training run on rays rendered from the depth-6
luminaire by the plain renderer (Sec. 4.2-4.4)."""
import numpy as np
import pytest

import paper_2207_05009_gb300 as plo
import plogen
from oracle import mlp as omlp

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_cuda(cuda_available):
    import torch
    return torch


def bf16(x):
    import torch
    return torch.from_numpy(np.ascontiguousarray(x, np.float32)).to(torch.bfloat16).to(torch.float64).numpy()


def unflatten(flat):
    Ws, bs, i = [], [], 0
    for (o, n) in omlp.layer_shapes(3):
        Ws.append(flat[i:i + o * n].reshape(o, n).astype(np.float64))
        i += o * n
        bs.append(flat[i:i + o].astype(np.float64))
        i += o
    assert i == flat.size
    return Ws, bs


def flatten(Ws, bs):
    return np.concatenate([np.concatenate([w.ravel(), b]) for w, b in zip(Ws, bs)])


def random_params(seed, scale=1.0):
    rng = np.random.default_rng(seed)
    Ws, bs = omlp.init_params(rng)
    Ws = [w * scale for w in Ws]
    bs = [rng.normal(0, 0.05, b.shape) for b in bs]
    bs[-1][0] = 1.0
    return flatten(Ws, bs).astype(np.float32)


def cosine(a, b):
    return float(np.dot(a, b) / (np.linalg.norm(a) * np.linalg.norm(b) + 1e-300))


def test_forward_matches_oracle(torch_cuda):
    torch = torch_cuda
    flat = random_params(1)
    net = plo.Mlp(l_max=8.0)
    net.set_params(flat)
    np.testing.assert_array_equal(net.get_params(), flat)
    pts = np.random.default_rng(2).random((10_000, 3)).astype(np.float32)
    raw = net.forward(torch.from_numpy(pts).cuda())
    torch.cuda.synchronize()
    net.check()
    raw = raw.cpu().numpy().astype(np.float64)
    Ws, bs = unflatten(flat)
    ref, _ = omlp.forward([bf16(w) for w in Ws], bs, omlp.positional_encoding(pts.astype(np.float64)))
    assert cosine(raw.ravel(), ref.ravel()) > 0.999
    assert np.linalg.norm(raw - ref) / np.linalg.norm(ref) < 3e-2


@pytest.mark.parametrize("loss,trans", [(plo.LOSS_PAPER, plo.TRANS_EXP), (plo.LOSS_MSE, plo.TRANS_EXP),
                                        (plo.LOSS_PAPER, plo.TRANS_LINEAR)])
def test_gradients_match_oracle(torch_cuda, loss, trans):
    torch = torch_cuda
    R, N = 64, 32
    flat = random_params(3, scale=0.5)
    net = plo.Mlp(l_max=6.0, loss=loss, transmittance=trans)
    net.set_params(flat)
    rays = plogen.rays_sphere(R, seed=4)
    rng = np.random.default_rng(5)
    jit = rng.random((R, N)).astype(np.float32)
    C_gt = rng.uniform(0, 5, (R, 3)).astype(np.float32)
    a_gt = rng.uniform(0, 1, R).astype(np.float32)
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    loss_gpu = net.train_step(dev(rays), dev(C_gt), dev(a_gt), n_samples=N, jitter=dev(jit))
    torch.cuda.synchronize()
    net.check()
    g = net.get_grads().astype(np.float64)
    Ws, bs = unflatten(flat)
    kind = {plo.LOSS_PAPER: "paper", plo.LOSS_MSE: "mse"}[loss]
    tname = "exp" if trans == plo.TRANS_EXP else "linear"
    L, dWs, dbs, _ = omlp.train_loss_and_grads([bf16(w) for w in Ws], bs, rays, jit.astype(np.float64),
                                               C_gt.astype(np.float64), a_gt.astype(np.float64), 6.0, kind=kind,
                                               transmittance=tname)
    ref = flatten(dWs, dbs)
    assert float(loss_gpu.item()) == pytest.approx(L, rel=2e-2)
    assert cosine(g, ref) > 0.999
    assert np.linalg.norm(g - ref) / np.linalg.norm(ref) < 1e-2 * 3
    # every layer's gradient points the same way
    i = 0
    for w, b in zip(dWs, dbs):
        n = w.size + b.size
        assert cosine(g[i:i + n], ref[i:i + n]) > 0.99
        i += n
    # the step moved the parameters by Adam's first update, ~lr * sign(g)
    p1 = net.get_params()
    moved = np.abs(p1 - flat)
    assert moved.max() <= 5e-4 * 1.01 and moved.max() > 1e-4


def test_training_on_rendered_targets_reduces_loss(torch_cuda):
    torch = torch_cuda
    tree = plogen.luminaire_tree(plogen.LUMINAIRE_D6)
    t = plo.Tree(tree)
    R = 4096
    batches = []
    for k in range(4):
        rays = torch.from_numpy(plogen.rays_sphere(R, seed=100 + k)).cuda()
        rgb, T, _ = plo.render(t, rays)
        batches.append((rays, rgb, 1.0 - T))
    torch.cuda.synchronize()
    l_max = float(max(b[1].max().item() for b in batches))
    net = plo.Mlp(l_max=l_max, total_steps=200)
    losses = []
    for step in range(60):
        rays, rgb, alpha = batches[step % 4]
        losses.append(float(net.train_step(rays, rgb, alpha, n_samples=64).item()))
    net.check()
    assert np.all(np.isfinite(losses))
    assert np.mean(losses[-8:]) < 0.7 * np.mean(losses[:4]), losses
