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


U32 = 2.0 ** -24  # unit roundoff of FP32


def to_np(t):
    return t.float().cpu().numpy().astype(np.float64)


def test_fused_trunk_equals_layer_by_layer_gemm(torch_cuda):
    """The layer-fused trunk (one kernel for layers 1-8, the tile kept in
    shared memory) against the single-layer tensor-core GEMM applied to each
    of its own stored inputs: bit for bit, on a ragged sample count whose
    tiles give the CTAs both full pairs and a lone tile."""
    torch = torch_cuda
    flat = random_params(3)
    net = plo.Mlp(l_max=8.0)
    net.set_params(flat)
    n = 152 * 128 * 3 + 77
    pts = np.random.default_rng(4).random((n, 3)).astype(np.float32)
    net.forward(torch.from_numpy(pts).cuda())
    H = [net.activation(l, n) for l in range(omlp.DEPTH + 1)]
    Ws, bs = unflatten(flat)
    for l in range(omlp.DEPTH):
        W = np.zeros((256, H[l].shape[1]), np.float32)
        W[:, :Ws[l].shape[1]] = Ws[l]
        Wd = torch.from_numpy(W).cuda().to(torch.bfloat16)
        bias = torch.from_numpy(bs[l].astype(np.float32)).cuda()
        out, err = plo.gemm_bf16(H[l].contiguous(), Wd, 0, bias=bias)
        torch.cuda.synchronize()
        assert int(err.item()) == 0
        assert torch.equal(out, H[l + 1]), (l, int((out != H[l + 1]).sum()))
    net.check()


def test_fused_backward_chain_equals_layer_by_layer_gemm(torch_cuda):
    """The layer-fused data-gradient chain of a training step (dZ_{l-1} =
    (dZ_l W_l) masked where H_l > 0, l = 7 .. 1, in one kernel) against the
    single-layer tensor-core GEMM with the mask epilogue applied to each of
    its own stored inputs: bit for bit, on 1,142 rays x 64 samples (571
    tiles: full pairs and lone tiles per CTA)."""
    torch = torch_cuda
    flat = random_params(5, scale=0.5)
    net = plo.Mlp(l_max=6.0)
    net.set_params(flat)
    R, N = 1142, 64
    rays = plogen.rays_sphere(R, seed=6)
    rng = np.random.default_rng(7)
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    net.train_step(dev(rays), dev(rng.uniform(0, 5, (R, 3)).astype(np.float32)),
                   dev(rng.uniform(0, 1, R).astype(np.float32)), n_samples=N)
    M = R * N
    H = [net.activation(l, M) for l in range(omlp.DEPTH + 1)]
    dZ = [net.activation(plo.MLP_DZ_BASE + l, M) for l in range(omlp.DEPTH)]
    Ws, _ = unflatten(flat)  # the weights the step's backward used (before its update)
    for l in range(omlp.DEPTH - 1, 0, -1):
        WT = torch.from_numpy(np.ascontiguousarray(Ws[l].T.astype(np.float32))).cuda().to(torch.bfloat16)
        out, err = plo.gemm_bf16(dZ[l], WT, 2, mask=H[l])
        torch.cuda.synchronize()
        assert int(err.item()) == 0
        assert torch.equal(out, dZ[l - 1]), (l, int((out != dZ[l - 1]).sum()))
    assert bool(dZ[0].abs().sum() > 0)
    net.check()


def test_forward_layers_match_oracle_elementwise(torch_cuda):
    """Every tensor-core layer of the forward pass, element by element: the
    GPU's own bf16 input of layer l, times the bf16 weights, plus the FP32
    bias, then ReLU, in FP64, against the GPU's bf16 output of that layer.
    Bound: one bf16 rounding (2^-8 relative) plus FP32 accumulation over K
    terms (K 2^-24 sum |w h|).  The encoded input is the bf16 rounding of the
    FP32 sin / cos of the encoding (2^-8 relative plus 2^-23)."""
    torch = torch_cuda
    flat = random_params(1)
    net = plo.Mlp(l_max=8.0)
    net.set_params(flat)
    np.testing.assert_array_equal(net.get_params(), flat)
    n = 4096
    pts = np.random.default_rng(2).random((n, 3)).astype(np.float32)
    raw = net.forward(torch.from_numpy(pts).cuda())
    H = [to_np(net.activation(l, n)) for l in range(omlp.DEPTH + 1)]
    torch.cuda.synchronize()
    net.check()
    raw = to_np(raw)
    Ws, bs = unflatten(flat)
    Wb = [bf16(w) for w in Ws]
    pe = omlp.positional_encoding(pts.astype(np.float64))
    assert np.all(H[0][:, 63] == 0)
    assert np.all(np.abs(H[0][:, :63] - pe) <= 2.0 ** -8 * np.abs(pe) + 2 * U32)
    for l in range(omlp.DEPTH):
        h_in = H[l][:, :Wb[l].shape[1]]
        ref = np.maximum(h_in @ Wb[l].T + bs[l], 0.0)
        acc = Wb[l].shape[1] * U32 * (np.abs(h_in) @ np.abs(Wb[l]).T + np.abs(bs[l]))
        err = np.abs(H[l + 1] - ref)
        assert np.all(err <= 2.0 ** -8 * np.abs(ref) + acc * (1 + 2.0 ** -8)), (l, float((err - acc).max()))
    ref = H[omlp.DEPTH] @ Wb[-1].T + bs[-1]
    acc = 256 * U32 * (np.abs(H[omlp.DEPTH]) @ np.abs(Wb[-1]).T + np.abs(bs[-1]))
    assert np.all(np.abs(raw - ref) <= acc + 1e-30)
    # and end to end against the FP64 oracle that rounds what the network
    # stores to bf16 (same precision decisions, independent of the GPU's
    # intermediate values)
    ref_b, _ = omlp.forward(Wb, bs, pe, storage="bf16")
    assert cosine(raw.ravel(), ref_b.ravel()) > 0.9999
    assert np.linalg.norm(raw - ref_b) / np.linalg.norm(ref_b) < 1e-2


def quad_inputs(R, N, seed):
    rng = np.random.default_rng(seed)
    rays = plogen.rays_sphere(R, seed=seed)
    raw = rng.normal(0.0, 1.0, (R * N, 49))
    # sigma_raw, ReLU clipping the negative ones; a per-ray scale spreads the
    # optical depth over ~0.02 .. 20, so rays range from clear to opaque
    raw[:, 0] = rng.uniform(-2.0, 30.0, R * N) * np.repeat(10.0 ** rng.uniform(-3, 0, R), N)
    delta = rng.uniform(0.2, 1.8, (R * N)) * (1.7 / N)
    C_gt = rng.uniform(0.0, 5.0, (R, 3))
    a_gt = rng.uniform(0.0, 1.0, R)
    return rays, raw.astype(np.float32), delta.astype(np.float32), C_gt.astype(np.float32), a_gt.astype(np.float32)


@pytest.mark.parametrize("loss,trans,N", [(plo.LOSS_PAPER, plo.TRANS_EXP, 64), (plo.LOSS_MSE, plo.TRANS_EXP, 128),
                                          (plo.LOSS_PAPER, plo.TRANS_LINEAR, 32),
                                          (plo.LOSS_REG, plo.TRANS_EXP, 256)])
def test_quadrature_matches_oracle_per_ray(torch_cuda, loss, trans, N):
    """The quadrature render and loss stage (k_quad) per ray and channel: C^
    and alpha^ within 1e-4 relative, the loss within 1e-4 relative, and
    d loss / d raw per element within one bf16 rounding (2^-8) plus 1e-4 of
    the largest gradient of that ray and column, against the oracle's
    composite / loss_terms / composite_backward on the same raw outputs and
    segment lengths."""
    torch = torch_cuda
    R, l_max = 96, 6.0
    rays, raw, delta, C_gt, a_gt = quad_inputs(R, N, seed=11 + N)
    net = plo.Mlp(l_max=l_max, loss=loss, transmittance=trans)
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    ray_out, draw = net.quad(dev(rays), dev(raw), dev(delta), dev(C_gt), dev(a_gt), N)
    torch.cuda.synchronize()
    ray_out, draw = to_np(ray_out), to_np(draw)
    kind = {plo.LOSS_PAPER: "paper", plo.LOSS_MSE: "mse", plo.LOSS_REG: "reg"}[loss]
    tname = "exp" if trans == plo.TRANS_EXP else "linear"
    Y = omlp.sh_matrix(rays[:, 3:].astype(np.float64), 3)
    C, alpha, cache = omlp.composite(raw.astype(np.float64).reshape(R, N, 49), delta.astype(np.float64).reshape(R, N),
                                     Y, l_max, tname)
    per_ray, dC, dA = omlp.loss_terms(C, alpha, C_gt.astype(np.float64), a_gt.astype(np.float64), l_max, kind)
    ref = omlp.composite_backward(cache, dC / R, dA / R).reshape(R * N, 49)
    np.testing.assert_allclose(ray_out[:, :3], C, rtol=1e-4, atol=0)
    np.testing.assert_allclose(ray_out[:, 3], alpha, rtol=1e-4, atol=1e-7)
    np.testing.assert_allclose(ray_out[:, 4], per_ray, rtol=1e-4, atol=1e-7)
    assert 0.05 < float(alpha.mean()) < 0.95  # both opaque and clear rays in the batch
    ref3 = ref.reshape(R, N, 49)
    tol = 2.0 ** -8 * np.abs(ref3) + 1e-5 * np.abs(ref3).max(axis=1, keepdims=True)
    # d loss / d sigma_j is a difference of FP32 prefix / suffix sums (exp:
    # T_{j+1} g_j - sum_{k>j} w_k g_k; linear: sums of g_k over the samples
    # where T is positive): its FP32 error scales with the sums' magnitude
    g_w = np.einsum("rnc,rc->rn", cache["c"], dC / R) + (dA / R)[:, None]
    wg = np.abs(cache["w"] * g_w)
    suffix = np.flip(np.cumsum(np.flip(wg, 1), 1), 1) - wg
    if tname == "exp":
        cancel = cache["T"][:, 1:] * np.abs(g_w) + suffix
    else:
        cancel = np.flip(np.cumsum(np.flip(np.abs(g_w), 1), 1), 1)
    tol[..., 0] += 1e-5 * cancel * delta.astype(np.float64).reshape(R, N)
    err = np.abs(draw.reshape(R, N, 49) - ref3)
    bad = np.argwhere(err > tol)
    assert bad.size == 0, (len(bad), [tuple(int(x) for x in b) for b in bad[:5]],
                           float((err / np.maximum(tol, 1e-300)).max()))


@pytest.mark.parametrize("loss,trans", [(plo.LOSS_PAPER, plo.TRANS_EXP), (plo.LOSS_MSE, plo.TRANS_EXP),
                                        (plo.LOSS_PAPER, plo.TRANS_LINEAR)])
def test_gradients_match_oracle(torch_cuda, loss, trans):
    """A training step's gradients against the FP64 oracle that stores
    activations and gradients in bf16 where the network does, on the GPU's
    own encoded samples: per layer (weights and biases) within 1e-2 of the
    layer's gradient norm, and the loss within 1e-3 relative."""
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
    X = to_np(net.activation(0, R * N))[:, :63]
    torch.cuda.synchronize()
    net.check()
    g = net.get_grads().astype(np.float64)
    Ws, bs = unflatten(flat)
    kind = {plo.LOSS_PAPER: "paper", plo.LOSS_MSE: "mse"}[loss]
    tname = "exp" if trans == plo.TRANS_EXP else "linear"
    L, dWs, dbs, _ = omlp.train_loss_and_grads([bf16(w) for w in Ws], bs, rays, jit.astype(np.float64),
                                               C_gt.astype(np.float64), a_gt.astype(np.float64), 6.0, kind=kind,
                                               transmittance=tname, storage="bf16", X=X)
    ref = flatten(dWs, dbs)
    # the oracle's activations are its own (bf16 roundings may fall on the
    # other side of a boundary), so the loss agrees to ~1e-4, not to FP32
    assert float(loss_gpu.item()) == pytest.approx(L, rel=1e-3)
    assert np.linalg.norm(g - ref) / np.linalg.norm(ref) < 1e-2
    i = 0
    for w, b in zip(dWs, dbs):
        n = w.size + b.size
        assert np.linalg.norm(g[i:i + n] - ref[i:i + n]) <= 1e-2 * np.linalg.norm(ref[i:i + n]), i
        i += n


def test_adam_matches_oracle_over_steps(torch_cuda):
    """Six training steps with the learning rate decaying over four (so the
    last steps run at lr1): after each step the FP32 masters equal the
    oracle's Adam (adam_update with lr_at) replayed on the gradients the GPU
    used, element by element.  Bound after k steps: k 1e-6 |p| for the FP32
    parameter roundings (2^-24 relative each, with margin) plus 1e-5 of the
    learning rates summed so far, for the FP32 constants of the GPU's
    update (0.9f, 0.999f and the FP32 bias corrections move an update by
    about 7e-6 of lr)."""
    torch = torch_cuda
    R, N, total, lr0, lr1 = 64, 32, 4, 5e-4, 5e-6
    flat = random_params(13, scale=0.5)
    net = plo.Mlp(l_max=6.0, total_steps=total, lr0=lr0, lr1=lr1)
    net.set_params(flat)
    rng = np.random.default_rng(14)
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    p = flat.astype(np.float64)
    m = np.zeros_like(p)
    v = np.zeros_like(p)
    lr_sum = 0.0
    for step in range(1, 7):
        rays = plogen.rays_sphere(R, seed=40 + step)
        jit = rng.random((R, N)).astype(np.float32)
        C_gt = rng.uniform(0, 5, (R, 3)).astype(np.float32)
        a_gt = rng.uniform(0, 1, R).astype(np.float32)
        net.train_step(dev(rays), dev(C_gt), dev(a_gt), n_samples=N, jitter=dev(jit))
        torch.cuda.synchronize()
        g = net.get_grads().astype(np.float64)
        lr = omlp.lr_at(step - 1, total, lr0, lr1)
        lr_sum += lr
        p0 = p
        p, m, v = omlp.adam_update(p, g, m, v, step, lr)
        got = net.get_params().astype(np.float64)
        err = np.abs(got - p)
        tol = 1e-6 * step * np.abs(p) + 1e-5 * lr_sum
        i = int(np.argmax(err / tol))
        assert err[i] <= tol[i], dict(step=step, index=i, p_before=p0[i], g=g[i], gpu=got[i], oracle=p[i],
                                      err=err[i], tol=tol[i])
        assert np.abs(got - p0).max() > 0.5 * lr  # the step moved the parameters
    assert net.step == 6
    assert omlp.lr_at(5, total, lr0, lr1) == pytest.approx(lr1)


def gt_batches(torch, n_batches, R=4096, seed0=100):
    """Training targets rendered from the depth-6 luminaire by the plain
    renderer (exponential transmittance, max(0, .) emission)."""
    t = plo.Tree(plogen.luminaire_tree(plogen.LUMINAIRE_D6))
    out = []
    for k in range(n_batches):
        rays = torch.from_numpy(plogen.rays_sphere(R, seed=seed0 + k)).cuda()
        rgb, T, _ = plo.render(t, rays)
        out.append((rays, rgb, 1.0 - T))
    torch.cuda.synchronize()
    return out


def emission_scale(batches):
    """L_max and the mean emission of the opaque part of the rays."""
    rgb = np.concatenate([b[1].cpu().numpy() for b in batches])
    alpha = np.concatenate([b[2].cpu().numpy() for b in batches])
    return float(rgb.max()), float(rgb.mean() / max(alpha.mean(), 1e-3))


def test_training_on_rendered_targets_reduces_loss(torch_cuda):
    batches = gt_batches(torch_cuda, 8)
    l_max, c0 = emission_scale(batches)
    net = plo.Mlp(l_max=l_max, total_steps=1000, init_radiance=c0)
    losses = []
    for step in range(240):
        rays, rgb, alpha = batches[step % 8]
        losses.append(float(net.train_step(rays, rgb, alpha, n_samples=128).item()))
    net.check()
    assert np.all(np.isfinite(losses))
    assert np.mean(losses[-16:]) < 0.6 * np.mean(losses[:8]), losses[::16]


def tree_from_morton(depth, codes, sigma, sh):
    """Canonical tree whose leaves at level `depth` are the given voxels."""
    from plogen import HostTree
    child = [[-1] * 8]
    for i, c in enumerate(codes):
        node = 0
        for l in range(depth - 1):
            slot = (int(c) >> (3 * (depth - 1 - l))) & 7
            if child[node][slot] == -1:
                child[node][slot] = len(child)
                child.append([-1] * 8)
            node = child[node][slot]
        child[node][int(c) & 7] = -i - 2
    return HostTree(depth, 3, np.array(child, np.int32), np.asarray(sigma, np.float32),
                    np.asarray(sh, np.float32).reshape(len(codes), 3, 16))


@pytest.mark.parametrize("S", [4, 256])
def test_distill_matches_oracle(torch_cuda, S):
    """S = 256 is the paper's sample count per kept voxel (Sec. 5)."""
    torch = torch_cuda
    import oracle
    from tests.parity import quantise_tree, relative_errors
    depth, seed = 4, 99
    flat = random_params(7, scale=0.6)
    net = plo.Mlp(l_max=5.0, jitter_seed=seed)
    net.set_params(flat)
    Ws, bs = unflatten(flat)
    Wb = [bf16(w) for w in Ws]
    _, sig_c, _, _ = omlp.distill_dense(Wb, bs, depth, None, sigma_thresh=0.0)
    thresh = float(np.median(sig_c[sig_c > 0]))
    tree = net.distill(depth, samples=S, sigma_thresh=thresh)
    G = 1 << depth
    idx = np.arange(G ** 3)
    ijk_all = np.stack([idx % G, (idx // G) % G, idx // (G * G)], 1)
    centres = torch.from_numpy(((ijk_all + 0.5) / G).astype(np.float32)).cuda()
    leaf, _ = plo.lookup(tree, centres)
    torch.cuda.synchronize()
    kept_gpu = leaf.cpu().numpy() >= 0
    # the keep decision is the same wherever the centre sigma is not within
    # the bf16 network's error (3%) of the threshold
    clear = np.abs(sig_c / thresh - 1.0) > 0.03
    np.testing.assert_array_equal(kept_gpu[clear], (sig_c >= thresh)[clear])
    assert 0.3 < kept_gpu.mean() < 0.7
    # leaf values over the GPU's kept set, from the oracle's network and jitter
    codes = omlp.morton_code(ijk_all[kept_gpu], depth)
    order = np.argsort(np.array(codes, dtype=np.int64))
    codes = [codes[i] for i in order]
    ijk = ijk_all[kept_gpu][order]
    jit = omlp.distill_jitter(seed, codes, S)
    raw_s, _ = omlp.forward(Wb, bs, omlp.positional_encoding(((ijk[:, None, :] + jit) / G).reshape(-1, 3)))
    raw_s = raw_s.reshape(len(codes), S, -1)
    sig = np.maximum(raw_s[..., 0], 0).mean(1)
    sh = raw_s[..., 1:].mean(1)
    ref_tree = tree_from_morton(depth, codes, sig, sh)
    rays = plogen.rays_sphere(4096, seed=8)
    rgb, T, _ = plo.render(tree, torch.from_numpy(rays).cuda(),
                           plo.RenderParams(activation=plo.ACT_SIGMOID, l_max=5.0))
    ref = oracle.render(ref_tree, rays, activation=oracle.SIGMOID, l_max=5.0)
    torch.cuda.synchronize()
    e_c, e_T = relative_errors(rgb.cpu().numpy(), T.cpu().numpy(), ref)
    assert e_c < 3e-2 and e_T < 3e-2, (e_c, e_T)
    # the device packer against the host one: the distilled tree exported to
    # the canonical format and packed again by plo_build_tree has the same
    # kept set (leaf ids in Morton order) and renders bit for bit the same
    host = tree.export()
    assert host.n_leaves == len(codes)
    plo.validate(host)
    again = plo.Tree(host)
    rgb2, T2, _ = plo.render(again, torch.from_numpy(rays).cuda(), plo.RenderParams(activation=plo.ACT_SIGMOID,
                                                                                     l_max=5.0))
    torch.cuda.synchronize()
    assert torch.equal(rgb2, rgb) and torch.equal(T2, T)
    # and the exported leaves equal the oracle's averages on the bf16 network
    # to the network's bf16 precision
    np.testing.assert_allclose(host.sigma, sig, rtol=3e-2, atol=1e-3 * float(np.abs(sig).max()))
    np.testing.assert_allclose(host.sh.reshape(len(codes), -1), sh.reshape(len(codes), -1), rtol=0,
                               atol=3e-2 * float(np.abs(sh).max()))
    # 16-bit distillation: the device's leaf encoding equals the host
    # packer's, as emulated by quantise_tree, bit for bit
    for name, prec in (("fp16", plo.PREC_FP16), ("bf16", plo.PREC_BF16)):
        t16 = net.distill(depth, samples=S, sigma_thresh=thresh, precision=prec)
        h16 = t16.export()
        q = quantise_tree(host, name)
        np.testing.assert_array_equal(h16.child, host.child)
        np.testing.assert_array_equal(h16.sigma, q.sigma)
        np.testing.assert_array_equal(h16.sh, q.sh)


def test_distill_depth_10_on_the_device(torch_cuda):
    """Depth 10 (1024^3 voxel centres, Sec. 5) end to end on the device.  The
    kept set is checked bit for bit on 200,000 random voxels: the centre
    pass and plo_mlp_forward encode the same FP32 centre the same way, so the
    network's sigma there is the same, and a voxel is a leaf of the packed
    tree (plo_lookup_points) exactly where it reaches the threshold."""
    torch = torch_cuda
    flat = random_params(7, scale=0.6)
    net = plo.Mlp(l_max=5.0, jitter_seed=99)
    net.set_params(flat)
    G = 1024
    rng = np.random.default_rng(21)
    probe = torch.from_numpy(((rng.integers(0, G, (65536, 3)) + 0.5) / G).astype(np.float32)).cuda()
    sig = torch.relu(net.forward(probe)[:, 0])
    thresh = float(torch.quantile(sig, 0.95))  # ~5% of the voxels: ~50M leaves
    tree = net.distill(10, samples=1, sigma_thresh=thresh)
    inf = tree.info()
    assert inf["depth"] == 10 and 0.01 * G ** 3 < inf["n_leaves"] < 0.2 * G ** 3
    ijk = rng.integers(0, G, (200_000, 3))
    centres = torch.from_numpy(((ijk + 0.5) / G).astype(np.float32)).cuda()
    kept = torch.relu(net.forward(centres)[:, 0]) >= thresh
    leaf, level = plo.lookup(tree, centres)
    torch.cuda.synchronize()
    assert torch.equal(leaf >= 0, kept)
    assert bool((level[kept] == 10).all())
    rays = torch.from_numpy(plogen.rays_sphere(65536, seed=9)).cuda()
    rgb, T, _ = plo.render(tree, rays, plo.RenderParams(activation=plo.ACT_SIGMOID, l_max=5.0))
    torch.cuda.synchronize()
    tree.check()
    assert bool(torch.isfinite(rgb).all()) and bool((T < 1).any())


def test_learned_gain_over_mse_and_untrained(torch_cuda):
    """The paper's loss ablation, repurposed on synthetic data: the distilled
    octree of a network trained with the paper's loss (HDR colour term + alpha
    term) reconstructs transparency better than one trained with plain MSE,
    and far better than the untrained network distilled the same way."""
    from paper_2207_05009_gb300 import learned
    gt = plo.Tree(plogen.luminaire_tree(plogen.LUMINAIRE_D6))
    train_b = learned.target_batches(gt, [plogen.rays_sphere(4096, seed=200 + k) for k in range(16)])
    test_b = learned.target_batches(gt, [plogen.rays_sphere(8192, seed=900)])
    l_max, _ = learned.emission_scale(train_b)
    errs = {}
    for name, loss, steps in (("paper", plo.LOSS_PAPER, 600), ("mse", plo.LOSS_MSE, 600),
                              ("untrained", plo.LOSS_PAPER, 0)):
        net, losses, _ = learned.train(train_b, steps, loss, l_max=l_max)
        errs[name] = learned.distilled_error(net, l_max, test_b, depth=6)
    assert errs["paper"].alpha_rmse < errs["mse"].alpha_rmse
    assert errs["paper"].alpha_rmse < 0.6 * errs["untrained"].alpha_rmse
    assert errs["paper"].rel_l2_radiance < errs["untrained"].rel_l2_radiance
