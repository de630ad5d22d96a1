"""Pins for the learned-part oracle: positional-encoding values, quadrature
closed forms, loss special cases, central finite differences of the full
training loss, Adam's first step, the learning-rate schedule, and the
distillation of a constant field."""
import math

import numpy as np
import pytest

import oracle
import plogen
from oracle import mlp
from tests.trees import chord


def test_positional_encoding_values():
    x = np.array([[0.0, 0.5, 0.25]])
    g = mlp.positional_encoding(x)
    assert g.shape == (1, 63)
    np.testing.assert_array_equal(g[0, :3], x[0])
    for j in range(10):
        s, c = g[0, 3 + 6 * j: 6 + 6 * j], g[0, 6 + 6 * j: 9 + 6 * j]
        assert s[0] == 0.0 and c[0] == 1.0                         # x = 0
        assert s[1] == pytest.approx(math.sin(2 ** j * math.pi / 2), abs=1e-12)
        assert c[1] == pytest.approx(math.cos(2 ** j * math.pi / 2), abs=1e-12)
    assert g[0, 3 + 1] == pytest.approx(1.0)   # sin(pi/2)
    assert g[0, 9 + 4] == pytest.approx(-1.0)  # cos(2 pi * 0.5)


def test_samples_lie_in_the_chord_and_are_ordered():
    rays = plogen.rays_sphere(64, seed=3)
    rng = np.random.default_rng(0)
    jit = rng.random((64, 16))
    t, delta, x, hit = mlp.stratified_samples(rays, jit)
    for i, r in enumerate(rays):
        ch = chord(r[:3], r[3:])
        assert hit[i] == (ch is not None)
        if ch is None:
            continue
        assert np.all(np.diff(t[i]) > 0)
        assert t[i, 0] >= ch[0] - 1e-12 and t[i, -1] <= ch[1] + 1e-12
        assert t[i, -1] + delta[i, -1] == pytest.approx(ch[1], abs=1e-12)
        assert np.all((x[i] >= -1e-9) & (x[i] <= 1 + 1e-9))


def test_composite_closed_forms():
    R, N = 5, 32
    rng = np.random.default_rng(1)
    delta = rng.uniform(0.001, 0.05, (R, N))
    K = 16
    raw = np.zeros((R, N, 1 + 3 * K))
    raw[..., 0] = 3.0                       # constant sigma
    raw[..., 1:] = rng.normal(size=3 * K)   # same coefficients everywhere
    Y = mlp.sh_matrix(np.tile([0.0, 0.0, 1.0], (R, 1)), 3)
    C, alpha, _ = mlp.composite(raw, delta, Y, 7.0, "exp")
    L = delta.sum(1)
    np.testing.assert_allclose(alpha, 1 - np.exp(-3.0 * L), rtol=1e-13)
    s = raw[0, 0, 1:].reshape(3, K) @ Y[0]
    phi = 7.0 / (1 + np.exp(-s))
    np.testing.assert_allclose(C, alpha[:, None] * phi[None], rtol=1e-12)
    C, alpha, _ = mlp.composite(raw, delta, Y, 7.0, "linear")
    np.testing.assert_allclose(alpha, np.minimum(1.0, 3.0 * L), rtol=1e-13)


def test_loss_special_cases():
    C = np.array([[1.0, 2.0, 3.0]])
    a = np.array([0.4])
    per, dC, dA = mlp.loss_terms(C, a, C, a, 10.0)
    assert per[0] == 0 and np.all(dC == 0) and dA[0] == 0
    per, dC, dA = mlp.loss_terms(C, a, np.zeros_like(C), np.zeros(1), 10.0, kind="paper")
    cn = C[0] / 10
    assert per[0] == pytest.approx(((cn / (cn + 0.01)) ** 2).sum() + 0.16)
    per, dC, _ = mlp.loss_terms(C, a, np.zeros_like(C), a, 10.0, kind="mse")
    assert per[0] == pytest.approx((cn ** 2).sum())
    np.testing.assert_allclose(dC[0], 2 * cn / 10)


def _batch(seed=0, R=6, N=12, l_max=3):
    rng = np.random.default_rng(seed)
    Ws, bs = mlp.init_params(rng, l_max)
    # small-scale weights so that the sigmoid and ReLUs are away from kinks
    Ws = [w * 0.5 for w in Ws]
    bs = [rng.normal(0, 0.05, b.shape) for b in bs]
    bs[-1][0] = 1.0
    rays = plogen.rays_sphere(R, seed=seed + 40)
    jit = rng.random((R, N))
    C_gt = rng.uniform(0, 5, (R, 3))
    a_gt = rng.uniform(0, 1, R)
    return Ws, bs, rays, jit, C_gt, a_gt


@pytest.mark.parametrize("kind,trans,seed", [("paper", "exp", 1), ("paper", "exp", 5), ("mse", "exp", 2),
                                              ("paper", "linear", 11), ("paper", "linear", 10)])
def test_gradients_match_central_differences(kind, trans, seed):
    Ws, bs, rays, jit, C_gt, a_gt = _batch(seed=seed)
    Lm = 6.0
    loss0, dWs, dbs, ex = mlp.train_loss_and_grads(Ws, bs, rays, jit, C_gt, a_gt, Lm, kind=kind,
                                                   transmittance=trans)
    # the loss holds its denominator constant: freeze it at the base point
    den = ex["C"] / Lm + 0.01

    def loss_at(Wmod=None, bmod=None):
        return mlp.train_loss_and_grads(Wmod or Ws, bmod or bs, rays, jit, C_gt, a_gt, Lm, kind=kind,
                                        transmittance=trans, denom=den)[0]

    def fd(setter, h):
        return (loss_at(*setter(+h)) - loss_at(*setter(-h))) / (2 * h)

    rng = np.random.default_rng(5)
    checks = 0
    for l in [0, 3, 7, 8]:
        scale = float(np.sqrt((dWs[l] ** 2).mean()))
        tries = 0
        done = 0
        while done < 4 and tries < 40:
            tries += 1
            i = rng.integers(0, Ws[l].shape[0])
            j = rng.integers(0, Ws[l].shape[1])

            def setter(h, i=i, j=j, l=l):
                W2 = [w.copy() for w in Ws]
                W2[l][i, j] += h
                return W2, None
            f1, f2 = fd(setter, 1e-5), fd(setter, 5e-6)
            if abs(f1 - f2) > 1e-4 * abs(f1) + 1e-6 * scale:
                continue  # a ReLU or clamp kink within the step: resample
            assert dWs[l][i, j] == pytest.approx(f1, rel=1e-4, abs=1e-5 * scale), (l, i, j)
            done += 1
            checks += 1
        k = int(np.argmax(np.abs(dbs[l])))

        def bset(h, k=k, l=l):
            b2 = [b.copy() for b in bs]
            b2[l][k] += h
            return None, b2
        assert dbs[l][k] == pytest.approx(fd(bset, 1e-5), rel=1e-4)
    assert checks == 16


def test_adam_first_step_and_schedule():
    g = np.array([0.3, -2.0, 1e-3])
    p, m, v = mlp.adam_update(np.zeros(3), g, np.zeros(3), np.zeros(3), 1, 1e-3)
    np.testing.assert_allclose(p, -1e-3 * g / (np.abs(g) + 1e-8), rtol=1e-12)
    assert mlp.lr_at(0, 1000) == pytest.approx(5e-4)
    assert mlp.lr_at(1000, 1000) == pytest.approx(5e-6)
    assert mlp.lr_at(500, 1000) == pytest.approx(5e-5)


def test_distill_constant_field():
    rng = np.random.default_rng(2)
    Ws, bs = mlp.init_params(rng)
    Ws = [w * 0 for w in Ws]
    bs = [b * 0 for b in bs]
    bs[-1][0] = 0.5
    bs[-1][1:] = np.arange(48) * 0.01
    jit = rng.random((8 ** 2 * 8, 8, 3))
    ijk, sig_c, sig, sh = mlp.distill_dense(Ws, bs, 3, jit)
    assert len(ijk) == 512 and np.all(sig_c == 0.5)
    np.testing.assert_allclose(sig, 0.5)
    np.testing.assert_allclose(sh.reshape(len(ijk), -1), np.tile(np.arange(48) * 0.01, (512, 1)))
    bs[-1][0] = 0.005  # below the 0.01 threshold: everything pruned
    ijk, *_ = mlp.distill_dense(Ws, bs, 3, None)
    assert len(ijk) == 0


def test_splitmix64_published_vectors_and_morton():
    # first two outputs of SplitMix64 seeded with 0 (reference implementation)
    assert mlp._mix64(0) == 0xE220A8397B1DCDAF
    assert mlp._mix64(0x9E3779B97F4A7C15) == 0x6E789E6AA1B965F4
    # Morton code: brute force over a 4^3 grid against the per-level slots
    ijk = np.array([[x, y, z] for z in range(4) for y in range(4) for x in range(4)])
    codes = mlp.morton_code(ijk, 2)
    for (x, y, z), c in zip(ijk, codes):
        s0 = (x >> 1) | ((y >> 1) << 1) | ((z >> 1) << 2)
        s1 = (x & 1) | ((y & 1) << 1) | ((z & 1) << 2)
        assert c == s0 * 8 + s1
    assert sorted(codes) == list(range(64))
    u = mlp.distill_jitter(3, [0, 17], 5)
    assert u.shape == (2, 5, 3) and np.all((u >= 0) & (u < 1))
    assert len(np.unique(u)) == u.size


# ---------------------------------------------------------------- the paper's full training setup
# (Sec. 4.2 extra 128-wide output layer; Sec. 4.3-4.4 coarse/fine networks)

def _paper_nets(seed, l_max=3):
    rng = np.random.default_rng(seed)
    nets = []
    for _ in range(2):
        Ws, bs = mlp.init_params_paper(rng, l_max)
        Ws = [w * 0.5 for w in Ws]
        bs = [rng.normal(0, 0.05, b.shape) for b in bs]
        bs[mlp.DEPTH][0] = 1.0  # sigma bias: a visible density
        nets.append((Ws, bs))
    return nets


def test_paper_head_shapes_and_forward_by_hand():
    (Ws, bs), _ = _paper_nets(0)
    assert [w.shape for w in Ws][-3:] == [(1, 256), (128, 256), (48, 128)]
    X = np.random.default_rng(1).normal(size=(5, 63))
    raw, H = mlp.forward_paper(Ws, bs, X)
    h = X
    for l in range(8):
        h = np.maximum(Ws[l] @ h.T + bs[l][:, None], 0).T
    feat = np.maximum(h @ Ws[9].T + bs[9], 0)
    np.testing.assert_allclose(raw[:, 0], h @ Ws[8][0] + bs[8][0], rtol=1e-12)
    np.testing.assert_allclose(raw[:, 1:], feat @ Ws[10].T + bs[10], rtol=1e-12, atol=1e-12)


def test_fine_samples_uniform_weights_closed_form():
    R, Nc, Nf = 3, 64, 128
    rays = plogen.rays_sphere(R, seed=5)
    t, delta, _, hit = mlp.stratified_samples(rays, np.zeros((R, Nc)))  # evenly spaced
    assert hit.all()
    xi = np.random.default_rng(2).random((R, Nf))
    tf = mlp.fine_samples(t, delta, np.full((R, Nc), 0.3), xi)
    t0, t1 = t[:, :1], (t[:, -1] + delta[:, -1])[:, None]
    u = (np.arange(Nf)[None] + xi) / Nf
    np.testing.assert_allclose(tf, t0 + u * (t1 - t0), rtol=1e-12, atol=1e-12)


def test_fine_samples_match_bisection_of_the_cdf():
    rng = np.random.default_rng(3)
    R, Nc, Nf = 4, 16, 40
    t = np.sort(rng.uniform(1, 3, (R, Nc)), 1)
    delta = np.concatenate([np.diff(t, axis=1), rng.uniform(0.01, 0.2, (R, 1))], 1)
    w = rng.random((R, Nc)) ** 3
    w[:, 5] = 0.0
    xi = rng.random((R, Nf))
    tf = mlp.fine_samples(t, delta, w, xi)
    for r in range(R):
        m = w[r] + 1e-5
        m = m / m.sum()

        def cdf(x):  # mass below x: piecewise-linear inside each segment
            inside = np.clip((x - t[r]) / delta[r], 0.0, 1.0)
            return float((m * inside).sum())
        for j in range(Nf):
            u = (j + xi[r, j]) / Nf
            lo, hi = t[r, 0], t[r, -1] + delta[r, -1]
            for _ in range(80):
                mid = 0.5 * (lo + hi)
                lo, hi = (mid, hi) if cdf(mid) < u else (lo, mid)
            assert tf[r, j] == pytest.approx(0.5 * (lo + hi), abs=1e-10)
    assert np.all(np.diff(tf, axis=1) >= 0)


def test_fine_samples_counts_follow_the_weights():
    # stratified draws (one per stratum of width 1/N_f) put N_f m_i +- 2 samples in segment i
    rng = np.random.default_rng(4)
    R, Nc, Nf = 6, 64, 128
    t = np.cumsum(rng.uniform(0.01, 0.03, (R, Nc)), 1)
    delta = np.concatenate([np.diff(t, axis=1), np.full((R, 1), 0.02)], 1)
    w = rng.random((R, Nc)) ** 4
    tf = mlp.fine_samples(t, delta, w, rng.random((R, Nf)))
    for r in range(R):
        m = (w[r] + 1e-5) / (w[r] + 1e-5).sum()
        seg = np.searchsorted(t[r], tf[r], side="right") - 1
        counts = np.bincount(seg, minlength=Nc)
        assert np.all(np.abs(counts - Nf * m) < 2.0)


def test_merge_is_sorted_and_tiles_the_chord():
    rng = np.random.default_rng(5)
    R = 4
    rays = plogen.rays_sphere(R, seed=6)
    t, delta, _, hit = mlp.stratified_samples(rays, rng.random((R, 64)))
    tf = mlp.fine_samples(t, delta, rng.random((R, 64)), rng.random((R, 128)))
    t1 = t[:, -1] + delta[:, -1]
    ta, da = mlp.merge_samples(t, tf, t1)
    assert ta.shape == (R, 192)
    assert np.all(np.diff(ta, axis=1) >= 0) and np.all(da >= 0)
    np.testing.assert_allclose(ta[:, 0] + da.sum(1), t1, rtol=1e-12)
    for r in range(R):
        np.testing.assert_array_equal(np.sort(np.concatenate([t[r], tf[r]])), ta[r])


def test_hier_loss_constant_field_closed_form():
    # zero weights: sigma and the SH sum are the biases everywhere, so both
    # passes see a uniform medium: alpha = 1 - exp(-sigma L), C = Phi alpha
    R, l_max = 5, 3
    K = (l_max + 1) ** 2
    Ws = [np.zeros(s) for s in mlp.layer_shapes_paper(l_max)]
    bs = [np.zeros(s[0]) for s in mlp.layer_shapes_paper(l_max)]
    rng = np.random.default_rng(6)
    bs[8][0] = 2.5
    bs[10][:] = rng.normal(0, 1, 3 * K)
    rays = plogen.rays_sphere(R, seed=7)
    Lm = 4.0
    C_gt, a_gt = rng.uniform(0, 3, (R, 3)), rng.random(R)
    jit = rng.random((R, 64))
    loss, _, _, ex = mlp.train_loss_and_grads_hier(Ws, bs, Ws, bs, rays, jit, rng.random((R, 128)), C_gt, a_gt, Lm)
    t, _, _, _ = mlp.stratified_samples(rays, jit)
    d = rays[:, 3:].astype(np.float64)
    ref = 0.0
    for r in range(R):
        # both passes integrate from the first coarse sample to the exit
        # (the fine samples are drawn inside the coarse segments)
        ch = chord(rays[r, :3], rays[r, 3:])
        L = 0.0 if ch is None else ch[1] - t[r, 0]
        alpha = 1 - math.exp(-2.5 * L)
        Y = oracle.sh_basis(l_max, d[r] / np.linalg.norm(d[r]))
        phi = Lm / (1 + np.exp(-(bs[10].reshape(3, K) @ Y)))
        C = phi * alpha
        np.testing.assert_allclose(ex["C_c"][r], C, rtol=1e-12)
        np.testing.assert_allclose(ex["C_f"][r], C, rtol=1e-12)
        assert ex["alpha_f"][r] == pytest.approx(alpha, rel=1e-12)
        cn, gn = C / Lm, C_gt[r] / Lm
        col = (((cn - gn) / (cn + 0.01)) ** 2).sum()
        ref += 2 * col + (alpha - a_gt[r]) ** 2
    assert loss == pytest.approx(ref / R, rel=1e-12)


@pytest.mark.parametrize("seed,trans", [(1, "exp"), (2, "exp"), (3, "linear")])
def test_hier_gradients_match_central_differences(seed, trans):
    (Wc, bc), (Wf, bf) = _paper_nets(seed)
    R = 4
    rng = np.random.default_rng(seed + 100)
    rays = plogen.rays_sphere(R, seed=seed + 60)
    jit, xi = rng.random((R, 8)), rng.random((R, 16))
    C_gt, a_gt = rng.uniform(0, 5, (R, 3)), rng.uniform(0, 1, R)
    Lm = 6.0
    loss0, (dWc, dbc), (dWf, dbf), ex = mlp.train_loss_and_grads_hier(Wc, bc, Wf, bf, rays, jit, xi, C_gt, a_gt, Lm,
                                                                     transmittance=trans)
    den = (ex["C_c"] / Lm + 0.01, ex["C_f"] / Lm + 0.01)
    tf = ex["t_fine"]

    def part(which, Wc2, bc2, Wf2, bf2):
        ex2 = mlp.train_loss_and_grads_hier(Wc2, bc2, Wf2, bf2, rays, jit, xi, C_gt, a_gt, Lm, transmittance=trans,
                                            denoms=den, t_fine=tf)[3]
        return ex2["loss_c"] if which == "c" else ex2["loss_f"]

    checks = 0
    for which, Ws, bs, dWs, dbs in (("c", Wc, bc, dWc, dbc), ("f", Wf, bf, dWf, dbf)):
        for l in [0, 7, 8, 9, 10]:
            scale = float(np.sqrt((dWs[l] ** 2).mean())) + 1e-300
            done = tries = 0
            while done < 2 and tries < 40:
                tries += 1
                i, j = rng.integers(0, Ws[l].shape[0]), rng.integers(0, Ws[l].shape[1])

                def f(h, i=i, j=j, l=l):
                    W2 = [w.copy() for w in Ws]
                    W2[l][i, j] += h
                    args = (W2, bs, Wf, bf) if which == "c" else (Wc, bc, W2, bs)
                    return part(which, *args)
                f1 = (f(1e-5) - f(-1e-5)) / 2e-5
                f2 = (f(5e-6) - f(-5e-6)) / 1e-5
                if abs(f1 - f2) > 1e-4 * abs(f1) + 1e-6 * scale:
                    continue
                assert dWs[l][i, j] == pytest.approx(f1, rel=1e-4, abs=1e-5 * scale), (which, l, i, j)
                done += 1
                checks += 1
    assert checks == 20


def test_adam_accumulates_moments_over_steps():
    """Closed forms of Adam's moments (Kingma & Ba, Algorithm 1) over several
    steps: with a constant gradient g the bias-corrected moments are g and
    g^2 at every step, so each step moves lr g / (|g| + eps); with a gradient
    of alternating sign (-1)^t g the first moment is the geometric sum
    (1 - b1) g (-1)^t (1 - (-b1)^t) / (1 + b1)."""
    b1, b2, eps = 0.9, 0.999, 1e-8
    g = np.array([0.3, -2.0, 1e-3, 5e-9])
    p, m, v = np.zeros(4), np.zeros(4), np.zeros(4)
    for t in range(1, 8):
        lr = mlp.lr_at(t - 1, 4)
        p_new, m, v = mlp.adam_update(p, g, m, v, t, lr)
        np.testing.assert_allclose(p - p_new, lr * g / (np.abs(g) + eps), rtol=1e-9)
        np.testing.assert_allclose(m, g * (1 - b1 ** t), rtol=1e-12)
        np.testing.assert_allclose(v, g * g * (1 - b2 ** t), rtol=1e-12)
        p = p_new
    m, v = np.zeros(4), np.zeros(4)
    p = np.zeros(4)
    for t in range(1, 9):
        gt = (-1.0) ** t * g
        p_new, m, v = mlp.adam_update(p, gt, m, v, t, 1e-3)
        m_ref = (1 - b1) * g * (-1.0) ** t * (1 - (-b1) ** t) / (1 + b1)
        np.testing.assert_allclose(m, m_ref, rtol=1e-12)
        mh, vh = m_ref / (1 - b1 ** t), g * g
        np.testing.assert_allclose(p - p_new, 1e-3 * mh / (np.sqrt(vh) + eps), rtol=1e-9)
        p = p_new
    # the schedule reaches lr1 at total_steps and stays there
    assert mlp.lr_at(4, 4) == pytest.approx(5e-6) and mlp.lr_at(9, 4) == pytest.approx(5e-6)


def test_bf16_rounding_pins():
    """round_bf16: 8 significant bits, nearest with ties to even; values
    already in bf16 are unchanged; the error is at most half a unit in the
    last place (2^-8 relative)."""
    exact = np.array([1.0, 1.5, -3.0, 2.0 ** -100, 0.0, 1.0 + 2 ** -7, 65280.0])
    np.testing.assert_array_equal(mlp.round_bf16(exact), exact)
    u = 2.0 ** -7  # spacing of bf16 in [1, 2)
    cases = {1 + u / 2: 1.0, 1 + 1.5 * u: 1 + 2 * u, 1 + u / 2 + 2 ** -20: 1 + u, -(1 + u / 2): -1.0,
             1 + 0.49 * u: 1.0, 2 + u: 2.0, 2 + 3 * u: 2 + 4 * u}
    for x, want in cases.items():
        assert mlp.round_bf16(np.array([x]))[0] == want, x
    x = np.random.default_rng(0).normal(0, 10, 100_000)
    r = mlp.round_bf16(x)
    assert np.all(np.abs(r - x) <= 2.0 ** -8 * np.abs(x) * (1 + 1e-6))
    bits = r.astype(np.float32).view(np.uint32)
    assert np.all(bits & 0xFFFF == 0)


def test_bf16_storage_rounds_only_what_the_network_stores():
    """Under storage='bf16' every stored activation is a bf16 value, the raw
    outputs are not rounded, the masks are the signs of the unrounded
    pre-activations, and the result stays within bf16 error of FP64."""
    rng = np.random.default_rng(3)
    Ws, bs = mlp.init_params(rng)
    X = mlp.positional_encoding(rng.random((64, 3)))
    masks = []
    raw_b, H_b = mlp.forward(Ws, bs, X, storage="bf16", masks=masks)
    raw_f, H_f = mlp.forward(Ws, bs, X)
    for h in H_b:
        np.testing.assert_array_equal(h, mlp.round_bf16(h))
    h = mlp.round_bf16(X)
    for l in range(mlp.DEPTH):
        z = h @ Ws[l].T + bs[l]
        np.testing.assert_array_equal(masks[l], z > 0)
        h = mlp.round_bf16(np.maximum(z, 0))
    np.testing.assert_array_equal(raw_b, h @ Ws[-1].T + bs[-1])
    assert np.linalg.norm(raw_b - raw_f) / np.linalg.norm(raw_f) < 2e-2
