"""FP64 oracle for the learned part: NeRF-SH network, quadrature render, the
paper's loss, its gradients, Adam, and the distillation into an octree.

TEST INFRASTRUCTURE ONLY (tests, smoke, the bench's CPU leg).  Plain numpy;
matrix products are the only library primitive.  Follows:
  - network (Sec. 4.2, "Network architecture"): Fourier positional encoding
    of the position, 8 fully connected layers of 256 with ReLU, a linear head
    to sigma and 3 (l_max+1)^2 SH coefficients; sigma = ReLU(raw);
  - emission (Eq. 6): Phi = L_max * sigmoid(sum_k c_k Y_k(d));
  - render (Sec. 4.1, Eq. 3-5): deterministic ray marching with stratified
    samples; exponential or linear (Eq. 4) transmittance; alpha = 1 - T;
  - loss (Sec. 4.3, Eq. 7-9): L = mean_r [ sum_ch ((C^ - C)/(lambda C^ + eps))^2
    + (alpha^ - alpha)^2 ] with eps = 0.01, computed on values divided by L_max
    (lambda = 1), the denominator held constant (no gradient through it);
  - Adam with the learning rate decaying exponentially from 5e-4 to 5e-6
    (Sec. 4.4);
  - distillation (Sec. 5, "Creating the plenoctree"): centre sample of each
    voxel, prune sigma < threshold, average jittered samples in kept voxels;
  - the paper's full setup (Sec. 4.2-4.4): the extra 128-wide SH output
    layer, coarse and fine networks, fine samples placed by the coarse
    weights, loss L_c + L_f + L_alpha.

The SH basis is the oracle's own (``oracle.sh_basis``, Legendre recursion).

Storage precision.  The workload fixes the network's arithmetic as BF16
weights and activations with FP32 accumulation.  With ``storage="bf16"`` the
forward and backward passes round what the network stores between layers to
bfloat16 (round to nearest even, through FP32), at these points: the encoded
input, every hidden ReLU output, d loss / d raw, and every hidden layer's
d loss / d pre-activation after its ReLU mask.  Sums stay in FP64.  The
default ``storage="fp64"`` rounds nothing.
"""
from __future__ import annotations

import math

import numpy as np

import oracle as _oracle

WIDTH = 256
DEPTH = 8
N_FREQ = 10
PE_DIM = 3 + 6 * N_FREQ  # 63


def n_out(l_max: int = 3) -> int:
    return 1 + 3 * (l_max + 1) ** 2


def layer_shapes(l_max: int = 3):
    """[(out, in)] for the 8 hidden layers and the head."""
    shapes = [(WIDTH, PE_DIM)] + [(WIDTH, WIDTH)] * (DEPTH - 1) + [(n_out(l_max), WIDTH)]
    return shapes


def init_params(rng: np.random.Generator, l_max: int = 3):
    """He-uniform weights, zero biases (FP64)."""
    Ws, bs = [], []
    for (o, i) in layer_shapes(l_max):
        lim = math.sqrt(6.0 / i)
        Ws.append(rng.uniform(-lim, lim, (o, i)))
        bs.append(np.zeros(o))
    return Ws, bs


def positional_encoding(x: np.ndarray) -> np.ndarray:
    """gamma(x) = [x, sin(2^j pi x), cos(2^j pi x)]_{j=0..9}, per component:
    x [M,3] -> [M,63] in the order x, then for each j sin (3), cos (3)."""
    feats = [x]
    for j in range(N_FREQ):
        f = (2.0 ** j) * math.pi * x
        feats.append(np.sin(f))
        feats.append(np.cos(f))
    return np.concatenate(feats, axis=1)


def round_bf16(x: np.ndarray) -> np.ndarray:
    """x rounded to bfloat16 (8 significant bits, FP32's exponent range):
    first to FP32, then the low 16 bits of the FP32 pattern rounded away,
    to nearest with ties to even.  Returned as FP64."""
    b = np.ascontiguousarray(x, np.float32).view(np.uint32).astype(np.uint64)
    b = (b + 0x7FFF + ((b >> 16) & 1)) & 0xFFFF0000
    return b.astype(np.uint32).view(np.float32).astype(np.float64)


def _store(x, storage):
    return round_bf16(x) if storage == "bf16" else x


def forward(Ws, bs, X, storage="fp64", masks=None):
    """MLP forward.  Returns (raw outputs [M, n_out], hidden activations,
    the stored ones under bf16 storage).  If `masks` is a list, the hidden
    layers' pre-activation signs (taken before rounding) are appended."""
    X = _store(X, storage)
    H = [X]
    h = X
    masks = [] if masks is None else masks
    for l in range(DEPTH):
        z = h @ Ws[l].T + bs[l]
        masks.append(z > 0)
        h = _store(np.maximum(z, 0.0), storage)
        H.append(h)
    raw = h @ Ws[DEPTH].T + bs[DEPTH]
    return raw, H


def backward(Ws, H, draw, storage="fp64", masks=None):
    """Gradients of the MLP parameters given d loss / d raw.  `masks` are
    the hidden layers' pre-activation signs (default: the stored outputs
    > 0)."""
    dWs = [None] * (DEPTH + 1)
    dbs = [None] * (DEPTH + 1)
    draw = _store(draw, storage)
    dWs[DEPTH] = draw.T @ H[DEPTH]
    dbs[DEPTH] = draw.sum(0)
    g = draw @ Ws[DEPTH]
    for l in range(DEPTH - 1, -1, -1):
        g = _store(g * (masks[l] if masks is not None else (H[l + 1] > 0)), storage)
        dWs[l] = g.T @ H[l]
        dbs[l] = g.sum(0)
        g = g @ Ws[l]
    return dWs, dbs


def clip_unit_cube(o, d):
    """[t0, t1] of each ray inside the unit cube (t0 clamped at 0), and a hit
    mask (positive-length intersection in front of the origin)."""
    with np.errstate(divide="ignore", invalid="ignore"):
        inv = 1.0 / d
        ta = (0.0 - o) * inv
        tb = (1.0 - o) * inv
    tlo = np.where(d == 0, np.where((o >= 0) & (o <= 1), -np.inf, np.inf), np.minimum(ta, tb))
    thi = np.where(d == 0, np.where((o >= 0) & (o <= 1), np.inf, -np.inf), np.maximum(ta, tb))
    t0 = tlo.max(1)
    t1 = thi.min(1)
    hit = (t0 < t1) & (t1 > 0)
    return np.maximum(t0, 0.0), t1, hit


def stratified_samples(rays, jitter):
    """Sample parameters per ray: t_j = t0 + (j + u_j)(t1 - t0)/N, segment
    lengths delta_j = t_{j+1} - t_j (the last one ends at t1), positions
    x_j = o + t_j d.  jitter u [R, N] in [0, 1).  Misses get zero lengths."""
    o, d = rays[:, :3].astype(np.float64), rays[:, 3:].astype(np.float64)
    R, N = jitter.shape
    t0, t1, hit = clip_unit_cube(o, d)
    t0 = np.where(hit, t0, 0.0)
    t1 = np.where(hit, t1, 0.0)
    span = (t1 - t0)[:, None]
    t = t0[:, None] + (np.arange(N)[None, :] + jitter) * span / N
    nxt = np.concatenate([t[:, 1:], t1[:, None]], axis=1)
    delta = np.where(hit[:, None], nxt - t, 0.0)
    x = o[:, None, :] + t[..., None] * d[:, None, :]
    return t, delta, x, hit


def sh_matrix(dirs, l_max):
    return np.stack([_oracle.sh_basis(l_max, v) for v in dirs])


def composite(raw, delta, Y, l_max_scale, transmittance="exp"):
    """Quadrature render of Eq. 3 for raw outputs [R, N, n_out].
    Returns (C [R,3], alpha [R], cache for backward)."""
    R, N, _ = raw.shape
    K = Y.shape[1]
    sigma = np.maximum(raw[..., 0], 0.0)
    coef = raw[..., 1:].reshape(R, N, 3, K)
    s = np.einsum("rnck,rk->rnc", coef, Y)
    sig = 1.0 / (1.0 + np.exp(-s))
    c = l_max_scale * sig
    a = sigma * delta
    cum = np.concatenate([np.zeros((R, 1)), np.cumsum(a, axis=1)], axis=1)  # [R, N+1]
    if transmittance == "exp":
        T = np.exp(-cum)
    else:
        T = np.maximum(0.0, 1.0 - cum)
    w = T[:, :-1] - T[:, 1:]
    C = np.einsum("rn,rnc->rc", w, c)
    alpha = w.sum(1)
    return C, alpha, dict(sigma=sigma, a=a, T=T, w=w, c=c, sig=sig, Y=Y, raw=raw, delta=delta,
                          transmittance=transmittance, l_max_scale=l_max_scale)


def loss_terms(C, alpha, C_gt, alpha_gt, l_max_scale, kind="paper", eps=0.01, lam=1.0, denom=None):
    """Per-ray loss and its gradient w.r.t. (C, alpha).  kind: 'paper'
    (HDR-regularised colour + alpha), 'reg' (colour only), 'mse' (plain MSE
    on normalised colour).  `denom` overrides the held-constant denominator."""
    Cn, Gn = C / l_max_scale, C_gt / l_max_scale
    if kind == "mse":
        den = np.ones_like(Cn)
    else:
        den = lam * Cn + eps if denom is None else denom
    r = (Cn - Gn) / den
    per_ray = (r ** 2).sum(1)
    dC = 2.0 * r / den / l_max_scale
    dA = np.zeros_like(alpha)
    if kind == "paper":
        per_ray = per_ray + (alpha - alpha_gt) ** 2
        dA = 2.0 * (alpha - alpha_gt)
    return per_ray, dC, dA


def composite_backward(cache, dC, dA):
    """d loss / d raw [R, N, n_out] from d loss / d C and d loss / d alpha."""
    w, c, T, a = cache["w"], cache["c"], cache["T"], cache["a"]
    sig, Y, raw, delta = cache["sig"], cache["Y"], cache["raw"], cache["delta"]
    R, N = w.shape
    K = Y.shape[1]
    dc = w[..., None] * dC[:, None, :]                       # d/dc_j
    ds = dc * cache["l_max_scale"] * sig * (1.0 - sig)       # through the sigmoid
    dcoef = np.einsum("rnc,rk->rnck", ds, Y).reshape(R, N, 3 * K)
    # d/da_j.  exp: dw_k/da_j = T_{j+1} for k = j, -w_k for k > j;
    # linear: T_k = max(0, 1 - cum_k), w_k = T_k - T_{k+1}.
    g_w = np.einsum("rnc,rc->rn", c, dC) + dA[:, None]      # d loss / d w_k
    if cache["transmittance"] == "exp":
        Tn = T[:, 1:]
        suffix = np.flip(np.cumsum(np.flip(w * g_w, 1), 1), 1)  # sum_{k>=j} w_k g_k
        after = suffix - w * g_w                                 # sum_{k>j}
        da = Tn * g_w - after
    else:
        # T_k depends on a_j (j < k) with slope -1 while 1 - cum_k > 0
        act = (1.0 - np.concatenate([np.zeros((R, 1)), np.cumsum(a, 1)], 1)) > 0  # [R, N+1]
        # w_k = T_k - T_{k+1}: d w_k / d a_j = -act_k [j<k] + act_{k+1} [j<k+1]
        # d loss/d a_j = sum_k g_k (act_{k+1}[j<=k] - act_k[j<k])
        gk_act_next = g_w * act[:, 1:]
        gk_act = g_w * act[:, :-1]
        s1 = np.flip(np.cumsum(np.flip(gk_act_next, 1), 1), 1)          # sum_{k>=j}
        s2 = np.flip(np.cumsum(np.flip(gk_act, 1), 1), 1) - gk_act      # sum_{k>j}
        da = s1 - s2
    dsigma = da * delta * (raw[..., 0] > 0)
    return np.concatenate([dsigma[..., None], dcoef], axis=2)


def train_loss_and_grads(Ws, bs, rays, jitter, C_gt, alpha_gt, l_max_scale, l_max=3, kind="paper",
                         transmittance="exp", denom=None, arch="linear", storage="fp64", X=None):
    """One training batch: returns (mean loss, dWs, dbs, extras).  arch:
    'linear' (linear head) or 'paper' (the 128-wide SH layer); storage:
    'fp64' or 'bf16' (see the module's header); X overrides the encoded
    samples [R * N, 63] (for example with another implementation's own
    rounding of them)."""
    fwd, bwd = (forward_paper, backward_paper) if arch == "paper" else (forward, backward)
    t, delta, x, hit = stratified_samples(rays, jitter)
    R, N = jitter.shape
    if X is None:
        X = positional_encoding(x.reshape(R * N, 3))
    masks = []
    raw, H = fwd(Ws, bs, X, storage=storage, masks=masks)
    raw = raw.reshape(R, N, -1)
    d = rays[:, 3:].astype(np.float64)
    Y = sh_matrix(d, l_max)
    C, alpha, cache = composite(raw, delta, Y, l_max_scale, transmittance)
    per_ray, dC, dA = loss_terms(C, alpha, C_gt, alpha_gt, l_max_scale, kind, denom=denom)
    loss = per_ray.mean()
    draw = composite_backward(cache, dC / R, dA / R).reshape(R * N, -1)
    dWs, dbs = bwd(Ws, H, draw, storage=storage, masks=masks)
    return loss, dWs, dbs, dict(C=C, alpha=alpha, raw=raw, draw=draw, X=X, delta=delta)


# ---------------------------------------------------------------- the paper's full training setup
# Sec. 4.2 (network architecture): the 8 x 256 trunk, then a 128-wide hidden
# layer whose output gives the 3 (l_max+1)^2 SH coefficients; sigma is read
# linearly from the trunk.  Sec. 4.3 / 4.4: a coarse and a fine network,
# N_c = 64 stratified samples for the coarse one and N_f = 128 more, placed
# by the coarse weights, for the fine one; loss L_c + L_f + L_alpha.

FEAT = 128


def layer_shapes_paper(l_max: int = 3):
    """[(out, in)]: 8 trunk layers, then sigma (1 x 256), the 128-wide
    feature layer (128 x 256) and the SH layer (3K x 128)."""
    K = (l_max + 1) ** 2
    return [(WIDTH, PE_DIM)] + [(WIDTH, WIDTH)] * (DEPTH - 1) + [(1, WIDTH), (FEAT, WIDTH), (3 * K, FEAT)]


def init_params_paper(rng: np.random.Generator, l_max: int = 3):
    Ws, bs = [], []
    for (o, i) in layer_shapes_paper(l_max):
        lim = math.sqrt(6.0 / i)
        Ws.append(rng.uniform(-lim, lim, (o, i)))
        bs.append(np.zeros(o))
    return Ws, bs


def forward_paper(Ws, bs, X, storage="fp64", masks=None):
    """Trunk, then raw sigma = W_s h8 + b_s and SH = W_c ReLU(W_f h8 + b_f) + b_c.
    Returns (raw [M, 1 + 3K] with sigma first, activations [X, h1..h8, feat]);
    `masks` as in forward, the 128-wide layer's last."""
    X = _store(X, storage)
    H = [X]
    h = X
    masks = [] if masks is None else masks
    for l in range(DEPTH):
        z = h @ Ws[l].T + bs[l]
        masks.append(z > 0)
        h = _store(np.maximum(z, 0.0), storage)
        H.append(h)
    sig = h @ Ws[DEPTH].T + bs[DEPTH]
    zf = h @ Ws[DEPTH + 1].T + bs[DEPTH + 1]
    masks.append(zf > 0)
    feat = _store(np.maximum(zf, 0.0), storage)
    H.append(feat)
    sh = feat @ Ws[DEPTH + 2].T + bs[DEPTH + 2]
    return np.concatenate([sig, sh], axis=1), H


def backward_paper(Ws, H, draw, storage="fp64", masks=None):
    """Parameter gradients of forward_paper given d loss / d raw.  `masks`:
    the pre-activation signs of the trunk layers and the 128-wide layer
    (default: the stored outputs > 0).  Under bf16 storage the gradient of
    the 128-wide layer and sigma's is stored as one bf16 block."""
    n = DEPTH + 3
    dWs, dbs = [None] * n, [None] * n
    draw = _store(draw, storage)
    mk = (lambda l: masks[l]) if masks is not None else (lambda l: H[l + 1] > 0)
    dsig, dsh = draw[:, :1], draw[:, 1:]
    h8, feat = H[DEPTH], H[DEPTH + 1]
    dWs[DEPTH + 2] = dsh.T @ feat
    dbs[DEPTH + 2] = dsh.sum(0)
    gf = _store((dsh @ Ws[DEPTH + 2]) * mk(DEPTH), storage)
    dWs[DEPTH + 1] = gf.T @ h8
    dbs[DEPTH + 1] = gf.sum(0)
    dWs[DEPTH] = dsig.T @ h8
    dbs[DEPTH] = dsig.sum(0)
    g = gf @ Ws[DEPTH + 1] + dsig @ Ws[DEPTH]
    for l in range(DEPTH - 1, -1, -1):
        g = _store(g * mk(l), storage)
        dWs[l] = g.T @ H[l]
        dbs[l] = g.sum(0)
        g = g @ Ws[l]
    return dWs, dbs


FINE_FLOOR = 1e-5


def fine_samples(t, delta, w, xi):
    """N_f samples per ray from the coarse pass.  Coarse sample i owns the
    segment [t_i, t_i + delta_i); the density is constant on each segment
    and its mass there is proportional to w_i + 1e-5 (the floor keeps
    the density defined where the coarse weights vanish).  Stratified
    u_j = (j + xi_j) / N_f is mapped through the inverse CDF:
    t = t_i + (u - C_i) / (C_{i+1} - C_i) * delta_i for C_i <= u < C_{i+1}.
    t, delta, w [R, N_c]; xi [R, N_f] in [0, 1).  Returns t_fine [R, N_f]
    (ascending in j)."""
    R, Nc = t.shape
    Nf = xi.shape[1]
    m = w + FINE_FLOOR
    C = np.concatenate([np.zeros((R, 1)), np.cumsum(m, axis=1)], axis=1)
    C = C / C[:, -1:]
    u = (np.arange(Nf)[None, :] + xi) / Nf
    out = np.empty((R, Nf))
    for r in range(R):
        i = np.searchsorted(C[r], u[r], side="right") - 1
        i = np.clip(i, 0, Nc - 1)
        frac = (u[r] - C[r, i]) / (C[r, i + 1] - C[r, i])
        out[r] = t[r, i] + frac * delta[r, i]
    return out


def merge_samples(t_coarse, t_fine, t1):
    """Union of the coarse and fine parameters per ray in ascending order,
    with delta_j = t_{j+1} - t_j and the last segment ending at t1."""
    t = np.sort(np.concatenate([t_coarse, t_fine], axis=1), axis=1, kind="stable")
    nxt = np.concatenate([t[:, 1:], t1[:, None]], axis=1)
    return t, nxt - t


def train_loss_and_grads_hier(Wc, bc, Wf, bf, rays, jitter, xi, C_gt, alpha_gt, l_max_scale, l_max=3,
                              transmittance="exp", arch="paper", denoms=(None, None), t_fine=None,
                              storage="fp64", X_coarse=None, X_fine=None):
    """One batch of the paper's training (Eq. finaloss): coarse colour loss
    L_c on N_c stratified samples (jitter [R, N_c]), fine colour loss L_f
    and alpha loss L_alpha on the coarse plus N_f fine samples (xi [R, N_f]).
    No gradient flows through the sample placement.  `denoms` overrides the
    held-constant loss denominators (coarse, fine); `t_fine` overrides the
    fine samples (to hold them fixed); storage and X_coarse / X_fine (the
    encoded samples of either pass) as in train_loss_and_grads.  Returns
    (mean loss, (dWc, dbc), (dWf, dbf), extras)."""
    fwd, bwd = (forward_paper, backward_paper) if arch == "paper" else (forward, backward)
    R, Nc = jitter.shape
    d = rays[:, 3:].astype(np.float64)
    o = rays[:, :3].astype(np.float64)
    Y = sh_matrix(d, l_max)
    t, delta, x, hit = stratified_samples(rays, jitter)
    mc, mf = [], []
    Xc = positional_encoding(x.reshape(R * Nc, 3)) if X_coarse is None else X_coarse
    raw_c, Hc = fwd(Wc, bc, Xc, storage=storage, masks=mc)
    raw_c = raw_c.reshape(R, Nc, -1)
    C_c, a_c, cache_c = composite(raw_c, delta, Y, l_max_scale, transmittance)
    per_c, dC_c, _ = loss_terms(C_c, a_c, C_gt, alpha_gt, l_max_scale, "reg", denom=denoms[0])
    t0, t1, _ = clip_unit_cube(o, d)
    t1 = np.where(hit, t1, 0.0)
    tf = fine_samples(t, delta, cache_c["w"], xi) if t_fine is None else t_fine
    ta, da = merge_samples(t, tf, t1)
    da = np.where(hit[:, None], da, 0.0)
    N = ta.shape[1]
    xa = o[:, None, :] + ta[..., None] * d[:, None, :]
    Xf = positional_encoding(xa.reshape(R * N, 3)) if X_fine is None else X_fine
    raw_f, Hf = fwd(Wf, bf, Xf, storage=storage, masks=mf)
    raw_f = raw_f.reshape(R, N, -1)
    C_f, a_f, cache_f = composite(raw_f, da, Y, l_max_scale, transmittance)
    per_f, dC_f, dA_f = loss_terms(C_f, a_f, C_gt, alpha_gt, l_max_scale, "paper", denom=denoms[1])
    loss = (per_c + per_f).mean()
    draw_c = composite_backward(cache_c, dC_c / R, np.zeros(R)).reshape(R * Nc, -1)
    draw_f = composite_backward(cache_f, dC_f / R, dA_f / R).reshape(R * N, -1)
    gc = bwd(Wc, Hc, draw_c, storage=storage, masks=mc)
    gf = bwd(Wf, Hf, draw_f, storage=storage, masks=mf)
    return loss, gc, gf, dict(C_c=C_c, C_f=C_f, alpha_f=a_f, t_fine=tf, t_all=ta, delta_all=da,
                              w_c=cache_c["w"], loss_c=per_c.mean(), loss_f=per_f.mean())


def lr_at(step: int, total: int, lr0=5e-4, lr1=5e-6) -> float:
    """Exponential decay from lr0 to lr1 over `total` steps (Sec. 4.4)."""
    return lr0 * (lr1 / lr0) ** (min(step, total) / max(total, 1))


def adam_update(p, g, m, v, step, lr, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam update (step counts from 1).  Returns new (p, m, v)."""
    m = b1 * m + (1 - b1) * g
    v = b2 * v + (1 - b2) * g * g
    mh = m / (1 - b1 ** step)
    vh = v / (1 - b2 ** step)
    return p - lr * mh / (np.sqrt(vh) + eps), m, v


def distill_dense(Ws, bs, depth, jitter, sigma_thresh=0.01, l_max=3):
    """Plenoctree extraction at `depth`: sigma of each voxel centre; voxels
    with sigma >= sigma_thresh are kept and get the average of ReLU(sigma)
    and of the raw SH coefficients over the jittered samples jitter
    [n_kept, S, 3] (offsets in [0,1)^3 inside the voxel).  Returns
    (kept voxel integer coords [n,3] in x-fastest order, sigma_centre of all
    voxels [G^3], averaged sigma [n], averaged SH [n, 3, K])."""
    G = 1 << depth
    idx = np.arange(G ** 3)
    ijk = np.stack([idx % G, (idx // G) % G, idx // (G * G)], 1)
    centres = (ijk + 0.5) / G
    raw, _ = forward(Ws, bs, positional_encoding(centres))
    sig_c = np.maximum(raw[:, 0], 0.0)
    kept = np.nonzero(sig_c >= sigma_thresh)[0]
    if jitter is None:
        return ijk[kept], sig_c, None, None
    S = jitter.shape[1]
    pts = (ijk[kept][:, None, :] + jitter[: len(kept)]) / G
    raw_s, _ = forward(Ws, bs, positional_encoding(pts.reshape(-1, 3)))
    raw_s = raw_s.reshape(len(kept), S, -1)
    sig = np.maximum(raw_s[..., 0], 0.0).mean(1)
    K = (l_max + 1) ** 2
    sh = raw_s[..., 1:].mean(1).reshape(len(kept), 3, K)
    return ijk[kept], sig_c, sig, sh


# ---------------------------------------------------------------- distillation sampling
# Voxels are addressed by their Morton code at depth D: the child slot
# (bx | by << 1 | bz << 2) of every level from the root, most significant
# first.  The jittered sample offsets inside a voxel come from the SplitMix64
# generator (Steele, Lea, Flood, "Fast splittable pseudorandom number
# generators", OOPSLA 2014), written here from its definition:
#   mix(z): z += 0x9E3779B97F4A7C15; z = (z ^ z>>30) * 0xBF58476D1CE4E5B9;
#           z = (z ^ z>>27) * 0x94D049BB133111EB; return z ^ z>>31
#   key = mix(mix(seed ^ 0xD15711) ^ (code * 0x9E3779B97F4A7C15 + 3 s + a))
#   u   = (key >> 40) / 2^24            (sample s, axis a)
_M64 = (1 << 64) - 1


def _mix64(z):
    z = (z + 0x9E3779B97F4A7C15) & _M64
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & _M64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & _M64
    return z ^ (z >> 31)


def morton_code(ijk, depth):
    """Morton code of integer voxel coords [n,3] at `depth`."""
    code = np.zeros(len(ijk), dtype=object)
    for l in range(depth):
        bit = depth - 1 - l
        slot = ((ijk[:, 0] >> bit) & 1) | (((ijk[:, 1] >> bit) & 1) << 1) | (((ijk[:, 2] >> bit) & 1) << 2)
        code = code * 8 + slot.astype(object)
    return code


def distill_jitter(seed, codes, S):
    """Offsets in [0,1)^3 of S samples in each voxel, [n, S, 3]."""
    k0 = _mix64(seed ^ 0xD15711)
    out = np.empty((len(codes), S, 3))
    for i, c in enumerate(codes):
        base = (int(c) * 0x9E3779B97F4A7C15) & _M64
        for s in range(S):
            for a in range(3):
                key = _mix64(k0 ^ ((base + 3 * s + a) & _M64))
                out[i, s, a] = (key >> 40) / 16777216.0
    return out
