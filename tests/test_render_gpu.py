"""GPU parity: plo_render_rays / plo_lookup_points / plo_trace_rays against
the FP64 oracle on the same seeded inputs (Eq. 3-5, Sec. 5)."""
import numpy as np
import pytest

import oracle
import paper_2207_05009_gb300 as plo
import plogen
from plogen import HostTree
from tests.parity import COND_ETA_LINEAR, RTOL_BF16, RTOL_FP16, RTOL_FP32, assert_radiance_close, quantise_tree
from tests.trees import random_tree, uniform_tree

pytestmark = pytest.mark.gpu

TRANS = {"exp": (plo.TRANS_EXP, oracle.EXPONENTIAL), "lin": (plo.TRANS_LINEAR, oracle.LINEAR),
         "lit": (plo.TRANS_LINEAR_LITERAL, oracle.LINEAR_LITERAL)}


@pytest.fixture(scope="module")
def torch_cuda(cuda_available):
    import torch
    return torch


@pytest.fixture(scope="module")
def d6():
    return plogen.luminaire_tree(plogen.LUMINAIRE_D6)


# device layouts: the octree, and bricks of side 8, 4 and 2 finest cells
LAYOUTS = {"octree": (plo.LAYOUT_OCTREE, 0), "bricks8": (plo.LAYOUT_BRICKS, 3), "bricks4": (plo.LAYOUT_BRICKS, 2),
           "bricks2": (plo.LAYOUT_BRICKS, 1)}
ALL_LAYOUTS = pytest.mark.parametrize("layout", list(LAYOUTS))
TWO_LAYOUTS = pytest.mark.parametrize("layout", ["octree", "bricks8"])


def gpu_render(torch, tree, rays, precision=plo.PREC_FP32, layout="octree", **kw):
    t = plo.Tree(tree, precision, *LAYOUTS[layout])
    r = torch.from_numpy(np.ascontiguousarray(rays)).cuda()
    st = torch.full((len(rays),), -7, dtype=torch.int32, device="cuda")
    rgb, T, _ = plo.render(t, r, plo.RenderParams(**kw), status=st)
    torch.cuda.synchronize()
    t.check()
    return rgb.cpu().numpy(), T.cpu().numpy(), st.cpu().numpy()


@TWO_LAYOUTS
@pytest.mark.parametrize("model", ["exp", "lin", "lit"])
def test_d6_luminaire_fp32_parity(torch_cuda, d6, model, layout):
    rays = plogen.rays_sphere(65536, seed=1)
    g_rgb, g_T, st = gpu_render(torch_cuda, d6, rays, transmittance=TRANS[model][0], layout=layout)
    ref = oracle.render(d6, rays, transmittance=TRANS[model][1])
    assert np.all(st == 0)
    eta = 0.0 if model == "exp" else COND_ETA_LINEAR
    assert_radiance_close(g_rgb, g_T, ref, RTOL_FP32, what=f"D6 {model}", cond_eta=eta)


def test_sigmoid_activation_parity(torch_cuda, d6):
    rays = plogen.rays_sphere(8192, seed=2)
    tree = HostTree(d6.depth, d6.sh_degree, d6.child, d6.sigma, d6.sh * 1e-3 - 0.5)
    g_rgb, g_T, _ = gpu_render(torch_cuda, tree, rays, activation=plo.ACT_SIGMOID, l_max=12.5)
    ref = oracle.render(tree, rays, activation=oracle.SIGMOID, l_max=12.5)
    assert_radiance_close(g_rgb, g_T, ref, RTOL_FP32, what="sigmoid")


@ALL_LAYOUTS
@pytest.mark.parametrize("seed", range(8))
def test_random_trees_all_degrees_ragged(torch_cuda, seed, layout):
    rng = np.random.default_rng(seed)
    deg = seed % 5
    tree = random_tree(1 + seed % 5, rng, sh_degree=deg)
    n = 1000 + 37 * seed  # not a multiple of the warp or block size
    rays = plogen.rays_sphere(n, seed=100 + seed, radius=1.5 + seed)
    g_rgb, g_T, st = gpu_render(torch_cuda, tree, rays, layout=layout)
    ref = oracle.render(tree, rays)
    assert np.all(st == 0)
    assert_radiance_close(g_rgb, g_T, ref, RTOL_FP32, what=f"random tree {seed}")


@ALL_LAYOUTS
def test_degenerate_trees(torch_cuda, layout):
    c = np.random.default_rng(0).normal(size=(3, 9)).astype(np.float32) + 2
    rays = plogen.rays_sphere(2000, seed=5)
    for tree in (uniform_tree(0, 2.0, c), uniform_tree(1, 0.7, c),
                 HostTree(0, 2, np.zeros((0, 8), np.int32), np.zeros(0, np.float32), np.zeros((0, 3, 9), np.float32))):
        g_rgb, g_T, st = gpu_render(torch_cuda, tree, rays, layout=layout)
        ref = oracle.render(tree, rays)
        assert_radiance_close(g_rgb, g_T, ref, RTOL_FP32, what=f"degenerate depth {tree.depth}")


def deep_chain_tree(depth, rng):
    """A path of nodes down to `depth` (the maximum, 16) with leaves beside it."""
    child = []
    sig, sh = [], []
    for lev in range(depth):
        row = []
        for s in range(8):
            if s == 0 and lev < depth - 1:
                row.append(len(child) + 1)
            else:
                sig.append(float(rng.uniform(0.5, 50.0)))
                sh.append(rng.normal(size=(3, 9)) + 1.0)
                row.append(-len(sig) - 1)
        child.append(row)
    return HostTree(depth, 2, np.array(child, np.int32), np.array(sig, np.float32), np.array(sh, np.float32))


@ALL_LAYOUTS
def test_max_depth_16(torch_cuda, layout):
    tree = deep_chain_tree(16, np.random.default_rng(3))
    rays = plogen.rays_sphere(4000, seed=6, radius=2.0, center=(0.0, 0.0, 0.0))
    g_rgb, g_T, st = gpu_render(torch_cuda, tree, rays, layout=layout)
    ref = oracle.render(tree, rays)
    assert np.all(st == 0)
    assert_radiance_close(g_rgb, g_T, ref, RTOL_FP32, what="depth 16")


@ALL_LAYOUTS
def test_edge_rays(torch_cuda, d6, layout):
    rng = np.random.default_rng(7)
    rays = []
    g = np.arange(65) / 64.0
    for _ in range(300):  # axis-parallel rays lying on cell planes
        a = rng.integers(0, 3)
        o = rng.choice(g, 3).astype(np.float64)
        o[a] = -1.0 if rng.random() < 0.5 else 2.0
        d = np.zeros(3)
        d[a] = 1.0 if o[a] < 0 else -1.0
        rays.append(np.concatenate([o, d]))
    for _ in range(300):  # origins inside the cube
        d = rng.normal(size=3)
        rays.append(np.concatenate([rng.random(3), d / np.linalg.norm(d)]))
    for _ in range(100):  # diagonal rays through cell corners
        o = rng.choice(g, 3) - 2.0
        rays.append(np.concatenate([o, np.ones(3) / np.sqrt(3)]))
    rays.append([0.5, 0.5, 0.5, 0.0, 0.0, 1.0])     # starts on the centre corner
    rays.append([1.0, 0.3, 0.3, 1.0, 0.0, 0.0])     # starts on a face, leaves at once
    rays.append([0.0, 0.2, 0.2, 0.0, 1.0, 0.0])     # slides along the x = 0 face
    rays = np.array(rays, np.float32)
    g_rgb, g_T, st = gpu_render(torch_cuda, d6, rays, layout=layout)
    ref = oracle.render(d6, rays)
    assert np.all(st == 0)
    assert_radiance_close(g_rgb, g_T, ref, RTOL_FP32, what="edge rays")


@TWO_LAYOUTS
def test_invalid_and_missing_rays(torch_cuda, d6, layout):
    rays = np.array([[np.nan, 0, 0, 0, 0, 1], [0, 0, -1, 0, 0, 0], [0.5, 0.5, -1, 0, 0, np.inf],
                     [5, 5, 5, 1, 0, 0], [0.5, 0.5, -1, 0, 0, -1]], np.float32)
    g_rgb, g_T, st = gpu_render(torch_cuda, d6, rays, layout=layout)
    ref = oracle.render(d6, rays)
    assert list(st) == [plo.RAY_INVALID] * 3 + [0, 0]
    assert np.all(np.isnan(g_rgb[:3])) and np.all(np.isnan(g_T[:3]))
    assert np.all(ref["status"][:3] == 3)
    np.testing.assert_array_equal(g_rgb[3:], 0.0)
    np.testing.assert_array_equal(g_T[3:], 1.0)


def test_empty_input_is_a_noop(torch_cuda, d6):
    import torch
    t = plo.Tree(d6)
    r = torch.empty((0, 6), device="cuda")
    rgb, T, _ = plo.render(t, r)
    torch.cuda.synchronize()
    assert rgb.shape == (0, 3) and T.shape == (0,)


@TWO_LAYOUTS
def test_early_stop_within_tail_bound(torch_cuda, d6, layout):
    rays = plogen.rays_sphere(65536, seed=9)
    g_rgb, g_T, _ = gpu_render(torch_cuda, d6, rays, t_stop=1e-4, layout=layout)
    full = oracle.render(d6, rays)
    stop = oracle.render(d6, rays, t_stop=1e-4)
    # same stop rule as the oracle: compare with the oracle's early-stopped
    # result, except for rays whose T crosses t_stop within the FP32 error
    near = np.abs(full["T"] - 1e-4) < 1e-6
    assert_radiance_close(g_rgb, g_T, stop, RTOL_FP32, mask=~near, what="t_stop")


def test_step_limit_is_reported(torch_cuda, d6):
    rays = plogen.rays_sphere(1024, seed=10)
    t = plo.Tree(d6)
    import torch
    st = torch.zeros(1024, dtype=torch.int32, device="cuda")
    plo.render(t, torch.from_numpy(rays).cuda(), plo.RenderParams(max_steps=3), status=st)
    torch.cuda.synchronize()
    assert (st.cpu().numpy() == plo.RAY_STEP_LIMIT).any()
    with pytest.raises(plo.PloError) as ei:
        t.check()
    assert ei.value.status == -5
    t.check()  # flag cleared


def test_world_bbox(torch_cuda, d6):
    tree = HostTree(d6.depth, d6.sh_degree, d6.child, d6.sigma, d6.sh, bbox_min=(-1.0, -2.0, 0.0),
                    bbox_max=(3.0, 2.0, 4.0))
    rays = plogen.rays_sphere(8192, seed=11, radius=9.0, center=(1.0, 0.0, 2.0))
    g_rgb, g_T, _ = gpu_render(torch_cuda, tree, rays)
    ref = oracle.render(tree, rays)
    assert_radiance_close(g_rgb, g_T, ref, RTOL_FP32, what="world bbox")


@TWO_LAYOUTS
@pytest.mark.parametrize("prec,name", [(plo.PREC_FP16, "fp16"), (plo.PREC_BF16, "bf16")])
def test_16bit_leaves(torch_cuda, d6, prec, name, layout):
    rays = plogen.rays_sphere(65536, seed=12)
    g_rgb, g_T, _ = gpu_render(torch_cuda, d6, rays, precision=prec, layout=layout)
    # arithmetic parity: the oracle on the exactly dequantised tree
    ref_q = oracle.render(quantise_tree(d6, name), rays)
    assert_radiance_close(g_rgb, g_T, ref_q, RTOL_FP32, what=f"{name} vs dequantised oracle")
    # storage error: the oracle on the original FP32 leaves
    ref = oracle.render(d6, rays)
    rtol = RTOL_FP16 if name == "fp16" else RTOL_BF16
    assert_radiance_close(g_rgb, g_T, ref, rtol, what=f"{name} vs FP32-leaf oracle")


@TWO_LAYOUTS
@pytest.mark.parametrize("prec,name", [(plo.PREC_FP32, "fp32"), (plo.PREC_FP16, "fp16"), (plo.PREC_BF16, "bf16")])
def test_sh_degree_4_leaves(torch_cuda, prec, name, layout):
    """l_max = 4 (K = 25, the largest degree of the paper's ablation, Sec.
    6.2) on the depth-6 luminaire's geometry: FP32 leaves against the FP64
    oracle, 16-bit leaves against the oracle on the dequantised tree."""
    tree = plogen.luminaire_tree(plogen.LUMINAIRE_D6.with_(sh_degree=4))
    assert tree.K == 25
    rays = plogen.rays_sphere(32768, seed=21)
    g_rgb, g_T, st = gpu_render(torch_cuda, tree, rays, precision=prec, layout=layout)
    assert np.all(st == 0)
    ref = oracle.render(tree if name == "fp32" else quantise_tree(tree, name), rays)
    assert_radiance_close(g_rgb, g_T, ref, RTOL_FP32, what=f"l_max 4 {name} {layout}")


def test_lookup_bit_exact(torch_cuda, d6):
    import torch
    rng = np.random.default_rng(13)
    g = np.arange(65) / 64.0
    pts = rng.random((20000, 3)).astype(np.float32)
    on = rng.random(pts.shape) < 0.3
    pts[on] = rng.choice(g, on.sum())
    pts[:50] = np.array([[0, 0, 0], [1, 1, 1], [0.5, 0.5, 0.5], [1, 0, 1], [-1e-7, 0.5, 0.5]] * 10)
    dirs = rng.normal(size=pts.shape).astype(np.float32)
    dirs[rng.random(dirs.shape) < 0.2] = 0.0
    t = plo.Tree(d6)
    for use_dir in (False, True):
        leaf, lev = plo.lookup(t, torch.from_numpy(pts).cuda(),
                               torch.from_numpy(dirs).cuda() if use_dir else None)
        ref, ref_lev = oracle.lookup(d6, pts, dirs if use_dir else None)
        np.testing.assert_array_equal(leaf.cpu().numpy(), ref)
        ok = ref >= -1
        np.testing.assert_array_equal(lev.cpu().numpy()[ok], ref_lev[ok])


def test_trace_matches_oracle_cell_sequence(torch_cuda, d6):
    import torch
    rays = plogen.rays_sphere(300, seed=14)
    t = plo.Tree(d6)
    M = 512
    leaf, tt, cnt = plo.trace(t, torch.from_numpy(rays).cuda(), M)
    leaf, tt, cnt = leaf.cpu().numpy(), tt.cpu().numpy().astype(np.float64), cnt.cpu().numpy()
    for i, r in enumerate(rays):
        ol, ot = oracle.trace(d6, r)
        keep_o = (ot[:, 1] - ot[:, 0]) >= 1e-6
        n = min(cnt[i], M)
        keep_g = (tt[i, :n, 1] - tt[i, :n, 0]) >= 1e-6
        np.testing.assert_array_equal(leaf[i, :n][keep_g], ol[keep_o], err_msg=f"ray {i}")
        np.testing.assert_allclose(tt[i, :n][keep_g], ot[keep_o], rtol=0, atol=2e-6)


def test_deterministic_and_host_path(torch_cuda, d6):
    import torch
    rays = plogen.rays_sphere(3 * (1 << 20) // 2, seed=15)  # spans two host-path chunks
    t = plo.Tree(d6)
    r = torch.from_numpy(rays).cuda()
    a = plo.render(t, r)
    b = plo.render(t, r)
    torch.cuda.synchronize()
    assert torch.equal(a[0], b[0]) and torch.equal(a[1], b[1])
    h_rgb, h_T = plo.render_host(t, rays)
    np.testing.assert_array_equal(h_rgb, a[0].cpu().numpy())
    np.testing.assert_array_equal(h_T, a[1].cpu().numpy())
    # four chunks of a quarter of the rays each, the last one ragged
    rays = plogen.rays_sphere(4 * (1 << 20) + 12345, seed=16)
    a = plo.render(t, torch.from_numpy(rays).cuda())
    h_rgb, h_T = plo.render_host(t, rays)
    np.testing.assert_array_equal(h_rgb, a[0].cpu().numpy())
    np.testing.assert_array_equal(h_T, a[1].cpu().numpy())


@pytest.mark.parametrize("prec", [plo.PREC_FP32, plo.PREC_FP16])
def test_ray_order_leaves_results_unchanged(torch_cuda, d6, prec):
    """Wavefronts of 2^23 rays or more are rendered in entry-cell order (a
    sorted scratch copy); the same rays rendered in launches below that size
    (in index order) give bit-identical outputs and statuses, including rays
    that miss the box and rays with non-finite components."""
    import torch
    rays = plogen.rays_room((1 << 23) + 4097, seed=17).copy()
    rays[::9973, :3] = (9.0, 9.0, 9.0)  # misses
    rays[5::99991, 3] = np.nan  # invalid
    t = plo.Tree(d6, prec)
    r = torch.from_numpy(rays).cuda()
    st = torch.full((len(rays),), -7, dtype=torch.int32, device="cuda")
    a_rgb, a_T, _ = plo.render(t, r, status=st)
    half = len(rays) // 2
    sts = [torch.full((n,), -7, dtype=torch.int32, device="cuda") for n in (half, len(rays) - half)]
    b = [plo.render(t, r[:half].contiguous(), status=sts[0]), plo.render(t, r[half:].contiguous(), status=sts[1])]
    torch.cuda.synchronize()
    t.check()
    b_rgb, b_T = torch.cat([b[0][0], b[1][0]]), torch.cat([b[0][1], b[1][1]])
    assert torch.equal(torch.nan_to_num(a_rgb, nan=-1.0), torch.nan_to_num(b_rgb, nan=-1.0))
    assert torch.equal(torch.nan_to_num(a_T, nan=-1.0), torch.nan_to_num(b_T, nan=-1.0))
    assert torch.equal(st, torch.cat(sts))
    assert bool(torch.isnan(a_T).any()) and bool((st == plo.RAY_INVALID).any())


# ---------------------------------------------------------------- sphere proxy (Sec. 5) and the
# sigma_min / alpha_max heuristics (Sec. 6.2)

def cube_rays(n, seed):
    """Origins uniform inside the unit cube, isotropic unit directions."""
    rng = np.random.default_rng(seed)
    d = rng.normal(size=(n, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    return np.concatenate([rng.uniform(0, 1, (n, 3)), d], 1).astype(np.float32)


@pytest.mark.parametrize("model", ["exp", "lin"])
@pytest.mark.parametrize("sphere", [(0.5, 0.5, 0.5, 0.4), (0.62, 0.45, 0.5, 0.55), (0.5, 0.5, 0.5, 0.9)])
@TWO_LAYOUTS
def test_sphere_proxy_parity(torch_cuda, d6, model, sphere, layout):
    rays = np.concatenate([plogen.rays_sphere(32768, seed=31), cube_rays(4096, 33)])
    g_rgb, g_T, st = gpu_render(torch_cuda, d6, rays, transmittance=TRANS[model][0], sphere=sphere, layout=layout)
    # the API takes the sphere in FP32: give the oracle the same values
    sphere = tuple(float(np.float32(v)) for v in sphere)
    ref = oracle.render(d6, rays, transmittance=TRANS[model][1], sphere=sphere)
    assert np.all(st == 0)
    eta = 0.0 if model == "exp" else COND_ETA_LINEAR
    assert_radiance_close(g_rgb, g_T, ref, RTOL_FP32, what=f"sphere {sphere} {model}", cond_eta=eta)
    box = oracle.render(d6, rays, transmittance=TRANS[model][1])
    clipped = np.abs(box["T"] - ref["T"]) > 1e-6
    if sphere[3] < 0.87:
        assert clipped.sum() > 100  # the ball cuts the luminaire: the clip is exercised
    else:
        assert not clipped.any()


@TWO_LAYOUTS
def test_paper_heuristics_parity(torch_cuda, d6, layout):
    rays = plogen.rays_sphere(65536, seed=32)
    hp = dict(sigma_min=0.1, saturate=True)
    g_rgb, g_T, _ = gpu_render(torch_cuda, d6, rays, t_stop=0.1, layout=layout, **hp)
    ref = oracle.render(d6, rays, t_stop=0.1, **hp)
    # rays whose running T passes within FP32 rounding of t_stop may stop one
    # leaf apart: find them by moving the threshold by 1e-5 either way
    lo = oracle.render(d6, rays, t_stop=0.1 * (1 - 1e-5), **hp)
    hi = oracle.render(d6, rays, t_stop=0.1 * (1 + 1e-5), **hp)
    near = (lo["n_leaf"] != hi["n_leaf"]) | ((lo["T"] == 0) != (hi["T"] == 0))
    assert near.mean() < 1e-3
    assert_radiance_close(g_rgb, g_T, ref, RTOL_FP32, mask=~near, what="sigma_min 0.1, alpha_max 0.9")
    saturated = ref["T"] == 0
    assert saturated.sum() > 1000
    assert np.all(g_T[saturated & ~near] == 0)
    # the preset in the binding is the same parameter set
    p = plo.RenderParams.paper_heuristics()
    assert (p.sigma_min, p.t_stop, p.saturate) == (0.1, 0.1, True)


def test_sphere_proxy_rejected_where_unsupported(torch_cuda, d6):
    import torch
    t = plo.Tree(d6)
    rays = torch.from_numpy(plogen.rays_sphere(64, seed=34)).cuda()
    sp = plo.RenderParams(sphere=(0.5, 0.5, 0.5, 0.4))
    with pytest.raises(plo.PloError) as ei:
        plo.trace(t, rays, 16, sp)
    assert ei.value.status == -7
    with pytest.raises(plo.PloError) as ei:
        plo.Batch([t], [0, 64], sp)
    assert ei.value.status == -7
    for bad in ((0.5, 0.5, 0.5, 0.0), (0.5, float("nan"), 0.5, 0.3)):
        with pytest.raises(plo.PloError) as ei:
            plo.render(t, rays, plo.RenderParams(sphere=bad))
        assert ei.value.status == -1
