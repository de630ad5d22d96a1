#!/usr/bin/env python
"""Throughput of the plenoctree luminaire render on GB300.

Workload (the at-scale configuration): a procedural luminaire octree of max
depth 10 (1024^3 finest cells, ~32M leaves, SH degree 3 = 16 coefficients x
RGB + sigma, 196 B per FP32 leaf) and a wavefront of 16,777,216 rays with
origins uniform in a 10 x 10 x 3 room and cosine-weighted directions, kept
only when they meet the luminaire's proxy box.  One step renders the whole
wavefront (proxy clip, octree walk, SH emission, compositing) with one
persistent kernel launch; inputs are resident in HBM and larger than L2.

Prints one JSON line (rank 0).  `value` is Mrays/s with FP32 leaves; the
`fp16` / `bf16` objects time the same rays with 16-bit leaves.
`--impl reference` times the FP64 CPU oracle on the host cores instead.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import re
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "Mrays/s plenoctree render (FP32 vs FP16 leaves) and % of HBM roofline"
UNIT = "Mrays/s"
FALLBACK_HBM_GBS = 6800.0


def parse_args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--rays", type=int, default=1 << 24)
    ap.add_argument("--depth", type=int, default=10)
    ap.add_argument("--cpu-sample", type=int, default=1 << 20, help="rays in the oracle's timed sample")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-batch", action="store_true", help="skip the 8-luminaire batched-render section")
    ap.add_argument("--no-pt", action="store_true", help="skip the path-tracer emitter timing")
    ap.add_argument("--no-variants", action="store_true",
                    help="skip the linear / sigma_min-alpha_max / sphere-proxy timings")
    ap.add_argument("--no-train", action="store_true", help="skip the training-step timing")
    ap.add_argument("--no-octopt", action="store_true", help="skip the direct leaf optimisation section")
    ap.add_argument("--octopt-fit-steps", type=int, default=1000)
    ap.add_argument("--no-distill", action="store_true",
                    help="skip the trained network's depth-10 distillation and its error")
    ap.add_argument("--distill-train-steps", type=int, default=2000)
    ap.add_argument("--train-timed-steps", type=int, default=60)
    ap.add_argument("--layout", choices=["octree", "bricks4", "bricks8"], default="octree",
                    help="device layout of the timed trees (plo_build_tree_ex)")
    ap.add_argument("--no-layouts", action="store_true",
                    help="skip the device-layout comparison (octree vs bricks of 4^3 and 8^3 cells)")
    ap.add_argument("--learned", action="store_true",
                    help="run the learned-part experiment (train, distill, error vs ground truth) instead")
    ap.add_argument("--train-steps", type=int, default=3000)
    ap.add_argument("--distill-depth", type=int, default=10)
    ap.add_argument("--no-hier", action="store_true", help="--learned: skip the coarse/fine arm")
    return ap.parse_args()


def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def max_over_ranks(x: float, dist, device) -> float:
    """The largest of every rank's value (the job's time is its slowest
    rank's); x itself without a process group."""
    if dist is None:
        return x
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(world: int, rays_per_rank: int, steps: int, seconds: float) -> float:
    """Whole-job Mrays/s: every rank renders its own rays_per_rank per step
    (weak scaling), over the slowest rank's time."""
    return world * rays_per_rank * steps / seconds / 1e6


def shard_seed(rank: int) -> int:
    """Seed of rank's rays: each rank renders a shard of its own."""
    return 11 + rank


def workload(depth: int, n_rays: int, seed: int):
    import plogen
    rec = plogen.LUMINAIRE_D10.with_(depth=depth)
    t0 = time.time()
    tree = plogen.luminaire_tree(rec)
    rays = plogen.rays_room(n_rays, seed=seed)
    return rec, tree, rays, time.time() - t0


class ClockSampler:
    """nvidia-smi clock / throttle-reason samples while the timed regions run."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        self.dev = device_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                                          "-lms", "200", "-i", str(self.dev)], stdout=subprocess.PIPE,
                                         stderr=subprocess.DEVNULL, text=True)
            self.reader = threading.Thread(target=self._read, daemon=True)
            self.reader.start()
        except (OSError, FileNotFoundError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"], "samples": 0}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.reader.join(timeout=2)
        sm, smax, power, reasons = [], [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
                power.append(float(parts[3]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "power_w_max": max(power) if power else None, "reasons": sorted(reasons), "samples": len(sm)}


def measured_peak():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(p) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return FALLBACK_HBM_GBS, "fallback"


def kernel_source_hash() -> str:
    """Hash of the render kernel's code (comments and whitespace left out,
    so that a comment edit keeps a capture taken on the same code)."""
    h = hashlib.sha256()
    for fn in ("render.cu", "tree.cu", "plo_internal.h"):
        with open(os.path.join(ROOT, "paper_2207_05009_gb300", "csrc", fn)) as f:
            src = f.read()
        src = re.sub(r"/\*.*?\*/", " ", src, flags=re.S)
        src = re.sub(r"//[^\n]*", " ", src)
        h.update(" ".join(src.split()).encode())
    return h.hexdigest()[:16]


def ncu_traffic(precision: str):
    """DRAM bytes per launch from the committed ncu summary, if it was taken
    on the current kernel source (else None)."""
    p = os.path.join(ROOT, "profiles", "render_d10_traffic.json")
    try:
        with open(p) as f:
            d = json.load(f)
    except (OSError, ValueError):
        return None
    if d.get("kernel_source_hash") != kernel_source_hash():
        return None
    return d.get("dram_bytes_per_launch", {}).get(precision)


def rel_errors(rgb, T, ref):
    scale = np.maximum(ref["bound"], 1e-30)
    e_c = np.abs(np.asarray(rgb, np.float64) - ref["rgb"]) / scale
    e_c[(ref["bound"] == 0) & (np.asarray(rgb) == 0)] = 0.0
    e_T = np.abs(np.asarray(T, np.float64) - ref["T"]) / np.maximum(ref["T"], 1e-3)
    return float(e_c.max()), float(e_T.max())


def batch_workload(seed: int = 4242, total: int = 12_000_000):
    """8 luminaires of depth 7-10 with SH degree 2 or 3 and ray counts drawn
    log-uniform in [1e3, 4e6], rescaled to ~12M in all (clamped to the range)."""
    import plogen
    rng = np.random.default_rng(seed)
    draws = np.exp(rng.uniform(np.log(1e3), np.log(4e6), 8))
    # rescale to the total, clamping to the range; repeat so that the clamped
    # entries' excess goes to the others (water-filling)
    counts = draws.copy()
    for _ in range(20):
        free = (counts > 1e3) & (counts < 4e6)
        fixed = counts[~free].sum()
        if free.any():
            counts[free] *= (total - fixed) / counts[free].sum()
        counts = np.clip(counts, 1e3, 4e6)
    counts = np.round(counts).astype(np.int64)
    recs = [plogen.LUMINAIRE_D10.with_(depth=d, sh_degree=2 + (i % 2), seed=1000 + i)
            for i, d in enumerate([7, 8, 9, 10, 7, 8, 9, 10])]
    return recs, counts


def run_batch(args, plo, torch, W, K):
    """Batched render of the 8-luminaire workload: one graph-replayed
    persistent launch (autotuned launch shape) vs 8 separate launches."""
    import plogen
    recs, counts = batch_workload()
    trees, rays = [], []
    for i, (rec, c) in enumerate(zip(recs, counts)):
        trees.append(plo.Tree(plogen.luminaire_tree(rec), plo.PREC_FP32))
        rays.append(plogen.rays_room(int(c), seed=300 + i))
    offs = np.concatenate([[0], np.cumsum(counts)])
    n = int(offs[-1])
    d_rays = torch.from_numpy(np.concatenate(rays)).cuda()
    rgb = torch.empty((n, 3), device="cuda")
    T = torch.empty(n, device="cuda")
    batch = plo.Batch(trees, offs)
    cfg, src = plo.autotune_cached(batch, f"batch8-{n}", d_rays, rgb, T)
    batch.capture(d_rays, rgb, T)
    stream = torch.cuda.current_stream()

    def time_it(fn):
        for _ in range(W):
            fn()
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(K):
            fn()
        b.record(stream)
        torch.cuda.synchronize()
        return a.elapsed_time(b) / K

    def separate():
        for t, (lo, hi) in zip(trees, zip(offs[:-1], offs[1:])):
            plo.render(t, d_rays[lo:hi], rgb=rgb[lo:hi], T=T[lo:hi])

    ms_batch = time_it(batch.replay)
    ref_rgb = rgb.clone()
    ms_sep = time_it(separate)
    same = bool(torch.equal(rgb, ref_rgb))
    for t in trees:
        t.check()
    return {"workload": "8 luminaires, depth 7-10, SH degree 2/3, ray counts log-uniform 1e3-4e6 rescaled to ~12M",
            "rays": n, "ray_counts": [int(c) for c in counts],
            "leaves": [int(t.info()["n_leaves"]) for t in trees],
            "persistent_graph": {"value": n / ms_batch / 1e3, "unit": UNIT, "ms_per_step": ms_batch,
                                 "launches_per_step": 1},
            "separate_launches": {"value": n / ms_sep / 1e3, "unit": UNIT, "ms_per_step": ms_sep,
                                  "launches_per_step": len(trees)},
            "speedup": ms_sep / ms_batch, "bitwise_equal": same, "config": cfg, "config_source": src}


def run_variants(plo, torch, tree32, rays, rgb, T, timed, rays_total):
    """Speed and error of the paper's render options on the same rays (FP32
    leaves): the linear transmittance model (Sec. 6.2 "Transmittance model"),
    the sigma_min = 0.1 / alpha_max = 0.9 heuristics (Sec. 6.2 "Performance vs
    Quality") and a sphere proxy around the luminaire (Sec. 5).  Errors are
    against the exact render with the box proxy and the same transmittance."""
    def outputs(params):
        plo.render(tree32, rays, params, rgb=rgb, T=T)
        return rgb.clone(), T.clone()

    def err(a, b):
        (c, t), (c0, t0) = a, b
        d = (c - c0).double()
        return {"rel_l2_radiance": float(d.norm() / c0.double().norm().clamp_min(1e-300)),
                "alpha_rmse": float((t - t0).double().pow(2).mean().sqrt()),
                "max_abs_alpha": float((t - t0).abs().max())}

    P = plo.RenderParams
    cases = {"exp": P(), "linear": P(transmittance=plo.TRANS_LINEAR),
             "exp_heuristics": P.paper_heuristics(),
             "linear_heuristics": P.paper_heuristics(transmittance=plo.TRANS_LINEAR),
             "exp_sphere_r0.5": P(sphere=(0.5, 0.5, 0.5, 0.5)),
             "exp_tstop_1e-4": P(t_stop=1e-4)}
    exact = {"exp": outputs(cases["exp"]), "linear": outputs(cases["linear"])}
    out = {}
    for name, p in cases.items():
        total, per_launch = timed(tree32, p)
        base = "linear" if p.transmittance == plo.TRANS_LINEAR else "exp"
        out[name] = {"value": rays_total / (total / 1e3) / 1e6, "unit": UNIT, "kernel_ms": per_launch,
                     "error_vs_exact": err(outputs(p), exact[base])}
    out["linear_speedup_vs_exp"] = out["linear"]["value"] / out["exp"]["value"]
    out["heuristics_speedup_exp"] = out["exp_heuristics"]["value"] / out["exp"]["value"]
    return out


def run_sh_degrees(plo, torch, depth, rays, rgb, T, timed, rays_total):
    """Render speed against the SH degree (Sec. 6.2's comparison of l_max 2,
    3 and 4): the same luminaire geometry and leaf densities with l_max = 2,
    3, 4 (9, 16, 25 coefficients per channel), FP32 leaves, the same rays."""
    import plogen
    out = {}
    for deg in (2, 3, 4):
        t = plo.Tree(plogen.luminaire_tree(plogen.LUMINAIRE_D10.with_(depth=depth, sh_degree=deg)))
        total, per_launch = timed(t)
        out[f"l_max_{deg}"] = {"value": rays_total / (total / 1e3) / 1e6, "unit": UNIT, "kernel_ms": per_launch,
                               "record_bytes_fp32": int(t.info()["sh_record_stride"])}
        t.free()
    out["l_max_4_vs_2"] = out["l_max_4"]["value"] / out["l_max_2"]["value"]
    return out


def run_pt(plo, torch, tree32, W, K):
    """The luminaire as an emitter in a path tracer (Sec. 3 Eq. 2, Sec. 5):
    paths per second with the octree luminaire, and with an opaque box of
    constant radiance in its place (the explicitly handled emitter); the
    overhead per sample is their time ratio minus one (Sec. 6.2 quotes 20%
    for its Mitsuba integration against the luminaires' real geometry)."""
    sc = dict(room_min=(-1.0, -1.0, -1.0), room_max=(2.0, 2.0, 2.0), albedo=[(0.6, 0.6, 0.6)] * 6,
              cam_pos=(0.5, 0.4, -0.9), cam_target=(0.5, 0.5, 0.5), cam_up=(0.0, 1.0, 0.0), fov_y=1.2, width=512,
              height=512, max_bounces=3, emitter=plo.PT_OCTREE, box_radiance=(1.0, 1.0, 1.0))
    spp = 4
    stream = torch.cuda.current_stream()
    out = {"scene": "room [-1,2]^3, diffuse walls (albedo 0.6), the depth-10 luminaire in [0,1]^3; "
                    f"{sc['width']}x{sc['height']} pixels, {spp} samples, {sc['max_bounces']} bounces, "
                    "2 luminaire queries per bounce"}
    for name, emitter in (("octree", plo.PT_OCTREE), ("constant_box", plo.PT_CONSTANT_BOX)):
        sc["emitter"] = emitter
        for _ in range(W):
            plo.pt_render(tree32, sc, spp, seed=1)
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for k in range(K):
            plo.pt_render(tree32, sc, spp, seed=2 + k)
        b.record(stream)
        torch.cuda.synchronize()
        ms = a.elapsed_time(b) / K
        paths = sc["width"] * sc["height"] * spp
        out[name] = {"ms_per_frame": ms, "paths_per_s": paths / (ms / 1e3),
                     "luminaire_queries_per_s": 2 * sc["max_bounces"] * paths / (ms / 1e3)}
    out["overhead_per_sample"] = out["octree"]["ms_per_frame"] / out["constant_box"]["ms_per_frame"] - 1.0
    return out


def measured_tflops():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(p) as f:
            d = json.load(f)
        return float(d["bf16_tflops_sustained"]), float(d["bf16_tflops"]), "measured"
    except (OSError, KeyError, ValueError):
        return 1700.0, 1900.0, "fallback"


def run_train(plo, torch, steps: int, W: int):
    """The training step of the learned part (Sec. 4.4): 4096 rays x 128
    samples per step on targets rendered from the depth-6 luminaire by the
    plain renderer, the paper's loss, linear-head network; `steps` timed
    steps after W warm-up steps (CUDA events), plus the tensor-core layers
    alone on the same shapes (524,288 rows): forward 256 -> 256 with the
    ReLU bits, data gradient through the mask, weight gradient with the bias
    sums."""
    import plogen
    from paper_2207_05009_gb300 import learned
    gt = plo.Tree(plogen.luminaire_tree(plogen.LUMINAIRE_D6))
    batches = learned.target_batches(gt, [plogen.rays_sphere(4096, seed=200 + k) for k in range(8)])
    l_max, c0 = learned.emission_scale(batches)
    net = plo.Mlp(l_max=l_max, total_steps=steps + W, init_radiance=c0)
    loss = torch.empty(1, device="cuda")
    stream = torch.cuda.current_stream()
    for k in range(W):
        rays, rgb, alpha = batches[k % 8]
        net.train_step(rays, rgb, alpha, n_samples=128, loss_out=loss)
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    for k in range(steps):
        rays, rgb, alpha = batches[k % 8]
        net.train_step(rays, rgb, alpha, n_samples=128, loss_out=loss)
    b.record(stream)
    torch.cuda.synchronize()
    net.check()
    ms = a.elapsed_time(b) / steps
    M = 4096 * 128
    trunk = 63 * 256 + 7 * 256 * 256
    flops = M * 2 * 3 * (trunk + 256 * 49)
    sustained, burst, src = measured_tflops()

    def time_op(fn, reps=10, batches=5):
        # median over batches of `reps` launches: one late launch (a clock
        # change, another process on the host) then moves no number
        for _ in range(2):
            fn()
        torch.cuda.synchronize()
        per = []
        for _ in range(batches):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for _ in range(reps):
                fn()
            e1.record(stream)
            torch.cuda.synchronize()
            per.append(e0.elapsed_time(e1) / reps)
        return float(np.median(per))

    g = torch.Generator(device="cuda").manual_seed(5)
    H = (torch.rand(M, 256, device="cuda", generator=g) - 0.3).to(torch.bfloat16)
    Wt = (torch.randn(256, 256, device="cuda", generator=g) * 0.06).to(torch.bfloat16)
    bias = torch.zeros(256, device="cuda")
    bits = torch.empty((M, 8), device="cuda", dtype=torch.int32)
    out = torch.empty((M, 256), device="cuda", dtype=torch.bfloat16)
    dW = torch.zeros(256, 256, device="cuda")
    db = torch.zeros(256, device="cuda")
    layer_flops = 2 * M * 256 * 256
    layers = {}
    for name, fn in (("forward_relu_bits", lambda: plo.gemm_bf16(H, Wt, 0, bias=bias, bits=bits, out=out)),
                     ("data_gradient_mask", lambda: plo.gemm_bf16(H, Wt, 3, bits=bits, out=out)),
                     ("weight_gradient_bias", lambda: plo.wgrad_bf16(H, H, dW, db=db))):
        t = time_op(fn)
        layers[name] = {"ms": t, "tflops": layer_flops / (t / 1e3) / 1e12}
    del H, out
    return {"workload": "4096 rays x 128 samples per step (524,288 network evaluations), paper loss, "
                        "8 x 256 trunk + linear head, targets from the depth-6 luminaire",
            "steps_timed": steps, "ms_per_step": ms, "tflops": flops / (ms / 1e3) / 1e12,
            "flops_per_step": flops, "peak_tflops_sustained": sustained,
            "frac_of_sustained": flops / (ms / 1e3) / 1e12 / sustained, "peak_source": f"{src} (MEASURED_PEAKS.json)",
            "final_loss": float(loss.item()), "layer_256x256_M524288": layers}


def run_distill(plo, torch, steps: int):
    """The learned part's end product (Sec. 5): a network trained `steps`
    steps with the paper's loss on targets rendered from the depth-6
    luminaire, distilled into a depth-10 octree (1024^3 voxel centres, 8
    jittered samples per kept voxel, sigma >= 0.01) on the device, and the
    distilled octree's render error against the ground-truth renders on
    65,536 test rays; depth 8 beside it, with 8 and with the paper's 256
    samples per kept voxel."""
    import plogen
    from paper_2207_05009_gb300 import learned
    gt = plo.Tree(plogen.luminaire_tree(plogen.LUMINAIRE_D6))
    train_b = learned.target_batches(gt, [plogen.rays_sphere(4096, seed=200 + k) for k in range(64)])
    test_b = learned.target_batches(gt, [plogen.rays_sphere(65536, seed=900)])
    l_max, _ = learned.emission_scale(train_b)
    net, losses, dt = learned.train(train_b, steps, plo.LOSS_PAPER, l_max=l_max)
    out = {"workload": f"paper loss, {steps} steps of 4096 rays x 128 samples on the depth-6 luminaire's "
                       "renders; distilled with 8 samples per kept voxel (depth 8 also with the paper's 256), "
                       "sigma >= 0.01; error on 65,536 test rays",
           "train_s": dt, "final_loss": float(np.mean(losses[-32:]))}
    for depth, samples in ((8, 8), (8, 256), (10, 8)):
        e = learned.distilled_error(net, l_max, test_b, depth=depth, samples=samples)
        d = e.__dict__
        d["samples_per_voxel"] = samples
        d["network_samples_per_s"] = e.leaves * samples / max(e.distill_s, 1e-9)
        out[f"depth{depth}" + ("" if samples == 8 else f"_samples{samples}")] = d
    del net
    torch.cuda.empty_cache()
    return out


def full_octree_child(depth: int) -> np.ndarray:
    """Canonical child table of the complete octree of `depth` levels
    (breadth-first node ids; the 8^depth leaves numbered in the order of
    their parents)."""
    rows = []
    for lev in range(depth):
        k = np.arange(8 ** lev, dtype=np.int64)[:, None] * 8 + np.arange(8)
        if lev + 1 < depth:
            rows.append((8 ** (lev + 1) - 1) // 7 + k)  # the next level's node ids
        else:
            rows.append(-k - 2)  # leaves
    return np.concatenate(rows).astype(np.int32)


def fit_octopt(plo, torch, init, l_max, batches, test_b, steps: int, W: int, total: int, **cfg):
    """Timed steps and a fit of the direct leaf optimisation; returns the
    step time and the packed result's error on the test rays."""
    from paper_2207_05009_gb300 import learned
    n = batches[0][0].shape[0]
    opt = plo.OctOpt(init, l_max, max_rays=n, total_steps=total, **cfg)
    loss = torch.empty(3, device="cuda")
    stream = torch.cuda.current_stream()
    first = None
    for k in range(W):
        opt.step(*batches[k % len(batches)], loss_out=loss)
        if first is None:
            first = float(loss[0].item())
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    for k in range(steps):
        opt.step(*batches[(W + k) % len(batches)], loss_out=loss)
    b.record(stream)
    torch.cuda.synchronize()
    opt.check()
    ms = a.elapsed_time(b) / steps
    for k in range(W + steps, total):
        opt.step(*batches[k % len(batches)], loss_out=loss)
    torch.cuda.synchronize()
    opt.check()
    fit = opt.build_tree()
    rel, psnr, a_rmse = learned.tree_error(fit, l_max, test_b)
    fit.free()
    opt.free()
    torch.cuda.empty_cache()
    return {"leaves": int(init.n_leaves), "rays_per_step": n, "steps_timed": steps, "ms_per_step": ms,
            "mrays_per_s": n / (ms / 1e3) / 1e6, "fit_steps": total, "first_loss": first,
            "final_loss": float(loss[0].item()), "error": {"rel_l2_radiance": rel, "psnr": psnr, "alpha_rmse": a_rmse}}


def run_octopt(plo, torch, steps: int, W: int, fit_steps: int):
    """Direct optimisation of the octree's leaves (Sec. 7's alternative to
    the network), fitted with the paper's loss, small TV weights and Adam to
    the plain renderer's images of the depth-8 luminaire (the network's
    targets), 65,536 rays per step, every leaf starting at sigma = 1 with
    the DC coefficient of the mean emission (the network's starting level):
    on the luminaire's own structure (497,856 leaves, SH degree 3), and on
    the complete depth-7 octree (2,097,152 leaves), which knows nothing of
    it.  `steps` timed steps after W warm-up steps (CUDA events); then each
    fit continues to `fit_steps` steps and the packed result is scored on
    65,536 test rays like the distilled network."""
    import plogen
    from paper_2207_05009_gb300 import learned
    gt_host = plogen.luminaire_tree(plogen.LUMINAIRE_D10.with_(depth=8))
    gt = plo.Tree(gt_host)
    n = 65536
    batches = learned.target_batches(gt, [plogen.rays_sphere(n, seed=300 + k) for k in range(16)])
    test_b = learned.target_batches(gt, [plogen.rays_sphere(n, seed=900)])
    gt.free()
    l_max, c0 = learned.emission_scale(batches)
    u = min(max(c0 / l_max, 1e-6), 1 - 1e-6)
    dc = np.log(u / (1 - u)) / 0.28209479177387814  # emission c0 in every direction
    total = max(fit_steps, steps + W)
    cfg = dict(lr_sigma=5.0, lr_sh=0.1, lr_decay=0.1, tv_sigma=1e-4, tv_sh=1e-5)
    out = {"workload": "the depth-8 luminaire's images (the network's targets) fitted from sigma = 1 and the mean "
                       "emission; paper loss, TV 1e-4 / 1e-5, Adam (5.0 / 0.1 decaying to a tenth); 65,536 rays per "
                       "step; SH degree 3"}
    for name, depth, child, nl in (("luminaire_structure", gt_host.depth, gt_host.child, gt_host.n_leaves),
                                   ("complete_depth7", 7, full_octree_child(7), 8 ** 7)):
        sh0 = np.zeros((nl, 3, gt_host.K), np.float32)
        sh0[:, :, 0] = dc
        init = plogen.HostTree(depth, gt_host.sh_degree, child, np.ones(nl, np.float32), sh0)
        out[name] = fit_octopt(plo, torch, init, l_max, batches, test_b, steps, W, total, **cfg)
    # the headline fields: the luminaire-structure fit
    for k in ("ms_per_step", "mrays_per_s", "first_loss", "final_loss", "error", "fit_steps", "rays_per_step",
              "steps_timed"):
        out[k] = out["luminaire_structure"][k]
    return out


def run_learned(args):
    """Train the NeRF-SH network on targets rendered from the depth-6
    luminaire (4096 rays x 128 samples per step, the paper's loss), distil it
    into an octree, and state the distilled octree's error against the ground
    truth next to the untrained network's, an MSE-trained network's, and the
    paper's full setup (coarse/fine networks with the 128-wide SH layer,
    64 + 128 samples, distilled from the fine network)."""
    import torch
    import paper_2207_05009_gb300 as plo
    import plogen
    from paper_2207_05009_gb300 import learned
    torch.cuda.set_device(0)
    gt = plo.Tree(plogen.luminaire_tree(plogen.LUMINAIRE_D6))
    train_b = learned.target_batches(gt, [plogen.rays_sphere(4096, seed=200 + k) for k in range(64)])
    test_b = learned.target_batches(gt, [plogen.rays_sphere(65536, seed=900)])
    l_max, c0 = learned.emission_scale(train_b)
    out = {"metric": "learned luminaire: distilled octree error vs ground truth", "data": "synthetic",
           "config": {"workload": "depth-6 luminaire targets, 4096 rays x 128 samples per step",
                      "train_steps": args.train_steps, "distill_depth": args.distill_depth, "l_max": l_max}}
    trunk = 63 * 256 + 7 * 256 * 256
    flops_step = 4096 * 128 * 2 * 3 * (trunk + 256 * 49)
    # coarse (64 samples) + fine (64 + 128 samples) with the 128-wide SH layer
    flops_hier = 4096 * (64 + 192) * 2 * 3 * (trunk + 256 + 256 * 128 + 128 * 48)
    arms = [("paper_loss", plo.LOSS_PAPER, args.train_steps), ("mse_loss", plo.LOSS_MSE, args.train_steps),
            ("untrained", plo.LOSS_PAPER, 0)]
    if not args.no_hier:
        arms.insert(1, ("paper_setup_coarse_fine", "hier", args.train_steps))
    for name, loss, steps in arms:
        if loss == "hier":
            coarse, net, losses, dt = learned.train_hier(train_b, steps, l_max=l_max)
            del coarse
            fl = flops_hier
        else:
            net, losses, dt = learned.train(train_b, steps, loss, l_max=l_max)
            fl = flops_step
        res = {"train_s": dt, "ms_per_step": dt / max(steps, 1) * 1e3,
               "tflops": fl * steps / max(dt, 1e-9) / 1e12 if steps else None,
               "final_loss": float(np.mean(losses[-32:])) if steps else None}
        e7 = learned.distilled_error(net, l_max, test_b, depth=7)
        res["depth7"] = e7.__dict__
        # the deepest distillation whose leaf count (predicted from depth 7,
        # 8x per level) fits comfortably in device memory: <= 400M leaves
        frac = e7.leaves / 8 ** 7
        depth = args.distill_depth
        while depth > 7 and frac * 8 ** depth > 400e6:
            depth -= 1
        if depth > 7:
            res[f"depth{depth}"] = learned.distilled_error(net, l_max, test_b, depth=depth).__dict__
        if depth < args.distill_depth:
            res["note"] = (f"depth {args.distill_depth} skipped: {frac:.1%} of depth-7 voxels are kept, "
                           f"~{frac * 8 ** args.distill_depth / 1e6:.0f}M leaves")
        out[name] = res
        del net
        torch.cuda.empty_cache()
    print(json.dumps(out), flush=True)
    return 0


def run_reference(args, world, rank):
    """FP64 oracle on the host cores, on bounded samples of the workload."""
    if rank != 0:
        return 0
    import oracle
    rec, tree, rays, gen_s = workload(args.depth, args.rays, seed=shard_seed(0))
    cores = len(os.sched_getaffinity(0))
    per_step = min(args.cpu_sample // 4 if args.cpu_sample >= 4 else 1, len(rays))
    for w in range(args.warmup):
        oracle.render(tree, rays[(w * 997) % max(1, len(rays) - 4096):][:4096], n_threads=cores)
    t0 = time.perf_counter()
    done = 0
    for k in range(args.steps):
        off = (k * per_step) % max(1, len(rays) - per_step + 1)
        oracle.render(tree, rays[off:off + per_step], n_threads=cores)
        done += per_step
    dt = time.perf_counter() - t0
    v = done / dt / 1e6
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": f"luminaire octree depth {args.depth}, SH degree 3, {args.rays} room rays",
                       "rays_per_step_sampled": per_step, "leaves": int(tree.n_leaves)},
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": f"{per_step} rays of the {args.rays}-ray wavefront per step"},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def main():
    args = parse_args()
    world, rank, local = dist_env()
    if args.learned:
        return run_learned(args) if rank == 0 else 0
    if args.impl == "reference":
        return run_reference(args, world, rank)

    import torch
    import paper_2207_05009_gb300 as plo

    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    K, W = args.steps, args.warmup
    assert W >= 3, "at least 3 warm-up steps"

    rec, tree, rays_np, gen_s = workload(args.depth, args.rays, seed=shard_seed(rank))
    n = len(rays_np)
    stream = torch.cuda.current_stream()
    t0 = time.time()
    lay = {"octree": (plo.LAYOUT_OCTREE, 0), "bricks4": (plo.LAYOUT_BRICKS, 2),
           "bricks8": (plo.LAYOUT_BRICKS, 3)}[args.layout]
    trees = {"fp32": plo.Tree(tree, plo.PREC_FP32, *lay), "fp16": plo.Tree(tree, plo.PREC_FP16, *lay),
             "bf16": plo.Tree(tree, plo.PREC_BF16, *lay)}
    build_s = time.time() - t0
    rays = torch.from_numpy(rays_np).cuda()
    rgb = torch.empty((n, 3), device="cuda")
    T = torch.empty(n, device="cuda")
    params = plo.RenderParams()

    def barrier():
        torch.cuda.synchronize()
        if dist is not None:
            dist.barrier()

    def timed(tr, params=params):
        for _ in range(W):
            plo.render(tr, rays, params, rgb=rgb, T=T)
        barrier()
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(K)]
        start, end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        start.record(stream)
        for a, b in evs:
            a.record(stream)
            plo.render(tr, rays, params, rgb=rgb, T=T)
            b.record(stream)
        end.record(stream)
        barrier()
        total = start.elapsed_time(end)
        per_launch = [a.elapsed_time(b) for a, b in evs]
        tr.check()
        total = max_over_ranks(total, dist, "cuda")
        return total, sum(per_launch) / len(per_launch)

    sampler = ClockSampler(torch.cuda.current_device())
    sampler.start()
    res = {}
    for name in ("fp32", "fp16", "bf16"):
        res[name] = timed(trees[name])
    layouts = None
    if not args.no_layouts:
        # the same rays on the other device layouts (plo_build_tree_ex), FP32
        # and FP16 leaves; the default layout's numbers are the lines above
        layouts = {}
        for lname, lay, blog in (("octree", plo.LAYOUT_OCTREE, 0), ("bricks4", plo.LAYOUT_BRICKS, 2),
                                 ("bricks8", plo.LAYOUT_BRICKS, 3)):
            layouts[lname] = {}
            for pname, prec in (("fp32", plo.PREC_FP32), ("fp16", plo.PREC_FP16)):
                tr = plo.Tree(tree, prec, lay, blog)
                total, per_launch = timed(tr)
                inf = tr.info()
                layouts[lname][pname] = {"value": job_rate(world, n, K, total / 1e3), "kernel_ms": per_launch,
                                         "structure_bytes": int(inf["node_bytes"] if lay == plo.LAYOUT_OCTREE
                                                                else inf["brick_bytes"] + 64 * inf["top_nodes"])}
                tr.free()
            layouts[lname]["fp16_speedup_vs_fp32"] = layouts[lname]["fp16"]["value"] / layouts[lname]["fp32"]["value"]
    variants = None if args.no_variants else run_variants(plo, torch, trees["fp32"], rays, rgb, T, timed,
                                                          world * n * K)
    pt = None if args.no_pt else run_pt(plo, torch, trees["fp32"], W, K)
    sh_degrees = None if args.no_variants else run_sh_degrees(plo, torch, args.depth, rays, rgb, T, timed,
                                                              world * n * K)
    train = None if args.no_train else run_train(plo, torch, args.train_timed_steps, W)
    distill = None if args.no_distill else run_distill(plo, torch, args.distill_train_steps)
    octopt = None if args.no_octopt else run_octopt(plo, torch, 20, W, args.octopt_fit_steps)
    e2e = None
    if not args.no_e2e:
        rays_h = torch.from_numpy(rays_np).pin_memory()
        rgb_h = torch.empty((n, 3), dtype=torch.float32).pin_memory()
        T_h = torch.empty(n, dtype=torch.float32).pin_memory()
        for _ in range(W):
            plo.render_host(trees["fp32"], rays_h, params, rgb=rgb_h, T=T_h)
        barrier()
        t1 = time.perf_counter()
        for _ in range(K):
            plo.render_host(trees["fp32"], rays_h, params, rgb=rgb_h, T=T_h)
        barrier()
        e2e_s = max_over_ranks(time.perf_counter() - t1, dist, "cuda")
        e2e = {"value": job_rate(world, n, K, e2e_s), "unit": UNIT, "h2d_bytes_per_step": n * 24,
               "d2h_bytes_per_step": n * 16, "ms_per_step": e2e_s / K * 1e3}
    batch = None
    if not args.no_batch:
        batch = run_batch(args, plo, torch, W, K)
    clocks = sampler.stop()

    # FP32 outputs of the last timed pass, for the parity spot check below
    plo.render(trees["fp32"], rays, params, rgb=rgb, T=T)
    out32 = (rgb[: args.cpu_sample].cpu().numpy(), T[: args.cpu_sample].cpu().numpy())
    plo.render(trees["fp16"], rays, params, rgb=rgb, T=T)
    out16 = (rgb[: args.cpu_sample].cpu().numpy(), T[: args.cpu_sample].cpu().numpy())
    plo.render(trees["bf16"], rays, params, rgb=rgb, T=T)
    outb16 = (rgb[: args.cpu_sample].cpu().numpy(), T[: args.cpu_sample].cpu().numpy())
    torch.cuda.synchronize()

    if rank != 0:
        if dist is not None:
            dist.barrier()
            dist.destroy_process_group()
        return 0

    # FP64 oracle on a bounded sample: CPU baseline, per-ray algorithmic
    # bytes, and a parity spot check of the timed launch configuration.
    cpu = None
    K16 = tree.K
    sample = min(args.cpu_sample, n)
    if not args.no_cpu:
        import oracle
        cores = len(os.sched_getaffinity(0))
        tc = time.perf_counter()
        ref = oracle.render(tree, rays_np[:sample], n_threads=cores)
        cpu_s = time.perf_counter() - tc
        cpu = {"value": sample / cpu_s / 1e6, "unit": UNIT, "cores": cores, "kind": "oracle",
               "sample": f"first {sample} rays of the {n}-ray wavefront ({cpu_s:.1f} s)"}
        # the same oracle on one thread, and on the 65,536-ray depth-6 set
        one = min(sample, 1 << 14)
        tc = time.perf_counter()
        oracle.render(tree, rays_np[:one], n_threads=1)
        cpu["one_thread"] = {"value": one / (time.perf_counter() - tc) / 1e6, "unit": UNIT, "cores": 1,
                             "sample": f"first {one} rays of the wavefront"}
        import plogen
        tree6, rays6 = plogen.luminaire_tree(plogen.LUMINAIRE_D6), plogen.rays_sphere(65536, seed=1)
        tc = time.perf_counter()
        oracle.render(tree6, rays6, n_threads=cores)
        cpu["depth6_65536_rays"] = {"value": 65536 / (time.perf_counter() - tc) / 1e6, "unit": UNIT,
                                    "cores": cores, "sample": "all 65,536 rays of the depth-6 (SH degree 2) set"}
        leaf_visits = float(ref["n_leaf"].mean())
        sh_visits = float(ref["n_sh"].mean())
        cells = float(ref["n_cell"].mean())
        # [radiance, T] max errors against the FP64 oracle on FP32 leaves
        parity = {"sample_rays": sample, "fp32_max_rel_err": rel_errors(*out32, ref),
                  "fp16_max_rel_err": rel_errors(*out16, ref),
                  "bf16_max_rel_err": rel_errors(*outb16, ref),
                  "metric": "[radiance, T]: |g - o| / sum_i w_i sum_k |c_k Y_k| per channel, "
                            "|T_g - T_o| / max(T_o, 1e-3)"}
    else:
        leaf_visits = sh_visits = cells = float("nan")
        parity = None

    peak, peak_kind = measured_peak()
    bytes_ray = {"fp32": 40 + 4 * leaf_visits + 12 * K16 * sh_visits,
                 "fp16": 40 + 4 * leaf_visits + (6 * K16 + 4) * sh_visits}
    bytes_ray["bf16"] = bytes_ray["fp16"]
    lines = {}
    for name, (total, per_launch) in res.items():
        mrays = job_rate(world, n, K, total / 1e3)
        ach = bytes_ray[name] * n / (per_launch / 1e3) / 1e9
        traffic = ncu_traffic(name)
        lines[name] = {"value": mrays, "ms_per_step": total / K, "kernel_ms": per_launch,
                       "roofline": {"bound": "hbm", "achieved": ach, "peak": peak, "unit": "GB/s",
                                    "frac": ach / peak, "traffic": traffic,
                                    "peak_source": f"{peak_kind} copy bandwidth (MEASURED_PEAKS.json hbm_gbs)",
                                    "frac_of_8TBs": ach / 8000.0,
                                    "algorithmic_bytes_per_ray": bytes_ray[name]}}
    info = trees["fp32"].info()
    line = {
        "metric": METRIC, "value": lines["fp32"]["value"], "unit": UNIT, "n_gpus": world, "steps": K,
        "warmup": W, "ms_per_step": lines["fp32"]["ms_per_step"], "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": f"luminaire octree depth {args.depth} ({tree.n_leaves} leaves, SH degree 3, "
                               f"K=16), {n} room rays per GPU meeting the proxy box",
                   "rays_per_gpu": n, "leaves": int(tree.n_leaves), "nodes": int(tree.n_nodes),
                   "emissive_leaves": int(info["n_sh_records"]),
                   "tree_bytes_fp32": int(info["node_bytes"] + info["sh_bytes"]),
                   "l2": "inputs larger than L2 (tree and rays each exceed 129 MB); no flush",
                   "parallelism": f"replicas x{world} (rays shard, no collective)",
                   "mean_cells_per_ray": cells, "mean_leaf_visits_per_ray": leaf_visits,
                   "mean_sh_reads_per_ray": sh_visits, "host_setup_s": round(gen_s + build_s, 1)},
        "clocks": clocks,
        "e2e": e2e,
        # per render call of 2^23 rays or more: the ray-order count, a
        # three-launch scan of its (bin, block) table, the positions, the
        # rays in order, k_render, the outputs back in ray order
        "gpu_launches": K * (8 if n >= (1 << 23) else 1),
        "roofline": lines["fp32"]["roofline"],
        "cpu_baseline": cpu,
        "fp16": {k: v for k, v in lines["fp16"].items()},
        "bf16": {k: v for k, v in lines["bf16"].items()},
        "fp16_speedup_vs_fp32": lines["fp16"]["value"] / lines["fp32"]["value"],
        "layout": {"timed": args.layout,
                   "n_bricks": int(info["n_bricks"]), "brick_bytes": int(info["brick_bytes"]),
                   "compared": layouts},
        "parity": parity,
        "batch": batch,
        "variants": variants,
        "path_tracer": pt,
        "sh_degrees": sh_degrees,
        "train": train,
        "distill": distill,
        "octopt": octopt,
    }
    line["fp16"]["roofline"]["frac"] = line["fp16"]["roofline"]["achieved"] / peak
    print(json.dumps(line), flush=True)
    if dist is not None:
        dist.barrier()
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
