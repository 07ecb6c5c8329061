#!/usr/bin/env python
"""Benchmark of the multi-resolution sampling hot path on GB300.

One step = one hybrid frame of the 200k-triangle procedural scene:
  render-tree rebuild (Morton codes, radix sort, hierarchical clustering in one
  launch) -> LRHS render 256x256 @ 64 spp -> HRLS render 1024x1024 @ 4 spp
  (+ albedo / normal / depth) -> x4 fusion CNN in BF16 on tcgen05 -> fallback
  gate (box-downsampled fused vs LRHS, RelMSE threshold 0.01).  The same frame
  over the Karras LBVH (radix tree + refit) is reported beside it.
Max depth 8 with Russian roulette from bounce 3 for both renders.

Prints one JSON line.  `value` is device-timed ms per frame (inputs resident in
HBM, L2 flushed between steps); `e2e` times the same frame through the public
API with the geometry uploaded from pinned host memory and the fused image read
back every step.  `--impl reference` times the CPU oracle on a bounded sample.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "ms/frame at equal PSNR, hybrid vs plain HR path trace; Msamples/s; conv TFLOP/s"
WORKLOAD = {
    "workload": "hybrid frame: procedural 200,968-triangle scene (seed 0), render tree rebuilt "
                "every step; LRHS 256x256 @ 64 spp + "
                "HRLS 1024x1024 @ 4 spp (albedo/normal/depth), max depth 8, roulette from bounce 3; "
                "x4 fusion CNN (12->64, 8 residual blocks, 64->3) in BF16 on tcgen05; fallback gate; "
                "the two renders run concurrently on two streams",
    "tree": "hierarchical clustering in one launch over the Morton-sorted triangles (the images "
            "are those of the LBVH bit for bit)",
    "scene_seed": 0, "lrhs": [256, 256, 64], "hrls": [1024, 1024, 4], "scale": 4,
    "max_depth": 8, "rr_start": 3, "precision": "bf16",
    "net_init": "trained before the timed region by the training recipe (reduced: see "
                "`training`); the seeded initialisation under --quick",
    "l2": "flushed between steps (512 MiB write)",
}
LR, HR, S = 256, 1024, 4
TREE = "hcluster"       # the frame's render tree (mrs_scene_set_tree)
SPP_LR, SPP_HR, DEPTH, RR = 64, 4, 8, 3
CONV_FLOP_PER_PX = 2 * 9 * (12 * 64 + 16 * 64 * 64 + 64 * 3)      # 1,196,928
# algorithmic HBM bytes per HR pixel of the 18 BF16 conv layers: input layer
# reads 12 channels (24 B) and writes 128 B; each residual block reads h,
# writes r, reads r and h, writes h (5 x 128 B); the head reads 128 B and
# writes 3 FP32 (12 B)
CONV_BYTES_PER_PX = (24 + 128) + 8 * 5 * 128 + (128 + 12)           # 5,412
# algorithmic FP32 work per traversal step: a node visit tests the ray against
# its two children's boxes (slab test, 12 FLOP per box), a triangle test is
# Moller-Trumbore (27 FLOP); the roofline peak counts an FMA as 2 FLOP
FLOP_PER_NODE_VISIT = 24
FLOP_PER_TRI_TEST = 27
# the kernel's own FP32 instruction count per step, from the source (pt.cu:
# slab() on both children, intersect() per triangle; built with --fmad=false),
# reported beside the algorithmic figure against the non-FMA issue rate
OPS_PER_NODE_VISIT = 52
OPS_PER_TRI_TEST = 50
# the BF16 training step's algorithmic FLOPs per HR pixel: forward, weight
# gradients of all 18 layers, input gradients of the 17 layers after the first
TRAIN_FLOP_PER_PX = 2 * CONV_FLOP_PER_PX + (CONV_FLOP_PER_PX - 2 * 9 * 12 * 64)


def _peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        d["source"] = "measured"
        return d
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0,
            "sm_max_mhz": 2070.0, "source": "fallback"}


class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled every 100 ms."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.rows = []
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append([x.strip() for x in line.split(",")])

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        if not self.rows:
            return None
        mhz = [float(r[1]) for r in self.rows if len(r) > 2 and r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in self.rows if len(r) > 2 and r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in self.rows for i in range(4)
                          if len(r) > 5 + i and r[5 + i].lower() == "active"})
        return {"sm_mhz": float(np.median(mhz)) if mhz else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons,
                "samples": len(self.rows)}


def _traffic(kernel, src):
    """The committed ncu DRAM-traffic record of `kernel` (profiles/traffic.json:
    bytes of one captured launch and the work units it processed), if the
    kernel source is unchanged since the capture (else None)."""
    p = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(p):
        return None
    with open(p) as f:
        d = json.load(f).get(kernel)
    if not d:
        return None
    with open(os.path.join(ROOT, "paper_2106_12802_gb300", "csrc", src), "rb") as f:
        sha = hashlib.sha256(f.read()).hexdigest()[:16]
    return d if d.get("src_sha256_16") == sha else None


def max_over_ranks(value, world, device=None):
    """The maximum of a per-rank number over all ranks (the slowest rank's
    time); the value itself at world size 1.  The reduction runs on `device`
    under NCCL and on the host under gloo."""
    if world <= 1:
        return float(value)
    import torch
    import torch.distributed as dist
    dev = device if (device is not None and dist.get_backend() == "nccl") else torch.device("cpu")
    t = torch.tensor([float(value)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def l2_copy_gbs(megabytes=32, reps=20, trials=5):
    """L2 bandwidth reference: bytes read + written per second by a device
    copy between two L2-resident buffers of `megabytes` MB (median of
    `trials` event-timed batches of `reps` copies, after a warm-up)."""
    import torch
    n = megabytes * (1 << 20) // 4
    a = torch.ones(n, dtype=torch.float32, device="cuda")
    b = torch.empty_like(a)
    b.copy_(a)
    ts = []
    for _ in range(trials):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(reps):
            b.copy_(a)
        e1.record()
        e1.synchronize()
        ts.append(e0.elapsed_time(e1))
    ms = float(np.median(ts))
    return 2 * n * 4 * reps / (ms * 1e-3) / 1e9


# ----------------------------------------------------------------------------
# CPU oracle (bounded samples of the same frame)
# ----------------------------------------------------------------------------
def oracle_frame_sample(desc, params, k=0, lr_rows=8, hr_rows=16, cnn_rows=4):
    """Times the oracle on a bounded sample of the hybrid frame and scales each
    part to a whole frame: `lr_rows` LRHS rows and `hr_rows` HRLS rows spread
    evenly over the image (every (H / rows)-th row from an offset that moves
    with the sample index k, so that samples cover the whole image), and the
    FP64 network on a strip of `cnn_rows` output rows plus its receptive-field
    halo.  Returns (ms_per_frame, detail)."""
    import oracle
    from oracle import cnn
    oracle.build()
    t0 = time.perf_counter()
    oracle.lbvh(desc["V"])
    t_build = time.perf_counter() - t0
    st_lr, st_hr = LR // lr_rows, HR // hr_rows
    seed = k
    t0 = time.perf_counter()
    oracle.render(desc, LR, LR, SPP_LR, DEPTH, RR, seed, rows=((7 * k) % st_lr, LR, st_lr))
    t_lr = max(time.perf_counter() - t0 - t_build, 1e-9)
    t0 = time.perf_counter()
    oracle.render(desc, HR, HR, SPP_HR, DEPTH, RR, seed + 1, rows=((13 * k) % st_hr, HR, st_hr))
    t_hr = max(time.perf_counter() - t0 - t_build, 1e-9)
    rng = np.random.default_rng(0)
    halo = 18                      # receptive field of the 18 stacked 3x3 convs
    rows = cnn_rows + 2 * halo
    lr = rng.uniform(0, 2, (1, (rows + S - 1) // S, HR // S, 3))
    hr = rng.uniform(0, 2, (1, lr.shape[1] * S, HR, 3))
    t0 = time.perf_counter()
    cnn.forward(params, lr, hr, hr, hr, S)
    t_cnn = time.perf_counter() - t0
    ms = 1e3 * (2 * t_build + t_lr * LR / lr_rows + t_hr * HR / hr_rows + t_cnn * HR / hr.shape[1])
    detail = (f"LBVH build x2; every {st_lr}th LRHS row ({lr_rows}/{LR}) and every {st_hr}th "
              f"HRLS row ({hr_rows}/{HR}) rendered (scaled by rows); FP64 CNN on a "
              f"{hr.shape[1]}x{HR} strip (scaled by rows)")
    return ms, detail


def oracle_frame_estimate(desc, params, samples=3):
    """Mean of `samples` bounded oracle samples of one frame (rows at
    different offsets); returns (ms_per_frame, detail)."""
    ms, detail = [], ""
    t0 = time.perf_counter()
    for k in range(samples):
        m, detail = oracle_frame_sample(desc, params, k)
        ms.append(m)
    wall = time.perf_counter() - t0
    return float(np.mean(ms)), (detail + f"; mean of {samples} samples (rows at different "
                                f"offsets), {wall:.1f} s wall")


def cpu_cores():
    import oracle
    try:
        import threadpoolctl
        blas = max([i.get("num_threads", 1) for i in threadpoolctl.threadpool_info()] or [1])
    except Exception:
        blas = os.cpu_count() or 1
    return max(oracle.num_threads(), blas)


def run_reference(args, rank, world):
    if rank != 0:
        return 0
    import oracle
    from oracle import cnn
    from synth import scenes
    desc = scenes.procedural(0)
    params = cnn.kaiming(0)
    oracle.build()
    for k in range(args.warmup):
        oracle_frame_sample(desc, params, 1000 + k)
    times = []
    t_all = time.perf_counter()
    for k in range(args.steps):
        ms, detail = oracle_frame_sample(desc, params, k)
        times.append(ms)
    wall = time.perf_counter() - t_all
    value = float(np.mean(times))
    cores = cpu_cores()
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "ms/frame",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup, "ms_per_step": value,
        "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "f32/f64",
        "data": "synthetic", "config": WORKLOAD,
        "cpu_baseline": {"value": value, "unit": "ms/frame", "cores": cores, "kind": "oracle",
                         "sample": detail + f"; {args.steps} samples, {wall:.1f} s wall"},
        "e2e": {"value": value, "unit": "ms/frame", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# ----------------------------------------------------------------------------
# equal-PSNR comparison: hybrid frame vs plain high-resolution path tracing
# ----------------------------------------------------------------------------
def train_net(mrs, s, n_scenes=800, steps=20000):
    """Trains the fusion network by the training recipe (seeded 200k-triangle
    scenes, seeds 1.. -- never the bench scene -- one 256^2 window of the
    1024^2 frame per scene with LRHS 64 spp, HRLS 4 spp and a 1024-spp
    target; 128^2 crops at batch 16, L1 on log(1 + x), Adam lr 1e-4, BF16
    training step) reduced to n_scenes scenes and `steps` steps, and scores
    the gain over the method without the network on 4 held-out scenes
    (512^2 windows, 4096-spp references).  Returns the net and the report."""
    from paper_2106_12802_gb300 import trainer
    net, rep = trainer.train_recipe(n_scenes=n_scenes, steps=steps, window=256, spp_tgt=1024,
                                    lr=1e-4, loss="l1log", eval_scenes=4, eval_size=512,
                                    eval_tgt=4096, log_every=0)
    rep["reduction"] = (f"{n_scenes} of the recipe's 2,000 scenes and {steps} steps; each scene "
                        "renders one 256^2 window of its 1024^2 frame (windows are bit-identical "
                        "to those pixels of the whole render)")
    return net, rep


def equal_psnr(mrs, scene, s, net, training, ref_spp=4096):
    """Renders a ref_spp reference of the bench scene, scores the hybrid frame
    (BF16 fusion with the trained net) and finds the plain HR spp that reaches
    the same sRGB PSNR (bisection on spp); returns both times (CUDA events,
    same renderer)."""
    import torch

    ref = mrs.render(scene, HR, HR, ref_spp, DEPTH, RR, 99991, aux=False, counts=False)["radiance"]
    ev = (torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))

    def timed(fn):
        fn()
        torch.cuda.synchronize()
        ev[0].record()
        r = fn()
        ev[1].record()
        torch.cuda.synchronize()
        return r, ev[0].elapsed_time(ev[1])

    ctx_lr, ctx_hr = mrs.RenderContext(), mrs.RenderContext()
    s_lr, s_hr = torch.cuda.Stream(), torch.cuda.Stream()

    def hybrid():
        main = torch.cuda.current_stream()
        s_lr.wait_stream(main)
        s_hr.wait_stream(main)
        with torch.cuda.stream(s_hr):
            hr = mrs.render(scene, HR, HR, SPP_HR, DEPTH, RR, 6, aux=True, counts=False, ctx=ctx_hr)
        with torch.cuda.stream(s_lr):
            lr = mrs.render(scene, LR, LR, SPP_LR, DEPTH, RR, 5, aux=False, counts=False,
                            ctx=ctx_lr)["radiance"]
        main.wait_stream(s_lr)
        main.wait_stream(s_hr)
        out = net.fuse(lr[None], hr["radiance"][None], hr["albedo"][None], hr["normal"][None], s,
                       precision="bf16")
        return out[0]

    fused, t_h = timed(hybrid)
    p_h = mrs.image_metrics(fused.contiguous(), ref)[0]
    cache = {}

    def plain_psnr(n):
        if n not in cache:
            img = mrs.render(scene, HR, HR, n, DEPTH, RR, 7, aux=False, counts=False)["radiance"]
            cache[n] = mrs.image_metrics(img, ref)[0]
        return cache[n]

    lo, hi = 1, 1
    while plain_psnr(hi) < p_h and hi < ref_spp // 4:
        lo, hi = hi, hi * 2
    while hi - lo > 1 and plain_psnr(hi) >= p_h:
        mid = (lo + hi) // 2
        if plain_psnr(mid) >= p_h:
            hi = mid
        else:
            lo = mid
    n_eq = hi
    # the plain render timed at its best first bounce of the tail kernel (the
    # image does not depend on it; many-wave renders favour a later start)
    t_by_tail = {}
    for tb in (0, 1, 2):
        c = mrs.RenderContext()
        c.set_tail(tb)
        _, t_by_tail[tb] = timed(lambda: mrs.render(scene, HR, HR, n_eq, DEPTH, RR, 7, aux=False,
                                                    counts=False, ctx=c))
        c.close()
    tail_best = min(t_by_tail, key=t_by_tail.get)
    t_p = t_by_tail[tail_best]
    # the method without the network: upsampled LRHS (zero-weight network)
    lr = mrs.render(scene, LR, LR, SPP_LR, DEPTH, RR, 5, aux=False, counts=False)["radiance"]
    hr = mrs.render(scene, HR, HR, SPP_HR, DEPTH, RR, 6, aux=True, counts=False)
    up = mrs.Net(np.zeros(mrs.NPARAMS, np.float32)).fuse(
        lr[None], hr["radiance"][None], hr["albedo"][None], hr["normal"][None], s, precision="fp32")
    p_lr_up = mrs.image_metrics(up[0].contiguous(), ref)[0]
    p_hrls = mrs.image_metrics(hr["radiance"], ref)[0]
    return {"reference_spp": ref_spp, "hybrid_psnr_db": p_h, "hybrid_ms": t_h,
            "upsampled_lrhs_psnr_db": p_lr_up, "hrls_psnr_db": p_hrls, "plain_spp_at_equal_psnr": n_eq,
            "plain_psnr_db": plain_psnr(n_eq), "plain_ms": t_p, "speedup_plain_over_hybrid": t_p / t_h,
            "plain_ms_by_tail_start": {str(k): v for k, v in t_by_tail.items()},
            "plain_tail_start": tail_best,
            "spp_avg_hybrid": SPP_LR / (s * s) + SPP_HR,
            "training": training}


# ----------------------------------------------------------------------------
# batched serving: many frames of uneven size, scale and spp in one CUDA graph
# ----------------------------------------------------------------------------
def batched_serving(mrs, params, n_jobs=32, seed=5, psnr_window=256, ref_spp=4096, reps=3,
                    tree="cluster"):
    """32 hybrid frames of 32 different seeded 200k-triangle scenes: HR in
    {512, 1024, 2048}^2, scale in {2, 4}, HRLS spp in {1, 2, 4, 8}, LRHS
    64 spp.  All 64 renders are one batched render (mrs_render_batch: the
    frames' paths share waves, one launch per wavefront stage over all of
    them); the fusion runs once per (size, scale) group of frames (N frames
    per launch) in BF16 or FP8; the device-side gate per frame; the whole
    batch is one CUDA graph per precision.  The autotuner picks the wave
    size, the tail kernel's first bounce and the conv's ring depth.  Every
    frame's fused image is scored (sRGB PSNR) against a ref_spp-spp render
    over its central psnr_window^2 window (a window render is bit-identical
    to those pixels of the whole render).  For comparison the same frames
    are also timed with one render call per frame (the batch as 64 separate
    renders in one graph).  The scenes are built once, before anything is
    timed, with the `tree` render tree (default: clustering in grid-wide
    rounds, the fastest to render over)."""
    import torch

    from paper_2106_12802_gb300 import autotune
    rng = np.random.default_rng(seed)
    frames = []
    for j in range(n_jobs):
        frames.append({"scene": mrs.Scene.seeded(200 + j), "hr": int(rng.choice([512, 1024, 2048])),
                       "s": int(rng.choice([2, 4])), "spp_h": int(rng.choice([1, 2, 4, 8])),
                       "seed": 1000 + j})
    for f in frames:
        f["scene"].set_tree(tree)
    net = mrs.Net(params)
    dev = torch.device("cuda")
    groups = {}
    for f in frames:
        groups.setdefault((f["hr"], f["s"]), []).append(f)
    bufs = {}
    for (H, s), fs in groups.items():
        n = len(fs)
        bufs[(H, s)] = {"lr": torch.empty((n, H // s, H // s, 3), device=dev),
                        "hr": torch.empty((n, H, H, 3), device=dev),
                        "alb": torch.empty((n, H, H, 3), device=dev),
                        "nrm": torch.empty((n, H, H, 3), device=dev),
                        "dep": torch.empty((n, H, H), device=dev),
                        "fused": torch.empty((n, H, H, 3), device=dev),
                        "out": torch.empty((n, H, H, 3), device=dev),
                        "used": torch.zeros((n, 2), dtype=torch.int32, device=dev),
                        "D": torch.zeros(n, dtype=torch.float64, device=dev)}
        for i, f in enumerate(fs):
            f["group"], f["index"] = (H, s), i
    jobs = []
    for f in frames:
        b, i, H, s = bufs[f["group"]], f["index"], f["hr"], f["s"]
        jobs.append({"scene": f["scene"], "W": H // s, "H": H // s, "spp": SPP_LR, "max_depth": DEPTH,
                     "rr_start": RR, "seed": f["seed"], "out": {"radiance": b["lr"][i]}})
        jobs.append({"scene": f["scene"], "W": H, "H": H, "spp": f["spp_h"], "max_depth": DEPTH,
                     "rr_start": RR, "seed": f["seed"] + 7,
                     "out": {"radiance": b["hr"][i], "albedo": b["alb"][i], "normal": b["nrm"][i],
                             "depth": b["dep"][i]}})
    ctx = mrs.RenderContext()

    def render_all():
        mrs.render_batch(ctx, jobs)

    def fuse_all(prec):
        for (H, s), b in bufs.items():
            net.fuse(b["lr"], b["hr"], b["alb"], b["nrm"], s, precision=prec, out=b["fused"])
            for i in range(b["lr"].shape[0]):
                mrs.gate_async(b["fused"][i:i + 1], b["lr"][i:i + 1], None, s, 0.01,
                               out=b["out"][i:i + 1], used=b["used"][i], D=b["D"][i:i + 1])

    # autotuning (outside the graph): wave size, tail start, conv ring depth
    tuned = {}
    tuned["wave"], t_wave = autotune.tune("batch:wave", [{"wave": c} for c in autotune.WAVE_CANDIDATES],
                                          lambda c: ctx.set_wave(c["wave"]), render_all, reps=1, cache=None)
    tuned["tail"], t_tail = autotune.tune("batch:tail", [{"tail": b} for b in autotune.TAIL_CANDIDATES],
                                          lambda c: ctx.set_tail(c["tail"]), render_all, reps=1, cache=None)
    tuned["ring"], t_ring = autotune.tune("batch:ring", [{"ring": r} for r in autotune.RING_CANDIDATES],
                                          lambda c: mrs.conv_set_ring(c["ring"]),
                                          lambda: fuse_all("bf16"), reps=2, cache=None)
    result = {"jobs": n_jobs, "distinct_scenes": n_jobs, "tree": tree,
              "hr_mix": {str(r): sum(1 for f in frames if f["hr"] == r) for r in (512, 1024, 2048)},
              "groups": {f"{H}x{H}/s{s}": len(fs) for (H, s), fs in groups.items()},
              "paths_per_batch": int(sum((f["hr"] // f["s"]) ** 2 * SPP_LR + f["hr"] ** 2 * f["spp_h"]
                                         for f in frames)),
              "autotuned": tuned, "autotune_ms": {"wave": t_wave, "tail": t_tail, "ring": t_ring}}

    def timed_graph(fn):
        side = torch.cuda.Stream()
        side.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(side):
            fn()                      # warm-up: sizes arenas, packs / calibrates weights
        torch.cuda.current_stream().wait_stream(side)
        torch.cuda.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g):
            fn()
        g.replay()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(reps):
            g.replay()
        e1.record()
        torch.cuda.synchronize()
        del g
        return e0.elapsed_time(e1) / reps

    renders_ms = timed_graph(render_all)
    # the same 64 renders as separate calls (one context per frame pair)
    ctx_f = mrs.RenderContext()
    ctx_f.set_wave(tuned["wave"]["wave"])
    ctx_f.set_tail(tuned["tail"]["tail"])

    def render_per_call():
        for jb in jobs:
            mrs.render(jb["scene"], jb["W"], jb["H"], jb["spp"], DEPTH, RR, jb["seed"],
                       out=jb["out"], ctx=ctx_f, counts=False)
    per_call_ms = timed_graph(render_per_call)
    ctx_f.close()
    refs = []
    for f in frames:
        H = f["hr"]
        w = min(psnr_window, H)
        win = ((H - w) // 2, (H - w) // 2, w, w)
        ref = mrs.render(f["scene"], H, H, ref_spp, DEPTH, RR, 99991, aux=False, counts=False,
                         window=win)["radiance"]
        refs.append((win, ref))
    per_frame = [{"hr": f["hr"], "s": f["s"], "hrls_spp": f["spp_h"]} for f in frames]
    for prec in ("bf16", "fp8"):
        ms = timed_graph(lambda: (render_all(), fuse_all(prec)))
        ps = []
        for f, (win, ref), pf in zip(frames, refs, per_frame):
            x0, y0, w, _ = win
            img = bufs[f["group"]]["fused"][f["index"], y0:y0 + w, x0:x0 + w].contiguous()
            p = mrs.image_metrics(img, ref)[0]
            pf[f"psnr_{prec}"] = round(p, 3)
            ps.append(p)
        result[prec] = {"ms_per_batch": ms, "ms_per_frame": ms / n_jobs,
                        "frames_per_s": n_jobs / ms * 1e3,
                        "mean_psnr_db_vs_4096spp": float(np.mean(ps)), "psnr_frames": len(ps)}
    result["renders_ms_batched"] = renders_ms
    result["renders_ms_one_call_per_render"] = per_call_ms
    result["render_msamples_per_s_batched"] = result["paths_per_batch"] / renders_ms / 1e3
    result["per_frame"] = per_frame
    result["psnr_note"] = (f"each frame's central {psnr_window}^2 window (the whole frame if smaller) "
                           f"against a {ref_spp}-spp window render")
    mrs.conv_set_ring(0)
    ctx.close()
    for f in frames:
        f["scene"].close()
    net.close()
    return result


# ----------------------------------------------------------------------------
# the spp study of Sec. 5 (Table comp_spp) on procedural scenes
# ----------------------------------------------------------------------------
def spp_study(mrs, s=S, size=512, train_scenes=12, steps=2000):
    """Trains the x4 network with the method's spp randomisation and scores it
    over the (LRHS spp, HRLS spp) grid of Table comp_spp on 4 held-out scenes
    against 2048-spp renders (mean sRGB PSNR / RelMSE, with the method
    without the network for comparison)."""
    from paper_2106_12802_gb300 import trainer
    t0 = time.perf_counter()
    data = trainer.make_dataset(range(500, 500 + train_scenes), size=size, s=s, spp_tgt=512,
                                spp_random=True, examples_per_scene=2, seed=2)
    net = mrs.Net(trainer.init_params(0))
    trainer.train(net, data, steps, batch=16, crop=128, s=s, lr=1e-3, seed=0, precision="bf16",
                  loss="robust")
    del data
    t_train = time.perf_counter() - t0
    g = trainer.spp_grid(net, range(600, 604), size=size, s=s, spp_tgt=2048)
    net.close()
    cells = [{"lrhs_spp": a, "hrls_spp": b, **{k: round(v, 4) for k, v in r.items()}}
             for (a, b), r in sorted(g.items())]
    return {"training": f"{train_scenes} procedural scenes x 2 examples at {size}^2, spp pairs "
                        f"drawn per example (Sec. 4), 512-spp targets; {steps} BF16 Adam steps, "
                        f"batch 16 x 128^2, robust loss ({t_train:.1f} s incl. rendering)",
            "eval": f"4 held-out scenes at {size}^2, x{s}, 2048-spp targets", "cells": cells}


# ----------------------------------------------------------------------------
# the method's own fusion network (Sec. 4): x4 two-encoder network at 1024^2
# ----------------------------------------------------------------------------
def paper_network(mrs, flush, s=S, reps=10):
    """Device time of the method's own x4 network (BF16 tensor cores, Kaiming
    weights: the time does not depend on them) on a 256^2 LRHS + 1024^2 HRLS
    frame, L2 flushed before every rep, plus one FP32 pass for reference."""
    import torch

    from paper_2106_12802_gb300 import rdn
    net = mrs.RDN(rdn.kaiming_params(s), s)
    g = torch.Generator(device="cuda").manual_seed(0)
    lr = torch.rand((1, LR, LR, 3), device="cuda", generator=g)
    hr = [torch.rand((1, HR, HR, 3), device="cuda", generator=g) for _ in range(3)]
    out = torch.empty((1, HR, HR, 3), device="cuda")
    for _ in range(2):
        net.fuse(lr, *hr, precision="bf16", out=out)
    torch.cuda.synchronize()
    ts = []
    for _ in range(reps):
        flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        net.fuse(lr, *hr, precision="bf16", out=out)
        e1.record()
        torch.cuda.synchronize()
        ts.append(e0.elapsed_time(e1))
    # one more rep with per-launch events for the conv share (events between
    # the launches serialise them, so this rep is not part of the timing)
    mrs.profile_read()
    mrs.profile_enable(True)
    flush.zero_()
    net.fuse(lr, *hr, precision="bf16", out=out)
    torch.cuda.synchronize()
    mrs.profile_enable(False)
    prof = mrs.profile_read()
    reps_prof = 1
    net.check()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    net.fuse(lr, *hr, precision="fp32", out=out)
    e1.record()
    torch.cuda.synchronize()
    fp32_ms = e0.elapsed_time(e1)
    # four frames per call (serving batch): the same launches cover 4x the
    # pixels, so the per-launch fixed cost is shared
    nb = 4
    lrb = lr.expand(nb, -1, -1, -1).contiguous()
    hrb = [t.expand(nb, -1, -1, -1).contiguous() for t in hr]
    outb = torch.empty((nb, HR, HR, 3), device="cuda")
    net.fuse(lrb, *hrb, precision="bf16", out=outb)
    tb = []
    for _ in range(5):
        flush.zero_()
        e0.record()
        net.fuse(lrb, *hrb, precision="bf16", out=outb)
        e1.record()
        torch.cuda.synchronize()
        tb.append(e0.elapsed_time(e1) / nb)
    del lrb, hrb, outb
    train = rdn_train_timing(mrs, flush, s, precision="fp32")
    train_bf16 = rdn_train_timing(mrs, flush, s, precision="bf16", reps=10, warmup=3)
    ms = float(np.median(ts))
    flop = rdn.flops_per_lr_pixel(s) * LR * LR
    peaks = _peaks()
    conv_ms = prof["conv_tc"][0] / reps_prof
    tf = flop / (ms * 1e-3) / 1e12
    res = {"network": "Sec. 4 two-encoder network, x4: H_lrhs, H_hrls, 2 deshuffles, 1x1 fuse, "
                      "3 RDG x 5 RDB x 4 convs, 2 shuffle upscalings, H_Rec; Kaiming weights",
           "lrhs": [LR, LR], "hr": [HR, HR], "bf16_ms": ms, "fp32_ms": fp32_ms,
           "bf16_ms_per_frame_batch4": float(np.median(tb)),
           "gflop": flop / 1e9, "bf16_tflops": tf,
           "tensor_frac_of_measured_sustained": tf / peaks["bf16_tflops_sustained"],
           "conv_tc_ms_events": conv_ms, "conv_tc_launches": prof["conv_tc"][1] // reps_prof,
           "conv_tc_tflops": flop / (conv_ms * 1e-3) / 1e12 if conv_ms else None,
           "l2": "flushed before every rep (512 MiB write)", "train_step_fp32": train,
           "train_step_bf16": train_bf16}
    net.close()
    return res


def rdn_train_flop_per_lr_pixel(s):
    """Multiply-adds x 2 of one training step per LR pixel: the forward, every
    layer's weight gradient (as much again) and every layer's input gradient
    except the two encoders' (their inputs are images)."""
    from paper_2106_12802_gb300 import rdn
    fwd = rdn.flops_per_lr_pixel(s)
    enc = 2 * 9 * 3 * 64 + 2 * 9 * 9 * 64 * s * s
    return 3 * fwd - enc


def rdn_train_timing(mrs, flush, s=S, N=16, crop=192, reps=3, warmup=2, precision="fp32"):
    """Device time of one training step of the method's own network at the
    paper's training batch (Sec. 4 "Implement details": mini-batch 16,
    192 x 192 HR patches at x4): forward with its activations kept, the
    robust loss, the backward of every step, Adam; FP32 on the SIMT cores or
    BF16 on the tensor cores.  Random radiance-like inputs on the device, L2
    flushed before every step."""
    import torch

    from paper_2106_12802_gb300 import rdn
    net = mrs.RDN(rdn.kaiming_params(s), s)
    g = torch.Generator(device="cuda").manual_seed(12)
    h = crop // s
    lr = torch.rand((N, h, h, 3), device="cuda", generator=g) * 2
    hr = torch.rand((N, crop, crop, 3), device="cuda", generator=g) * 2
    alb = torch.rand((N, crop, crop, 3), device="cuda", generator=g)
    nrm = torch.rand((N, crop, crop, 3), device="cuda", generator=g) * 2 - 1
    tgt = torch.rand((N, crop, crop, 3), device="cuda", generator=g) * 2
    for _ in range(warmup):
        net.train_step(lr, hr, alb, nrm, tgt, lr=1e-4, loss="robust", beta=0.1, sync_loss=False,
                       precision=precision)
    torch.cuda.synchronize()
    ts = []
    for _ in range(reps):
        flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        net.train_step(lr, hr, alb, nrm, tgt, lr=1e-4, loss="robust", beta=0.1, sync_loss=False,
                       precision=precision)
        e1.record()
        torch.cuda.synchronize()
        ts.append(e0.elapsed_time(e1))
    net.close()
    ms = float(np.median(ts))
    flop = rdn_train_flop_per_lr_pixel(s) * N * h * h
    tf = flop / (ms * 1e-3) / 1e12
    res = {"batch": [N, crop, crop], "scale": s, "loss": "robust, beta 0.1", "optimizer": "Adam, lr 1e-4",
           "ms": ms, "tflop_per_step": flop / 1e12, "tflops": tf}
    if precision == "fp32":
        sm = torch.cuda.get_device_properties(0).multi_processor_count
        fp32_peak = sm * 128 * 2 * 2.07e9 / 1e12   # TFLOP/s: FP32 lanes x FMA x max SM clock
        res.update({"precision": "fp32 (SIMT)", "fp32_frac": tf / fp32_peak, "fp32_peak_tflops": fp32_peak})
    else:
        res.update({"precision": "bf16 (tensor cores: forward, input and weight gradients)",
                    "tensor_frac_of_measured_sustained": tf / _peaks()["bf16_tflops_sustained"]})
    return res


def fp8_gemm_tflops(n=8192, reps=10):
    """Dense FP8-E4M3 GEMM throughput of the vendor library (torch._scaled_mm,
    n^3, best of `reps`): the denominator for the FP8 fusion, which the peaks
    file does not measure.  None (with the reason) where it is unavailable."""
    import torch
    try:
        a = torch.randn(n, n, device="cuda").to(torch.float8_e4m3fn)
        b = torch.randn(n, n, device="cuda").to(torch.float8_e4m3fn).t()
        one = torch.ones((), device="cuda")
        torch._scaled_mm(a, b, one, one, out_dtype=torch.bfloat16)
        torch.cuda.synchronize()
        best = None
        for _ in range(reps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            torch._scaled_mm(a, b, one, one, out_dtype=torch.bfloat16)
            e1.record()
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1)
            best = ms if best is None else min(best, ms)
        return 2.0 * n ** 3 / (best * 1e-3) / 1e12, "torch._scaled_mm e4m3 %d^3, best of %d" % (n, reps)
    except Exception as e:  # noqa: BLE001
        return None, "unavailable: %s" % str(e).splitlines()[0][:120]


def fusion_precisions(mrs, net, flush, reps=10):
    """Device time of the x4 fusion network alone at 1024^2 (L2 flushed before
    every rep) in BF16, FP8-E4M3 and FP32, with the tensor-core rates against
    the measured BF16 and FP8 GEMM peaks, and the FP8 / BF16 output agreement."""
    import torch
    g = torch.Generator(device="cuda").manual_seed(3)
    lr = torch.rand((1, LR, LR, 3), device="cuda", generator=g)
    hr = [torch.rand((1, HR, HR, 3), device="cuda", generator=g) for _ in range(3)]
    outs = {}
    res = {"hr": [HR, HR], "scale": S, "l2": "flushed before every rep (512 MiB write)"}
    flop = CONV_FLOP_PER_PX * HR * HR
    peaks = _peaks()
    fp8_peak, fp8_src = fp8_gemm_tflops()
    for prec in ("bf16", "fp8", "fp32"):
        out = torch.empty((1, HR, HR, 3), device="cuda")
        net.fuse(lr, *hr, S, precision=prec, out=out)
        torch.cuda.synchronize()
        ts = []
        for _ in range(reps if prec != "fp32" else 2):
            flush.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            net.fuse(lr, *hr, S, precision=prec, out=out)
            e1.record()
            torch.cuda.synchronize()
            ts.append(e0.elapsed_time(e1))
        ms = float(np.median(ts))
        tf = flop / (ms * 1e-3) / 1e12
        res[prec] = {"ms": ms, "tflops": tf}
        outs[prec] = out
    res["bf16"]["tensor_frac_of_measured_sustained"] = res["bf16"]["tflops"] / peaks["bf16_tflops_sustained"]
    res["fp8"]["tensor_frac_of_fp8_gemm"] = res["fp8"]["tflops"] / fp8_peak if fp8_peak else None
    res["fp8_gemm_tflops"] = fp8_peak
    res["fp8_gemm_source"] = fp8_src
    res["fp8_vs_bf16_psnr_db"] = mrs.image_metrics(outs["fp8"][0].contiguous(),
                                                   outs["bf16"][0].contiguous())[0]
    res["bf16_vs_fp32_psnr_db"] = mrs.image_metrics(outs["bf16"][0].contiguous(),
                                                    outs["fp32"][0].contiguous())[0]
    return res


def train_step_timing(mrs, params, flush, N=16, crop=128, s=S, reps=10, warmup=3):
    """Device time of one BF16 training step of the fusion network at the
    training batch (N crops of crop x crop HR pixels, x s): forward with every
    activation kept, loss, tensor-core input and weight gradients, Adam.  The
    inputs are random radiance-like images already on the device; L2 flushed
    before every step; median of `reps` event-timed steps.  The per-family
    split comes from one extra step with events around every launch."""
    import torch
    g = torch.Generator(device="cuda").manual_seed(11)
    h = crop // s
    lr = torch.rand((N, h, h, 3), device="cuda", generator=g) * 2
    hr = torch.rand((N, crop, crop, 3), device="cuda", generator=g) * 2
    alb = torch.rand((N, crop, crop, 3), device="cuda", generator=g)
    nrm = torch.rand((N, crop, crop, 3), device="cuda", generator=g) * 2 - 1
    tgt = torch.rand((N, crop, crop, 3), device="cuda", generator=g) * 2
    net = mrs.Net(params)
    net.set_loss("l1log")
    args = (lr, hr, alb, nrm, tgt, s)
    for _ in range(warmup):
        mrs.train_step(net, *args, lr=1e-4, precision="bf16", sync_loss=False)
    torch.cuda.synchronize()
    ts = []
    for _ in range(reps):
        flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        mrs.train_step(net, *args, lr=1e-4, precision="bf16", sync_loss=False)
        e1.record()
        torch.cuda.synchronize()
        ts.append(e0.elapsed_time(e1))
    mrs.profile_read()
    mrs.profile_enable(True)
    flush.zero_()
    mrs.train_step(net, *args, lr=1e-4, precision="bf16", sync_loss=False)
    torch.cuda.synchronize()
    mrs.profile_enable(False)
    prof = mrs.profile_read()
    net.close()
    ms = float(np.median(ts))
    flop = TRAIN_FLOP_PER_PX * N * crop * crop
    tf = flop / (ms * 1e-3) / 1e12
    peaks = _peaks()
    return {"batch": [N, crop, crop], "scale": s, "precision": "bf16", "loss": "l1log",
            "optimizer": "Adam, lr 1e-4", "ms": ms, "tflop_per_step": flop / 1e12,
            "tflops": tf, "tensor_frac_of_measured_sustained": tf / peaks["bf16_tflops_sustained"],
            "family_ms_events": {k: round(v[0], 4) for k, v in prof.items() if v[1]},
            "l2": "flushed before every step (512 MiB write)",
            "flop_note": "forward + weight gradients of 18 layers + input gradients of the 17 "
                         "layers after the first, 2 FLOP per multiply-add"}


# ----------------------------------------------------------------------------
# GPU arm
# ----------------------------------------------------------------------------
def run_gpu(args, rank, world):
    import torch
    import torch.distributed as dist

    import paper_2106_12802_gb300 as mrs
    from paper_2106_12802_gb300 import trainer
    from synth import scenes

    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    mrs.load()
    stream = torch.cuda.current_stream()
    desc = scenes.procedural(0)
    scene = mrs.Scene(desc)
    scene.set_tree(TREE)
    # the network: trained on held-out scenes before anything is timed (the
    # timed frame and the equal-PSNR comparison use the same weights);
    # --quick keeps the Kaiming initialisation (timing does not depend on the
    # weights, the gate's decision does)
    if args.quick:
        net, training = mrs.Net(trainer.init_params(0)), None
    else:
        net, training = train_net(mrs, S)
    params = net.get_params()

    lrhs = torch.empty((1, LR, LR, 3), device=dev)
    hrls = torch.empty((1, HR, HR, 3), device=dev)
    alb = torch.empty((1, HR, HR, 3), device=dev)
    nrm = torch.empty((1, HR, HR, 3), device=dev)
    dep = torch.empty((1, HR, HR), device=dev)
    fused = torch.empty((1, HR, HR, 3), device=dev)
    out = torch.empty((1, HR, HR, 3), device=dev)
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    gate_info = {}
    # the LRHS and HRLS renders are independent: they run concurrently on two
    # streams with render contexts of their own, so that the low-occupancy
    # last bounces of one overlap the other's bulk
    ctx_lr, ctx_hr = mrs.RenderContext(), mrs.RenderContext()
    s_lr, s_hr = torch.cuda.Stream(), torch.cuda.Stream()

    def renders(seed, serial=False):
        # serial: both renders one after the other on the main stream (the
        # profiled frames, so that each kernel's events time that kernel alone)
        s_a, s_b = (stream, stream) if serial else (s_hr, s_lr)
        s_a.wait_stream(stream)
        s_b.wait_stream(stream)
        with torch.cuda.stream(s_a):
            mrs.render(scene, HR, HR, SPP_HR, DEPTH, RR, seed + 1, ctx=ctx_hr,
                       out={"radiance": hrls[0], "albedo": alb[0], "normal": nrm[0], "depth": dep[0]})
        with torch.cuda.stream(s_b):
            mrs.render(scene, LR, LR, SPP_LR, DEPTH, RR, seed, ctx=ctx_lr, out={"radiance": lrhs[0]})
        stream.wait_stream(s_a)
        stream.wait_stream(s_b)

    # the gate's decision stays on the device (no host synchronisation inside
    # a frame); it is read after the frames
    used_d = torch.zeros(2, dtype=torch.int32, device=dev)
    D_d = torch.zeros(1, dtype=torch.float64, device=dev)

    def frame(seed, serial=False):
        scene.rebuild()
        renders(seed, serial)
        net.fuse(lrhs, hrls, alb, nrm, S, precision="bf16", out=fused)
        mrs.gate_async(fused, lrhs, None, S, 0.01, out=out, used=used_d, D=D_d)

    for k in range(args.warmup):
        frame(1000 + k)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()

    # ---- timed region: device-resident inputs, L2 flushed between steps -----
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    launches0 = mrs.kernel_launches()
    with ClockSampler(local) as clk:
        torch.cuda.synchronize()
        for k in range(args.steps):
            flush.zero_()
            ev[k][0].record(stream)
            frame(k)
            ev[k][1].record(stream)
        torch.cuda.synchronize()
    launches = (mrs.kernel_launches() - launches0) // max(args.steps, 1)
    step_ms = [a.elapsed_time(b) for a, b in ev]
    gate_info.update(used_plain=bool(used_d[0].item()), D=float(D_d.item()))
    # per-kernel-family split from extra frames with CUDA events around every
    # launch (outside the timed region: the events serialise the launches),
    # the two renders one after the other so that no kernel's events also
    # cover the other render's kernels
    prof_steps = max(3, args.steps // 4)
    mrs.profile_read()
    mrs.profile_enable(True)
    for k in range(prof_steps):
        flush.zero_()
        frame(500 + k, serial=True)
    torch.cuda.synchronize()
    mrs.profile_enable(False)
    prof = mrs.profile_read()
    t_local = max_over_ranks(float(np.sum(step_ms)), world, dev)
    if world > 1:
        dist.barrier()
    ms_frame = t_local / (args.steps * world)

    # ---- end to end through the public API with host buffers -----------------
    Vh = torch.from_numpy(np.ascontiguousarray(desc["V"], np.float32)).pin_memory()
    out_h = torch.empty((1, HR, HR, 3), dtype=torch.float32).pin_memory()
    used_h = torch.empty(2, dtype=torch.int32).pin_memory()
    D_h = torch.empty(1, dtype=torch.float64).pin_memory()

    def frame_e2e(seed):
        # geometry in from pinned host memory; image and gate decision back,
        # one synchronisation per frame
        scene.update_vertices(Vh)
        renders(seed)
        net.fuse(lrhs, hrls, alb, nrm, S, precision="bf16", out=fused)
        mrs.gate_async(fused, lrhs, None, S, 0.01, out=out, used=used_d, D=D_d)
        out_h.copy_(out, non_blocking=True)
        used_h.copy_(used_d, non_blocking=True)
        D_h.copy_(D_d, non_blocking=True)
        torch.cuda.synchronize()

    frame_e2e(0)
    e2e_steps = max(3, min(args.steps, 10))
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for k in range(e2e_steps):
        frame_e2e(k)
    e2e_ms = 1e3 * (time.perf_counter() - t0) / e2e_steps
    h2d = Vh.numel() * 4
    d2h = out_h.numel() * 4 + used_h.numel() * 4 + D_h.numel() * 8
    # the two copies alone (device-timed, same pinned buffers), to split the
    # end-to-end time into copies and the rest
    v_dev = torch.empty(Vh.shape, dtype=torch.float32, device=dev)
    c0, c1, c2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
    c0.record(stream)
    v_dev.copy_(Vh, non_blocking=True)
    c1.record(stream)
    out_h.copy_(out, non_blocking=True)
    c2.record(stream)
    torch.cuda.synchronize()
    copy_ms = {"h2d_ms": c0.elapsed_time(c1), "d2h_ms": c1.elapsed_time(c2)}
    del v_dev

    # ---- context measurements (outside the timed region) --------------------
    extra = {}
    if rank == 0 and not args.quick and not args.no_equal_psnr:
        extra["equal_psnr"] = equal_psnr(mrs, scene, S, net, "the bench's trained network "
                                         "(`training`)")
    if rank == 0 and not args.quick and not args.no_batched:
        extra["batched_serving"] = batched_serving(mrs, params)
    if rank == 0 and not args.no_paper_network:
        extra["paper_network_x4"] = paper_network(mrs, flush)
    if rank == 0 and not args.quick:
        extra["fusion_precisions_1024"] = fusion_precisions(mrs, net, flush)
    if rank == 0:
        extra["train_step"] = train_step_timing(mrs, trainer.init_params(0), flush)
    if rank == 0 and not args.quick and not args.no_spp_study:
        extra["spp_study_x4"] = spp_study(mrs)
    if rank == 0:
        stats_lr = mrs.render_stats(scene, LR, LR, SPP_LR, DEPTH, RR, 0)
        stats_hr = mrs.render_stats(scene, HR, HR, SPP_HR, DEPTH, RR, 1)
        cnt_lr = mrs.render(scene, LR, LR, SPP_LR, DEPTH, RR, 0, aux=False)["counts"]
        cnt_hr = mrs.render(scene, HR, HR, SPP_HR, DEPTH, RR, 1, aux=False)["counts"]
        # closest-hit segments of bounces >= 1 (the tail kernel's units)
        tail_segments = int(cnt_lr[1:].sum().item() + cnt_hr[1:].sum().item())
    else:
        stats_lr = stats_hr = None
        tail_segments = None
    if rank == 0 and not args.quick:
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        plain = mrs.render(scene, HR, HR, 64, DEPTH, RR, 7)
        torch.cuda.synchronize()
        e0.record(stream)
        plain = mrs.render(scene, HR, HR, 64, DEPTH, RR, 8, out=plain)
        e1.record(stream)
        torch.cuda.synchronize()
        pms = e0.elapsed_time(e1)
        rays = int(plain["counts"].sum().item() + plain["shadow_counts"].sum().item())
        # the same render over the other trees (the radix tree, and clustering
        # in grid-wide rounds)
        tree_ms = {}
        for kind in ("lbvh", "cluster"):
            scene.set_tree(kind)
            plain = mrs.render(scene, HR, HR, 64, DEPTH, RR, 8, out=plain)
            torch.cuda.synchronize()
            e0.record(stream)
            plain = mrs.render(scene, HR, HR, 64, DEPTH, RR, 8, out=plain)
            e1.record(stream)
            torch.cuda.synchronize()
            tree_ms[kind] = e0.elapsed_time(e1)
        scene.set_tree(TREE)
        extra["plain_path_trace_1024_64spp"] = {
            "tree": TREE, "ms": pms, "msamples_per_s": HR * HR * 64 / pms / 1e3,
            "mrays_per_s": rays / pms / 1e3,
            "lbvh_tree_ms": tree_ms["lbvh"],
            "lbvh_tree_msamples_per_s": HR * HR * 64 / tree_ms["lbvh"] / 1e3,
            "cluster_tree_ms": tree_ms["cluster"],
            "cluster_tree_msamples_per_s": HR * HR * 64 / tree_ms["cluster"] / 1e3}
        # the timed frame again with its tree rebuilt as the Karras LBVH (radix
        # tree and refit) instead (same steps, same L2 flush; the images are the
        # same bit for bit), and both builds alone
        scene.set_tree("lbvh")
        for k in range(3):
            frame(2000 + k)
        hev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
               for _ in range(args.steps)]
        torch.cuda.synchronize()
        for k in range(args.steps):
            flush.zero_()
            hev[k][0].record(stream)
            frame(k)
            hev[k][1].record(stream)
        torch.cuda.synchronize()
        build_ms = {}
        for kind in ("lbvh", TREE):
            scene.set_tree(kind)
            torch.cuda.synchronize()
            e0.record(stream)
            for _ in range(10):
                scene.rebuild()
            e1.record(stream)
            torch.cuda.synchronize()
            build_ms[kind] = e0.elapsed_time(e1) / 10
        extra["frame_lbvh_tree"] = {
            "ms_per_step": float(np.mean([a.elapsed_time(b) for a, b in hev])),
            "tree_build_ms": build_ms}

    peaks = _peaks()
    conv_ms = prof["conv_tc"][0] / prof_steps
    conv_flop = CONV_FLOP_PER_PX * HR * HR
    family_ms = {k: v[0] / prof_steps for k, v in prof.items() if v[1]}
    # the conv stack against both of its rooflines: arithmetic intensity
    # 1,196,928 / 5,412 = 221 FLOP/B is below the measured ridge (about 256),
    # so HBM is the binding one
    conv_roof = None
    if conv_ms:
        c_tf = conv_flop / (conv_ms * 1e-3) / 1e12
        c_gbs = CONV_BYTES_PER_PX * HR * HR / (conv_ms * 1e-3) / 1e9
        conv_roof = {"tflops": c_tf, "tensor_frac": c_tf / peaks["bf16_tflops_sustained"],
                     "hbm_gbs": c_gbs, "hbm_frac": c_gbs / peaks["hbm_gbs"],
                     "flop_per_byte": CONV_FLOP_PER_PX / CONV_BYTES_PER_PX,
                     "ridge_flop_per_byte": peaks["bf16_tflops_sustained"] * 1e3 / peaks["hbm_gbs"],
                     "bound": "hbm" if CONV_FLOP_PER_PX / CONV_BYTES_PER_PX <
                     peaks["bf16_tflops_sustained"] * 1e3 / peaks["hbm_gbs"] else "tensor"}
    dom = max(family_ms, key=family_ms.get)
    roofline = None
    conv_tr = _traffic("k_conv_fold", "conv_tc.cu")
    conv_traffic = conv_tr["dram_bytes_per_launch"] if conv_tr else None
    if conv_roof is not None:
        conv_roof["traffic_per_64to64_launch"] = conv_traffic
        conv_roof["algorithmic_bytes_per_64to64_launch"] = 5 * 128 * HR * HR // 2
    if dom == "conv_tc":
        ach = CONV_BYTES_PER_PX * HR * HR / (conv_ms * 1e-3) / 1e9
        roofline = {"kernel": "k_conv_fold (tcgen05 implicit-GEMM 3x3 conv)", "bound": "hbm",
                    "achieved": ach, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                    "frac": ach / peaks["hbm_gbs"], "traffic": conv_traffic,
                    "peak_source": peaks["source"] + " HBM copy"}
    elif dom in ("trace", "shadow", "tail") and stats_lr:
        # traversal work of the kernel's own launches: the tail kernel's share
        # (late bounces, closest-hit and shadow rays) is counted apart
        def work(kind, part):
            tail = stats_lr["tail_" + kind] + stats_hr["tail_" + kind]
            return tail if part == "tail" else stats_lr[kind] + stats_hr[kind] - tail
        kinds = {"trace": ("",), "shadow": ("shadow_",), "tail": ("", "shadow_")}[dom]
        visits = sum(work(k + "visits", dom) for k in kinds)
        tests = sum(work(k + "tests", dom) for k in kinds)
        flop = FLOP_PER_NODE_VISIT * visits + FLOP_PER_TRI_TEST * tests
        ops = OPS_PER_NODE_VISIT * visits + OPS_PER_TRI_TEST * tests
        kms = family_ms[dom]
        launches_per_frame = prof[dom][1] / prof_steps
        sms = torch.cuda.get_device_properties(dev).multi_processor_count
        clock = peaks["sm_max_mhz"] * 1e6
        peak = sms * 128 * 2 * clock / 1e12          # FP32 FMA lanes, 2 FLOP each
        ach = flop / (kms * 1e-3) / 1e12
        ops_peak = sms * 128 * clock / 1e12
        ops_ach = ops / (kms * 1e-3) / 1e12
        # DRAM traffic of one launch, scaled from a small-case ncu capture by
        # the launch's units (bounce >= 1 closest-hit segments for the tail)
        tr = _traffic(f"k_{dom}", "pt.cu")
        traffic = None
        if tr and dom == "tail" and tail_segments and tr.get("units"):
            traffic = tr["dram_bytes_per_launch"] / tr["units"] * tail_segments / launches_per_frame
        elif tr and dom != "tail":
            traffic = tr["dram_bytes_per_launch"]
        l2_gbs = None
        if tr and tr.get("lts_bytes_per_launch") and dom == "tail" and tail_segments and tr.get("units"):
            l2_gbs = (tr["lts_bytes_per_launch"] / tr["units"] * tail_segments) / (kms * 1e-3) / 1e9
        l2_peak = l2_copy_gbs() if rank == 0 else None
        label = {"trace": "k_trace (closest-hit traversal, bounce 0)",
                 "shadow": "k_shadow (shadow-ray traversal, bounce 0)",
                 "tail": "k_tail (traversal, shading and shadow rays of bounces >= 1)"}[dom]
        roofline = {"kernel": label, "bound": "alu", "achieved": ach,
                    "peak": peak, "unit": "TFLOP/s", "frac": ach / peak,
                    "traffic": traffic,
                    "peak_source": f"{sms} SMs x 128 FP32 lanes x 2 FLOP (FMA) x "
                                   f"{peaks['sm_max_mhz']} MHz",
                    "flop_per_frame": flop, "flop_per_node_visit": FLOP_PER_NODE_VISIT,
                    "flop_per_tri_test": FLOP_PER_TRI_TEST, "node_visits_per_frame": visits,
                    "tri_tests_per_frame": tests, "kernel_ms_per_frame": kms,
                    "launches_per_frame": launches_per_frame,
                    "tail_segments_per_frame": tail_segments,
                    "traffic_note": ("per launch, from one small-case ncu capture "
                                     "(profiles/traffic.json) scaled by bounce >= 1 segments"
                                     if traffic else "no capture of the current source"),
                    "instruction_count": {"ops_per_frame": ops, "achieved_tops": ops_ach,
                                          "peak_tops": ops_peak, "frac": ops_ach / ops_peak,
                                          "note": "FP32 instructions counted from the source "
                                                  "(52 per node visit, 50 per triangle test; "
                                                  "--fmad=false) against the non-FMA issue rate"},
                    "l2": {"achieved_gbs": l2_gbs, "copy_gbs": l2_peak,
                           "frac": l2_gbs / l2_peak if l2_gbs and l2_peak else None,
                           "peak_source": "measured here: device copy between two 32 MB "
                                          "L2-resident buffers, read + write bytes"}}

    if rank == 0:
        cpu = None
        if not args.quick and not args.no_cpu_baseline:
            from oracle import cnn
            cms, detail = oracle_frame_estimate(desc, cnn.kaiming(0))
            cpu = {"value": cms, "unit": "ms/frame", "cores": cpu_cores(), "kind": "oracle",
                   "sample": detail}
        line = {
            "metric": METRIC, "value": ms_frame, "unit": "ms/frame", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": t_local / args.steps,
            "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "bf16",
            "data": "synthetic", "config": WORKLOAD,
            "parallelism": "replicas" if world > 1 else "single-gpu",
            "e2e": {"value": e2e_ms, "unit": "ms/frame", "h2d_bytes_per_step": h2d,
                    "d2h_bytes_per_step": d2h, **copy_ms},
            "roofline": roofline, "cpu_baseline": cpu, "clocks": clk.summary(),
            "gpu_launches": int(launches),
            "stage_ms_per_frame": {k: round(v, 4) for k, v in family_ms.items()},
            "stage_note": f"per-kernel-family CUDA-event totals over {prof_steps} extra frames "
                          "after the timed region (events around every launch, the two renders "
                          "one after the other on one stream): the families sum to about a "
                          "serialised frame, more than the timed frame, whose renders overlap",
            "conv_tflops": conv_flop / (conv_ms * 1e-3) / 1e12 if conv_ms else None,
            "conv_roofline": conv_roof,
            "gate": gate_info, "training": training, **extra,
        }
        print(json.dumps(line), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=40)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="mrs", choices=["mrs", "reference"])
    ap.add_argument("--quick", action="store_true", help="skip context measurements")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-equal-psnr", action="store_true")
    ap.add_argument("--no-batched", action="store_true")
    ap.add_argument("--no-paper-network", action="store_true")
    ap.add_argument("--no-spp-study", action="store_true")
    args = ap.parse_args()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        backend = "gloo" if args.impl == "reference" else "nccl"
        if backend == "nccl":
            import torch
            torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
        dist.init_process_group(backend)
    if args.impl == "reference":
        rc = run_reference(args, rank, world)
    else:
        rc = run_gpu(args, rank, world)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return rc


if __name__ == "__main__":
    sys.exit(main())
