"""Training-data generation, training loop and evaluation of the fusion network.

The learned part of the method (Sec. 4): the network is trained on
(LRHS, HRLS + albedo / normal, high-spp target) triples that this renderer
produces from seeded procedural scenes, and judged against the high-spp
render.  All rendering, convolution, loss, optimiser and metric arithmetic
runs in libmrs.so; this module only orchestrates calls and slices crops.
"""
from __future__ import annotations

import numpy as np
import torch

from . import fusion
from .fusion import NPARAMS
from .render import Scene, render as render_image

LAYERS = [(12, 64)] + [(64, 64)] * 16 + [(64, 3)]


def init_params(seed: int, resid_gain: float = 0.1) -> np.ndarray:
    """Kaiming-normal weights (std sqrt(2 / (9 Cin))) with the second conv of
    every residual block scaled by `resid_gain` and the 3-channel head set to
    zero, so that an untrained network outputs the upsampled LRHS exactly and
    training starts from the method-without-network baseline."""
    rng = np.random.default_rng(np.random.SeedSequence([0x696E6974, int(seed)]))
    parts = []
    for i, (ci, co) in enumerate(LAYERS):
        w = rng.normal(0.0, np.sqrt(2.0 / (9 * ci)), (co, 3, 3, ci))
        if 1 <= i <= 16 and i % 2 == 0:
            w *= resid_gain
        if i == len(LAYERS) - 1:
            w[:] = 0.0
        parts += [w.ravel(), np.zeros(co)]
    p = np.concatenate(parts).astype(np.float32)
    assert p.size == NPARAMS
    return p


def render_example(scene, size, s, spp_lr, spp_hr, spp_tgt, depth, rr, seed, lr_grid=1):
    """One training triple: LRHS [1,size/s,size/s,3], HRLS + albedo + normal
    [1,size,size,3], target [1,size,size,3] (independent seeds per render).
    lr_grid = s renders the LRHS on the sparse grid (nearest-neighbour LR, the
    paper's low-resolution images); 1 jitters over the whole LR pixel."""
    lr = render_image(scene, size // s, size // s, spp_lr, depth, rr, 3 * seed + 0, aux=False,
                       counts=False, grid=lr_grid)["radiance"]
    hr = render_image(scene, size, size, spp_hr, depth, rr, 3 * seed + 1, aux=True, counts=False)
    tg = render_image(scene, size, size, spp_tgt, depth, rr, 3 * seed + 2, aux=False,
                       counts=False)["radiance"]
    return {"lrhs": lr[None], "hrls": hr["radiance"][None], "albedo": hr["albedo"][None],
            "normal": hr["normal"][None], "target": tg[None]}


# spp sets of the method's training (Sec. 4, implementation details): each
# training example draws its HRLS spp and its LRHS spp from these, with the
# HRLS spp below the LRHS spp
SPP_HRLS_SET = (1, 2, 3, 4, 5, 6, 7, 8, 12, 16, 32)
SPP_LRHS_SET = (2, 3, 4, 5, 6, 7, 8, 12, 16, 32, 64, 128, 250, 1000, 4000)


def random_spp_pair(rng, spp_tgt):
    """(spp_lr, spp_hr) drawn uniformly from the two sets with spp_hr <
    spp_lr; LRHS values at or above the target's spp are left out (a noisier
    target than the input would make no sense)."""
    lr_set = [v for v in SPP_LRHS_SET if v < spp_tgt]
    hr_set = [v for v in SPP_HRLS_SET if v < max(lr_set)]
    if not lr_set or not hr_set:
        raise ValueError(f"spp_tgt={spp_tgt} leaves no valid (LRHS, HRLS) spp pair")
    while True:
        hr = int(hr_set[int(rng.integers(len(hr_set)))])
        lr = int(lr_set[int(rng.integers(len(lr_set)))])
        if hr < lr:
            return lr, hr


def make_dataset(scene_seeds, size=256, s=4, spp_lr=64, spp_hr=4, spp_tgt=256, depth=8, rr=3,
                 scene_fn=None, spp_random=False, examples_per_scene=1, seed=0, lr_grid=1):
    """Render `examples_per_scene` examples per procedural scene seed (render
    seeds differ per example); with spp_random each example draws its (LRHS,
    HRLS) spp with random_spp_pair, else uses (spp_lr, spp_hr).  Tensors stay
    on the GPU; each example records its spp under "spp"."""
    from synth import scenes
    scene_fn = scene_fn or (lambda sd: scenes.procedural(sd, n_spheres=24, n_large=8))
    rng = np.random.default_rng(np.random.SeedSequence([0x737070, int(seed)]))
    data = []
    for sd in scene_seeds:
        sc = Scene(scene_fn(sd))
        for e in range(examples_per_scene):
            a, b = random_spp_pair(rng, spp_tgt) if spp_random else (spp_lr, spp_hr)
            ex = render_example(sc, size, s, a, b, spp_tgt, depth, rr, sd + 100003 * e, lr_grid)
            ex["spp"] = (a, b)
            data.append(ex)
        sc.close()
    torch.cuda.synchronize()
    return data


def random_batch(data, batch, crop, s, rng):
    """`batch` random crops (crop x crop HR, aligned to the scale) from `data`."""
    keys = ("lrhs", "hrls", "albedo", "normal", "target")
    out = {k: [] for k in keys}
    for _ in range(batch):
        ex = data[int(rng.integers(len(data)))]
        H = ex["hrls"].shape[1]
        y = int(rng.integers(0, (H - crop) // s + 1)) * s
        x = int(rng.integers(0, (H - crop) // s + 1)) * s
        out["lrhs"].append(ex["lrhs"][:, y // s:(y + crop) // s, x // s:(x + crop) // s])
        for k in keys[1:]:
            out[k].append(ex[k][:, y:y + crop, x:x + crop])
    return {k: torch.cat(v).contiguous() for k, v in out.items()}


def train(net, data, steps, batch=16, crop=128, s=4, lr=1e-4, seed=0, log_every=0, precision="fp32",
          loss=None, beta=0.1):
    """Adam on random crops of `data`; precision "fp32" (SIMT) or "bf16"
    (tensor cores, FP32 master weights); `loss` ("l1log" / "robust"), when
    given, sets the net's training loss first."""
    rng = np.random.default_rng(seed)
    if loss is not None:
        net.set_loss(loss, beta)
    losses = []
    for i in range(steps):
        b = random_batch(data, batch, crop, s, rng)
        sync = bool(log_every) and (i % log_every == 0 or i == steps - 1)
        loss = fusion.train_step(net, b["lrhs"], b["hrls"], b["albedo"], b["normal"], b["target"],
                                 s, lr=lr, sync_loss=sync, precision=precision)
        if sync:
            losses.append((i, loss))
    torch.cuda.synchronize()
    return losses


def evaluate(net, data, s=4, precision="fp32"):
    """Mean sRGB PSNR / RelMSE against the target of: the fused image, the
    method without the network (upsampled LRHS, via a zero-weight network)
    and the HRLS input."""
    zero = fusion.Net(np.zeros(NPARAMS, np.float32))
    acc = {"fused": [], "upsampled_lrhs": [], "hrls": []}
    for ex in data:
        fused = net.fuse(ex["lrhs"], ex["hrls"], ex["albedo"], ex["normal"], s, precision=precision)
        up = zero.fuse(ex["lrhs"], ex["hrls"], ex["albedo"], ex["normal"], s, precision="fp32")
        for k, img in (("fused", fused), ("upsampled_lrhs", up), ("hrls", ex["hrls"])):
            psnr, rel, _ = fusion.image_metrics(img, ex["target"])
            acc[k].append((psnr, rel))
    zero.close()
    return {k: {"psnr": float(np.mean([a for a, _ in v])), "relmse": float(np.mean([b for _, b in v]))}
            for k, v in acc.items()}


# the spp grid of the method's spp study (Sec. 5, Table comp_spp): LRHS spp
# rows, HRLS spp columns, cells with HRLS spp below LRHS spp
SPP_GRID_LRHS = (2, 4, 8, 16, 32, 64, 128)
SPP_GRID_HRLS = (1, 2, 4)


def spp_grid(net, scene_seeds, size=256, s=4, spp_tgt=1024, depth=8, rr=3, lr_spps=SPP_GRID_LRHS,
             hr_spps=SPP_GRID_HRLS, precision="bf16", scene_fn=None, seed=7):
    """Mean sRGB PSNR / RelMSE against a spp_tgt render, over the scenes of
    `scene_seeds`, of the fused image and of the method without the network
    (upsampled LRHS) for every (LRHS spp, HRLS spp) cell with HRLS < LRHS.
    Returns {(lr_spp, hr_spp): {"psnr", "relmse", "up_psnr", "up_relmse"}}."""
    from synth import scenes
    scene_fn = scene_fn or (lambda sd: scenes.procedural(sd, n_spheres=24, n_large=8))
    zero = fusion.Net(np.zeros(NPARAMS, np.float32))
    acc = {}
    for k, sd in enumerate(scene_seeds):
        sc = Scene(scene_fn(sd))
        tgt = render_image(sc, size, size, spp_tgt, depth, rr, 1000 * seed + 3 * k, aux=False,
                           counts=False)["radiance"]
        for a in lr_spps:
            lr = render_image(sc, size // s, size // s, a, depth, rr, 1000 * seed + 3 * k + 1,
                              aux=False, counts=False)["radiance"][None]
            for b in hr_spps:
                if b >= a:
                    continue
                hr = render_image(sc, size, size, b, depth, rr, 1000 * seed + 3 * k + 2, aux=True,
                                  counts=False)
                args = (lr, hr["radiance"][None], hr["albedo"][None], hr["normal"][None], s)
                fused = net.fuse(*args, precision=precision)
                up = zero.fuse(*args, precision="fp32")
                p, r, _ = fusion.image_metrics(fused[0].contiguous(), tgt)
                pu, ru, _ = fusion.image_metrics(up[0].contiguous(), tgt)
                acc.setdefault((a, b), []).append((p, r, pu, ru))
        sc.close()
    zero.close()
    return {key: {"psnr": float(np.mean([v[0] for v in vals])),
                  "relmse": float(np.mean([v[1] for v in vals])),
                  "up_psnr": float(np.mean([v[2] for v in vals])),
                  "up_relmse": float(np.mean([v[3] for v in vals]))}
            for key, vals in acc.items()}


# ----------------------------------------------------------------------------
# the fusion network's training recipe on many seeded scenes: every example
# is a window of a full-resolution frame (the pixel scale the network serves)
# ----------------------------------------------------------------------------
def make_window_dataset(scene_seeds, frame=1024, window=256, s=4, spp_lr=64, spp_hr=4,
                        spp_tgt=1024, depth=8, rr=3, seed=0, scene_kind="procedural"):
    """One example per seeded scene (the library's own generator,
    Scene.seeded): a random window x window crop of the frame x frame image,
    aligned to the scale, rendered as LRHS (the matching window of the
    frame / s image at spp_lr), HRLS + albedo + normal (spp_hr) and a spp_tgt
    target.  Returns the list of examples (tensors on the GPU) and the
    number of paths rendered."""
    rng = np.random.default_rng(np.random.SeedSequence([0x77696E, int(seed)]))
    data, paths = [], 0
    for sd in scene_seeds:
        sc = Scene.seeded(int(sd), scene_kind)
        sc.set_tree("cluster")      # built once, rendered at > 1000 spp: the faster tree
        x0 = int(rng.integers(0, (frame - window) // s + 1)) * s
        y0 = int(rng.integers(0, (frame - window) // s + 1)) * s
        lw = (x0 // s, y0 // s, window // s, window // s)
        hw = (x0, y0, window, window)
        base = 3 * int(sd)
        lr = render_image(sc, frame // s, frame // s, spp_lr, depth, rr, base, aux=False,
                          counts=False, window=lw)["radiance"]
        hr = render_image(sc, frame, frame, spp_hr, depth, rr, base + 1, aux=True, counts=False,
                          window=hw)
        tg = render_image(sc, frame, frame, spp_tgt, depth, rr, base + 2, aux=False, counts=False,
                          window=hw)["radiance"]
        data.append({"lrhs": lr[None], "hrls": hr["radiance"][None], "albedo": hr["albedo"][None],
                     "normal": hr["normal"][None], "target": tg[None], "spp": (spp_lr, spp_hr),
                     "scene": int(sd), "window": hw})
        paths += (window // s) ** 2 * spp_lr + window * window * (spp_hr + spp_tgt)
        sc.close()
    torch.cuda.synchronize()
    return data, paths


def train_recipe(n_scenes=2000, steps=20000, frame=1024, window=256, spp_tgt=1024, batch=16,
                 crop=128, s=4, lr=1e-4, loss="l1log", precision="bf16", eval_scenes=4,
                 eval_size=512, eval_tgt=4096, init_seed=0, log_every=1000):
    """The training recipe end to end: data from n_scenes seeded scenes
    (seeds 1 .. n_scenes), `steps` Adam steps on batch x crop^2 crops with the
    given loss and learning rate, then the gain over the method without the
    network on held-out scenes (seeds 100001 ..; eval_size^2 windows of the
    frame, eval_tgt-spp references).  Returns (net, report dict)."""
    import time
    t0 = time.perf_counter()
    data, paths = make_window_dataset(range(1, 1 + n_scenes), frame, window, s,
                                      spp_tgt=spp_tgt, seed=1)
    t_data = time.perf_counter() - t0
    net = fusion.Net(seed=init_seed)
    t0 = time.perf_counter()
    losses = train(net, data, steps, batch=batch, crop=crop, s=s, lr=lr, seed=0,
                   log_every=log_every, precision=precision, loss=loss)
    t_train = time.perf_counter() - t0
    del data
    ev, _ = make_window_dataset(range(100001, 100001 + eval_scenes), frame, eval_size, s,
                                spp_tgt=eval_tgt, seed=2)
    res = evaluate(net, ev, s=s, precision=precision)
    del ev
    report = {
        "scenes": n_scenes, "frame": frame, "window": window, "spp": [64, 4, spp_tgt],
        "paths_rendered": paths, "data_s": round(t_data, 2),
        "steps": steps, "batch": [batch, crop, crop], "loss": loss, "optimizer": f"Adam lr {lr}",
        "precision": precision, "train_s": round(t_train, 2),
        "ms_per_step": round(1e3 * t_train / max(steps, 1), 3),
        "loss_log": [(int(i), round(float(v), 5)) for i, v in losses],
        "eval": {"scenes": eval_scenes, "size": eval_size, "reference_spp": eval_tgt, **res},
        "gain_db_over_upsampled_lrhs": res["fused"]["psnr"] - res["upsampled_lrhs"]["psnr"],
        "gain_db_over_hrls": res["fused"]["psnr"] - res["hrls"]["psnr"],
    }
    return net, report


def loss_study(n_scenes=160, steps=6000, betas=(0.01, 0.1, 1.0, 100.0), window=256, spp_tgt=1024,
               lr=1e-4, eval_scenes=4, eval_size=512, eval_tgt=4096, seed=0):
    """The method's loss ablation (Sec. 5, Fig. comp_loss): nets trained on the
    same data (n_scenes seeded scenes, one window each, as train_recipe), the
    same batch draws and the same initialisation with the robust loss l_r at
    each beta of `betas` and with L1 on log(1 + x), scored on the same
    held-out windows.  l_r with a large beta (|e| / (beta + |e|) ~ |e| / beta)
    is L1 on radiance up to scale, which Adam does not see.  Returns
    {loss name: {"psnr", "relmse", "gain_db_over_upsampled_lrhs"}}."""
    data, _ = make_window_dataset(range(1, 1 + n_scenes), 1024, window, 4, spp_tgt=spp_tgt, seed=1)
    ev, _ = make_window_dataset(range(100001, 100001 + eval_scenes), 1024, eval_size, 4,
                                spp_tgt=eval_tgt, seed=2)
    runs = [("l1log", "l1log", 0.1)] + [(f"robust_beta_{b:g}", "robust", b) for b in betas]
    out = {}
    for name, loss, beta in runs:
        net = fusion.Net(seed=seed)
        train(net, data, steps, batch=16, crop=128, s=4, lr=lr, seed=0, precision="bf16",
              loss=loss, beta=beta)
        r = evaluate(net, ev, s=4, precision="bf16")
        out[name] = {"psnr": r["fused"]["psnr"], "relmse": r["fused"]["relmse"],
                     "gain_db_over_upsampled_lrhs": r["fused"]["psnr"] - r["upsampled_lrhs"]["psnr"]}
        net.close()
    out["upsampled_lrhs"] = {"psnr": r["upsampled_lrhs"]["psnr"], "relmse": r["upsampled_lrhs"]["relmse"]}
    return out


def main(argv=None):
    """python -m paper_2106_12802_gb300.trainer recipe --scenes 2000 --steps 20000 [--save f]
    python -m paper_2106_12802_gb300.trainer loss-study --scenes 160 --steps 6000"""
    import argparse
    import json
    ap = argparse.ArgumentParser()
    ap.add_argument("cmd", choices=["recipe", "loss-study"])
    ap.add_argument("--scenes", type=int, default=2000)
    ap.add_argument("--steps", type=int, default=20000)
    ap.add_argument("--window", type=int, default=256)
    ap.add_argument("--spp-tgt", type=int, default=1024)
    ap.add_argument("--lr", type=float, default=1e-4)
    ap.add_argument("--loss", default="l1log")
    ap.add_argument("--eval-scenes", type=int, default=4)
    ap.add_argument("--save", default=None, help="checkpoint file for the trained net")
    a = ap.parse_args(argv)
    if a.cmd == "loss-study":
        print(json.dumps(loss_study(a.scenes, a.steps, window=a.window, spp_tgt=a.spp_tgt,
                                    lr=a.lr, eval_scenes=a.eval_scenes)), flush=True)
        return 0
    net, rep = train_recipe(a.scenes, a.steps, window=a.window, spp_tgt=a.spp_tgt, lr=a.lr,
                            loss=a.loss, eval_scenes=a.eval_scenes)
    if a.save:
        fusion.save_checkpoint(net, a.save, seed=0)
    print(json.dumps(rep), flush=True)
    return 0


if __name__ == "__main__":
    import sys
    sys.exit(main())
