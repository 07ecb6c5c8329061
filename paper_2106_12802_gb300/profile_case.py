"""Small, self-contained cases of the hot kernels, for profilers (ncu).

This is the package's profiling entry point: every command recorded under
profiles/ runs one of these cases.

  python -m paper_2106_12802_gb300.profile_case fuse   --size 1024 --prec bf16
  python -m paper_2106_12802_gb300.profile_case render --size 512 --spp 4 [--tree hcluster]
  python -m paper_2106_12802_gb300.profile_case rdn    --size 1024 --prec bf16
  python -m paper_2106_12802_gb300.profile_case train  --batch 16 --crop 128
  python -m paper_2106_12802_gb300.profile_case rdn_train --batch 16 --crop 192 --prec bf16
  python -m paper_2106_12802_gb300.profile_case tree   --kind cluster

`fuse` runs the x4 fusion network at size x size output (inputs random,
Kaiming weights); `rdn` the method's own x4 two-encoder network (the same);
`render` renders the 200k-triangle procedural scene (seed 0, depth 8, roulette
from bounce 3; over the radix tree, or --tree cluster / hcluster) and prints its per-bounce ray counts, whose bounce >= 1 part is
the number of closest-hit segments the tail kernel traces (the unit that a
traffic capture of one tail launch is divided by); `train` runs BF16 training
steps of the fusion network on a random batch; `rdn_train` training steps of
the method's own x4 network (the paper's batch: 16 crops of 192^2; a BF16
step after the first replays its recorded graph); `tree` rebuilds the
procedural scene's render tree (--kind lbvh or cluster).  Each case runs one
warm-up call first, so the second call's launches are steady-state (ncu: skip
the first call's launches with -s).
"""
from __future__ import annotations

import argparse
import json
import os
import sys

import numpy as np


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("case", choices=["fuse", "render", "rdn", "train", "rdn_train", "tree"])
    ap.add_argument("--kind", default="cluster")
    ap.add_argument("--tree", default="lbvh")
    ap.add_argument("--size", type=int, default=1024)
    ap.add_argument("--prec", default="bf16")
    ap.add_argument("--spp", type=int, default=4)
    ap.add_argument("--depth", type=int, default=8)
    ap.add_argument("--batch", type=int, default=16)
    ap.add_argument("--crop", type=int, default=128)
    a = ap.parse_args(argv)
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import torch

    import paper_2106_12802_gb300 as mrs
    from synth import scenes

    if a.case == "fuse":
        rng = np.random.default_rng(0)
        params = (rng.normal(0, 1, mrs.NPARAMS) * 0.03).astype(np.float32)
        net = mrs.Net(params)
        H = W = a.size
        s = 4
        g = torch.Generator(device="cuda").manual_seed(0)
        lr = torch.rand((1, H // s, W // s, 3), device="cuda", generator=g)
        hr = torch.rand((1, H, W, 3), device="cuda", generator=g)
        for _ in range(2):
            out = net.fuse(lr, hr, hr, hr, s, precision=a.prec)
        torch.cuda.synchronize()
        print("fuse ok", float(out.abs().mean()))
    elif a.case == "rdn":
        from paper_2106_12802_gb300 import rdn
        s = 4
        net = mrs.RDN(rdn.kaiming_params(s), s)
        H = W = a.size
        g = torch.Generator(device="cuda").manual_seed(0)
        lr = torch.rand((1, H // s, W // s, 3), device="cuda", generator=g)
        hr = torch.rand((1, H, W, 3), device="cuda", generator=g)
        for _ in range(2):
            out = net.fuse(lr, hr, hr, hr, precision=a.prec)
        torch.cuda.synchronize()
        net.check()
        print("rdn ok", float(out.abs().mean()))
    elif a.case == "train":
        from paper_2106_12802_gb300 import trainer
        s = 4
        N, c = a.batch, a.crop
        g = torch.Generator(device="cuda").manual_seed(11)
        t = [torch.rand((N, c // s, c // s, 3), device="cuda", generator=g) * 2] + \
            [torch.rand((N, c, c, 3), device="cuda", generator=g) for _ in range(4)]
        net = mrs.Net(trainer.init_params(0))
        for _ in range(2):
            loss = mrs.train_step(net, *t, s, lr=1e-4, precision=a.prec)
        print("train ok", loss)
    elif a.case == "rdn_train":
        from paper_2106_12802_gb300 import rdn
        s = 4
        N, c = a.batch, a.crop
        net = mrs.RDN(rdn.kaiming_params(s), s)
        g = torch.Generator(device="cuda").manual_seed(12)
        t = [torch.rand((N, c // s, c // s, 3), device="cuda", generator=g) * 2] + \
            [torch.rand((N, c, c, 3), device="cuda", generator=g) for _ in range(4)]
        for _ in range(2):
            loss = net.train_step(*t, lr=1e-4, loss="robust", beta=0.1, precision=a.prec)
        print("rdn_train ok", loss)
    elif a.case == "tree":
        sc = mrs.Scene(scenes.procedural(0))
        sc.set_tree(a.kind)
        for _ in range(2):
            sc.rebuild()
        torch.cuda.synchronize()
        print("tree ok", sc.tree())
    else:
        sc = mrs.Scene(scenes.procedural(0))
        sc.set_tree(a.tree)
        for _ in range(2):
            r = mrs.render(sc, a.size, a.size, a.spp, a.depth, rr_start=3, seed=0)
        torch.cuda.synchronize()
        counts = r["counts"].cpu().numpy().astype(np.int64)
        print(json.dumps({"render": [a.size, a.size, a.spp, a.depth],
                          "mean": float(r["radiance"].mean()),
                          "counts": counts.tolist(),
                          "tail_segments": int(counts[1:].sum())}))
    return 0


if __name__ == "__main__":
    sys.exit(main())
