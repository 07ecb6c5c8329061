"""Small, self-contained cases of the hot kernels for profilers (ncu).

  python -m paper_2106_12802_gb300.profile_case fuse   --size 1024 --prec bf16
  python -m paper_2106_12802_gb300.profile_case render --size 256 --spp 4
  python -m paper_2106_12802_gb300.profile_case rdn    --size 1024 --prec bf16

`fuse` runs the x4 fusion network once at size x size output (inputs random,
Kaiming weights); `rdn` the method's own x4 two-encoder network (the same);
`render` renders the 200k-triangle procedural scene once.
Each case runs one warm-up call first, so the profiled launches are steady-state.
"""
from __future__ import annotations

import argparse
import os
import sys

import numpy as np


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("case", choices=["fuse", "render", "rdn"])
    ap.add_argument("--size", type=int, default=1024)
    ap.add_argument("--prec", default="bf16")
    ap.add_argument("--spp", type=int, default=4)
    ap.add_argument("--depth", type=int, default=8)
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
    else:
        sc = mrs.Scene(scenes.procedural(0))
        for _ in range(2):
            r = mrs.render(sc, a.size, a.size, a.spp, a.depth, rr_start=3, seed=0)
        torch.cuda.synchronize()
        print("render ok", float(r["radiance"].mean()))
    return 0


if __name__ == "__main__":
    sys.exit(main())
