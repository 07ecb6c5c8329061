"""Python binding of the method's own fusion network (mrs_rdn_*).

Marshalling only: every computation runs in libmrs.so's kernels.
"""
from __future__ import annotations

import ctypes

import numpy as np
import torch

from ._lib import call, load
from .fusion import LOSSES, _prec
from .render import _dev, _ptr, _stream


def layers(scale: int, hr_channels: int = 9):
    """[(name, k, cin, cout)] in parameter order, as include/mrs.h documents
    it: H_lrhs, H_hrls, fuse (1x1), 3 groups x 5 blocks x 4 convs, the
    log2(scale) upsampling convs, H_Rec."""
    D = {2: 1, 4: 2, 8: 3}[scale]
    L = [("H_lrhs", 3, 3, 64), ("H_hrls", 3, hr_channels, 64), ("fuse", 1, 64 + 64 * scale * scale, 64)]
    L += [(f"rdg{g}.rdb{b}.conv{c}", 3, 64 * c, 64) for g in range(3) for b in range(5)
          for c in range(1, 5)]
    L += [(f"up{d}", 3, 64, 256) for d in range(D)] + [("H_rec", 3, 64, 3)]
    return L


def kaiming_params(scale: int, hr_channels: int = 9, seed: int = 0, fusion_damp: float = 0.1):
    """Kaiming-normal weights (std sqrt(2 / (k^2 Cin))), zero biases, the
    blocks' local-fusion convs scaled by fusion_damp (random weights for
    throughput measurements; each block adds its fusion output to its input)."""
    rng = np.random.default_rng(np.random.SeedSequence([0x6B726E, int(seed), scale, hr_channels]))
    parts = []
    for name, k, ci, co in layers(scale, hr_channels):
        w = rng.normal(0.0, np.sqrt(2.0 / (k * k * ci)), (co, k, k, ci))
        if name.endswith("conv4"):
            w *= fusion_damp
        parts += [w.ravel(), np.zeros(co)]
    return np.concatenate(parts).astype(np.float32)


def flops_per_lr_pixel(scale: int, hr_channels: int = 9) -> int:
    """2 x multiply-adds of one forward pass per LR pixel (H_hrls and H_Rec
    at scale^2 HR pixels, the i-th upsampling conv at 4^i LR pixels)."""
    total, up = 0, 0
    for name, k, ci, co in layers(scale, hr_channels):
        f = 2 * k * k * ci * co
        if name in ("H_hrls", "H_rec"):
            f *= scale * scale
        elif name.startswith("up"):
            f *= 4 ** up
            up += 1
        total += f
    return total


def nparams(scale: int, hr_channels: int = 9) -> int:
    load()
    n = ctypes.c_int64()
    call("mrs_rdn_nparams", int(scale), int(hr_channels), ctypes.byref(n))
    return int(n.value)


class RDN:
    """Two-encoder fusion network of Sec. 4 (H_lrhs, H_hrls + deshuffle, 1x1
    fuse, 3 x 5 residual dense blocks, shuffle upscaling, H_Rec) for one
    scale (2, 4 or 8) and HRLS input width (9, or 18 with the extra layers)."""

    def __init__(self, params, scale: int, hr_channels: int = 9):
        load()
        p = np.ascontiguousarray(params, dtype=np.float32)
        h = ctypes.c_void_p()
        call("mrs_rdn_create", int(scale), int(hr_channels), ctypes.c_void_p(p.ctypes.data),
             int(p.size), ctypes.byref(h))
        self.handle = h
        self.scale = int(scale)
        self.hr_channels = int(hr_channels)

    def close(self):
        if getattr(self, "handle", None):
            call("mrs_rdn_free", self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def fuse(self, lrhs, hrls, albedo, normal, precision="bf16", extra=None, out=None,
             stream=None):
        """lrhs [N,h,w,3], hrls / albedo / normal [N,H,W,3] (extra [N,H,W,9]
        when hr_channels is 18) float32 CUDA tensors -> I_SR [N,H,W,3]."""
        for t in (lrhs, hrls, albedo, normal) + ((extra,) if extra is not None else ()):
            _dev(t, torch.float32)
        N, H, W, _ = hrls.shape
        if out is None:
            out = torch.empty((N, H, W, 3), dtype=torch.float32, device=hrls.device)
        call("mrs_rdn_fuse", self.handle, _ptr(lrhs), _ptr(hrls), _ptr(albedo), _ptr(normal),
             _ptr(extra), N, H, W, _prec(precision), _ptr(out), _stream(stream))
        return out

    def check(self):
        """Raises if a tensor-core wait of an earlier fuse gave up."""
        call("mrs_rdn_check", self.handle)

    @property
    def nparams(self):
        return nparams(self.scale, self.hr_channels)

    def train_step(self, lrhs, hrls, albedo, normal, target, lr=1e-4, loss="robust", beta=0.1,
                   extra=None, out=None, sync_loss=True, precision="fp32", stream=None):
        """One Adam step on a batch (CUDA float32 NHWC tensors as in fuse plus
        target [N,H,W,3]); returns the mean loss, or None when sync_loss is
        False (no host synchronisation).  out [N,H,W,3] receives I_SR."""
        for t in (lrhs, hrls, albedo, normal, target) + ((extra,) if extra is not None else ()):
            _dev(t, torch.float32)
        if out is not None:
            _dev(out, torch.float32)
        N, H, W, _ = hrls.shape
        v = ctypes.c_double()
        call("mrs_rdn_train_step", self.handle, _ptr(lrhs), _ptr(hrls), _ptr(albedo), _ptr(normal),
             _ptr(extra), _ptr(target), N, H, W, LOSSES[loss] if isinstance(loss, str) else int(loss),
             float(beta), float(lr), _prec(precision), _ptr(out),
             ctypes.byref(v) if sync_loss else None, _stream(stream))
        return float(v.value) if sync_loss else None

    def get_grads(self):
        g = np.zeros(self.nparams, np.float32)
        call("mrs_rdn_get_grads", self.handle, ctypes.c_void_p(g.ctypes.data), g.size)
        return g

    def get_state(self):
        p, m, v = (np.zeros(self.nparams, np.float32) for _ in range(3))
        step = ctypes.c_int64()
        call("mrs_rdn_get_state", self.handle, *(ctypes.c_void_p(a.ctypes.data) for a in (p, m, v)),
             p.size, ctypes.byref(step))
        return {"params": p, "adam_m": m, "adam_v": v, "step": int(step.value)}

    def get_params(self):
        return self.get_state()["params"]

    def set_state(self, st):
        p, m, v = (np.ascontiguousarray(st[k], np.float32) for k in ("params", "adam_m", "adam_v"))
        call("mrs_rdn_set_state", self.handle, *(ctypes.c_void_p(a.ctypes.data) for a in (p, m, v)),
             p.size, int(st["step"]))
