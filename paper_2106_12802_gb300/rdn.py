"""Python binding of the method's own fusion network (mrs_rdn_*).

Marshalling only: every computation runs in libmrs.so's kernels.
"""
from __future__ import annotations

import ctypes

import numpy as np
import torch

from ._lib import call, load
from .fusion import _prec
from .render import _dev, _ptr, _stream


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
