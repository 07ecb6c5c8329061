"""Python binding of the fusion-network, metric and gate entry points.

Marshalling only: every computation runs in libmrs.so's kernels.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np
import torch

from ._lib import call, load
from .render import _dev, _ptr, _stream

NPARAMS = 599555
NPARAMS_EXTRA = 604739      # 21 input channels: + diffuse, specular, variance of the HRLS
PREC = {"fp32": 0, "bf16": 1, "fp8": 2}


LOSSES = {"l1log": 0, "robust": 1}


def _prec(p):
    return PREC[p] if isinstance(p, str) else int(p)


class Net:
    """Fusion network handle (FP32 master weights + packed BF16/FP8 copies +
    Adam state) created from a flat float32 parameter array of NPARAMS
    (12 input channels) or NPARAMS_EXTRA values (21: the extra HRLS layers)."""

    def __init__(self, params=None, *, seed=None, input_channels=12, resid_gain=0.1):
        """Net(params) copies a flat parameter array in; Net(seed=k) makes the
        library's seeded initialisation (mrs_net_create_seeded) for a net of
        `input_channels` (12 or 21) input channels."""
        load()
        h = ctypes.c_void_p()
        if params is None:
            if seed is None:
                raise ValueError("give params or seed")
            call("mrs_net_create_seeded", int(input_channels), int(seed), float(resid_gain),
                 ctypes.byref(h))
        else:
            p = np.ascontiguousarray(params, dtype=np.float32)
            assert p.size in (NPARAMS, NPARAMS_EXTRA), p.size
            call("mrs_net_create", ctypes.c_void_p(p.ctypes.data), p.size, ctypes.byref(h))
        self.handle = h
        c = ctypes.c_int32()
        call("mrs_net_input_channels", h, ctypes.byref(c))
        self.input_channels = int(c.value)
        self.nparams = NPARAMS_EXTRA if self.input_channels == 21 else NPARAMS

    def set_loss(self, loss="l1log", beta=0.1):
        """Training loss of train_step: "l1log" (L1 on log(1 + x)) or "robust"
        (the paper's l_r with factor beta)."""
        call("mrs_net_set_loss", self.handle, LOSSES[loss] if isinstance(loss, str) else int(loss),
             float(beta))

    def close(self):
        if getattr(self, "handle", None):
            call("mrs_net_free", self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_params(self, params):
        p = np.ascontiguousarray(params, dtype=np.float32)
        assert p.size == self.nparams
        call("mrs_net_set_params", self.handle, ctypes.c_void_p(p.ctypes.data))

    def get_params(self):
        out = np.zeros(self.nparams, np.float32)
        call("mrs_net_get_params", self.handle, ctypes.c_void_p(out.ctypes.data))
        return out

    def fuse(self, lrhs, hrls, albedo, normal, scale, precision="bf16", out=None, stream=None,
             extra=None):
        """lrhs [N,h,w,3], others [N,H,W,3] float32 CUDA tensors -> [N,H,W,3].
        extra [N,H,W,9] (diffuse, specular, variance) for a 21-channel net."""
        for t in (lrhs, hrls, albedo, normal) + ((extra,) if extra is not None else ()):
            _dev(t, torch.float32)
        N, H, W, _ = hrls.shape
        if out is None:
            out = torch.empty((N, H, W, 3), dtype=torch.float32, device=hrls.device)
        if extra is None:
            call("mrs_fuse", self.handle, _ptr(lrhs), _ptr(hrls), _ptr(albedo), _ptr(normal), N, H,
                 W, scale, _prec(precision), _ptr(out), _stream(stream))
        else:
            call("mrs_fuse_extra", self.handle, _ptr(lrhs), _ptr(hrls), _ptr(albedo), _ptr(normal),
                 _ptr(extra), N, H, W, scale, _prec(precision), _ptr(out), _stream(stream))
        return out


def _np_ptr(a):
    return ctypes.c_void_p(a.ctypes.data)


def train_step(net, lrhs, hrls, albedo, normal, target, scale, lr=1e-4, precision="fp32",
               sync_loss=True, stream=None, loss=None, beta=0.1, extra=None):
    """One Adam step on a batch (CUDA float32 NHWC tensors); returns the loss
    (float) or None when sync_loss is False (no host synchronisation).
    `loss` ("l1log" / "robust"), when given, first sets the net's loss.
    extra [N,H,W,9] for a 21-channel net."""
    for t in (lrhs, hrls, albedo, normal, target) + ((extra,) if extra is not None else ()):
        _dev(t, torch.float32)
    if loss is not None:
        net.set_loss(loss, beta)
    N, H, W, _ = hrls.shape
    loss = ctypes.c_double()
    lp = ctypes.byref(loss) if sync_loss else None
    if extra is None:
        call("mrs_train_step", net.handle, _ptr(lrhs), _ptr(hrls), _ptr(albedo), _ptr(normal),
             _ptr(target), N, H, W, scale, float(lr), _prec(precision), lp, _stream(stream))
    else:
        call("mrs_train_step_extra", net.handle, _ptr(lrhs), _ptr(hrls), _ptr(albedo),
             _ptr(normal), _ptr(extra), _ptr(target), N, H, W, scale, float(lr), _prec(precision),
             lp, _stream(stream))
    return float(loss.value) if sync_loss else None


def get_grads(net):
    out = np.zeros(net.nparams, np.float32)
    call("mrs_net_get_grads", net.handle, _np_ptr(out))
    return out


def get_state(net):
    p, m, v = (np.zeros(net.nparams, np.float32) for _ in range(3))
    step = ctypes.c_int64()
    call("mrs_net_get_state", net.handle, _np_ptr(p), _np_ptr(m), _np_ptr(v), ctypes.byref(step))
    return {"params": p, "adam_m": m, "adam_v": v, "step": int(step.value)}


def set_state(net, st):
    p, m, v = (np.ascontiguousarray(st[k], np.float32) for k in ("params", "adam_m", "adam_v"))
    call("mrs_net_set_state", net.handle, _np_ptr(p), _np_ptr(m), _np_ptr(v), int(st["step"]))




def save_checkpoint(net, path, seed=0):
    """Checkpoint of the net (weights, Adam state and step, loss) and `seed`
    to `path` through mrs_net_save (flat little-endian file with a
    checksum)."""
    call("mrs_net_save", net.handle, os.fsencode(str(path)), int(seed))


def load_checkpoint(net, path):
    """Restores a save_checkpoint file into `net` (mrs_net_load); returns the
    stored seed."""
    seed = ctypes.c_uint64()
    call("mrs_net_load", net.handle, os.fsencode(str(path)), ctypes.byref(seed))
    return int(seed.value)


def conv3x3(x, w, b, relu=False, precision="fp32", stream=None):
    """One 3x3 conv layer: x [N,H,W,cin] CUDA float32, w [cout,3,3,cin], b [cout] numpy."""
    _dev(x, torch.float32)
    N, H, W, cin = x.shape
    w = np.ascontiguousarray(w, np.float32)
    b = np.ascontiguousarray(b, np.float32)
    cout = w.shape[0]
    out = torch.empty((N, H, W, cout), dtype=torch.float32, device=x.device)
    call("mrs_conv3x3", _ptr(x), N, H, W, cin, cout, ctypes.c_void_p(w.ctypes.data),
         ctypes.c_void_p(b.ctypes.data), int(relu), _prec(precision), _ptr(out), _stream(stream))
    return out


def conv3x3_wgrad(x, dy, precision="fp32", stream=None):
    """Weight / bias gradients of a 3x3 conv: x [N,H,W,cin], dy [N,H,W,cout]
    CUDA float32 -> (dw [cout,3,3,cin], db [cout]) numpy float32."""
    _dev(x, torch.float32)
    _dev(dy, torch.float32)
    N, H, W, cin = x.shape
    cout = dy.shape[3]
    if tuple(dy.shape[:3]) != (N, H, W):
        raise ValueError("x and dy must share N, H, W")
    dw = np.zeros((cout, 3, 3, cin), np.float32)
    db = np.zeros(cout, np.float32)
    call("mrs_conv3x3_wgrad", _ptr(x), _ptr(dy), N, H, W, cin, cout, _prec(precision),
         ctypes.c_void_p(dw.ctypes.data), ctypes.c_void_p(db.ctypes.data), _stream(stream))
    return dw, db


def conv_set_ring(stages: int):
    """Input-row ring depth of every later tensor-core conv launch (0: the
    most that fits; 3 .. 12 otherwise).  Results do not depend on it."""
    call("mrs_conv_set_ring", int(stages))


DGRAD_MODES = {"linear": 0, "relu_mask": 1, "residual": 2}


def conv3x3_dgrad(dy, w, mode="linear", aux=None, precision="fp32", stream=None):
    """Input gradient of a 3x3 conv with the training step's epilogue:
    dy [N,H,W,cout] CUDA float32, w [cout,3,3,cin] numpy, aux [N,H,W,cin]
    CUDA float32 (the ReLU output for "relu_mask", the incoming gradient for
    "residual") -> out [N,H,W,cin] CUDA float32."""
    _dev(dy, torch.float32)
    N, H, W, cout = dy.shape
    w = np.ascontiguousarray(w, np.float32)
    if w.shape[0] != cout:
        raise ValueError("w must be [cout, 3, 3, cin] with cout = dy.shape[3]")
    cin = w.shape[3]
    if aux is not None:
        _dev(aux, torch.float32)
        if tuple(aux.shape) != (N, H, W, cin):
            raise ValueError("aux must be [N, H, W, cin]")
    out = torch.empty((N, H, W, cin), dtype=torch.float32, device=dy.device)
    call("mrs_conv3x3_dgrad", _ptr(dy), N, H, W, cin, cout, ctypes.c_void_p(w.ctypes.data),
         DGRAD_MODES[mode], _ptr(aux) if aux is not None else None, _prec(precision), _ptr(out),
         _stream(stream))
    return out


def image_metrics(x, ref, lam1=0.5, lam2=0.01, stream=None):
    """(sRGB PSNR, RelMSE, linear MSE) reduced in float64 on the GPU."""
    _dev(x, torch.float32)
    _dev(ref, torch.float32)
    out = (ctypes.c_double * 3)()
    call("mrs_image_metrics", _ptr(x), _ptr(ref), x.numel(), lam1, lam2, out, _stream(stream))
    return float(out[0]), float(out[1]), float(out[2])


def gate_async(fused, lrhs, plain, scale, tau=0.01, out=None, used=None, D=None, stream=None):
    """Device-side fallback gate (no host sync; capturable).  Returns (out,
    used[int32 x2 device], D[float64 device])."""
    N, H, W, _ = fused.shape
    if out is None:
        out = torch.empty_like(fused)
    if used is None:
        used = torch.zeros(2, dtype=torch.int32, device=fused.device)
    if D is None:
        D = torch.zeros(1, dtype=torch.float64, device=fused.device)
    call("mrs_gate_async", _ptr(fused), _ptr(lrhs), _ptr(plain), N, H, W, scale, float(tau),
         _ptr(out), _ptr(used), _ptr(D), _stream(stream))
    return out, used, D


def gate(fused, lrhs, plain, scale, tau=0.01, out=None, stream=None):
    """Fallback gate: returns (out, used_plain, D)."""
    N, H, W, _ = fused.shape
    if out is None:
        out = torch.empty_like(fused)
    used = ctypes.c_int32()
    D = ctypes.c_double()
    call("mrs_gate", _ptr(fused), _ptr(lrhs), _ptr(plain), N, H, W, scale, float(tau), _ptr(out),
         ctypes.byref(used), ctypes.byref(D), _stream(stream))
    return out, bool(used.value), float(D.value)
