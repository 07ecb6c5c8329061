"""Float64 oracle of the image metrics and the hybrid-render fallback gate.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

* srgb: linear -> sRGB transfer of Eq. cvt_color (Sec. 3.2).
* relmse: lambda1 * (I_SR - I_HR)^2 / (I_HR^2 + lambda2), averaged over all
  pixels and channels (Sec. 5; lambda1 = 0.5, lambda2 = 0.01 for the paper's
  own dataset, 1 and 1e-4 for the Gharbi protocol).
* psnr: 10 log10(1 / MSE) of the sRGB images (peak 1), Sec. 5.
* spp_avg: spp_LRHS / s^2 + spp_HRLS (Sec. 5.1).
* clip: firefly clipping of radiance at 100 (Sec. 3.2).
* box_down and gate: the fused image, box-downsampled by s, is compared with
  LRHS by RelMSE; above the threshold the plain render is used instead.

Pins (tests/test_oracle_metrics.py): hand-computed values on 2x2 images, the
piecewise branches of Eq. cvt_color at their boundaries, identical images
(RelMSE 0, PSNR +inf), and a fused image off by a known factor for the gate.
"""
from __future__ import annotations

import numpy as np


def srgb(lin):
    l = np.asarray(lin, dtype=np.float64)
    out = np.where(l <= 0.0, 0.0, 12.92 * l)
    mid = (l > 0.0031308) & (l < 1.0)
    out = np.where(mid, 1.055 * np.power(np.where(mid, l, 1.0), 1.0 / 2.4) - 0.055, out)
    return np.where(l >= 1.0, 1.0, out)


def clamp01(lin):
    """Gharbi-protocol transfer: s = min(1, max(0, l))."""
    return np.clip(np.asarray(lin, dtype=np.float64), 0.0, 1.0)


def relmse(x, ref, lam1=0.5, lam2=0.01):
    x = np.asarray(x, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    return float(np.mean(lam1 * (x - ref) ** 2 / (ref * ref + lam2)))


def psnr(x, ref, transfer=srgb):
    mse = float(np.mean((transfer(x) - transfer(ref)) ** 2))
    return float("inf") if mse == 0.0 else 10.0 * np.log10(1.0 / mse)


def spp_avg(spp_lrhs, spp_hrls, s):
    return spp_lrhs / (s * s) + spp_hrls


def clip(x, limit=100.0):
    return np.minimum(np.asarray(x, dtype=np.float64), limit)


def box_down(x, s):
    """Mean over each s x s block of an [..., H, W, C] image."""
    x = np.asarray(x, dtype=np.float64)
    *lead, H, W, C = x.shape
    return x.reshape(*lead, H // s, s, W // s, s, C).mean(axis=(-4, -2))


def gate(fused, lrhs, s, tau=0.01):
    """(use_plain, D) with D = RelMSE(box_down(fused, s), LRHS)."""
    d = relmse(box_down(fused, s), lrhs)
    return d > tau, d
