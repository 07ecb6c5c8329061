"""Autotuner for launch parameters the library exposes, with a JSON cache.

Currently: the render wave size (paths per wave, which sizes the path-state
arena and sets how many sample passes share one wavefront).  Results are keyed
by (parameter, image size, spp, depth, SM count) and stored in a JSON file.
"""
from __future__ import annotations

import json
import os

import torch

from .render import render

DEFAULT_CACHE = os.path.join(os.path.expanduser("~"), ".cache", "mrs_autotune.json")
WAVE_CANDIDATES = (1 << 22, 1 << 23, 1 << 24, 1 << 25)


def _key(W, H, spp, depth):
    sms = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    return f"render_wave:{W}x{H}:spp{spp}:d{depth}:sm{sms}"


def _load(path):
    try:
        with open(path) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def tune_wave(scene, W, H, spp, depth, rr=None, cache=DEFAULT_CACHE, candidates=WAVE_CANDIDATES,
              reps=2):
    """Pick the fastest wave size for this render shape (timed with CUDA
    events), set it on the scene and return (wave, {candidate: ms})."""
    db = _load(cache) if cache else {}
    key = _key(W, H, spp, depth)
    if key in db:
        scene.set_wave(db[key]["wave"])
        return db[key]["wave"], db[key]["ms"]
    out = render(scene, W, H, spp, depth, rr, 0, aux=False, counts=False)
    times = {}
    for c in candidates:
        if c < W * H and c != candidates[0]:
            continue
        scene.set_wave(c)
        render(scene, W, H, spp, depth, rr, 1, out=out)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for k in range(reps):
            render(scene, W, H, spp, depth, rr, 2 + k, out=out)
        e1.record()
        torch.cuda.synchronize()
        times[c] = e0.elapsed_time(e1) / reps
    best = min(times, key=times.get)
    scene.set_wave(best)
    if cache:
        db[key] = {"wave": best, "ms": {str(k): v for k, v in times.items()}}
        os.makedirs(os.path.dirname(cache), exist_ok=True)
        with open(cache, "w") as f:
            json.dump(db, f, indent=1)
    return best, times
