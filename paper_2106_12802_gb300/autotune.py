"""Autotuner for the launch parameters the library exposes, with a JSON cache.

Tunable parameters:
  * the render wave size (paths per wave: the capacity of the wavefront's ray
    queues and the size of the path-state arena; for a batch, how many jobs'
    samples share one set of launches) -- Scene.set_wave / RenderContext.set_wave
  * the first bounce of the render's persistent tail kernel -- set_tail
  * the input-row ring depth of the tensor-core convolution (how far the TMA
    producer runs ahead of the MMAs) -- fusion.conv_set_ring
The traversal kernels' block size (256 threads, 8 resident blocks per SM at 32
registers) and the convolution's tile (one 128-pixel row, the MMA's M) are
fixed by the kernels' register and tensor-memory layouts.

A tuning run times a workload (a callable) under each candidate setting with
CUDA events and keeps the fastest; results are keyed by (workload key, SM
count) and stored in a JSON file (cache=None: no file).
"""
from __future__ import annotations

import json
import os

import torch

from .render import render

DEFAULT_CACHE = os.path.join(os.path.expanduser("~"), ".cache", "mrs_autotune.json")
WAVE_CANDIDATES = (1 << 22, 1 << 23, 1 << 24, 1 << 25)
TAIL_CANDIDATES = (0, 1, 2)
RING_CANDIDATES = (4, 6, 8, 0)


def _sms():
    return torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count


def _load(path):
    try:
        with open(path) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def _store(path, db):
    os.makedirs(os.path.dirname(path), exist_ok=True)
    with open(path, "w") as f:
        json.dump(db, f, indent=1)


def tune(key, candidates, apply, run, reps=2, warmup=1, cache=DEFAULT_CACHE):
    """Times run() under each candidate setting (apply(candidate) first; the
    candidates are JSON-able values), leaves the fastest applied and returns
    (best, {candidate: ms}).  A cached result for (key, SM count) is applied
    without timing."""
    full = f"{key}:sm{_sms()}"
    db = _load(cache) if cache else {}
    if full in db:
        best = db[full]["best"]
        apply(best)
        return best, db[full]["ms"]
    times = {}
    for c in candidates:
        apply(c)
        for _ in range(warmup):
            run()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(reps):
            run()
        e1.record()
        torch.cuda.synchronize()
        times[json.dumps(c)] = e0.elapsed_time(e1) / reps
    best = json.loads(min(times, key=times.get))
    apply(best)
    if cache:
        db[full] = {"best": best, "ms": times}
        _store(cache, db)
    return best, times


def tune_wave(scene, W, H, spp, depth, rr=None, cache=DEFAULT_CACHE, candidates=WAVE_CANDIDATES,
              reps=2):
    """The fastest wave size for one render shape (set on the scene); returns
    (wave, {candidate: ms})."""
    out = render(scene, W, H, spp, depth, rr, 0, aux=False, counts=False)
    cands = [c for c in candidates if c >= W * H or c == candidates[0]]
    seed = iter(range(1, 1 << 30))
    return tune(f"render_wave:{W}x{H}:spp{spp}:d{depth}", cands, scene.set_wave,
                lambda: render(scene, W, H, spp, depth, rr, next(seed), out=out), reps=reps,
                cache=cache)
