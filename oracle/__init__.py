"""CPU oracle of the multi-resolution sampling renderer and fusion network.

TEST INFRASTRUCTURE ONLY: the slow, obviously-correct reference the CUDA
library is checked against.  It shares no code with the CUDA path; only
`tests/`, `__graft_entry__.smoke()` and `bench.py`'s CPU-baseline leg may
import it.  The product path never routes through it.

* `render`, `lbvh`, `cast`, `philox*`: ctypes wrappers over `orc_pt.c`, a plain
  C path tracer compiled with -ffp-contract=off (see that file's header).
* `cnn`: the fusion network forward/backward, loss and Adam in float64 numpy.
* `rdn`: the method's own two-encoder fusion network (Sec. 4) forward in
  float64 numpy.
* `metrics`: linear->sRGB (Eq. cvt_color), RelMSE and PSNR (Sec. 5), average
  spp (Sec. 5.1), box downsampling and the fallback gate.

Functions whose results are not fixed by a closed form or library routine are
still pinned by tests: see each module's header.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "liborc.so")
_lock = threading.Lock()
_est_lock = threading.Lock()   # the estimator switch is process-global in orc_pt.c
_lib = None


def build(force: bool = False) -> str:
    """Compile orc_pt.c into oracle/_build/liborc.so (gcc, -ffp-contract=off)."""
    src = os.path.join(_HERE, "orc_pt.c")
    if not force and os.path.exists(_SO) and os.path.getmtime(_SO) >= os.path.getmtime(src):
        return _SO
    os.makedirs(_BUILD, exist_ok=True)
    tmp = _SO + f".{os.getpid()}.tmp"
    cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fopenmp",
           "-shared", "-fPIC", "-o", tmp, src, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _SO)
    return _SO


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = ctypes.CDLL(_SO)
            P = ctypes.c_void_p
            i32, u32, u64 = ctypes.c_int, ctypes.c_uint32, ctypes.c_uint64
            L.orc_philox4x32_10.argtypes = [P, P, P]
            L.orc_philox_uniforms.argtypes = [u32, u32, u32, u64, P]
            L.orc_sincos2pi.argtypes = [P, i32, P, P]
            L.orc_morton.argtypes = [P, i32, P]
            L.orc_lbvh.argtypes = [P, i32, P, P, P, P, P]
            L.orc_lbvh.restype = i32
            L.orc_cast.argtypes = [P, i32, P, P, i32, i32, P, P]
            L.orc_cast.restype = i32
            L.orc_render.argtypes = [P, i32, P, P, P, P, i32, P, P, i32, i32, i32, i32, i32,
                                     i32, u64, i32, i32, i32, i32, P, P, P, P, P, P, P, P, P]
            L.orc_render.restype = i32
            L.orc_num_threads.restype = i32
            L.orc_set_estimator.argtypes = [i32]
            L.orc_bsdf_eval_batch.argtypes = [P, P, P, i32, P, P]
            L.orc_bsdf_sample_batch.argtypes = [P, P, P, i32, P, P, P, P]
            _lib = L
    return _lib


def _p(a):
    return ctypes.c_void_p(a.ctypes.data) if a is not None else None


def philox4x32_10(ctr, key):
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    out = np.zeros(4, dtype=np.uint32)
    lib().orc_philox4x32_10(_p(c), _p(k), _p(out))
    return out


def philox_uniforms(pixel: int, sample: int, bounce: int, seed: int):
    """The 8 uniforms of one (pixel, sample, bounce): dims 0..7."""
    out = np.zeros(8, dtype=np.float32)
    lib().orc_philox_uniforms(pixel, sample, bounce, seed, _p(out))
    return out


def sincos2pi(u):
    u = np.ascontiguousarray(u, dtype=np.float32)
    c = np.zeros_like(u)
    s = np.zeros_like(u)
    lib().orc_sincos2pi(_p(u), u.size, _p(c), _p(s))
    return c, s


def morton(V):
    V = np.ascontiguousarray(V, dtype=np.float32)
    out = np.zeros(len(V), dtype=np.uint32)
    lib().orc_morton(_p(V), len(V), _p(out))
    return out


def lbvh(V):
    """Returns dict(morton, order, left, right, box) of the binary radix tree."""
    V = np.ascontiguousarray(V, dtype=np.float32)
    n = len(V)
    r = {
        "morton": np.zeros(n, np.uint32),
        "order": np.zeros(n, np.int32),
        "left": np.zeros(max(n - 1, 0), np.int32),
        "right": np.zeros(max(n - 1, 0), np.int32),
        "box": np.zeros((max(2 * n - 1, 0), 6), np.float32),
    }
    if n:
        rc = lib().orc_lbvh(_p(V), n, _p(r["morton"]), _p(r["order"]),
                            _p(r["left"]) if n > 1 else None,
                            _p(r["right"]) if n > 1 else None, _p(r["box"]))
        assert rc == 0
    return r


def cast(V, orig, dirs, brute: bool = False):
    """Closest hit per ray through the LBVH (or by brute force)."""
    V = np.ascontiguousarray(V, dtype=np.float32)
    o = np.ascontiguousarray(orig, dtype=np.float32)
    d = np.ascontiguousarray(dirs, dtype=np.float32)
    prim = np.zeros(len(o), np.int32)
    t = np.zeros(len(o), np.float32)
    rc = lib().orc_cast(_p(V), len(V), _p(o), _p(d), len(o), int(brute), _p(prim), _p(t))
    assert rc == 0
    return prim, t


def bsdf_eval(mat, wo, wi):
    """f (without cosine) [n,3] and sampling pdf [n] of one material row
    (type, albedo rgb, alpha, Le rgb) for local directions wo, wi [n,3]
    (shading normal +z)."""
    m = np.ascontiguousarray(mat, dtype=np.float32).reshape(8)
    wo = np.ascontiguousarray(np.broadcast_to(wo, np.shape(wi)), dtype=np.float32)
    wi = np.ascontiguousarray(wi, dtype=np.float32)
    n = len(wi)
    f = np.zeros((n, 3), np.float32)
    pdf = np.zeros(n, np.float32)
    lib().orc_bsdf_eval_batch(_p(m), _p(wo), _p(wi), n, _p(f), _p(pdf))
    return f, pdf


def bsdf_sample(mat, wo, u):
    """Sample wi for local wo [n,3] with uniforms u [n,2]: returns wi [n,3],
    weight = f cos / pdf [n,3], pdf [n] and ok [n] (False: below the surface)."""
    m = np.ascontiguousarray(mat, dtype=np.float32).reshape(8)
    u = np.ascontiguousarray(u, dtype=np.float32)
    n = len(u)
    wo = np.ascontiguousarray(np.broadcast_to(wo, (n, 3)), dtype=np.float32)
    wi = np.zeros((n, 3), np.float32)
    wt = np.zeros((n, 3), np.float32)
    pdf = np.zeros(n, np.float32)
    ok = np.zeros(n, np.int32)
    lib().orc_bsdf_sample_batch(_p(m), _p(wo), _p(u), n, _p(wi), _p(wt), _p(pdf), _p(ok))
    return wi, wt, pdf, ok.astype(bool)


ESTIMATORS = {"mis": 0, "light": 1, "bsdf": 2}


def num_threads() -> int:
    return int(lib().orc_num_threads())


def render(scene, W, H, spp, max_depth, rr_start=None, seed=0, rows=None, threads=0, grid=1,
           estimator="mis"):
    """Path-trace the scene; returns dict(radiance[H,W,3], albedo, normal,
    depth[H,W], counts[max_depth+1], shadow_counts[max_depth+1]).

    rr_start=None disables Russian roulette.  rows=(r0, r1) renders only those
    image rows (the result then has r1-r0 rows), rows=(r0, r1, step) only every
    step-th of them -- used for bounded samples.
    grid=g > 1 samples each pixel only inside the centre sub-pixel of its g x g
    block (nearest-neighbour downsampling of a g-times finer render).
    Also returns the extra layers diffuse, specular and variance [H,W,3]:
    the radiance of the samples whose first hit is Lambertian / GGX, and the
    per-channel sample variance of the pixel mean.

    estimator selects how lights and the environment are reached: "mis" (the
    renderer's: next-event estimation and BSDF sampling, power heuristic),
    "light" (next-event estimation only) or "bsdf" (BSDF sampling only).  The
    last two exist to test the first: all three estimate the same integral."""
    if rr_start is None:
        rr_start = 1 << 30
    r0, r1, step = (0, H, 1) if rows is None else (tuple(rows) + (1,))[:3]
    h = max(0, (r1 - r0 + step - 1) // step)
    out = {
        "radiance": np.zeros((h, W, 3), np.float32),
        "albedo": np.zeros((h, W, 3), np.float32),
        "normal": np.zeros((h, W, 3), np.float32),
        "depth": np.zeros((h, W), np.float32),
        "diffuse": np.zeros((h, W, 3), np.float32),
        "specular": np.zeros((h, W, 3), np.float32),
        "variance": np.zeros((h, W, 3), np.float32),
        "counts": np.zeros(max_depth + 1, np.uint64),
        "shadow_counts": np.zeros(max_depth + 1, np.uint64),
    }
    s = scene
    L = lib()
    with _est_lock:
        L.orc_set_estimator(ESTIMATORS[estimator])
        try:
            rc = _render_call(s, W, H, spp, max_depth, rr_start, grid, seed, r0, r1, step, threads,
                              out)
        finally:
            L.orc_set_estimator(0)
    if rc != 0:
        raise ValueError(f"orc_render failed ({rc})")
    return out


def _render_call(s, W, H, spp, max_depth, rr_start, grid, seed, r0, r1, step, threads, out):
    return lib().orc_render(_p(s["V"]), len(s["V"]), _p(s["tri_mat"]), _p(s["tri_light"]),
                          _p(s["mats"]), _p(s["lights"]), len(s["lights"]), _p(s["env"]),
                          _p(s["cam"]), W, H, spp, max_depth, rr_start, grid, seed, r0, r1, step,
                          threads,
                          _p(out["radiance"]), _p(out["albedo"]), _p(out["normal"]),
                          _p(out["depth"]), _p(out["diffuse"]), _p(out["specular"]),
                          _p(out["variance"]), _p(out["counts"]), _p(out["shadow_counts"]))
