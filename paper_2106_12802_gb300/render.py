"""Python binding of the scene / LBVH / path-tracing entry points.

Marshalling only: every computation runs in libmrs.so's kernels.
"""
from __future__ import annotations

import ctypes

import numpy as np
import torch

from ._lib import call, load


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else None


def _hptr(a):
    return ctypes.c_void_p(a.ctypes.data) if a is not None and a.size else None


def _stream(stream=None):
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _dev(t, dtype):
    assert t.is_cuda and t.dtype == dtype and t.is_contiguous(), (t.device, t.dtype)
    return t


class _SceneParams(ctypes.Structure):
    _fields_ = [("n_spheres", ctypes.c_int32), ("n_large", ctypes.c_int32),
                ("sphere_subdiv", ctypes.c_int32), ("aspect", ctypes.c_float)]


SCENE_KINDS = {"cornell": 0, "procedural": 1}


class Scene:
    """Device-resident scene + LBVH (mrs_build_scene).  `desc` is the dict of
    arrays produced by the seeded scene generators; Scene.seeded builds a
    generated scene inside the library instead (mrs_build_scene_seeded)."""

    @classmethod
    def seeded(cls, seed, kind="procedural", n_spheres=64, n_large=31, sphere_subdiv=4,
               aspect=1.0, stream=None):
        load()
        self = cls.__new__(cls)
        prm = _SceneParams(n_spheres, n_large, sphere_subdiv, aspect)
        h = ctypes.c_void_p()
        call("mrs_build_scene_seeded", int(seed) & (2**64 - 1), SCENE_KINDS[kind],
             ctypes.byref(prm), _stream(stream), ctypes.byref(h))
        self.handle = h
        self.desc = None
        k = SCENE_KINDS[kind]
        if k == 0:
            self.n = 12 + 2 * 20 * 4 ** sphere_subdiv
        else:
            self.n = 2 + n_large * 5120 + (n_spheres - n_large) * 1280 + 6
        return self

    def __init__(self, desc, stream=None):
        load()
        self.desc = desc
        self.n = int(len(desc["V"]))
        V = np.ascontiguousarray(desc["V"], np.float32)
        tm = np.ascontiguousarray(desc["tri_mat"], np.int32)
        tl = np.ascontiguousarray(desc["tri_light"], np.int32)
        mats = np.ascontiguousarray(desc["mats"], np.float32)
        lights = np.ascontiguousarray(desc["lights"], np.float32)
        env = np.ascontiguousarray(desc["env"], np.float32)
        cam = np.ascontiguousarray(desc["cam"], np.float32)
        h = ctypes.c_void_p()
        call("mrs_build_scene", _hptr(V), self.n, _hptr(tm), _hptr(tl), _hptr(mats), len(mats),
             _hptr(lights), len(lights), _hptr(env), _hptr(cam), _stream(stream), ctypes.byref(h))
        self.handle = h

    def close(self):
        if getattr(self, "handle", None):
            call("mrs_free_scene", self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def rebuild(self, stream=None):
        call("mrs_scene_rebuild", self.handle, _stream(stream))

    def update_vertices(self, V, stream=None):
        """Upload new vertices (pinned or pageable host float32 [n,3,3] array or
        CPU tensor) and rebuild the LBVH."""
        if isinstance(V, torch.Tensor):
            assert V.device.type == "cpu" and V.dtype == torch.float32 and V.is_contiguous()
            ptr = ctypes.c_void_p(V.data_ptr())
        else:
            V = np.ascontiguousarray(V, np.float32)
            ptr = ctypes.c_void_p(V.ctypes.data)
        call("mrs_scene_update_vertices", self.handle, ptr, self.n, _stream(stream))

    def set_wave(self, paths: int):
        call("mrs_scene_set_wave", self.handle, int(paths))

    def set_tail(self, bounce: int):
        """First bounce of the tail kernel (-1: automatic; > max_depth: none)."""
        call("mrs_scene_set_tail", self.handle, int(bounce))

    TREES = {"lbvh": 0, "cluster": 1, "hcluster": 2}

    def set_tree(self, kind: str = "cluster", stream=None):
        """Render tree: "lbvh" (the radix tree, the default: cheapest build),
        "cluster" (locally-ordered clustering in grid-wide rounds: faster
        renders, slower build) or "hcluster" (the same clustering inside the
        radix tree's subtrees, one launch); rebuilds it."""
        call("mrs_scene_set_tree", self.handle, self.TREES[kind], _stream(stream))

    def tree(self) -> str:
        """The render tree in use ("lbvh" also when clustering gave up)."""
        k = ctypes.c_int32()
        call("mrs_scene_get_tree", self.handle, ctypes.byref(k))
        return {v: n for n, v in self.TREES.items()}[k.value]

    def export_nodes(self):
        """The render tree: dict(ns, box [ns-1, 2, 6] child boxes, child
        [ns-1, 2] ids (< ns - 1 internal, else leaf ns - 1 + k), order [ns])."""
        ns = ctypes.c_int32()
        call("mrs_scene_export_nodes", self.handle, None, 0, None, ctypes.byref(ns))
        ns = int(ns.value)
        raw = np.zeros((max(ns - 1, 1), 16), np.float32)
        order = np.zeros(max(ns, 1), np.int32)
        call("mrs_scene_export_nodes", self.handle, ctypes.c_void_p(raw.ctypes.data), raw.size,
             ctypes.c_void_p(order.ctypes.data), ctypes.byref(ctypes.c_int32()))
        raw = raw[: max(ns - 1, 0)]
        return {"ns": ns, "box": raw[:, :12].reshape(-1, 2, 6).copy(),
                "child": raw[:, 12:14].copy().view(np.int32), "order": order[:ns]}

    def export_bvh(self, stream=None):
        n = self.n
        dev = torch.device("cuda")
        out = {
            "morton": torch.zeros(n, dtype=torch.int32, device=dev),
            "order": torch.zeros(n, dtype=torch.int32, device=dev),
            "left": torch.zeros(max(n - 1, 1), dtype=torch.int32, device=dev),
            "right": torch.zeros(max(n - 1, 1), dtype=torch.int32, device=dev),
            "box": torch.zeros((max(2 * n - 1, 1), 6), dtype=torch.float32, device=dev),
        }
        call("mrs_scene_export_bvh", self.handle, _ptr(out["morton"]), _ptr(out["order"]),
             _ptr(out["left"]), _ptr(out["right"]), _ptr(out["box"]), _stream(stream))
        torch.cuda.synchronize()
        r = {k: v.cpu().numpy() for k, v in out.items()}
        r["morton"] = r["morton"].view(np.uint32)
        r["left"] = r["left"][: max(n - 1, 0)]
        r["right"] = r["right"][: max(n - 1, 0)]
        r["box"] = r["box"][: max(2 * n - 1, 0)]
        return r

    def cast(self, orig, dirs, stream=None):
        o = _dev(orig, torch.float32)
        d = _dev(dirs, torch.float32)
        n = o.shape[0]
        prim = torch.empty(n, dtype=torch.int32, device=o.device)
        t = torch.empty(n, dtype=torch.float32, device=o.device)
        call("mrs_cast", self.handle, _ptr(o), _ptr(d), n, _ptr(prim), _ptr(t), _stream(stream))
        return prim, t


class RenderContext:
    """A path-state arena of its own (mrs_ctx): renders of one scene through
    different contexts may run concurrently on different streams."""

    def __init__(self):
        load()
        h = ctypes.c_void_p()
        call("mrs_ctx_create", ctypes.byref(h))
        self.handle = h

    def set_wave(self, paths: int):
        call("mrs_ctx_set_wave", self.handle, int(paths))

    def set_tail(self, bounce: int):
        """First bounce of the tail kernel (-1: automatic; > max_depth: none)."""
        call("mrs_ctx_set_tail", self.handle, int(bounce))

    def close(self):
        if getattr(self, "handle", None):
            call("mrs_ctx_free", self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class _RenderOut(ctypes.Structure):
    _fields_ = [(k, ctypes.c_void_p) for k in ("radiance", "albedo", "normal", "depth", "diffuse",
                                               "specular", "variance", "counts", "shadow_counts")]


def render(scene: Scene, W, H, spp, max_depth, rr_start=None, seed=0, aux=True, counts=True,
           out=None, stream=None, ctx: RenderContext | None = None, grid=1, layers=False,
           window=None):
    """mrs_render (or mrs_render_ctx when ctx is given) into device tensors;
    returns dict of (device) tensors.  grid > 1 renders on the sparse
    camera-sampling grid (mrs_render_grid): each pixel samples only the centre
    sub-pixel of its grid x grid block, the paper's nearest-neighbour LR.
    layers=True also returns the extra HRLS layers diffuse, specular and
    variance (mrs_render_layers).  window=(x0, y0, w, h) renders only that
    window of the W x H image (mrs_render_window; outputs [h, w, ...])."""
    dev = torch.device("cuda")
    if window is not None:
        x0, y0, ww, hh = (int(v) for v in window)
        if out is None:
            out = {"radiance": torch.empty((hh, ww, 3), dtype=torch.float32, device=dev)}
            if aux:
                out["albedo"] = torch.empty((hh, ww, 3), dtype=torch.float32, device=dev)
                out["normal"] = torch.empty((hh, ww, 3), dtype=torch.float32, device=dev)
                out["depth"] = torch.empty((hh, ww), dtype=torch.float32, device=dev)
            if counts:
                out["counts"] = torch.zeros(max_depth + 1, dtype=torch.int64, device=dev)
                out["shadow_counts"] = torch.zeros(max_depth + 1, dtype=torch.int64, device=dev)
            if layers:
                for k in ("diffuse", "specular", "variance"):
                    out[k] = torch.empty((hh, ww, 3), dtype=torch.float32, device=dev)
        ro = _RenderOut(*[_ptr(out.get(k)) for k, _ in _RenderOut._fields_])
        call("mrs_render_window", ctx.handle if ctx is not None else None, scene.handle, W, H, x0,
             y0, ww, hh, spp, max_depth, -1 if rr_start is None else rr_start,
             int(seed) & 0xFFFFFFFFFFFFFFFF, int(grid), ctypes.byref(ro), _stream(stream))
        return out
    if out is None:
        out = {"radiance": torch.empty((H, W, 3), dtype=torch.float32, device=dev)}
        if aux:
            out["albedo"] = torch.empty((H, W, 3), dtype=torch.float32, device=dev)
            out["normal"] = torch.empty((H, W, 3), dtype=torch.float32, device=dev)
            out["depth"] = torch.empty((H, W), dtype=torch.float32, device=dev)
        if counts:
            out["counts"] = torch.zeros(max_depth + 1, dtype=torch.int64, device=dev)
            out["shadow_counts"] = torch.zeros(max_depth + 1, dtype=torch.int64, device=dev)
        if layers:
            for k in ("diffuse", "specular", "variance"):
                out[k] = torch.empty((H, W, 3), dtype=torch.float32, device=dev)
    bufs = (_ptr(out["radiance"]), _ptr(out.get("albedo")), _ptr(out.get("normal")),
            _ptr(out.get("depth")), _ptr(out.get("counts")), _ptr(out.get("shadow_counts")),
            _stream(stream))
    head = (W, H, spp, max_depth, -1 if rr_start is None else rr_start, int(seed) & 0xFFFFFFFFFFFFFFFF)
    args = head + bufs
    if any(k in out for k in ("diffuse", "specular", "variance")):
        ro = _RenderOut(*[_ptr(out.get(k)) for k, _ in _RenderOut._fields_])
        call("mrs_render_layers", ctx.handle if ctx is not None else None, scene.handle, *head,
             int(grid), ctypes.byref(ro), _stream(stream))
    elif grid != 1:
        call("mrs_render_grid", ctx.handle if ctx is not None else None, scene.handle, *head,
             int(grid), *bufs)
    elif ctx is None:
        call("mrs_render", scene.handle, *args)
    else:
        call("mrs_render_ctx", ctx.handle, scene.handle, *args)
    return out


class _RenderJob(ctypes.Structure):
    _fields_ = [("scene", ctypes.c_void_p), ("W", ctypes.c_int32), ("H", ctypes.c_int32),
                ("spp", ctypes.c_int32), ("max_depth", ctypes.c_int32),
                ("rr_start", ctypes.c_int32), ("seed", ctypes.c_uint64), ("grid", ctypes.c_int32),
                ("radiance", ctypes.c_void_p), ("albedo", ctypes.c_void_p),
                ("normal", ctypes.c_void_p), ("depth", ctypes.c_void_p)]


def render_batch(ctx, jobs, stream=None):
    """mrs_render_batch: jobs is a list of dicts with scene, W, H, spp,
    max_depth, and optionally rr_start, seed, grid, aux (default True) and
    out (dict of device tensors).  Returns the list of output dicts
    (radiance [H,W,3]; albedo, normal [H,W,3], depth [H,W] when aux)."""
    dev = torch.device("cuda")
    arr = (_RenderJob * len(jobs))()
    outs = []
    for i, j in enumerate(jobs):
        W, H = int(j["W"]), int(j["H"])
        out = j.get("out")
        if out is None:
            out = {"radiance": torch.empty((H, W, 3), dtype=torch.float32, device=dev)}
            if j.get("aux", True):
                out["albedo"] = torch.empty((H, W, 3), dtype=torch.float32, device=dev)
                out["normal"] = torch.empty((H, W, 3), dtype=torch.float32, device=dev)
                out["depth"] = torch.empty((H, W), dtype=torch.float32, device=dev)
        rr = j.get("rr_start")
        arr[i] = _RenderJob(j["scene"].handle.value, W, H, int(j["spp"]), int(j["max_depth"]),
                            -1 if rr is None else int(rr), int(j.get("seed", 0)) & (2**64 - 1),
                            int(j.get("grid", 1)), _ptr(out["radiance"]).value,
                            *[(_ptr(out[k]).value if out.get(k) is not None else None)
                              for k in ("albedo", "normal", "depth")])
        outs.append(out)
    call("mrs_render_batch", ctx.handle, arr, len(jobs), _stream(stream))
    return outs


def render_stats(scene: Scene, W, H, spp, max_depth, rr_start=None, seed=0, stream=None):
    """Node visits / triangle tests of the closest-hit and shadow traversals
    (all bounces), and the part of them done in the tail kernel (tail_*)."""
    dev = torch.device("cuda")
    rad = torch.empty((H, W, 3), dtype=torch.float32, device=dev)
    st = torch.zeros(8, dtype=torch.int64, device=dev)
    call("mrs_render_stats", scene.handle, W, H, spp, max_depth, -1 if rr_start is None else rr_start,
         int(seed), _ptr(rad), _ptr(st), _stream(stream))
    v = st.cpu().tolist()
    names = ("visits", "tests", "shadow_visits", "shadow_tests")
    out = dict(zip(names, v[:4]))
    out.update({"tail_" + k: x for k, x in zip(names, v[4:])})
    return out


PROFILE_KERNELS = ["trace", "shade", "shadow", "raygen", "accumulate", "tree", "conv_tc",
                   "conv_simt", "input", "metrics", "train", "wgrad_tc", "tail"]


def profile_enable(on=True):
    call("mrs_profile_enable", int(bool(on)))


def profile_read():
    """{kernel family: (total ms, launches)} since the last read (synchronises)."""
    out = {}
    for i, name in enumerate(PROFILE_KERNELS):
        ms = ctypes.c_double()
        n = ctypes.c_int64()
        call("mrs_profile_read", i, ctypes.byref(ms), ctypes.byref(n))
        out[name] = (float(ms.value), int(n.value))
    return out


def philox_uniforms(triples, seed, stream=None):
    tr = _dev(triples, torch.int32)
    n = tr.shape[0]
    out = torch.empty((n, 8), dtype=torch.float32, device=tr.device)
    call("mrs_philox_uniforms", _ptr(tr), n, int(seed), _ptr(out), _stream(stream))
    return out
