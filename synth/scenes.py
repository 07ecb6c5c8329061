"""Seeded synthetic scenes: the shared input generator of the renderer.

This module only *describes* scenes (triangles, materials, lights, camera).  It
holds none of the rendering arithmetic; both the CUDA path and the CPU oracle
consume the arrays it returns.  Every value is produced in float64 and rounded
once to float32, so a scene is a pure function of its arguments.  The two
measured workloads (cornell_box, procedural) come from scenegen.c, which the
CUDA library also links for its seeded scene build; the small analytic test
scenes are built here in numpy.

Scene dictionary (all arrays C-contiguous):

  V          float32 [N, 3, 3]  triangle vertices v0, v1, v2 (world space)
  tri_mat    int32   [N]        material index per triangle
  tri_light  int32   [N]        index of the area light the triangle belongs
                                to, or -1 (used for MIS of BSDF-sampled hits)
  mats       float32 [M, 8]     type (0 Lambert, 1 GGX), albedo rgb, GGX alpha,
                                emitted radiance rgb (one-sided, along the
                                triangle's geometric normal cross(v1-v0, v2-v0))
  lights     float32 [L, 12]    quad lights: p0, e1, e2, Le (point = p0+u e1+v e2,
                                emitting along normalize(cross(e1, e2)))
  env        float32 [3]        constant environment radiance
  cam        float32 [12]       eye, forward, right * tan(fov/2) * aspect,
                                up * tan(fov/2)

The two workloads are the ones the renderer is measured on: a Cornell box of
5 Lambertian quads, two r=0.25 spheres (one Lambert, one GGX alpha 0.3) and one
Le=15 quad light; and a procedural field of 64 noise-displaced icospheres on a
ground plane (about 200k triangles) under 3 quad lights and an environment of
0.5.  The paper renders its scenes with Blender Cycles (Sec. 3.1-3.2); these
procedural stand-ins replace its dataset.
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
import threading

import numpy as np

LAMBERT = 0
GGX = 1

# --------------------------------------------------------------------------
# geometry helpers (float64)
# --------------------------------------------------------------------------


def _icosahedron():
    t = (1.0 + math.sqrt(5.0)) / 2.0
    v = np.array([
        [-1, t, 0], [1, t, 0], [-1, -t, 0], [1, -t, 0],
        [0, -1, t], [0, 1, t], [0, -1, -t], [0, 1, -t],
        [t, 0, -1], [t, 0, 1], [-t, 0, -1], [-t, 0, 1],
    ], dtype=np.float64)
    v /= np.linalg.norm(v, axis=1, keepdims=True)
    f = np.array([
        [0, 11, 5], [0, 5, 1], [0, 1, 7], [0, 7, 10], [0, 10, 11],
        [1, 5, 9], [5, 11, 4], [11, 10, 2], [10, 7, 6], [7, 1, 8],
        [3, 9, 4], [3, 4, 2], [3, 2, 6], [3, 6, 8], [3, 8, 9],
        [4, 9, 5], [2, 4, 11], [6, 2, 10], [8, 6, 7], [9, 8, 1],
    ], dtype=np.int64)
    return v, f


_ICO_CACHE: dict[int, tuple[np.ndarray, np.ndarray]] = {}


def icosphere(subdiv: int):
    """Unit icosphere with 20 * 4**subdiv outward-wound faces (float64)."""
    if subdiv in _ICO_CACHE:
        return _ICO_CACHE[subdiv]
    v, f = _icosahedron()
    verts = [tuple(x) for x in v]
    for _ in range(subdiv):
        cache: dict[tuple[int, int], int] = {}

        def mid(a, b):
            key = (a, b) if a < b else (b, a)
            if key in cache:
                return cache[key]
            p = (np.array(verts[a]) + np.array(verts[b])) * 0.5
            p /= np.linalg.norm(p)
            verts.append(tuple(p))
            cache[key] = len(verts) - 1
            return cache[key]

        nf = []
        for a, b, c in f:
            ab, bc, ca = mid(a, b), mid(b, c), mid(c, a)
            nf += [[a, ab, ca], [b, bc, ab], [c, ca, bc], [ab, bc, ca]]
        f = np.array(nf, dtype=np.int64)
    out = (np.array(verts, dtype=np.float64), f)
    _ICO_CACHE[subdiv] = out
    return out


def _quad_tris(p0, e1, e2):
    """Two triangles covering p0 + [0,1] e1 + [0,1] e2, wound so that their
    geometric normal is along cross(e1, e2)."""
    p0, e1, e2 = (np.asarray(x, dtype=np.float64) for x in (p0, e1, e2))
    a, b, c, d = p0, p0 + e1, p0 + e1 + e2, p0 + e2
    return np.array([[a, b, c], [a, c, d]], dtype=np.float64)


def camera(eye, target, up, fov_deg, aspect=1.0):
    eye, target, up = (np.asarray(x, dtype=np.float64) for x in (eye, target, up))
    fwd = target - eye
    fwd /= np.linalg.norm(fwd)
    right = np.cross(fwd, up)
    right /= np.linalg.norm(right)
    upv = np.cross(right, fwd)
    th = math.tan(math.radians(fov_deg) * 0.5)
    return np.concatenate([eye, fwd, right * th * aspect, upv * th]).astype(np.float32)


class _Builder:
    def __init__(self):
        self.tris: list[np.ndarray] = []
        self.tri_mat: list[np.ndarray] = []
        self.tri_light: list[np.ndarray] = []
        self.mats: list[list[float]] = []
        self.lights: list[np.ndarray] = []

    def material(self, kind, albedo, alpha=1.0, Le=(0.0, 0.0, 0.0)):
        self.mats.append([float(kind), *map(float, albedo), float(alpha), *map(float, Le)])
        return len(self.mats) - 1

    def add(self, tris, mat, light=-1):
        tris = np.asarray(tris, dtype=np.float64).reshape(-1, 3, 3)
        self.tris.append(tris)
        self.tri_mat.append(np.full(len(tris), mat, dtype=np.int32))
        self.tri_light.append(np.full(len(tris), light, dtype=np.int32))

    def quad_light(self, p0, e1, e2, Le):
        li = len(self.lights)
        self.lights.append(np.concatenate([p0, e1, e2, Le]).astype(np.float64))
        m = self.material(LAMBERT, (0, 0, 0), 1.0, Le)
        self.add(_quad_tris(p0, e1, e2), m, li)

    def finish(self, env, cam):
        V = np.concatenate(self.tris) if self.tris else np.zeros((0, 3, 3))
        return {
            "V": np.ascontiguousarray(V, dtype=np.float32),
            "tri_mat": np.ascontiguousarray(np.concatenate(self.tri_mat) if self.tri_mat
                                            else np.zeros(0), dtype=np.int32),
            "tri_light": np.ascontiguousarray(np.concatenate(self.tri_light) if self.tri_light
                                              else np.zeros(0), dtype=np.int32),
            "mats": np.ascontiguousarray(np.array(self.mats, dtype=np.float32).reshape(-1, 8)),
            "lights": np.ascontiguousarray(np.array(self.lights, dtype=np.float32).reshape(-1, 12)),
            "env": np.asarray(env, dtype=np.float32).reshape(3).copy(),
            "cam": np.asarray(cam, dtype=np.float32).reshape(12).copy(),
        }


# --------------------------------------------------------------------------
# scenes
# --------------------------------------------------------------------------


# --------------------------------------------------------------------------
# the measured workloads: generated by scenegen.c (the same code the CUDA
# library links for its seeded scene build)
# --------------------------------------------------------------------------
_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "libsynth.so")
_lock = threading.Lock()
_lib = None
CORNELL, PROCEDURAL = 0, 1


class _Params(ctypes.Structure):
    _fields_ = [("n_spheres", ctypes.c_int32), ("n_large", ctypes.c_int32),
                ("sphere_subdiv", ctypes.c_int32), ("aspect", ctypes.c_float)]


def build(force: bool = False) -> str:
    """Compile scenegen.c into synth/_build/libsynth.so (gcc, -ffp-contract=off)."""
    src = [os.path.join(_HERE, f) for f in ("scenegen.c", "scenegen.h")]
    if not force and os.path.exists(_SO) and all(os.path.getmtime(_SO) >= os.path.getmtime(f)
                                                 for f in src):
        return _SO
    os.makedirs(_BUILD, exist_ok=True)
    tmp = _SO + f".{os.getpid()}.tmp"
    subprocess.run(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-shared",
                    "-fPIC", "-o", tmp, src[0], "-lm"], check=True)
    os.replace(tmp, _SO)
    return _SO


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = ctypes.CDLL(_SO)
            P = ctypes.c_void_p
            L.synth_scene_counts.argtypes = [ctypes.c_int32, ctypes.POINTER(_Params), P, P, P]
            L.synth_scene_counts.restype = ctypes.c_int
            L.synth_scene_generate.argtypes = [ctypes.c_uint64, ctypes.c_int32,
                                               ctypes.POINTER(_Params), P, P, P, P, P, P, P]
            L.synth_scene_generate.restype = ctypes.c_int
            _lib = L
    return _lib


def generate(kind: int, seed: int = 0, n_spheres: int = 64, n_large: int = 31,
             sphere_subdiv: int = 4, aspect: float = 1.0):
    """The scene dictionary of scenegen.c for (kind, seed, parameters)."""
    L = _load()
    prm = _Params(n_spheres, n_large, sphere_subdiv, aspect)
    nt, nm, nl = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32()
    if L.synth_scene_counts(kind, ctypes.byref(prm), ctypes.byref(nt), ctypes.byref(nm),
                            ctypes.byref(nl)):
        raise ValueError("invalid scene kind or parameters")
    d = {"V": np.zeros((nt.value, 3, 3), np.float32), "tri_mat": np.zeros(nt.value, np.int32),
         "tri_light": np.zeros(nt.value, np.int32), "mats": np.zeros((nm.value, 8), np.float32),
         "lights": np.zeros((nl.value, 12), np.float32), "env": np.zeros(3, np.float32),
         "cam": np.zeros(12, np.float32)}
    p = [ctypes.c_void_p(d[k].ctypes.data) for k in ("V", "tri_mat", "tri_light", "mats", "lights",
                                                      "env", "cam")]
    if L.synth_scene_generate(int(seed) & (2**64 - 1), kind, ctypes.byref(prm), *p):
        raise RuntimeError("scene generation failed")
    return d


def cornell_box(sphere_subdiv: int = 4, aspect: float = 1.0):
    """Cornell box: 5 Lambertian quads (white 0.75, red/green 0.6), a Lambert
    and a GGX (alpha 0.3) sphere of radius 0.25, one quad light with Le=15.

    Box spans x in [-1,1], y in [0,2], z in [-1,1]; the camera looks down -z.
    """
    return generate(CORNELL, 0, sphere_subdiv=sphere_subdiv, aspect=aspect)


def procedural(seed: int, n_spheres: int = 64, n_large: int = 31, aspect: float = 1.0):
    """Seeded field of noise-displaced icospheres on a ground plane.

    64 spheres with radius U(0.1, 1) placed in a 20 x 20 area; the n_large
    largest (ties by index) use subdivision 4 (5120 tris), the rest 3 (1280),
    so the default scene has 31*5120 + 33*1280 + 2 = 200,962 triangles plus
    6 light triangles.  Displacement is value noise of amplitude 0.2*r.
    Materials are 50/50 Lambert/GGX with alpha U(0.05, 1) and albedo
    U(0.1, 0.9) per channel; 3 quad lights with Le U(5, 20) facing down;
    environment 0.5.
    """
    return generate(PROCEDURAL, seed, n_spheres=n_spheres, n_large=n_large, aspect=aspect)


def furnace_sphere(Le: float, rho: float, subdiv: int = 2):
    """Closed emissive Lambertian sphere (inward normals), camera at its centre:
    every path sees Le * sum_k rho^k exactly (white-furnace closed form)."""
    b = _Builder()
    m = b.material(LAMBERT, (rho, rho, rho), 1.0, (Le, Le, Le))
    v, f = icosphere(subdiv)
    b.add(v[f][:, ::-1, :] * 5.0, m)   # reversed winding: normals point inward
    cam = camera((0, 0, 0), (0, 0, -1), (0, 1, 0), 60.0)
    return b.finish((0.0, 0.0, 0.0), cam)


def sky_plane(rho: float, L_sky: float):
    """Large diffuse plane under a uniform sky, viewed straight down through a
    narrow field of view (all camera rays hit the plane): L = rho * L_sky."""
    b = _Builder()
    m = b.material(LAMBERT, (rho, rho, rho))
    b.add(_quad_tris((-50, 0, -50), (0, 0, 100), (100, 0, 0)), m)
    cam = camera((0, 5, 0), (0, 0, 0), (0, 0, -1), 30.0)
    return b.finish((L_sky, L_sky, L_sky), cam)


LIGHTS_OVER_PLANE = (
    # p0, e1, e2, Le of two disjoint quads at height 1 facing down
    # (cross(e1, e2) = x^ x z^ = -y); different areas and colours
    ((-0.7, 1.0, -0.5), (0.5, 0.0, 0.0), (0.0, 0.0, 0.8), (6.0, 3.0, 1.5)),
    ((0.1, 1.0, -0.2), (0.4, 0.0, 0.0), (0.0, 0.0, 0.6), (2.0, 5.0, 8.0)),
)


def lights_over_plane(kind: int = LAMBERT, albedo=(0.6, 0.6, 0.6), alpha: float = 1.0,
                      env: float = 0.3):
    """A large plane y = 0 under the two quad lights of LIGHTS_OVER_PLANE and a
    uniform environment, seen straight down by a camera at height 0.5 (below
    the lights, which stay out of view): every camera ray hits the plane, and
    at one scattering event its pixel sees only direct light."""
    b = _Builder()
    m = b.material(kind, albedo, alpha)
    b.add(_quad_tris((-50, 0, -50), (0, 0, 100), (100, 0, 0)), m)
    for p0, e1, e2, le in LIGHTS_OVER_PLANE:
        b.quad_light(np.array(p0), np.array(e1), np.array(e2), np.array(le))
    cam = camera((0.0, 0.5, 0.0), (0.0, 0.0, 0.0), (0, 0, -1), 50.0)
    return b.finish((env, env, env), cam)


def random_triangles(seed: int, n: int, spread: float = 1.0, size: float = 0.3):
    """n random triangles in a cube (for BVH / intersection tests)."""
    rng = np.random.default_rng(np.random.SeedSequence([0x747269, int(seed)]))
    c = rng.uniform(-spread, spread, (n, 1, 3))
    V = c + rng.uniform(-size, size, (n, 3, 3))
    b = _Builder()
    m = b.material(LAMBERT, (0.5, 0.5, 0.5))
    b.add(V, m)
    cam = camera((0, 0, 4 * spread), (0, 0, 0), (0, 1, 0), 40.0)
    return b.finish((0.0, 0.0, 0.0), cam)


def random_rays(seed: int, n: int, spread: float = 1.0):
    """n rays (origin, unit direction) aimed through a cube of half-size spread."""
    rng = np.random.default_rng(np.random.SeedSequence([0x726179, int(seed)]))
    o = rng.normal(size=(n, 3))
    o = o / np.linalg.norm(o, axis=1, keepdims=True) * (3.0 * spread)
    tgt = rng.uniform(-spread, spread, (n, 3))
    d = tgt - o
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    return o.astype(np.float32), d.astype(np.float32)
