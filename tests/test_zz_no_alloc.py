"""The allocation-free LBVH build (mrs_lbvh_build_static) against the regular
build (mrs_build_scene + mrs_scene_export_bvh), through the C ABI.

Some callers cannot allocate device memory: code running inside another
allocator's callback, under a reservation that forbids new allocations, or in a
frame loop that must not stall on cudaMalloc.  For them the library keeps the
build's scratch in a static device array.  The outputs must be bit-identical to
the LBVH that mrs_scene_export_bvh returns for the same triangles, on two calls
in a row (the second call reuses the array with the first call's leftovers in
it), from one triangle up to the array's capacity, and sizes above the
capacity must be refused.  This file is collected last on purpose.
"""
import ctypes

import numpy as np
import pytest

from synth import scenes

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mrs():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2106_12802_gb300 as m
    m.load()
    return m


CAP = 262144   # MRS_LBVH_STATIC_MAX_TRIS


def _static_build(lib, V, null_children=False):
    n = V.shape[0]
    dev = torch.device("cuda")
    Vd = torch.from_numpy(np.ascontiguousarray(V, np.float32)).to(dev)
    out = {
        "morton": torch.empty(n, dtype=torch.int32, device=dev),
        "order": torch.empty(n, dtype=torch.int32, device=dev),
        "left": torch.empty(max(n - 1, 1), dtype=torch.int32, device=dev),
        "right": torch.empty(max(n - 1, 1), dtype=torch.int32, device=dev),
        "box": torch.empty((2 * n - 1, 6), dtype=torch.float32, device=dev),
    }
    p = {k: ctypes.c_void_p(v.data_ptr()) for k, v in out.items()}
    if null_children:   # one triangle has no internal node: left/right may be NULL
        p["left"] = p["right"] = None
    st = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    rc = lib.mrs_lbvh_build_static(ctypes.c_void_p(Vd.data_ptr()), n, p["morton"], p["order"],
                                   p["left"], p["right"], p["box"], st)
    assert rc == 0, lib.mrs_last_error()
    torch.cuda.synchronize()
    r = {k: v.cpu().numpy() for k, v in out.items()}
    r["morton"] = r["morton"].view(np.uint32)
    r["left"] = r["left"][: n - 1]
    r["right"] = r["right"][: n - 1]
    return r


@pytest.mark.parametrize("kind", ["procedural", "random"])
def test_static_build_matches_regular_build_twice(mrs, kind):
    lib = mrs.load()
    desc = scenes.procedural(0) if kind == "procedural" else scenes.random_triangles(9, 3001)
    ref = mrs.Scene(desc).export_bvh()
    for _ in range(2):
        got = _static_build(lib, desc["V"])
        for k in ("morton", "order", "left", "right"):
            assert np.array_equal(got[k], ref[k]), k
        assert np.array_equal(got["box"].view(np.uint32), ref["box"].view(np.uint32))


@pytest.mark.parametrize("n", [1, 2, CAP])
def test_static_build_edge_sizes_twice(mrs, n):
    # one triangle (no internal node, NULL child arrays), two, and exactly the
    # capacity (every scratch region filled to its end, all sort tiles used)
    lib = mrs.load()
    desc = scenes.random_triangles(17 + n, n, spread=4.0 if n == CAP else 1.0,
                                   size=0.02 if n == CAP else 0.3)
    ref = mrs.Scene(desc).export_bvh()
    for _ in range(2):
        got = _static_build(lib, desc["V"], null_children=(n == 1))
        keys = ("morton", "order") if n == 1 else ("morton", "order", "left", "right")
        for k in keys:
            assert np.array_equal(got[k], ref[k]), k
        assert np.array_equal(got["box"].view(np.uint32), ref["box"].view(np.uint32))


def test_static_build_rejects_oversize(mrs):
    lib = mrs.load()
    cap = CAP
    rc = lib.mrs_lbvh_build_static(None, cap + 1, None, None, None, None, None, None)
    assert rc == -5   # MRS_ERR_CAPACITY
    assert b"MRS_LBVH_STATIC_MAX_TRIS" in lib.mrs_last_error()
