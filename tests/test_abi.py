"""CPU checks of the C-ABI library: it builds, loads, exports every entry point
declared in include/*.h, and rejects invalid arguments before touching CUDA."""
import ctypes
import glob
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = open(h).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        names |= set(re.findall(r"\b(mrs_[a-z0-9_]+)\s*\(", src))
    return names


@pytest.fixture(scope="module")
def lib():
    from paper_2106_12802_gb300 import _lib
    return _lib.load()


def test_header_declares_entry_points():
    names = declared_symbols()
    for want in ("mrs_build_scene", "mrs_render", "mrs_free_scene", "mrs_status_string"):
        assert want in names


def test_library_exports_every_declared_symbol(lib):
    from paper_2106_12802_gb300 import _lib
    out = subprocess.run(["nm", "-D", "--defined-only", _lib.library_path()],
                         capture_output=True, text=True, check=True).stdout
    exported = set(re.findall(r"\b(mrs_[a-z0-9_]+)\b", out))
    missing = declared_symbols() - exported
    assert not missing, missing
    for name in declared_symbols():
        assert hasattr(lib, name)


def test_binding_signatures_cover_header():
    from paper_2106_12802_gb300 import _lib
    assert declared_symbols() <= set(_lib.SIGS)


def test_invalid_arguments_rejected_without_cuda(lib):
    assert lib.mrs_status_string(0) == b"ok"
    assert lib.mrs_status_string(-1) == b"invalid argument"
    # NULL scene handle
    assert lib.mrs_render(None, 8, 8, 1, 1, -1, 0, None, None, None, None, None, None, None) == -1
    assert b"scene" in lib.mrs_last_error()
    assert lib.mrs_scene_rebuild(None, None) == -1
    # NULL out pointer, negative sizes
    assert lib.mrs_build_scene(None, 0, None, None, None, 0, None, 0, None, None, None, None) == -1
    h = ctypes.c_void_p()
    assert lib.mrs_build_scene(None, -5, None, None, None, 0, None, 0, None, None, None,
                               ctypes.byref(h)) == -1
    assert lib.mrs_philox_uniforms(None, -1, 0, None, None) == -1
    assert lib.mrs_free_scene(None) == 0
    # tail-kernel switch: NULL handles, out-of-range bounce
    assert lib.mrs_scene_set_tail(None, 1) == -1
    assert lib.mrs_ctx_set_tail(None, 1) == -1
    assert lib.mrs_status_string(-7) == b"invalid checkpoint file"
    assert lib.mrs_status_string(-8) == b"file I/O error"


def test_boundary_calls_of_the_method_reject_bad_arguments(lib):
    # the seeded scene build, checkpoint save / load and the seeded network
    # refuse invalid arguments before any device work
    from paper_2106_12802_gb300.render import _SceneParams
    h = ctypes.c_void_p()
    assert lib.mrs_build_scene_seeded(0, 1, None, None, None) == -1           # out NULL
    assert lib.mrs_build_scene_seeded(0, 7, None, None, ctypes.byref(h)) == -1  # unknown kind
    for prm in (_SceneParams(0, 0, 4, 1.0), _SceneParams(64, 65, 4, 1.0),
                _SceneParams(64, 31, 4, 0.0), _SceneParams(64, 31, 7, 1.0)):
        kind = 0 if prm.sphere_subdiv == 7 else 1
        assert lib.mrs_build_scene_seeded(3, kind, ctypes.byref(prm), None, ctypes.byref(h)) == -1
        assert h.value is None
    assert lib.mrs_render_batch(None, None, 0, None) == -1                    # no context
    assert lib.mrs_render_window(None, None, 8, 8, 0, 0, 4, 4, 1, 1, -1, 0, 1, None, None) == -1
    assert lib.mrs_net_save(None, b"/nonexistent/x.ckpt", 0) == -1
    assert lib.mrs_net_load(None, b"x.ckpt", None) == -1
    assert lib.mrs_net_create_seeded(13, 0, ctypes.c_float(0.1), ctypes.byref(h)) == -1
    assert lib.mrs_net_create_seeded(12, 0, ctypes.c_float(2.0), ctypes.byref(h)) == -1
    assert lib.mrs_net_create_seeded(12, 0, ctypes.c_float(0.1), None) == -1


def test_rdn_host_helpers_match_the_oracle_layout():
    # the binding's documented parameter layout, Kaiming initialiser and FLOP
    # count agree with the oracle's network definition and with the library
    from oracle import rdn as ordn
    from paper_2106_12802_gb300 import rdn
    for s in (2, 4, 8):
        for c in (9, 18):
            assert rdn.layers(s, c) == ordn.layers_for(s, c)
            assert rdn.nparams(s, c) == ordn.nparams(s, c) == rdn.kaiming_params(s, c).size
            assert rdn.flops_per_lr_pixel(s, c) == ordn.flops_per_lr_pixel(s, c)
