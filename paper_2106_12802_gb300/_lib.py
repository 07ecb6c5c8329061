"""ctypes loader for libmrs.so and the C-ABI signatures of include/mrs.h.

Argument marshalling only.  If the library is missing or fails to load, every
call raises: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os
import threading

from . import build as _build

_lock = threading.Lock()
_lib = None

P = ctypes.c_void_p
I32 = ctypes.c_int32
I64 = ctypes.c_int64
U64 = ctypes.c_uint64
F32 = ctypes.c_float
F64 = ctypes.c_double

# name -> argtypes (restype is always int32 mrs_status unless listed in _RES)
SIGS = {
    "mrs_build_scene": [P, I32, P, P, P, I32, P, I32, P, P, P, P],
    "mrs_build_scene_seeded": [U64, I32, P, P, P],
    "mrs_scene_rebuild": [P, P],
    "mrs_scene_set_tree": [P, I32, P],
    "mrs_scene_get_tree": [P, P],
    "mrs_scene_export_nodes": [P, P, I64, P, P],
    "mrs_scene_update_vertices": [P, P, I32, P],
    "mrs_free_scene": [P],
    "mrs_scene_export_bvh": [P, P, P, P, P, P, P],
    "mrs_cast": [P, P, P, I32, P, P, P],
    "mrs_lbvh_build_static": [P, I32, P, P, P, P, P, P],
    "mrs_render": [P, I32, I32, I32, I32, I32, U64, P, P, P, P, P, P, P],
    "mrs_scene_set_wave": [P, I64],
    "mrs_ctx_create": [P],
    "mrs_ctx_free": [P],
    "mrs_ctx_set_wave": [P, I64],
    "mrs_ctx_set_tail": [P, I32],
    "mrs_scene_set_tail": [P, I32],
    "mrs_render_ctx": [P, P, I32, I32, I32, I32, I32, U64, P, P, P, P, P, P, P],
    "mrs_render_grid": [P, P, I32, I32, I32, I32, I32, U64, I32, P, P, P, P, P, P, P],
    "mrs_render_layers": [P, P, I32, I32, I32, I32, I32, U64, I32, P, P],
    "mrs_render_window": [P, P, I32, I32, I32, I32, I32, I32, I32, I32, I32, U64, I32, P, P],
    "mrs_render_batch": [P, P, I32, P],
    "mrs_render_stats": [P, I32, I32, I32, I32, I32, U64, P, P, P],
    "mrs_profile_enable": [I32],
    "mrs_profile_read": [I32, P, P],
    "mrs_philox_uniforms": [P, I32, U64, P, P],
    "mrs_net_create": [P, I32, P],
    "mrs_net_free": [P],
    "mrs_net_set_params": [P, P],
    "mrs_net_get_params": [P, P],
    "mrs_fuse": [P, P, P, P, P, I32, I32, I32, I32, I32, P, P],
    "mrs_fuse_extra": [P, P, P, P, P, P, I32, I32, I32, I32, I32, P, P],
    "mrs_net_input_channels": [P, P],
    "mrs_image_metrics": [P, P, I64, F64, F64, P, P],
    "mrs_train_step": [P, P, P, P, P, P, I32, I32, I32, I32, F32, I32, P, P],
    "mrs_train_step_extra": [P, P, P, P, P, P, P, I32, I32, I32, I32, F32, I32, P, P],
    "mrs_net_get_grads": [P, P],
    "mrs_conv3x3_dgrad": [P, I32, I32, I32, I32, I32, P, I32, P, I32, P, P],
    "mrs_conv_set_ring": [I32],
    "mrs_net_save": [P, ctypes.c_char_p, U64],
    "mrs_net_load": [P, ctypes.c_char_p, P],
    "mrs_net_create_seeded": [I32, U64, F32, P],
    "mrs_net_get_state": [P, P, P, P, P],
    "mrs_net_set_state": [P, P, P, P, I64],
    "mrs_gate": [P, P, P, I32, I32, I32, I32, F64, P, P, P, P],
    "mrs_gate_async": [P, P, P, I32, I32, I32, I32, F64, P, P, P, P],
    "mrs_conv3x3": [P, I32, I32, I32, I32, I32, P, P, I32, I32, P, P],
    "mrs_conv3x3_wgrad": [P, P, I32, I32, I32, I32, I32, I32, P, P, P],
    "mrs_net_set_loss": [P, I32, F32],
    "mrs_rdn_nparams": [I32, I32, P],
    "mrs_rdn_create": [I32, I32, P, I64, P],
    "mrs_rdn_free": [P],
    "mrs_rdn_fuse": [P, P, P, P, P, P, I32, I32, I32, I32, P, P],
    "mrs_rdn_check": [P],
    "mrs_rdn_train_step": [P, P, P, P, P, P, P, I32, I32, I32, I32, F32, F32, I32, P, P, P],
    "mrs_rdn_get_grads": [P, P, I64],
    "mrs_rdn_get_state": [P, P, P, P, I64, P],
    "mrs_rdn_set_state": [P, P, P, P, I64, I64],
    "mrs_selftest_wait_timeout": [I32, P],
    "mrs_status_string": [I32],
    "mrs_last_error": [],
    "mrs_kernel_launches": [],
}
_RES = {"mrs_status_string": ctypes.c_char_p, "mrs_last_error": ctypes.c_char_p,
        "mrs_kernel_launches": ctypes.c_uint64}


def kernel_launches() -> int:
    return int(load().mrs_kernel_launches())


class MrsError(RuntimeError):
    def __init__(self, fn, status, detail):
        super().__init__(f"{fn} failed: status {status}: {detail}")
        self.status = status


def library_path() -> str:
    return _build.SO


def load(build_if_missing: bool = True):
    """Load libmrs.so (building it first if it is missing and nvcc exists)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(_build.SO):
                if not build_if_missing:
                    raise RuntimeError(f"CUDA library not built: {_build.SO}")
                _build.build()
            L = ctypes.CDLL(_build.SO)
            for name, args in SIGS.items():
                fn = getattr(L, name)
                fn.argtypes = args
                fn.restype = _RES.get(name, I32)
            _lib = L
    return _lib


def call(name, *args):
    L = load()
    st = getattr(L, name)(*args)
    if st != 0:
        detail = (L.mrs_last_error() or b"").decode(errors="replace")
        raise MrsError(name, st, detail)
    return st
