"""ctypes view of libtcgs.so (include/tcgs.h).  Argument marshalling only.

Loading fails loudly when the library is missing and cannot be built: there is
no CPU fallback anywhere in this package.
"""
from __future__ import annotations

import ctypes
import os
import threading

from . import build as _build

c_int32, c_int64, c_float, c_void_p, c_size_t = (ctypes.c_int32, ctypes.c_int64, ctypes.c_float, ctypes.c_void_p,
                                                 ctypes.c_size_t)

TCGS_OK, TCGS_ERR_INVALID, TCGS_ERR_CUDA, TCGS_ERR_CAPACITY, TCGS_ERR_TIMEOUT, TCGS_ERR_UNSUPPORTED = range(6)
TCGS_ERR_SCRATCH_LIMIT = 6
TCGS_BIN_SORT_NOALLOC_SCRATCH_BYTES = 64 * 1024 * 1024
(TCGS_FP32, TCGS_TC_FP16, TCGS_TC_FP16_SPLIT, TCGS_TC_FP8, TCGS_TC_TF32, TCGS_TC_FP16_GLOBAL,
 TCGS_TC_TF32_GLOBAL, TCGS_FP32_FRAG2MAT) = range(8)
PRECISIONS = {"fp32": TCGS_FP32, "tc_fp16": TCGS_TC_FP16, "tc_fp16_split": TCGS_TC_FP16_SPLIT, "tc_fp8": TCGS_TC_FP8,
              "tc_tf32": TCGS_TC_TF32, "tc_fp16_global": TCGS_TC_FP16_GLOBAL, "tc_tf32_global": TCGS_TC_TF32_GLOBAL,
              "fp32_frag2mat": TCGS_FP32_FRAG2MAT}


class tcgs_camera(ctypes.Structure):
    _fields_ = [("width", c_int32), ("height", c_int32), ("fx", c_float), ("fy", c_float), ("cx", c_float),
                ("cy", c_float), ("viewmat", c_float * 12), ("campos", c_float * 3), ("near_z", c_float),
                ("tan_fovx", c_float), ("tan_fovy", c_float)]


class tcgs_render_opts(ctypes.Structure):
    _fields_ = [("precision", c_int32), ("alpha_max", c_float), ("early_cull", c_int32), ("tile_cull", c_int32),
                ("tile_stats", c_void_p), ("device_status", c_void_p), ("tile_order", c_void_p),
                ("work_counter", c_void_p), ("pixels_per_thread", c_int32)]


TCGS_MAX_VIEWS = 16
TCGS_MLP_IN, TCGS_MLP_HIDDEN, TCGS_MLP_PARAMS = 8, 32, 1377
TILE_STATS_WORDS = 8


class tcgs_view(ctypes.Structure):
    _fields_ = [("cam", tcgs_camera), ("tile_ranges", c_void_p), ("ids_sorted", c_void_p), ("mean2d", c_void_p),
                ("conic", c_void_p), ("rgb", c_void_p), ("img", c_void_p), ("T_final", c_void_p),
                ("n_contrib", c_void_p), ("tile_stats", c_void_p)]


# name -> (restype, argtypes); the same names and order as include/tcgs.h
P_CAM = ctypes.POINTER(tcgs_camera)
P_OPT = ctypes.POINTER(tcgs_render_opts)
V = c_void_p
SIGNATURES = {
    "tcgs_status_string": (ctypes.c_char_p, [ctypes.c_int]),
    "tcgs_version": (ctypes.c_int, []),
    "tcgs_kernel_launches": (ctypes.c_uint64, []),
    "tcgs_project": (c_int32, [P_CAM, c_int32, c_int32, V, V, V, V, V, V, V, V, V, V, V, V]),
    "tcgs_project_bwd": (c_int32, [P_CAM, c_int32, c_int32] + [V] * 12 + [V]),
    "tcgs_bin_sort_workspace_size": (c_size_t, [c_int32, c_int64, c_int32]),
    "tcgs_bin_sort": (c_int32, [P_CAM, c_int32, V, V, V, c_int64, V, c_size_t, V, V, V, V, V]),
    "tcgs_bin_sort_noalloc": (c_int32, [P_CAM, c_int32, V, V, V, c_int64, V, V, V, V, V]),
    "tcgs_bin_sort_exact": (c_int32, [P_CAM, c_int32, V, V, V, V, V, c_int64, V, c_size_t, V, V, V, V, V]),
    "tcgs_tile_order": (c_int32, [P_CAM, V, V, V]),
    "tcgs_render_fwd": (c_int32, [P_CAM, P_OPT, V, V, V, V, V, V, V, V, V, V, V]),
    "tcgs_render_bwd": (c_int32, [P_CAM, P_OPT, V, V, V, V, V, V, V, V, V, V, V, V, V, V, V, V]),
    "tcgs_render_fwd_batched": (c_int32, [c_int32, V, P_OPT, V, V, V, c_int32, V, c_int32, V]),
    "tcgs_tile_features": (c_int32, [P_CAM, V, V, V, V, V, V, V, V, V]),
    "tcgs_feature_norm": (c_int32, [V, c_int32, V, V]),
    "tcgs_mlp_fwd": (c_int32, [V, V, V, c_int32, V, V]),
    "tcgs_mlp_bwd": (c_int32, [V, V, V, V, c_int32, V, V, V]),
    "tcgs_adam_step": (c_int32, [V, V, V, V, c_int32, c_float, c_float, c_float, c_float, c_int32, V]),
    "tcgs_sched_order_workspace_size": (c_size_t, [c_int32]),
    "tcgs_sched_order": (c_int32, [V, V, c_int32, V, V, c_size_t, V]),
    "tcgs_frag2mat_beta": (c_int32, [P_CAM, c_int32, V, V, V, V, V, c_int32, V, c_int32, V, V, V]),
    "tcgs_selftest_bounded_wait": (c_int32, [V, ctypes.c_uint32, V]),
    "tcgs_microbench_ex2": (c_int32, [V, c_int32, c_int32, V]),
    "tcgs_tc_wave_tiles": (c_int32, []),
}

_lock = threading.Lock()
_lib = None


def library_path() -> str:
    return _build.LIB


def load(build_if_needed: bool = True) -> ctypes.CDLL:
    """Load libtcgs.so (building it with nvcc first if it is missing or stale)."""
    global _lib
    with _lock:
        if _lib is None:
            if build_if_needed:
                _build.build()
            if not os.path.exists(_build.LIB):
                raise RuntimeError(f"libtcgs.so not found at {_build.LIB}; build it with "
                                   "paper_2505_24796_gb300.build.build()")
            lib = ctypes.CDLL(_build.LIB)
            for name, (res, args) in SIGNATURES.items():
                fn = getattr(lib, name)
                fn.restype = res
                fn.argtypes = args
            _lib = lib
    return _lib


class TcgsError(RuntimeError):
    def __init__(self, name, code):
        msg = load(False).tcgs_status_string(code).decode()
        super().__init__(f"{name} failed: {msg} (status {code})")
        self.code = code


def check(name: str, code: int) -> None:
    if code != TCGS_OK:
        raise TcgsError(name, code)
