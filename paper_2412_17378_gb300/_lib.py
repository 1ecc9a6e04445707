"""ctypes loader of libbgs.so (the C ABI declared in include/bgs.h).

Loading fails loudly: there is no CPU or PyTorch fallback for any entry point.  The
library is built in-tree by ``paper_2412_17378_gb300.build`` (called on first use if the
shared object is missing or stale and nvcc is available).
"""
from __future__ import annotations

import ctypes
import os
import threading

from . import build as _build

_lock = threading.Lock()
_lib = None

BGS_OK = 0
BGS_ERR_INVALID = -1
BGS_ERR_CAPACITY = -2
BGS_ERR_CUDA = -3
BGS_ERR_DEVICE_CHECK = -4

MODE_AUTO, MODE_PIXEL, MODE_GAUSSIAN, MODE_STATIC, MODE_SELECT = 0, 1, 2, 3, 4
MODES = {"auto": MODE_AUTO, "pixel": MODE_PIXEL, "gaussian": MODE_GAUSSIAN, "static": MODE_STATIC,
         "select": MODE_SELECT}

CHECK_INDEX, CHECK_RANGE, CHECK_OVERFLOW, CHECK_QUEUE = 1, 2, 4, 8

# names every build of the library exports (checked by the CPU test suite)
EXPORTS = [
    "bgs_plan_desc_default", "bgs_plan_create", "bgs_plan_destroy", "bgs_plan_set", "bgs_plan_get",
    "bgs_plan_reserve", "bgs_workspace_size", "bgs_check", "bgs_plan_stats", "bgs_plan_reset_stats",
    "bgs_plan_num_sms", "bgs_last_error", "bgs_preprocess", "bgs_bin_and_sort", "bgs_render_forward",
    "bgs_render_backward", "bgs_probe_pipe_rates", "bgs_debug_exp2", "bgs_plan_timing", "bgs_plan_kernel_ms",
    "bgs_render_forward_noalloc", "bgs_preprocess_batched", "bgs_bin_and_sort_batched",
    "bgs_preprocess_backward", "bgs_preprocess_backward_batched", "bgs_plan_selector", "bgs_plan_selector_reset",
    "bgs_plan_inject_fault", "bgs_plan_selector_restore",
    "bgs_render_forward_batched", "bgs_render_backward_batched", "bgs_graph_begin", "bgs_graph_end",
    "bgs_graph_launch", "bgs_autotune_render", "bgs_render_forward_batched_vc", "bgs_render_backward_batched_vc",
    "bgs_sh_to_rgb", "bgs_sh_to_rgb_backward",
]


class BgsError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"bgs error {code}: {msg}")
        self.code = code


class PlanDesc(ctypes.Structure):
    _fields_ = [("heavy_threshold", ctypes.c_int32), ("gw_pixels", ctypes.c_int32),
                ("queue_chunk", ctypes.c_int32), ("blocks_per_sm", ctypes.c_int32),
                ("lpt_order", ctypes.c_int32), ("device", ctypes.c_int32), ("pixel_rows", ctypes.c_int32),
                ("select_period", ctypes.c_int32), ("bin_block", ctypes.c_int32),
                ("gw_segment", ctypes.c_int32)]


class Camera(ctypes.Structure):
    _fields_ = [("width", ctypes.c_int32), ("height", ctypes.c_int32), ("fx", ctypes.c_float),
                ("fy", ctypes.c_float), ("cx", ctypes.c_float), ("cy", ctypes.c_float),
                ("viewmat", ctypes.c_float * 16), ("near_plane", ctypes.c_float), ("lowpass", ctypes.c_float)]


class View(ctypes.Structure):
    _fields_ = [("cam", Camera), ("out_color", ctypes.c_void_p), ("out_depth", ctypes.c_void_p),
                ("out_alpha", ctypes.c_void_p), ("final_T", ctypes.c_void_p), ("n_contrib", ctypes.c_void_p),
                ("n_eval", ctypes.c_void_p), ("dL_dcolor", ctypes.c_void_p), ("dL_ddepth", ctypes.c_void_p),
                ("dL_dalpha", ctypes.c_void_p)]


BIN_NO_SYNC = 1


class Stats(ctypes.Structure):
    _fields_ = [("eval_pairs", ctypes.c_uint64), ("contrib_pairs", ctypes.c_uint64), ("items", ctypes.c_uint64),
                ("check_bits", ctypes.c_uint32), ("last_num_items", ctypes.c_uint32),
                ("host_launches", ctypes.c_uint64)]


def library_path() -> str:
    return _build.LIB


def load(build_if_needed: bool = True):
    """Returns the loaded ctypes library, building it first if needed."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        path = _build.LIB
        if build_if_needed and not _build.up_to_date():
            _build.build()
        if not os.path.exists(path):
            raise OSError(f"libbgs.so not found at {path}; build it with "
                          "`python -m paper_2412_17378_gb300.build`")
        lib = ctypes.CDLL(path)
        P, i32, i64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64
        lib.bgs_last_error.restype = ctypes.c_char_p
        lib.bgs_plan_desc_default.argtypes = [ctypes.POINTER(PlanDesc)]
        lib.bgs_plan_desc_default.restype = None
        lib.bgs_plan_create.argtypes = [ctypes.POINTER(PlanDesc), ctypes.POINTER(P)]
        lib.bgs_plan_destroy.argtypes = [P]
        lib.bgs_plan_set.argtypes = [P, ctypes.POINTER(PlanDesc)]
        lib.bgs_plan_get.argtypes = [P, ctypes.POINTER(PlanDesc)]
        lib.bgs_plan_reserve.argtypes = [P, i64, i64, i64, i64]
        lib.bgs_workspace_size.argtypes = [P, i64, i64, i64, i64]
        lib.bgs_workspace_size.restype = ctypes.c_size_t
        lib.bgs_check.argtypes = [P, P]
        lib.bgs_plan_stats.argtypes = [P, ctypes.POINTER(Stats), P]
        lib.bgs_plan_reset_stats.argtypes = [P, P]
        lib.bgs_plan_num_sms.argtypes = [P]
        lib.bgs_plan_selector.argtypes = [P, ctypes.POINTER(i32), ctypes.POINTER(i64), ctypes.POINTER(i64),
                                          ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double)]
        lib.bgs_plan_selector_reset.argtypes = [P]
        lib.bgs_plan_inject_fault.argtypes = [P, ctypes.c_uint32]
        lib.bgs_plan_selector_restore.argtypes = [P, i32, i64, i64, ctypes.c_double, ctypes.c_double]
        lib.bgs_plan_timing.argtypes = [P, i32]
        lib.bgs_plan_kernel_ms.argtypes = [P, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(i32),
                                           ctypes.POINTER(ctypes.c_double), ctypes.POINTER(i32)]
        lib.bgs_preprocess.argtypes = [P, i64, P, P, P, P, ctypes.POINTER(Camera), i32, i32, P, P, P, P, P, P]
        lib.bgs_bin_and_sort.argtypes = [P, i64, P, P, P, P, i32, i32, i32, i32, P, i64, P,
                                         ctypes.POINTER(i64), ctypes.POINTER(i64), P]
        lib.bgs_render_forward.argtypes = [P, i64, P, P, P, P, P, i64, P, i32, i32, i32, i32, P, i32,
                                           P, P, P, P, P, P, P]
        lib.bgs_render_backward.argtypes = [P, i64, P, P, P, P, P, i64, P, i32, i32, i32, i32, P, i32,
                                            P, P, P, P, P, P, P, P, P, P, P]
        lib.bgs_probe_pipe_rates.argtypes = [P, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double), P]
        lib.bgs_debug_exp2.argtypes = [P, P, i64, P]
        VP = ctypes.POINTER(View)
        lib.bgs_preprocess_batched.argtypes = [P, i32, VP, i64, P, P, P, P, i32, i32, P, P, P, P, P, P]
        lib.bgs_preprocess_backward.argtypes = [P, i64, P, P, P, ctypes.POINTER(Camera), P, P, P, P, P, P, P, P]
        lib.bgs_preprocess_backward_batched.argtypes = [P, i32, VP, i64, P, P, P, P, P, P, P, P, P, P, P]
        lib.bgs_bin_and_sort_batched.argtypes = [P, i32, VP, i64, P, P, P, P, i32, i32, P, i64, P, i32,
                                                 ctypes.POINTER(i64), ctypes.POINTER(i64), P]
        lib.bgs_render_forward_batched.argtypes = [P, i32, VP, i64, P, P, P, P, P, i64, P, i32, i32, P, i32, P]
        lib.bgs_render_backward_batched.argtypes = [P, i32, VP, i64, P, P, P, P, P, i64, P, i32, i32, P, i32,
                                                    P, P, P, P, P, P]
        lib.bgs_render_forward_batched_vc.argtypes = lib.bgs_render_forward_batched.argtypes
        lib.bgs_render_backward_batched_vc.argtypes = lib.bgs_render_backward_batched.argtypes
        lib.bgs_sh_to_rgb.argtypes = [P, i32, VP, i64, i32, i32, P, P, P, P, P]
        lib.bgs_sh_to_rgb_backward.argtypes = [P, i32, VP, i64, i32, i32, P, P, P, P, P, P]
        lib.bgs_autotune_render.argtypes = [P, i32, VP, i64, P, P, P, P, P, i64, P, i32, i32, P, i32,
                                            P, P, P, P, ctypes.POINTER(ctypes.c_double), P]
        lib.bgs_graph_begin.argtypes = [P, P]
        lib.bgs_graph_end.argtypes = [P, P]
        lib.bgs_graph_launch.argtypes = [P, P]
        lib.bgs_render_forward_noalloc.argtypes = [i64, P, P, P, P, P, i64, P, i32, i32, i32, i32, P,
                                                   P, P, P, P, P, P, ctypes.POINTER(ctypes.c_uint32), P]
        _lib = lib
        return lib


def check(code: int, what: str = "") -> int:
    if code != BGS_OK:
        msg = load().bgs_last_error().decode(errors="replace")
        raise BgsError(code, f"{what}: {msg}" if what else msg)
    return code
