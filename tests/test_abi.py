"""CPU checks of the boundary: the C-ABI library builds for sm_103a, loads, and exports
every symbol include/bgs.h declares; host-only calls behave.  No kernel runs here."""
import ctypes
import os
import re
import subprocess

import pytest

from paper_2412_17378_gb300 import _lib, build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "bgs.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(bgs_[a-z0-9_]+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = _declared()
    for required in ("bgs_preprocess", "bgs_bin_and_sort", "bgs_render_forward", "bgs_render_backward",
                     "bgs_plan_create", "bgs_plan_destroy", "bgs_workspace_size", "bgs_last_error", "bgs_check"):
        assert required in names


def test_library_builds_and_exports_every_declared_symbol():
    path = build.build()
    assert os.path.exists(path)
    lib = ctypes.CDLL(path)
    for name in _declared():
        assert hasattr(lib, name), name
    assert set(_lib.EXPORTS) <= set(_declared())
    # the exported dynamic symbols are plain C names (extern "C")
    out = subprocess.run(["nm", "-D", "--defined-only", path], capture_output=True, text=True).stdout
    for name in _declared():
        assert re.search(rf"\bT {name}$", out, re.M), name


def test_build_targets_sm_103a_only():
    assert build.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]


def test_host_only_calls():
    lib = _lib.load()
    d = _lib.PlanDesc()
    lib.bgs_plan_desc_default(ctypes.byref(d))
    assert (d.heavy_threshold, d.gw_pixels, d.queue_chunk, d.lpt_order, d.device, d.pixel_rows,
            d.select_period, d.bin_block, d.gw_segment) == (512, 4, 1, 1, -1, 2, 1000, 0, 2048)
    assert lib.bgs_workspace_size(None, 10, 10, 10, 10) == 0
    # NULL output pointer is rejected before any CUDA call
    assert lib.bgs_plan_create(ctypes.byref(d), None) == _lib.BGS_ERR_INVALID
    assert b"NULL" in lib.bgs_last_error()
    # invalid knobs are rejected before any CUDA call
    h = ctypes.c_void_p()
    d.select_period = 0
    assert lib.bgs_plan_create(ctypes.byref(d), ctypes.byref(h)) == _lib.BGS_ERR_INVALID
    d.select_period = 1000
    d.bin_block = 100  # not a multiple of 32
    assert lib.bgs_plan_create(ctypes.byref(d), ctypes.byref(h)) == _lib.BGS_ERR_INVALID
    d.bin_block = 0
    d.gw_pixels = 3
    assert lib.bgs_plan_create(ctypes.byref(d), ctypes.byref(h)) == _lib.BGS_ERR_INVALID
    d.gw_pixels = 4
    for bad in (0, 128, 1000):  # segment lengths are multiples of 256
        d.gw_segment = bad
        assert lib.bgs_plan_create(ctypes.byref(d), ctypes.byref(h)) == _lib.BGS_ERR_INVALID
    d.gw_segment = 2048
    # the selector query rejects a NULL plan
    assert lib.bgs_plan_selector(None, None, None, None, None, None) == _lib.BGS_ERR_INVALID
    # argument checks of the entry points run before any device work
    assert lib.bgs_render_forward(None, 0, None, None, None, None, None, 0, None, 16, 16, 16, 16, None, 0,
                                  None, None, None, None, None, None, None) == _lib.BGS_ERR_INVALID
    assert lib.bgs_debug_exp2(None, None, -1, None) == _lib.BGS_ERR_INVALID
