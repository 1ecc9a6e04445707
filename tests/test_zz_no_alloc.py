"""The allocation-free forward entry point (bgs_render_forward_noalloc), through the C ABI,
on two calls in a row: against the FP64 oracle (the image parity bar, integer outputs
exact) and against the regular entry point (bgs_render_forward), and its check-bit report.

Callers that cannot let the library allocate device memory (a host application that owns
all device memory under a fixed budget, a plugin inside such a process, a runtime that
forbids allocations after start-up) use this entry point; its scratch lives in a fixed
device array shared by all calls, so the second call also checks that the array is reset
between calls.  This file is named so that pytest collects it last."""
import ctypes

import numpy as np
import pytest

import oracle
from helpers import compare_images, oracle_render_inputs, scene, to_gpu

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _call_noalloc(lib, g, W, H, tile, bg, point_list=None, report=True):
    dev = "cuda"
    out = dict(color=torch.empty((3, H, W), device=dev), depth=torch.empty((H, W), device=dev),
               alpha=torch.empty((H, W), device=dev), final_T=torch.empty((H, W), device=dev),
               n_contrib=torch.empty((H, W), dtype=torch.int32, device=dev),
               n_eval=torch.empty((H, W), dtype=torch.int32, device=dev))
    p = lambda t: ctypes.c_void_p(t.data_ptr())
    bgv = (ctypes.c_float * 3)(*bg)
    bits = ctypes.c_uint32(0xdead)
    pl = g["point_list"] if point_list is None else point_list
    code = lib.bgs_render_forward_noalloc(
        g["means2D"].shape[0], p(g["means2D"]), p(g["conic_opacity"]), p(g["colors"]), p(g["depths"]),
        p(pl), g["K"], p(g["ranges"]), W, H, tile[0], tile[1], bgv, p(out["color"]), p(out["depth"]),
        p(out["alpha"]), p(out["final_T"]), p(out["n_contrib"]), p(out["n_eval"]),
        ctypes.byref(bits) if report else None, ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    torch.cuda.synchronize()
    return code, bits.value, {k: v.cpu().numpy() for k, v in out.items()}


def test_noalloc_forward_matches_oracle_and_regular_entry_point():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2412_17378_gb300 import _lib, raster
    lib = _lib.load()
    plan = raster.Plan()
    cases = [(scene("cfg1"), None, (16, 16), (0.0, 0.0, 0.0)),
             (scene("cfg1", 0.3), (100, 70), (16, 8), (0.1, 0.5, 0.9))]  # smaller, ragged: scratch reused
    for sc, size, tile, bg in cases:
        if size is not None:
            W, H = size
            sc["cameras"][0].update(W=W, H=H, cx=(W - 1) / 2, cy=(H - 1) / 2, fx=W, fy=W)
        inp = oracle_render_inputs(sc, tile=tile)
        W, H = inp["W"], inp["H"]
        g = to_gpu(inp)
        code, bits, got = _call_noalloc(lib, g, W, H, tile, bg)
        assert code == 0 and bits == 0, lib.bgs_last_error()
        ref = oracle.render(inp["means2D"], inp["conic_opacity"], inp["colors"], inp["depths"], inp["point_list"],
                            inp["ranges"], W, H, tile[0], tile[1], bg=bg)
        compare_images(got["color"], ref, what=f"noalloc {W}x{H}")
        un = ref["flags"] == 0
        np.testing.assert_array_equal(got["n_contrib"][un], ref["n_contrib"][un])
        np.testing.assert_array_equal(got["n_eval"][un], ref["n_eval"][un])
        np.testing.assert_allclose(got["final_T"], ref["final_T"], atol=2e-3)
        reg = raster.render_forward(plan, g["means2D"], g["conic_opacity"], g["colors"], g["depths"],
                                    g["point_list"], g["K"], g["ranges"], W, H, tile, bg, "pixel", n_eval=True)
        torch.cuda.synchronize()
        reg = {k: v.cpu().numpy() for k, v in reg.items()}
        # same tolerance as the cross-kernel agreement test: equal up to float32 reassociation
        assert np.abs(got["color"] - reg["color"]).max() < 1e-4
        np.testing.assert_array_equal(got["n_contrib"][un], reg["n_contrib"][un])
    plan.close()


def test_noalloc_reports_check_bits():
    """An index >= N in the point list (skipped by the kernel's bounds check) is reported
    through the host word; the next clean call reports nothing (the array is reset)."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2412_17378_gb300 import _lib
    lib = _lib.load()
    inp = oracle_render_inputs(scene("cfg1", 0.3))
    g = to_gpu(inp)
    bad = g["point_list"].clone()
    bad[5] = 10 ** 8
    code, bits, _ = _call_noalloc(lib, g, inp["W"], inp["H"], (16, 16), (0.0, 0.0, 0.0), point_list=bad)
    assert code == -4 and bits & 1, (code, bits)
    code, bits, _ = _call_noalloc(lib, g, inp["W"], inp["H"], (16, 16), (0.0, 0.0, 0.0))
    assert code == 0 and bits == 0
    code, bits, _ = _call_noalloc(lib, g, inp["W"], inp["H"], (16, 16), (0.0, 0.0, 0.0), point_list=bad,
                                  report=False)
    assert code == 0 and bits == 0xdead  # without a host word nothing is reported or written
