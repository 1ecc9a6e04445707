"""The allocation-free forward entry point (bgs_render_forward_noalloc) against the
regular one (bgs_render_forward), through the C ABI, on two calls in a row.

Callers that cannot let the library allocate device memory (a host application that
owns all device memory under a fixed budget, a plugin inside such a process, a runtime
that forbids allocations after start-up) use this entry point; its scratch lives in a
fixed device array shared by all calls, so the second call also checks that the array
is reset between calls.  This file is named so that pytest collects it last."""
import ctypes

import numpy as np
import pytest

import oracle
from helpers import oracle_render_inputs, scene, to_gpu

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _call_noalloc(lib, g, W, H, tile, bg):
    dev = "cuda"
    out = dict(color=torch.empty((3, H, W), device=dev), depth=torch.empty((H, W), device=dev),
               alpha=torch.empty((H, W), device=dev), final_T=torch.empty((H, W), device=dev),
               n_contrib=torch.empty((H, W), dtype=torch.int32, device=dev),
               n_eval=torch.empty((H, W), dtype=torch.int32, device=dev))
    p = lambda t: ctypes.c_void_p(t.data_ptr())
    bgv = (ctypes.c_float * 3)(*bg)
    code = lib.bgs_render_forward_noalloc(
        g["means2D"].shape[0], p(g["means2D"]), p(g["conic_opacity"]), p(g["colors"]), p(g["depths"]),
        p(g["point_list"]), g["K"], p(g["ranges"]), W, H, tile[0], tile[1], bgv, p(out["color"]), p(out["depth"]),
        p(out["alpha"]), p(out["final_T"]), p(out["n_contrib"]), p(out["n_eval"]),
        ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert code == 0, lib.bgs_last_error()
    torch.cuda.synchronize()
    return {k: v.cpu().numpy() for k, v in out.items()}


def test_noalloc_forward_matches_regular_entry_point():
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
        got = _call_noalloc(lib, g, W, H, tile, bg)
        ref = raster.render_forward(plan, g["means2D"], g["conic_opacity"], g["colors"], g["depths"],
                                    g["point_list"], g["K"], g["ranges"], W, H, tile, bg, "pixel", n_eval=True)
        torch.cuda.synchronize()
        ref = {k: v.cpu().numpy() for k, v in ref.items()}
        flags = oracle.render(inp["means2D"], inp["conic_opacity"], inp["colors"], inp["depths"], inp["point_list"],
                              inp["ranges"], W, H, tile[0], tile[1], bg=bg)["flags"]
        un = flags == 0
        # same tolerance as the cross-kernel agreement test: equal up to float32 reassociation
        assert np.abs(got["color"] - ref["color"]).max() < 1e-4
        assert np.abs(got["final_T"] - ref["final_T"]).max() < 1e-4
        np.testing.assert_array_equal(got["n_contrib"][un], ref["n_contrib"][un])
        np.testing.assert_array_equal(got["n_eval"][un], ref["n_eval"][un])
    plan.close()
