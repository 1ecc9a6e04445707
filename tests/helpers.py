"""Shared helpers of the parity tests: build oracle-side inputs from a seeded scene,
move them to the GPU, and compare images / gradients with the stated tolerances.

Tolerances of the parity bar:
  * images: max |GPU - oracle| <= 2e-3 per channel over pixels the oracle does not flag
    as decision-ambiguous, and >= 99.9% of all pixels within 1e-4;
  * integer outputs (n_contrib, n_eval, binning) bit-exact outside flagged pixels;
  * gradients: relative L2 error <= 1e-3 per tensor.
"""
from __future__ import annotations

import numpy as np

import oracle
from paper_2412_17378_gb300 import scenes

IMG_MAX_ABS = 2e-3
IMG_FRAC_TOL = 1e-4
IMG_FRAC_MIN = 0.999
GRAD_REL_L2 = 1e-3


def oracle_render_inputs(scene: dict, view: int = 0, tile=(16, 16)):
    """FP64 oracle projection of a scene, rounded to the float32 render inputs that both
    the GPU path and the oracle renderer consume, plus the oracle's binning."""
    g, cam = scene["gaussians"], scene["cameras"][view]
    pp = oracle.preprocess(g["means3D"], g["log_scales"], g["quats"], g["opacities"], cam, tile[0], tile[1])
    m2 = pp["means2D"].astype(np.float32)
    co = pp["conic_opacity"].astype(np.float32)
    dp = pp["depth"].astype(np.float32)
    r = pp["radius"].astype(np.int32)
    pl, rg = oracle.bin_tiles(m2, r, dp, cam["W"], cam["H"], tile[0], tile[1])
    return dict(means2D=m2, conic_opacity=co, colors=np.ascontiguousarray(g["colors"], np.float32), depths=dp,
                radii=r, point_list=pl, ranges=rg, W=cam["W"], H=cam["H"], tile=tuple(tile), cam=cam, pre=pp)


def to_gpu(inp: dict):
    import torch
    d = "cuda"
    return dict(
        means2D=torch.from_numpy(inp["means2D"]).to(d), conic_opacity=torch.from_numpy(inp["conic_opacity"]).to(d),
        colors=torch.from_numpy(inp["colors"]).to(d), depths=torch.from_numpy(inp["depths"]).to(d),
        radii=torch.from_numpy(inp["radii"]).to(d),
        point_list=torch.from_numpy(inp["point_list"].astype(np.int32) if inp["point_list"].size else
                                    np.zeros(1, np.int32)).to(d),
        ranges=torch.from_numpy(inp["ranges"].astype(np.int32)).to(d), K=int(inp["point_list"].size))


def compare_images(gpu_color: np.ndarray, ref: dict, flags: np.ndarray | None = None, what: str = ""):
    """Asserts the image parity bar; returns (max_abs_unflagged, frac_within)."""
    ref_c = ref["color"]
    diff = np.abs(gpu_color.astype(np.float64) - ref_c).max(axis=0)
    fl = ref["flags"] if flags is None else flags
    unflagged = fl == 0
    max_abs = float(diff[unflagged].max()) if unflagged.any() else 0.0
    frac = float((diff <= IMG_FRAC_TOL).mean())
    assert max_abs <= IMG_MAX_ABS, f"{what}: max abs {max_abs:.3e} over unflagged pixels"
    assert frac >= IMG_FRAC_MIN, f"{what}: only {frac:.5f} of pixels within {IMG_FRAC_TOL}"
    return max_abs, frac


def rel_l2(a, b) -> float:
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    nb = np.linalg.norm(b)
    return float(np.linalg.norm(a - b) / nb) if nb > 0 else float(np.linalg.norm(a))


def scene(name: str, scale: float = 1.0):
    return scenes.scene_config(name, scale)
