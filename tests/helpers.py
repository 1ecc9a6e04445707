"""Shared helpers of the parity tests: build oracle-side inputs from a seeded scene,
move them to the GPU, and compare images / gradients with the stated tolerances.

Tolerances of the parity bar:
  * images: max |GPU - oracle| <= 2e-3 per channel over pixels the oracle does not flag
    as decision-ambiguous, and >= 99.9% of all pixels within 1e-4;
  * integer outputs (n_contrib, n_eval, binning) bit-exact outside flagged pixels;
  * gradients, per tensor: relative L2 error <= 1e-3, and element-wise
    |GPU - oracle| <= 1e-3 |oracle| + eps S wherever |oracle| > 1e-6 max |oracle|
    (``compare_grads``).  S is the oracle's sum of |term| over the per-pair terms of that
    gradient sum (``render_backward(..., abs_terms=True)``): any float32 evaluation of a
    sum whose terms carry relative errors <= eps is off by at most eps S (the classical
    bound of floating-point summation), however the terms cancel.  eps (``term_eps``)
    is the per-term error of the kernels: each term's own roundings plus the
    transmittance recovered back to front by one rcp.approx and one multiply per
    accumulated pair (2 ulp each), i.e. (2 n_contrib_max + 32) units of 2^-24.
    The gradients of the projection and of the spherical-harmonics colour are chain rules
    evaluated per Gaussian, not sums over pixels; there S is the norm of the Gaussian's own
    gradient vector (its row) and eps is ROW_EPS_PROJECTION / ROW_EPS_SH: float32
    evaluation of the inverse 2D covariance and its derivative (or of the basis polynomials
    at a float32 direction) determines a small component only to a fraction of the
    Gaussian's largest one, and the FP64 oracle itself moves such components by up to 0.5 %
    under one-ulp perturbations of its float32 inputs.
"""
from __future__ import annotations

import numpy as np

import oracle
from paper_2412_17378_gb300 import scenes

IMG_MAX_ABS = 2e-3
IMG_FRAC_TOL = 1e-4
IMG_FRAC_MIN = 0.999
GRAD_REL_L2 = 1e-3
GRAD_ELEM_REL = 1e-3     # element-wise relative bound ...
GRAD_ELEM_FLOOR = 1e-6   # ... on the elements with |ref| > GRAD_ELEM_FLOOR * max |ref|
ROW_EPS_PROJECTION = 3e-4  # per-Gaussian allowance of the projection backward (x the row norm)
ROW_EPS_SH = 1e-4          # per-Gaussian allowance of the spherical-harmonics backward


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


def term_eps(n_contrib_max: int) -> float:
    """Per-term relative error bound of the render backward's float32 terms: a term's own
    roundings (16 ulp) plus the transmittance T_i, recovered from the final T by one
    rcp.approx and one multiply per accumulated pair behind it (2 ulp each); ulp = 2^-24."""
    return (2.0 * n_contrib_max + 32.0) * 2.0 ** -24


def grad_errors(g, r, s=None, eps=0.0):
    """Element-wise comparison of one gradient array against the oracle's: (checked
    elements, failing elements, worst |g - r| / bound over the checked ones, rel-L2, mask
    of the failing elements), bound = GRAD_ELEM_REL |r| + eps s."""
    g = np.asarray(g, np.float64)
    r = np.asarray(r, np.float64)
    a = np.abs(r)
    m = float(a.max()) if a.size else 0.0
    sel = a > GRAD_ELEM_FLOOR * m
    err = np.abs(g - r)
    bound = GRAD_ELEM_REL * a + (eps * np.asarray(s, np.float64) if s is not None else 0.0)
    ratio = np.where(sel, err / np.maximum(bound, 1e-300), 0.0)
    bad = sel & (err > bound)
    return int(sel.sum()), int(bad.sum()), float(ratio.max()) if ratio.size else 0.0, rel_l2(g, r), bad


def compare_grad(g, r, what="", rel_l2_max=GRAD_REL_L2, s=None, eps=0.0, row_eps=None):
    """Asserts the gradient parity bar on one array: rel-L2 <= rel_l2_max and, element-wise,
    |g - r| <= GRAD_ELEM_REL |r| + eps s wherever |r| > GRAD_ELEM_FLOOR max |r| (s: the
    oracle's sum of |term| per element, or None).  With row_eps, s is the L2 norm of each
    element's row (the first axis: one Gaussian's gradient) and eps = row_eps.  Returns
    (checked elements, worst ratio to the element-wise bound)."""
    g = np.asarray(g, np.float64)
    r = np.asarray(r, np.float64)
    if row_eps is not None:
        rn = np.linalg.norm(r.reshape(r.shape[0], -1), axis=1)
        s = np.broadcast_to(rn.reshape((-1,) + (1,) * (r.ndim - 1)), r.shape)
        eps = row_eps
    n, nbad, worst, e, bad = grad_errors(g, r, s, eps)
    assert e <= rel_l2_max, f"{what}: rel-L2 {e:.3e}"
    if nbad:
        w = np.unravel_index(np.argmax(np.where(bad, np.abs(g - r) / np.maximum(np.abs(r), 1e-300), 0)), r.shape)
        extra = f" sum|term| {float(np.asarray(s)[w]):.3e}" if s is not None else ""
        raise AssertionError(f"{what}: {nbad} of {n} elements beyond the bound (worst {worst:.2f}x; at "
                             f"{tuple(int(x) for x in w)}: got {g[w]:.6e} ref {r[w]:.6e}{extra})")
    return n, worst


def compare_grads(got, ref, keys=("means2D", "conic", "opacity", "colors"), what="", idx=None, n_contrib_max=None):
    """compare_grad on every listed tensor of a render-gradient dict against the oracle's
    ``render_backward(..., abs_terms=True)`` output (rows ``idx`` only, when given), with the
    summation allowance eps = term_eps(n_contrib_max) times the oracle's sum of |term|.
    Returns {key: (checked elements, worst ratio)}."""
    eps = term_eps(n_contrib_max) if n_contrib_max is not None else 0.0
    res = {}
    for k in keys:
        g, r = np.asarray(got[k]), np.asarray(ref[k])
        s = ref.get("abs_" + k)
        if idx is not None:
            g, r = g[idx], r[idx]
            s = None if s is None else s[idx]
        res[k] = compare_grad(g, r, f"{what} {k}", s=s, eps=eps if s is not None else 0.0)
    return res
