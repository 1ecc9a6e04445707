"""FP64 CPU oracle of the tile-based 3DGS rasterizer (Balanced 3DGS, arXiv 2412.17378).

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py``.  The product path never
imports it.  The arithmetic lives in ``orc.c`` (plain C, double precision, OpenMP over
pixels / tiles); this module only compiles it and marshals numpy arrays.

Each wrapper cites the passage of the paper it follows:

* ``preprocess``   -- Eq. 1-3 (Sec. 2.1): 3D covariance, EWA projection, conic, radius.
* ``bin_tiles``    -- the per-tile depth-sorted Gaussian lists (``point_list`` of
  Algorithms 1-6, the "patch" pre-processing of the Sec. 4.3 footnote);
  ``bin_tiles_subset`` builds the same lists for chosen tiles only.
* ``render``       -- Eq. 4 under Algorithm 5's per-pair rules (Appendix A).
* ``render_backward`` -- the analytic gradient of ``render`` (not in the paper, which
  only names the backward pass in Sec. 3; derived from Eq. 4 directly).
* ``preprocess_backward`` -- the chain rule through the projection of Eq. 2-3 (the
  paper prints no backward; ``project64`` is the same projection from FP64 inputs, for
  finite differences).

Parity status: pinned by closed forms, invariants, brute force and FP64 finite
differences (``tests/test_oracle_pins.py``); the paper prints no numeric example, so
nothing is pinned to a value printed in the paper.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "orc.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liborc.so")
_lock = threading.Lock()
_lib = None

# per-pixel ambiguity flags written by ``render`` (see orc.c)
FLAG_ALPHA_EDGE = 1
FLAG_T_EDGE = 2
FLAG_CLAMP_EDGE = 4
FLAG_POWER_EDGE = 8


def build(force: bool = False) -> str:
    """Compile ``orc.c`` into ``_build/liborc.so`` (gcc, -O2, OpenMP, no FP contraction)."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off",
           "-fno-fast-math", _SRC, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIB_PATH)
            P = ctypes.c_void_p
            i64, i32, d = ctypes.c_int64, ctypes.c_int, ctypes.c_double
            lib.orc_num_threads.restype = i32
            lib.orc_set_threads.argtypes = [i32]
            lib.orc_tile_rect.argtypes = [ctypes.c_float, ctypes.c_float, i32, i32, i32, i32, i32, P]
            lib.orc_preprocess.argtypes = [i64, P, P, P, P, i32, i32, d, d, d, d, P, d, d, i32, i32,
                                           P, P, P, P, P, P]
            lib.orc_project64.argtypes = [i64, P, P, P, i32, i32, d, d, d, d, P, d, d, P, P, P, P]
            lib.orc_preprocess_backward.argtypes = [i64, P, P, P, i32, i32, d, d, d, d, P, d, d, P, P, P, P, P, P,
                                                    P]
            lib.orc_bin.argtypes = [i64, P, P, P, i32, i32, i32, i32, i64, P, P]
            lib.orc_bin.restype = i64
            lib.orc_depth_order.argtypes = [i64, P, P, P]
            lib.orc_depth_order.restype = i64
            lib.orc_bin_subset.argtypes = [i64, P, P, i32, i32, i32, i32, i64, P, P, i64, i64, P, P]
            lib.orc_bin_subset.restype = i64
            lib.orc_render.argtypes = [i32, i32, i32, i32, P, P, P, P, P, P, P, i64, P,
                                       P, P, P, P, P, P, P, P]
            lib.orc_render_backward.argtypes = [i32, i32, i32, i32, i64, P, P, P, P, P, P, P,
                                                P, P, P, i64, P, P, P, P, P, P, P, P]
            lib.orc_sh_to_rgb.argtypes = [i64, i32, i32, i32, P, P, P, P, P]
            lib.orc_sh_to_rgb_backward.argtypes = [i64, i32, i32, i32, P, P, P, P, P, P]
            _lib = lib
    return _lib


def _p(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _f32(a):
    return np.ascontiguousarray(a, dtype=np.float32)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def num_threads() -> int:
    return _load().orc_num_threads()


def set_threads(n: int) -> None:
    _load().orc_set_threads(int(n))


def tile_rect(u: float, v: float, r: int, W: int, H: int, tw: int, th: int):
    """Tile rectangle [x0, x1) x [y0, y1) of a Gaussian (float32 decision)."""
    out = np.zeros(4, np.int32)
    _load().orc_tile_rect(ctypes.c_float(u), ctypes.c_float(v), int(r), W, H, tw, th, _p(out))
    return tuple(int(x) for x in out)


def preprocess(means3D, log_scales, quats, opacities, cam: dict, tile_w=16, tile_h=16):
    """Eq. 1-3: per-Gaussian projection.  ``cam`` holds W, H, fx, fy, cx, cy,
    viewmat (4x4 row-major world->camera), near, lowpass.

    Returns a dict of FP64 means2D [N,2], conic_opacity [N,4], depth [N], the int32
    radius [N], radius_raw [N] (3 sqrt(lambda_max) before the ceil) and
    tiles_touched [N]."""
    lib = _load()
    m3, ls, q, op = _f32(means3D), _f32(log_scales), _f32(quats), _f32(opacities)
    N = m3.shape[0]
    V = _f64(np.asarray(cam["viewmat"], np.float64).reshape(16))
    out = dict(means2D=np.zeros((N, 2)), conic_opacity=np.zeros((N, 4)), depth=np.zeros(N),
               radius=np.zeros(N, np.int32), radius_raw=np.zeros(N),
               tiles_touched=np.zeros(N, np.int32))
    lib.orc_preprocess(N, _p(m3), _p(ls), _p(q), _p(op), int(cam["W"]), int(cam["H"]),
                       float(cam["fx"]), float(cam["fy"]), float(cam["cx"]), float(cam["cy"]),
                       _p(V), float(cam.get("near", 0.2)), float(cam.get("lowpass", 0.3)),
                       tile_w, tile_h, _p(out["means2D"]), _p(out["conic_opacity"]),
                       _p(out["depth"]), _p(out["radius"]), _p(out["radius_raw"]),
                       _p(out["tiles_touched"]))
    return out


def _cam_args(cam: dict):
    V = _f64(np.asarray(cam["viewmat"], np.float64).reshape(16))
    return V, (int(cam["W"]), int(cam["H"]), float(cam["fx"]), float(cam["fy"]), float(cam["cx"]),
               float(cam["cy"]))


def project64(means3D, log_scales, quats, cam: dict):
    """The projection of ``preprocess`` (Eq. 1-3) from FP64 inputs: means2D [N,2],
    conic [N,3] (a, b, c), depth [N] and valid [N] (0 where culled)."""
    lib = _load()
    m3, ls, q = _f64(means3D), _f64(log_scales), _f64(quats)
    N = m3.shape[0]
    V, (W, H, fx, fy, cx, cy) = _cam_args(cam)
    out = dict(means2D=np.zeros((N, 2)), conic=np.zeros((N, 3)), depth=np.zeros(N), valid=np.zeros(N, np.int32))
    lib.orc_project64(N, _p(m3), _p(ls), _p(q), W, H, fx, fy, cx, cy, _p(V), float(cam.get("near", 0.2)),
                      float(cam.get("lowpass", 0.3)), _p(out["means2D"]), _p(out["conic"]), _p(out["depth"]),
                      _p(out["valid"]))
    return out


def preprocess_backward(means3D, log_scales, quats, cam: dict, dL_dmeans2D, dL_dconic, dL_ddepth=None,
                        radius=None):
    """Chain rule through the projection (Eq. 2-3): dL/d(means2D [N,2], conic [N,3],
    depth [N]) -> dL/d(means3D [N,3], log_scales [N,3], quats [N,4]) in FP64.  Gaussians
    with radius 0 (when ``radius`` is given) or culled get zero."""
    lib = _load()
    m3, ls, q = _f64(means3D), _f64(log_scales), _f64(quats)
    N = m3.shape[0]
    V, (W, H, fx, fy, cx, cy) = _cam_args(cam)
    gm, gc = _f64(dL_dmeans2D).reshape(N, 2), _f64(dL_dconic).reshape(N, 3)
    gd = None if dL_ddepth is None else _f64(dL_ddepth).reshape(N)
    rad = None if radius is None else np.ascontiguousarray(radius, np.int32)
    out = dict(means3D=np.zeros((N, 3)), log_scales=np.zeros((N, 3)), quats=np.zeros((N, 4)))
    lib.orc_preprocess_backward(N, _p(m3), _p(ls), _p(q), W, H, fx, fy, cx, cy, _p(V), float(cam.get("near", 0.2)),
                                float(cam.get("lowpass", 0.3)), _p(rad), _p(gm), _p(gc), _p(gd),
                                _p(out["means3D"]), _p(out["log_scales"]), _p(out["quats"]))
    return out


def sh_to_rgb(sh, means3D, campos, degree: int):
    """View-dependent colour of Sec. 2.1 from real orthonormal spherical harmonics of
    degree <= 3 in FP64: sh [N, K, 3] (K >= (degree+1)^2 coefficient rows), means3D [N,3],
    campos [V,3] (or [3]).  Returns rgb [V,N,3] and clamped [V,N,3] (uint8, 1 where the
    channel sum + 1/2 was negative and the colour clamped to 0)."""
    lib = _load()
    c = _f64(sh)
    N, K = c.shape[0], c.shape[1]
    m3 = _f64(means3D).reshape(N, 3)
    cp = _f64(campos).reshape(-1, 3)
    V = cp.shape[0]
    rgb = np.zeros((V, N, 3))
    clamped = np.zeros((V, N, 3), np.uint8)
    lib.orc_sh_to_rgb(N, V, int(degree), K, _p(c), _p(m3), _p(cp), _p(rgb), _p(clamped))
    return rgb, clamped


def sh_to_rgb_backward(sh, means3D, campos, degree: int, dL_drgb):
    """Gradients of ``sh_to_rgb`` in FP64: dL_drgb [V,N,3] -> dL/dsh [N,K,3] and
    dL/dmeans3D [N,3] (through the view direction), summed over the V views."""
    lib = _load()
    c = _f64(sh)
    N, K = c.shape[0], c.shape[1]
    m3 = _f64(means3D).reshape(N, 3)
    cp = _f64(campos).reshape(-1, 3)
    V = cp.shape[0]
    g = _f64(dL_drgb).reshape(V, N, 3)
    d_sh, d_m = np.zeros((N, K, 3)), np.zeros((N, 3))
    lib.orc_sh_to_rgb_backward(N, V, int(degree), K, _p(c), _p(m3), _p(cp), _p(g), _p(d_sh), _p(d_m))
    return d_sh, d_m


def bin_tiles(means2D, radius, depth, W, H, tile_w=16, tile_h=16, capacity=None):
    """Per-tile depth-sorted lists from float32 means / depths and int radii.

    Returns (point_list uint32 [K], ranges uint32 [T,2])."""
    lib = _load()
    m2, r, dep = _f32(means2D), np.ascontiguousarray(radius, np.int32), _f32(depth)
    N = m2.shape[0]
    T = ((W + tile_w - 1) // tile_w) * ((H + tile_h - 1) // tile_h)
    ranges = np.zeros((T, 2), np.uint32)
    if capacity is None:
        K = -lib.orc_bin(N, _p(m2), _p(r), _p(dep), W, H, tile_w, tile_h, -1, None, _p(ranges))
        capacity = max(int(K), 0)
    pl = np.zeros(max(capacity, 1), np.uint32)
    K = lib.orc_bin(N, _p(m2), _p(r), _p(dep), W, H, tile_w, tile_h, capacity, _p(pl), _p(ranges))
    if K < 0:
        raise ValueError(f"capacity {capacity} < {-K}")
    return pl[:K].copy(), ranges


def depth_order(radius, depth):
    """The visible Gaussians (radius > 0) in the stable depth order of the per-tile lists
    (float32 depth bits, ties by index): uint32 [n_visible]."""
    lib = _load()
    r, dep = np.ascontiguousarray(radius, np.int32), _f32(depth)
    order = np.zeros(max(r.size, 1), np.uint32)
    n = lib.orc_depth_order(r.size, _p(r), _p(dep), _p(order))
    return order[:n].copy()


def bin_tiles_subset(means2D, radius, depth, W, H, tiles, tile_w=16, tile_h=16, order=None):
    """The lists of ``bin_tiles`` for the listed tile ids only (distinct), one after the
    other; ranges [T,2] holds their spans and (0, 0) for every other tile.  ``order`` is
    ``depth_order(radius, depth)`` (computed when not given).

    Returns (point_list uint32 [K], ranges uint32 [T,2])."""
    lib = _load()
    m2, r = _f32(means2D), np.ascontiguousarray(radius, np.int32)
    sel = np.ascontiguousarray(tiles, np.int64)
    assert np.unique(sel).size == sel.size, "tile ids must be distinct"
    od = depth_order(r, depth) if order is None else np.ascontiguousarray(order, np.uint32)
    N = m2.shape[0]
    T = ((W + tile_w - 1) // tile_w) * ((H + tile_h - 1) // tile_h)
    ranges = np.zeros((T, 2), np.uint32)
    args = (N, _p(m2), _p(r), W, H, tile_w, tile_h, sel.size, _p(sel), _p(od), od.size)
    K = -lib.orc_bin_subset(*args, -1, None, _p(ranges))
    pl = np.zeros(max(int(K), 1), np.uint32)
    K = lib.orc_bin_subset(*args, pl.size, _p(pl), _p(ranges))
    if K < 0:
        raise ValueError("bin_tiles_subset: list storage")
    return pl[:K].copy(), ranges


def render(means2D, conic_opacity, colors, depth, point_list, ranges, W, H, tile_w=16, tile_h=16,
           bg=(0.0, 0.0, 0.0), pixels=None):
    """Eq. 4 under Algorithm 5 for every pixel (or for the linear pixel ids in
    ``pixels``).  Inputs are promoted to FP64.  Returns a dict with color [3,H,W]
    (or [3,P]), depth, alpha, final_T, n_contrib, n_eval, n_acc and the ambiguity flags."""
    lib = _load()
    m2, co, cl, dp = _f64(means2D), _f64(conic_opacity), _f64(colors), _f64(depth)
    pl = np.ascontiguousarray(point_list, np.uint32)
    rg = np.ascontiguousarray(ranges, np.uint32)
    bgv = _f64(np.asarray(bg, np.float64).reshape(3))
    if pixels is None:
        P, shape, pix = W * H, (H, W), None
    else:
        pix = np.ascontiguousarray(pixels, np.int64)
        P, shape = pix.shape[0], (pix.shape[0],)
    out = dict(color=np.zeros((3,) + shape), depth=np.zeros(shape), alpha=np.zeros(shape),
               final_T=np.zeros(shape), n_contrib=np.zeros(shape, np.int32),
               n_eval=np.zeros(shape, np.int32), n_acc=np.zeros(shape, np.int32),
               flags=np.zeros(shape, np.uint8))
    if pl.size == 0:
        pl = np.zeros(1, np.uint32)
    lib.orc_render(W, H, tile_w, tile_h, _p(m2), _p(co), _p(cl), _p(dp), _p(pl), _p(rg), _p(bgv),
                   P, _p(pix), _p(out["color"]), _p(out["depth"]), _p(out["alpha"]),
                   _p(out["final_T"]), _p(out["n_contrib"]), _p(out["n_eval"]), _p(out["n_acc"]),
                   _p(out["flags"]))
    return out


def render_backward(means2D, conic_opacity, colors, depth, point_list, ranges, W, H, dL_dcolor,
                    dL_ddepth=None, dL_dalpha=None, tile_w=16, tile_h=16, bg=(0.0, 0.0, 0.0),
                    tiles=None, mask=None, abs_terms=False):
    """Analytic FP64 gradient of ``render`` w.r.t. means2D, conic (a,b,c), opacity,
    colors and depths, summed over pixels.  ``tiles`` restricts the visited tiles,
    ``mask`` (uint8 [N]) the Gaussians that receive gradients.  With ``abs_terms`` the
    dict also holds ``abs_<name>``: per element, the sum of the absolute values of the
    per-pair terms of that gradient sum (its condition; used by test tolerances)."""
    lib = _load()
    m2, co, cl, dp = _f64(means2D), _f64(conic_opacity), _f64(colors), _f64(depth)
    N = m2.shape[0]
    pl = np.ascontiguousarray(point_list, np.uint32)
    if pl.size == 0:
        pl = np.zeros(1, np.uint32)
    rg = np.ascontiguousarray(ranges, np.uint32)
    bgv = _f64(np.asarray(bg, np.float64).reshape(3))
    gC = _f64(dL_dcolor)
    gD = None if dL_ddepth is None else _f64(dL_ddepth)
    gA = None if dL_dalpha is None else _f64(dL_dalpha)
    tl = None if tiles is None else np.ascontiguousarray(tiles, np.int64)
    mk = None if mask is None else np.ascontiguousarray(mask, np.uint8)
    out = dict(means2D=np.zeros((N, 2)), conic=np.zeros((N, 3)), opacity=np.zeros(N),
               colors=np.zeros((N, 3)), depths=np.zeros(N))
    ab = np.zeros((N, 10)) if abs_terms else None
    lib.orc_render_backward(W, H, tile_w, tile_h, N, _p(m2), _p(co), _p(cl), _p(dp), _p(pl), _p(rg),
                            _p(bgv), _p(gC), _p(gD), _p(gA), 0 if tl is None else tl.shape[0],
                            _p(tl), _p(mk), _p(out["means2D"]), _p(out["conic"]),
                            _p(out["opacity"]), _p(out["colors"]), _p(out["depths"]), _p(ab))
    if abs_terms:
        out.update(abs_means2D=ab[:, 0:2].copy(), abs_conic=ab[:, 2:5].copy(), abs_opacity=ab[:, 5].copy(),
                   abs_colors=ab[:, 6:9].copy(), abs_depths=ab[:, 9].copy())
    return out
