"""Thin Python binding of the C ABI (include/bgs.h) plus a torch.autograd.Function.

Every function here only checks and marshals arguments (device pointers of CUDA
tensors, the current CUDA stream) and calls the library; every step of the render path
runs in the library's kernels.  PyTorch provides device memory and streams.  The names
follow the C entry points: ``preprocess`` -> bgs_preprocess, ``bin_and_sort`` ->
bgs_bin_and_sort, ``render_forward`` / ``render_backward`` -> bgs_render_forward /
bgs_render_backward.
"""
from __future__ import annotations

import ctypes

import numpy as np
import torch

from . import _lib
from ._lib import MODES, BgsError, check

__all__ = ["Plan", "camera_struct", "preprocess", "preprocess_backward", "bin_and_sort", "render_forward",
           "render_backward", "PreprocessFunction",
           "render_forward_noalloc",
           "RenderFunction", "render", "tile_counts", "preprocess_batched", "preprocess_backward_batched",
           "bin_and_sort_batched", "alloc_view_outputs", "render_forward_batched", "render_backward_batched",
           "sh_to_rgb", "sh_to_rgb_backward", "SHFunction", "autotune_render", "graph_begin", "graph_end",
           "graph_launch", "probe_pipe_rates", "debug_exp2", "BgsError", "MODES"]


def _stream(device) -> ctypes.c_void_p:
    return ctypes.c_void_p(torch.cuda.current_stream(device).cuda_stream)


def _ptr(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _req(t: torch.Tensor, name: str, dtype, shape=None):
    if not isinstance(t, torch.Tensor):
        raise TypeError(f"{name} must be a torch.Tensor")
    if not t.is_cuda:
        raise ValueError(f"{name} must be a CUDA tensor (there is no CPU path)")
    if t.dtype != dtype:
        raise TypeError(f"{name} must be {dtype}, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if shape is not None and tuple(t.shape) != tuple(shape):
        raise ValueError(f"{name} has shape {tuple(t.shape)}, expected {tuple(shape)}")
    return t


class Plan:
    """Owns a bgs_plan: tuning knobs and the library-managed workspace."""

    def __init__(self, heavy_threshold: int = 512, gw_pixels: int = 4, queue_chunk: int = 1,
                 blocks_per_sm: int = 0, lpt_order: bool = True, device=None, pixel_rows: int = 2,
                 select_period: int = 1000, bin_block: int = 0, gw_segment: int = 2048):
        self._lib = _lib.load()
        if device is None:
            device = torch.cuda.current_device()
        self.device = torch.device("cuda", device if isinstance(device, int) else torch.device(device).index or 0)
        d = _lib.PlanDesc()
        self._lib.bgs_plan_desc_default(ctypes.byref(d))
        d.heavy_threshold, d.gw_pixels, d.queue_chunk = heavy_threshold, gw_pixels, queue_chunk
        d.blocks_per_sm, d.lpt_order, d.device = blocks_per_sm, int(bool(lpt_order)), self.device.index
        d.pixel_rows = pixel_rows
        d.select_period = select_period
        d.bin_block = bin_block
        d.gw_segment = gw_segment
        h = ctypes.c_void_p()
        check(self._lib.bgs_plan_create(ctypes.byref(d), ctypes.byref(h)), "bgs_plan_create")
        self.handle = h

    def desc(self) -> dict:
        d = _lib.PlanDesc()
        check(self._lib.bgs_plan_get(self.handle, ctypes.byref(d)), "bgs_plan_get")
        return {k: getattr(d, k) for k, _ in _lib.PlanDesc._fields_}

    def set(self, **kw):
        d = _lib.PlanDesc()
        check(self._lib.bgs_plan_get(self.handle, ctypes.byref(d)), "bgs_plan_get")
        for k, v in kw.items():
            setattr(d, k, int(v))
        check(self._lib.bgs_plan_set(self.handle, ctypes.byref(d)), "bgs_plan_set")

    def selector(self) -> dict:
        """State of the "select" mode (Sec. 4.4): switched, calls, measurements and the last
        balanced / static forward timings in ms."""
        sw, calls, meas = ctypes.c_int32(), ctypes.c_int64(), ctypes.c_int64()
        tb, ts = ctypes.c_double(), ctypes.c_double()
        check(self._lib.bgs_plan_selector(self.handle, ctypes.byref(sw), ctypes.byref(calls), ctypes.byref(meas),
                                          ctypes.byref(tb), ctypes.byref(ts)), "bgs_plan_selector")
        return dict(switched=bool(sw.value), calls=calls.value, measurements=meas.value, balanced_ms=tb.value,
                    static_ms=ts.value)

    def state_dict(self) -> dict:
        """The plan's resumable state: its knobs (device excluded) and the selector's state --
        what a training run checkpoints to resume with the same kernels (plain JSON types)."""
        knobs = {k: int(v) for k, v in self.desc().items() if k != "device"}
        return {"knobs": knobs, "selector": self.selector()}

    def load_state_dict(self, state: dict):
        """Restores a state_dict() (knobs, then the selector)."""
        self.set(**state["knobs"])
        sel = state["selector"]
        check(self._lib.bgs_plan_selector_restore(self.handle, int(bool(sel["switched"])), int(sel["calls"]),
                                                  int(sel["measurements"]), float(sel["balanced_ms"]),
                                                  float(sel["static_ms"])), "bgs_plan_selector_restore")

    def inject_fault(self, which: int):
        """bgs_plan_inject_fault: a host-side fault for tests (e.g. _lib.CHECK_QUEUE)."""
        check(self._lib.bgs_plan_inject_fault(self.handle, int(which)), "bgs_plan_inject_fault")

    def selector_reset(self):
        check(self._lib.bgs_plan_selector_reset(self.handle), "bgs_plan_selector_reset")

    @property
    def num_sms(self) -> int:
        return self._lib.bgs_plan_num_sms(self.handle)

    def reserve(self, max_gaussians: int, max_entries: int, max_tiles: int, max_pixels: int):
        check(self._lib.bgs_plan_reserve(self.handle, max_gaussians, max_entries, max_tiles, max_pixels),
              "bgs_plan_reserve")

    def check(self):
        """Raises BgsError if a device-side check tripped (synchronises the stream)."""
        check(self._lib.bgs_check(self.handle, _stream(self.device)), "bgs_check")

    def stats(self) -> dict:
        s = _lib.Stats()
        check(self._lib.bgs_plan_stats(self.handle, ctypes.byref(s), _stream(self.device)), "bgs_plan_stats")
        return {k: getattr(s, k) for k, _ in _lib.Stats._fields_}

    def timing(self, enable: bool):
        """Turns CUDA-event timing of the render kernels on / off."""
        check(self._lib.bgs_plan_timing(self.handle, int(bool(enable))), "bgs_plan_timing")

    def kernel_ms(self):
        """(forward ms, forward launches, backward ms, backward launches) recorded since the last call."""
        f, b = ctypes.c_double(0), ctypes.c_double(0)
        nf, nb = ctypes.c_int32(0), ctypes.c_int32(0)
        check(self._lib.bgs_plan_kernel_ms(self.handle, ctypes.byref(f), ctypes.byref(nf), ctypes.byref(b),
                                           ctypes.byref(nb)), "bgs_plan_kernel_ms")
        return f.value, nf.value, b.value, nb.value

    def reset_stats(self):
        check(self._lib.bgs_plan_reset_stats(self.handle, _stream(self.device)), "bgs_plan_reset_stats")

    def close(self):
        if getattr(self, "handle", None) is not None and self.handle.value:
            self._lib.bgs_plan_destroy(self.handle)
            self.handle = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def camera_struct(cam: dict) -> _lib.Camera:
    c = _lib.Camera()
    c.width, c.height = int(cam["W"]), int(cam["H"])
    c.fx, c.fy, c.cx, c.cy = float(cam["fx"]), float(cam["fy"]), float(cam["cx"]), float(cam["cy"])
    V = np.asarray(cam["viewmat"], np.float64).reshape(16)
    for k in range(16):
        c.viewmat[k] = float(V[k])
    c.near_plane = float(cam.get("near", 0.2))
    c.lowpass = float(cam.get("lowpass", 0.3))
    return c


def preprocess(plan: Plan, means3D, log_scales, quats, opacities, cam: dict, tile=(16, 16), out=None):
    """bgs_preprocess: returns dict(means2D [N,2], conic_opacity [N,4], depths [N], radii [N] int32,
    tiles_touched [N] int32 holding uint32)."""
    N = means3D.shape[0]
    _req(means3D, "means3D", torch.float32, (N, 3))
    _req(log_scales, "log_scales", torch.float32, (N, 3))
    _req(quats, "quats", torch.float32, (N, 4))
    _req(opacities, "opacities", torch.float32, (N,))
    dev = means3D.device
    if out is None:
        out = dict(means2D=torch.empty((N, 2), device=dev), conic_opacity=torch.empty((N, 4), device=dev),
                   depths=torch.empty(N, device=dev), radii=torch.empty(N, dtype=torch.int32, device=dev),
                   tiles_touched=torch.empty(N, dtype=torch.int32, device=dev))
    c = camera_struct(cam)
    check(plan._lib.bgs_preprocess(plan.handle, N, _ptr(means3D), _ptr(log_scales), _ptr(quats), _ptr(opacities),
                                   ctypes.byref(c), tile[0], tile[1], _ptr(out["means2D"]),
                                   _ptr(out["conic_opacity"]), _ptr(out["depths"]), _ptr(out["radii"]),
                                   _ptr(out["tiles_touched"]), _stream(dev)), "bgs_preprocess")
    return out


def _grads_out(N, dev, out):
    if out is None:
        out = dict(means3D=torch.empty((N, 3), device=dev), log_scales=torch.empty((N, 3), device=dev),
                   quats=torch.empty((N, 4), device=dev))
    return out


def preprocess_backward(plan: Plan, means3D, log_scales, quats, cam: dict, radii, dL_dmeans2D, dL_dconic,
                        dL_ddepths=None, out=None):
    """bgs_preprocess_backward: dL/d(means2D [N,2], conic [N,3], depths [N]) -> dict of
    dL/d(means3D [N,3], log_scales [N,3], quats [N,4])."""
    N = means3D.shape[0]
    _req(means3D, "means3D", torch.float32, (N, 3))
    _req(log_scales, "log_scales", torch.float32, (N, 3))
    _req(quats, "quats", torch.float32, (N, 4))
    _req(radii, "radii", torch.int32, (N,))
    _req(dL_dmeans2D, "dL_dmeans2D", torch.float32, (N, 2))
    _req(dL_dconic, "dL_dconic", torch.float32, (N, 3))
    if dL_ddepths is not None:
        _req(dL_ddepths, "dL_ddepths", torch.float32, (N,))
    dev = means3D.device
    out = _grads_out(N, dev, out)
    c = camera_struct(cam)
    check(plan._lib.bgs_preprocess_backward(plan.handle, N, _ptr(means3D), _ptr(log_scales), _ptr(quats),
                                            ctypes.byref(c), _ptr(radii), _ptr(dL_dmeans2D), _ptr(dL_dconic),
                                            _ptr(dL_ddepths), _ptr(out["means3D"]), _ptr(out["log_scales"]),
                                            _ptr(out["quats"]), _stream(dev)), "bgs_preprocess_backward")
    return out


def bin_and_sort(plan: Plan, means2D, radii, depths, W: int, H: int, tile=(16, 16), point_list=None,
                 conic_opacity=None):
    """bgs_bin_and_sort: returns (point_list int32 [>=K] holding uint32, ranges int32 [T,2], K).
    Grows ``point_list`` (a torch buffer) when the entry count exceeds its capacity.  With
    ``conic_opacity`` each tile's list is cut where every pixel of the tile is certified to
    have stopped (the render's outputs are unchanged)."""
    N = means2D.shape[0]
    _req(means2D, "means2D", torch.float32, (N, 2))
    _req(radii, "radii", torch.int32, (N,))
    _req(depths, "depths", torch.float32, (N,))
    if conic_opacity is not None:
        _req(conic_opacity, "conic_opacity", torch.float32, (N, 4))
    dev = means2D.device
    tx, ty = (W + tile[0] - 1) // tile[0], (H + tile[1] - 1) // tile[1]
    ranges = torch.empty((tx * ty, 2), dtype=torch.int32, device=dev)
    if point_list is None:
        point_list = torch.empty(max(4 * N, 1024), dtype=torch.int32, device=dev)
    K = ctypes.c_int64(0)
    need = ctypes.c_int64(0)
    for _ in range(2):
        code = plan._lib.bgs_bin_and_sort(plan.handle, N, _ptr(means2D), _ptr(radii), _ptr(depths),
                                          _ptr(conic_opacity) if conic_opacity is not None else None, W, H, tile[0],
                                          tile[1], _ptr(point_list), point_list.numel(), _ptr(ranges),
                                          ctypes.byref(K), ctypes.byref(need), _stream(dev))
        if code == _lib.BGS_ERR_CAPACITY and need.value > point_list.numel():
            point_list = torch.empty(int(need.value * 1.1) + 1024, dtype=torch.int32, device=dev)
            continue
        check(code, "bgs_bin_and_sort")
        break
    return point_list, ranges, int(K.value)


def render_forward(plan: Plan, means2D, conic_opacity, colors, depths, point_list, num_entries: int, ranges,
                   W: int, H: int, tile=(16, 16), bg=(0.0, 0.0, 0.0), mode="auto", n_eval: bool = False, out=None):
    """bgs_render_forward: returns dict(color [3,H,W], depth, alpha, final_T, n_contrib[, n_eval])."""
    N = means2D.shape[0]
    _req(means2D, "means2D", torch.float32, (N, 2))
    _req(conic_opacity, "conic_opacity", torch.float32, (N, 4))
    _req(colors, "colors", torch.float32, (N, 3))
    _req(depths, "depths", torch.float32, (N,))
    _req(point_list, "point_list", torch.int32)
    _req(ranges, "ranges", torch.int32)
    dev = means2D.device
    if out is None:
        out = dict(color=torch.empty((3, H, W), device=dev), depth=torch.empty((H, W), device=dev),
                   alpha=torch.empty((H, W), device=dev), final_T=torch.empty((H, W), device=dev),
                   n_contrib=torch.empty((H, W), dtype=torch.int32, device=dev))
        if n_eval:
            out["n_eval"] = torch.empty((H, W), dtype=torch.int32, device=dev)
    bgv = (ctypes.c_float * 3)(*[float(v) for v in bg])
    m = MODES[mode] if isinstance(mode, str) else int(mode)
    check(plan._lib.bgs_render_forward(plan.handle, N, _ptr(means2D), _ptr(conic_opacity), _ptr(colors),
                                       _ptr(depths), _ptr(point_list), int(num_entries), _ptr(ranges), W, H, tile[0],
                                       tile[1], bgv, m, _ptr(out["color"]), _ptr(out["depth"]), _ptr(out["alpha"]),
                                       _ptr(out["final_T"]), _ptr(out["n_contrib"]), _ptr(out.get("n_eval")),
                                       _stream(dev)), "bgs_render_forward")
    return out


def render_backward(plan: Plan, means2D, conic_opacity, colors, depths, point_list, num_entries: int, ranges,
                    W: int, H: int, final_T, n_contrib, dL_dcolor, dL_ddepth=None, dL_dalpha=None, tile=(16, 16),
                    bg=(0.0, 0.0, 0.0), mode="auto", out=None):
    """bgs_render_backward: returns dict(means2D [N,2], conic [N,3], opacity [N], colors [N,3], depths [N])."""
    N = means2D.shape[0]
    _req(final_T, "final_T", torch.float32, (H, W))
    _req(n_contrib, "n_contrib", torch.int32, (H, W))
    _req(dL_dcolor, "dL_dcolor", torch.float32, (3, H, W))
    if dL_ddepth is not None:
        _req(dL_ddepth, "dL_ddepth", torch.float32, (H, W))
    if dL_dalpha is not None:
        _req(dL_dalpha, "dL_dalpha", torch.float32, (H, W))
    dev = means2D.device
    if out is None:
        out = dict(means2D=torch.empty((N, 2), device=dev), conic=torch.empty((N, 3), device=dev),
                   opacity=torch.empty(N, device=dev), colors=torch.empty((N, 3), device=dev),
                   depths=torch.empty(N, device=dev))
    bgv = (ctypes.c_float * 3)(*[float(v) for v in bg])
    m = MODES[mode] if isinstance(mode, str) else int(mode)
    check(plan._lib.bgs_render_backward(plan.handle, N, _ptr(means2D), _ptr(conic_opacity), _ptr(colors),
                                        _ptr(depths), _ptr(point_list), int(num_entries), _ptr(ranges), W, H,
                                        tile[0], tile[1], bgv, m, _ptr(final_T), _ptr(n_contrib), _ptr(dL_dcolor),
                                        _ptr(dL_ddepth), _ptr(dL_dalpha), _ptr(out["means2D"]), _ptr(out["conic"]),
                                        _ptr(out["opacity"]), _ptr(out["colors"]), _ptr(out.get("depths")),
                                        _stream(dev)), "bgs_render_backward")
    return out


def render_forward_noalloc(means2D, conic_opacity, colors, depths, point_list, num_entries: int, ranges, W: int,
                           H: int, tile=(16, 16), bg=(0.0, 0.0, 0.0), n_eval: bool = False, out=None):
    """bgs_render_forward_noalloc: the allocation-free forward (no plan; the library keeps
    its scratch in a fixed device array).  ``out`` may pass preallocated output tensors."""
    N = means2D.shape[0]
    _req(means2D, "means2D", torch.float32, (N, 2))
    _req(conic_opacity, "conic_opacity", torch.float32, (N, 4))
    _req(colors, "colors", torch.float32, (N, 3))
    _req(depths, "depths", torch.float32, (N,))
    dev = means2D.device
    if out is None:
        out = dict(color=torch.empty((3, H, W), device=dev), depth=torch.empty((H, W), device=dev),
                   alpha=torch.empty((H, W), device=dev), final_T=torch.empty((H, W), device=dev),
                   n_contrib=torch.empty((H, W), dtype=torch.int32, device=dev))
        if n_eval:
            out["n_eval"] = torch.empty((H, W), dtype=torch.int32, device=dev)
    bgv = (ctypes.c_float * 3)(*[float(v) for v in bg])
    with torch.cuda.device(dev):
        check(_lib.load().bgs_render_forward_noalloc(
            N, _ptr(means2D), _ptr(conic_opacity), _ptr(colors), _ptr(depths), _ptr(point_list), int(num_entries),
            _ptr(ranges), W, H, tile[0], tile[1], bgv, _ptr(out["color"]), _ptr(out["depth"]), _ptr(out["alpha"]),
            _ptr(out["final_T"]), _ptr(out["n_contrib"]), _ptr(out.get("n_eval")), _stream(dev)),
            "bgs_render_forward_noalloc")
    return out


class RenderFunction(torch.autograd.Function):
    """Differentiable render of projected Gaussians: (means2D, conic_opacity, colors, depths)
    -> (color [3,H,W], depth [H,W], alpha [H,W]).  The backward calls bgs_render_backward,
    which recomputes the blend from the stored final T and last-contributor index."""

    @staticmethod
    def forward(ctx, means2D, conic_opacity, colors, depths, binning, plan, W, H, tile, bg, mode):
        point_list, ranges, K = binning
        out = render_forward(plan, means2D.contiguous(), conic_opacity.contiguous(), colors.contiguous(),
                             depths.contiguous(), point_list, K, ranges, W, H, tile, bg, mode)
        ctx.plan, ctx.W, ctx.H, ctx.tile, ctx.bg, ctx.mode, ctx.K = plan, W, H, tile, bg, mode, K
        ctx.save_for_backward(means2D, conic_opacity, colors, depths, point_list, ranges, out["final_T"],
                              out["n_contrib"])
        ctx.mark_non_differentiable(out["final_T"], out["n_contrib"])
        return out["color"], out["depth"], out["alpha"], out["final_T"], out["n_contrib"]

    @staticmethod
    def backward(ctx, g_color, g_depth, g_alpha, _g_T, _g_n):
        means2D, conic_opacity, colors, depths, point_list, ranges, final_T, n_contrib = ctx.saved_tensors
        g = render_backward(ctx.plan, means2D, conic_opacity, colors, depths, point_list, ctx.K, ranges, ctx.W,
                            ctx.H, final_T, n_contrib,
                            g_color.contiguous() if g_color is not None else torch.zeros_like(final_T).expand(3, -1, -1).contiguous(),
                            None if g_depth is None else g_depth.contiguous(),
                            None if g_alpha is None else g_alpha.contiguous(),
                            ctx.tile, ctx.bg, ctx.mode)
        d_conic = torch.cat([g["conic"], g["opacity"][:, None]], 1)
        return g["means2D"], d_conic, g["colors"], g["depths"], None, None, None, None, None, None, None


class PreprocessFunction(torch.autograd.Function):
    """Differentiable projection (Eq. 1-3): (means3D, log_scales, quats, opacities) ->
    (means2D, conic_opacity, depths, radii).  The backward calls bgs_preprocess_backward;
    the opacity column of conic_opacity passes its gradient straight to opacities."""

    @staticmethod
    def forward(ctx, means3D, log_scales, quats, opacities, plan, cam, tile):
        m3, ls, q = means3D.contiguous(), log_scales.contiguous(), quats.contiguous()
        out = preprocess(plan, m3, ls, q, opacities.contiguous(), cam, tile)
        ctx.plan, ctx.cam = plan, cam
        ctx.save_for_backward(m3, ls, q, out["radii"])
        ctx.mark_non_differentiable(out["radii"])
        return out["means2D"], out["conic_opacity"], out["depths"], out["radii"]

    @staticmethod
    def backward(ctx, g_means2D, g_conic_opacity, g_depths, _g_radii):
        m3, ls, q, radii = ctx.saved_tensors
        N = m3.shape[0]
        z = lambda *shape: torch.zeros(shape, device=m3.device)
        gm = g_means2D.contiguous() if g_means2D is not None else z(N, 2)
        gco = g_conic_opacity if g_conic_opacity is not None else z(N, 4)
        gd = g_depths.contiguous() if g_depths is not None else None
        g = preprocess_backward(ctx.plan, m3, ls, q, ctx.cam, radii, gm, gco[:, :3].contiguous(), gd)
        return g["means3D"], g["log_scales"], g["quats"], gco[:, 3].contiguous(), None, None, None


def render(plan: Plan, means2D, conic_opacity, colors, depths, binning, W, H, tile=(16, 16), bg=(0.0, 0.0, 0.0),
           mode="auto"):
    """Differentiable render; returns (color, depth, alpha)."""
    color, depth, alpha, _, _ = RenderFunction.apply(means2D, conic_opacity, colors, depths, binning, plan, W, H,
                                                     tuple(tile), tuple(bg), mode)
    return color, depth, alpha


# ---- batched views (many cameras, one Gaussian set) and graph capture --------------------

def _views(cams, outs=None, grads=None, fw=None):
    arr = (_lib.View * len(cams))()
    for v, cam in enumerate(cams):
        arr[v].cam = camera_struct(cam)
        if outs is not None:
            o = outs[v]
            arr[v].out_color, arr[v].out_depth = o["color"].data_ptr(), o["depth"].data_ptr()
            arr[v].out_alpha, arr[v].final_T = o["alpha"].data_ptr(), o["final_T"].data_ptr()
            arr[v].n_contrib = o["n_contrib"].data_ptr()
            arr[v].n_eval = o["n_eval"].data_ptr() if "n_eval" in o else None
        if fw is not None:
            arr[v].final_T, arr[v].n_contrib = fw[v]["final_T"].data_ptr(), fw[v]["n_contrib"].data_ptr()
        if grads is not None:
            gv = grads[v]
            arr[v].dL_dcolor = gv["color"].data_ptr()
            arr[v].dL_ddepth = gv["depth"].data_ptr() if gv.get("depth") is not None else None
            arr[v].dL_dalpha = gv["alpha"].data_ptr() if gv.get("alpha") is not None else None
    return arr


def tile_counts(cams, tile=(16, 16)):
    """Tiles per view and the total of the global tile space."""
    per = [((c["W"] + tile[0] - 1) // tile[0]) * ((c["H"] + tile[1] - 1) // tile[1]) for c in cams]
    return per, sum(per)


def preprocess_batched(plan: Plan, means3D, log_scales, quats, opacities, cams, tile=(16, 16), out=None):
    """bgs_preprocess_batched: records v * N + g; returns dict of [V*N, ...] tensors."""
    N, V = means3D.shape[0], len(cams)
    _req(means3D, "means3D", torch.float32, (N, 3))
    _req(log_scales, "log_scales", torch.float32, (N, 3))
    _req(quats, "quats", torch.float32, (N, 4))
    _req(opacities, "opacities", torch.float32, (N,))
    dev, R = means3D.device, N * V
    if out is None:
        out = dict(means2D=torch.empty((R, 2), device=dev), conic_opacity=torch.empty((R, 4), device=dev),
                   depths=torch.empty(R, device=dev), radii=torch.empty(R, dtype=torch.int32, device=dev),
                   tiles_touched=torch.empty(R, dtype=torch.int32, device=dev))
    vw = _views(cams)
    check(plan._lib.bgs_preprocess_batched(plan.handle, V, vw, N, _ptr(means3D), _ptr(log_scales), _ptr(quats),
                                           _ptr(opacities), tile[0], tile[1], _ptr(out["means2D"]),
                                           _ptr(out["conic_opacity"]), _ptr(out["depths"]), _ptr(out["radii"]),
                                           _ptr(out["tiles_touched"]), _stream(dev)), "bgs_preprocess_batched")
    return out


def preprocess_backward_batched(plan: Plan, means3D, log_scales, quats, cams, radii, dL_dmeans2D, dL_dconic,
                                dL_ddepths=None, out=None):
    """bgs_preprocess_backward_batched: record gradients [V*N, ...] -> Gaussian gradients
    [N, ...] summed over the views."""
    N, V = means3D.shape[0], len(cams)
    R = N * V
    _req(means3D, "means3D", torch.float32, (N, 3))
    _req(log_scales, "log_scales", torch.float32, (N, 3))
    _req(quats, "quats", torch.float32, (N, 4))
    _req(radii, "radii", torch.int32, (R,))
    _req(dL_dmeans2D, "dL_dmeans2D", torch.float32, (R, 2))
    _req(dL_dconic, "dL_dconic", torch.float32, (R, 3))
    if dL_ddepths is not None:
        _req(dL_ddepths, "dL_ddepths", torch.float32, (R,))
    dev = means3D.device
    out = _grads_out(N, dev, out)
    vw = _views(cams)
    check(plan._lib.bgs_preprocess_backward_batched(plan.handle, V, vw, N, _ptr(means3D), _ptr(log_scales),
                                                    _ptr(quats), _ptr(radii), _ptr(dL_dmeans2D), _ptr(dL_dconic),
                                                    _ptr(dL_ddepths), _ptr(out["means3D"]), _ptr(out["log_scales"]),
                                                    _ptr(out["quats"]), _stream(dev)),
          "bgs_preprocess_backward_batched")
    return out


def bin_and_sort_batched(plan: Plan, means2D, radii, depths, cams, tile=(16, 16), point_list=None, ranges=None,
                         no_sync: bool = False, conic_opacity=None):
    """bgs_bin_and_sort_batched: returns (point_list, ranges [sum T_v, 2], K).  With no_sync the call
    only enqueues work (graph capture): K is returned as -1 and an overflow raises a device check.
    With ``conic_opacity`` [V*N, 4] the lists are truncated as in ``bin_and_sort``."""
    R = means2D.shape[0]
    V = len(cams)
    assert R % V == 0
    N = R // V
    _req(means2D, "means2D", torch.float32, (R, 2))
    _req(radii, "radii", torch.int32, (R,))
    _req(depths, "depths", torch.float32, (R,))
    if conic_opacity is not None:
        _req(conic_opacity, "conic_opacity", torch.float32, (R, 4))
    dev = means2D.device
    _, T = tile_counts(cams, tile)
    if ranges is None:
        ranges = torch.empty((T, 2), dtype=torch.int32, device=dev)
    if point_list is None:
        point_list = torch.empty(max(4 * R, 1024), dtype=torch.int32, device=dev)
    vw = _views(cams)
    K, need = ctypes.c_int64(0), ctypes.c_int64(0)
    flags = _lib.BIN_NO_SYNC if no_sync else 0
    for _ in range(2):
        code = plan._lib.bgs_bin_and_sort_batched(plan.handle, V, vw, N, _ptr(means2D), _ptr(radii), _ptr(depths),
                                                  _ptr(conic_opacity) if conic_opacity is not None else None,
                                                  tile[0], tile[1], _ptr(point_list), point_list.numel(),
                                                  _ptr(ranges), flags, ctypes.byref(K), ctypes.byref(need),
                                                  _stream(dev))
        if code == _lib.BGS_ERR_CAPACITY and not no_sync and need.value > point_list.numel():
            point_list = torch.empty(int(need.value * 1.1) + 1024, dtype=torch.int32, device=dev)
            continue
        check(code, "bgs_bin_and_sort_batched")
        break
    return point_list, ranges, (-1 if no_sync else int(K.value))


def alloc_view_outputs(cams, device, n_eval=False):
    outs = []
    for c in cams:
        H, W = c["H"], c["W"]
        o = dict(color=torch.empty((3, H, W), device=device), depth=torch.empty((H, W), device=device),
                 alpha=torch.empty((H, W), device=device), final_T=torch.empty((H, W), device=device),
                 n_contrib=torch.empty((H, W), dtype=torch.int32, device=device))
        if n_eval:
            o["n_eval"] = torch.empty((H, W), dtype=torch.int32, device=device)
        outs.append(o)
    return outs


def render_forward_batched(plan: Plan, means2D, conic_opacity, colors, depths, point_list, num_entries: int, ranges,
                           cams, tile=(16, 16), bg=(0.0, 0.0, 0.0), mode="auto", outs=None, n_eval=False):
    """bgs_render_forward_batched: returns the list of per-view output dicts.  colors is
    [N, 3] (shared by the views) or, for view-dependent colours, [V*N, 3] (one row per
    record, e.g. from sh_to_rgb; bgs_render_forward_batched_vc)."""
    R, V = means2D.shape[0], len(cams)
    N = R // V
    assert R == N * V and colors.shape[0] in (N, R)
    per_view = colors.shape[0] == R and V > 1
    _req(means2D, "means2D", torch.float32, (R, 2))
    _req(conic_opacity, "conic_opacity", torch.float32, (R, 4))
    _req(colors, "colors", torch.float32, (colors.shape[0], 3))
    _req(depths, "depths", torch.float32, (R,))
    dev = means2D.device
    if outs is None:
        outs = alloc_view_outputs(cams, dev, n_eval)
    vw = _views(cams, outs=outs)
    bgv = (ctypes.c_float * 3)(*[float(v) for v in bg])
    m = MODES[mode] if isinstance(mode, str) else int(mode)
    fn = plan._lib.bgs_render_forward_batched_vc if per_view else plan._lib.bgs_render_forward_batched
    check(fn(plan.handle, V, vw, N, _ptr(means2D), _ptr(conic_opacity), _ptr(colors), _ptr(depths),
             _ptr(point_list), int(num_entries), _ptr(ranges), tile[0], tile[1], bgv, m, _stream(dev)),
          "bgs_render_forward_batched")
    return outs


def render_backward_batched(plan: Plan, means2D, conic_opacity, colors, depths, point_list, num_entries: int, ranges,
                            cams, fw_outs, grads_in, tile=(16, 16), bg=(0.0, 0.0, 0.0), mode="auto", out=None):
    """bgs_render_backward_batched: grads_in[v] = dict(color=[3,H,W], depth=None|[H,W], alpha=None|[H,W]).
    Returns dict(means2D [V*N,2], conic [V*N,3], opacity [V*N], colors, depths [V*N]) with colors
    [N,3] summed over the views, or [V*N,3] per record when colors is [V*N,3] (view-dependent)."""
    R, V = means2D.shape[0], len(cams)
    N = R // V
    assert R == N * V and colors.shape[0] in (N, R)
    per_view = colors.shape[0] == R and V > 1
    dev = means2D.device
    if out is None:
        out = dict(means2D=torch.empty((R, 2), device=dev), conic=torch.empty((R, 3), device=dev),
                   opacity=torch.empty(R, device=dev), colors=torch.empty((colors.shape[0], 3), device=dev),
                   depths=torch.empty(R, device=dev))
    vw = _views(cams, fw=fw_outs, grads=grads_in)
    bgv = (ctypes.c_float * 3)(*[float(v) for v in bg])
    m = MODES[mode] if isinstance(mode, str) else int(mode)
    fn = plan._lib.bgs_render_backward_batched_vc if per_view else plan._lib.bgs_render_backward_batched
    check(fn(plan.handle, V, vw, N, _ptr(means2D), _ptr(conic_opacity), _ptr(colors), _ptr(depths),
             _ptr(point_list), int(num_entries), _ptr(ranges), tile[0], tile[1], bgv, m, _ptr(out["means2D"]),
             _ptr(out["conic"]), _ptr(out["opacity"]), _ptr(out["colors"]), _ptr(out.get("depths")), _stream(dev)),
          "bgs_render_backward_batched")
    return out


# ---- view-dependent colour from spherical harmonics (Sec. 2.1) ---------------------------

def sh_to_rgb(plan: Plan, sh, means3D, cams, degree: int, clamped: bool = False, out=None):
    """bgs_sh_to_rgb: sh [N, K, 3] (K >= (degree+1)^2), means3D [N, 3], cams: list of V camera
    dicts (their viewmats give the camera centres).  Returns rgb [V*N, 3] (and, with
    clamped=True, the clamp flags [V*N, 3] uint8)."""
    N, V = means3D.shape[0], len(cams)
    _req(sh, "sh", torch.float32)
    assert sh.dim() == 3 and sh.shape[0] == N and sh.shape[2] == 3 and sh.shape[1] >= (degree + 1) ** 2
    _req(means3D, "means3D", torch.float32, (N, 3))
    dev = means3D.device
    rgb = out if out is not None else torch.empty((V * N, 3), device=dev)
    cl = torch.empty((V * N, 3), dtype=torch.uint8, device=dev) if clamped else None
    vw = _views(cams)
    check(plan._lib.bgs_sh_to_rgb(plan.handle, V, vw, N, int(degree), sh.shape[1], _ptr(sh), _ptr(means3D),
                                  _ptr(rgb), _ptr(cl), _stream(dev)), "bgs_sh_to_rgb")
    return (rgb, cl) if clamped else rgb


def sh_to_rgb_backward(plan: Plan, sh, means3D, cams, degree: int, dL_drgb):
    """bgs_sh_to_rgb_backward: dL_drgb [V*N, 3] -> (dL/dsh [N, K, 3], dL/dmeans3D [N, 3]),
    summed over the views."""
    N, V = means3D.shape[0], len(cams)
    _req(dL_drgb, "dL_drgb", torch.float32, (V * N, 3))
    dev = means3D.device
    d_sh, d_m = torch.empty_like(sh), torch.empty((N, 3), device=dev)
    vw = _views(cams)
    check(plan._lib.bgs_sh_to_rgb_backward(plan.handle, V, vw, N, int(degree), sh.shape[1], _ptr(sh),
                                           _ptr(means3D), _ptr(dL_drgb), _ptr(d_sh), _ptr(d_m), _stream(dev)),
          "bgs_sh_to_rgb_backward")
    return d_sh, d_m


class SHFunction(torch.autograd.Function):
    """Differentiable view-dependent colour: (sh [N,K,3], means3D [N,3]) -> rgb [V*N,3]."""

    @staticmethod
    def forward(ctx, sh, means3D, plan, cams, degree):
        sh, m3 = sh.contiguous(), means3D.contiguous()
        ctx.plan, ctx.cams, ctx.degree = plan, cams, degree
        ctx.save_for_backward(sh, m3)
        return sh_to_rgb(plan, sh, m3, cams, degree)

    @staticmethod
    def backward(ctx, g_rgb):
        sh, m3 = ctx.saved_tensors
        d_sh, d_m = sh_to_rgb_backward(ctx.plan, sh, m3, ctx.cams, ctx.degree, g_rgb.contiguous())
        return d_sh, d_m, None, None, None


def autotune_render(plan: Plan, means2D, conic_opacity, colors, depths, point_list, num_entries: int, ranges, cams,
                    tile=(16, 16), bg=(0.0, 0.0, 0.0), backward: bool = True, outs=None, grads_in=None, out=None):
    """bgs_autotune_render: times candidate plan knobs (pixel rows per lane, heavy-tile threshold,
    pixels per Gaussian-wise item, queue chunk) on this frame and keeps the fastest in the plan.
    Works for one view (cams of length 1) or several.  Returns (best ms, chosen knobs)."""
    R, N, V = means2D.shape[0], colors.shape[0], len(cams)
    dev = means2D.device
    if outs is None:
        outs = alloc_view_outputs(cams, dev)
    if backward and grads_in is None:
        grads_in = [dict(color=torch.zeros((3, c["H"], c["W"]), device=dev)) for c in cams]
    if backward and out is None:
        out = dict(means2D=torch.empty((R, 2), device=dev), conic=torch.empty((R, 3), device=dev),
                   opacity=torch.empty(R, device=dev), colors=torch.empty((N, 3), device=dev))
    vw = _views(cams, outs=outs, grads=grads_in if backward else None)
    bgv = (ctypes.c_float * 3)(*[float(v) for v in bg])
    best = ctypes.c_double(0)
    g = out or {}
    check(plan._lib.bgs_autotune_render(plan.handle, V, vw, N, _ptr(means2D), _ptr(conic_opacity), _ptr(colors),
                                        _ptr(depths), _ptr(point_list), int(num_entries), _ptr(ranges), tile[0],
                                        tile[1], bgv, int(bool(backward)), _ptr(g.get("means2D")),
                                        _ptr(g.get("conic")), _ptr(g.get("opacity")), _ptr(g.get("colors")),
                                        ctypes.byref(best), _stream(dev)), "bgs_autotune_render")
    return best.value, plan.desc()


def graph_begin(plan: Plan):
    check(plan._lib.bgs_graph_begin(plan.handle, _stream(plan.device)), "bgs_graph_begin")


def graph_end(plan: Plan):
    check(plan._lib.bgs_graph_end(plan.handle, _stream(plan.device)), "bgs_graph_end")


def graph_launch(plan: Plan):
    check(plan._lib.bgs_graph_launch(plan.handle, _stream(plan.device)), "bgs_graph_launch")


def probe_pipe_rates(plan: Plan):
    """Measured (FP32 FMA, MUFU ex2) operations per SM per clock on the plan's device."""
    a, b = ctypes.c_double(0), ctypes.c_double(0)
    check(plan._lib.bgs_probe_pipe_rates(plan.handle, ctypes.byref(a), ctypes.byref(b), _stream(plan.device)),
          "bgs_probe_pipe_rates")
    return a.value, b.value


def debug_exp2(x: torch.Tensor) -> torch.Tensor:
    _req(x, "x", torch.float32)
    y = torch.empty_like(x)
    check(_lib.load().bgs_debug_exp2(_ptr(x), _ptr(y), x.numel(), _stream(x.device)), "bgs_debug_exp2")
    return y
