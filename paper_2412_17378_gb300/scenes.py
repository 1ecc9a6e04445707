"""Seeded synthetic scenes and cameras for the balanced splat renderer.

This module draws random inputs only: Gaussian parameters, camera poses and target
images.  It contains none of the rasterizer's arithmetic (no projection, binning or
blending), so both the CUDA path and the FP64 oracle can consume its output.

The paper's measurements use an internal driving dataset (first training iteration,
960x540, Sec. 5.1-5.2) that is not available; these scenes stand in for it.  They are
shaped after its first-iteration imbalance: per-thread list lengths "from hundreds to
hundreds of thousands" (Sec. 5.2.1), i.e. a few dense clusters over a sparse background.

Conventions (shared by every scene):
  * camera looks down +z; ``viewmat`` is the row-major 4x4 world->camera transform;
  * fx = fy = W, cx = (W-1)/2, cy = (H-1)/2, near plane 0.2, low-pass 0.3;
  * quaternions are (w, x, y, z), drawn as normalised 4-D normal vectors (uniform on S^3);
  * opacities are already passed through the sigmoid;
  * colors are RGB in [0, 1] (SH degree 0); background black.
"""
from __future__ import annotations

import math

import numpy as np

__all__ = ["camera", "look_at_camera", "scene_config", "CONFIGS", "frustum_uniform",
           "cluster_points", "veil_points", "arc_cameras", "target_image"]


def camera(W: int, H: int, viewmat=None, fx: float | None = None, fy: float | None = None,
           cx: float | None = None, cy: float | None = None, near: float = 0.2,
           lowpass: float = 0.3) -> dict:
    """Pinhole camera dict (fx = fy = W unless given, principal point at the image centre)."""
    fx = float(W) if fx is None else float(fx)
    fy = fx if fy is None else float(fy)
    return dict(W=int(W), H=int(H), fx=fx, fy=fy,
                cx=(W - 1) / 2.0 if cx is None else float(cx),
                cy=(H - 1) / 2.0 if cy is None else float(cy),
                viewmat=np.eye(4) if viewmat is None else np.asarray(viewmat, np.float64),
                near=float(near), lowpass=float(lowpass))


def look_at_camera(W: int, H: int, eye, target, up=(0.0, -1.0, 0.0)) -> dict:
    """Camera at ``eye`` whose +z axis points at ``target`` (image y grows along ``up``'s
    opposite, matching the identity camera whose image y axis is world +y)."""
    eye = np.asarray(eye, np.float64)
    f = np.asarray(target, np.float64) - eye
    f /= np.linalg.norm(f)
    # image x axis (camera +x) and y axis (camera +y) so that the identity pose is recovered
    # for eye = 0, target = +z
    y_hint = -np.asarray(up, np.float64)
    x = np.cross(y_hint, f)
    x /= np.linalg.norm(x)
    y = np.cross(f, x)
    R = np.stack([x, y, f])            # rows: camera axes in world coordinates
    V = np.eye(4)
    V[:3, :3] = R
    V[:3, 3] = -R @ eye
    return camera(W, H, viewmat=V)


def frustum_uniform(rng, n: int, W: int, H: int, z_lo=2.0, z_hi=6.0):
    """Points uniform in depth z ~ U[z_lo, z_hi] and uniform over the identity camera's
    image cross-section at that depth (fx = fy = W)."""
    z = rng.uniform(z_lo, z_hi, n)
    u = rng.uniform(0.0, W, n)
    v = rng.uniform(0.0, H, n)
    f = float(W)
    x = (u - (W - 1) / 2.0) / f * z
    y = (v - (H - 1) / 2.0) / f * z
    return np.stack([x, y, z], 1)


def cluster_points(rng, n: int, W: int, H: int, pu: float, pv: float, z: float, sigma: float):
    """Isotropic 3-D normal cluster centred on the identity camera's ray through pixel
    (pu*W, pv*H) at depth z."""
    f = float(W)
    c = np.array([(pu * W - (W - 1) / 2.0) / f * z, (pv * H - (H - 1) / 2.0) / f * z, z])
    return c[None, :] + sigma * rng.standard_normal((n, 3))


def _quats(rng, n):
    q = rng.standard_normal((n, 4))
    return q / np.linalg.norm(q, axis=1, keepdims=True)


def _sigmoid(x):
    return 1.0 / (1.0 + np.exp(-x))


def _gaussians(means, log_scales, quats, opac, colors):
    f = lambda a: np.ascontiguousarray(a, np.float32)
    return dict(means3D=f(means), log_scales=f(log_scales), quats=f(quats), opacities=f(opac),
                colors=f(colors))


def arc_cameras(sizes, radius=4.0, centre=(0.0, 0.0, 4.0), yaw_deg=30.0):
    """Cameras on a +-yaw arc of the given radius around ``centre``, all looking at it.
    ``sizes`` is a list of (W, H); camera k sits at yaw linspace(-yaw, yaw)[k]."""
    centre = np.asarray(centre, np.float64)
    cams = []
    n = len(sizes)
    yaws = np.linspace(-yaw_deg, yaw_deg, n) if n > 1 else np.zeros(1)
    for (W, H), yd in zip(sizes, yaws):
        t = math.radians(yd)
        eye = centre + radius * np.array([math.sin(t), 0.0, -math.cos(t)])
        cams.append(look_at_camera(W, H, eye, centre))
    return cams


def target_image(seed: int, W: int, H: int):
    """Random L2-loss target image, float32 [3,H,W], U[0,1]."""
    rng = np.random.default_rng([seed, 7])
    return rng.uniform(0.0, 1.0, (3, H, W)).astype(np.float32)


def _config1(scale=1.0):
    rng = np.random.default_rng(0)
    N = max(1, int(10_000 * scale))
    means = np.stack([rng.uniform(-1, 1, N), rng.uniform(-1, 1, N), rng.uniform(2, 6, N)], 1)
    g = _gaussians(means, rng.normal(-3.5, 0.5, (N, 3)), _quats(rng, N),
                   _sigmoid(rng.normal(0, 1, N)), rng.uniform(0, 1, (N, 3)))
    return dict(name="cfg1_256x256_10k", gaussians=g, cameras=[camera(256, 256)], backward=False)


def _clustered(rng, N, W, H, frac_cluster=0.8, sigma_c=0.189):
    nc = int(round(N * frac_cluster))
    pts = np.concatenate([cluster_points(rng, nc, W, H, 0.3, 0.6, 4.0, sigma_c),
                          frustum_uniform(rng, N - nc, W, H)])
    return pts


def _config2(scale=1.0, W=1920, H=1080):
    rng = np.random.default_rng(2)
    N = max(1, int(1_000_000 * scale))
    means = _clustered(rng, N, 1920, 1080)
    g = _gaussians(means, rng.normal(-4.0, 0.7, (N, 3)), _quats(rng, N),
                   _sigmoid(rng.normal(0, 1.5, N)), rng.uniform(0, 1, (N, 3)))
    return dict(name=f"cfg2_{W}x{H}_{N}", gaussians=g, cameras=[camera(W, H)], backward=True)


def _config3(stage: str, scale=1.0):
    W, H = 1280, 720
    if stage == "early":
        rng = np.random.default_rng([3, 0])
        N = max(1, int(100_000 * scale))
        ls = rng.normal(-2.0, 0.5, (N, 3))
        op = rng.uniform(0.05, 0.3, N)
    else:
        rng = np.random.default_rng([3, 1])
        N = max(1, int(3_000_000 * scale))
        ls = rng.normal(-5.0, 0.5, (N, 3))
        op = rng.uniform(0.5, 1.0, N)
    means = frustum_uniform(rng, N, W, H)
    g = _gaussians(means, ls, _quats(rng, N), op, rng.uniform(0, 1, (N, 3)))
    return dict(name=f"cfg3{stage}_{W}x{H}_{N}", gaussians=g, cameras=[camera(W, H)], backward=True)


def drift_scene(frac: float, scale=1.0, seed: int = 31) -> dict:
    """A stage of a synthetic training run between config 3-early (frac = 0: 100k large,
    faint Gaussians) and config 3-late (frac = 1: 3M small, opaque ones) at 1280x720:
    the Gaussian count grows geometrically, the mean log-scale falls linearly from -2 to
    -5 and the opacity range moves from U[0.05, 0.3] to U[0.5, 1] -- the densification /
    sharpening drift behind the paper's inflection point (Sec. 4.4, Sec. 5.2.2)."""
    f = min(max(float(frac), 0.0), 1.0)
    W, H = 1280, 720
    rng = np.random.default_rng([seed, int(round(1000 * f))])
    N = max(1, int(100_000 * (30.0 ** f) * scale))
    ls = rng.normal(-2.0 - 3.0 * f, 0.5, (N, 3))
    op = rng.uniform(0.05 + 0.45 * f, 0.3 + 0.7 * f, N)
    means = frustum_uniform(rng, N, W, H)
    g = _gaussians(means, ls, _quats(rng, N), op, rng.uniform(0, 1, (N, 3)))
    return dict(name=f"drift{f:.2f}_{W}x{H}_{N}", gaussians=g, cameras=[camera(W, H)], backward=True)


def _config4(scale=1.0):
    rng = np.random.default_rng(4)
    N = max(1, int(2_000_000 * scale))
    means = _clustered(rng, N, 1920, 1080)
    g = _gaussians(means, rng.normal(-4.0, 0.7, (N, 3)), _quats(rng, N),
                   _sigmoid(rng.normal(0, 1.5, N)), rng.uniform(0, 1, (N, 3)))
    sizes = []
    for k in range(16):
        sizes.append((640, 360) if k % 4 == 0 else ((1920, 1080) if k % 4 == 2 else (1280, 720)))
    return dict(name=f"cfg4_16views_{N}", gaussians=g, cameras=arc_cameras(sizes), backward=True)


def _config5(scale=1.0, sigma_c=(0.25, 0.2, 0.15)):
    rng = np.random.default_rng(5)
    N = max(1, int(4_000_000 * scale))
    W, H = 3840, 2160
    n1, n2, n3 = int(0.6 * N), int(0.2 * N), int(0.1 * N)
    pts = np.concatenate([cluster_points(rng, n1, W, H, 0.3, 0.6, 4.0, sigma_c[0]),
                          cluster_points(rng, n2, W, H, 0.7, 0.35, 3.5, sigma_c[1]),
                          cluster_points(rng, n3, W, H, 0.55, 0.5, 5.0, sigma_c[2]),
                          frustum_uniform(rng, N - n1 - n2 - n3, W, H)])
    g = _gaussians(pts, rng.normal(-4.5, 1.0, (N, 3)), _quats(rng, N),
                   _sigmoid(rng.normal(0.5, 1.5, N)), rng.uniform(0, 1, (N, 3)))
    cams = [camera(W, H)] + arc_cameras([(1920, 1080)] * 8)
    return dict(name=f"cfg5_4k+8x1080p_{N}", gaussians=g, cameras=cams, backward=True)


def veil_points(rng, n: int, W: int, H: int, u0: float, v0: float, half: float, z_lo=2.0, z_hi=6.0):
    """Points whose projections fall uniformly in the (2 half)^2 pixel window centred on
    (u0, v0) of the identity camera (fx = fy = W), depth z ~ U[z_lo, z_hi]."""
    z = rng.uniform(z_lo, z_hi, n)
    u = rng.uniform(u0 - half, u0 + half, n)
    v = rng.uniform(v0 - half, v0 + half, n)
    f = float(W)
    return np.stack([(u - (W - 1) / 2.0) / f * z, (v - (H - 1) / 2.0) / f * z, z], 1)


def _heavy(scale=1.0, W=1920, H=1080):
    """A frame with a few ultra-heavy tiles: config 2's clustered scene at a fifth of its
    Gaussians, plus a veil of 100k faint Gaussians (opacity U[0.001, 0.0045], most of
    their pairs below the 1/255 cut; projected sigma ~ 5 px) over a 48 x 48 pixel window
    in front of the scene (z in [1, 1.9]).  The ~35 tiles under the veil get lists of
    tens of thousands of entries, and their pixels walk through the whole veil (its
    transmittance stays near 0.5) before the scene behind it stops them, while the rest
    of the frame is light: the workload for which the paper's Gaussian-wise parallelism
    is meant (Sec. 4.2)."""
    rng = np.random.default_rng(6)
    Nb = max(1, int(200_000 * scale))
    Nv = max(1, int(100_000 * scale))
    bg = _clustered(rng, Nb, W, H)
    veil = veil_points(rng, Nv, W, H, 0.62 * W, 0.4 * H, 24.0, 1.0, 1.9)
    means = np.concatenate([bg, veil])
    ls = np.concatenate([rng.normal(-4.0, 0.7, (Nb, 3)), rng.normal(-5.6, 0.15, (Nv, 3))])
    op = np.concatenate([_sigmoid(rng.normal(0, 1.5, Nb)), rng.uniform(0.001, 0.0045, Nv)])
    g = _gaussians(means, ls, _quats(rng, Nb + Nv), op, rng.uniform(0, 1, (Nb + Nv, 3)))
    return dict(name=f"heavy_{W}x{H}_{Nb}+{Nv}veil", gaussians=g, cameras=[camera(W, H)], backward=True)


def fd_crop_scene(seed: int = 5, n: int = 512, size: int = 64):
    """512 Gaussians whose centres fall in a 64x64 crop, rendered as a 64x64 image: the
    camera's principal point is shifted so that the crop becomes the whole image."""
    rng = np.random.default_rng([seed, 64])
    Wf = 1920
    z = rng.uniform(3.0, 5.0, n)
    u = rng.uniform(0.0, size, n)
    v = rng.uniform(0.0, size, n)
    x = (u - (size - 1) / 2.0) / Wf * z
    y = (v - (size - 1) / 2.0) / Wf * z
    means = np.stack([x, y, z], 1)
    g = _gaussians(means, rng.normal(-5.5, 0.4, (n, 3)), _quats(rng, n),
                   _sigmoid(rng.normal(0.0, 1.0, n)), rng.uniform(0, 1, (n, 3)))
    cam = camera(size, size, fx=Wf, fy=Wf)
    return dict(name=f"fdcrop_{size}x{size}_{n}", gaussians=g, cameras=[cam], backward=True)


CONFIGS = {
    "cfg1": _config1,
    "cfg2": _config2,
    "cfg3early": lambda scale=1.0: _config3("early", scale),
    "cfg3late": lambda scale=1.0: _config3("late", scale),
    "cfg4": _config4,
    "cfg5": _config5,
    "heavy": _heavy,
    "fdcrop": lambda scale=1.0: fd_crop_scene(),
}


def scene_config(name: str, scale: float = 1.0) -> dict:
    """Scene dict: ``gaussians`` (float32 arrays), ``cameras`` (list of camera dicts),
    ``backward`` (whether the config trains).  ``scale`` shrinks the Gaussian count."""
    return CONFIGS[name](scale=scale)
