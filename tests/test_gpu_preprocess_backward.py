"""GPU parity of the projection backward (bgs_preprocess_backward and its batched form)
against the FP64 oracle's chain rule through Eq. 2-3, and of the differentiable chain
projection -> render through torch autograd against the oracle's composed gradients."""
import numpy as np
import pytest

import oracle
from helpers import ROW_EPS_PROJECTION, ROW_EPS_SH, compare_grad, scene, term_eps
from paper_2412_17378_gb300 import scenes

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def R():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2412_17378_gb300 import raster
    return raster


def _gpu(a):
    return torch.from_numpy(np.ascontiguousarray(a, np.float32)).cuda()


def _rotated_scene(n=3000, seed=21):
    """Gaussians around the view axis of a rotated, translated camera, some beyond the
    tangent clamp, with unnormalised quaternions."""
    rng = np.random.default_rng(seed)
    cam = scenes.look_at_camera(320, 200, eye=(0.4, -0.3, -1.0), target=(0.0, 0.1, 3.0))
    V = cam["viewmat"]
    lim = 1.3 * cam["W"] / (2 * cam["fx"])
    z = rng.uniform(1.0, 6.0, n)
    t = np.stack([rng.uniform(-1.6, 1.6, n) * lim * z, rng.uniform(-0.9, 0.9, n) * lim * z, z], 1)
    m3 = np.linalg.solve(V[:3, :3], (t - V[:3, 3]).T).T
    g = dict(means3D=m3.astype(np.float32), log_scales=rng.normal(-3.0, 0.7, (n, 3)).astype(np.float32),
             quats=(rng.normal(size=(n, 4)) * rng.uniform(0.5, 2.0, (n, 1))).astype(np.float32),
             opacities=rng.uniform(0.05, 0.95, n).astype(np.float32))
    return g, cam


@pytest.mark.parametrize("which", ["rotated", "cfg2"])
def test_projection_backward_matches_oracle(R, which):
    if which == "rotated":
        g, cam = _rotated_scene()
    else:
        s = scene("cfg2", 0.02)
        g, cam = s["gaussians"], s["cameras"][0]
    plan = R.Plan()
    d = {k: _gpu(v) for k, v in g.items()}
    pre = R.preprocess(plan, d["means3D"], d["log_scales"], d["quats"], d["opacities"], cam)
    radii = pre["radii"]
    n = radii.numel()
    rng = np.random.default_rng(3)
    gm, gc, gd = rng.normal(size=(n, 2)), rng.normal(size=(n, 3)), rng.normal(size=n)
    got = R.preprocess_backward(plan, d["means3D"], d["log_scales"], d["quats"], cam, radii, _gpu(gm), _gpu(gc),
                                _gpu(gd))
    torch.cuda.synchronize()
    rad = radii.cpu().numpy()
    assert (rad > 0).sum() > n // 4
    ref = oracle.preprocess_backward(g["means3D"].astype(np.float64), g["log_scales"].astype(np.float64),
                                     g["quats"].astype(np.float64), cam, gm, gc, gd, radius=rad)
    for k in ("means3D", "log_scales", "quats"):
        out = got[k].cpu().numpy()
        assert not out[rad == 0].any(), k
        compare_grad(out, ref[k], k, row_eps=ROW_EPS_PROJECTION)
    plan.close()


def test_projection_backward_batched_sums_views(R):
    s = scene("cfg2", 0.004)
    g = s["gaussians"]
    cams = scenes.arc_cameras([(160, 96), (250, 130), (96, 64)], yaw_deg=20.0)
    plan = R.Plan()
    d = {k: _gpu(v) for k, v in g.items()}
    pre = R.preprocess_batched(plan, d["means3D"], d["log_scales"], d["quats"], d["opacities"], cams)
    N, V = g["means3D"].shape[0], len(cams)
    rng = np.random.default_rng(4)
    gm, gc, gd = rng.normal(size=(N * V, 2)), rng.normal(size=(N * V, 3)), rng.normal(size=N * V)
    got = R.preprocess_backward_batched(plan, d["means3D"], d["log_scales"], d["quats"], cams, pre["radii"],
                                        _gpu(gm), _gpu(gc), _gpu(gd))
    torch.cuda.synchronize()
    rad = pre["radii"].cpu().numpy()
    ref = {k: 0.0 for k in ("means3D", "log_scales", "quats")}
    for v, cam in enumerate(cams):
        sl = slice(v * N, (v + 1) * N)
        r = oracle.preprocess_backward(g["means3D"].astype(np.float64), g["log_scales"].astype(np.float64),
                                       g["quats"].astype(np.float64), cam, gm[sl], gc[sl], gd[sl], radius=rad[sl])
        for k in ref:
            ref[k] = ref[k] + r[k]
    for k in ref:
        compare_grad(got[k].cpu().numpy(), ref[k], f"batched {k}", row_eps=ROW_EPS_PROJECTION)
    plan.close()


def test_autograd_chain_projection_then_render(R):
    """torch autograd through PreprocessFunction and RenderFunction equals the oracle's
    render backward composed with its projection backward, on the GPU's projected inputs."""
    s = scene("cfg1", 0.3)
    g, cam = s["gaussians"], s["cameras"][0]
    W, H = cam["W"], cam["H"]
    plan = R.Plan()
    p = {k: _gpu(v).requires_grad_(k != "colors") for k, v in g.items()}
    m2, co, dp, radii = R.PreprocessFunction.apply(p["means3D"], p["log_scales"], p["quats"], p["opacities"], plan,
                                                   cam, (16, 16))
    binning = R.bin_and_sort(plan, m2.detach(), radii, dp.detach(), W, H)
    colors = _gpu(g["colors"]).requires_grad_(True)
    color, _, _ = R.render(plan, m2, co, colors, dp, binning, W, H, mode="pixel")
    # oracle on the same float32 projected values
    m2n, con, dpn = (t.detach().cpu().numpy() for t in (m2, co, dp))
    radn = radii.cpu().numpy()
    opl, org = oracle.bin_tiles(m2n, radn, dpn, W, H)
    ref_f = oracle.render(m2n, con, g["colors"], dpn, opl, org, W, H)
    rng = np.random.default_rng(5)
    gC = rng.normal(size=(3, H, W)).astype(np.float32)
    gC[:, ref_f["flags"] != 0] = 0
    (color * _gpu(gC)).sum().backward()
    ref_r = oracle.render_backward(m2n, con, g["colors"], dpn, opl, org, W, H, gC, abs_terms=True)
    eps = term_eps(int(ref_f["n_contrib"].max()))
    ref_p = oracle.preprocess_backward(g["means3D"].astype(np.float64), g["log_scales"].astype(np.float64),
                                       g["quats"].astype(np.float64), cam, ref_r["means2D"], ref_r["conic"],
                                       ref_r.get("depths"), radius=radn)
    for k in ("means3D", "log_scales", "quats"):
        compare_grad(p[k].grad.cpu().numpy(), ref_p[k], f"chain {k}", row_eps=ROW_EPS_PROJECTION)
    compare_grad(p["opacities"].grad.cpu().numpy(), ref_r["opacity"], "chain opacities", s=ref_r["abs_opacity"],
                 eps=eps)
    compare_grad(colors.grad.cpu().numpy(), ref_r["colors"], "chain colors", s=ref_r["abs_colors"], eps=eps)
    plan.close()


def test_autograd_chain_with_sh_colours(R):
    """The documented training step: PreprocessFunction, SHFunction (degree 3), binning and
    the differentiable render under torch autograd.  Every leaf gradient equals the oracle's
    render backward composed with its SH backward and projection backward (means3D takes
    both the projection's and the view direction's terms)."""
    s = scene("cfg1", 0.3)
    g, cam = s["gaussians"], s["cameras"][0]
    W, H = cam["W"], cam["H"]
    N = g["means3D"].shape[0]
    plan = R.Plan()
    p = {k: _gpu(v).requires_grad_(True) for k, v in g.items() if k != "colors"}
    rng = np.random.default_rng(8)
    sh_np = (rng.normal(size=(N, 16, 3)) * 0.05).astype(np.float32)  # view-dependent, never clamped
    sh_np[:, 0, :] += 1.0
    sh = _gpu(sh_np).requires_grad_(True)
    m2, co, dp, radii = R.PreprocessFunction.apply(p["means3D"], p["log_scales"], p["quats"], p["opacities"], plan,
                                                   cam, (16, 16))
    colors = R.SHFunction.apply(sh, p["means3D"], plan, [cam], 3)
    binning = R.bin_and_sort(plan, m2.detach(), radii, dp.detach(), W, H)
    color, _, _ = R.render(plan, m2, co, colors, dp, binning, W, H, mode="pixel")
    m2n, con, dpn, coln = (t.detach().cpu().numpy() for t in (m2, co, dp, colors))
    radn = radii.cpu().numpy()
    opl, org = oracle.bin_tiles(m2n, radn, dpn, W, H)
    ref_f = oracle.render(m2n, con, coln, dpn, opl, org, W, H)
    gC = rng.normal(size=(3, H, W)).astype(np.float32)
    gC[:, ref_f["flags"] != 0] = 0
    (color * _gpu(gC)).sum().backward()
    ref_r = oracle.render_backward(m2n, con, coln, dpn, opl, org, W, H, gC, abs_terms=True)
    eps = term_eps(int(ref_f["n_contrib"].max()))
    ref_p = oracle.preprocess_backward(g["means3D"].astype(np.float64), g["log_scales"].astype(np.float64),
                                       g["quats"].astype(np.float64), cam, ref_r["means2D"], ref_r["conic"],
                                       ref_r.get("depths"), radius=radn)
    Vm = np.asarray(cam["viewmat"], np.float64)
    campos = -np.linalg.solve(Vm[:3, :3], Vm[:3, 3])
    # no colour channel near the clamp at 0, so both sides take the same clamp decisions
    rgb_ref, _ = oracle.sh_to_rgb(sh_np.astype(np.float64), g["means3D"].astype(np.float64), campos, 3)
    assert rgb_ref.min() > 1e-3
    d_sh, d_m_sh = oracle.sh_to_rgb_backward(sh_np.astype(np.float64), g["means3D"].astype(np.float64), campos, 3,
                                             ref_r["colors"].reshape(1, N, 3))
    compare_grad(sh.grad.cpu().numpy(), d_sh, "sh chain: sh", row_eps=ROW_EPS_SH)
    compare_grad(p["means3D"].grad.cpu().numpy(), ref_p["means3D"] + d_m_sh, "sh chain: means3D",
                 row_eps=ROW_EPS_PROJECTION)
    for k in ("log_scales", "quats"):
        compare_grad(p[k].grad.cpu().numpy(), ref_p[k], f"sh chain: {k}", row_eps=ROW_EPS_PROJECTION)
    compare_grad(p["opacities"].grad.cpu().numpy(), ref_r["opacity"], "sh chain: opacities", s=ref_r["abs_opacity"],
                 eps=eps)
    plan.close()
