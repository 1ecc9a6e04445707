"""GPU parity of the view-dependent colour path (spherical harmonics of degree <= 3, Sec. 2.1)
and of the batched render with per-view colours, against the FP64 oracle on the same
float32 inputs."""
import numpy as np
import pytest

import oracle
from helpers import ROW_EPS_SH, compare_grad, compare_images, rel_l2, term_eps
from paper_2412_17378_gb300 import scenes

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

# float32 basis values (|Y| <= 1.1) and sums of up to 16 terms against FP64
SH_ATOL = 2e-6
SH_GRAD_REL = 2e-5
AMBIG = 1e-5  # channels whose pre-clamp value is this close to 0 may clamp differently


@pytest.fixture(scope="module")
def R():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2412_17378_gb300 import raster
    return raster


def _centre(cam):
    """Camera centre of a world -> camera viewmat, solved independently with numpy."""
    M = np.asarray(cam["viewmat"], np.float64)
    return -np.linalg.solve(M[:3, :3], M[:3, 3])


def _cams(V):
    if V == 1:
        return [scenes.camera(64, 48, viewmat=np.array([[1, 0, 0, 0.3], [0, 1, 0, -0.2], [0, 0, 1, 0.5],
                                                        [0, 0, 0, 1]], np.float64))]
    return scenes.arc_cameras([(64, 48)] * V, yaw_deg=25.0)


def _inputs(N, K, seed):
    rng = np.random.default_rng(seed)
    sh = (rng.normal(size=(N, K, 3)) * 0.3).astype(np.float32)
    sh[:, 0, :] = rng.normal(0.5, 1.5, size=(N, 3))  # ~6 % of the channels clamp at every degree
    m = (rng.normal(size=(N, 3)) + np.array([0.0, 0.0, 4.0])).astype(np.float32)
    return sh, m


def _oracle_fwd(sh, m, cams, degree):
    cp = np.stack([_centre(c) for c in cams])
    rgb, cl = oracle.sh_to_rgb(sh.astype(np.float64), m.astype(np.float64), cp, degree)
    # the pre-clamp value: rgb where unclamped; 1 - rgb(-sh) where clamped (-s + 1/2 > 1 there)
    neg = sh.astype(np.float64).copy()
    neg[:, :(degree + 1) ** 2, :] *= -1
    rgb_neg, _ = oracle.sh_to_rgb(neg, m.astype(np.float64), cp, degree)
    s = np.where(cl == 1, 1.0 - rgb_neg, rgb)
    return rgb.reshape(-1, 3), cl.reshape(-1, 3), s.reshape(-1, 3), cp


@pytest.mark.parametrize("V", [1, 3])
@pytest.mark.parametrize("degree", [0, 1, 2, 3])
def test_sh_forward_matches_oracle(R, degree, V):
    plan = R.Plan()
    sh, m = _inputs(3000, 16, 40 + degree)
    cams = _cams(V)
    rgb, cl = R.sh_to_rgb(plan, torch.from_numpy(sh).cuda(), torch.from_numpy(m).cuda(), cams, degree, clamped=True)
    torch.cuda.synchronize()
    ref, ref_cl, s, _ = _oracle_fwd(sh, m, cams, degree)
    rgb, cl = rgb.cpu().numpy(), cl.cpu().numpy()
    sure = np.abs(s) > AMBIG
    assert sure.mean() > 0.99 and (ref_cl == 1).any()
    np.testing.assert_array_equal(cl[sure], ref_cl[sure])
    np.testing.assert_allclose(rgb[sure], ref[sure], rtol=0, atol=SH_ATOL * 2)
    assert np.abs(rgb[~sure]).max(initial=0.0) <= AMBIG + SH_ATOL
    plan.close()


@pytest.mark.parametrize("V", [1, 3])
@pytest.mark.parametrize("degree", [0, 1, 2, 3])
def test_sh_backward_matches_oracle(R, degree, V):
    plan = R.Plan()
    N = 3000
    sh, m = _inputs(N, 16, 60 + degree)
    cams = _cams(V)
    _, _, s, cp = _oracle_fwd(sh, m, cams, degree)
    g = np.random.default_rng(7).normal(size=(V * N, 3)).astype(np.float32)
    g[np.abs(s) <= AMBIG] = 0.0  # ambiguous clamp decisions pass no gradient on either side
    d_sh, d_m = R.sh_to_rgb_backward(plan, torch.from_numpy(sh).cuda(), torch.from_numpy(m).cuda(), cams, degree,
                                     torch.from_numpy(g).cuda())
    torch.cuda.synchronize()
    r_sh, r_m = oracle.sh_to_rgb_backward(sh.astype(np.float64), m.astype(np.float64), cp, degree,
                                          g.reshape(V, N, 3).astype(np.float64))
    compare_grad(d_sh.cpu().numpy(), r_sh, f"degree {degree} V {V} sh", SH_GRAD_REL, row_eps=ROW_EPS_SH)
    if degree == 0:
        assert np.abs(d_m.cpu().numpy()).max() == 0.0  # the DC term does not depend on the direction
    else:
        compare_grad(d_m.cpu().numpy(), r_m, f"degree {degree} V {V} means3D", SH_GRAD_REL, row_eps=ROW_EPS_SH)
    plan.close()


@pytest.mark.parametrize("stride,offset", [(9, 0), (16, 0), (16, 1), (10, 0)])
def test_sh_strides_and_alignment(R, stride, offset):
    """Degree 2 (9 rows) in row blocks of 9, 10 and 16 rows, and at a pointer that is not
    16-byte aligned: the scalar and float4 load paths agree with the oracle, and gradient
    rows past the 9 used ones are zero."""
    plan = R.Plan()
    N, degree = 2000, 2
    sh, m = _inputs(N, stride, 80 + stride)
    cams = _cams(2)
    store = torch.zeros(N * stride * 3 + 4, device="cuda")
    store[offset:offset + sh.size] = torch.from_numpy(sh.ravel()).cuda()
    sh_t = store[offset:offset + sh.size].view(N, stride, 3)
    assert (sh_t.data_ptr() % 16 == 0) == (offset == 0)
    rgb = R.sh_to_rgb(plan, sh_t, torch.from_numpy(m).cuda(), cams, degree)
    ref, ref_cl, s, cp = _oracle_fwd(sh, m, cams, degree)
    sure = np.abs(s) > AMBIG
    np.testing.assert_allclose(rgb.cpu().numpy()[sure], ref[sure], rtol=0, atol=SH_ATOL * 2)
    g = np.random.default_rng(9).normal(size=(2 * N, 3)).astype(np.float32)
    g[~sure] = 0.0
    d_sh, d_m = R.sh_to_rgb_backward(plan, sh_t, torch.from_numpy(m).cuda(), cams, degree,
                                     torch.from_numpy(g).cuda())
    r_sh, r_m = oracle.sh_to_rgb_backward(sh.astype(np.float64), m.astype(np.float64), cp, degree,
                                          g.reshape(2, N, 3).astype(np.float64))
    d_sh = d_sh.cpu().numpy()
    compare_grad(d_sh, r_sh, "strided sh", SH_GRAD_REL, row_eps=ROW_EPS_SH)
    assert (d_sh[:, 9:, :] == 0).all()
    compare_grad(d_m.cpu().numpy(), r_m, "strided means3D", SH_GRAD_REL, row_eps=ROW_EPS_SH)
    plan.close()


def test_sh_autograd_function(R):
    plan = R.Plan()
    N, degree = 1500, 3
    sh, m = _inputs(N, 16, 90)
    cams = _cams(2)
    sh_t = torch.from_numpy(sh).cuda().requires_grad_(True)
    m_t = torch.from_numpy(m).cuda().requires_grad_(True)
    rgb = R.SHFunction.apply(sh_t, m_t, plan, cams, degree)
    w = torch.from_numpy(np.random.default_rng(3).normal(size=(2 * N, 3)).astype(np.float32)).cuda()
    _, _, s, cp = _oracle_fwd(sh, m, cams, degree)
    w[torch.from_numpy(np.abs(s) <= AMBIG).cuda()] = 0.0
    (rgb * w).sum().backward()
    r_sh, r_m = oracle.sh_to_rgb_backward(sh.astype(np.float64), m.astype(np.float64), cp, degree,
                                          w.cpu().numpy().reshape(2, N, 3).astype(np.float64))
    compare_grad(sh_t.grad.cpu().numpy(), r_sh, "autograd sh", SH_GRAD_REL, row_eps=ROW_EPS_SH)
    compare_grad(m_t.grad.cpu().numpy(), r_m, "autograd means3D", SH_GRAD_REL, row_eps=ROW_EPS_SH)
    plan.close()


def test_batched_render_with_view_dependent_colours(R):
    """Three views of one Gaussian set whose colours come from degree-3 SH per view: the
    batched render takes colours [V*N, 3] (bgs_render_*_batched_vc); every view's image and
    per-record colour gradient match the oracle run on that view with those colours."""
    s = scenes.scene_config("cfg2", 0.004)
    g = s["gaussians"]
    N = g["means3D"].shape[0]
    cams = scenes.arc_cameras([(160, 96), (250, 130), (96, 64)], yaw_deg=20.0)
    V = len(cams)
    plan = R.Plan(heavy_threshold=40, gw_pixels=2)
    sh = (np.random.default_rng(12).normal(size=(N, 16, 3)) * 0.2).astype(np.float32)
    sh[:, 0, :] += 1.0
    rgb = R.sh_to_rgb(plan, torch.from_numpy(sh).cuda(), torch.from_numpy(g["means3D"].astype(np.float32)).cuda(),
                      cams, 3)
    rgb_np = rgb.cpu().numpy().astype(np.float64)
    per_view = []
    for cam in cams:
        pp = oracle.preprocess(g["means3D"], g["log_scales"], g["quats"], g["opacities"], cam)
        per_view.append(dict(means2D=pp["means2D"].astype(np.float32), conic_opacity=pp["conic_opacity"].astype(np.float32),
                             depths=pp["depth"].astype(np.float32), radii=pp["radius"].astype(np.int32)))
    st = lambda k: torch.from_numpy(np.concatenate([pv[k] for pv in per_view])).cuda()
    m2, co, dp = st("means2D"), st("conic_opacity"), st("depths")
    pl, rg, K = R.bin_and_sort_batched(plan, m2, st("radii"), dp, cams)
    outs = R.render_forward_batched(plan, m2, co, rgb, dp, pl, K, rg, cams, mode="auto")
    rng = np.random.default_rng(13)
    grads_in, refs, nc_max = [], [], 0
    for v, cam in enumerate(cams):
        pv = per_view[v]
        opl, org = oracle.bin_tiles(pv["means2D"], pv["radii"], pv["depths"], cam["W"], cam["H"])
        cols = rgb_np[v * N:(v + 1) * N]
        ref = oracle.render(pv["means2D"], pv["conic_opacity"], cols, pv["depths"], opl, org, cam["W"], cam["H"])
        compare_images(outs[v]["color"].cpu().numpy(), ref, what=f"view {v}")
        gC = rng.normal(size=(3, cam["H"], cam["W"])).astype(np.float32)
        gC[:, ref["flags"] != 0] = 0
        grads_in.append(dict(color=torch.from_numpy(gC).cuda(), depth=None, alpha=None))
        refs.append((opl, org, cols, gC))
        nc_max = max(nc_max, int(ref["n_contrib"].max()))
    gr = R.render_backward_batched(plan, m2, co, rgb, dp, pl, K, rg, cams, outs, grads_in, mode="auto")
    torch.cuda.synchronize()
    plan.check()
    assert gr["colors"].shape == (V * N, 3)
    for v, cam in enumerate(cams):
        opl, org, cols, gC = refs[v]
        pv = per_view[v]
        og = oracle.render_backward(pv["means2D"], pv["conic_opacity"], cols, pv["depths"], opl, org, cam["W"],
                                    cam["H"], gC, abs_terms=True)
        compare_grad(gr["colors"][v * N:(v + 1) * N].cpu().numpy(), og["colors"], f"view {v} colors",
                     s=og["abs_colors"], eps=term_eps(nc_max))
    plan.close()


@pytest.mark.parametrize("degree,stride,N", [(1, 4, 1000), (3, 16, 257), (3, 16, 1)])
def test_sh_staged_rows_single_view(R, degree, stride, N):
    """Coefficient arrays holding exactly the used rows (degree 1 in rows of 4, degree 3 in
    rows of 16) take the shared-memory staged kernels; N = 257 and 1 leave partial blocks."""
    plan = R.Plan()
    sh, m = _inputs(N, stride, 100 + N)
    cams = _cams(1)
    rgb = R.sh_to_rgb(plan, torch.from_numpy(sh).cuda(), torch.from_numpy(m).cuda(), cams, degree)
    ref, ref_cl, s, cp = _oracle_fwd(sh, m, cams, degree)
    sure = np.abs(s) > AMBIG
    np.testing.assert_allclose(rgb.cpu().numpy()[sure], ref[sure], rtol=0, atol=SH_ATOL * 2)
    g = np.random.default_rng(11).normal(size=(N, 3)).astype(np.float32)
    g[~sure] = 0.0
    d_sh, d_m = R.sh_to_rgb_backward(plan, torch.from_numpy(sh).cuda(), torch.from_numpy(m).cuda(), cams, degree,
                                     torch.from_numpy(g).cuda())
    r_sh, r_m = oracle.sh_to_rgb_backward(sh.astype(np.float64), m.astype(np.float64), cp, degree,
                                          g.reshape(1, N, 3).astype(np.float64))
    compare_grad(d_sh.cpu().numpy(), r_sh, f"staged degree {degree} N {N} sh", SH_GRAD_REL, row_eps=ROW_EPS_SH)
    compare_grad(d_m.cpu().numpy(), r_m, f"staged degree {degree} N {N} means3D", SH_GRAD_REL, row_eps=ROW_EPS_SH)
    plan.close()
