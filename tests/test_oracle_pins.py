"""Pins of the FP64 oracle against facts fixed by the paper and by mathematics.

Nothing here compares the oracle with itself.  Each test checks it against an
independent route to the same number: a library routine (scipy's normal density,
scipy's rotation, numpy's eigen-solver, numerical Jacobians), a closed form that the
paper's equations reduce to in a special case, an invariant, brute force without
tiles on tiny scenes, or FP64 central finite differences.  The paper prints no
numeric worked example, so no test can pin the image to a printed value.
"""
from fractions import Fraction
import math

import numpy as np
import pytest
from scipy.spatial.transform import Rotation
from scipy.stats import multivariate_normal

import oracle
from paper_2412_17378_gb300 import scenes

ALPHA_MIN = 1.0 / 255.0


def _unnorm_gauss(x, mean, cov):
    """exp(-1/2 d^T cov^-1 d) from scipy's normalised density (Eq. 3)."""
    return multivariate_normal(mean=mean, cov=cov).pdf(x) * 2 * np.pi * math.sqrt(np.linalg.det(cov))


def _single(mean, cov, o, color, depth=3.0, W=32, H=32, r=None, tile=16):
    conic = np.linalg.inv(cov)
    co = np.array([[conic[0, 0], conic[0, 1], conic[1, 1], o]])
    r = int(max(W, H) * 2) if r is None else r
    pl, rg = oracle.bin_tiles(np.array([mean], np.float32), np.array([r]), np.array([depth], np.float32),
                              W, H, tile, tile)
    out = oracle.render(np.array([mean]), co, np.array([color]), np.array([depth]), pl, rg, W, H,
                        tile, tile)
    return out, co


def test_single_gaussian_matches_scipy_density():
    """Eq. 3-4 with one Gaussian: C = c * min(0.99, o G') where alpha >= 1/255."""
    mean = np.array([13.3, 17.8])
    cov = np.array([[9.0, 3.5], [3.5, 5.0]])  # anisotropic, non-zero off-diagonal
    o, color = 0.8, np.array([0.2, 0.5, 0.9])
    out, _ = _single(mean, cov, o, color)
    ys, xs = np.mgrid[0:32, 0:32]
    pts = np.stack([xs.ravel(), ys.ravel()], 1).astype(np.float64)
    G = _unnorm_gauss(pts, mean, cov).reshape(32, 32)
    alpha = np.minimum(0.99, o * G)
    alpha[alpha < ALPHA_MIN] = 0.0
    for ch in range(3):
        np.testing.assert_allclose(out["color"][ch], color[ch] * alpha, rtol=1e-12, atol=1e-14)
    np.testing.assert_allclose(out["final_T"], 1.0 - alpha, rtol=1e-12, atol=1e-14)
    np.testing.assert_allclose(out["depth"], 3.0 * alpha, rtol=1e-12, atol=1e-14)
    assert out["n_contrib"].max() == 1


def test_alpha_clamp_and_threshold():
    """alpha = min(0.99, o G); pairs with alpha < 1/255 are skipped (Algorithm 5)."""
    cov = np.array([[4.0, 0.0], [0.0, 4.0]])
    out, _ = _single(np.array([10.0, 10.0]), cov, 1.0, np.array([1.0, 1.0, 1.0]))
    assert out["color"][0, 10, 10] == pytest.approx(0.99, abs=1e-15)
    assert out["final_T"][10, 10] == pytest.approx(0.01, abs=1e-15)
    # choose the opacity so that alpha at pixel (10, 14) sits just below / above 1/255
    G = _unnorm_gauss(np.array([10.0, 14.0]), np.array([10.0, 10.0]), cov)
    for o, expect in [((ALPHA_MIN * (1 - 1e-5)) / G, 0.0), ((ALPHA_MIN * (1 + 1e-5)) / G, 1.0)]:
        out, _ = _single(np.array([10.0, 10.0]), cov, o, np.array([1.0, 1.0, 1.0]))
        got = out["color"][0, 14, 10]
        if expect == 0.0:
            assert got == 0.0
        else:
            assert got == pytest.approx(ALPHA_MIN * (1 + 1e-5), rel=1e-9)


def test_two_gaussians_front_to_back():
    """Eq. 4 with two Gaussians: C = c1 a1 + c2 a2 (1 - a1), nearer first."""
    m1, m2 = np.array([12.0, 15.0]), np.array([17.0, 14.0])
    c1m, c2m = np.array([[6.0, 1.0], [1.0, 4.0]]), np.array([[5.0, -2.0], [-2.0, 7.0]])
    o1, o2 = 0.7, 0.6
    col1, col2 = np.array([1.0, 0.0, 0.3]), np.array([0.0, 1.0, 0.6])
    k1, k2 = np.linalg.inv(c1m), np.linalg.inv(c2m)
    co = np.array([[k1[0, 0], k1[0, 1], k1[1, 1], o1], [k2[0, 0], k2[0, 1], k2[1, 1], o2]])
    ys, xs = np.mgrid[0:32, 0:32]
    pts = np.stack([xs.ravel(), ys.ravel()], 1).astype(np.float64)

    def alpha(m, c, o):
        a = np.minimum(0.99, o * _unnorm_gauss(pts, m, c))
        a[a < ALPHA_MIN] = 0
        return a.reshape(32, 32)

    a1, a2 = alpha(m1, c1m, o1), alpha(m2, c2m, o2)
    for depths, (fa, fc, ba, bc) in [((2.0, 5.0), (a1, col1, a2, col2)), ((5.0, 2.0), (a2, col2, a1, col1))]:
        pl, rg = oracle.bin_tiles(np.stack([m1, m2]).astype(np.float32), np.array([64, 64]),
                                  np.array(depths, np.float32), 32, 32)
        out = oracle.render(np.stack([m1, m2]), co, np.stack([col1, col2]), np.array(depths), pl, rg, 32, 32)
        for ch in range(3):
            expect = fc[ch] * fa + bc[ch] * ba * (1 - fa)
            np.testing.assert_allclose(out["color"][ch], expect, rtol=1e-12, atol=1e-14)
        np.testing.assert_allclose(out["final_T"], (1 - fa) * (1 - ba), rtol=1e-12, atol=1e-14)


def test_early_stop_excludes_stopping_gaussian():
    """Algorithm 5: the pair whose T' would fall below 1e-4 is not accumulated and T keeps
    its previous value.  With alpha = 1/2 per layer, 0.5^13 >= 1e-4 > 0.5^14, so 13
    layers are accumulated, the 14th is visited and stops the pixel."""
    n = 20
    means = np.tile(np.array([[8.0, 8.0]]), (n, 1))
    co = np.tile(np.array([[0.5, 0.0, 0.5, 0.5]]), (n, 1))  # G = 1 at the centre, alpha = 0.5
    cols = np.tile(np.array([[0.25, 0.5, 1.0]]), (n, 1))
    depths = np.arange(1, n + 1, dtype=np.float64)
    pl, rg = oracle.bin_tiles(means.astype(np.float32), np.full(n, 40), depths.astype(np.float32), 16, 16)
    out = oracle.render(means, co, cols, depths, pl, rg, 16, 16)
    T13 = 0.5 ** 13
    assert out["final_T"][8, 8] == T13
    assert out["n_contrib"][8, 8] == 13
    assert out["n_eval"][8, 8] == 14
    np.testing.assert_allclose(out["color"][:, 8, 8], cols[0] * (1 - T13), rtol=1e-14)
    # depth-weighted sum: sum_{k=1..13} k * 0.5 * 0.5^(k-1)
    expect_d = sum(k * 0.5 ** k for k in range(1, 14))
    assert out["depth"][8, 8] == pytest.approx(expect_d, rel=1e-14)


@pytest.fixture(scope="module")
def cfg1_inputs():
    s = scenes.scene_config("cfg1")
    g, cam = s["gaussians"], s["cameras"][0]
    pp = oracle.preprocess(g["means3D"], g["log_scales"], g["quats"], g["opacities"], cam)
    m2 = pp["means2D"].astype(np.float32)
    co = pp["conic_opacity"].astype(np.float32)
    dp = pp["depth"].astype(np.float32)
    pl, rg = oracle.bin_tiles(m2, pp["radius"], dp, 256, 256)
    return dict(m2=m2, co=co, dp=dp, cl=g["colors"], r=pp["radius"], pl=pl, rg=rg, W=256, H=256)


def test_weights_and_transmittance_telescope(cfg1_inputs):
    """sum_i w_i + T_final = 1 (Eq. 4's weights telescope) and out_alpha = 1 - T_final."""
    c = cfg1_inputs
    out = oracle.render(c["m2"], c["co"], c["cl"], c["dp"], c["pl"], c["rg"], c["W"], c["H"])
    assert np.abs(out["alpha"] + out["final_T"] - 1.0).max() < 1e-12
    assert out["final_T"].min() >= 1e-4
    assert (out["n_contrib"] <= out["n_eval"]).all()


def test_permutation_of_gaussians_leaves_image(cfg1_inputs):
    """Relabelling the Gaussians (distinct depths) does not change the image."""
    c = dict(cfg1_inputs)
    dp = c["dp"].copy()
    while True:  # make the float32 depths distinct (ties would be broken by index)
        order = np.argsort(dp, kind="stable")
        dup = order[1:][dp[order[1:]] == dp[order[:-1]]]
        if dup.size == 0:
            break
        dp[dup] = np.nextafter(dp[dup], np.float32(np.inf))
    c["dp"] = dp
    c["pl"], c["rg"] = oracle.bin_tiles(c["m2"], c["r"], dp, c["W"], c["H"])
    perm = np.random.default_rng(11).permutation(len(c["dp"]))
    out0 = oracle.render(c["m2"], c["co"], c["cl"], c["dp"], c["pl"], c["rg"], c["W"], c["H"])
    pl, rg = oracle.bin_tiles(c["m2"][perm], c["r"][perm], c["dp"][perm], c["W"], c["H"])
    out1 = oracle.render(c["m2"][perm], c["co"][perm], c["cl"][perm], c["dp"][perm], pl, rg, c["W"], c["H"])
    np.testing.assert_array_equal(out0["color"], out1["color"])
    np.testing.assert_array_equal(out0["n_contrib"], out1["n_contrib"])


def test_sampled_pixels_equal_full_render(cfg1_inputs):
    c = cfg1_inputs
    out = oracle.render(c["m2"], c["co"], c["cl"], c["dp"], c["pl"], c["rg"], c["W"], c["H"])
    pix = np.random.default_rng(3).choice(c["W"] * c["H"], 500, replace=False)
    sub = oracle.render(c["m2"], c["co"], c["cl"], c["dp"], c["pl"], c["rg"], c["W"], c["H"], pixels=pix)
    np.testing.assert_array_equal(sub["color"], out["color"].reshape(3, -1)[:, pix])
    np.testing.assert_array_equal(sub["n_eval"], out["n_eval"].ravel()[pix])


def _brute_force_pixel(px, py, means, co, cols, depths, idx_order):
    """Algorithm 5 on one pixel over a globally depth-sorted list (no tiles)."""
    T, C = 1.0, np.zeros(3)
    for g in idx_order:
        cov = np.linalg.inv(np.array([[co[g, 0], co[g, 1]], [co[g, 1], co[g, 2]]]))
        G = _unnorm_gauss(np.array([px, py], float), means[g], cov)
        a = min(0.99, co[g, 3] * G)
        if a < ALPHA_MIN:
            continue
        Tn = T * (1 - a)
        if Tn < 1e-4:
            break
        C += cols[g] * a * T
        T = Tn
    return C, T


def test_brute_force_without_tiles():
    """Tiny scene whose every Gaussian covers every tile: the tiled oracle equals a
    per-pixel walk over all Gaussians sorted globally by (depth, index)."""
    rng = np.random.default_rng(5)
    n, W, H = 48, 32, 32
    means = rng.uniform(0, 32, (n, 2))
    A = rng.normal(0, 1.0, (n, 2, 2))
    covs = A @ A.transpose(0, 2, 1) * 6 + np.eye(2) * 2
    conics = np.linalg.inv(covs)
    co = np.stack([conics[:, 0, 0], conics[:, 0, 1], conics[:, 1, 1], rng.uniform(0.2, 0.95, n)], 1)
    cols = rng.uniform(0, 1, (n, 3))
    depths = rng.uniform(1, 5, n).astype(np.float32).astype(np.float64)
    depths[5] = depths[9]  # a tie, broken by index
    pl, rg = oracle.bin_tiles(means.astype(np.float32), np.full(n, 100), depths.astype(np.float32), W, H, 16, 16)
    out = oracle.render(means.astype(np.float32).astype(np.float64), co, cols, depths, pl, rg, W, H, 16, 16)
    means64 = means.astype(np.float32).astype(np.float64)
    order = np.lexsort((np.arange(n), depths))
    for py in range(0, H, 3):
        for px in range(0, W, 3):
            C, T = _brute_force_pixel(px, py, means64, co, cols, depths, order)
            np.testing.assert_allclose(out["color"][:, py, px], C, rtol=1e-10, atol=1e-12)
            assert out["final_T"][py, px] == pytest.approx(T, rel=1e-10)


def test_binning_matches_per_tile_lexsort():
    """Each tile's list = the Gaussians whose rectangle covers it, ordered by
    (float32 depth, index) -- checked against numpy's lexsort per tile."""
    rng = np.random.default_rng(8)
    n, W, H, tw, th = 400, 100, 70, 16, 8
    m2 = rng.uniform(-20, 120, (n, 2)).astype(np.float32)
    r = rng.integers(0, 30, n).astype(np.int32)
    dp = rng.choice(np.linspace(1, 2, 50), n).astype(np.float32)  # many ties
    pl, rg = oracle.bin_tiles(m2, r, dp, W, H, tw, th)
    tx, ty = (W + tw - 1) // tw, (H + th - 1) // th
    rects = np.array([oracle.tile_rect(float(m2[i, 0]), float(m2[i, 1]), int(r[i]), W, H, tw, th)
                      for i in range(n)])
    for t in range(tx * ty):
        x, y = t % tx, t // tx
        inc = np.nonzero((r > 0) & (rects[:, 0] <= x) & (x < rects[:, 1]) & (rects[:, 2] <= y) & (y < rects[:, 3]))[0]
        expect = inc[np.lexsort((inc, dp[inc]))]
        np.testing.assert_array_equal(pl[rg[t, 0]:rg[t, 1]], expect)


def test_subset_binning_matches_per_tile_lexsort():
    """bin_tiles_subset: the lists of the chosen tiles only, each the Gaussians whose
    rectangle covers the tile ordered by (float32 depth, index) -- numpy's lexsort per
    tile -- and empty spans for every other tile."""
    rng = np.random.default_rng(18)
    n, W, H, tw, th = 400, 100, 70, 16, 8
    m2 = rng.uniform(-20, 120, (n, 2)).astype(np.float32)
    r = rng.integers(0, 30, n).astype(np.int32)
    dp = rng.choice(np.linspace(1, 2, 50), n).astype(np.float32)  # many ties
    tx, ty = (W + tw - 1) // tw, (H + th - 1) // th
    sel = rng.permutation(tx * ty)[:13]
    pl, rg = oracle.bin_tiles_subset(m2, r, dp, W, H, sel, tw, th)
    order = oracle.depth_order(r, dp)
    vis = np.nonzero(r > 0)[0]
    np.testing.assert_array_equal(order, vis[np.lexsort((vis, dp[vis]))])
    pl2, rg2 = oracle.bin_tiles_subset(m2, r, dp, W, H, sel, tw, th, order=order)
    np.testing.assert_array_equal(pl2, pl)
    np.testing.assert_array_equal(rg2, rg)
    rects = np.array([oracle.tile_rect(float(m2[i, 0]), float(m2[i, 1]), int(r[i]), W, H, tw, th)
                      for i in range(n)])
    total = 0
    for t in range(tx * ty):
        if t not in set(sel.tolist()):
            assert rg[t, 0] == rg[t, 1] == 0
            continue
        x, y = t % tx, t // tx
        inc = np.nonzero((r > 0) & (rects[:, 0] <= x) & (x < rects[:, 1]) & (rects[:, 2] <= y) & (y < rects[:, 3]))[0]
        expect = inc[np.lexsort((inc, dp[inc]))]
        np.testing.assert_array_equal(pl[rg[t, 0]:rg[t, 1]], expect)
        total += expect.size
    assert pl.size == total > 0


def test_tile_rect_is_exact_floor():
    """The rectangle bounds are floor((u - r)/tw) and floor((u + r + tw - 1)/tw),
    clamped: compared with exact rational arithmetic away from rounding ties."""
    rng = np.random.default_rng(9)
    W, H, tw, th = 1920, 1080, 16, 8
    for _ in range(2000):
        u, v = np.float32(rng.uniform(-50, 1970)), np.float32(rng.uniform(-50, 1130))
        r = int(rng.integers(1, 200))
        got = oracle.tile_rect(float(u), float(v), r, W, H, tw, th)
        vals = [(Fraction(float(u)) - r) / tw, (Fraction(float(u)) + r + tw - 1) / tw,
                (Fraction(float(v)) - r) / th, (Fraction(float(v)) + r + th - 1) / th]
        if any(abs(q - round(q)) < Fraction(1, 10000) for q in vals):
            continue
        lim = [(W + tw - 1) // tw] * 2 + [(H + th - 1) // th] * 2
        expect = [min(max(math.floor(q), 0), L) for q, L in zip(vals, lim)]
        assert list(got) == expect


# ----------------------------------------------------------------------------- projection


def _numeric_jacobian(f, p, h=1e-6):
    J = np.zeros((2, 3))
    for k in range(3):
        e = np.zeros(3)
        e[k] = h
        J[:, k] = (f(p + e) - f(p - e)) / (2 * h)
    return J


def test_projection_against_scipy_rotation_and_numeric_jacobian():
    """Eq. 2: Sigma' = J W Sigma W^T J^T (+ low-pass), with Sigma from scipy's rotation
    (quaternion in scalar-last order) and J from central differences of the pinhole map."""
    rng = np.random.default_rng(12)
    n = 40
    W_, H_ = 640, 480
    V = np.eye(4)
    V[:3, :3] = Rotation.from_euler("xyz", [0.1, -0.2, 0.05]).as_matrix()
    V[:3, 3] = [0.1, -0.2, 0.3]
    cam = scenes.camera(W_, H_, viewmat=V, fx=500.0, fy=520.0)
    # points in front of the camera and inside the tangent clamp
    pc = np.stack([rng.uniform(-0.5, 0.5, n), rng.uniform(-0.4, 0.4, n), rng.uniform(2, 5, n)], 1)
    world = (pc - V[:3, 3]) @ V[:3, :3]  # invert the rigid transform
    ls = rng.normal(-3.0, 0.6, (n, 3))
    q = rng.normal(size=(n, 4))
    op = rng.uniform(0.1, 0.9, n)
    pp = oracle.preprocess(world.astype(np.float32), ls.astype(np.float32), q.astype(np.float32),
                           op.astype(np.float32), cam)
    world32 = world.astype(np.float32).astype(np.float64)
    for i in range(n):
        qq = q.astype(np.float32).astype(np.float64)[i]
        R = Rotation.from_quat([qq[1], qq[2], qq[3], qq[0]]).as_matrix()
        S = np.diag(np.exp(ls.astype(np.float32).astype(np.float64)[i]))
        Sig = R @ S @ S @ R.T
        pcam = V[:3, :3] @ world32[i] + V[:3, 3]
        proj = lambda p: np.array([500.0 * p[0] / p[2] + cam["cx"], 520.0 * p[1] / p[2] + cam["cy"]])
        J = _numeric_jacobian(proj, pcam)
        cov2 = J @ V[:3, :3] @ Sig @ V[:3, :3].T @ J.T + 0.3 * np.eye(2)
        conic = np.linalg.inv(cov2)
        got = pp["conic_opacity"][i]
        np.testing.assert_allclose(got[:3], [conic[0, 0], conic[0, 1], conic[1, 1]], rtol=1e-6, atol=1e-12)
        assert got[3] == np.float32(op[i])
        np.testing.assert_allclose(pp["means2D"][i], proj(pcam), rtol=1e-12)
        assert pp["depth"][i] == pytest.approx(pcam[2], rel=1e-12)
        lam = np.linalg.eigvalsh(cov2).max()
        mid, det = 0.5 * np.trace(cov2), np.linalg.det(cov2)
        if mid * mid - det > 0.1:
            assert pp["radius_raw"][i] == pytest.approx(3 * math.sqrt(lam), rel=1e-9)
        if abs(pp["radius_raw"][i] - round(pp["radius_raw"][i])) > 1e-6 and pp["radius"][i] > 0:
            assert pp["radius"][i] == math.ceil(3 * math.sqrt(lam)) or mid * mid - det <= 0.1


def test_isotropic_gaussian_on_axis():
    """An isotropic Gaussian of scale s on the optical axis at depth z projects to a
    circle of pixel std fx s / z: conic = I / ((fx s/z)^2 + lowpass)."""
    s, z, fx = 0.02, 4.0, 800.0
    cam = scenes.camera(400, 300, fx=fx, fy=fx)
    for lowpass in (0.0, 0.3):
        cam["lowpass"] = lowpass
        pp = oracle.preprocess(np.array([[0, 0, z]], np.float32), np.full((1, 3), math.log(s), np.float32),
                               np.array([[1, 0, 0, 0]], np.float32), np.array([0.5], np.float32), cam)
        var = (fx * np.float64(np.float32(s)) / z) ** 2
        var = (fx * math.exp(np.float64(np.float32(math.log(s)))) / z) ** 2 + lowpass
        np.testing.assert_allclose(pp["conic_opacity"][0, :3], [1 / var, 0.0, 1 / var], rtol=1e-9, atol=1e-15)
        np.testing.assert_allclose(pp["means2D"][0], [cam["cx"], cam["cy"]], atol=1e-12)
        # isotropic: discriminant 0 is floored at 0.1
        assert pp["radius_raw"][0] == pytest.approx(3 * math.sqrt(var + math.sqrt(0.1)), rel=1e-12)


def test_near_cull_and_quaternion_scale():
    cam = scenes.camera(64, 64)
    m = np.array([[0, 0, 0.15], [0, 0, 0.25], [0.01, 0.02, 3.0]], np.float32)
    ls = np.full((3, 3), -3.0, np.float32)
    q = np.array([[1, 0, 0, 0], [1, 0, 0, 0], [0.3, -0.2, 0.5, 0.4]], np.float32)
    pp1 = oracle.preprocess(m, ls, q, np.full(3, 0.5, np.float32), cam)
    pp2 = oracle.preprocess(m, ls, q * 4, np.full(3, 0.5, np.float32), cam)
    assert pp1["radius"][0] == 0 and pp1["tiles_touched"][0] == 0
    assert pp1["radius"][1] > 0
    np.testing.assert_allclose(pp1["conic_opacity"], pp2["conic_opacity"], rtol=1e-12)


def test_tangent_clamp():
    """Off-axis points beyond 1.3 tan(fov/2) use the Jacobian at the clamped point."""
    W_, fx = 100, 100.0
    cam = scenes.camera(W_, W_, fx=fx, fy=fx, lowpass=0.0)
    z = 2.0
    x = 3.0 * z * (W_ / (2 * fx))  # 3 half-widths off axis, beyond the 1.3 clamp
    pp = oracle.preprocess(np.array([[x, 0, z]], np.float32), np.full((1, 3), math.log(0.05), np.float32),
                           np.array([[1, 0, 0, 0]], np.float32), np.array([0.5], np.float32), cam)
    xc = 1.3 * (W_ / (2 * fx)) * z
    proj = lambda p: np.array([fx * p[0] / p[2], fx * p[1] / p[2]])
    J = _numeric_jacobian(proj, np.array([xc, 0.0, z]))
    s2 = math.exp(np.float64(np.float32(math.log(0.05)))) ** 2
    cov2 = J @ (np.eye(3) * s2) @ J.T
    conic = np.linalg.inv(cov2)
    np.testing.assert_allclose(pp["conic_opacity"][0, :3], [conic[0, 0], conic[0, 1], conic[1, 1]], rtol=1e-6)


# ----------------------------------------------------------------------------- gradient


@pytest.fixture(scope="module")
def fd_scene():
    s = scenes.scene_config("fdcrop")
    g, cam = s["gaussians"], s["cameras"][0]
    pp = oracle.preprocess(g["means3D"], g["log_scales"], g["quats"], g["opacities"], cam)
    W = H = 64
    m2, co, dp = pp["means2D"], pp["conic_opacity"], pp["depth"]
    pl, rg = oracle.bin_tiles(m2.astype(np.float32), pp["radius"], dp.astype(np.float32), W, H)
    rng = np.random.default_rng(21)
    gC, gD, gA = rng.normal(size=(3, H, W)), rng.normal(size=(H, W)) * 0.1, rng.normal(size=(H, W))
    return dict(m2=m2, co=co, cl=g["colors"].astype(np.float64), dp=dp, pl=pl, rg=rg, W=W, H=H,
                gC=gC, gD=gD, gA=gA, bg=np.array([0.2, 0.4, 0.1]))


def _loss(s, m2, co, cl, dp):
    out = oracle.render(m2, co, cl, dp, s["pl"], s["rg"], s["W"], s["H"], bg=s["bg"])
    L = (s["gC"] * out["color"]).sum() + (s["gD"] * out["depth"]).sum() + (s["gA"] * out["alpha"]).sum()
    return L, out


def test_backward_matches_central_differences(fd_scene):
    """FP64 central differences of L = <gC, C> + <gD, D> + <gA, A> against the analytic
    gradient, with a non-black background; parameters whose perturbation changes a
    discrete decision (skip / stop / clamp) are not compared."""
    s = fd_scene
    grad = oracle.render_backward(s["m2"], s["co"], s["cl"], s["dp"], s["pl"], s["rg"], s["W"], s["H"],
                                  s["gC"], s["gD"], s["gA"], bg=s["bg"])
    assert np.abs(grad["opacity"]).max() > 0
    _, base = _loss(s, s["m2"], s["co"], s["cl"], s["dp"])
    contrib = np.unique(s["pl"])
    rng = np.random.default_rng(4)
    checks = []
    for g in rng.choice(contrib, 40, replace=False):
        for field, k, key in [("m2", 0, ("means2D", 0)), ("m2", 1, ("means2D", 1)), ("co", 0, ("conic", 0)),
                              ("co", 1, ("conic", 1)), ("co", 2, ("conic", 2)), ("co", 3, ("opacity", None)),
                              ("cl", 1, ("colors", 1)), ("dp", None, ("depths", None))]:
            checks.append((g, field, k, key))
    compared = 0
    for g, field, k, (gname, gk) in checks:
        arrs = {f: s[f].copy() for f in ("m2", "co", "cl", "dp")}
        x0 = arrs[field][g] if k is None else arrs[field][g, k]
        # step from the parameter's natural scale (the conic's diagonal for its three
        # entries), so that FP64 round-off in L stays far below the tolerance
        scale = {"m2": 1.0, "co": 0.5 * (arrs["co"][g, 0] + arrs["co"][g, 2]) if k != 3 else 1.0,
                 "cl": 1.0, "dp": abs(x0)}[field]
        h = 1e-5 * scale
        vals, outs = [], []
        for sign in (1, -1):
            a = {f: v.copy() for f, v in arrs.items()}
            if k is None:
                a[field][g] = x0 + sign * h
            else:
                a[field][g, k] = x0 + sign * h
            L, out = _loss(s, a["m2"], a["co"], a["cl"], a["dp"])
            vals.append(L)
            outs.append(out)
        if not (np.array_equal(outs[0]["n_contrib"], outs[1]["n_contrib"])
                and np.array_equal(outs[0]["n_eval"], outs[1]["n_eval"])
                and np.array_equal(outs[0]["n_contrib"], base["n_contrib"])
                and np.array_equal(outs[0]["n_acc"], outs[1]["n_acc"])
                and np.array_equal(outs[0]["flags"], outs[1]["flags"])):
            continue
        fd = (vals[0] - vals[1]) / (2 * h)
        an = grad[gname][g] if gk is None else grad[gname][g, gk]
        assert an == pytest.approx(fd, rel=2e-5, abs=1e-7 * (1 + abs(fd))), (g, field, k)
        compared += 1
    assert compared > 250


def test_backward_tile_subset_and_mask(fd_scene):
    """Restricting to a tile subset and a Gaussian mask gives the same per-Gaussian
    gradients as the full pass for Gaussians whose rectangles lie inside the subset."""
    s = fd_scene
    full = oracle.render_backward(s["m2"], s["co"], s["cl"], s["dp"], s["pl"], s["rg"], s["W"], s["H"], s["gC"])
    N = s["m2"].shape[0]
    mask = np.zeros(N, np.uint8)
    mask[::7] = 1
    sub = oracle.render_backward(s["m2"], s["co"], s["cl"], s["dp"], s["pl"], s["rg"], s["W"], s["H"], s["gC"],
                                 tiles=np.arange(16), mask=mask)
    np.testing.assert_allclose(sub["opacity"][mask == 1], full["opacity"][mask == 1], rtol=1e-12, atol=1e-15)
    assert (sub["opacity"][mask == 0] == 0).all()


def test_backward_term_magnitudes(fd_scene):
    """The per-element sums of |term| that the gradient tests use as tolerance scales:
    never below |gradient| (triangle inequality); equal to it when every term has one sign
    (colour terms alpha T dL/dC under a positive dL/dC); equal to the gradient of
    L = <|gC|, C> for the colour terms (their weights are the same); and zero exactly
    where the gradient receives no term."""
    s = fd_scene
    g = oracle.render_backward(s["m2"], s["co"], s["cl"], s["dp"], s["pl"], s["rg"], s["W"], s["H"], s["gC"],
                               s["gD"], s["gA"], bg=s["bg"], abs_terms=True)
    for k in ("means2D", "conic", "opacity", "colors", "depths"):
        assert (g["abs_" + k] >= np.abs(g[k]) * (1 - 1e-12) - 1e-300).all(), k
    pos = oracle.render_backward(s["m2"], s["co"], s["cl"], s["dp"], s["pl"], s["rg"], s["W"], s["H"],
                                 np.abs(s["gC"]), bg=s["bg"], abs_terms=True)
    np.testing.assert_allclose(pos["abs_colors"], pos["colors"], rtol=1e-12, atol=0)
    np.testing.assert_allclose(g["abs_colors"], pos["colors"], rtol=1e-12, atol=0)
    touched = np.zeros(s["m2"].shape[0], bool)
    touched[np.unique(s["pl"])] = True
    assert (g["abs_opacity"][~touched] == 0).all() and (g["opacity"][~touched] == 0).all()
    assert (g["abs_means2D"] > np.abs(g["means2D"]) * 1.001).any()  # cancellation does occur


def test_oracle_regression_snapshot():
    """The oracle still reproduces tests/golden/cfg1_oracle_snapshot.txt."""
    import importlib.util
    import os
    here = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
    spec = importlib.util.spec_from_file_location("make_golden", os.path.join(here, "make_golden.py"))
    mg = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mg)
    stored = {}
    for line in open(os.path.join(here, "cfg1_oracle_snapshot.txt")):
        if line.startswith("#"):
            continue
        k, v = line.split()
        stored[k] = float(v)
    for k, v in mg.snapshot():
        assert v == pytest.approx(stored[k], rel=1e-12, abs=1e-15), k


# --------------------------------------------------------------------- projection backward

def _projection_fd_scene():
    """40 anisotropic Gaussians seen by a rotated, translated camera: quaternions of
    non-unit norm, a third of the centres beyond the tangent clamp (|x/z| well above
    1.3 tan(fov/2)), none within 5 % of the clamp edge."""
    rng = np.random.default_rng(11)
    cam = scenes.look_at_camera(96, 64, eye=(0.3, -0.2, -1.0), target=(0.1, 0.05, 3.0))
    cam["lowpass"] = 0.3
    n = 40
    V = cam["viewmat"]
    lim_x, lim_y = 1.3 * cam["W"] / (2 * cam["fx"]), 1.3 * cam["H"] / (2 * cam["fy"])
    pts = []
    while len(pts) < n:
        z = rng.uniform(1.5, 5.0)
        tx = rng.uniform(-2.2, 2.2) * lim_x * z if len(pts) % 3 == 0 else rng.uniform(-0.9, 0.9) * lim_x * z
        ty = rng.uniform(-0.9, 0.9) * lim_y * z
        if abs(abs(tx / z) - lim_x) < 0.05 * lim_x:
            continue
        t = np.array([tx, ty, z])
        pts.append(np.linalg.solve(V[:3, :3], t - V[:3, 3]))  # world point with camera coords t
    m3 = np.array(pts)
    ls = rng.normal(-2.0, 0.6, (n, 3))
    q = rng.normal(size=(n, 4)) * rng.uniform(0.5, 2.0, (n, 1))
    return m3, ls, q, cam


def test_projection_backward_matches_central_differences():
    m3, ls, q, cam = _projection_fd_scene()
    n = m3.shape[0]
    rng = np.random.default_rng(12)
    gm, gc, gd = rng.normal(size=(n, 2)), rng.normal(size=(n, 3)) * 100.0, rng.normal(size=n)
    base = oracle.project64(m3, ls, q, cam)
    assert base["valid"].all()
    got = oracle.preprocess_backward(m3, ls, q, cam, gm, gc, gd)

    def loss(m3_, ls_, q_):
        o = oracle.project64(m3_, ls_, q_, cam)
        return np.sum(gm * o["means2D"], axis=1) + np.sum(gc * o["conic"], axis=1) + gd * o["depth"]

    for name, arr in (("means3D", m3), ("log_scales", ls), ("quats", q)):
        fd = np.zeros_like(arr)
        for k in range(arr.shape[1]):
            h = 1e-6 * np.maximum(1.0, np.abs(arr[:, k]))
            a_p, a_m = arr.copy(), arr.copy()
            a_p[:, k] += h
            a_m[:, k] -= h
            args_p = [m3, ls, q]
            args_m = [m3, ls, q]
            idx = ("means3D", "log_scales", "quats").index(name)
            args_p[idx], args_m[idx] = a_p, a_m
            fd[:, k] = (loss(*args_p) - loss(*args_m)) / (2 * h)  # per-Gaussian losses are independent
        scale = np.abs(fd).max(axis=1, keepdims=True) + 1e-12
        err = np.abs(got[name] - fd) / scale
        assert err.max() < 1e-5, (name, float(err.max()))


def test_projection_backward_zero_for_culled_and_radius_zero():
    m3, ls, q, cam = _projection_fd_scene()
    n = m3.shape[0]
    m3 = m3.copy()
    # Gaussian 0 behind the near plane
    V = cam["viewmat"]
    m3[0] = np.linalg.solve(V[:3, :3], np.array([0.0, 0.0, 0.1]) - V[:3, 3])
    radius = np.ones(n, np.int32)
    radius[1] = 0  # off-screen: passes no gradient
    g = oracle.preprocess_backward(m3, ls, q, cam, np.ones((n, 2)), np.ones((n, 3)), np.ones(n), radius=radius)
    for k in ("means3D", "log_scales", "quats"):
        assert not g[k][:2].any(), k
        assert np.abs(g[k][2:]).sum() > 0, k


def test_projection_backward_quaternion_gradient_is_tangent():
    """The projection depends on q only through q / |q|: the gradient is orthogonal to q
    and scales as 1 / |q|."""
    m3, ls, q, cam = _projection_fd_scene()
    n = m3.shape[0]
    rng = np.random.default_rng(13)
    gm, gc = rng.normal(size=(n, 2)), rng.normal(size=(n, 3))
    g1 = oracle.preprocess_backward(m3, ls, q, cam, gm, gc)["quats"]
    g2 = oracle.preprocess_backward(m3, ls, 2.0 * q, cam, gm, gc)["quats"]
    np.testing.assert_allclose(np.sum(g1 * q, axis=1), 0.0, atol=1e-9 * np.abs(g1).max())
    np.testing.assert_allclose(g2, 0.5 * g1, rtol=1e-9, atol=1e-15)


# ---- view-dependent colour: spherical harmonics of degree <= 3 (Sec. 2.1) ----------------

def _sh_values(dirs, degree=3):
    """Y_k(d) for unit directions dirs [M,3], read back through the oracle's colour with one
    small coefficient at a time (0.1 Y + 1/2 stays positive, so nothing is clamped)."""
    K = (degree + 1) ** 2
    M = dirs.shape[0]
    out = np.zeros((M, K))
    for k in range(K):
        sh = np.zeros((M, K, 3))
        sh[:, k, 0] = 0.1
        rgb, clamped = oracle.sh_to_rgb(sh, dirs, np.zeros(3), degree)
        assert not clamped.any()
        out[:, k] = (rgb[0, :, 0] - 0.5) / 0.1
    return out


def _real_sh_scipy(l, m, dirs):
    """Real orthonormal SH with the Condon-Shortley phase from scipy's complex ones:
    sqrt(2) Re Y_l^m (m > 0), sqrt(2) Im Y_l^|m| (m < 0), Y_l^0 (m = 0)."""
    import scipy.special as sp
    theta = np.arccos(np.clip(dirs[:, 2], -1, 1))
    phi = np.arctan2(dirs[:, 1], dirs[:, 0])
    if hasattr(sp, "sph_harm_y"):
        Y = sp.sph_harm_y(l, abs(m), theta, phi)
    else:
        Y = sp.sph_harm(abs(m), l, phi, theta)
    if m > 0:
        return math.sqrt(2) * Y.real
    if m < 0:
        return math.sqrt(2) * Y.imag
    return Y.real


def _random_dirs(n, seed):
    d = np.random.default_rng(seed).normal(size=(n, 3))
    return d / np.linalg.norm(d, axis=1, keepdims=True)


def test_sh_basis_equals_scipy_real_harmonics():
    dirs = _random_dirs(200, 11)
    Y = _sh_values(dirs)
    k = 0
    for l in range(4):
        for m in range(-l, l + 1):
            np.testing.assert_allclose(Y[:, k], _real_sh_scipy(l, m, dirs), rtol=0, atol=1e-12, err_msg=f"l={l} m={m}")
            k += 1


def test_sh_basis_orthonormal_on_the_sphere():
    """Gauss-Legendre in cos(theta) x uniform phi integrates products of two degree-3
    harmonics exactly: the Gram matrix must be the identity."""
    ct, wt = np.polynomial.legendre.leggauss(8)
    nphi = 16
    phi = 2 * np.pi * np.arange(nphi) / nphi
    st = np.sqrt(1 - ct ** 2)
    dirs = np.stack([np.outer(st, np.cos(phi)).ravel(), np.outer(st, np.sin(phi)).ravel(),
                     np.repeat(ct, nphi)], axis=1)
    w = np.repeat(wt, nphi) * (2 * np.pi / nphi)
    Y = _sh_values(dirs)
    gram = (Y * w[:, None]).T @ Y
    np.testing.assert_allclose(gram, np.eye(16), atol=1e-12)


def test_sh_addition_theorem():
    """sum_m Y_lm(d)^2 = (2l + 1) / (4 pi) for every direction and degree."""
    Y = _sh_values(_random_dirs(64, 12))
    k = 0
    for l in range(4):
        s = (Y[:, k:k + 2 * l + 1] ** 2).sum(axis=1)
        np.testing.assert_allclose(s, (2 * l + 1) / (4 * np.pi), rtol=1e-13)
        k += 2 * l + 1


def test_sh_degree0_closed_form_and_clamp():
    rng = np.random.default_rng(13)
    sh = rng.normal(size=(50, 1, 3))
    m = rng.normal(size=(50, 3)) * 3
    rgb, clamped = oracle.sh_to_rgb(sh, m, np.array([0.3, -0.1, 0.2]), 0)
    s = sh[:, 0, :] / (2 * math.sqrt(math.pi)) + 0.5
    np.testing.assert_allclose(rgb[0], np.maximum(s, 0), rtol=0, atol=1e-15)
    np.testing.assert_array_equal(clamped[0], (s < 0).astype(np.uint8))
    # a clamped channel passes no gradient (to its coefficients or, through it, to the mean)
    g = np.ones((1, 50, 3))
    d_sh, d_m = oracle.sh_to_rgb_backward(sh, m, np.array([0.3, -0.1, 0.2]), 0, g)
    np.testing.assert_allclose(d_sh[:, 0, :], np.where(s < 0, 0.0, 1 / (2 * math.sqrt(math.pi))), atol=1e-15)
    np.testing.assert_allclose(d_m, 0.0, atol=1e-15)  # degree 0 does not depend on the direction
    assert clamped.any() and not clamped.all()


@pytest.mark.parametrize("degree", [1, 2, 3])
def test_sh_backward_matches_central_differences(degree):
    rng = np.random.default_rng(20 + degree)
    N, K = 6, 16
    sh = rng.normal(size=(N, K, 3)) * 0.3
    m = rng.normal(size=(N, 3)) + np.array([0.0, 0.0, 3.0])
    cp = np.array([[0.0, 0.0, 0.0], [0.4, -0.3, 0.2]])
    g = rng.normal(size=(2, N, 3))
    rgb, clamped = oracle.sh_to_rgb(sh, m, cp, degree)
    assert not clamped.any()
    d_sh, d_m = oracle.sh_to_rgb_backward(sh, m, cp, degree, g)
    L = lambda s_, m_: (oracle.sh_to_rgb(s_, m_, cp, degree)[0] * g).sum()
    h = 1e-6
    fd_m = np.zeros_like(m)
    for i in range(N):
        for a in range(3):
            mp, mm = m.copy(), m.copy()
            mp[i, a] += h
            mm[i, a] -= h
            fd_m[i, a] = (L(sh, mp) - L(sh, mm)) / (2 * h)
    np.testing.assert_allclose(d_m, fd_m, rtol=1e-6, atol=1e-8)
    nk = (degree + 1) ** 2
    fd_s = np.zeros_like(sh)
    for i in range(N):
        for k in range(K):
            for c in range(3):
                sp_, sm_ = sh.copy(), sh.copy()
                sp_[i, k, c] += h
                sm_[i, k, c] -= h
                fd_s[i, k, c] = (L(sp_, m) - L(sm_, m)) / (2 * h)
    np.testing.assert_allclose(d_sh, fd_s, rtol=1e-6, atol=1e-8)
    assert np.all(d_sh[:, nk:, :] == 0)  # rows past (degree + 1)^2 are not read
