"""Parity at the benchmark's full size (1920x1080, 1M Gaussians, 80% clustered) in the
benchmark's launch configurations, on outputs the oracle computes one by one: binning
compared in full, sampled pixels (random ones and every pixel of the heaviest tiles) and
the gradients, element by element, of sampled Gaussians -- those of the heaviest and
lightest tiles and random ones (the oracle visits the tiles their rectangles cover)."""
import numpy as np
import pytest

import oracle
from helpers import IMG_FRAC_MIN, IMG_FRAC_TOL, IMG_MAX_ABS, compare_grads, oracle_render_inputs, scene, to_gpu

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def big():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    inp = oracle_render_inputs(scene("cfg2"))
    return inp


def test_fullsize_binning_bit_exact(big):
    from paper_2412_17378_gb300 import raster as R
    plan = R.Plan()
    g = to_gpu(big)
    pl, rg, K = R.bin_and_sort(plan, g["means2D"], g["radii"], g["depths"], big["W"], big["H"])
    torch.cuda.synchronize()
    assert K == big["point_list"].size
    np.testing.assert_array_equal(rg.cpu().numpy().astype(np.uint32), big["ranges"])
    np.testing.assert_array_equal(pl[:K].cpu().numpy().astype(np.uint32), big["point_list"])
    plan.close()


# the benchmark's candidate launch configurations: pixel-wise items only (its tuned choice
# on this scene) and a mixed list with Gaussian-wise items for the heavy tiles
@pytest.mark.parametrize("knobs", [dict(mode="auto", heavy_threshold=1 << 30, gw_pixels=4),
                                   dict(mode="auto", heavy_threshold=4096, gw_pixels=2)])
def test_fullsize_sampled_forward_and_backward(big, knobs):
    from paper_2412_17378_gb300 import raster as R
    W, H = big["W"], big["H"]
    plan = R.Plan(heavy_threshold=knobs["heavy_threshold"], gw_pixels=knobs["gw_pixels"])
    g = to_gpu(big)
    out = R.render_forward(plan, g["means2D"], g["conic_opacity"], g["colors"], g["depths"], g["point_list"], g["K"],
                           g["ranges"], W, H, (16, 16), (0.0, 0.0, 0.0), knobs["mode"], n_eval=True)
    torch.cuda.synchronize()
    plan.check()
    # sampled pixels: 4000 random + every pixel of the 3 heaviest tiles
    rng = np.random.default_rng(0)
    lens = big["ranges"][:, 1].astype(np.int64) - big["ranges"][:, 0]
    tx = (W + 15) // 16
    heavy = np.argsort(-lens)[:3]
    pix = [rng.choice(W * H, 4000, replace=False)]
    for t in heavy:
        ys, xs = np.mgrid[(t // tx) * 16:(t // tx) * 16 + 16, (t % tx) * 16:(t % tx) * 16 + 16]
        pix.append((ys * W + xs).ravel())
    pix = np.unique(np.concatenate(pix))
    ref = oracle.render(big["means2D"], big["conic_opacity"], big["colors"], big["depths"], big["point_list"],
                        big["ranges"], W, H, pixels=pix)
    got = out["color"].reshape(3, -1)[:, torch.from_numpy(pix).cuda()].cpu().numpy()
    diff = np.abs(got - ref["color"]).max(axis=0)
    un = ref["flags"] == 0
    assert diff[un].max() <= IMG_MAX_ABS, diff[un].max()
    assert (diff <= IMG_FRAC_TOL).mean() >= IMG_FRAC_MIN
    nc = out["n_contrib"].reshape(-1)[torch.from_numpy(pix).cuda()].cpu().numpy()
    np.testing.assert_array_equal(nc[un], ref["n_contrib"][un])

    # gradients, element-wise, of a sample of Gaussians: every Gaussian that contributes to
    # the 3 heaviest tiles (the list entries before the tiles' largest n_contrib), every
    # Gaussian of the 3 lightest non-empty tiles, and 300 random visible ones
    sample = [rng.choice(np.nonzero(big["radii"] > 0)[0], 300, replace=False)]
    nc_ref = ref["n_contrib"]
    for t in heavy:
        ys, xs = np.mgrid[(t // tx) * 16:(t // tx) * 16 + 16, (t % tx) * 16:(t % tx) * 16 + 16]
        sel = np.isin(pix, (ys * W + xs).ravel())
        top = int(nc_ref[sel].max())
        sample.append(big["point_list"][big["ranges"][t, 0]:big["ranges"][t, 0] + top])
    light = [t for t in np.argsort(lens, kind="stable") if lens[t] > 0][:3]
    for t in light:
        sample.append(big["point_list"][big["ranges"][t, 0]:big["ranges"][t, 1]])
    sample = np.unique(np.concatenate(sample).astype(np.int64))
    assert sample.size > 300
    mask = np.zeros(big["radii"].size, np.uint8)
    mask[sample] = 1
    tiles = set()
    for i in sample:
        x0, x1, y0, y1 = oracle.tile_rect(float(big["means2D"][i, 0]), float(big["means2D"][i, 1]),
                                          int(big["radii"][i]), W, H, 16, 16)
        for y in range(y0, y1):
            for x in range(x0, x1):
                tiles.add(y * tx + x)
    tiles = np.array(sorted(tiles), np.int64)
    # upstream gradient: random, zero on the decision-ambiguous pixels of these tiles
    gC = rng.normal(size=(3, H, W)).astype(np.float32)
    tp = []
    for t in tiles:
        ys, xs = np.mgrid[(t // tx) * 16:min((t // tx) * 16 + 16, H), (t % tx) * 16:min((t % tx) * 16 + 16, W)]
        tp.append((ys * W + xs).ravel())
    tp = np.concatenate(tp)
    fwd_tp = oracle.render(big["means2D"], big["conic_opacity"], big["colors"], big["depths"], big["point_list"],
                           big["ranges"], W, H, pixels=tp)
    fl = fwd_tp["flags"]
    gC.reshape(3, -1)[:, tp[fl != 0]] = 0
    gr = R.render_backward(plan, g["means2D"], g["conic_opacity"], g["colors"], g["depths"], g["point_list"], g["K"],
                           g["ranges"], W, H, out["final_T"], out["n_contrib"], torch.from_numpy(gC).cuda(), None, None,
                           (16, 16), (0.0, 0.0, 0.0), knobs["mode"])
    torch.cuda.synchronize()
    plan.check()
    og = oracle.render_backward(big["means2D"], big["conic_opacity"], big["colors"], big["depths"], big["point_list"],
                                big["ranges"], W, H, gC, tiles=tiles, mask=mask, abs_terms=True)
    got = {k: gr[k].cpu().numpy() for k in ("means2D", "conic", "opacity", "colors")}
    nc_max = int(fwd_tp["n_contrib"].max())  # the deepest walk of the visited tiles
    compare_grads(got, og, what=f"full size {knobs}", idx=sample, n_contrib_max=nc_max)
    plan.close()
