"""List truncation in binning (bgs_bin_and_sort with conic_opacity): each tile's list is cut
where every pixel of the tile is certified to have stopped (Algorithm 5).  Checked against
the FP64 oracle's complete lists: every truncated list is a prefix of the oracle's list, at
least as long as the oracle's largest n_eval over the tile's pixels, and rendering from the
truncated lists gives the oracle's images, integer outputs and gradients."""
import numpy as np
import pytest

import oracle
from helpers import compare_grads, compare_images, oracle_render_inputs, scene, to_gpu
from paper_2412_17378_gb300 import scenes

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def R():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2412_17378_gb300 import raster
    return raster


@pytest.fixture(scope="module")
def dense():
    """A dense, opaque single view: config 2's clustered distribution at 200k Gaussians, with
    scales and opacities raised so that cluster tiles saturate early."""
    s = scene("cfg2", 0.2)
    g = s["gaussians"]
    g["log_scales"] = (g["log_scales"] + 1.0).astype(np.float32)
    g["opacities"] = np.clip(g["opacities"] * 1.3, 0.0, 0.999).astype(np.float32)
    s["cameras"][0].update(W=960, H=540, cx=479.5, cy=269.5, fx=960.0, fy=960.0)
    inp = oracle_render_inputs(s)
    ref = oracle.render(inp["means2D"], inp["conic_opacity"], inp["colors"], inp["depths"], inp["point_list"],
                        inp["ranges"], inp["W"], inp["H"])
    return inp, ref


def _tile_max(a, W, H, tile=(16, 16)):
    tx, ty = (W + tile[0] - 1) // tile[0], (H + tile[1] - 1) // tile[1]
    pad = np.zeros((ty * tile[1], tx * tile[0]), a.dtype)
    pad[:H, :W] = a
    return pad.reshape(ty, tile[1], tx, tile[0]).max(axis=(1, 3)).reshape(-1)


def _check_prefixes(pl_t, rg_t, pl_full, rg_full, need, base=0, shift=0):
    """Every truncated list: a prefix of the full list, no shorter than the tile's need."""
    n_cut = 0
    for t in range(rg_full.shape[0]):
        a, b = int(rg_t[t, 0]), int(rg_t[t, 1])
        fa, fb = int(rg_full[t, 0]), int(rg_full[t, 1])
        L, F = b - a, fb - fa
        assert L <= F, t
        assert L >= min(F, int(need[t])), (t, L, need[t])
        if L:
            np.testing.assert_array_equal(pl_t[a:b] - shift, pl_full[fa:fa + L], err_msg=f"tile {t}")
        n_cut += L < F
    return n_cut


def test_truncated_lists_are_covering_prefixes(R, dense):
    inp, ref = dense
    W, H = inp["W"], inp["H"]
    g = to_gpu(inp)
    plan = R.Plan()
    pl, rg, K = R.bin_and_sort(plan, g["means2D"], g["radii"], g["depths"], W, H,
                               conic_opacity=g["conic_opacity"])
    torch.cuda.synchronize()
    plan.check()
    pl, rg = pl[:K].cpu().numpy().view(np.uint32), rg.cpu().numpy().view(np.uint32)
    need = _tile_max(ref["n_eval"], W, H)
    n_cut = _check_prefixes(pl, rg, inp["point_list"], inp["ranges"], need)
    full = int(inp["point_list"].size)
    assert n_cut > 0 and K < 0.5 * full, (K, full)  # the dense cluster's tiles are cut
    plan.close()


@pytest.mark.parametrize("mode", ["pixel", "gaussian", "static"])
def test_render_from_truncated_lists_matches_oracle(R, dense, mode):
    inp, ref = dense
    W, H = inp["W"], inp["H"]
    g = to_gpu(inp)
    plan = R.Plan(heavy_threshold=256, gw_pixels=4)
    pl, rg, K = R.bin_and_sort(plan, g["means2D"], g["radii"], g["depths"], W, H,
                               conic_opacity=g["conic_opacity"])
    out = R.render_forward(plan, g["means2D"], g["conic_opacity"], g["colors"], g["depths"], pl, K, rg, W, H,
                           (16, 16), (0.0, 0.0, 0.0), mode, n_eval=True)
    torch.cuda.synchronize()
    plan.check()
    o = {k: v.cpu().numpy() for k, v in out.items()}
    compare_images(o["color"], ref, what=f"truncated {mode}")
    un = ref["flags"] == 0
    np.testing.assert_array_equal(o["n_contrib"][un], ref["n_contrib"][un])
    np.testing.assert_array_equal(o["n_eval"][un], ref["n_eval"][un])
    if mode == "gaussian":
        return
    rng = np.random.default_rng(31)
    gC = rng.normal(size=(3, H, W)).astype(np.float32)
    gC[:, ~un] = 0
    gr = R.render_backward(plan, g["means2D"], g["conic_opacity"], g["colors"], g["depths"], pl, K, rg, W, H,
                           out["final_T"], out["n_contrib"], torch.from_numpy(gC).cuda(), None, None, (16, 16),
                           (0.0, 0.0, 0.0), mode)
    torch.cuda.synchronize()
    plan.check()
    og = oracle.render_backward(inp["means2D"], inp["conic_opacity"], inp["colors"], inp["depths"],
                                inp["point_list"], inp["ranges"], W, H, gC, abs_terms=True)
    compare_grads({k: v.cpu().numpy() for k, v in gr.items()}, og, what=f"truncated {mode}",
                  n_contrib_max=int(ref["n_contrib"].max()))
    plan.close()


@pytest.mark.parametrize("W,H", [(1280, 720), (64, 48)])
def test_truncation_on_small_tile_grids(R, W, H):
    """Tile grids whose credit counters are small (a few KB of shared memory beside the
    kernel's fixed tables): truncation runs and keeps covering prefixes."""
    s = scene("cfg3early", 0.1)
    s["cameras"][0].update(W=W, H=H, cx=(W - 1) / 2, cy=(H - 1) / 2, fx=W, fy=W)
    inp = oracle_render_inputs(s)
    ref = oracle.render(inp["means2D"], inp["conic_opacity"], inp["colors"], inp["depths"], inp["point_list"],
                        inp["ranges"], W, H)
    g = to_gpu(inp)
    plan = R.Plan()
    pl, rg, K = R.bin_and_sort(plan, g["means2D"], g["radii"], g["depths"], W, H,
                               conic_opacity=g["conic_opacity"])
    torch.cuda.synchronize()
    plan.check()
    pl, rg = pl[:K].cpu().numpy().view(np.uint32), rg.cpu().numpy().view(np.uint32)
    _check_prefixes(pl, rg, inp["point_list"], inp["ranges"], _tile_max(ref["n_eval"], W, H))
    plan.close()


def test_batched_truncation_per_view(R):
    """Three uneven views of one clustered scene: each view's truncated lists are covering
    prefixes of that view's oracle lists (record indices v N + g)."""
    s = scenes.scene_config("cfg2", 0.02)
    g = s["gaussians"]
    g["log_scales"] = (g["log_scales"] + 0.8).astype(np.float32)
    cams = scenes.arc_cameras([(320, 180), (250, 130), (480, 270)], yaw_deg=20.0)
    per_view = []
    for cam in cams:
        pp = oracle.preprocess(g["means3D"], g["log_scales"], g["quats"], g["opacities"], cam)
        per_view.append(dict(means2D=pp["means2D"].astype(np.float32), conic_opacity=pp["conic_opacity"].astype(np.float32),
                             depths=pp["depth"].astype(np.float32), radii=pp["radius"].astype(np.int32)))
    N = g["means3D"].shape[0]
    st = lambda k: torch.from_numpy(np.concatenate([pv[k] for pv in per_view])).cuda()
    plan = R.Plan()
    pl, rg, K = R.bin_and_sort_batched(plan, st("means2D"), st("radii"), st("depths"), cams,
                                       conic_opacity=st("conic_opacity"))
    torch.cuda.synchronize()
    plan.check()
    pl, rg = pl[:K].cpu().numpy().view(np.uint32).astype(np.int64), rg.cpu().numpy().view(np.uint32)
    per, _ = R.tile_counts(cams)
    base, cut, full = 0, 0, 0
    for v, (cam, pv) in enumerate(zip(cams, per_view)):
        opl, org = oracle.bin_tiles(pv["means2D"], pv["radii"], pv["depths"], cam["W"], cam["H"])
        ref = oracle.render(pv["means2D"], pv["conic_opacity"], g["colors"], pv["depths"], opl, org, cam["W"],
                            cam["H"])
        need = _tile_max(ref["n_eval"], cam["W"], cam["H"])
        cut += _check_prefixes(pl, rg[base:base + per[v]], opl, org, need, shift=v * N)
        base += per[v]
        full += opl.size
    assert cut > 0 and K < full
    plan.close()
