"""GPU parity of the Gaussian-wise path (Sec. 4.2-4.3, Algorithm 6) with long lists split
into segments walked by separate warps and merged per pixel: stacks of more than 10^4
faint Gaussians (alpha about 0.001, below the 1/255 cut, mixed with alpha about 0.0045),
whose pixels walk the whole list or stop deep inside it, against the FP64 oracle element by
element; several segment lengths, pixel groups and tile shapes; the fallback to unsplit
lists when the split would exceed its item budget; the heavy-veil frame.  Marked ``gpu``."""
import numpy as np
import pytest

import oracle
from helpers import compare_images, oracle_render_inputs, scene, to_gpu

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

# alpha of the accepted layers: the geometric transmittance (1 - A)^k crosses 1e-4 half-way
# between k = 2042 and k = 2043 (ln(1e-4) / ln(1 - A) = 2042.5), so every pixel's stop is a
# quarter of a step (0.22 %) away from the threshold on either side
A_HI = 1.0 - np.exp(np.log(1e-4) / 2042.5)
A_LO = 0.001  # below 1/255: visited, never accumulated


@pytest.fixture(scope="module")
def R():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2412_17378_gb300 import raster
    return raster


def stack(kind: str, W=32, H=32, tile=(16, 16), n=12000, seed=0):
    """n Gaussians centred on the image, wide enough that G is within 1e-4 of 1 at every
    pixel (so a layer's alpha is its opacity to that precision), in depth order 1..n."""
    rng = np.random.default_rng(seed)
    if kind == "faint":        # nothing accumulated: every pixel walks all n entries
        o = np.full(n, A_LO)
    elif kind == "mixed":      # every 5th layer accumulated: stop at entry 5 * 2042 + 1
        o = np.where(np.arange(n) % 5 == 0, A_HI, A_LO)
    elif kind == "uniform":    # every layer accumulated: stop at entry 2043
        o = np.full(n, A_HI)
    elif kind == "open":       # every 10th layer accumulated: 1200 layers, no stop
        o = np.where(np.arange(n) % 10 == 0, A_HI, A_LO)
    else:
        raise ValueError(kind)
    cx, cy = W / 2.0 + 0.25, H / 2.0 + 0.25  # no pixel centre at dx = dy = 0 (power 0)
    inp = dict(means2D=np.tile([[cx, cy]], (n, 1)).astype(np.float32),
               conic_opacity=np.stack([np.full(n, 2e-7), np.zeros(n), np.full(n, 2e-7), o], 1).astype(np.float32),
               colors=rng.uniform(0, 1, (n, 3)).astype(np.float32), depths=np.arange(1, n + 1, dtype=np.float32),
               radii=np.full(n, int(max(W, H) + 8), np.int32), W=W, H=H, tile=tuple(tile), cam=dict(W=W, H=H))
    inp["point_list"], inp["ranges"] = oracle.bin_tiles(inp["means2D"], inp["radii"], inp["depths"], W, H, *tile)
    return inp


def render(R, plan, inp, mode, bg=(0.0, 0.0, 0.0)):
    g = to_gpu(inp)
    out = R.render_forward(plan, g["means2D"], g["conic_opacity"], g["colors"], g["depths"], g["point_list"], g["K"],
                           g["ranges"], inp["W"], inp["H"], inp["tile"], bg, mode, n_eval=True)
    torch.cuda.synchronize()
    plan.check()
    return {k: v.detach().cpu().numpy() for k, v in out.items()}


def oracle_ref(inp, bg=(0.0, 0.0, 0.0)):
    return oracle.render(inp["means2D"], inp["conic_opacity"], inp["colors"], inp["depths"], inp["point_list"],
                         inp["ranges"], inp["W"], inp["H"], inp["tile"][0], inp["tile"][1], bg=bg)


def check(out, ref, what):
    compare_images(out["color"], ref, what=what)
    un = ref["flags"] == 0
    np.testing.assert_array_equal(out["n_contrib"][un], ref["n_contrib"][un], err_msg=what)
    np.testing.assert_array_equal(out["n_eval"][un], ref["n_eval"][un], err_msg=what)
    np.testing.assert_allclose(out["final_T"][un], ref["final_T"][un], rtol=2e-3, atol=1e-6, err_msg=what)
    np.testing.assert_allclose(out["final_T"], ref["final_T"], atol=2e-3, err_msg=what)
    np.testing.assert_allclose(out["alpha"], ref["alpha"], atol=2e-3, err_msg=what)
    np.testing.assert_allclose(out["depth"][un], ref["depth"][un], rtol=2e-3, atol=2e-3, err_msg=what)


STACK_STOPS = {"faint": (0, 12000), "mixed": (5 * 2041 + 1, 5 * 2042 + 1), "uniform": (2042, 2043),
               "open": (10 * 1199 + 1, 12000)}


@pytest.mark.parametrize("kind", list(STACK_STOPS))
@pytest.mark.parametrize("P,L", [(4, 256), (4, 2048), (1, 512), (8, 256), (2, 1024), (16, 256), (16, 2048)])
def test_heavy_stacks_match_oracle(R, kind, P, L):
    inp = stack(kind)
    ref = oracle_ref(inp)
    # the closed form of the geometric stack pins the oracle's integer outputs here
    nc, ne = STACK_STOPS[kind]
    assert (ref["n_contrib"] == nc).all() and (ref["n_eval"] == ne).all() and (ref["flags"] == 0).all()
    plan = R.Plan(heavy_threshold=64, gw_pixels=P, gw_segment=L)
    try:
        plan.reset_stats()
        out = render(R, plan, inp, "gaussian")
        check(out, ref, f"{kind} P={P} L={L}")
        st = plan.stats()
        assert st["eval_pairs"] == int(ref["n_eval"].sum()) and st["contrib_pairs"] == int(ref["n_acc"].sum())
        out = render(R, plan, inp, "auto")
        check(out, ref, f"{kind} auto P={P} L={L}")
    finally:
        plan.close()


@pytest.mark.parametrize("kind", ["mixed", "uniform"])
@pytest.mark.parametrize("W,H,tile,P", [(37, 29, (16, 8), 8), (50, 21, (32, 8), 4), (17, 40, (8, 8), 2),
                                        (45, 27, (16, 16), 16)])
def test_heavy_stacks_ragged_tiles(R, kind, W, H, tile, P):
    """Partial pixel groups (the tile's visible part not a multiple of P) and ragged tiles."""
    inp = stack(kind, W, H, tile, n=11000, seed=1)
    ref = oracle_ref(inp, bg=(0.3, 0.1, 0.7))
    plan = R.Plan(heavy_threshold=0, gw_pixels=P, gw_segment=256)
    try:
        check(render(R, plan, inp, "gaussian", bg=(0.3, 0.1, 0.7)), ref, f"{kind} {W}x{H} {tile} P={P}")
    finally:
        plan.close()


def test_pixel_and_gaussian_items_agree_on_stacks(R):
    inp = stack("mixed", n=10500, seed=2)
    plan = R.Plan(heavy_threshold=64, gw_pixels=4, gw_segment=512)
    try:
        ref = oracle_ref(inp)
        outs = {m: render(R, plan, inp, m) for m in ("pixel", "gaussian", "static")}
        for m, o in outs.items():
            check(o, ref, m)
        assert np.abs(outs["gaussian"]["color"] - outs["pixel"]["color"]).max() < 1e-4
    finally:
        plan.close()


@pytest.mark.parametrize("P", [1, 2, 4, 8, 16])
@pytest.mark.parametrize("L", [256, 768])
def test_cfg1_short_segments(R, P, L):
    """Every tile Gaussian-wise with short segments: most pixels stop in a later segment."""
    inp = oracle_render_inputs(scene("cfg1"))
    ref = oracle_ref(inp)
    plan = R.Plan(heavy_threshold=0, gw_pixels=P, gw_segment=L)
    try:
        plan.reset_stats()
        out = render(R, plan, inp, "gaussian")
        check(out, ref, f"cfg1 P={P} L={L}")
        st = plan.stats()
        tot = ref["n_eval"].sum()
        assert abs(st["eval_pairs"] - int(tot)) <= 1e-5 * tot + 10
        assert st["items"] == st["last_num_items"]
    finally:
        plan.close()


def test_overlapping_ranges_fall_back_to_unsplit_lists(R):
    """Every tile's range spans the whole point list (the ranges overlap): splitting would
    need more items than the list's budget, so the lists are walked unsplit -- same result."""
    inp = stack("mixed", n=12000, seed=3)
    K = inp["point_list"].size
    ntiles = inp["ranges"].shape[0]
    # one tile's list, shared by every tile
    t0 = inp["ranges"][0]
    pl = inp["point_list"][t0[0]:t0[1]].copy()
    inp["point_list"] = pl
    inp["ranges"] = np.tile(np.array([[0, pl.size]], np.uint32), (ntiles, 1))
    assert ntiles > 1 and K == ntiles * pl.size
    ref = oracle_ref(inp)
    plan = R.Plan(heavy_threshold=0, gw_pixels=4, gw_segment=256)
    try:
        check(render(R, plan, inp, "gaussian"), ref, "overlapping ranges")
    finally:
        plan.close()


@pytest.fixture(scope="module")
def heavy():
    return oracle_render_inputs(scene("heavy", 0.5))


@pytest.mark.parametrize("mode", ["gaussian", "auto"])
def test_heavy_veil_frame_matches_oracle(R, heavy, mode):
    inp = heavy
    ref = oracle_ref(inp)
    n = (inp["ranges"][:, 1] - inp["ranges"][:, 0]).astype(np.int64)
    assert n.max() > 10_000
    plan = R.Plan(heavy_threshold=2048, gw_pixels=4, gw_segment=2048)
    try:
        check(render(R, plan, inp, mode), ref, f"heavy {mode}")
    finally:
        plan.close()


def test_autotuner_picks_gaussian_wise_on_the_heavy_frame(R):
    """On the heavy-veil frame (truncated lists) the tuner's per-tile selector keeps
    Gaussian-wise items for the veil's tiles: split lists beat the pixel-wise walk there."""
    s = scene("heavy")
    g, cam = s["gaussians"], s["cameras"][0]
    W, H = cam["W"], cam["H"]
    d = {k: torch.from_numpy(v).cuda() for k, v in g.items()}
    plan = R.Plan()
    try:
        pp = R.preprocess(plan, d["means3D"], d["log_scales"], d["quats"], d["opacities"], cam)
        pl, rg, K = R.bin_and_sort(plan, pp["means2D"], pp["radii"], pp["depths"], W, H,
                                   conic_opacity=pp["conic_opacity"])
        nmax = int((rg[:, 1] - rg[:, 0]).max())
        best, desc = R.autotune_render(plan, pp["means2D"], pp["conic_opacity"], d["colors"], pp["depths"], pl, K,
                                       rg, [cam], backward=False)
        assert desc["heavy_threshold"] < nmax, desc
        # the chosen knobs render what the pixel-wise items render
        a = R.render_forward(plan, pp["means2D"], pp["conic_opacity"], d["colors"], pp["depths"], pl, K, rg, W, H,
                             mode="auto")
        b = R.render_forward(plan, pp["means2D"], pp["conic_opacity"], d["colors"], pp["depths"], pl, K, rg, W, H,
                             mode="pixel")
        torch.cuda.synchronize()
        plan.check()
        assert (a["color"] - b["color"]).abs().max().item() < 2e-3
        assert (a["n_contrib"] != b["n_contrib"]).float().mean().item() < 1e-4
    finally:
        plan.close()


# ----------------------------------------------------------------- segmented backward

def _backward(R, plan, inp, mode, seed=0, extra=True, bg=(0.2, 0.4, 0.6)):
    """Forward then backward on one plan (a Gaussian-wise forward that split lists makes the
    backward walk those tiles segment by segment); the oracle's gradient for the same
    upstream gradients, with its |term| sums."""
    from helpers import compare_grads  # noqa: F401  (used by the callers)
    W, H = inp["W"], inp["H"]
    rng = np.random.default_rng(seed)
    ref_f = oracle_ref(inp, bg=bg)
    gC = rng.normal(size=(3, H, W)).astype(np.float32)
    gD = (0.1 * rng.normal(size=(H, W))).astype(np.float32) if extra else None
    gA = rng.normal(size=(H, W)).astype(np.float32) if extra else None
    fl = ref_f["flags"] != 0
    gC[:, fl] = 0
    if extra:
        gD[fl] = 0
        gA[fl] = 0
    ref = oracle.render_backward(inp["means2D"], inp["conic_opacity"], inp["colors"], inp["depths"],
                                 inp["point_list"], inp["ranges"], W, H, gC, gD, gA, inp["tile"][0], inp["tile"][1],
                                 bg=bg, abs_terms=True)
    g = to_gpu(inp)
    out = R.render_forward(plan, g["means2D"], g["conic_opacity"], g["colors"], g["depths"], g["point_list"], g["K"],
                           g["ranges"], W, H, inp["tile"], bg, mode)
    dev = lambda a: None if a is None else torch.from_numpy(a).cuda()
    plan.reset_stats()
    grads = R.render_backward(plan, g["means2D"], g["conic_opacity"], g["colors"], g["depths"], g["point_list"],
                              g["K"], g["ranges"], W, H, out["final_T"], out["n_contrib"], dev(gC), dev(gD), dev(gA),
                              inp["tile"], bg, mode)
    torch.cuda.synchronize()
    plan.check()
    return {k: v.detach().cpu().numpy() for k, v in grads.items()}, ref, int(ref_f["n_contrib"].max()), plan.stats()


@pytest.mark.parametrize("kind", ["mixed", "uniform", "open"])
@pytest.mark.parametrize("P,L,rows", [(4, 256, 2), (8, 2048, 4), (16, 512, 1)])
def test_segmented_backward_on_heavy_stacks(R, kind, P, L, rows):
    """The backward of a forward that split the stack's lists walks every segment on its own
    from the boundary state the merge stored; element-wise against the oracle."""
    from helpers import compare_grads
    inp = stack(kind, n=11000, seed=4)
    plan = R.Plan(heavy_threshold=64, gw_pixels=P, gw_segment=L, pixel_rows=rows)
    try:
        got, ref, ncmax, st = _backward(R, plan, inp, "auto")
        # one pixel-wise item per (sub-block, segment): more items than the tiles' sub-blocks
        per_tile = (16 // 8) * (16 // (4 * rows))
        assert st["last_num_items"] > 4 * per_tile, st
        compare_grads(got, ref, keys=("means2D", "conic", "opacity", "colors", "depths"),
                      what=f"{kind} P={P} L={L}", n_contrib_max=ncmax)
    finally:
        plan.close()


def test_segmented_backward_equals_the_unsegmented_walk(R):
    """Same frame, same upstream gradients: the segmented walk (after a Gaussian-wise forward)
    and the plain walk from the last contributor (after a pixel-wise forward) agree to the
    per-tensor parity bar (rel-L2 1e-3): the plain walk recovers T through ~10^4 divisions
    from the final T, the segmented one from each segment's end (both are within the
    element-wise oracle bounds, tested above)."""
    inp = stack("mixed", 37, 29, (16, 8), n=10500, seed=5)
    plan = R.Plan(heavy_threshold=64, gw_pixels=8, gw_segment=256)
    try:
        seg, ref, _, st_seg = _backward(R, plan, inp, "auto", seed=3)
        pix, _, _, st_pix = _backward(R, plan, inp, "pixel", seed=3)
        assert st_seg["last_num_items"] > st_pix["last_num_items"]
        for k in ("means2D", "conic", "opacity", "colors", "depths"):
            d = np.linalg.norm(seg[k] - pix[k]) / max(np.linalg.norm(pix[k]), 1e-30)
            assert d < 1e-3, (k, d)
    finally:
        plan.close()


def test_segmented_backward_on_the_heavy_veil_frame(R, heavy):
    from helpers import compare_grads
    inp = heavy
    plan = R.Plan(heavy_threshold=2048, gw_pixels=8, gw_segment=2048, pixel_rows=2)
    try:
        got, ref, ncmax, st = _backward(R, plan, inp, "auto", extra=False, bg=(0.0, 0.0, 0.0))
        compare_grads(got, ref, what="heavy veil", n_contrib_max=ncmax)
    finally:
        plan.close()
