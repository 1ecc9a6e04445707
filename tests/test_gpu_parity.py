"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle on the same seeded
float32 inputs.  Marked ``gpu``; run on a GB300 with ``pytest -m gpu``."""
import numpy as np
import pytest

import oracle
from helpers import (IMG_FRAC_MIN, IMG_FRAC_TOL, IMG_MAX_ABS, compare_grads, compare_images, oracle_render_inputs,
                     rel_l2, scene, to_gpu)

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

MODES = ["static", "pixel", "gaussian", "auto"]


@pytest.fixture(scope="module")
def R():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2412_17378_gb300 import raster
    return raster


@pytest.fixture(scope="module")
def plan(R):
    p = R.Plan(heavy_threshold=64, gw_pixels=4)
    yield p
    p.close()


@pytest.fixture(scope="module")
def cfg1():
    return oracle_render_inputs(scene("cfg1"))


def _np(t):
    return t.detach().cpu().numpy()


def _render_gpu(R, plan, inp, mode, bg=(0.0, 0.0, 0.0)):
    g = to_gpu(inp)
    out = R.render_forward(plan, g["means2D"], g["conic_opacity"], g["colors"], g["depths"], g["point_list"], g["K"],
                           g["ranges"], inp["W"], inp["H"], inp["tile"], bg, mode, n_eval=True)
    torch.cuda.synchronize()
    plan.check()
    return {k: _np(v) for k, v in out.items()}, g


# --------------------------------------------------------------------------------- a1 / a2

def test_preprocess_matches_oracle(R, plan):
    s = scene("cfg2", 0.05)
    g, cam = s["gaussians"], s["cameras"][0]
    d = {k: torch.from_numpy(v).cuda() for k, v in g.items()}
    out = R.preprocess(plan, d["means3D"], d["log_scales"], d["quats"], d["opacities"], cam)
    torch.cuda.synchronize()
    ref = oracle.preprocess(g["means3D"], g["log_scales"], g["quats"], g["opacities"], cam)
    rad = _np(out["radii"])
    ok = ref["radius"] > 0
    # radii: exact except where 3 sqrt(lambda) lies within 1e-4 of an integer
    near_int = np.abs(ref["radius_raw"] - np.round(ref["radius_raw"])) < 1e-4
    mism = (rad != ref["radius"]) & ~near_int
    assert mism.sum() <= 1e-4 * len(rad), mism.sum()
    both = ok & (rad > 0)
    np.testing.assert_allclose(_np(out["means2D"])[both], ref["means2D"][both], rtol=2e-6, atol=2e-4)
    np.testing.assert_allclose(_np(out["depths"])[both], ref["depth"][both], rtol=1e-6)
    co = _np(out["conic_opacity"])[both]
    rco = ref["conic_opacity"][both]
    scale = np.abs(rco[:, :3]).max(axis=1, keepdims=True)
    assert np.abs(co[:, :3] - rco[:, :3]).max() / 1 <= 1e-3 * scale.max()
    assert (np.abs(co[:, :3] - rco[:, :3]) <= 2e-4 * scale + 1e-7).mean() > 0.999
    np.testing.assert_array_equal(co[:, 3], rco[:, 3].astype(np.float32))


@pytest.mark.parametrize("name,scale,tile,W_H", [("cfg1", 1.0, (16, 16), None), ("cfg2", 0.02, (16, 8), None),
                                                 ("cfg1", 1.0, (16, 16), (250, 130)),
                                                 # 65536 tiles: counters exceed shared memory -> radix-sort path
                                                 ("cfg1", 0.1, (8, 4), (2048, 1024))])
def test_binning_bit_exact(R, plan, name, scale, tile, W_H):
    s = scene(name, scale)
    if W_H is not None:
        s["cameras"][0]["W"], s["cameras"][0]["H"] = W_H
    inp = oracle_render_inputs(s, tile=tile)
    g = to_gpu(inp)
    pl, rg, K = R.bin_and_sort(plan, g["means2D"], g["radii"], g["depths"], inp["W"], inp["H"], tile)
    torch.cuda.synchronize()
    assert K == inp["point_list"].size
    np.testing.assert_array_equal(_np(rg).astype(np.uint32), inp["ranges"])
    np.testing.assert_array_equal(_np(pl)[:K].astype(np.uint32), inp["point_list"])


@pytest.mark.parametrize("bin_block", [32, 96, 512, 2560, 4096])
def test_binning_block_sizes_bit_exact(R, bin_block):
    """The counting blocks' size changes the work split only: single-word masks (32), a block
    smaller than one 512-Gaussian pass (96), one pass (512), several passes with a partial
    last one (2560 = 5 x 512) -- the path large frames take -- and whole passes (4096)."""
    s = scene("cfg2", 0.02)
    s["cameras"][0].update(W=700, H=300, cx=349.5, cy=149.5)
    inp = oracle_render_inputs(s)
    g = to_gpu(inp)
    p = R.Plan(bin_block=bin_block)
    pl, rg, K = R.bin_and_sort(p, g["means2D"], g["radii"], g["depths"], inp["W"], inp["H"])
    torch.cuda.synchronize()
    assert K == inp["point_list"].size
    np.testing.assert_array_equal(_np(rg).astype(np.uint32), inp["ranges"])
    np.testing.assert_array_equal(_np(pl)[:K].astype(np.uint32), inp["point_list"])
    p.close()


def test_binning_degenerate_inputs(R):
    """No visible Gaussian, one Gaussian covering every tile, and all Gaussians at one depth."""
    p = R.Plan(bin_block=64)
    W, H = 100, 60
    n = 300
    rng = np.random.default_rng(8)
    m2 = np.stack([rng.uniform(0, W, n), rng.uniform(0, H, n)], 1).astype(np.float32)
    cases = {"none visible": (np.zeros(n, np.int32), rng.uniform(1, 5, n)),
             "one covers all": (np.where(np.arange(n) == 7, 500, 0).astype(np.int32), rng.uniform(1, 5, n)),
             "equal depths": (rng.integers(1, 40, n).astype(np.int32), np.full(n, 2.5))}
    for what, (radii, depth) in cases.items():
        dp = depth.astype(np.float32)
        opl, org = oracle.bin_tiles(m2, radii, dp, W, H)
        pl, rg, K = R.bin_and_sort(p, torch.from_numpy(m2).cuda(), torch.from_numpy(radii).cuda(),
                                   torch.from_numpy(dp).cuda(), W, H)
        torch.cuda.synchronize()
        assert K == opl.size, what
        np.testing.assert_array_equal(_np(rg).astype(np.uint32), org, err_msg=what)
        np.testing.assert_array_equal(_np(pl)[:K].astype(np.uint32), opl, err_msg=what)
    p.close()


# --------------------------------------------------------------------------------- a4 / a5

@pytest.mark.parametrize("mode", MODES)
def test_forward_cfg1_matches_oracle(R, plan, cfg1, mode):
    inp = cfg1
    ref = oracle.render(inp["means2D"], inp["conic_opacity"], inp["colors"], inp["depths"], inp["point_list"],
                        inp["ranges"], inp["W"], inp["H"])
    out, _ = _render_gpu(R, plan, inp, mode)
    compare_images(out["color"], ref, what=mode)
    un = ref["flags"] == 0
    np.testing.assert_array_equal(out["n_contrib"][un], ref["n_contrib"][un])
    np.testing.assert_array_equal(out["n_eval"][un], ref["n_eval"][un])
    np.testing.assert_allclose(out["final_T"], ref["final_T"], atol=2e-3)
    np.testing.assert_allclose(out["alpha"], ref["alpha"], atol=2e-3)
    np.testing.assert_allclose(out["depth"][un], ref["depth"][un], atol=2e-3 * 6)


@pytest.mark.parametrize("mode", MODES)
@pytest.mark.parametrize("W,H,tile", [(100, 70, (16, 16)), (67, 33, (16, 8)), (32, 32, (32, 8))])
def test_forward_ragged_and_tile_shapes(R, plan, mode, W, H, tile):
    s = scene("cfg1", 0.3)
    cam = s["cameras"][0]
    cam.update(W=W, H=H, cx=(W - 1) / 2, cy=(H - 1) / 2, fx=W, fy=W)
    inp = oracle_render_inputs(s, tile=tile)
    bg = (0.1, 0.5, 0.9)
    ref = oracle.render(inp["means2D"], inp["conic_opacity"], inp["colors"], inp["depths"], inp["point_list"],
                        inp["ranges"], W, H, tile[0], tile[1], bg=bg)
    out, _ = _render_gpu(R, plan, inp, mode, bg)
    compare_images(out["color"], ref, what=f"{mode} {W}x{H}")


@pytest.mark.parametrize("mode", MODES)
def test_forward_edge_cases(R, plan, mode):
    """Empty scene, all Gaussians culled, one opaque stack that stops early."""
    W = H = 48
    cam = dict(W=W, H=H)
    # (1) no Gaussian touches any tile
    inp = dict(means2D=np.full((5, 2), -1e4, np.float32), conic_opacity=np.tile([[1, 0, 1, 0.5]], (5, 1)).astype(np.float32),
               colors=np.ones((5, 3), np.float32), depths=np.arange(1, 6, dtype=np.float32), radii=np.zeros(5, np.int32),
               W=W, H=H, tile=(16, 16), cam=cam)
    inp["point_list"], inp["ranges"] = oracle.bin_tiles(inp["means2D"], inp["radii"], inp["depths"], W, H)
    out, _ = _render_gpu(R, plan, inp, mode, (0.2, 0.3, 0.4))
    assert np.allclose(out["color"][0], 0.2) and np.allclose(out["final_T"], 1.0) and (out["n_contrib"] == 0).all()
    # (2) 40 identical layers with alpha 0.5 at the centre pixel: 13 accumulated, the 14th stops
    n = 40
    inp["means2D"] = np.tile([[24.0, 24.0]], (n, 1)).astype(np.float32)
    inp["conic_opacity"] = np.tile([[0.02, 0.0, 0.02, 0.5]], (n, 1)).astype(np.float32)
    inp["colors"] = np.tile([[0.25, 0.5, 1.0]], (n, 1)).astype(np.float32)
    inp["depths"] = np.arange(1, n + 1, dtype=np.float32)
    inp["radii"] = np.full(n, 30, np.int32)
    inp["point_list"], inp["ranges"] = oracle.bin_tiles(inp["means2D"], inp["radii"], inp["depths"], W, H)
    ref = oracle.render(inp["means2D"], inp["conic_opacity"], inp["colors"], inp["depths"], inp["point_list"],
                        inp["ranges"], W, H)
    out, _ = _render_gpu(R, plan, inp, mode)
    assert out["n_contrib"][24, 24] == 13 and out["n_eval"][24, 24] == 14
    compare_images(out["color"], ref, what=f"stack {mode}")


def test_all_kernels_agree(R, plan, cfg1):
    """Sec. 4: load balancing changes no result -- every mode gives the same image up to
    float32 reassociation, with identical integer outputs outside ambiguous pixels."""
    outs = {m: _render_gpu(R, plan, cfg1, m)[0] for m in MODES}
    ref = oracle.render(cfg1["means2D"], cfg1["conic_opacity"], cfg1["colors"], cfg1["depths"], cfg1["point_list"],
                        cfg1["ranges"], cfg1["W"], cfg1["H"])
    un = ref["flags"] == 0
    for m in MODES[1:]:
        assert np.abs(outs[m]["color"] - outs["static"]["color"]).max() < 1e-4
        np.testing.assert_array_equal(outs[m]["n_contrib"][un], outs["static"]["n_contrib"][un])
    # same sequential arithmetic per pixel: equal up to the compiler's FMA contraction choices
    np.testing.assert_allclose(outs["pixel"]["color"], outs["static"]["color"], rtol=0, atol=1e-6)


def test_stats_count_evaluated_pairs(R, plan, cfg1):
    plan.reset_stats()
    out, _ = _render_gpu(R, plan, cfg1, "auto")
    st = plan.stats()
    ref = oracle.render(cfg1["means2D"], cfg1["conic_opacity"], cfg1["colors"], cfg1["depths"], cfg1["point_list"],
                        cfg1["ranges"], cfg1["W"], cfg1["H"])
    assert abs(st["eval_pairs"] - int(ref["n_eval"].sum())) <= 1e-5 * ref["n_eval"].sum() + 10
    assert abs(st["contrib_pairs"] - int(ref["n_acc"].sum())) <= 1e-5 * ref["n_acc"].sum() + 10
    assert st["items"] == st["last_num_items"]


# --------------------------------------------------------------------------------- a6

def _backward_case(R, plan, inp, mode, bg=(0.0, 0.0, 0.0), with_extra=True, seed=0):
    W, H = inp["W"], inp["H"]
    rng = np.random.default_rng(seed)
    ref_f = oracle.render(inp["means2D"], inp["conic_opacity"], inp["colors"], inp["depths"], inp["point_list"],
                          inp["ranges"], W, H, inp["tile"][0], inp["tile"][1], bg=bg)
    gC = rng.normal(size=(3, H, W)).astype(np.float32)
    gD = (0.1 * rng.normal(size=(H, W))).astype(np.float32) if with_extra else None
    gA = rng.normal(size=(H, W)).astype(np.float32) if with_extra else None
    flagged = ref_f["flags"] != 0  # decision-ambiguous pixels pass no gradient on either side
    gC[:, flagged] = 0
    if with_extra:
        gD[flagged] = 0
        gA[flagged] = 0
    ref = oracle.render_backward(inp["means2D"], inp["conic_opacity"], inp["colors"], inp["depths"],
                                 inp["point_list"], inp["ranges"], W, H, gC, gD, gA, inp["tile"][0], inp["tile"][1],
                                 bg=bg, abs_terms=True)
    ref["nc_max"] = int(ref_f["n_contrib"].max())
    out, g = _render_gpu(R, plan, inp, mode, bg)
    dev = lambda a: None if a is None else torch.from_numpy(a).cuda()
    grads = R.render_backward(plan, g["means2D"], g["conic_opacity"], g["colors"], g["depths"], g["point_list"],
                              g["K"], g["ranges"], W, H, dev(out["final_T"]), dev(out["n_contrib"]), dev(gC),
                              dev(gD), dev(gA), inp["tile"], bg, mode)
    torch.cuda.synchronize()
    plan.check()
    return {k: _np(v) for k, v in grads.items()}, ref


@pytest.mark.parametrize("mode", MODES)
def test_backward_cfg1_matches_oracle(R, plan, cfg1, mode):
    got, ref = _backward_case(R, plan, cfg1, mode, bg=(0.3, 0.2, 0.1))
    compare_grads(got, ref, ("means2D", "conic", "opacity", "colors", "depths"), what=f"cfg1 {mode}",
                  n_contrib_max=ref["nc_max"])


@pytest.mark.parametrize("mode", ["static", "pixel"])
def test_backward_fd_crop(R, plan, mode):
    """The 512-Gaussian 64x64 crop whose oracle gradient is pinned by central differences."""
    inp = oracle_render_inputs(scene("fdcrop"))
    got, ref = _backward_case(R, plan, inp, mode, with_extra=False, seed=3)
    compare_grads(got, ref, what=f"fdcrop {mode}", n_contrib_max=ref["nc_max"])


@pytest.mark.parametrize("mode,threshold", [("pixel", 64), ("auto", 1 << 30), ("auto", 64)])
def test_backward_reuses_or_rebuilds_forward_state(R, cfg1, mode, threshold):
    """A backward on the arrays of the plan's last forward reuses its packed records (and
    builds its own, cost-ordered work list); after a forward on other arrays it rebuilds
    the records; a plan that ran no forward builds them.  All three give the same
    gradients."""
    W, H, tile = cfg1["W"], cfg1["H"], cfg1["tile"]
    rng = np.random.default_rng(4)
    gC = torch.from_numpy(rng.normal(size=(3, H, W)).astype(np.float32)).cuda()
    gA, gB = to_gpu(cfg1), to_gpu(cfg1)  # same values, different arrays

    def fwd(pl, g):
        return R.render_forward(pl, g["means2D"], g["conic_opacity"], g["colors"], g["depths"], g["point_list"],
                                g["K"], g["ranges"], W, H, tile, (0.0, 0.0, 0.0), mode)

    def bwd(pl, g, out):
        gr = R.render_backward(pl, g["means2D"], g["conic_opacity"], g["colors"], g["depths"], g["point_list"],
                               g["K"], g["ranges"], W, H, out["final_T"], out["n_contrib"], gC, None, None, tile,
                               (0.0, 0.0, 0.0), mode)
        torch.cuda.synchronize()
        pl.check()
        return {k: _np(v) for k, v in gr.items()}

    plans = [R.Plan(heavy_threshold=threshold) for _ in range(3)]
    out = fwd(plans[0], gA)
    reused = bwd(plans[0], gA, out)
    fwd(plans[1], gA)
    fwd(plans[1], gB)  # the plan now holds gB's records
    rebuilt = bwd(plans[1], gA, out)
    fresh = bwd(plans[2], gA, out)
    for k in ("means2D", "conic", "opacity", "colors"):
        assert rel_l2(reused[k], fresh[k]) < 1e-6, k
        assert rel_l2(rebuilt[k], fresh[k]) < 1e-6, k
    for pl in plans:
        pl.close()


# --------------------------------------------------------------------------------- device checks

def test_device_checks_report_bad_indices_and_ranges(R, plan, cfg1):
    g = to_gpu(cfg1)
    W, H = cfg1["W"], cfg1["H"]
    bad = g["point_list"].clone()
    bad[7] = 10 ** 8  # index >= N: the kernels' bounds check skips it and raises a flag
    for mode in MODES:
        R.render_forward(plan, g["means2D"], g["conic_opacity"], g["colors"], g["depths"], bad, g["K"], g["ranges"],
                         W, H, (16, 16), (0, 0, 0), mode)
        with pytest.raises(R.BgsError) as e:
            plan.check()
        assert e.value.code == -4
    rg = g["ranges"].clone()
    rg[3, 1] = g["K"] + 100  # past num_entries: the tile renders empty and a flag is raised
    R.render_forward(plan, g["means2D"], g["conic_opacity"], g["colors"], g["depths"], g["point_list"], g["K"], rg,
                     W, H, (16, 16), (0, 0, 0), "auto")
    with pytest.raises(R.BgsError):
        plan.check()
    plan.check()  # bits were cleared


def test_queue_drain_check_reports_injected_fault(R, cfg1):
    """Every persistent pass checks that it ran each queued item exactly once.  A host-side
    fault (the queue marked exhausted before the pass) must surface as BGS_CHECK_QUEUE;
    the next, clean passes report nothing."""
    from paper_2412_17378_gb300 import _lib
    p = R.Plan(heavy_threshold=64)
    g = to_gpu(cfg1)
    W, H = cfg1["W"], cfg1["H"]
    rng = np.random.default_rng(9)
    gC = torch.from_numpy(rng.normal(size=(3, H, W)).astype(np.float32)).cuda()

    def fwd(mode):
        return R.render_forward(p, g["means2D"], g["conic_opacity"], g["colors"], g["depths"], g["point_list"], g["K"],
                                g["ranges"], W, H, (16, 16), (0, 0, 0), mode)

    def bwd(out, mode):
        R.render_backward(p, g["means2D"], g["conic_opacity"], g["colors"], g["depths"], g["point_list"], g["K"],
                          g["ranges"], W, H, out["final_T"], out["n_contrib"], gC, None, None, (16, 16), (0, 0, 0),
                          mode)

    for mode in ("auto", "pixel", "gaussian"):
        out = fwd(mode)
        bwd(out, mode)
        torch.cuda.synchronize()
        p.check()  # clean passes
        p.inject_fault(_lib.CHECK_QUEUE)
        out = fwd(mode)
        with pytest.raises(R.BgsError) as e:
            p.check()
        assert e.value.code == -4 and "queue" in str(e.value)
        out = fwd(mode)
        p.inject_fault(_lib.CHECK_QUEUE)
        bwd(out, mode)
        with pytest.raises(R.BgsError) as e:
            p.check()
        assert "queue" in str(e.value)
        bwd(out, mode)
        torch.cuda.synchronize()
        p.check()
    p.close()


def test_exp2_accuracy(R):
    """The render kernels' exponential (ex2.approx.ftz) against float64 2^x on the range the
    blend uses (alpha >= 1/255 needs 2^x >= 1/255 with x <= 0)."""
    x = np.linspace(-30.0, 0.0, 200001).astype(np.float32)
    y = _np(R.debug_exp2(torch.from_numpy(x).cuda()))
    ref = np.exp2(x.astype(np.float64))
    rel = np.abs(y - ref) / ref
    assert rel.max() < 2.0 ** -21, rel.max()


@pytest.mark.parametrize("rows", [1, 2, 4, 8])
def test_pixel_rows_sub_tiles(R, cfg1, rows):
    """Every sub-tile size of the pixel-wise items (8 x 4, 8 x 8, 8 x 16, 16 x 16) gives the
    oracle's image and gradients."""
    p = R.Plan(heavy_threshold=1 << 30, pixel_rows=rows)
    ref = oracle.render(cfg1["means2D"], cfg1["conic_opacity"], cfg1["colors"], cfg1["depths"], cfg1["point_list"],
                        cfg1["ranges"], cfg1["W"], cfg1["H"])
    out, _ = _render_gpu(R, p, cfg1, "auto")
    compare_images(out["color"], ref, what=f"rows {rows}")
    got, gref = _backward_case(R, p, cfg1, "pixel", seed=rows)
    compare_grads(got, gref, what=f"rows {rows}", n_contrib_max=gref["nc_max"])
    p.close()


@pytest.mark.parametrize("rows", [4, 8])
@pytest.mark.parametrize("W,H,tile", [(100, 70, (16, 16)), (67, 33, (16, 8)), (32, 32, (32, 8)), (40, 24, (8, 8))])
def test_pixel_items_on_ragged_images_and_tiles(R, rows, W, H, tile):
    """Items larger than the tile or than its part inside the image (16 x 16 items on 16 x 8
    or 8 x 8 tiles, ragged image edges) render only their in-tile, in-image pixels."""
    s = scene("cfg1", 0.3)
    cam = s["cameras"][0]
    cam.update(W=W, H=H, cx=(W - 1) / 2, cy=(H - 1) / 2, fx=W, fy=W)
    inp = oracle_render_inputs(s, tile=tile)
    ref = oracle.render(inp["means2D"], inp["conic_opacity"], inp["colors"], inp["depths"], inp["point_list"],
                        inp["ranges"], W, H, tile[0], tile[1])
    p = R.Plan(heavy_threshold=1 << 30, pixel_rows=rows)
    out, _ = _render_gpu(R, p, inp, "pixel")
    compare_images(out["color"], ref, what=f"rows {rows} {W}x{H} {tile}")
    got, gref = _backward_case(R, p, inp, "pixel", seed=7)
    compare_grads(got, gref, what=f"rows {rows} {W}x{H} {tile}", n_contrib_max=gref["nc_max"])
    p.close()


def test_autotuner_choice_keeps_parity(R, cfg1):
    p = R.Plan()
    g = to_gpu(cfg1)
    cam = dict(W=cfg1["W"], H=cfg1["H"], fx=256.0, fy=256.0, cx=127.5, cy=127.5, viewmat=np.eye(4))
    best_ms, knobs = R.autotune_render(p, g["means2D"], g["conic_opacity"], g["colors"], g["depths"],
                                       g["point_list"], g["K"], g["ranges"], [cam])
    assert best_ms > 0 and knobs["pixel_rows"] in (1, 2, 4, 8) and knobs["queue_chunk"] in (1, 2, 4)
    ref = oracle.render(cfg1["means2D"], cfg1["conic_opacity"], cfg1["colors"], cfg1["depths"], cfg1["point_list"],
                        cfg1["ranges"], cfg1["W"], cfg1["H"])
    out, _ = _render_gpu(R, p, cfg1, "auto")
    compare_images(out["color"], ref, what="tuned")
    p.close()


_WL_CACHE = {}


def _worklist_scene(W, H):
    if (W, H) not in _WL_CACHE:
        s = scene("cfg1", 0.3)
        cam = s["cameras"][0]
        cam.update(W=W, H=H, cx=(W - 1) / 2, cy=(H - 1) / 2, fx=0.25 * W, fy=0.25 * W)
        inp = oracle_render_inputs(s)
        ref = oracle.render(inp["means2D"], inp["conic_opacity"], inp["colors"], inp["depths"], inp["point_list"],
                            inp["ranges"], W, H)
        _WL_CACHE[(W, H)] = (inp, ref)
    return _WL_CACHE[(W, H)]


@pytest.mark.parametrize("W,H", [(1000, 700), (4096, 4208)])
@pytest.mark.parametrize("lpt", [True, False])
@pytest.mark.parametrize("mode", ["pixel", "gaussian", "auto"])
def test_worklist_small_and_large_tile_grids(R, W, H, lpt, mode):
    """The work list of a3 (Sec. 4.1 / 4.3) on 2772 and 67328 tiles, with and without the
    heaviest-first order and with every tile kind: every item must run exactly once (the
    drain check) and the image must match the oracle."""
    inp, ref = _worklist_scene(W, H)
    p = R.Plan(heavy_threshold=8, gw_pixels=4, lpt_order=lpt)
    p.reset_stats()
    out, _ = _render_gpu(R, p, inp, mode)
    compare_images(out["color"], ref, what=f"worklist {mode} lpt={lpt} {W}x{H}")
    un = ref["flags"] == 0
    np.testing.assert_array_equal(out["n_contrib"][un], ref["n_contrib"][un])
    st = p.stats()
    assert st["items"] == st["last_num_items"] > 0
    p.close()
