"""GPU parity of the batched path (many views of one Gaussian set in one persistent launch)
and of graph capture / replay.  Each view is checked against the FP64 oracle run on that
view alone."""
import numpy as np
import pytest

import oracle
from helpers import compare_grad, compare_images, rel_l2, term_eps
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
def batch():
    """Three uneven views (one ragged) of a 4000-Gaussian clustered scene on a +-20 deg arc."""
    s = scenes.scene_config("cfg2", 0.004)
    g = s["gaussians"]
    cams = scenes.arc_cameras([(160, 96), (250, 130), (96, 64)], yaw_deg=20.0)
    per_view = []
    for cam in cams:
        pp = oracle.preprocess(g["means3D"], g["log_scales"], g["quats"], g["opacities"], cam)
        per_view.append(dict(means2D=pp["means2D"].astype(np.float32),
                             conic_opacity=pp["conic_opacity"].astype(np.float32),
                             depths=pp["depth"].astype(np.float32), radii=pp["radius"].astype(np.int32)))
    return dict(g=g, cams=cams, per_view=per_view, N=g["means3D"].shape[0])


def _stack(batch, key):
    return torch.from_numpy(np.concatenate([pv[key] for pv in batch["per_view"]])).cuda()


def test_batched_binning_equals_per_view_oracle(R, batch):
    plan = R.Plan()
    cams, N = batch["cams"], batch["N"]
    pl, rg, K = R.bin_and_sort_batched(plan, _stack(batch, "means2D"), _stack(batch, "radii"), _stack(batch, "depths"),
                                       cams)
    torch.cuda.synchronize()
    pl, rg = pl.cpu().numpy().astype(np.int64), rg.cpu().numpy().astype(np.int64)
    per, _ = R.tile_counts(cams)
    base_t, total = 0, 0
    for v, (cam, pv) in enumerate(zip(cams, batch["per_view"])):
        opl, org = oracle.bin_tiles(pv["means2D"], pv["radii"], pv["depths"], cam["W"], cam["H"])
        grg = rg[base_t:base_t + per[v]]
        nonempty = grg[:, 1] > grg[:, 0]
        assert (org[:, 1] - org[:, 0] == (grg[:, 1] - grg[:, 0])).all()
        for t in np.nonzero(nonempty)[0]:
            np.testing.assert_array_equal(pl[grg[t, 0]:grg[t, 1]] - v * N, opl[org[t, 0]:org[t, 1]])
        base_t += per[v]
        total += opl.size
    assert K == total
    plan.close()


def _oracle_view(batch, v, bg=(0.0, 0.0, 0.0)):
    cam, pv = batch["cams"][v], batch["per_view"][v]
    opl, org = oracle.bin_tiles(pv["means2D"], pv["radii"], pv["depths"], cam["W"], cam["H"])
    out = oracle.render(pv["means2D"], pv["conic_opacity"], batch["g"]["colors"], pv["depths"], opl, org, cam["W"],
                        cam["H"], bg=bg)
    return out, opl, org


@pytest.mark.parametrize("mode", ["pixel", "gaussian", "auto"])
def test_batched_forward_backward_match_oracle(R, batch, mode):
    plan = R.Plan(heavy_threshold=40, gw_pixels=2)
    cams, N = batch["cams"], batch["N"]
    m2, co, dp = _stack(batch, "means2D"), _stack(batch, "conic_opacity"), _stack(batch, "depths")
    colors = torch.from_numpy(batch["g"]["colors"]).cuda()
    pl, rg, K = R.bin_and_sort_batched(plan, m2, _stack(batch, "radii"), dp, cams)
    bg = (0.2, 0.1, 0.4)
    outs = R.render_forward_batched(plan, m2, co, colors, dp, pl, K, rg, cams, bg=bg, mode=mode, n_eval=True)
    rng = np.random.default_rng(5)
    grads_in, refs = [], []
    for v in range(len(cams)):
        ref, opl, org = _oracle_view(batch, v, bg)
        refs.append((ref, opl, org))
        compare_images(outs[v]["color"].cpu().numpy(), ref, what=f"view {v} {mode}")
        un = ref["flags"] == 0
        np.testing.assert_array_equal(outs[v]["n_contrib"].cpu().numpy()[un], ref["n_contrib"][un])
        gC = rng.normal(size=(3, cams[v]["H"], cams[v]["W"])).astype(np.float32)
        gC[:, ~un] = 0
        grads_in.append(dict(color=torch.from_numpy(gC).cuda(), depth=None, alpha=None))
    gr = R.render_backward_batched(plan, m2, co, colors, dp, pl, K, rg, cams, outs, grads_in, bg=bg, mode=mode)
    torch.cuda.synchronize()
    plan.check()
    col_sum, col_abs = np.zeros((N, 3)), np.zeros((N, 3))
    eps = term_eps(max(int(r[0]["n_contrib"].max()) for r in refs))
    for v in range(len(cams)):
        ref, opl, org = refs[v]
        pv = batch["per_view"][v]
        og = oracle.render_backward(pv["means2D"], pv["conic_opacity"], batch["g"]["colors"], pv["depths"], opl, org,
                                    cams[v]["W"], cams[v]["H"], grads_in[v]["color"].cpu().numpy(), bg=bg,
                                    abs_terms=True)
        sl = slice(v * N, (v + 1) * N)
        for k in ("means2D", "conic", "opacity"):
            compare_grad(gr[k][sl].cpu().numpy(), og[k], f"view {v} {mode} {k}", s=og["abs_" + k], eps=eps)
        col_sum += og["colors"]
        col_abs += og["abs_colors"]
    compare_grad(gr["colors"].cpu().numpy(), col_sum, f"{mode} colors summed over the views", s=col_abs, eps=eps)
    plan.close()


def test_batched_preprocess_equals_single_view(R, batch):
    plan = R.Plan()
    g, cams = batch["g"], batch["cams"]
    d = {k: torch.from_numpy(v).cuda() for k, v in g.items()}
    outb = R.preprocess_batched(plan, d["means3D"], d["log_scales"], d["quats"], d["opacities"], cams)
    N = batch["N"]
    for v, cam in enumerate(cams):
        o1 = R.preprocess(plan, d["means3D"], d["log_scales"], d["quats"], d["opacities"], cam)
        for k in ("means2D", "conic_opacity", "depths", "radii"):
            assert torch.equal(outb[k][v * N:(v + 1) * N], o1[k]), (v, k)
    plan.close()


def test_graph_capture_replays_the_step(R, batch):
    """A whole batched step (projection, binning without host sync, forward, backward)
    captured once and replayed twice gives the eager step's outputs."""
    plan = R.Plan()
    g, cams, N = batch["g"], batch["cams"], batch["N"]
    d = {k: torch.from_numpy(v).cuda() for k, v in g.items()}
    V = len(cams)
    side = torch.cuda.Stream()
    rng = np.random.default_rng(2)
    grads_in = [dict(color=torch.from_numpy(rng.normal(size=(3, c["H"], c["W"])).astype(np.float32)).cuda())
                for c in cams]

    def step(state):
        pre = R.preprocess_batched(plan, d["means3D"], d["log_scales"], d["quats"], d["opacities"], cams,
                                   out=state.get("pre"))
        state["pre"] = pre
        pl, rg, _ = R.bin_and_sort_batched(plan, pre["means2D"], pre["radii"], pre["depths"], cams,
                                           point_list=state["pl"], ranges=state.get("rg"), no_sync=True)
        state["rg"] = rg
        outs = R.render_forward_batched(plan, pre["means2D"], pre["conic_opacity"], d["colors"], pre["depths"], pl,
                                        pl.numel(), rg, cams, outs=state.get("outs"))
        state["outs"] = outs
        gr = R.render_backward_batched(plan, pre["means2D"], pre["conic_opacity"], d["colors"], pre["depths"], pl,
                                       pl.numel(), rg, cams, outs, grads_in, out=state.get("gr"))
        state["gr"] = gr
        return state

    with torch.cuda.stream(side):
        # eager run with a synchronising binning to size the point_list
        pre = R.preprocess_batched(plan, d["means3D"], d["log_scales"], d["quats"], d["opacities"], cams)
        _, _, K = R.bin_and_sort_batched(plan, pre["means2D"], pre["radii"], pre["depths"], cams)
        state = dict(pl=torch.empty(int(K * 1.2) + 64, dtype=torch.int32, device="cuda"))
        step(state)  # eager, grows every workspace
        side.synchronize()
        eager = {k: v.clone() for k, v in state["gr"].items()}
        eager_img = [o["color"].clone() for o in state["outs"]]
        R.graph_begin(plan)
        step(state)
        R.graph_end(plan)
        for _ in range(2):
            for o in state["outs"]:
                o["color"].zero_()
            state["gr"]["opacity"].zero_()
            R.graph_launch(plan)
            side.synchronize()
            for v in range(V):
                assert torch.equal(state["outs"][v]["color"], eager_img[v])
            for k in ("means2D", "conic", "colors"):
                assert rel_l2(state["gr"][k].cpu().numpy(), eager[k].cpu().numpy()) < 1e-5, k
    plan.check()
    plan.close()


def test_no_sync_binning_flags_overflow(R, batch):
    plan = R.Plan()
    cams = batch["cams"]
    m2, rd, dp = _stack(batch, "means2D"), _stack(batch, "radii"), _stack(batch, "depths")
    pl = torch.empty(100, dtype=torch.int32, device="cuda")  # far too small
    R.bin_and_sort_batched(plan, m2, rd, dp, cams, point_list=pl, no_sync=True)
    with pytest.raises(R.BgsError) as e:
        plan.check()
    assert e.value.code == -4 and "overflow" in str(e.value)
    plan.close()
