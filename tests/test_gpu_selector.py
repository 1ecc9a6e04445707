"""The self-adaptive kernel selection of Sec. 4.4 (render mode "select"): balanced kernels
until a timing (every select_period forward calls, the first included) finds the static
pixel-wise forward faster, then the static kernels for good.  The images and gradients do
not depend on the choice."""
import numpy as np
import pytest

from helpers import oracle_render_inputs, rel_l2, scene, to_gpu

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def R():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2412_17378_gb300 import raster
    return raster


@pytest.mark.parametrize("name,scale", [("cfg1", 1.0), ("cfg2", 0.05)])
def test_selector_times_switches_once_and_keeps_results(R, name, scale):
    inp = oracle_render_inputs(scene(name, scale))
    W, H, tile = inp["W"], inp["H"], inp["tile"]
    g = to_gpu(inp)
    rng = np.random.default_rng(6)
    gC = torch.from_numpy(rng.normal(size=(3, H, W)).astype(np.float32)).cuda()

    def run(plan, mode):
        out = R.render_forward(plan, g["means2D"], g["conic_opacity"], g["colors"], g["depths"], g["point_list"],
                               g["K"], g["ranges"], W, H, tile, (0.0, 0.0, 0.0), mode)
        gr = R.render_backward(plan, g["means2D"], g["conic_opacity"], g["colors"], g["depths"], g["point_list"],
                               g["K"], g["ranges"], W, H, out["final_T"], out["n_contrib"], gC, None, None, tile,
                               (0.0, 0.0, 0.0), mode)
        torch.cuda.synchronize()
        plan.check()
        return out, gr

    ref_out, ref_gr = run(R.Plan(), "pixel")
    plan = R.Plan(select_period=2)
    history = []
    for it in range(7):
        out, gr = run(plan, "select")
        history.append(plan.selector())
        assert (out["color"] - ref_out["color"]).abs().max().item() < 1e-5
        assert torch.equal(out["n_contrib"], ref_out["n_contrib"])
        for k in ("means2D", "conic", "opacity", "colors"):
            assert rel_l2(gr[k].cpu().numpy(), ref_gr[k].cpu().numpy()) < 1e-5, (it, k)
    st = history[-1]
    assert st["calls"] == 7
    # timings at calls 0, 2, 4, 6 until the switch; none after it
    switch_at = next((i for i, h in enumerate(history) if h["switched"]), None)
    if switch_at is None:
        assert st["measurements"] == 4
        assert st["static_ms"] >= st["balanced_ms"] > 0
    else:
        assert switch_at % 2 == 0
        assert st["measurements"] == switch_at // 2 + 1
        assert history[switch_at]["static_ms"] < history[switch_at]["balanced_ms"]
        assert all(h["switched"] for h in history[switch_at:])  # irreversible
        assert all(h["measurements"] == st["measurements"] for h in history[switch_at:])
    plan.selector_reset()
    st = plan.selector()
    assert (st["switched"], st["calls"], st["measurements"]) == (False, 0, 0)
    plan.close()


def test_selector_is_single_view(R):
    from paper_2412_17378_gb300 import scenes
    plan = R.Plan()
    cams = scenes.arc_cameras([(64, 48), (80, 48)])
    n = 8
    z = torch.zeros
    m2, co, dp = z((2 * n, 2)).cuda(), z((2 * n, 4)).cuda(), z(2 * n).cuda()
    pl, rg = z(4, dtype=torch.int32).cuda(), z((12 + 15, 2), dtype=torch.int32).cuda()
    with pytest.raises(R.BgsError):
        R.render_forward_batched(plan, m2, co, z((n, 3)).cuda(), dp, pl, 0, rg, cams, mode="select")
    plan.close()


def test_plan_state_round_trips_through_json(R):
    """Checkpoint / resume: the knobs and the selector state survive a JSON round trip."""
    import json
    a = R.Plan(heavy_threshold=2048, pixel_rows=4, select_period=7, bin_block=4096)
    assert a._lib.bgs_plan_selector_restore(a.handle, 1, 1234, 3, 0.5, 0.4) == 0
    state = json.loads(json.dumps(a.state_dict()))
    b = R.Plan()
    b.load_state_dict(state)
    assert b.state_dict() == a.state_dict()
    assert b.selector()["switched"] and b.selector()["calls"] == 1234
    from paper_2412_17378_gb300._lib import check
    with pytest.raises(R.BgsError):  # more measurements than calls: refused
        check(b._lib.bgs_plan_selector_restore(b.handle, 0, 1, 5, 0.0, 0.0), "restore")
    a.close()
    b.close()
