"""Host logic of bench.py that shapes the reported numbers, on CPU: the roofline arithmetic
of the render kernels (the op-count model against closed forms worked by hand), which ncu
captures may supply the `traffic` figure, the knob parser and the per-tile evaluated-pair
histogram."""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)
bench = pytest.importorskip("bench")


@pytest.fixture
def peaks_1ghz(monkeypatch):
    """A 1000 MHz maximum SM clock, whatever MEASURED_PEAKS.json holds."""
    monkeypatch.setattr(bench, "load_peaks", lambda: ({"sm_max_mhz": 1000.0}, "test"))


def test_roofline_backward_fp32_bound(peaks_1ghz):
    # 100 SMs at 1 GHz, 128 FP32 lanes, ex2 at 32 / SM / clock.  Backward: 9 FP32 ops + 1 ex2
    # per visited pair (1e9), 18 + 1 rcp per accumulated pair (1e8):
    #   FP32: (9e9 + 1.8e9) / (100 * 128 * 1e9 / s) = 0.84375 ms;  MUFU: 1.1e9 / (100 * 32 * 1e9 / s) = 0.34375 ms
    # so the bound is 0.84375 ms for 1e9 evaluated pairs, and a 1 ms launch reaches 0.84375 of it.
    r = bench.roofline_obj("backward", 1e9, 1e8, 1e9, 5.0, 1.0, 100, 128.0, 32.0, None)
    assert r["kernel"] == "k_backward_balanced" and r["bound"] == "alu" and r["unit"] == "Gpair/s"
    assert r["achieved"] == pytest.approx(1000.0)         # 1e9 pairs in 1 ms
    assert r["peak"] == pytest.approx(1000.0 / 0.84375)
    assert r["frac"] == pytest.approx(0.84375)
    assert r["frac"] == pytest.approx(r["achieved"] / r["peak"])
    assert r["frac_at_measured_clock"] is None


def test_roofline_backward_mufu_bound_and_measured_clock(peaks_1ghz):
    # ex2 at 8 / SM / clock: MUFU 1.1e9 / (100 * 8 * 1e9 / s) = 1.375 ms > FP32 0.84375 ms
    r = bench.roofline_obj("backward", 1e9, 1e8, 1e9, 5.0, 1.0, 100, 128.0, 8.0, 500.0)
    assert r["frac"] == pytest.approx(1.375)
    # at a 500 MHz measured clock the same launch is twice as close to that clock's bound
    assert r["frac_at_measured_clock"] == pytest.approx(2 * 1.375)


def test_roofline_forward_and_duration_scaling(peaks_1ghz):
    # forward: 8 FP32 + 1 ex2 per evaluated pair, + 7 per accumulated pair:
    #   FP32 (8e9 + 7e8) / 1.28e13 per s = 0.6796875 ms;  MUFU 1e9 / 3.2e12 per s = 0.3125 ms
    r = bench.roofline_obj("forward", 1e9, 1e8, 1e9, 1.0, 5.0, 100, 128.0, 32.0, None)
    assert r["kernel"] == "k_forward_balanced"
    assert r["frac"] == pytest.approx(0.6796875)
    r2 = bench.roofline_obj("forward", 1e9, 1e8, 1e9, 2.0, 5.0, 100, 128.0, 32.0, None)
    assert r2["frac"] == pytest.approx(r["frac"] / 2) and r2["peak"] == pytest.approx(r["peak"])


def _summary(path, digest, files, traffic=123456, config="cfg2", knobs="pixel_rows=4,heavy_threshold=2147483647"):
    path.write_text(f"# test capture\n\nconfig: {config}\nknobs: {knobs}\ntraffic_bytes_per_launch: {traffic}\n"
                    f"kernel_source_sha256_16: {digest} ({', '.join(files)})\n")


TUNED = {"pixel_rows": 4, "heavy_threshold": 2 ** 31 - 1}


def test_profiled_traffic_reads_a_current_capture(tmp_path, monkeypatch):
    files = ["render_bwd.cu", "bgs_internal.cuh"]
    p = tmp_path / "cap.md"
    _summary(p, bench.kernel_code_hash(files), files)
    monkeypatch.setitem(bench.PROFILED, "k_test", [str(p)])
    assert bench.profiled_traffic("k_test", "cfg2", TUNED) == (123456, str(p))
    # several captures: the one of the run's workload is used
    q = tmp_path / "cap5.md"
    _summary(q, bench.kernel_code_hash(files), files, traffic=777, config="cfg5")
    monkeypatch.setitem(bench.PROFILED, "k_test", [str(p), str(q)])
    assert bench.profiled_traffic("k_test", "cfg5", TUNED) == (777, str(q))
    assert bench.profiled_traffic("k_test", "cfg5@0.25", TUNED)[0] is None  # a reduced scale is another workload


def test_profiled_traffic_rejects_stale_or_foreign_captures(tmp_path, monkeypatch):
    files = ["render_bwd.cu", "bgs_internal.cuh"]
    p = tmp_path / "cap.md"
    _summary(p, "0" * 16, files)  # recorded against other kernel sources
    monkeypatch.setitem(bench.PROFILED, "k_test", [str(p)])
    t, why = bench.profiled_traffic("k_test", "cfg2", TUNED)
    assert t is None and "changed" in why
    _summary(p, bench.kernel_code_hash(files), files)
    assert bench.profiled_traffic("k_test", "cfg4", TUNED)[0] is None           # another workload
    assert bench.profiled_traffic("k_test", "cfg2", dict(TUNED, pixel_rows=2))[0] is None  # other knobs
    assert bench.profiled_traffic("k_test", "cfg2", dict(TUNED, heavy_threshold=512))[0] is None
    assert bench.profiled_traffic("k_unknown", "cfg2", TUNED)[0] is None


def test_apply_knobs_parses_the_profiler_command_line():
    seen = {}

    class FakePlan:
        def set(self, **kw):
            seen.update(kw)

    kw = bench.apply_knobs(FakePlan(), "pixel_rows=4,heavy_threshold=2147483647,")
    assert kw == seen == {"pixel_rows": 4, "heavy_threshold": 2147483647}
    assert bench.apply_knobs(FakePlan(), "") == {}


def test_tile_eval_histogram_on_ragged_views():
    """Per-tile sums of n_eval over 16x16 tiles of two views with ragged edges, against a brute
    force over pixel coordinates; the log2 bins count every nonempty tile once."""
    torch = pytest.importorskip("torch")
    import numpy as np
    rng = np.random.default_rng(5)
    shapes = [(35, 20), (16, 50)]  # (H, W): 3x2 and 1x4 tiles
    outs, cams, expect = [], [], []
    for H, W in shapes:
        ne = rng.integers(0, 300, (H, W))
        ne[:16, :16] = 0  # one empty tile per view
        outs.append({"n_eval": torch.from_numpy(ne.astype(np.int32))})
        cams.append({"W": W, "H": H})
        for ty in range((H + 15) // 16):
            for tx in range((W + 15) // 16):
                expect.append(sum(int(ne[y, x]) for y in range(ty * 16, min(H, ty * 16 + 16))
                                  for x in range(tx * 16, min(W, tx * 16 + 16))))
    expect = np.array(expect, dtype=np.float64)
    h = bench.tile_eval_histogram(outs, cams)
    assert h["tiles"] == expect.size == 10
    assert h["max"] == expect.max() and h["mean"] == pytest.approx(expect.mean())
    assert h["max_over_mean"] == pytest.approx(expect.max() / expect.mean())
    assert h["log2_hist"]["0"] == 2
    assert sum(h["log2_hist"].values()) == expect.size
    for b, n in h["log2_hist"].items():
        if b != "0":
            k = int(b[2:])
            assert n == int(((expect >= 2 ** k) & (expect < 2 ** (k + 1))).sum())


def test_oracle_sample_counts_the_full_render_pairs_of_its_tiles():
    """The CPU baseline's sample (bench.oracle_sample_run): the evaluated pairs it times on a
    fixed set of tiles, from the oracle's own binning of those tiles only, equal the full-frame
    oracle render's n_eval summed over the same tiles; a second call reuses the kept sample."""
    import numpy as np
    import oracle
    from paper_2412_17378_gb300 import scenes
    sc = scenes.scene_config("cfg1", 1.0)
    n = 24
    r1 = bench.oracle_sample_run(sc, 0.5, n_tiles=n)
    r2 = bench.oracle_sample_run(sc, 0.5, n_tiles=n)
    assert r1[5] == r2[5] == n and r1[3] == r2[3] > 0 and r1[4] > 0
    assert sum(1 for k in bench._ORACLE_SAMPLES if k[0] == id(sc)) == 1
    # the same tiles of the full frame
    g, cam = sc["gaussians"], sc["cameras"][0]
    W, H = cam["W"], cam["H"]
    pp = oracle.preprocess(g["means3D"], g["log_scales"], g["quats"], g["opacities"], cam)
    m2, co, dp = (pp[k].astype(np.float32) for k in ("means2D", "conic_opacity", "depth"))
    pl, rg = oracle.bin_tiles(m2, pp["radius"], dp, W, H)
    full = oracle.render(m2, co, g["colors"], dp, pl, rg, W, H)
    tx, T = (W + 15) // 16, ((W + 15) // 16) * ((H + 15) // 16)
    tiles = np.random.default_rng(0).permutation(T)[:n]
    ne = full["n_eval"].reshape(H, W)
    expect = sum(int(ne[(t // tx) * 16:(t // tx) * 16 + 16, (t % tx) * 16:(t % tx) * 16 + 16].sum()) for t in tiles)
    assert r1[3] == expect
