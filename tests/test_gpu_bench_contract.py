"""bench.py's JSON line on a GPU: one run of the smallest workload prints exactly one line with
every key its consumers read (metric, value, timing, roofline, CPU baseline, end-to-end,
kernel launches, clocks), with consistent values."""
import json
import os
import subprocess
import sys

import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_bench_json_line_contract():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    r = subprocess.run([sys.executable, "bench.py", "--config", "cfg1", "--steps", "3", "--warmup", "3",
                        "--cpu-seconds", "1"], cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.strip().startswith("{")]
    assert len(lines) == 1, r.stdout[-2000:]
    L = json.loads(lines[0])
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better", "scaling",
              "vs_baseline", "dtype", "data", "config", "roofline", "cpu_baseline", "e2e", "gpu_launches", "clocks"):
        assert k in L, k
    assert L["n_gpus"] == 1 and L["steps"] == 3 and L["warmup"] == 3 and L["higher_is_better"] is True
    assert L["value"] > 0 and L["ms_per_step"] > 0 and L["gpu_launches"] > 0
    assert L["unit"] == "pairs/s" and L["scaling"] == "weak" and "workload" in L["config"]
    roof = L["roofline"]
    for k in ("bound", "achieved", "peak", "unit", "frac", "traffic"):
        assert k in roof, k
    assert roof["bound"] == "alu" and abs(roof["frac"] - roof["achieved"] / roof["peak"]) < 1e-9
    cpu = L["cpu_baseline"]
    assert cpu["kind"] == "oracle" and cpu["value"] > 0 and cpu["cores"] >= 1 and cpu["sample"]
    e2e = L["e2e"]
    assert e2e["value"] > 0 and e2e["unit"] == L["unit"] and e2e["h2d_bytes_per_step"] > 0
    # the step's rendered images (3 x 256 x 256 floats) and its loss come back every step
    assert e2e["d2h_bytes_per_step"] == 3 * 256 * 256 * 4 + 4
    assert e2e["value"] < L["value"]  # copies are inside its timed region
    assert e2e["images_match_serial"] is True
    # the pipelined end-to-end loop computes what the serial one does
    assert e2e["serial"]["ms_per_step"] > 0 and e2e["loss_matches_serial"] is True and e2e["loss"] > 0
    clk = L["clocks"]
    assert clk["sm_mhz"] > 0 and clk["sm_max_mhz"] > 0 and isinstance(clk["reasons"], list)
    assert clk["samples"] >= clk["samples_in_timed_region"] >= 0


def test_bench_default_steps_cover_clock_samples():
    """Without --steps the timed region is sized to about a second of replays (at least 10
    steps), so the clock sampler records samples inside it."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    r = subprocess.run([sys.executable, "bench.py", "--config", "cfg1", "--warmup", "3", "--cpu-seconds", "1"],
                       cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.strip().startswith("{")]
    assert len(lines) == 1, r.stdout[-2000:]
    L = json.loads(lines[0])
    assert L["steps"] >= 10
    assert L["steps"] * L["ms_per_step"] >= 250.0  # about a second of replays, host waits included in the sizing
    clk = L["clocks"]
    if clk["samples"] > 0:
        assert clk["samples_in_timed_region"] >= 1
