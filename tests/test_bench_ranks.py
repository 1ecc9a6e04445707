"""The multi-rank (replicas) path of bench.py on CPU: two gloo ranks agree on the maximum
of their timed regions, the whole-job value counts every rank's units, and the reference
arm runs on rank 0 only."""
import contextlib
import io
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, q):
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ms = bench.max_over_ranks(10.0 + 3.0 * rank, world, "cpu")
    dist.barrier()
    dist.destroy_process_group()
    q.put((rank, ms))


def test_two_gloo_ranks_take_the_maximum():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    got = dict(q.get(timeout=10) for _ in range(2))
    assert got == {0: 13.0, 1: 13.0}


def test_whole_job_value_counts_every_rank():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.whole_job_value(1e6, 1, 2.0) == pytest.approx(5e8)
    assert bench.whole_job_value(1e6, 4, 2.0) == pytest.approx(2e9)
    assert bench.max_over_ranks(7.5, 1, "cpu") == 7.5


def test_reference_arm_runs_on_rank_zero_only(monkeypatch):
    sys.path.insert(0, ROOT)
    import bench
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")
    monkeypatch.setattr(sys, "argv", ["bench.py", "--impl", "reference", "--gpus", "2", "--steps", "1",
                                      "--warmup", "0"])
    out = io.StringIO()
    with contextlib.redirect_stdout(out):
        bench.main()
    assert out.getvalue() == ""


def test_kernel_code_hash_ignores_comments_only(tmp_path, monkeypatch):
    """A profile capture stays valid across comment edits of its kernel's sources and is
    retired by any code edit (bench.kernel_code_hash)."""
    import bench
    csrc = tmp_path / "paper_2412_17378_gb300" / "csrc"
    csrc.mkdir(parents=True)
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    f = csrc / "k.cu"
    f.write_text('// kernel\n__global__ void k(int *p) { p[0] = 1; /* one */ }\nconst char *s = "a // b";\n')
    h0 = bench.kernel_code_hash(["k.cu"])
    f.write_text('// the kernel, reworded\n__global__ void k(int *p) {\n    p[0] = 1;  // one\n}\n'
                 'const char *s = "a // b";\n')
    assert bench.kernel_code_hash(["k.cu"]) == h0
    f.write_text('// kernel\n__global__ void k(int *p) { p[0] = 2; /* one */ }\nconst char *s = "a // b";\n')
    assert bench.kernel_code_hash(["k.cu"]) != h0
    f.write_text('// kernel\n__global__ void k(int *p) { p[0] = 1; /* one */ }\nconst char *s = "a // c";\n')
    assert bench.kernel_code_hash(["k.cu"]) != h0  # string literals are code


def test_reference_arm_json_line():
    """--impl reference (the FP64 oracle on the host cores) prints one line with the keys the
    ratio is computed from, its own e2e (no device copies) and a cpu_baseline of itself."""
    import json
    import subprocess
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--config", "cfg1", "--steps", "1",
                        "--warmup", "1"], cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.strip().startswith("{")]
    assert len(lines) == 1
    L = json.loads(lines[0])
    assert L["impl"] == "reference" and L["value"] > 0 and L["unit"] == "pairs/s" and L["higher_is_better"] is True
    assert L["cpu_baseline"]["kind"] == "oracle" and L["cpu_baseline"]["value"] == L["value"]
    assert L["e2e"] == {"value": L["value"], "unit": L["unit"], "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
