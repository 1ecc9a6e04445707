"""Benchmark of the balanced splat render path on one GB300 (or N replicas).

A step is one pass of the whole hot path over one synthetic frame (every view of the
workload):
  a1 projection -> a2 binning + sort -> a3 work list -> a5 balanced forward
  -> L2 loss gradient (torch) -> a6 balanced backward,
enqueued without host synchronisation, captured once as a CUDA graph and replayed.
Default workload: the large stress configuration -- 4M Gaussians in three dense clusters
over a sparse background, one 3840x2160 view plus eight 1920x1080 views on an arc, forward
+ backward (the largest configuration that fits one GPU); ``--config cfg2`` selects the
imbalanced single view (1920x1080, 1M Gaussians, 80% in one cluster).

The metric is Gaussian-pixel pairs per second: pairs = (pixel, list entry) pairs the
sequential rule visits (sum of n_eval over the frame), divided by the step time.  The
JSON line also carries ms/frame, the plain pixel-wise 16x16 static-grid kernel on the
same inputs, the roofline of the dominant render kernel and the FP64 CPU oracle timed on
a bounded sample of the same frame.

  python bench.py [--gpus N --steps K --warmup W] [--config cfg2] [--impl reference]
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "fwd+bwd render ms/frame & Gaussian-pixel pairs/s vs pixel-wise kernel, 1 GB300"
WORKLOADS = {
    "cfg1": "single view 256x256, 10k Gaussians uniform in a box, fwd+bwd",
    "cfg2": "imbalanced single view 1920x1080, 1M Gaussians (80% clustered), fwd+bwd",
    "cfg3early": "training-stage sweep, early: 1280x720, 100k large low-opacity Gaussians, fwd+bwd",
    "cfg3late": "training-stage sweep, late: 1280x720, 3M small opaque Gaussians, fwd+bwd",
    "cfg4": "16 uneven views (4x640x360, 8x1280x720, 4x1920x1080) of 2M clustered Gaussians, fwd+bwd",
    "cfg5": "3840x2160 + 8x1920x1080 views of 4M Gaussians in 3 clusters, fwd+bwd",
    "heavy": "single view 1920x1080: 200k clustered Gaussians and a veil of 100k faint ones over ~35 tiles "
             "(lists of 2-8e4 entries walked to their ends), fwd+bwd",
}
DEFAULT_CONFIG = "cfg5"

# Algorithmic per-pair operation counts of the sequential rule (Algorithm 5 and its
# derivative), counted at source level for the formulation the kernels implement, as the
# minimum a kernel must issue (the dx terms of a pixel column -- dx, qa dx^2, qb dx -- are
# shared by the 4 pixels of a lane: 1 op per pair):
#  forward, every evaluated pair: shared dx terms (1), dy (1), power (2 FMA), o*G and the
#          0.99 clamp (2), the power <= 0 and alpha >= 1/255 tests (2) = 8 FP32-pipe ops
#          + 1 MUFU ex2; every accumulated pair: T' = T - T alpha (1 FMA), the T test, w,
#          4 FMA (colour, depth) = 7 (the accumulated alpha is 1 - T, written once per pixel);
#  backward, every pair before the last contributor: the forward's 8 + the n_contrib test
#          = 9, + 1 ex2 (recompute); every accumulated pair: 1-alpha, T/(1-alpha), w,
#          3 colour FMA, c . dL/dC (3), minus R . dL/dC (1), dL/dalpha (1), the R . dL/dC
#          update (1), clamp test, dL/dpower, its dy product and 3 sums = 18 FP32-pipe ops
#          + 1 MUFU rcp (dL/dopacity is the dL/dpower sum over o, once per record).
# (The warp reductions and atomics of the backward are aggregation overhead, not counted.)
FWD_EVAL_FP32, FWD_EVAL_MUFU, FWD_ACC_FP32 = 8, 1, 7
BWD_EVAL_FP32, BWD_EVAL_MUFU, BWD_ACC_FP32, BWD_ACC_MUFU = 9, 1, 18, 1
FP32_LANES_PER_SM_CLK = 128


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=None,
                    help="timed steps (default: enough graph replays for about 1 s, at least 10; 10 for the "
                         "reference arm and --quick)")
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--config", default=DEFAULT_CONFIG)
    ap.add_argument("--scale", type=float, default=1.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-tune", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=15.0, help="budget of the oracle sample")
    ap.add_argument("--mode", default="auto", choices=["auto", "pixel", "gaussian", "static"],
                    help="render mode of the timed steps")
    ap.add_argument("--knobs", default="",
                    help="plan knobs for the timed steps when not tuning, e.g. pixel_rows=4,heavy_threshold=2147483647")
    ap.add_argument("--selector-drift", type=int, default=0, metavar="STAGES",
                    help="run the Sec. 4.4 selector (mode 'select', a timing every stage) over STAGES scenes "
                         "drifting from config 3-early to 3-late and print its record as one JSON line")
    ap.add_argument("--full-lists", action="store_true",
                    help="bin complete per-tile lists (no truncation where every pixel of a tile has stopped)")
    ap.add_argument("--quick", action="store_true",
                    help="only the timed steps (no tuning, baselines, e2e or oracle): for profiler runs")
    return ap.parse_args()


def apply_knobs(plan, spec):
    """Sets plan knobs given as 'name=value,...' (the tuner's knob names)."""
    kw = {}
    for item in filter(None, spec.split(",")):
        k, v = item.split("=")
        kw[k.strip()] = int(v)
    if kw:
        plan.set(**kw)
    return kw


def max_over_ranks(ms_total: float, world: int, device) -> float:
    """The timed region's length as the job sees it: the maximum over the ranks (every
    rank ran the same number of steps; the slowest one bounds the job)."""
    if world <= 1:
        return ms_total
    import torch
    import torch.distributed as dist
    t = torch.tensor([ms_total], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_value(units_per_rank_step: float, world: int, ms_step: float) -> float:
    """Whole-job throughput: the units all ranks processed in one step over the step time
    (weak scaling: every rank renders its own copy of the workload)."""
    return units_per_rank_step * world / (ms_step / 1e3)


def dist_init(args):
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


class ClockSampler:
    """nvidia-smi clock / throttle-reason samples (every 50 ms) around the timed region; the
    summary keeps the samples whose host time falls inside the marked window."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int, period_ms: int = 50):
        self.gpu = gpu_index
        self.period = period_ms
        self.proc = None
        self.path = None
        self.window = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.f = open(self.path, "w")
            self.t0 = time.time()
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu=timestamp,{self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", str(self.period)], stdout=self.f,
                                         stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def mark(self, t_begin: float, t_end: float):
        """Host wall-clock bounds (time.time()) of the timed region."""
        self.window = (t_begin, t_end)

    @staticmethod
    def _stamp(text: str):
        import datetime
        try:
            return datetime.datetime.strptime(text.strip(), "%Y/%m/%d %H:%M:%S.%f").timestamp()
        except ValueError:
            return None

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.close()
        rows = []
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 10:
                continue
            try:
                rows.append((self._stamp(parts[0]), float(parts[2]), float(parts[3]),
                             {n for n, v in zip(names, parts[6:10]) if v.lower() == "active"}))
            except ValueError:
                continue
        os.unlink(self.path)
        inside = rows
        if self.window is not None:
            lo, hi = self.window
            inside = [r for r in rows if r[0] is not None and lo - 0.05 <= r[0] <= hi + 0.05]
        use = inside if inside else rows
        reasons = set().union(*[r[3] for r in use]) if use else set()
        return {"sm_mhz": float(np.median([r[1] for r in use])) if use else None,
                "sm_max_mhz": max(r[2] for r in use) if use else None, "reasons": sorted(reasons),
                "samples": len(rows), "samples_in_timed_region": len(inside), "period_ms": self.period}


def cpu_model() -> str:
    """The host CPU's model name (lscpu), for the oracle's timing line."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.strip().startswith("Model name"):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    return "unknown"


def tile_eval_histogram(outs, cams, tile=16):
    """Per-tile evaluated pairs (sum of n_eval over the tile's pixels), all views: summary
    statistics and a log2 histogram (bin k counts tiles with 2^k <= pairs < 2^(k+1); bin
    "0" the empty tiles)."""
    per = []
    for o, c in zip(outs, cams):
        ne = o["n_eval"].double()
        H, W = ne.shape
        ty, tx = (H + tile - 1) // tile, (W + tile - 1) // tile
        pad = ne.new_zeros(ty * tile, tx * tile)
        pad[:H, :W] = ne
        per.append(pad.reshape(ty, tile, tx, tile).sum(dim=(1, 3)).reshape(-1).cpu().numpy())
    per = np.concatenate(per)
    hist = {}
    nz = per[per > 0]
    hist["0"] = int((per == 0).sum())
    if nz.size:
        k = np.floor(np.log2(nz)).astype(int)
        for b in range(int(k.max()) + 1):
            hist[f"2^{b}"] = int((k == b).sum())
    return {"tiles": int(per.size), "max": float(per.max()), "mean": float(per.mean()),
            "p99": float(np.percentile(per, 99)), "max_over_mean": float(per.max() / max(per.mean(), 1e-9)),
            "log2_hist": hist}


PROFILED = {  # ncu summaries carrying the DRAM traffic of a dominant kernel, per workload and knobs
    "k_backward_balanced": ["profiles/k_backward_balanced_cfg5_4k+8x1080p_4M.md",
                            "profiles/k_backward_balanced_cfg2_1920x1080_1M.md"],
    "k_forward_balanced": ["profiles/k_forward_pixel_cfg5_4k+8x1080p_4M.md",
                           "profiles/k_forward_pixel_cfg2_1920x1080_1M.md"],
}


def time_enqueued(stream, fns, rounds=6, skip=2):
    """Median device time of each callable in fns: every round enqueues fns[0], fns[1], ...
    between CUDA events on `stream`, and the host synchronises only once all rounds are
    enqueued, so the host-side cost of a call overlaps the device work of the rounds before
    it instead of landing between its events.  The first `skip` rounds are not counted."""
    import torch
    ev = [[torch.cuda.Event(enable_timing=True) for _ in range(len(fns) + 1)] for _ in range(rounds)]
    for r in range(rounds):
        ev[r][0].record(stream)
        for j, f in enumerate(fns):
            f()
            ev[r][j + 1].record(stream)
    stream.synchronize()
    return [float(np.median([ev[r][j].elapsed_time(ev[r][j + 1]) for r in range(skip, rounds)]))
            for j in range(len(fns))]


def _strip_comments(src: str) -> str:
    """C/C++/CUDA source without its comments (string and character literals kept)."""
    out, i, n = [], 0, len(src)
    while i < n:
        c = src[i]
        if c in "\"'":
            j = i + 1
            while j < n and src[j] != c:
                j += 2 if src[j] == "\\" else 1
            out.append(src[i:j + 1])
            i = j + 1
        elif src.startswith("//", i):
            j = src.find("\n", i)
            i = n if j < 0 else j
        elif src.startswith("/*", i):
            j = src.find("*/", i + 2)
            i = n if j < 0 else j + 2
            out.append(" ")
        else:
            out.append(c)
            i += 1
    return "".join(out)


def kernel_code_hash(files) -> str:
    """First 16 hex digits of the SHA-256 of the named csrc files' code, comments removed and
    whitespace collapsed: an edit of a comment does not retire a profile capture, an edit of
    the code does."""
    import hashlib
    h = hashlib.sha256()
    for f in files:
        src = open(os.path.join(ROOT, "paper_2412_17378_gb300", "csrc", f)).read()
        h.update(" ".join(_strip_comments(src).split()).encode())
    return h.hexdigest()[:16]


def profiled_traffic(kernel: str, config: str, tuned: dict):
    """DRAM read + write bytes per launch of the kernel from a committed ncu summary taken on
    this workload (its `config:` line) with these knobs (its `knobs:` line), whose kernel
    source files are unchanged since (their code hash is recorded in the summary); else
    (None, reason)."""
    reason = "no capture for this kernel"
    for path in PROFILED.get(kernel, []):
        if not os.path.exists(os.path.join(ROOT, path)):
            continue
        fields = {}
        for line in open(os.path.join(ROOT, path)):
            if ":" in line and line.split(":")[0] in ("traffic_bytes_per_launch", "kernel_source_sha256_16", "config",
                                                      "knobs"):
                k, v = line.split(":", 1)
                fields[k] = v.strip()
        if "traffic_bytes_per_launch" not in fields or "config" not in fields:
            reason = "capture has no traffic line"
            continue
        knobs = dict(kv.split("=") for kv in fields.get("knobs", "").split(",") if "=" in kv)
        if fields["config"] != config or any(int(tuned.get(k, -1)) != int(v) for k, v in knobs.items()):
            reason = f"no capture for workload {config} with these knobs"
            continue
        digest, files = fields["kernel_source_sha256_16"].split(" ", 1)
        if kernel_code_hash(files.strip("()").split(", ")) != digest:
            reason = "kernel code changed since the capture"
            continue
        return int(fields["traffic_bytes_per_launch"]), path
    return None, reason


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        return json.load(open(p)), "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


# ----------------------------------------------------------------------------- oracle leg

_ORACLE_SETUP = {}
_ORACLE_SAMPLES = {}


def oracle_setup(scene):
    """Oracle projection of every view of the frame (done once, outside any timed region):
    per view the float32 render inputs (for the oracle's binning), the same values as float64
    arrays (the form its render takes them in, so that no timed call converts the whole
    Gaussian set), the depth order and the view's tile count."""
    key = id(scene)
    if key not in _ORACLE_SETUP:
        import oracle
        g = scene["gaussians"]
        views = []
        for cam in scene["cameras"]:
            pp = oracle.preprocess(g["means3D"], g["log_scales"], g["quats"], g["opacities"], cam)
            m2, co, dp = (pp[k].astype(np.float32) for k in ("means2D", "conic_opacity", "depth"))
            W, H = cam["W"], cam["H"]
            views.append(dict(m2=m2, co=co, dp=dp, radius=pp["radius"], W=W, H=H,
                              m2d=m2.astype(np.float64), cod=co.astype(np.float64), dpd=dp.astype(np.float64),
                              T=((W + 15) // 16) * ((H + 15) // 16), order=oracle.depth_order(pp["radius"], dp)))
            del pp
        _ORACLE_SETUP[key] = dict(views=views, colors=np.ascontiguousarray(g["colors"], np.float64))
    return _ORACLE_SETUP[key]


def oracle_sample_run(scene, budget_s: float, rng_seed: int = 0, threads: int = 0, n_tiles: int = 0):
    """Times the FP64 oracle's render forward + backward on a bounded sample of the frame's
    tiles (chosen uniformly at random over the tiles of all views), sized to about
    ``budget_s`` seconds of CPU work (or of ``n_tiles`` tiles when given), on all host cores
    (threads = 0) or the given number of threads.  Only the render forward + backward is
    timed; the sampled tiles' lists are built beforehand by the oracle's own binning
    (``bin_tiles_subset``).  Returns (pairs/s, cores, description, measured pairs, seconds,
    tiles sampled)."""
    import oracle
    if threads:
        all_threads = oracle.num_threads()
        oracle.set_threads(threads)
        try:
            return oracle_sample_run(scene, budget_s, rng_seed, n_tiles=n_tiles)
        finally:
            oracle.set_threads(all_threads)
    setup = oracle_setup(scene)
    views, cl = setup["views"], setup["colors"]
    base = np.cumsum([0] + [v["T"] for v in views])
    T = int(base[-1])
    order = np.random.default_rng(rng_seed).permutation(T)

    def sample(tiles_global):
        """Per view: the sampled tiles, their lists (the oracle's binning) and pixels; built
        once per sample and kept (untimed)."""
        ck = (id(scene), rng_seed, tiles_global.size)
        if ck not in _ORACLE_SAMPLES:
            per = []
            for vi, v in enumerate(views):
                sel = np.sort(tiles_global[(tiles_global >= base[vi]) & (tiles_global < base[vi + 1])] - base[vi])
                if sel.size == 0:
                    continue
                W, H = v["W"], v["H"]
                tx = (W + 15) // 16
                pl, rg = oracle.bin_tiles_subset(v["m2"], v["radius"], v["dp"], W, H, sel, order=v["order"])
                pix = []
                for t in sel:
                    x0, y0 = (t % tx) * 16, (t // tx) * 16
                    ys, xs = np.mgrid[y0:min(y0 + 16, H), x0:min(x0 + 16, W)]
                    pix.append((ys * W + xs).ravel())
                per.append((vi, sel, pl, rg, np.concatenate(pix)))
            _ORACLE_SAMPLES[ck] = per
        return _ORACLE_SAMPLES[ck]

    def run(tiles_global):
        pairs, dt = 0, 0.0
        for vi, sel, pl, rg, pix in sample(tiles_global):
            v = views[vi]
            W, H = v["W"], v["H"]
            t0 = time.perf_counter()
            out = oracle.render(v["m2d"], v["cod"], cl, v["dpd"], pl, rg, W, H, pixels=pix)
            gC = np.zeros((3, H, W))
            gC.reshape(3, -1)[:, pix] = out["color"]
            oracle.render_backward(v["m2d"], v["cod"], cl, v["dpd"], pl, rg, W, H, gC, tiles=sel.astype(np.int64))
            dt += time.perf_counter() - t0
            pairs += int(out["n_eval"].sum())
        return pairs, dt

    if n_tiles:
        n = min(T, n_tiles)
        pairs, dt = run(order[:n])
    else:
        n = 16
        pairs, dt = run(order[:n])
        while dt < budget_s / 4 and n < T:
            # grow by 4x at least, or straight to about half the budget at the rate measured
            n = min(T, max(4 * n, int(n * budget_s / (2.0 * max(dt, 1e-3)))))
            pairs, dt = run(order[:n])
    where = f"{len(views)} views" if len(views) > 1 else "the frame"
    desc = f"{n} random 16x16 tiles of {T} ({100.0 * n / T:.1f}% of {where}), render fwd+bwd"
    return pairs / dt, oracle.num_threads(), desc, pairs, dt, n


def reference_arm(args):
    rank, world, _ = dist_init(args)
    if rank != 0:
        return
    if args.steps is None:
        args.steps = 10
    from paper_2412_17378_gb300 import scenes
    scene = scenes.scene_config(args.config, args.scale)
    per_step = max(2.0, 60.0 / max(1, args.steps + args.warmup))
    # the first warm-up step sizes a random tile sample to about per_step seconds of oracle
    # work (its lists are built once, untimed); every step renders that sample forward and
    # backward
    n_tiles = 0
    for k in range(max(1, args.warmup)):
        n_tiles = oracle_sample_run(scene, per_step, n_tiles=n_tiles)[5]
    t_all, p_all = 0.0, 0
    rate = cores = desc = None
    for k in range(args.steps):
        rate, cores, desc, pairs, dt, _ = oracle_sample_run(scene, per_step, n_tiles=n_tiles)
        t_all += dt
        p_all += pairs
    value = p_all / t_all
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "pairs/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * t_all / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic (seeded; stands in for the paper's internal dataset)",
            "config": {"workload": WORKLOADS.get(args.config, args.config), "sample": desc},
            "cpu_baseline": {"value": value, "unit": "pairs/s", "cores": cores, "kind": "oracle", "sample": desc},
            "e2e": {"value": value, "unit": "pairs/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ----------------------------------------------------------------------------- GPU arm

def selector_drift(args):
    """The self-adaptive selection of Sec. 4.4 over a synthetic training drift: at every
    stage the selector times the balanced forward against the static pixel-wise forward
    (select_period = 1) until the static one wins, then keeps it.  Two balanced kernels
    are guarded: "combined" = the plan defaults (tiles with lists longer than 512 entries
    rendered Gaussian-wise, the paper's fine-grained combined kernel), and "tuned" = the
    knobs bgs_autotune_render picks on the first stage."""
    import torch
    from paper_2412_17378_gb300 import raster, scenes
    torch.cuda.set_device(0)
    plans = {"combined": raster.Plan(select_period=1), "tuned": raster.Plan(select_period=1)}
    rows = {k: [] for k in plans}
    tuned = None
    for k in range(args.selector_drift):
        frac = k / max(1, args.selector_drift - 1)
        sc = scenes.drift_scene(frac)
        g, cam = sc["gaussians"], sc["cameras"][0]
        W, H = cam["W"], cam["H"]
        d = {n: torch.from_numpy(v).cuda() for n, v in g.items()}
        for name, plan in plans.items():
            pre = raster.preprocess(plan, d["means3D"], d["log_scales"], d["quats"], d["opacities"], cam)
            pl, rg, K = raster.bin_and_sort(plan, pre["means2D"], pre["radii"], pre["depths"], W, H)
            if name == "tuned" and tuned is None:
                _, knobs = raster.autotune_render(plan, pre["means2D"], pre["conic_opacity"], d["colors"],
                                                  pre["depths"], pl, K, rg, [cam])
                tuned = {n: knobs[n] for n in ("pixel_rows", "heavy_threshold", "gw_pixels", "queue_chunk")}
            for m in ("auto", "static"):  # warm both kernels on this frame
                raster.render_forward(plan, pre["means2D"], pre["conic_opacity"], d["colors"], pre["depths"], pl, K,
                                      rg, W, H, mode=m)
            before = plan.selector()
            raster.render_forward(plan, pre["means2D"], pre["conic_opacity"], d["colors"], pre["depths"], pl, K, rg,
                                  W, H, mode="select")
            torch.cuda.synchronize()
            st = plan.selector()
            measured = st["measurements"] > before["measurements"]
            rows[name].append({"stage": k, "frac": round(frac, 3), "gaussians": int(g["means3D"].shape[0]),
                               "entries": int(K), "balanced_ms": st["balanced_ms"] if measured else None,
                               "static_ms": st["static_ms"] if measured else None, "switched": st["switched"]})
    out = {"rule": "Sec. 4.4: time the balanced forward against the static pixel-wise forward every "
                   "select_period forward calls; switch once, irreversibly", "tuned_knobs": tuned}
    for name, r in rows.items():
        out[name] = {"stages": r, "switched_at_stage": next((x["stage"] for x in r if x["switched"]), None)}
    print(json.dumps({"selector_drift": out}), flush=True)
    for plan in plans.values():
        plan.close()


def main():
    args = parse()
    if args.impl == "reference":
        return reference_arm(args)
    if args.selector_drift:
        return selector_drift(args)
    if args.mode == "static":
        raise SystemExit("--mode static: the static kernel is timed as the baseline of every full run")
    import torch
    rank, world, local = dist_init(args)
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    from paper_2412_17378_gb300 import scenes
    scene = scenes.scene_config(args.config, args.scale)
    main_views(args, scene, rank, world, local)
    if world > 1:
        torch.distributed.destroy_process_group()


def main_views(args, scene, rank, world, local):
    """One step = the whole path for every camera of the workload: projection of all views,
    binning without host synchronisation, one persistent forward launch, the L2 loss
    gradients and one persistent backward launch, captured once as a CUDA graph and
    replayed K times.  pairs = evaluated (pixel, entry) pairs summed over the views."""
    import torch
    from paper_2412_17378_gb300 import raster, scenes
    g, cams = scene["gaussians"], scene["cameras"]
    V = len(cams)
    dev = torch.device("cuda", local)
    host = {k: torch.from_numpy(v).pin_memory() for k, v in g.items()}
    d = {k: v.to(dev) for k, v in host.items()}
    seeds = [2] if V == 1 else [4 + v for v in range(V)]
    targets_h = [torch.from_numpy(scenes.target_image(sd, c["W"], c["H"])).pin_memory() for sd, c in zip(seeds, cams)]
    targets = [t.to(dev) for t in targets_h]
    N = d["means3D"].shape[0]
    plan = raster.Plan(device=local)
    # list truncation: on unless --full-lists; the tuner keeps whichever binning is faster
    opt = {"truncate": not args.full_lists}
    side = torch.cuda.Stream(device=dev)
    state = {}
    if args.quick:
        args.no_tune = args.no_cpu_baseline = True
    tuned = {}
    if args.knobs:  # fixed knobs from the first step on (profiler runs)
        tuned = dict(apply_knobs(plan, args.knobs), source="--knobs")

    def step(no_sync=True, mode=args.mode, before_forward=None, inp=None, oset=""):
        # inp: (device inputs, device targets) to read, the resident set by default; oset:
        # which set of image outputs (and their loss gradients) the step writes
        dd, tgs = inp if inp is not None else (d, targets)
        pre = raster.preprocess_batched(plan, dd["means3D"], dd["log_scales"], dd["quats"], dd["opacities"], cams,
                                        out=state.get("pre"))
        state["pre"] = pre
        pl, rg, K = raster.bin_and_sort_batched(plan, pre["means2D"], pre["radii"], pre["depths"], cams,
                                                point_list=state.get("pl"), ranges=state.get("rg"), no_sync=no_sync,
                                                conic_opacity=pre["conic_opacity"] if opt["truncate"] else None)
        state["pl"], state["rg"] = pl, rg
        ne = pl.numel() if no_sync else K
        if before_forward is not None:
            before_forward()
        outs = raster.render_forward_batched(plan, pre["means2D"], pre["conic_opacity"], dd["colors"], pre["depths"],
                                             pl, ne, rg, cams, mode=mode, outs=state.get("outs" + oset))
        state["outs" + oset] = outs
        if "gin" + oset not in state:
            state["gin" + oset] = [dict(color=torch.empty_like(o["color"])) for o in outs]
        gin = state["gin" + oset]
        for o, gi, t in zip(outs, gin, tgs):
            torch.sub(o["color"], t, out=gi["color"])
        gr = raster.render_backward_batched(plan, pre["means2D"], pre["conic_opacity"], dd["colors"], pre["depths"],
                                            pl, ne, rg, cams, outs, gin, mode=mode, out=state.get("gr"))
        state["gr"] = gr
        return K

    with torch.cuda.stream(side):
        K = step(no_sync=False)  # sizes the point_list and every workspace
        pre = state["pre"]
        # the complete lists' entry count (the truncation factor; untimed)
        _, _, K_full = raster.bin_and_sort_batched(plan, pre["means2D"], pre["radii"], pre["depths"], cams)
        state["pl"] = torch.empty(int(max(K, K_full) * 1.15) + 1024, dtype=torch.int32, device=dev)
        # ---- binning alone (a2: depth sort + per-tile lists), CUDA events, no host sync, with
        # and without list truncation; tuning keeps the faster ----
        bin_t = {}
        for tr in (True, False):
            bin_t[tr], = time_enqueued(side, [lambda: raster.bin_and_sort_batched(
                plan, pre["means2D"], pre["radii"], pre["depths"], cams, point_list=state["pl"], ranges=state["rg"],
                no_sync=True, conic_opacity=pre["conic_opacity"] if tr else None)])
        if not args.knobs and not args.no_tune and not args.full_lists and len(bin_t) == 2:
            opt["truncate"] = bin_t[True] <= bin_t[False]
        bin_ms = bin_t[opt["truncate"]]
        tuned["truncate_lists"] = opt["truncate"]
        K = step(no_sync=False)  # the chosen binning's lists and entry count
        # ---- knobs: autotuner (bgs_autotune_render), --knobs, or the plan defaults ----
        if not args.knobs and not args.no_tune:
            best_ms, knobs = raster.autotune_render(plan, pre["means2D"], pre["conic_opacity"], d["colors"],
                                                    pre["depths"], state["pl"], K, state["rg"], cams,
                                                    outs=state["outs"], grads_in=state["gin"], out=state["gr"])
            tuned.update({k: knobs[k] for k in ("pixel_rows", "heavy_threshold", "gw_pixels", "queue_chunk",
                                                "gw_segment")})
            tuned["render_ms"] = round(best_ms, 4)
        # ---- frame statistics (evaluated / contributing pairs, backward pairs) ----
        plan.reset_stats()
        l0 = plan.stats()["host_launches"]
        K = step(no_sync=False)
        st = plan.stats()
        eval_pairs, contrib_pairs = st["eval_pairs"], st["contrib_pairs"]
        launches_per_step = st["host_launches"] - l0
        bwd_pairs = int(sum(o["n_contrib"].sum().item() for o in state["outs"]))
        rgh = state["rg"].cpu().numpy().reshape(-1, 2).view(np.uint32)  # list positions reach past 2^31
        lens = rgh[:, 1].astype(np.int64) - rgh[:, 0].astype(np.int64)
        # per-tile evaluated pairs (the imbalance the balanced kernels address)
        outs_ne = raster.render_forward_batched(plan, pre["means2D"], pre["conic_opacity"], d["colors"],
                                                pre["depths"], state["pl"], K, state["rg"], cams, n_eval=True)
        tile_hist = tile_eval_histogram(outs_ne, cams)
        del outs_ne
        n_tiles = int(rgh.shape[0])
        # algorithmic bytes: read means2D, radii, depths once (16 B per record; + 16 B of conic
        # and opacity with list truncation), write the point list (4 B per kept entry) and the
        # ranges (8 B per tile)
        bin_bytes = (32 if opt["truncate"] else 16) * N * V + 4 * K + 8 * n_tiles
        # ---- render kernels alone (CUDA events around the persistent launches) ----
        plan.timing(True)
        for _ in range(3):
            step()
        side.synchronize()
        plan.kernel_ms()
        for _ in range(max(3, (args.steps or 10) // 2)):
            step()
        f_ms, nf, b_ms, nb = plan.kernel_ms()
        plan.timing(False)
        fwd_ms, bwd_ms = f_ms / max(nf, 1), b_ms / max(nb, 1)
        # ---- the timed region: graph replays of the whole step ----
        raster.graph_begin(plan)
        step()
        raster.graph_end(plan)
        for _ in range(args.warmup):
            raster.graph_launch(plan)
        side.synchronize()
        plan.check()
        if world > 1:
            torch.distributed.barrier()
        # nvidia-smi samples every 50 ms: ~1 s of untimed replays of the same graph right
        # before the timed region (the sampler's start-up and the GPU's clock ramp), then the
        # timed region, whose host-side window selects the samples that are reported
        clocks = ClockSampler(local)
        clocks.start()
        n_load, t_load = 0, time.perf_counter()
        if not args.quick:
            while time.perf_counter() - t_load < 1.0:
                for _ in range(4):
                    raster.graph_launch(plan)
                side.synchronize()
                n_load += 4
        if args.steps is None:
            # about 1 s of timed replays (the clock samples fall inside), at least 10; the same
            # count on every rank
            step_s = (time.perf_counter() - t_load) / n_load if n_load else 0.0
            k = max(10, int(math.ceil(1.0 / step_s))) if step_s > 0 else 10
            args.steps = int(max_over_ranks(float(k), world, dev))
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        side.synchronize()
        if world > 1:
            torch.distributed.barrier()
        t_wall0 = time.time()
        e0.record(side)
        for _ in range(args.steps):
            raster.graph_launch(plan)
        e1.record(side)
        side.synchronize()
        clocks.mark(t_wall0, time.time())
        ms_total = e0.elapsed_time(e1)
        clk = clocks.stop()
        clk["note"] = ("median over the samples taken inside the timed region (host wall-clock window); "
                       "~1 s of untimed replays of the same step precede it")
        plan.check()
        ms_total = max_over_ranks(ms_total, world, dev)
        ms_step = ms_total / args.steps
        value = whole_job_value(eval_pairs, world, ms_step)
        if args.quick:
            if rank == 0:
                print(json.dumps({"metric": METRIC, "value": value, "unit": "pairs/s", "ms_per_step": ms_step,
                                  "render_ms_per_step": {"forward": fwd_ms, "backward": bwd_ms},
                                  "tuned": tuned, "note": "--quick profiling run"}), flush=True)
            plan.close()
            return
        # ---- end to end: inputs from pinned host memory, images and loss read back, every step ----
        # One captured graph per step (torch.cuda.graph, whose private memory pool keeps the
        # loss reduction's workspace alive for the replays).  Every step copies its inputs in
        # from pinned host memory and its rendered images (every view's colour planes) and
        # its loss out to pinned host memory.
        h2d = sum(v.numel() * v.element_size() for v in host.values()) + sum(
            t.numel() * t.element_size() for t in targets_h)
        img_bytes = sum(3 * c["W"] * c["H"] * 4 for c in cams)
        d2h = img_bytes + 4
        copy_s = torch.cuda.Stream(device=dev)
        copy_out = torch.cuda.Stream(device=dev)  # the pipelined steps' image read-back
        imgs_h = [[torch.empty((3, c["H"], c["W"]), pin_memory=True) for c in cams] for _ in range(2)]
        loss_h = torch.empty(1, pin_memory=True)
        loss_hp = torch.empty(2, pin_memory=True)  # the pipelined steps' losses, by step parity

        def loss_to_host(dst, oset=""):
            loss = sum((gi["color"] * gi["color"]).sum() for gi in state["gin" + oset]) * 0.5
            dst.copy_(loss.reshape(1), non_blocking=True)

        def images_to_host(dst, oset=""):
            for h, o in zip(dst, state["outs" + oset]):
                h.copy_(o["color"], non_blocking=True)

        # (1) serial: a step copies its own inputs, computes from them, then copies its images
        # and loss out; the host waits for them before launching the next step
        ev_fork, ev_join = torch.cuda.Event(), torch.cuda.Event()

        def serial_body(i):
            ev_fork.record(side)
            copy_s.wait_event(ev_fork)
            with torch.cuda.stream(copy_s):
                d["colors"].copy_(host["colors"], non_blocking=True)
                for t, th in zip(targets, targets_h):
                    t.copy_(th, non_blocking=True)
                ev_join.record(copy_s)
            for k in host:
                if k != "colors":
                    d[k].copy_(host[k], non_blocking=True)
            step(before_forward=lambda: side.wait_event(ev_join))
            images_to_host(imgs_h[0])
            loss_to_host(loss_h)

        # (2) pipelined, as a prefetching loader runs: two device input sets and two image
        # output sets; step i computes from input set i % 2 (filled while step i - 1 ran) into
        # output set i % 2, while a second stream copies step i + 1's inputs into the other
        # input set and a third copies step i - 1's images (the other output set) to the host
        # (the two directions at once).  A set is overwritten only after the step that read it
        # has ended (the steps run in order on one stream, and a step's graph ends after its
        # copies).
        bufs = [(d, targets), ({k: torch.empty_like(v) for k, v in d.items()}, [torch.empty_like(t) for t in targets])]
        osets = ["", "_b"]
        step(oset="_b")  # allocates the second output set
        side.synchronize()
        pev = [(torch.cuda.Event(), torch.cuda.Event(), torch.cuda.Event()) for _ in range(2)]

        def pipelined_body(i):
            k = i % 2
            ev_f, ev_j, ev_o = pev[k]
            ev_f.record(side)
            copy_s.wait_event(ev_f)
            copy_out.wait_event(ev_f)
            with torch.cuda.stream(copy_s):
                nd, nt = bufs[1 - k]
                for key in host:
                    nd[key].copy_(host[key], non_blocking=True)
                for t, th in zip(nt, targets_h):
                    t.copy_(th, non_blocking=True)
                ev_j.record(copy_s)
            with torch.cuda.stream(copy_out):
                images_to_host(imgs_h[1 - k], osets[1 - k])  # the previous step's images
                ev_o.record(copy_out)
            step(inp=bufs[k], oset=osets[k])
            loss_to_host(loss_hp[k:k + 1], osets[k])
            side.wait_event(ev_j)
            side.wait_event(ev_o)

        def capture(body, n):
            """n CUDA graphs of body(0..n-1) (torch.cuda.graph: its private memory pool keeps
            the loss reduction's workspace alive for the replays); None if capture fails."""
            try:
                for i in range(2):
                    body(i)
                side.synchronize()
                graphs = []
                for i in range(n):
                    g = torch.cuda.CUDAGraph()
                    with torch.cuda.graph(g, stream=side, capture_error_mode="thread_local"):
                        body(i)
                    graphs.append(g)
                side.synchronize()
                return graphs, None
            except Exception as exc:  # capture refused: time the same body eagerly
                side.synchronize()
                return None, f"{type(exc).__name__}: {exc}"[:200]

        def run_e2e(graphs, body, lag):
            """ms per step over the timed steps and the last loss.  lag 0: the host waits for
            each step and reads its loss before launching the next; lag 1: it launches step i,
            then waits for step i - 1 and reads that step's loss (one step in flight, every
            loss read inside the timed region); the last step's images are copied out after
            it, inside the timed region."""
            done = [torch.cuda.Event(), torch.cuda.Event()]

            def launch(i):
                if graphs is not None:
                    graphs[i % len(graphs)].replay()
                else:
                    body(i)
                done[i % 2].record(side)

            def read(i):
                done[i % 2].synchronize()
                return float(loss_hp[i % 2]) if lag else float(loss_h[0])

            def run(n):
                last = None
                for i in range(n):
                    launch(i)
                    if not lag:
                        last = read(i)
                    elif i > 0:
                        last = read(i - 1)
                if lag:
                    last = read(n - 1)
                    with torch.cuda.stream(side):
                        images_to_host(imgs_h[(n - 1) % 2], osets[(n - 1) % 2])
                    side.synchronize()
                return last

            run(4)  # an even count keeps the pipelined input sets in phase
            side.synchronize()
            t0 = time.perf_counter()
            last = run(args.steps)
            return max_over_ranks(1e3 * (time.perf_counter() - t0), world, dev) / args.steps, last

        g_serial, err_serial = capture(serial_body, 1)
        serial_ms, loss_serial = run_e2e(g_serial, serial_body, 0)
        img_serial = imgs_h[0][0][:, ::97, ::89].clone()
        g_pipe, err_pipe = capture(pipelined_body, 2)
        e2e_ms, loss_pipe = run_e2e(g_pipe, pipelined_body, 1)
        img_pipe = imgs_h[(args.steps - 1) % 2][0][:, ::97, ::89].clone()
        del g_serial, g_pipe
        e2e_how = ("two CUDA graphs alternating over two device input sets and two image output sets: each step "
                   "copies the next step's inputs in (pinned host memory, second stream) and the previous step's "
                   "images out (third stream) while it computes, then copies its loss out; the host reads step i's loss after "
                   "launching step i + 1" if err_pipe is None else "eager, pipelined: " + err_pipe)
        serial_how = ("one CUDA graph per step: H2D copies (colours and targets on a second stream, overlapping "
                      "projection and binning), the step, the D2H copies of its images and loss, host wait"
                      if err_serial is None else "eager: " + err_serial)
        loss_match = abs(loss_pipe - loss_serial) <= 1e-6 * max(1.0, abs(loss_serial))
        images_match = bool(torch.equal(img_serial, img_pipe))
        # ---- projection (a1) and its backward alone, CUDA events ----
        gr = state["gr"]
        proj_ms = tuple(time_enqueued(side, [
            lambda: raster.preprocess_batched(plan, d["means3D"], d["log_scales"], d["quats"], d["opacities"], cams,
                                              out=state["pre"]),
            lambda: raster.preprocess_backward_batched(plan, d["means3D"], d["log_scales"], d["quats"], cams,
                                                       pre["radii"], gr["means2D"], gr["conic"], gr.get("depths"))]))
        # algorithmic bytes: forward reads 44 B per Gaussian and writes 36 B per record;
        # backward reads 40 B per Gaussian + 28 B per record and writes 40 B per Gaussian
        proj_bytes = (44 * N + 36 * N * V, 80 * N + 28 * N * V)
        # ---- view-dependent colour from degree-3 spherical harmonics (Sec. 2.1) alone ----
        gen = torch.Generator(device=dev)
        gen.manual_seed(17)
        sh_coef = 0.2 * torch.randn((N, 16, 3), device=dev, generator=gen)
        g_rgb = torch.randn((V * N, 3), device=dev, generator=gen)
        rgb_sh = torch.empty((V * N, 3), device=dev)
        sh_ms = tuple(time_enqueued(side, [
            lambda: raster.sh_to_rgb(plan, sh_coef, d["means3D"], cams, 3, out=rgb_sh),
            lambda: raster.sh_to_rgb_backward(plan, sh_coef, d["means3D"], cams, 3, g_rgb)]))
        # algorithmic bytes: forward reads 192 B of coefficients + 12 B of mean per Gaussian and
        # writes 12 B per record; backward reads 204 B per Gaussian + 12 B per record and
        # writes 192 + 12 B per Gaussian
        sh_bytes = (204 * N + 12 * N * V, 408 * N + 12 * N * V)
        # ---- plain pixel-wise 16x16 static grid on the same inputs ----
        # (single-view kernel: a view at a time, each with its own binning; render kernels
        # only, summed over the views)
        sf = sb = 0.0
        for v, c in enumerate(cams):
            W, H = c["W"], c["H"]
            sl = slice(v * N, (v + 1) * N)
            m2, co, dp = pre["means2D"][sl], pre["conic_opacity"][sl], pre["depths"][sl]
            if V == 1:
                pl, rg, Kv = state["pl"], state["rg"], K
            else:
                pl, rg, Kv = raster.bin_and_sort(plan, m2, pre["radii"][sl], dp, W, H,
                                                 conic_opacity=co if opt["truncate"] else None)

            def static_pass():
                fw = raster.render_forward(plan, m2, co, d["colors"], dp, pl, Kv, rg, W, H, (16, 16),
                                           (0.0, 0.0, 0.0), "static")
                raster.render_backward(plan, m2, co, d["colors"], dp, pl, Kv, rg, W, H, fw["final_T"],
                                       fw["n_contrib"], state["gin"][v]["color"], None, None, (16, 16),
                                       (0.0, 0.0, 0.0), "static")

            plan.timing(True)
            static_pass()
            side.synchronize()
            plan.kernel_ms()
            reps = max(2, args.steps // 2) if V == 1 else 2
            for _ in range(reps):
                static_pass()
            sf_ms, snf, sb_ms, snb = plan.kernel_ms()
            plan.timing(False)
            sf += sf_ms / max(snf, 1)
            sb += sb_ms / max(snb, 1)
            del pl, rg
        static = {"forward_ms": sf, "backward_ms": sb, "total_ms": sf + sb,
                  "pairs_per_s_render": eval_pairs / ((sf + sb) / 1e3),
                  "speedup_render": (sf + sb) / (fwd_ms + bwd_ms)}
    fp32_rate, ex2_rate = raster.probe_pipe_rates(plan)
    dom = "forward" if fwd_ms >= bwd_ms else "backward"
    roof = roofline_obj(dom, eval_pairs, contrib_pairs, bwd_pairs, fwd_ms, bwd_ms, plan.num_sms, fp32_rate, ex2_rate,
                        clk.get("sm_mhz"))
    roof["traffic"], roof["traffic_source"] = profiled_traffic(
        roof["kernel"], args.config if args.scale == 1.0 else f"{args.config}@{args.scale}", tuned)
    if roof["traffic"] is not None:
        roof["traffic_unit"] = "bytes per launch (DRAM read + write, ncu)"
    # ---- FP64 CPU oracle on a bounded sample of every view (rank 0, one GPU) ----
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        rate, cores, desc, _, _, _ = oracle_sample_run(scene, args.cpu_seconds)
        rate1, _, desc1, _, _, _ = oracle_sample_run(scene, 2.0, threads=1)
        cpu = {"value": rate, "unit": "pairs/s", "cores": cores, "kind": "oracle", "sample": desc,
               "cpu_model": cpu_model(),
               "single_thread": {"value": rate1, "unit": "pairs/s", "cores": 1, "sample": desc1}}
    peaks, _ = load_peaks()
    hbm = float(peaks.get("hbm_gbs", 6800.0))
    binning = {"ms": bin_ms, "algorithmic_bytes": int(bin_bytes), "GB_s": bin_bytes / (bin_ms / 1e3) / 1e9,
               "hbm_peak_GB_s": hbm, "frac_of_hbm": bin_bytes / (bin_ms / 1e3) / 1e9 / hbm,
               "entries_kept": int(K), "entries_full_lists": int(K_full),
               "truncated": bool(opt["truncate"]),
               "ms_by_mode": {("truncated" if k else "full_lists"): v for k, v in bin_t.items()},
               "note": "depth sort + counting-sort binning; each tile's list cut after the depth block where "
                       "every pixel of the tile is certified to have stopped (entries_kept of entries_full_lists "
                       "written); algorithmic bytes = 32 B per projected record read (16 without truncation) + "
                       "4 B per kept entry + 8 B per tile written"}
    projection = {"forward_ms": proj_ms[0], "backward_ms": proj_ms[1],
                  "forward_GB_s": proj_bytes[0] / (proj_ms[0] / 1e3) / 1e9,
                  "backward_GB_s": proj_bytes[1] / (proj_ms[1] / 1e3) / 1e9, "hbm_peak_GB_s": hbm,
                  "note": "a1 projection and its backward (chain rule to means3D, log_scales, quats); "
                          "algorithmic bytes: forward 44 B per Gaussian + 36 B per record, backward 80 B per "
                          "Gaussian + 28 B per record"}
    sh_row = {"degree": 3, "forward_ms": sh_ms[0], "backward_ms": sh_ms[1],
              "forward_GB_s": sh_bytes[0] / (sh_ms[0] / 1e3) / 1e9,
              "backward_GB_s": sh_bytes[1] / (sh_ms[1] / 1e3) / 1e9, "hbm_peak_GB_s": hbm,
              "frac_of_hbm": [sh_bytes[0] / (sh_ms[0] / 1e3) / 1e9 / hbm, sh_bytes[1] / (sh_ms[1] / 1e3) / 1e9 / hbm],
              "note": "view-dependent colour of every record from 16 x 3 coefficients per Gaussian (seeded "
                      "synthetic) and its backward; algorithmic bytes: forward 204 B per Gaussian + 12 B per "
                      "record, backward 408 B per Gaussian + 12 B per record"}
    sizes = sorted(set(f"{c['W']}x{c['H']}" for c in cams))
    config = {"workload": WORKLOADS.get(args.config, f"{V} views ({', '.join(sizes)}) of {N} Gaussians"),
              "gaussians": N, "views": V, "image": sizes[0] if V == 1 else sizes, "tile": "16x16",
              "step": "projection, binning, forward, L2 loss gradient, backward; one CUDA graph replay",
              "l2": "working set per step > L2 (point list and tile histogram), no flush",
              "parallelism": "replicas" if world > 1 else "single GPU", "tuned": tuned}
    line = {
        "metric": METRIC, "value": value, "unit": "pairs/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32",
        "data": "synthetic (seeded; stands in for the paper's internal dataset)",
        "config": config,
        "ms_per_frame": ms_step / V,
        "render_ms_per_step": {"forward": fwd_ms, "backward": bwd_ms, "total": fwd_ms + bwd_ms},
        "pixelwise_static": static,
        "frame": {"eval_pairs": eval_pairs, "contrib_pairs": contrib_pairs, "bwd_pairs": bwd_pairs, "entries": K,
                  "tile_list_max": int(lens.max()), "tile_list_mean": float(lens.mean()),
                  "tile_list_p99": float(np.percentile(lens, 99)), "tile_eval_pairs": tile_hist},
        "binning": binning,
        "projection": projection,
        "spherical_harmonics": sh_row,
        "roofline": roof,
        "cpu_baseline": cpu,
        "e2e": {"value": whole_job_value(eval_pairs, world, e2e_ms), "unit": "pairs/s", "h2d_bytes_per_step": int(h2d),
                "d2h_bytes_per_step": int(d2h), "ms_per_step": e2e_ms, "how": e2e_how,
                "serial": {"value": whole_job_value(eval_pairs, world, serial_ms), "ms_per_step": serial_ms,
                           "how": serial_how},
                "loss": loss_pipe, "loss_matches_serial": bool(loss_match), "images_match_serial": images_match,
                "d2h": "every view's rendered colour planes + the loss"},
        "gpu_launches": int(launches_per_step * args.steps), "gpu_launches_per_step": int(launches_per_step),
        "gpu_launches_note": "libbgs kernels per graph replay, not counting CUB sort/scan kernels",
        "clocks": clk,
    }
    if rank == 0:
        print(json.dumps(line), flush=True)
    plan.close()


def roofline_obj(dom, eval_pairs, contrib_pairs, bwd_pairs, fwd_ms, bwd_ms, sms, fp32_rate, ex2_rate, clk_meas_mhz):
    """Roofline of the dominant render kernel (see the module docstring for the op counts)."""
    peaks, peak_src = load_peaks()
    clk_peak = float(peaks.get("sm_max_mhz", 2070.0)) * 1e6

    def t_min(fp32_ops, mufu_ops, clk):
        return max(fp32_ops / (sms * FP32_LANES_PER_SM_CLK * clk), mufu_ops / (sms * ex2_rate * clk))

    fwd_ops = (FWD_EVAL_FP32 * eval_pairs + FWD_ACC_FP32 * contrib_pairs, FWD_EVAL_MUFU * eval_pairs)
    bwd_ops = (BWD_EVAL_FP32 * bwd_pairs + BWD_ACC_FP32 * contrib_pairs,
               BWD_EVAL_MUFU * bwd_pairs + BWD_ACC_MUFU * contrib_pairs)
    ops, dur = (fwd_ops, fwd_ms) if dom == "forward" else (bwd_ops, bwd_ms)
    achieved = eval_pairs / (dur / 1e3)
    peak = eval_pairs / t_min(*ops, clk_peak)
    clk_meas = (clk_meas_mhz or 0) * 1e6
    return {"bound": "alu", "kernel": f"k_{dom}_balanced", "achieved": achieved / 1e9, "peak": peak / 1e9,
            "unit": "Gpair/s", "frac": achieved / peak, "traffic": None,
            "model": "max(FP32-pipe ops / (SMs*128*clk), MUFU ops / (SMs*ex2_rate*clk)) at the max SM clock",
            "peak_source": f"derived from unit counts; SM clock {clk_peak/1e6:.0f} MHz ({peak_src}); "
                           f"probed ex2 {ex2_rate:.1f}/SM/clk, fp32 {fp32_rate:.1f}/SM/clk",
            "frac_at_measured_clock": (achieved / (eval_pairs / t_min(*ops, clk_meas))) if clk_meas else None}



if __name__ == "__main__":
    main()
