"""View sharding of a multi-view training step (the paper's multi-GPU future work, Sec. 5.3)
on CPU: the view partition, and the one exchange step -- a SUM all-reduce of per-Gaussian
gradients -- over two gloo ranks, fed with the FP64 oracle's per-view gradients.  The ranks'
reduced gradients must equal the sum over all views computed in one process."""
import os
import socket
import sys

import numpy as np
import pytest

torch = pytest.importorskip("torch")
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

from paper_2412_17378_gb300 import scenes  # noqa: E402
from paper_2412_17378_gb300.shard import GRAD_KEYS, partition_views  # noqa: E402


def test_partition_covers_every_view_once_and_balances_pixels():
    cams = scenes.scene_config("cfg4", 0.001)["cameras"]  # 4 x 640x360, 8 x 1280x720, 4 x 1920x1080
    px = [c["W"] * c["H"] for c in cams]
    for world in (1, 2, 3, 4, 16, 20):
        parts = partition_views(cams, world)
        assert len(parts) == world
        flat = sorted(v for p in parts for v in p)
        assert flat == list(range(len(cams)))
        loads = [sum(px[v] for v in p) for p in parts]
        if world <= len(cams):
            # LPT: no rank exceeds the mean by more than the largest single view
            assert max(loads) <= sum(px) / world + max(px)
        assert partition_views(cams, world) == parts  # deterministic
    assert partition_views(cams, 2, loads=[1.0] * 15 + [100.0])[0] == [15]  # explicit loads
    with pytest.raises(ValueError):
        partition_views(cams, 0)


def _per_view_grads():
    """FP64 oracle gradients of L = 1/2 sum_v ||C_v - target_v||^2 for every view of a small
    4-view scene: per view, the render backward composed with the projection backward."""
    import oracle
    s = scenes.scene_config("cfg2", 0.002)
    g = s["gaussians"]
    cams = scenes.arc_cameras([(64, 48), (80, 40), (48, 48), (96, 32)], yaw_deg=20.0)
    out = []
    for k, cam in enumerate(cams):
        pp = oracle.preprocess(g["means3D"], g["log_scales"], g["quats"], g["opacities"], cam)
        m2, co, dp = (pp[x].astype(np.float32) for x in ("means2D", "conic_opacity", "depth"))
        pl, rg = oracle.bin_tiles(m2, pp["radius"], dp, cam["W"], cam["H"])
        f = oracle.render(m2, co, g["colors"], dp, pl, rg, cam["W"], cam["H"])
        tgt = scenes.target_image(10 + k, cam["W"], cam["H"])
        r = oracle.render_backward(m2, co, g["colors"], dp, pl, rg, cam["W"], cam["H"], f["color"] - tgt)
        p = oracle.preprocess_backward(g["means3D"].astype(np.float64), g["log_scales"].astype(np.float64),
                                       g["quats"].astype(np.float64), cam, r["means2D"], r["conic"],
                                       radius=pp["radius"])
        out.append(dict(means3D=p["means3D"], log_scales=p["log_scales"], quats=p["quats"], opacities=r["opacity"],
                        colors=r["colors"]))
    return cams, out


def _free_port():
    with socket.socket() as sk:
        sk.bind(("127.0.0.1", 0))
        return sk.getsockname()[1]


def _rank_main(rank, world, port, q):
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    from paper_2412_17378_gb300.shard import allreduce_gaussian_grads
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    cams, per_view = _per_view_grads()
    mine = partition_views(cams, world)[rank]
    local = {k: torch.zeros(per_view[0][k].shape, dtype=torch.float64) for k in GRAD_KEYS}
    for v in mine:
        for k in GRAD_KEYS:
            local[k] += torch.from_numpy(per_view[v][k])
    allreduce_gaussian_grads(local)
    dist.barrier()
    dist.destroy_process_group()
    q.put((rank, mine, {k: t.numpy() for k, t in local.items()}))


def test_two_gloo_ranks_sum_the_views_gradients():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = {}
    for _ in range(2):
        rank, mine, grads = q.get(timeout=300)
        got[rank] = (mine, grads)
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    assert sorted(got[0][0] + got[1][0]) == [0, 1, 2, 3] and got[0][0] and got[1][0]
    _, per_view = _per_view_grads()
    for k in GRAD_KEYS:
        total = sum(pv[k] for pv in per_view)
        assert np.abs(total).max() > 0, k
        for r in (0, 1):  # every rank ends with the sum over all views
            np.testing.assert_allclose(got[r][1][k], total, rtol=1e-12, atol=1e-14 * np.abs(total).max())
